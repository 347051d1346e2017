"""The debug build (device-side bounds checks on every state, class, set slot
and chunk bound; DFA_EBOUNDS on a failed check) gives the oracle's answer on
the paper's workloads and on every kind of launch: Algorithms 2 and 3, Eq. 13
sets, Sec. 4.2 placement, tables in shared memory and through L2, byte rows,
multi-pass chunks of a 20000-state DFA, batches with graph replay, the
pipelined host path and groups of DFAs sharing one stage.  Runs in its own process, which loads the debug library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_finds_no_bounds_violation():
    from paper_1210_5093_gb300 import build
    build.build()
    assert os.path.exists(build.OUT_DEBUG)
    env = dict(os.environ, DFA_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_bounds_cases.py")],
                       env=env, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug-bounds parity ok" in r.stdout
