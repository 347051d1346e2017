"""dfa_match on host input: the segmented copy/match pipeline.

Host strings of at least two first-segment lengths are copied and matched
segment by segment, each later segment as a continuation launch whose first
chunk looks back into the previous segment and whose Eq. (8) merge starts
from the previous segment's final state.  The answer must equal the oracle's
(bit-exact: final state, accept bit, status) for every segment layout, every
lookahead depth, pinned and pageable buffers, and bytes outside Sigma on
either side of a segment boundary."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm():
    import torch
    assert torch.cuda.is_available()
    from paper_1210_5093_gb300 import build
    build.build()
    import paper_1210_5093_gb300 as dm
    return dm


def _segments(n, first):
    """The segment lengths the library uses (doubling up to an eighth of the
    string; a short remainder joins the last segment), restated to place bytes
    at the boundaries."""
    cap = max(first, n // 8)
    out, pos, nxt = [], 0, first
    while pos < n:
        take = min(nxt, n - pos)
        if n - pos - take < nxt // 2:
            take = n - pos
        out.append(take)
        pos += take
        nxt = min(nxt * 2, cap)
    return out


def _pinned(data):
    import torch
    t = torch.empty(len(data), dtype=torch.uint8, pin_memory=True)
    t.numpy()[:] = data
    return t


@pytest.mark.parametrize("first", [(1 << 20) + 7, 300_001])
def test_pipeline_equals_oracle(dm, first):
    w = gen.regex_workload(5, (6 << 20) + 12345)
    assert len(_segments(len(w.data), first)) >= 3
    d = dm.Dfa.from_spec(w.spec)
    d.set_tuning(host_segment_bytes=first)
    want = oracle.Dfa.from_spec(w.spec).run(w.data)
    host = _pinned(w.data)
    for r in (0, 1, 2, 4):
        assert d.match(host, lookahead=r) == want, r
    assert d.match(w.data) == want               # pageable numpy buffer
    d.set_tuning(host_segment_bytes=0xFFFFFFFF)  # whole copy first
    assert d.match(host) == want


def test_pipeline_accepting_end_and_small_dfa(dm):
    w = gen.regex_workload(6, 5 << 20)
    word = np.frombuffer(w.spec.meta["planted_words"][0], dtype=np.uint8)
    data = w.data.copy()
    data[-len(word):] = word
    d = dm.Dfa.from_spec(w.spec)
    d.set_tuning(host_segment_bytes=1 << 20)
    st, fs, acc = d.match(_pinned(data))
    assert st == 0 and acc
    assert (st, fs, acc) == oracle.Dfa.from_spec(w.spec).run(data)
    p = gen.plain_workload(2, (4 << 20) + 3)
    dp = dm.Dfa.from_spec(p.spec)
    dp.set_tuning(host_segment_bytes=(1 << 20) - 5)
    assert dp.match(_pinned(p.data)) == oracle.Dfa.from_spec(p.spec).run(p.data)


def test_pipeline_bytes_outside_sigma_at_boundaries(dm):
    spec = gen.protein_dfa(3)
    d = dm.Dfa.from_spec(spec)
    first = 1 << 19
    d.set_tuning(host_segment_bytes=first)
    data = gen.protein_text(3, 3 << 20)
    seg = _segments(len(data), first)
    assert len(seg) >= 3
    b1, b2 = seg[0], seg[0] + seg[1]
    for pos in (0, b1 - 1, b1, b1 + 1, b2 - 2, b2, len(data) - 1):
        bad = data.copy()
        bad[pos] = ord("B")
        for r in (1, 4):
            st, _, _ = d.match(_pinned(bad), lookahead=r)
            assert st == dm.ESYMBOL, (pos, r)
    st, fs, acc = d.match(_pinned(data), lookahead=4)
    assert (st, fs, acc) == oracle.Dfa.from_spec(spec).run(data)
