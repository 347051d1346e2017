"""CPU checks of the C ABI: the library loads, exports exactly what
include/dfamatch.h declares, and its host-side steps (DFA compilation, Eq. 11/12
initial-state sets, alphabet classes, the Eq. 6-7 partition) agree with the
oracle.  No CUDA call is made here (dfa_create_host does none)."""
import ctypes
import os
import re

import numpy as np
import pytest

import gen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dm():
    from paper_1210_5093_gb300 import build
    build.build()
    import paper_1210_5093_gb300 as dm
    dm.lib()
    return dm


def _header_functions():
    src = open(os.path.join(ROOT, "include", "dfamatch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dfa_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(dm):
    names = _header_functions()
    assert len(names) >= 20
    L = ctypes.CDLL(dm.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(dm.SIGNATURES) == names


def test_strerror(dm):
    assert dm.strerror(0) == "ok"
    assert "alphabet" in dm.strerror(dm.ESYMBOL)


def _compare_isets(dm, spec):
    d = dm.Dfa.from_spec(spec, host_only=True)
    o = oracle.Dfa.from_spec(spec)
    flags, imax = o.isets()
    info = d.info()
    assert info.i_max == imax
    assert info.num_states_ext == spec.num_states + 1
    assert abs(info.gamma - imax / spec.num_states) < 1e-12
    cls = d.class_of_bytes()
    sym = spec.symbol_of_byte()
    for b in range(256):
        if sym[b] < 0:
            assert cls[b] == 0xFFFF
            continue
        want = np.nonzero(flags[sym[b]])[0].tolist()
        assert d.iset(int(cls[b])) == want, b
    # bytes share a class exactly when their symbols have identical columns
    ext = np.vstack([np.where(spec.delta < 0, spec.num_states, spec.delta),
                     np.full((1, spec.num_symbols), spec.num_states)])
    valid = [b for b in range(256) if sym[b] >= 0]
    for i, b1 in enumerate(valid[:40]):
        for b2 in valid[i + 1:i + 40]:
            same = np.array_equal(ext[:, sym[b1]], ext[:, sym[b2]])
            assert (cls[b1] == cls[b2]) == same
    assert d.iset(info.num_classes) == [spec.q0]                       # start set
    assert d.iset(info.num_classes + 1) == list(range(spec.num_states + 1))  # all of Q
    excluded = o.excluded()
    assert info.num_excluded == int(excluded.sum())
    return d, info


@pytest.mark.parametrize("seed", range(4))
def test_compile_random_small(dm, seed):
    spec = gen.random_dfa(40 + seed, 3 + 2 * seed, 2 + seed, num_finals=2, missing=0.3 * (seed % 2))
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[97:97 + spec.num_symbols] = np.arange(spec.num_symbols)
    spec.byte_to_symbol = m
    _compare_isets(dm, spec)


def test_compile_256_distinct_classes(dm):
    spec = gen.random_dfa(77, 60, 256, num_finals=3)
    d, info = _compare_isets(dm, spec)
    assert info.num_classes == 256
    assert sorted(set(d.class_of_bytes().tolist())) == list(range(256))


def test_compile_workload_dfas(dm):
    d, info = _compare_isets(dm, gen.plain_dfa(1))
    assert info.state_bytes == 1 and info.placement == 0
    spec = gen.regex_dfa(2)
    d, info = _compare_isets(dm, spec)
    assert info.num_classes == 32 and info.state_bytes == 2 and info.i_max == 241
    spec = gen.protein_dfa(3)
    d, info = _compare_isets(dm, spec)
    assert info.num_classes == 20 and info.i_max == int(np.ceil(0.35 * 1288 - 1e-9))


def test_compile_paper_examples(dm):
    from tests._golden import dfa_from, load, symbol_map
    for name in ("w1_fig1.txt", "w2_fig6.txt"):
        f = load(name)
        Q, syms, delta, q0, finals = dfa_from(f)
        spec = gen.DfaSpec(Q, len(syms), delta, q0, np.array(finals, dtype=np.uint32),
                           symbol_map(syms))
        d, info = _compare_isets(dm, spec)
        assert info.i_max == int(f["imax"][0][0])


def test_compile_rejects_bad_input(dm):
    good = np.zeros((2, 2), dtype=np.int32)
    with pytest.raises(dm.DfaError):
        dm.Dfa(2, 2, np.array([[0, 5], [0, 0]]), 0, [1], np.zeros(256, np.uint8), host_only=True)
    with pytest.raises(dm.DfaError):
        dm.Dfa(2, 2, good, 3, [1], np.zeros(256, np.uint8), host_only=True)   # q0 out of range
    with pytest.raises(dm.DfaError):
        dm.Dfa(2, 2, good, 0, [7], np.zeros(256, np.uint8), host_only=True)   # final out of range
    with pytest.raises(dm.DfaError):
        dm.Dfa(2, 2, good, 0, [1], None, host_only=True)                    # identity needs 256
    bad_map = np.zeros(256, np.uint8)
    bad_map[5] = 9
    with pytest.raises(dm.DfaError):
        dm.Dfa(2, 2, good, 0, [1], bad_map, host_only=True)
    d = dm.Dfa(2, 2, good, 0, [1], np.zeros(256, np.uint8), host_only=True)
    with pytest.raises(dm.DfaError) as e:
        d.match(b"ab")
    assert e.value.status == dm.EHOSTONLY
    with pytest.raises(dm.DfaError) as e:      # placement needs the device image too
        d.match(b"ab", boundary_window=16)
    assert e.value.status == dm.EHOSTONLY


@pytest.mark.parametrize("n", [0, 1, 36, 12345, 4 << 20, 10**10 + 7])
@pytest.mark.parametrize("P", [1, 2, 3, 1000])
@pytest.mark.parametrize("m", [1, 2, 241])
def test_partition_matches_oracle(dm, n, P, m):
    got = dm.partition(n, P, m).tolist()
    assert got == oracle.chunk_starts(n, P, m)


@pytest.mark.parametrize("which", ["reject", "accept"])
def test_compile_excluded_states_by_hand(dm, which):
    """The product's compiler leaves out the same states as the oracle on the
    hand-built DFAs whose sets are written out in test_oracle_pins: a
    non-accepting absorbing state besides q_e is excluded, an accepting
    absorbing state and a state that loops on one symbol only are kept."""
    from tests.test_oracle_pins import ABSORB_ACCEPT, ABSORB_REJECT
    d = ABSORB_REJECT if which == "reject" else ABSORB_ACCEPT
    m = np.array([i if i < d["num_symbols"] else 0xFF for i in range(256)], dtype=np.uint8)
    spec = gen.DfaSpec(d["num_states"], d["num_symbols"], np.array(d["delta"], dtype=np.int32),
                       d["q0"], np.array(d["finals"], dtype=np.uint32), m)
    dd, info = _compare_isets(dm, spec)
    cls = dd.class_of_bytes()
    if which == "reject":
        assert info.num_excluded == 2 and info.i_max == 2
        assert dd.iset(int(cls[0])) == [0, 1] and dd.iset(int(cls[1])) == [3]
    else:
        assert info.num_excluded == 1 and info.i_max == 2
        assert dd.iset(int(cls[0])) == [1, 2] and dd.iset(int(cls[1])) == [0, 1]


def test_compile_large_dfas_and_the_state_limit(dm):
    """|Q| up to 65534 compiles (q_e is state 65534; ids are 16-bit with
    0xFFFF reserved), with 32-bit table entries above 32767 states; 65535 is
    rejected.  The I-sets of a 5000-state DFA equal the oracle's."""
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[97:101] = np.arange(4)
    spec = gen.random_dfa(5, 5000, 4, num_finals=3, missing=0.05, byte_to_symbol=m)
    d, info = _compare_isets(dm, spec)
    assert info.state_bytes == 2
    m2 = np.full(256, 0xFF, dtype=np.uint8)
    m2[97:99] = np.arange(2)
    big = gen.random_dfa(6, 65534, 2, num_finals=1, byte_to_symbol=m2)
    d = dm.Dfa.from_spec(big, host_only=True)
    info = d.info()
    assert info.num_states_ext == 65535 and info.state_bytes == 4 and info.placement == 1
    too_big = np.zeros((65535, 2), dtype=np.int32)
    with pytest.raises(dm.DfaError) as e:
        dm.Dfa(65535, 2, too_big, 0, [1], m2, host_only=True)
    assert e.value.status == dm.EINVAL


def test_byte_rows_chosen_for_at_most_16_live_states(dm):
    """Byte rows (16 next-state codes per class row) are used exactly when a
    chain can visit at most 16 states: |Q| + 1 <= 16, or |Q| = 16 with q_e
    unreachable (no -1 in delta), and the table is in shared memory."""
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[97:100] = np.arange(3)
    cases = [(gen.plain_dfa(1), 1),                                          # 16 states, no -1
             (gen.random_dfa(3, 15, 3, missing=0.2, byte_to_symbol=m), 1),   # q_e is the 16th
             (gen.random_dfa(4, 16, 3, missing=0.2, byte_to_symbol=m), 0),   # 17 live states
             (gen.random_dfa(5, 8, 3, byte_to_symbol=m), 1),
             (gen.regex_dfa(2), 0)]
    for spec, want in cases:
        d = dm.Dfa.from_spec(spec, host_only=True)
        assert d.info().byte_rows == want, spec.name


def test_debug_library_exports_the_same_symbols(dm):
    """The debug build (DFA_DEBUG_BOUNDS) is the same ABI."""
    import ctypes
    from paper_1210_5093_gb300 import build
    build.build()
    L = ctypes.CDLL(build.OUT_DEBUG)
    for name in dm.SIGNATURES:
        assert hasattr(L, name), name
    assert L.dfa_strerror  # loads without a GPU
