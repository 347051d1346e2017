"""Pins the oracle to the worked examples printed in the paper (tests/golden)."""
from fractions import Fraction

import numpy as np

import oracle
from tests._golden import dfa_from, load, state, symbol_map


def _dfa(name):
    f = load(name)
    Q, syms, delta, q0, finals = dfa_from(f)
    return f, Q, syms, oracle.Dfa(Q, len(syms), delta, q0, finals, symbol_map(syms))


def test_fig1_sequential_run():
    f, Q, syms, d = _dfa("w1_fig1.txt")
    st, fs, acc = d.run(f["input"][0][0].encode())
    assert st == 0
    assert fs == state(f["final_state"][0][0], Q)
    assert acc == bool(int(f["accept"][0][0]))


def test_fig1_isets_and_imax():
    f, Q, syms, d = _dfa("w1_fig1.txt")
    flags, imax = d.isets()
    for a, *states in f["iset"]:
        assert sorted(np.nonzero(flags[syms.index(a)])[0].tolist()) == [int(s) for s in states]
    assert imax == int(f["imax"][0][0])


def test_fig1_state_map_of_chunk2():
    f, Q, syms, d = _dfa("w1_fig1.txt")
    starts = [int(x) for x in f["starts_equal"][0]]
    text = f["input"][0][0].encode()
    # Sec. 4.1 matches chunk c2 for both q0 and q1; Algorithm 2 (all states).
    for chunk, j, tok in f["map_chunk"]:
        k = int(chunk)
        seg = text[starts[k]:starts[k + 1]]
        s = int(j)
        for ch in seg:
            s = d.delta_star(s, [syms.index(chr(ch))])
        assert s == state(tok, Q)
    # and Algorithm 3 on that chunking reaches the same final state
    st, fs, acc, maps = d.chunked(text, starts, want_maps=True)
    assert st == 0 and fs == state(f["final_state"][0][0], Q)
    # chunk 2's lookahead symbol is b, so only q1 is matched: L_2[q1] = q1
    assert maps[2][1] == 1


def test_fig1_balanced_partition():
    f, Q, syms, d = _dfa("w1_fig1.txt")
    n = len(f["input"][0][0])
    assert oracle.chunk_starts(n, 3, 2) == [int(x) for x in f["starts_balanced_m2"][0]]
    assert oracle.chunk_starts(n, 3, 1) == [int(x) for x in f["starts_equal"][0]]


def test_fig6_isets_partition_and_chunks():
    f, Q, syms, d = _dfa("w2_fig6.txt")
    text = f["input"][0][0]
    flags, imax = d.isets()
    for a, *states in f["iset"]:
        assert np.nonzero(flags[syms.index(a)])[0].tolist() == [int(s) for s in states]
    assert imax == int(f["imax"][0][0])
    n = len(text)
    assert oracle.l0(n, 3, imax) == int(f["l0_imax"][0][0])
    assert oracle.l0(n, 3, Q) == int(f["l0_q"][0][0])
    starts = oracle.chunk_starts(n, 3, imax)
    for k, s in f["chunk"]:
        k = int(k)
        assert text[starts[k]:starts[k + 1]] == s
    for k, *states in f["chunk_iset"]:
        k = int(k)
        look = syms.index(text[starts[k] - 1])
        assert np.nonzero(flags[look])[0].tolist() == [int(s) for s in states]


def test_fig6_run_rejects_in_error_state():
    f, Q, syms, d = _dfa("w2_fig6.txt")
    text = f["input"][0][0].encode()
    st, fs, acc = d.run(text)
    assert st == 0 and fs == state(f["final_state"][0][0], Q) and acc is False
    st, fs2, acc2, _ = d.chunked(text, oracle.chunk_starts(len(text), 3, 2))
    assert (fs2, acc2) == (fs, acc)


def test_table1_weighted_partition():
    f = load("w3_table1.txt")
    n = int(f["n"][0][0])
    m = int(f["states_to_match"][0][0])
    w = oracle.weights([int(x) for x in f["capacity"][0]])
    assert w == [Fraction(x) for x in f["weight"][0]]
    L0 = oracle.l0(n, 3, m, w)
    assert L0 == Fraction(f["l0"][0][0])
    weighted = [L0 * w[0]] + [L0 * wk / m for wk in w[1:]]
    assert weighted == [Fraction(x) for x in f["weighted"][0]]
    ranges = oracle.partition(n, 3, m, w)
    assert ranges == [(int(a), int(b)) for a, b in f["range"]]


def test_sbase_table_and_ibase():
    f2 = load("w2_fig6.txt")
    Q, syms, delta, q0, finals = dfa_from(f2)
    d = oracle.Dfa(Q, len(syms), delta, q0, finals, symbol_map(syms))
    f = load("w4_sbase.txt")
    sbase = [int(x) for x in f["sbase"][0]]
    # the oracle's delta extended by the error-state row is SBase read as state ids
    ext = [d.delta_star(q, [a]) for q in range(Q + 1) for a in range(len(syms))]
    assert ext == sbase
    ibase = [syms.index(ch) for ch in f["input"][0][0]]
    assert ibase == [int(x) for x in f["ibase"][0]]
    st, fs, acc = d.run(f["input"][0][0].encode())
    assert fs == Q  # state 4 is q_e
