"""Pins the oracle's boundary placement (Sec. 4.2's suggestion: cut the input
right after symbols whose initial-state set is small) to
cases whose answer is fixed by construction, and to properties that any
correct placement has:

* a DFA whose reset symbol c has the one-state set {q0} while a and b have
  sets of all four states, on strings where c sits at hand-picked positions:
  the placed starts are known without running anything;
* a window of 0, or Algorithm 2, leaves the partition of Eqs. (6)-(7);
* on the workload DFAs: starts stay strictly increasing and within the
  window, no chunk starts after a symbol with a larger set than its nominal
  start had, and Algorithm 3 on the placed chunks still gives Algorithm 1's
  answer (the every-chunking invariant, failure-freedom of Sec. 4.4).

A placement that ignores the window, breaks ties toward the larger position
or prefers the farther of two equal candidates fails one of these.
"""
import numpy as np
import pytest

import gen
import oracle

A, B, C = 0, 1, 2


def _reset_dfa():
    """4 states over {a, b, c}: a rotates, b stays, c resets to q0.
    I_a = I_b = Q (size 4), I_c = {q0} (size 1)."""
    delta = [[(q + 1) % 4, q, 0] for q in range(4)]
    return oracle.Dfa(4, 3, np.array(delta, dtype=np.int32).ravel(), 0, [3])


def _string(n, c_at, fill=A):
    s = np.full(n, fill, dtype=np.uint8)
    s[1::2] = B
    for i in c_at:
        s[i] = C
    return s


def test_reset_dfa_sets():
    d = _reset_dfa()
    flags, imax = d.isets()
    assert flags.sum(axis=1).tolist() == [4, 4, 1] and imax == 4


def test_constructed_placement():
    d = _reset_dfa()
    # n = 64, P = 4, m = 1: nominal starts 16, 32, 48; shortest later chunk 16, so
    # the window is min(8, 16 // 4) = 4.
    #   c at 13 -> p = 14 (distance 2) is the only cheap candidate near 16;
    #   c at 29 and 33 -> p = 30 and p = 34 tie at distance 2: the smaller wins;
    #   c at 40 -> p = 41 is 7 away from 48, outside the window: 48 stays.
    s = _string(64, [13, 29, 33, 40])
    assert oracle.boundary_window(64, 4, 1, 8) == 4
    assert oracle.boundary_starts(d, s, 4, 1, 8) == [0, 14, 30, 48, 64]
    # a cheap symbol right before the nominal start keeps it (distance 0)
    s2 = _string(64, [15, 30, 46])
    assert oracle.boundary_starts(d, s2, 4, 1, 8) == [0, 16, 31, 47, 64]
    # window 1: only p in [S-1, S+1]; every cheap candidate above is within 1
    assert oracle.boundary_starts(d, s2, 4, 1, 1) == [0, 16, 31, 47, 64]
    # ... and c at 13, 29, 50 is 2-3 positions away: a window of 1 keeps Eqs. (6)-(7)
    s3 = _string(64, [13, 29, 50])
    assert oracle.boundary_starts(d, s3, 4, 1, 1) == [0, 16, 32, 48, 64]


def test_bytes_outside_sigma_are_never_preferred():
    # bytes through a map: 'a','b','c' are symbols, '!' is outside Sigma
    d0 = _reset_dfa()
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[ord("a")], m[ord("b")], m[ord("c")] = A, B, C
    d = oracle.Dfa(4, 3, d0.delta.ravel(), 0, [3], m)
    s = bytearray(b"ab" * 32)
    s[15] = ord("!")          # the nominal start 16 follows a byte outside Sigma
    s[17] = ord("c")          # p = 18: set {q0}
    assert oracle.boundary_starts(d, bytes(s), 4, 1, 8)[1] == 18
    s[17] = ord("a")          # no cheap symbol: any in-Sigma neighbour beats '!'
    assert oracle.boundary_starts(d, bytes(s), 4, 1, 8)[1] == 15


def test_window_zero_and_algorithm2_keep_eqs_6_7():
    w = gen.regex_workload(2, 1 << 18)
    d = oracle.Dfa.from_spec(w.spec)
    nominal = oracle.chunk_starts(len(w.data), 37, 1)
    assert oracle.boundary_starts(d, w.data, 37, 1, 0) == nominal
    assert oracle.boundary_starts(d, w.data, 37, 1, 256, lookahead=0) == nominal
    # multiplicity m = 3 shifts the nominal starts (Eq. 10); placement starts from them
    nominal3 = oracle.chunk_starts(len(w.data), 37, 3)
    assert oracle.boundary_starts(d, w.data, 37, 3, 0) == nominal3


@pytest.mark.parametrize("maker,P,window", [("regex", 64, 256), ("regex", 500, 32),
                                            ("protein", 64, 64), ("plain", 1024, 8)])
def test_placement_properties_and_invariant(maker, P, window):
    w = {"regex": lambda: gen.regex_workload(2, 1 << 20),
         "protein": lambda: gen.protein_workload(3, 1 << 20),
         "plain": lambda: gen.plain_workload(1, 1 << 20)}[maker]()
    d = oracle.Dfa.from_spec(w.spec)
    n = len(w.data)
    nominal = oracle.chunk_starts(n, P, 1)
    placed = oracle.boundary_starts(d, w.data, P, 1, window)
    wl = oracle.boundary_window(n, P, 1, window)
    assert placed[0] == 0 and placed[-1] == n
    assert all(a < b for a, b in zip(placed, placed[1:]))
    flags, _ = d.isets()
    size = flags.sum(axis=1)
    sym = d.symbols(w.data)
    for k in range(1, P):
        assert abs(placed[k] - nominal[k]) <= wl
        assert size[sym[placed[k] - 1]] <= size[sym[nominal[k] - 1]]
    st, fs, acc, _ = d.chunked(w.data, placed)
    assert (st, fs, acc) == d.run(w.data)


def test_placement_shrinks_the_regex_work():
    """Eq. 16's matching term sum_k L_k |I_k| on the placed chunks, against the
    nominal ones: the regex-shaped text always has a small-set symbol nearby."""
    w = gen.regex_workload(2, 1 << 20)
    d = oracle.Dfa.from_spec(w.spec)
    n, P = len(w.data), 128
    flags, _ = d.isets()
    size = flags.sum(axis=1)
    sym = d.symbols(w.data)

    def work(starts):
        lens = np.diff(np.asarray(starts))
        sets = [1] + [int(size[sym[s - 1]]) for s in starts[1:-1]]
        return int((lens * np.asarray(sets)).sum())

    w_nom = work(oracle.chunk_starts(n, P, 1))
    w_placed = work(oracle.boundary_starts(d, w.data, P, 1, 256))
    assert w_placed * 4 < w_nom
