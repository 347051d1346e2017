"""ORACLE - test infrastructure only.

A plain CPU statement of what the speculative DFA membership test of Ko, Jung,
Han & Burgstaller computes, used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with ``paper_1210_5093_gb300`` and does not import it.

* ``run``        - Algorithm 1 (sequential matching), in C (oracle.c).
* ``isets``      - Eq. (11)/(12): initial-state sets and I_max, in C.
* ``chunked``    - Algorithm 3 for a given partition plus the merge of Eq. (8), in C.
* ``compose``    - Eq. (9).
* ``partition``  - Eqs. (4)-(7) and (10) in exact rational arithmetic.
* ``weights``    - Eq. (1).
* ``iset_word``  - Eq. (13) for one word of r reverse-lookahead symbols, in C.
* ``isets_r``    - Eq. (13) for every word of length r, by enumeration
                   (exponential; small DFAs only).
* ``boundary_starts`` - Sec. 4.2's boundary placement: each chunk start moved,
                   within a bounded window, to the position whose reverse-
                   lookahead symbol has the smallest initial-state set.

Parity is pinned for every function here by tests/test_oracle_*.py (worked
examples printed in the paper, closed-form languages, brute force over all
short strings and the every-chunking invariant).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading
from fractions import Fraction
from math import floor
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_lib_lock = threading.Lock()  # first use may come from several threads at once

OK, EINVAL, ESYMBOL, ENOMEM = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no vector flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d.%d" % (os.getpid(), threading.get_ident())
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        return _load()


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        p, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run.argtypes = [u32, u32, p, u32, p, p, p, u64, p, p]
        lib.oracle_excluded.argtypes = [u32, u32, p, p, p]
        lib.oracle_isets.restype = u32
        lib.oracle_isets.argtypes = [u32, u32, p, p, p]
        lib.oracle_chunked.restype = ctypes.c_int
        lib.oracle_chunked.argtypes = [u32, u32, p, u32, p, p, p, u64, u32, p, p, p, p]
        lib.oracle_compose.argtypes = [u32, p, p, p]
        lib.oracle_iset_word.restype = u32
        lib.oracle_iset_word.argtypes = [u32, u32, p, p, p, u32, p]
        lib.oracle_delta_star.restype = u32
        lib.oracle_delta_star.argtypes = [u32, u32, p, u32, p, u32]
        _lib = lib
    return _lib


class Dfa:
    """The oracle's own view of a DFA: the user's delta as given (int32, -1 = q_e)."""

    def __init__(self, num_states: int, num_symbols: int, delta, q0: int, finals,
                 byte_to_symbol=None):
        self.Q = int(num_states)
        self.S = int(num_symbols)
        self.delta = np.ascontiguousarray(np.asarray(delta, dtype=np.int32).reshape(self.Q, self.S))
        self.q0 = int(q0)
        self.final_flags = np.zeros(self.Q + 1, dtype=np.uint8)
        for f in np.asarray(finals, dtype=np.int64).ravel():
            self.final_flags[int(f)] = 1
        self.map = None if byte_to_symbol is None else np.ascontiguousarray(
            np.asarray(byte_to_symbol, dtype=np.uint8))

    @classmethod
    def from_spec(cls, spec) -> "Dfa":
        return cls(spec.num_states, spec.num_symbols, spec.delta, spec.q0, spec.finals,
                   spec.byte_to_symbol)

    def _mp(self):
        return None if self.map is None else self.map.ctypes.data

    # ---------------------------------------------------------- Algorithm 1
    def run(self, data) -> tuple:
        """Returns (status, final_state, accept)."""
        buf = _as_u8(data)
        fs = ctypes.c_uint32(0)
        acc = ctypes.c_int32(0)
        st = _L().oracle_run(self.Q, self.S, self.delta.ctypes.data, self.q0,
                             self.final_flags.ctypes.data, self._mp(), buf.ctypes.data,
                             len(buf), ctypes.byref(fs), ctypes.byref(acc))
        if st != OK:
            return st, None, None
        return OK, int(fs.value), bool(acc.value)

    # ---------------------------------------------------------- Eqs. 11-12
    def excluded(self) -> np.ndarray:
        out = np.zeros(self.Q + 1, dtype=np.uint8)
        _L().oracle_excluded(self.Q, self.S, self.delta.ctypes.data,
                             self.final_flags.ctypes.data, out.ctypes.data)
        return out.astype(bool)

    def isets(self) -> tuple:
        """Returns (flags [S, Q+1] bool, I_max)."""
        out = np.zeros((self.S, self.Q + 1), dtype=np.uint8)
        imax = _L().oracle_isets(self.Q, self.S, self.delta.ctypes.data,
                                 self.final_flags.ctypes.data, out.ctypes.data)
        return out.astype(bool), int(imax)

    def iset(self, symbol: int) -> list:
        flags, _ = self.isets()
        return [int(s) for s in np.nonzero(flags[symbol])[0]]

    # ---------------------------------------------------------- Algorithm 3
    def chunked(self, data, starts: Sequence[int], want_maps: bool = False) -> tuple:
        """Algorithm 3 on the chunking `starts` (P+1 boundaries) and Eq. (8).
        Returns (status, final, accept, maps [P, Q+1] or None)."""
        buf = _as_u8(data)
        st_arr = np.ascontiguousarray(np.asarray(starts, dtype=np.uint64))
        P = len(st_arr) - 1
        maps = np.zeros((P, self.Q + 1), dtype=np.uint32) if want_maps else None
        fs = ctypes.c_uint32(0)
        acc = ctypes.c_int32(0)
        st = _L().oracle_chunked(self.Q, self.S, self.delta.ctypes.data, self.q0,
                                 self.final_flags.ctypes.data, self._mp(), buf.ctypes.data,
                                 len(buf), P, st_arr.ctypes.data,
                                 None if maps is None else maps.ctypes.data,
                                 ctypes.byref(fs), ctypes.byref(acc))
        if st != OK:
            return st, None, None, None
        return OK, int(fs.value), bool(acc.value), maps

    def delta_star(self, q: int, word: Sequence[int]) -> int:
        w = np.ascontiguousarray(np.asarray(word, dtype=np.uint32))
        return int(_L().oracle_delta_star(self.Q, self.S, self.delta.ctypes.data, q,
                                          w.ctypes.data if len(w) else None, len(w)))

    # ---------------------------------------------------------- Eq. 13
    def iset_word(self, word: Sequence[int]) -> list:
        """I_{sigma_1..sigma_r} of Eq. (13) for one symbol word, ascending."""
        w = np.ascontiguousarray(np.asarray(word, dtype=np.uint32))
        out = np.zeros(self.Q + 1, dtype=np.uint8)
        _L().oracle_iset_word(self.Q, self.S, self.delta.ctypes.data, self.final_flags.ctypes.data,
                              w.ctypes.data if len(w) else None, len(w), out.ctypes.data)
        return [int(s) for s in np.nonzero(out)[0]]

    def symbols(self, data) -> np.ndarray:
        """Symbol index of every byte (-1 outside Sigma)."""
        b = _as_u8(data).astype(np.int64)
        if self.map is None:
            return b
        m = self.map.astype(np.int64)
        m[m == 0xFF] = -1
        return m[b]

    def isets_r(self, r: int) -> dict:
        """{word: set of states} for every word of r symbols (Eq. 13 with the
        same exclusion as Algorithm 3/4).  Exponential in r."""
        excl = self.excluded()
        out = {}
        for word in itertools.product(range(self.S), repeat=r):
            img = set()
            for x in range(self.Q + 1):
                t = self.delta_star(x, word)
                if not excl[t]:
                    img.add(t)
            out[word] = img
        return out

    def imax_r(self, r: int) -> int:
        return max(len(v) for v in self.isets_r(r).values())


def compose(Li, Lj) -> np.ndarray:
    """Eq. (9): the map of chunk i followed by chunk j."""
    a = np.ascontiguousarray(np.asarray(Li, dtype=np.uint32))
    b = np.ascontiguousarray(np.asarray(Lj, dtype=np.uint32))
    out = np.zeros_like(a)
    _L().oracle_compose(len(a), a.ctypes.data, b.ctypes.data, out.ctypes.data)
    return out


def _as_u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    a = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
    return a


# ------------------------------------------------------------- Eqs. 1, 4-7, 10


def weights(capacities: Sequence) -> list:
    """Eq. (1): w_k = m_k / ((1/|P|) sum_i m_i), exactly."""
    m = [Fraction(x) for x in capacities]
    mean = sum(m) / len(m)
    return [x / mean for x in m]


def partition(n: int, P: int, m: int, w: Optional[Sequence] = None) -> list:
    """Inclusive (start, end) ranges of Eqs. (6)-(7), with Eq. (5) for L_0 and
    the number of states to match per subsequent chunk `m` (|Q| in Sec. 4.1,
    I_max in Eq. 10).  Exact rational arithmetic; w defaults to all ones."""
    w = [Fraction(1)] * P if w is None else [Fraction(x) for x in w]
    m = Fraction(m)
    L0 = Fraction(n) * m / (w[0] * m + sum(w[1:]))            # Eq. (5)/(10)

    # bound[k] = floor(L0 w0 + (1/m) sum_{1<=i<k} L0 w_i), accumulated left to right
    bound = [None] * (P + 1)
    acc = Fraction(0)
    for k in range(1, P + 1):
        bound[k] = floor(L0 * w[0] + acc / m)
        if k < P:
            acc += L0 * w[k]
    out = []
    for k in range(P):
        start = 0 if k == 0 else bound[k]                     # Eq. (6)
        end = n - 1 if k == P - 1 else bound[k + 1] - 1       # Eq. (7)
        out.append((start, end))
    return out


def chunk_starts(n: int, P: int, m: int) -> list:
    """Boundaries [start_0, ..., start_{P-1}, n] of the unweighted partition."""
    return [s for s, _ in partition(n, P, m)] + [n]


def l0(n: int, P: int, m: int, w: Optional[Sequence] = None) -> Fraction:
    w = [Fraction(1)] * P if w is None else [Fraction(x) for x in w]
    return Fraction(n) * m / (w[0] * m + sum(w[1:]))


# ------------------------------------------------------------- Sec. 4.2 boundaries

NOT_IN_SIGMA_COST = 65536  # larger than any initial-state set (|Q| <= 65535)


def boundary_window(n: int, P: int, m: int, window: int, lookahead: int = 1) -> int:
    """The window actually searched around each Eqs. (6)-(7) chunk start:
    at most a quarter of floor(n / (m + P - 1)), the shortest chunk after the
    first, so placed starts stay strictly increasing and no chunk grows by more
    than half of that length.  Algorithm 2 (no lookahead symbol) and empty
    chunks get no window."""
    if lookahead == 0 or window == 0 or P <= 1:
        return 0
    return min(int(window), (n // (m + P - 1)) // 4)


def boundary_starts(dfa: "Dfa", data, P: int, m: int, window: int, lookahead: int = 1) -> list:
    """Sec. 4.2 suggests, when the initial-state sets differ much in size, cutting
    the input right after symbols whose set is small.  Reading taken here: start with the boundaries of
    Eqs. (6)-(7); move the start S of every chunk k >= 1 to the position p in
    [S - w, S + w] (w from boundary_window) that minimises, in this order, the
    size |I_sigma| (Eq. 11) of the symbol sigma = Str[p - 1] before it, the
    distance |p - S| and p itself.  A byte outside Sigma costs more than any
    set.  The nominal start is a candidate, so no chunk starts after a symbol
    with a larger set than Eqs. (6)-(7) gave it; the paper's concern that a
    small-set symbol may be missing (a speed-down) is bounded by the window.
    Returns the P+1 boundaries [0, ..., n]."""
    buf = _as_u8(data)
    n = len(buf)
    starts = chunk_starts(n, P, m)
    w = boundary_window(n, P, m, window, lookahead)
    if w == 0:
        return starts
    flags, _ = dfa.isets()
    size = flags.sum(axis=1).astype(np.int64)               # |I_sigma| for every symbol
    out = list(starts)
    for k in range(1, P):
        S = starts[k]
        sym = dfa.symbols(buf[S - w - 1:S + w])             # symbols before p = S-w .. S+w
        best = None
        for i, p in enumerate(range(S - w, S + w + 1)):
            cost = int(size[sym[i]]) if sym[i] >= 0 else NOT_IN_SIGMA_COST
            key = (cost, abs(p - S), p)
            if best is None or key < best:
                best = key
        out[k] = best[2]
    return out
