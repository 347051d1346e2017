"""Seeded synthetic inputs: DFAs shaped like the paper's regex (PCRE) and
protein (PROSITE) workloads, plus the strings they are matched against.

This module is shared by the tests, ``bench.py`` and the smoke check.  It holds
none of the membership test's arithmetic: it only *builds* transition tables
and byte strings.  Expected results never come from here; they come from the
oracle.  The one routine that walks a DFA, :func:`sync_words`, only chooses
which words to plant so that accepting paths occur in the text.

All randomness is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in counter
form, implemented once in ``gen.c``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdfagen.so")
_lib = None
_lib_lock = threading.Lock()  # first use may come from several threads at once

# stream ids (any distinct constants)
S_DELTA, S_FINAL, S_GAMMA, S_TARGET, S_PERM, S_CLASSMAP, S_TEXT, S_PLANT, S_PLANTW, \
    S_WORDS, S_FREQ, S_MISSING, S_LENS, S_PICK, S_MIX = range(1, 16)


def build(force: bool = False) -> str:
    """Compile gen.c into libdfagen.so (gcc, no GPU)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d.%d" % (os.getpid(), threading.get_ident())
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src,
                               "-o", tmp])
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
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        lib.gen_key.restype = u64
        lib.gen_key.argtypes = [u64, u64]
        lib.gen_u64.argtypes = [u64, u64, u64, p]
        lib.gen_bytes_uniform.argtypes = [u64, p, u64, ctypes.c_int]
        lib.gen_bytes_categorical.argtypes = [u64, p, p, ctypes.c_int, p, u64, ctypes.c_int]
        lib.gen_plant_words.argtypes = [u64, u64, u64, p, p, ctypes.c_int, p, u64, ctypes.c_int]
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def key(seed: int, stream: int) -> int:
    return int(_L().gen_key(seed & (2**64 - 1), stream))


def draws(k: int, n: int, start: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    if n:
        _L().gen_u64(k, start, n, out.ctypes.data)
    return out


def below(u, k: int):
    """Uniform integer in [0, k) from a 64-bit draw (multiply-high of the top 32 bits)."""
    return ((np.asarray(u, dtype=np.uint64) >> np.uint64(32)) * np.uint64(k)) >> np.uint64(32)


def unit(u):
    """Uniform double in [0, 1) from a 64-bit draw."""
    return (np.asarray(u, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def permutation(k: int, n: int) -> np.ndarray:
    """Fisher-Yates shuffle of range(n) driven by stream k."""
    a = np.arange(n, dtype=np.int64)
    d = draws(k, max(n, 1))
    for i in range(n - 1, 0, -1):
        j = int(below(d[i], i + 1))
        a[i], a[j] = a[j], a[i]
    return a


# ----------------------------------------------------------------- DFA spec


@dataclass
class DfaSpec:
    """A DFA in the form the C-ABI takes: delta[q, a] (-1 = implicit error state)."""
    num_states: int
    num_symbols: int
    delta: np.ndarray                      # int32 [num_states, num_symbols]
    q0: int
    finals: np.ndarray                     # uint32 [num_finals]
    byte_to_symbol: Optional[np.ndarray]   # uint8 [256], 0xFF = not in Sigma; None = identity
    name: str = ""
    meta: dict = field(default_factory=dict)

    def symbol_of_byte(self) -> np.ndarray:
        if self.byte_to_symbol is None:
            return np.arange(256, dtype=np.int32)
        m = self.byte_to_symbol.astype(np.int32)
        m[m == 0xFF] = -1
        return m


def _sample_distinct(k: int, n: int, count: int, exclude=()) -> np.ndarray:
    pool = [x for x in permutation(k, n).tolist() if x not in set(exclude)]
    return np.array(sorted(pool[:count]), dtype=np.uint32)


def random_dfa(seed: int, num_states: int, num_symbols: int, num_finals: int = 1,
               missing: float = 0.0, byte_to_symbol=None, q0: int = 0) -> DfaSpec:
    """delta uniform over the states; a fraction `missing` of entries is -1."""
    d = draws(key(seed, S_DELTA), num_states * num_symbols)
    delta = below(d, num_states).astype(np.int32).reshape(num_states, num_symbols)
    if missing > 0:
        m = unit(draws(key(seed, S_MISSING), num_states * num_symbols)) < missing
        delta[m.reshape(num_states, num_symbols)] = -1
    finals = _sample_distinct(key(seed, S_FINAL), num_states, min(num_finals, num_states))
    return DfaSpec(num_states, num_symbols, delta, q0, finals, byte_to_symbol,
                   name=f"random{num_states}x{num_symbols}")


def plain_dfa(seed: int) -> DfaSpec:
    """Plain single-test workload: |Q|=16, 256 byte symbols, delta uniform, q0=0,
    4 accepting states other than q0."""
    d = draws(key(seed, S_DELTA), 16 * 256)
    delta = below(d, 16).astype(np.int32).reshape(16, 256)
    finals = _sample_distinct(key(seed, S_FINAL), 16, 4, exclude=(0,))
    return DfaSpec(16, 256, delta, 0, finals, None, name="plain16")


PRINTABLE = np.arange(0x20, 0x7F, dtype=np.uint8)          # 95 printable ASCII bytes
AMINO = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8)  # 20 one-letter codes


def class_dfa(seed: int, num_states: int, num_classes: int, gamma_lo: float, gamma_hi: float,
              num_finals: int, alphabet: str = "byte", name: str = "") -> DfaSpec:
    """Regex/protein-shaped DFA.

    Per class c a target set T_c of ceil(gamma_c*|Q|) states is drawn, gamma_c
    log-uniform in [gamma_lo, gamma_hi] with one class pinned at each end;
    delta(q, c) is uniform over T_c with every element of T_c hit, so the image
    of delta(., c) is exactly T_c.

    alphabet="byte": 256 byte symbols folded onto num_classes identical columns
    (the 95 printable bytes are spread over all classes; the rest are assigned
    at random); delta is returned unfolded (num_symbols=256, identity byte map)
    so the class folding is left to the compiler.  num_classes == 256 gives an
    unfolded table.
    alphabet="protein": 20 symbols (the amino-acid letters); bytes outside
    them are not in Sigma.
    """
    Q = num_states
    C = num_classes
    g = unit(draws(key(seed, S_GAMMA), C))
    lo, hi = math.log(max(gamma_lo, 1.0 / Q)), math.log(gamma_hi)
    gam = np.exp(lo + g * (hi - lo))
    order = permutation(key(seed, S_GAMMA + 100), C)
    gam[order[0]] = gamma_hi
    if C > 1:
        gam[order[1]] = max(gamma_lo, 1.0 / Q)
    sizes = np.minimum(Q, np.ceil(gam * Q - 1e-9).astype(np.int64))
    sizes = np.maximum(sizes, 1)
    tab = np.empty((Q, C), dtype=np.int32)
    for c in range(C):
        tk = key(seed, S_TARGET * 1000 + c)
        T = permutation(tk, Q)[: sizes[c]]
        pi = permutation(key(seed, S_PERM * 1000 + c), Q)
        d = draws(key(seed, S_TARGET * 1000 + c + 500), Q)
        col = np.empty(Q, dtype=np.int64)
        col[pi[: sizes[c]]] = T
        rest = pi[sizes[c]:]
        col[rest] = T[below(d[: len(rest)], sizes[c]).astype(np.int64)]
        tab[:, c] = col
    finals = _sample_distinct(key(seed, S_FINAL), Q, num_finals, exclude=(0,))
    meta = {"gamma_c": gam.tolist(), "target_sizes": sizes.tolist()}
    if alphabet == "protein":
        assert C == len(AMINO)
        b2s = np.full(256, 0xFF, dtype=np.uint8)
        b2s[AMINO] = np.arange(len(AMINO), dtype=np.uint8)
        spec = DfaSpec(Q, C, tab, 0, finals, b2s, name=name or f"protein{Q}", meta=meta)
        spec.meta["letters"] = AMINO
        return spec
    # byte alphabet: fold 256 bytes onto C classes
    if C == 256:
        cls_of_byte = permutation(key(seed, S_CLASSMAP), 256)
    else:
        cls_of_byte = np.empty(256, dtype=np.int64)
        pr = permutation(key(seed, S_CLASSMAP), len(PRINTABLE))
        for r, idx in enumerate(pr.tolist()):
            cls_of_byte[PRINTABLE[idx]] = r % C
        others = np.setdiff1d(np.arange(256), PRINTABLE)
        d = draws(key(seed, S_CLASSMAP + 100), len(others))
        cls_of_byte[others] = below(d, C).astype(np.int64)
    delta = tab[:, cls_of_byte].astype(np.int32)
    meta["class_of_byte"] = cls_of_byte
    meta["letters"] = PRINTABLE
    return DfaSpec(Q, 256, np.ascontiguousarray(delta), 0, finals, None,
                   name=name or f"regex{Q}", meta=meta)


def regex_dfa(seed: int) -> DfaSpec:
    """Regex-shaped workload DFA: |Q|=512, bytes folded to 32 classes,
    gamma_c in [0.02, 0.47], 16 accepting states."""
    return class_dfa(seed, 512, 32, 0.02, 0.47, 16, "byte", name="regex512")


def protein_dfa(seed: int) -> DfaSpec:
    """Protein-shaped workload DFA: 20 amino-acid letters, |Q|=1288,
    gamma_c in [0.02, 0.35], 13 accepting states (about 1% of |Q|)."""
    return class_dfa(seed, 1288, 20, 0.02, 0.35, 13, "protein", name="protein1288")


# ------------------------------------------------------------ closed forms


def mod_counter_dfa(k: int, num_symbols: int = 2, counted: int = 0) -> DfaSpec:
    """Accepts strings whose number of `counted` symbols is 0 mod k.  Every
    symbol permutes the states, so every initial-state set is all of Q."""
    delta = np.empty((k, num_symbols), dtype=np.int32)
    for q in range(k):
        for a in range(num_symbols):
            delta[q, a] = (q + 1) % k if a == counted else q
    return DfaSpec(k, num_symbols, delta, 0, np.array([0], dtype=np.uint32), None,
                   name=f"mod{k}")


def suffix_dfa(word, num_symbols: int) -> DfaSpec:
    """Accepts strings ending in `word` (the Knuth-Morris-Pratt automaton).
    State i = length of the longest suffix of the input that is a prefix of word."""
    w = list(word)
    k = len(w)
    delta = np.empty((k + 1, num_symbols), dtype=np.int32)
    for q in range(k + 1):
        for a in range(num_symbols):
            s = w[:q] + [a]
            j = min(len(s), k)
            while j > 0 and s[len(s) - j:] != w[:j]:
                j -= 1
            delta[q, a] = j
    return DfaSpec(k + 1, num_symbols, delta, 0, np.array([k], dtype=np.uint32), None,
                   name="suffix")


# ------------------------------------------------------------------ strings


def uniform_bytes(seed: int, n: int, stream: int = S_TEXT) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)
    if n:
        _L().gen_bytes_uniform(key(seed, stream), out.ctypes.data, n, _threads())
    return out


def _cdf32(weights) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    c = np.floor(np.cumsum(w) / w.sum() * 2.0 ** 32).astype(np.uint64)
    c[-1] = np.uint64(2 ** 32)
    return c


def categorical_bytes(seed: int, n: int, symbols, weights, stream: int = S_TEXT,
                      out: Optional[np.ndarray] = None) -> np.ndarray:
    syms = np.ascontiguousarray(np.asarray(symbols, dtype=np.uint8))
    cdf = _cdf32(weights)
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    if n:
        _L().gen_bytes_categorical(key(seed, stream), cdf.ctypes.data, syms.ctypes.data,
                                   len(syms), out.ctypes.data, n, _threads())
    return out


def plant(seed: int, buf: np.ndarray, words, rate: float) -> np.ndarray:
    """Overwrite buf in place with words starting at each position with probability `rate`."""
    if not words or rate <= 0 or len(buf) == 0:
        return buf
    flat = np.frombuffer(b"".join(bytes(bytearray(w)) for w in words), dtype=np.uint8).copy()
    offs = np.zeros(len(words) + 1, dtype=np.uint32)
    offs[1:] = np.cumsum([len(w) for w in words])
    r = min(int(rate * 2.0 ** 64), 2 ** 64 - 1)
    _L().gen_plant_words(key(seed, S_PLANT), key(seed, S_PLANTW), r, flat.ctypes.data,
                         offs.ctypes.data, len(words), buf.ctypes.data, len(buf), _threads())
    return buf


def zipf_text(seed: int, n: int, s: float = 1.1, letters=PRINTABLE,
              out: Optional[np.ndarray] = None) -> np.ndarray:
    """Zipf(s) over the given letters with a seeded rank -> letter permutation."""
    ranks = np.arange(1, len(letters) + 1, dtype=np.float64)
    perm = permutation(key(seed, S_PERM + 77), len(letters))
    return categorical_bytes(seed, n, np.asarray(letters)[perm], ranks ** (-s), out=out)


def protein_freqs(seed: int) -> np.ndarray:
    """A fixed, seeded 20-entry background frequency table (weights in [1, 4))."""
    return 1.0 + 3.0 * unit(draws(key(seed, S_FREQ), len(AMINO)))


def protein_text(seed: int, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    return categorical_bytes(seed, n, AMINO, protein_freqs(seed), out=out)


# ------------------------------------------------------------ planted words


def _image(delta_by_letter: np.ndarray, S: np.ndarray, letter_col: int) -> np.ndarray:
    return np.unique(delta_by_letter[S, letter_col])


def sync_words(spec: DfaSpec, letters, count: int, seed: int, maxlen: int = 64):
    """Words over `letters` that drive *every* state into an accepting state.

    Greedy set shrinking (Eppstein, SIAM J. Comput. 1990): starting from all
    states, append the letter whose image of the current set is smallest until
    one state is left, then a shortest path from it into F.  A short random
    prefix makes the words differ.  Raises if a word longer than maxlen would be
    needed.
    """
    letters = [int(x) for x in letters]
    sym = spec.symbol_of_byte()
    Qe = spec.num_states + 1
    cols = np.empty((Qe, len(letters)), dtype=np.int64)
    for li, b in enumerate(letters):
        a = sym[b]
        col = spec.delta[:, a].astype(np.int64)
        col[col < 0] = spec.num_states
        cols[: spec.num_states, li] = col
        cols[spec.num_states, li] = spec.num_states
    fin = np.zeros(Qe, dtype=bool)
    fin[spec.finals.astype(np.int64)] = True
    words = []
    k = key(seed, S_WORDS)
    d = draws(k, 64 * count * 8)
    di = 0
    tries = 0
    while len(words) < count:
        tries += 1
        if tries > 20 * count:
            raise RuntimeError("no synchronising word within %d letters" % maxlen)
        plen = 1 + int(below(d[di % len(d)], 4)); di += 1
        w = []
        S = np.arange(spec.num_states, dtype=np.int64)
        for _ in range(plen):
            li = int(below(d[di % len(d)], len(letters))); di += 1
            w.append(li)
            S = np.unique(cols[S, li])
        while len(S) > 1 and len(w) < maxlen:
            best, bl = None, None
            for li in range(len(letters)):
                im = np.unique(cols[S, li])
                if best is None or len(im) < len(best):
                    best, bl = im, li
            if len(best) == len(S):
                # no single letter shrinks the set: take a random letter and keep going
                bl = int(below(d[di % len(d)], len(letters))); di += 1
                best = np.unique(cols[S, bl])
            S = best
            w.append(bl)
        if len(S) != 1:
            continue
        # shortest path from the single state into F
        s0 = int(S[0])
        prev = {s0: None}
        frontier = [s0]
        goal = s0 if fin[s0] else None
        while goal is None and frontier:
            nxt = []
            for s in frontier:
                for li in range(len(letters)):
                    t = int(cols[s, li])
                    if t not in prev:
                        prev[t] = (s, li)
                        if fin[t]:
                            goal = t
                            break
                        nxt.append(t)
                if goal is not None:
                    break
            frontier = nxt
        if goal is None:
            continue
        path = []
        t = goal
        while prev[t] is not None:
            s, li = prev[t]
            path.append(li)
            t = s
        w += path[::-1]
        if len(w) <= maxlen:
            word = bytes(letters[li] for li in w)
            if word not in words:
                words.append(word)
    return words


# ---------------------------------------------------------------- workloads


@dataclass
class Workload:
    name: str
    spec: DfaSpec
    data: np.ndarray
    num_chunks: int = 0          # 0 = let the planner choose
    recipe: str = ""


def plain_workload(seed: int = 1, n: int = 4 << 20) -> Workload:
    spec = plain_dfa(seed)
    return Workload("plain16_4MiB", spec, uniform_bytes(seed, n), 1024,
                    "|Q|=16, 256 byte symbols, delta uniform, 4 MiB uniform bytes, 1024 chunks")


def regex_workload(seed: int = 2, n: int = 1 << 30, words=None) -> Workload:
    spec = regex_dfa(seed)
    if words is None:
        words = sync_words(spec, PRINTABLE, 16, seed)
    data = zipf_text(seed, n)
    plant(seed, data, words, 1e-3)
    spec.meta["planted_words"] = words
    return Workload("regex512_%s" % _size_name(n), spec, data, 0,
                    "|Q|=512, 32 byte classes, Zipf(1.1) printable text, 0.1% planted words")


def protein_workload(seed: int = 3, n: int = 10 * 10**9, words=None) -> Workload:
    spec = protein_dfa(seed)
    if words is None:
        words = sync_words(spec, AMINO, 16, seed)
    data = protein_text(seed, n)
    plant(seed, data, words, 1e-6)
    spec.meta["planted_words"] = words
    return Workload("protein1288_%s" % _size_name(n), spec, data, 0,
                    "|Q|=1288, 20 amino-acid letters, i.i.d. residues, motifs at 1e-6")


# |Q| of the protein-shaped DFAs matched together on one protein text (a
# group of PROSITE-like patterns of growing size; their joint tables, 21 rows
# of 16-bit entries each, total about 64 KB)
PROTEIN_GROUP_SIZES = (16, 32, 64, 100, 160, 240, 340, 480)


def protein_group_dfas(seed: int = 7, sizes=PROTEIN_GROUP_SIZES):
    """Protein-shaped DFAs over the 20 amino-acid letters (gamma_c in
    [0.02, 0.35], as protein_dfa), one per entry of sizes."""
    return [class_dfa(seed * 100 + i, q, 20, 0.02, 0.35, max(1, q // 100), "protein",
                      name="protein%d" % q) for i, q in enumerate(sizes)]


def _size_name(n: int) -> str:
    if n >= 10**9 and n % 10**9 == 0:
        return "%dGB" % (n // 10**9)
    for unit_, nm in ((1 << 30, "GiB"), (1 << 20, "MiB"), (1 << 10, "KiB")):
        if n >= unit_ and n % unit_ == 0:
            return "%d%s" % (n // unit_, nm)
    return "%dB" % n


def batch_dfas(seed: int, count: int = 64, q_lo: int = 8, q_hi: int = 1288):
    """The batched mix: |Q| log-uniform in [q_lo, q_hi]; a quarter byte-folded
    (32 classes), a quarter byte-unfolded (256 classes), half protein-lettered;
    gamma_max log-uniform in [0.02, 0.47]."""
    u = unit(draws(key(seed, S_MIX), 3 * count))
    specs = []
    for i in range(count):
        Q = int(round(math.exp(math.log(q_lo) + u[3 * i] * (math.log(q_hi) - math.log(q_lo)))))
        gmax = math.exp(math.log(0.02) + u[3 * i + 1] * (math.log(0.47) - math.log(0.02)))
        gmax = max(gmax, 1.0 / Q)
        kind = i % 4
        nf = max(1, Q // 100)
        s = seed * 1000 + i
        if kind == 0:
            specs.append(class_dfa(s, Q, 32, 0.02, gmax, nf, "byte", name=f"b32_{i}"))
        elif kind == 1:
            specs.append(class_dfa(s, Q, 256, 0.02, gmax, nf, "byte", name=f"b256_{i}"))
        else:
            specs.append(class_dfa(s, Q, 20, 0.02, gmax, nf, "protein", name=f"p20_{i}"))
    return specs


def batch_lengths(seed: int, count: int, lo: int = 256, hi: int = 64 << 20) -> np.ndarray:
    u = unit(draws(key(seed, S_LENS), count))
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_picks(seed: int, count: int, num_dfas: int) -> np.ndarray:
    return below(draws(key(seed, S_PICK), count), num_dfas).astype(np.int64)


def batch_text(seed: int, spec: DfaSpec, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Input for one batched test: Zipf printable text for byte DFAs, residues for protein DFAs."""
    if spec.byte_to_symbol is not None:
        return protein_text(seed, n, out=out)
    return zipf_text(seed, n, out=out)
