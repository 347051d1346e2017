"""Pins the oracle to facts fixed by the mathematics rather than by itself:

* brute force over every string of length <= 8 on tiny DFAs, against membership
  decided by a different method (backward propagation of the accepting set);
* closed-form languages (a*bc* through Python's `re`, "count of a mod k == 0",
  "ends with w" through str.endswith);
* the every-chunking invariant of Algorithm 3 (failure-freedom, Sec. 4.4);
* the lemma of Sec. 4.3 (I_max,r is non-increasing in r) and k-locality;
* Eq. (9) composition against the sequential merge of Eq. (8);
* Eqs. (6)-(7) in exact arithmetic against the closed integer form.

It also checks that plausible mistakes are caught: a chunked merge that uses a
wrong lookahead symbol, or drops one initial state, fails the invariant.
"""
import itertools
import re

import numpy as np
import pytest

import gen
import oracle


def _ext(spec):
    """delta with the error-state row appended (test-side, numpy)."""
    Q = spec.num_states
    d = spec.delta.astype(np.int64).copy()
    d[d < 0] = Q
    return np.vstack([d, np.full((1, spec.num_symbols), Q, dtype=np.int64)])


def _backward_accepts(spec, words):
    """Membership by backward set propagation: B_n = F, B_i = delta^-1(B_{i+1}, w_i);
    accept iff q0 in B_0.  words: int array [N, L]."""
    ext = _ext(spec)
    Q = spec.num_states
    N, L = words.shape
    B = np.zeros((N, Q + 1), dtype=bool)
    B[:, spec.finals.astype(np.int64)] = True
    rows = np.arange(N)[:, None]
    for i in range(L - 1, -1, -1):
        B = B[rows, ext[:, words[:, i]].T]
    return B[:, spec.q0]


def _all_words(k, L):
    if L == 0:
        return np.zeros((1, 0), dtype=np.int64)
    return np.array(list(itertools.product(range(k), repeat=L)), dtype=np.int64)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_all_short_strings(k, seed):
    Q = 2 + seed % 5
    spec = gen.random_dfa(1000 + 10 * k + seed, Q, k, num_finals=1 + seed % 2,
                          missing=0.2 if seed % 2 else 0.0)
    d = oracle.Dfa.from_spec(spec)
    for L in range(0, 9):
        words = _all_words(k, L)
        expect = _backward_accepts(spec, words)
        for w, e in zip(words, expect):
            st, fs, acc = d.run(bytes(w.astype(np.uint8)))
            assert st == 0 and acc == bool(e), (L, w)


def test_closed_form_fig1_language_against_re():
    delta = np.array([[0, 1, -1], [-1, -1, 1]], dtype=np.int32)
    m = np.full(256, 0xFF, dtype=np.uint8)
    for i, ch in enumerate(b"abc"):
        m[ch] = i
    d = oracle.Dfa(2, 3, delta, 0, [1], m)
    pat = re.compile(r"a*bc*")
    for L in range(0, 8):
        for w in itertools.product("abc", repeat=L):
            s = "".join(w)
            _, _, acc = d.run(s.encode())
            assert acc == bool(pat.fullmatch(s)), s


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_closed_form_mod_counter(k):
    spec = gen.mod_counter_dfa(k, 3, counted=0)
    d = oracle.Dfa.from_spec(spec)
    flags, imax = d.isets()
    assert imax == k and flags[:, :k].all()   # every I_c = Q, gamma = 1
    data = gen.uniform_bytes(7 + k, 5000) % 3
    for n in (0, 1, 17, 999, 5000):
        _, fs, acc = d.run(data[:n])
        assert acc == (int(np.count_nonzero(data[:n] == 0)) % k == 0)
        assert fs == int(np.count_nonzero(data[:n] == 0)) % k


@pytest.mark.parametrize("word", [[0, 1, 1], [1, 0, 1, 0], [2, 2, 0, 1, 2]])
def test_closed_form_suffix_automaton(word):
    spec = gen.suffix_dfa(word, 3)
    d = oracle.Dfa.from_spec(spec)
    data = gen.uniform_bytes(11, 4000) % 3
    data[1000:1000 + len(word)] = word
    for n in range(0, 1100, 7):
        s = data[:n]
        _, _, acc = d.run(s)
        assert acc == bytes(s).endswith(bytes(word))
    # k-local (Sec. 7): k lookahead symbols determine the state, I_max,k = 1
    assert d.imax_r(len(word)) == 1


def _weak_compositions(n, parts):
    for cuts in itertools.combinations_with_replacement(range(n + 1), parts - 1):
        yield [0] + list(cuts) + [n]


@pytest.mark.parametrize("seed", range(5))
def test_every_chunking_equals_sequential(seed):
    spec = gen.random_dfa(500 + seed, 3 + seed, 2 + seed % 2, num_finals=2,
                          missing=0.15 * (seed % 3))
    d = oracle.Dfa.from_spec(spec)
    data = gen.uniform_bytes(600 + seed, 12) % spec.num_symbols
    for n in (0, 1, 5, 12):
        s = data[:n]
        _, fs, acc = d.run(s)
        for parts in (1, 2, 3, 4):
            for starts in _weak_compositions(n, parts):
                st, f2, a2, _ = d.chunked(s, starts)
                assert st == 0 and (f2, a2) == (fs, acc), (n, starts)


def test_random_chunkings_large_input():
    spec = gen.regex_dfa(9)
    d = oracle.Dfa.from_spec(spec)
    data = gen.zipf_text(9, 200_000)
    _, fs, acc = d.run(data)
    k = gen.key(9, 99)
    for trial in range(4):
        P = 1 + int(gen.below(gen.draws(k, 1, trial), 300)[0])
        cuts = np.sort(gen.below(gen.draws(k, P - 1, 1000 * (trial + 1)), len(data) + 1))
        starts = [0] + cuts.astype(np.int64).tolist() + [len(data)]
        st, f2, a2, _ = d.chunked(data, starts)
        assert (f2, a2) == (fs, acc)
    for P in (1, 2, 1024):
        st, f2, a2, _ = d.chunked(data, oracle.chunk_starts(len(data), P, 241))
        assert (f2, a2) == (fs, acc)


def _planted_wrong_merge(spec, data, starts, mistake):
    """Algorithm 3 restated in Python with one deliberate mistake."""
    ext = _ext(spec)
    Q = spec.num_states
    d = oracle.Dfa.from_spec(spec)
    flags, _ = d.isets()
    s = spec.q0
    for i in range(len(starts) - 1):
        a, b = starts[i], starts[i + 1]
        if i == 0 or a == 0:
            I = [spec.q0]
        else:
            look = data[a] if (mistake == "lookahead" and a < len(data)) else data[a - 1]
            I = list(np.nonzero(flags[look])[0])
            if mistake == "drop" and len(I) > 1:
                I = I[1:]
        L = list(range(Q + 1))
        for j in I:
            t = j
            for x in data[a:b]:
                t = ext[t, x]
            L[j] = t
        s = L[s]
    return s


@pytest.mark.parametrize("mistake", ["lookahead", "drop"])
def test_invariant_catches_planted_mistakes(mistake):
    caught = False
    for seed in range(40):
        spec = gen.random_dfa(700 + seed, 4, 2, num_finals=1)
        d = oracle.Dfa.from_spec(spec)
        data = (gen.uniform_bytes(800 + seed, 10) % 2).tolist()
        _, fs, _ = d.run(np.array(data, dtype=np.uint8))
        for starts in _weak_compositions(10, 3):
            if _planted_wrong_merge(spec, data, starts, mistake) != fs:
                caught = True
                break
        if caught:
            break
    assert caught


@pytest.mark.parametrize("seed", range(8))
def test_lemma_imax_nonincreasing(seed):
    spec = gen.random_dfa(900 + seed, 4 + seed % 3, 2 + seed % 2, num_finals=1,
                          missing=0.25 * (seed % 2))
    d = oracle.Dfa.from_spec(spec)
    vals = [d.imax_r(r) for r in range(1, 5)]
    assert all(a >= b for a, b in zip(vals, vals[1:])), vals
    _, imax1 = d.isets()
    assert vals[0] == imax1


@pytest.mark.parametrize("seed", range(4))
def test_eq13_word_sets_match_enumeration(seed):
    spec = gen.random_dfa(950 + seed, 5 + seed, 2 + seed % 2, num_finals=1, missing=0.2 * (seed % 2))
    d = oracle.Dfa.from_spec(spec)
    flags, _ = d.isets()
    for a in range(spec.num_symbols):                       # r = 1 is Eq. (11)
        assert d.iset_word([a]) == np.nonzero(flags[a])[0].tolist()
    for r in (2, 3):
        for word, img in d.isets_r(r).items():             # enumeration over all x in Q
            assert d.iset_word(list(word)) == sorted(img)
            assert set(img) <= set(np.nonzero(flags[word[-1]])[0].tolist())   # lemma per word


def test_composition_eq9_matches_sequential_merge():
    # each symbol permutes the states, so the chunk maps stay non-constant
    delta = np.stack([gen.permutation(gen.key(31, a), 7) for a in range(3)], axis=1)
    spec = gen.DfaSpec(7, 3, delta.astype(np.int32), 0, np.array([2, 5], dtype=np.uint32), None)
    d = oracle.Dfa.from_spec(spec)
    data = gen.uniform_bytes(32, 3000) % 3
    starts = oracle.chunk_starts(len(data), 9, 1)
    # Algorithm 2 style maps (all states) so composition is defined everywhere
    Q = spec.num_states
    maps = []
    for i in range(9):
        L = [d.delta_star(j, data[starts[i]:starts[i + 1]].tolist()) for j in range(Q + 1)]
        maps.append(np.array(L, dtype=np.uint32))
    # binary reduction (Eq. 9) in a tree equals left-to-right composition
    level = maps
    while len(level) > 1:
        nxt = [oracle.compose(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    _, fs, _ = d.run(data)
    assert level[0][spec.q0] == fs
    # and composing in the other order generally differs (no accidental symmetry)
    assert any(not np.array_equal(oracle.compose(maps[i], maps[i + 1]),
                                  oracle.compose(maps[i + 1], maps[i])) for i in range(8))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 36, 1000, 4 << 20, 10**10 + 7])
@pytest.mark.parametrize("P", [1, 2, 3, 7, 1024])
@pytest.mark.parametrize("m", [1, 2, 4, 241])
def test_partition_exact_and_tiles(n, P, m):
    r = oracle.partition(n, P, m)
    assert r[0][0] == 0 and r[-1][1] == n - 1
    for (a, b), (c, _) in zip(r, r[1:]):
        assert c == b + 1                      # contiguous, no gap or overlap
    # closed integer form of Eqs. (6) and (10) with w = 1
    for k in range(1, P):
        assert r[k][0] == (n * (m + k - 1)) // (m + P - 1)


# ---------------------------------------------------------------- excluded states
# Algorithm 3 leaves the error state q_e out of every initial-state set; the
# oracle's reading extends that to every non-accepting state that loops on all
# symbols (a run that reaches one never leaves it and is rejected) and keeps
# accepting absorbing states.  The two DFAs below are built by hand so that
# each plausible variant of the rule gives different sets: "exclude only q_e"
# puts q2 of ABSORB_REJECT into I_a; "also exclude accepting absorbing states"
# drops q1 of ABSORB_ACCEPT from I_a and I_b; "exclude states that loop on
# some symbol" drops q2 of ABSORB_ACCEPT from I_a.  Expected sets are written
# out from Eq. (11) by hand: I_sigma = image of delta(., sigma) over Q + {q_e},
# minus the excluded states.

# symbols a = 0, b = 1; -1 = q_e (state 4 here, state 3 below)
ABSORB_REJECT = dict(num_states=4, num_symbols=2, q0=0, finals=[3], delta=[
    [1, 2],    # q0: a -> q1, b -> q2
    [1, 3],    # q1: a -> q1, b -> q3
    [2, 2],    # q2: non-accepting, loops on a and b (absorbing, not q_e)
    [0, -1],   # q3: accepting; b -> q_e
])
ABSORB_ACCEPT = dict(num_states=3, num_symbols=2, q0=0, finals=[1], delta=[
    [1, 0],    # q0: a -> q1, b -> q0
    [1, 1],    # q1: accepting and absorbing
    [2, 0],    # q2: loops on a only
])


def _hand_dfa(d):
    return oracle.Dfa(d["num_states"], d["num_symbols"], np.array(d["delta"], dtype=np.int32),
                      d["q0"], d["finals"], None if d["num_symbols"] == 256 else
                      np.array([i if i < d["num_symbols"] else 0xFF for i in range(256)],
                               dtype=np.uint8))


def test_excluded_non_accepting_absorbing_state_besides_qe():
    o = _hand_dfa(ABSORB_REJECT)
    # q2 loops on every symbol and is not accepting; q_e (index 4) is the paper's error state
    assert o.excluded().tolist() == [False, False, True, False, True]
    flags, imax = o.isets()
    # I_a: q0->q1, q1->q1, q2->q2, q3->q0, q_e->q_e  = {q0, q1, q2, q_e} minus {q2, q_e}
    assert np.nonzero(flags[0])[0].tolist() == [0, 1]
    # I_b: q0->q2, q1->q3, q2->q2, q3->q_e, q_e->q_e = {q2, q3, q_e} minus {q2, q_e}
    assert np.nonzero(flags[1])[0].tolist() == [3]
    assert imax == 2


def test_excluded_keeps_accepting_absorbing_and_partial_loops():
    o = _hand_dfa(ABSORB_ACCEPT)
    # only q_e (index 3, unreachable here) is excluded: q1 is absorbing but
    # accepting, q2 loops on a but leaves on b
    assert o.excluded().tolist() == [False, False, False, True]
    flags, imax = o.isets()
    # I_a: q0->q1, q1->q1, q2->q2, q_e->q_e = {q1, q2, q_e} minus {q_e}
    assert np.nonzero(flags[0])[0].tolist() == [1, 2]
    # I_b: q0->q0, q1->q1, q2->q0, q_e->q_e = {q0, q1, q_e} minus {q_e}
    assert np.nonzero(flags[1])[0].tolist() == [0, 1]
    assert imax == 2


@pytest.mark.parametrize("which", ["reject", "accept"])
def test_excluded_states_keep_every_chunking_exact(which):
    """Excluding absorbing states never changes the answer (their identity
    entries in L_k are already right): every chunking of every string of
    length <= 7 equals Algorithm 1, and Algorithm 1 equals backward
    propagation of F."""
    d = ABSORB_REJECT if which == "reject" else ABSORB_ACCEPT
    o = _hand_dfa(d)
    spec = gen.DfaSpec(d["num_states"], d["num_symbols"], np.array(d["delta"], dtype=np.int32),
                       d["q0"], np.array(d["finals"], dtype=np.uint32), o.map)
    for L in range(0, 8):
        words = _all_words(2, L)
        want = _backward_accepts(spec, words)
        for w, acc in zip(words, want):
            data = np.array(w, dtype=np.uint8)
            st, fs, a = o.run(data)
            assert st == 0 and a == bool(acc)
            for cuts in itertools.combinations(range(1, L), min(2, max(0, L - 1))):
                starts = [0, *cuts, L]
                st2, fs2, a2, _ = o.chunked(data, starts)
                assert (st2, fs2, a2) == (st, fs, a), (w, starts)


def test_oracle_first_use_from_many_threads():
    """The CPU baseline runs the oracle on all host cores at once: concurrent
    builds and first loads of the C library must not collide."""
    import concurrent.futures as cf
    spec = gen.random_dfa(7, 9, 256, num_finals=2)
    data = gen.uniform_bytes(8, 10000)
    want = oracle.Dfa.from_spec(spec).run(data)

    def one(_):
        oracle.build(force=True)
        return oracle.Dfa.from_spec(spec).run(data)
    with cf.ThreadPoolExecutor(4) as ex:
        assert set(ex.map(one, range(4))) == {want}
