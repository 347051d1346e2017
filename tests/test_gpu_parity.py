"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact
(final state and accept bit; the answer of a membership test is unique, so the
tolerance is zero).  Covers the paper's examples, random and closed-form DFAs,
every workload DFA, empty/ragged inputs, bytes outside Sigma, Algorithm 2
(lookahead 0), the multiplicity of Eq. (10), the async and batched entry
points, and the full-size regex- and protein-shaped workloads."""
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


def _expect(spec, data):
    st, fs, acc = oracle.Dfa.from_spec(spec).run(data)
    return st, fs, acc


def _check(dm, d, spec, data, **kw):
    st, fs, acc = d.match(data, **kw)
    est, efs, eacc = _expect(spec, data)
    assert st == est, (st, est, kw)
    if st == 0:
        assert (fs, acc) == (efs, eacc), kw


def test_paper_examples(dm):
    from tests._golden import dfa_from, load, symbol_map
    for name in ("w1_fig1.txt", "w2_fig6.txt"):
        f = load(name)
        Q, syms, delta, q0, finals = dfa_from(f)
        spec = gen.DfaSpec(Q, len(syms), delta, q0, np.array(finals, np.uint32), symbol_map(syms))
        d = dm.Dfa.from_spec(spec)
        text = f["input"][0][0].encode()
        for P in (1, 2, 3, 5, 12, 36, 100):
            for m in (1, 2, 4):
                _check(dm, d, spec, text, num_chunks=P, multiplicity=m)
        for n in range(len(text) + 1):
            _check(dm, d, spec, text[:n], num_chunks=3)


@pytest.mark.parametrize("seed", range(6))
def test_random_dfas_many_chunkings(dm, seed):
    Q = [2, 5, 17, 60, 255, 300][seed]
    S = [2, 3, 7, 256, 20, 64][seed]
    spec = gen.random_dfa(3000 + seed, Q, S, num_finals=max(1, Q // 5),
                          missing=0.02 if seed % 2 else 0.0)
    if S != 256:
        m = np.full(256, 0xFF, dtype=np.uint8)
        m[:S] = np.arange(S)
        spec.byte_to_symbol = m
    d = dm.Dfa.from_spec(spec)
    data = gen.uniform_bytes(4000 + seed, 300_000)
    if S != 256:
        data = (data % S).astype(np.uint8)
    for n in (0, 1, 7, 8, 9, 15, 16, 17, 100, 1000, 4097, 65537, 300_000):
        for P in (0, 1, 2, 3, 17, 1024):
            _check(dm, d, spec, data[:n], num_chunks=P)


def test_one_dfa_from_many_host_threads(dm):
    """Matching calls only read a dfa_t: eight host threads matching host and
    device strings through one dfa_t at once all get the oracle's answers."""
    import threading
    import torch
    w = gen.regex_workload(2, 8 << 20)
    d = dm.Dfa.from_spec(w.spec)
    xs = [w.data[i * 700_001: i * 700_001 + 3_000_000 - 17 * i] for i in range(8)]
    want = [oracle.Dfa.from_spec(w.spec).run(x) for x in xs]
    devs = [torch.from_numpy(x.copy()).cuda() if i % 2 else x for i, x in enumerate(xs)]
    got = [None] * len(xs)
    errors = []

    def one(i):
        try:
            for _ in range(3):
                got[i] = d.match(devs[i], num_chunks=0 if i < 4 else 100 + i)
        except Exception as e:      # reported below
            errors.append(e)
    ts = [threading.Thread(target=one, args=(i,)) for i in range(len(xs))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    assert got == want


def test_random_options(dm):
    """Random DFAs, inputs and launch options together: sizes 1-700 states over
    1-40 symbols on random byte subsets, missing entries, bytes outside Sigma,
    chunk counts, multiplicities, lookahead depths 0-4, placement windows and
    tunings, each answer against the oracle (Algorithm 1)."""
    done = 0
    for case in range(40):
        u = gen.unit(gen.draws(gen.key(7000 + case, 3), 32))
        Q = 1 + int(u[0] ** 2 * 700)
        S = 1 + int(u[1] * 40)
        m = np.full(256, 0xFF, dtype=np.uint8)
        alphabet = gen.permutation(gen.key(7000 + case, 4), 256)[: S + int(u[2] * 3 * S)]
        m[alphabet] = np.arange(len(alphabet)) % S
        spec = gen.random_dfa(7100 + case, Q, S, num_finals=max(1, Q // 3),
                              missing=0.15 * u[3], byte_to_symbol=m)
        d = dm.Dfa.from_spec(spec)
        n = int(u[4] ** 2 * 400_000)
        x = alphabet[gen.below(gen.draws(gen.key(7200 + case, 5), n), len(alphabet))].astype(np.uint8)
        if u[5] < 0.25 and n:
            outside = np.nonzero(m == 0xFF)[0]
            x[int(u[6] * n)] = outside[int(u[7] * len(outside))]
        if u[8] < 0.5:
            try:      # a K too small for the DFA's largest set is refused (DFA_EINVAL)
                d.set_tuning(states_per_thread=[2, 4, 8, 16][int(u[9] * 4)],
                             tiles_per_cta=1 + int(u[10] * 16), ctas_per_sm=1 + int(u[11] * 3))
            except dm.DfaError as e:
                assert e.status == dm.EINVAL
        for trial in range(4):
            v = gen.unit(gen.draws(gen.key(7300 + case, 6 + trial), 8))
            kw = {"num_chunks": 0 if v[0] < 0.4 else 1 + int(v[1] ** 2 * 5000),
                  "lookahead": int(v[2] * 5) if Q < 4096 else 1}
            if kw["lookahead"] >= 1 and v[3] < 0.3:
                kw["boundary_window"] = [1, 16, 256, 4096][int(v[4] * 4)]
            if v[5] < 0.3:
                kw["multiplicity"] = 1 + int(v[6] * 8)
            _check(dm, d, spec, x, **kw)
            done += 1
    assert done == 160


@pytest.mark.parametrize("Q,S,missing", [(16, 256, 0.0), (15, 5, 0.2), (8, 3, 0.0),
                                         (3, 2, 0.3), (12, 40, 0.05)])
def test_byte_row_dfas(dm, Q, S, missing):
    """DFAs whose chains visit at most 16 states are stepped by byte permutes
    of 16-byte class rows.  Codes with bit 3 of the state set (states 8-15)
    take the upper half of a row; q_e is the 16th state when |Q| = 15.  Every
    chains-per-thread choice, Algorithm 2, Eq. 13 sets and a batch, against
    the oracle."""
    import torch
    spec = gen.random_dfa(5000 + Q, Q, S, num_finals=max(1, Q // 4), missing=missing)
    if S != 256:
        m = np.full(256, 0xFF, dtype=np.uint8)
        m[:S] = np.arange(S)
        spec.byte_to_symbol = m
    d = dm.Dfa.from_spec(spec)
    assert d.info().byte_rows == 1
    data = gen.uniform_bytes(6000 + Q, 1 << 20)
    if S != 256:
        data = (data % S).astype(np.uint8)
    for K in (2, 4, 8, 16):
        d.set_tuning(states_per_thread=K)
        for n in (0, 1, 17, 4097, 1 << 20):
            for P in (0, 1, 3, 1024):
                _check(dm, d, spec, data[:n], num_chunks=P)
    _check(dm, d, spec, data, lookahead=0)
    _check(dm, d, spec, data, lookahead=3, num_chunks=500)
    _check(dm, d, spec, data, boundary_window=64)
    xs = [data[: 1000 * (i + 1) + i] for i in range(5)]
    res = dm.match_batch([d] * 5, [torch.from_numpy(x).cuda() for x in xs])
    for x, (fs, acc, st) in zip(xs, res):
        assert (st, fs, acc) == _expect(spec, x)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_mod_counter_gamma_one(dm, k):
    spec = gen.mod_counter_dfa(k, 3)
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[:3] = np.arange(3)
    spec.byte_to_symbol = m
    d = dm.Dfa.from_spec(spec)
    assert d.info().i_max == k
    data = (gen.uniform_bytes(77, 1 << 20) % 3).astype(np.uint8)
    for n in (0, 5, 1000, 1 << 20):
        _check(dm, d, spec, data[:n])
        _check(dm, d, spec, data[:n], num_chunks=999)


def test_suffix_automaton(dm):
    word = [1, 0, 2, 2, 1]
    spec = gen.suffix_dfa(word, 3)
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[:3] = np.arange(3)
    spec.byte_to_symbol = m
    d = dm.Dfa.from_spec(spec)
    data = (gen.uniform_bytes(78, 1 << 20) % 3).astype(np.uint8)
    data[-5:] = word
    for n in (5, 4096, 1 << 20):
        st, fs, acc = d.match(data[:n])
        assert acc == bytes(data[:n]).endswith(bytes(word))
        _check(dm, d, spec, data[:n], num_chunks=333)


def test_plain_workload_full_size(dm):
    w = gen.plain_workload(1)
    d = dm.Dfa.from_spec(w.spec)
    _check(dm, d, w.spec, w.data, num_chunks=w.num_chunks)
    _check(dm, d, w.spec, w.data)
    for seed in range(2, 6):
        data = gen.uniform_bytes(seed, (4 << 20) - seed * 1111)
        _check(dm, d, w.spec, data, num_chunks=1024)


@pytest.mark.parametrize("maker,n", [("regex", 16 << 20), ("protein", 16 << 20)])
def test_shaped_workloads_reduced(dm, maker, n):
    w = gen.regex_workload(2, n) if maker == "regex" else gen.protein_workload(3, n)
    d = dm.Dfa.from_spec(w.spec)
    _check(dm, d, w.spec, w.data)
    for P in (1, 7, 4096, 100_000):
        _check(dm, d, w.spec, w.data, num_chunks=P)
    # ragged lengths and an accepted ending (a planted word drives every state into F)
    word = np.frombuffer(w.spec.meta["planted_words"][0], dtype=np.uint8)
    data = w.data[: n - 12345].copy()
    data[-len(word):] = word
    st, fs, acc = d.match(data)
    assert st == 0 and acc
    _check(dm, d, w.spec, data)


def test_symbols_outside_sigma(dm):
    spec = gen.protein_dfa(3)
    d = dm.Dfa.from_spec(spec)
    data = gen.protein_text(3, 1 << 20)
    for pos in (0, 1, 4095, 4096, 500_000, (1 << 20) - 1):
        bad = data.copy()
        bad[pos] = ord("B")
        for P in (0, 1, 2, 1000):
            st, fs, acc = d.match(bad, num_chunks=P)
            assert st == dm.ESYMBOL, (pos, P)
    st, _, _ = d.match(data)
    assert st == 0


def test_empty_and_tiny_inputs(dm):
    spec = gen.regex_dfa(2)
    d = dm.Dfa.from_spec(spec)
    st, fs, acc = d.match(b"")
    assert (st, fs) == (0, spec.q0)
    for n in range(1, 40):
        _check(dm, d, spec, gen.zipf_text(5, n))
        _check(dm, d, spec, gen.zipf_text(5, n), num_chunks=n + 3)


def test_algorithm2_and_multiplicity(dm):
    for spec, data in ((gen.regex_dfa(2), gen.zipf_text(2, 3 << 20)),
                       (gen.plain_dfa(1), gen.uniform_bytes(1, 3 << 20))):
        d = dm.Dfa.from_spec(spec)
        for la in (0, 1):
            for m in (1, 3, 241):
                _check(dm, d, spec, data, lookahead=la, multiplicity=m)
                _check(dm, d, spec, data, lookahead=la, multiplicity=m, num_chunks=5000)


def test_async_with_torch_buffers(dm):
    import torch
    w = gen.regex_workload(2, 8 << 20)
    d = dm.Dfa.from_spec(w.spec)
    dev = torch.from_numpy(w.data).cuda()
    ws = torch.empty(d.workspace_size(dev.numel()), dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            d.match_async(dev, out, ws, stream=s)
    s.synchronize()
    (fs, acc, st), = dm.results_from(out)
    est, efs, eacc = _expect(w.spec, w.data)
    assert (st, fs, acc) == (0, efs, eacc)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DfaError):
        d.match_async(dev, out, small)


def _batch_mix(seed, count, max_len):
    specs = gen.batch_dfas(seed, 8)
    lens = gen.batch_lengths(seed, count, 1, max_len)
    lens[:3] = [0, 1, 2]
    picks = gen.batch_picks(seed, count, len(specs))
    datas = [gen.batch_text(seed * 7919 + i, specs[picks[i]], int(lens[i])) for i in range(count)]
    return specs, picks, datas


def test_batch_matches_oracle_and_graph_replay(dm):
    import torch
    specs, picks, datas = _batch_mix(11, 300, 1 << 20)
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    tens = [torch.from_numpy(x).cuda() for x in datas]
    expect = [_expect(specs[picks[i]], datas[i]) for i in range(len(datas))]
    res = dm.match_batch([dfas[p] for p in picks], tens)
    for (fs, acc, st), (est, efs, eacc) in zip(res, expect):
        assert st == est and (st != 0 or (fs, acc) == (efs, eacc))
    b = dm.Batch([dfas[p] for p in picks], tens)
    out = torch.zeros(12 * len(tens), dtype=torch.uint8, device="cuda")
    for graph in (False, True, True):
        out.zero_()
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        assert dm.results_from(out) == res
    # the same tests one at a time give the same answers
    for i in range(0, len(tens), 37):
        st, fs, acc = dfas[picks[i]].match(tens[i])
        assert (fs, acc) == res[i][:2] or st != 0


@pytest.fixture(scope="module")
def regex_1gib():
    """The benchmark's regex workload at full size, on the device, with the
    oracle's answer (Algorithm 1 on the whole GiB, computed once)."""
    import torch
    w = gen.regex_workload(2, 1 << 30)
    dev = torch.from_numpy(w.data).cuda()
    return w, dev, _expect(w.spec, w.data)


@pytest.fixture(scope="module")
def protein_10gb():
    import torch
    w = gen.protein_workload(3, 10 * 10**9)
    dev = torch.from_numpy(w.data).cuda()
    return w, dev, _expect(w.spec, w.data)


def _async_answer(dm, d, dev, **kw):
    import torch
    ws = torch.empty(d.workspace_size(dev.numel(), **kw), dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    d.match_async(dev, out, ws, **kw)
    torch.cuda.synchronize()
    (fs, acc, st), = dm.results_from(out)
    return (st, fs, acc) if st == 0 else (st, None, None)


@pytest.mark.slow
@pytest.mark.parametrize("tuning", ["default", "autotuned", "fixed_2_2_2"])
@pytest.mark.parametrize("window", [0, 256])
def test_regex_full_size_1GiB(dm, regex_1gib, tuning, window):
    """The benchmarked configurations at the size they are timed: the starts of
    Eqs. 6-7 (the headline) and Sec. 4.2 placement within 256 bytes, under the
    library defaults, the autotuner's pick on this input, and K = 2 with 2
    tiles and 2 CTAs per SM."""
    w, dev, want = regex_1gib
    d = dm.Dfa.from_spec(w.spec)
    if tuning == "autotuned":
        d.autotune(dev, boundary_window=window)
    elif tuning == "fixed_2_2_2":
        d.set_tuning(states_per_thread=2, tiles_per_cta=2, ctas_per_sm=2, boundary_window=window)
    assert _async_answer(dm, d, dev, boundary_window=window) == want


@pytest.mark.slow
@pytest.mark.parametrize("window", [0, 256])
def test_regex_full_size_1GiB_pinned_host_pipeline(dm, regex_1gib, window):
    """dfa_match on a pinned 1 GiB host buffer: the segmented copy/match
    pipeline the end-to-end figure times, twice in a row."""
    w, dev, want = regex_1gib
    import torch
    d = dm.Dfa.from_spec(w.spec)
    pinned = torch.from_numpy(w.data).pin_memory()
    for _ in range(2):
        assert d.match(pinned, boundary_window=window) == want


@pytest.mark.slow
@pytest.mark.parametrize("tuning,window", [("default", 0), ("autotuned", 0), ("default", 256),
                                           ("autotuned", 256)])
def test_protein_full_size_10GB(dm, protein_10gb, tuning, window):
    w, dev, want = protein_10gb
    d = dm.Dfa.from_spec(w.spec)
    if tuning == "autotuned":
        d.autotune(dev[: 1 << 30], boundary_window=window)
    assert _async_answer(dm, d, dev, boundary_window=window) == want


def _expected_set_sizes(spec, data, P, r):
    """|I_k| per chunk from the oracle: Eq. (13) on the min(r, Start(k)) symbols
    before chunk k (Eq. 11 when that is one symbol); 1 for the start set."""
    od = oracle.Dfa.from_spec(spec)
    starts = oracle.chunk_starts(len(data), P, 1)
    sym = od.symbols(data)
    out = []
    for k in range(P):
        st = starts[k]
        if k == 0 or st == 0:
            out.append(1)
            continue
        j = min(r, st) if r >= 1 else 0
        out.append(len(od.iset_word(sym[st - j:st].tolist())))
    return out


@pytest.mark.parametrize("r", [2, 3, 4])
def test_lookahead_r_symbols_parity(dm, r):
    from tests._golden import dfa_from, load, symbol_map
    for name in ("w1_fig1.txt", "w2_fig6.txt"):
        f = load(name)
        Q, syms, delta, q0, finals = dfa_from(f)
        spec = gen.DfaSpec(Q, len(syms), delta, q0, np.array(finals, np.uint32), symbol_map(syms))
        d = dm.Dfa.from_spec(spec)
        text = f["input"][0][0].encode()
        for P in (1, 2, 3, 7, 36):
            _check(dm, d, spec, text, num_chunks=P, lookahead=r)
    for seed in range(3):
        spec = gen.random_dfa(6000 + seed, [5, 40, 300][seed], [2, 7, 20][seed], num_finals=3,
                              missing=0.05 * seed)
        m = np.full(256, 0xFF, dtype=np.uint8)
        m[:spec.num_symbols] = np.arange(spec.num_symbols)
        spec.byte_to_symbol = m
        d = dm.Dfa.from_spec(spec)
        data = (gen.uniform_bytes(6100 + seed, 200_000) % spec.num_symbols).astype(np.uint8)
        for n in (0, 1, 2, 3, 5, 100, 200_000):
            for P in (0, 2, 3, 77, 5000):
                _check(dm, d, spec, data[:n], num_chunks=P, lookahead=r)
    for w in (gen.regex_workload(2, 8 << 20), gen.protein_workload(3, 8 << 20)):
        d = dm.Dfa.from_spec(w.spec)
        for P in (0, 3000):
            _check(dm, d, w.spec, w.data, num_chunks=P, lookahead=r)


@pytest.mark.parametrize("r", [1, 2, 4])
def test_lookahead_sets_equal_eq13(dm, r):
    import torch
    for w in (gen.regex_workload(2, 1 << 20), gen.protein_workload(3, 1 << 20)):
        d = dm.Dfa.from_spec(w.spec)
        dev = torch.from_numpy(w.data).cuda()
        P = 2000
        got = d.plan_sets(dev, num_chunks=P, lookahead=r).tolist()
        assert got == _expected_set_sizes(w.spec, w.data, P, r)
        if r > 1:  # the lemma of Sec. 4.3, chunk by chunk
            one = d.plan_sets(dev, num_chunks=P, lookahead=1)
            assert all(a <= b for a, b in zip(got, one.tolist()))


def test_lookahead_sets_with_bad_byte(dm):
    spec = gen.protein_dfa(3)
    d = dm.Dfa.from_spec(spec)
    data = gen.protein_text(3, 1 << 20)
    for pos in (0, 2, 1000, 4096, 4097):
        bad = data.copy()
        bad[pos] = ord("J")
        for r in (2, 4):
            st, _, _ = d.match(bad, num_chunks=256, lookahead=r)
            assert st == dm.ESYMBOL


def test_many_dfas_on_one_input(dm):
    """Several DFAs matched against the same input in one launch (the paper's
    representation allows one input to be run by several DFAs, Sec. 5): each
    result equals that DFA run alone and the oracle."""
    import torch
    # 8 DFAs, as the bench's several-DFA leg: the regex-shaped DFA, 6 byte DFAs of
    # the batched mix and one 256-class table read through L2
    specs = [gen.regex_dfa(2)] + [s for s in gen.batch_dfas(21, 16) if s.byte_to_symbol is None][:6]
    specs.append(gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte"))
    assert len(specs) == 8
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    x = gen.zipf_text(22, 3 << 20)
    dev = torch.from_numpy(x).cuda()
    res = dm.match_batch(dfas, [dev] * len(dfas))
    for (fs, acc, st), s, d in zip(res, specs, dfas):
        est, efs, eacc = _expect(s, x)
        assert (st, fs, acc) == (est, efs, eacc)
        assert d.match(dev) == (st, fs, acc)


def test_batch_dfa_switch_keeps_each_tests_own_dfa(dm):
    """Regression: a test finished at the start of a tile of another DFA must
    take its accept flags and state count from its own DFA.  Here DFA A
    accepts in every state and DFA B in none, so every accept bit is
    determined by the test's DFA; B also has more states than A."""
    import torch
    a = gen.random_dfa(71, 20, 256)
    a.finals = np.arange(20, dtype=np.uint32)
    b = gen.random_dfa(72, 300, 256, num_finals=0)
    b.finals = np.zeros(0, dtype=np.uint32)
    da, db = dm.Dfa.from_spec(a), dm.Dfa.from_spec(b)
    lens = gen.batch_lengths(73, 400, 1, 200_000)
    datas = [gen.uniform_bytes(74 + i, int(n)) for i, n in enumerate(lens)]
    dfas = [da if i % 2 == 0 else db for i in range(len(datas))]
    tens = [torch.from_numpy(x).cuda() for x in datas]
    res = dm.match_batch(dfas, tens)
    for i, (fs, acc, st) in enumerate(res):
        spec = a if i % 2 == 0 else b
        assert (st, fs, acc) == _expect(spec, datas[i])
        assert acc == (i % 2 == 0)


@pytest.mark.parametrize("kind", ["u16_large", "u8_256classes"])
def test_l2_placed_tables(dm, kind):
    """Tables that do not fit shared memory (or whose row offsets need more
    than 16 bits) are read through L2: 256 byte classes x 1288 states (uint16,
    659 KB) and 256 classes x 255 states (uint8, 66 KB)."""
    import torch
    if kind == "u16_large":
        spec = gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte")
    else:
        spec = gen.random_dfa(82, 255, 256, num_finals=20, missing=0.01)
    d = dm.Dfa.from_spec(spec)
    info = d.info()
    assert info.placement == 1 and info.num_classes == 256
    data = gen.zipf_text(83, 6 << 20) if kind == "u16_large" else gen.uniform_bytes(83, 6 << 20)
    for P in (0, 1, 5, 3000):
        for r in (1, 2):
            _check(dm, d, spec, data, num_chunks=P, lookahead=r)
    _check(dm, d, spec, data[: 12345], num_chunks=50)
    # batched together with a shared-memory DFA
    small = gen.regex_dfa(2)
    ds = dm.Dfa.from_spec(small)
    xs = [data[: 100_000 * (i + 1)] for i in range(6)]
    dev = [torch.from_numpy(x).cuda() for x in xs]
    res = dm.match_batch([d, ds, d, ds, d, ds], dev)
    for i, (fs, acc, st) in enumerate(res):
        spec_i = spec if i % 2 == 0 else small
        assert (st, fs, acc) == _expect(spec_i, xs[i])


def test_largest_dfa_and_k16(dm):
    """|Q| = 4095 (the largest DFA whose running maps stay in shared memory), a
    dense 20-letter alphabet so I_max is large and the planner needs K = 16 to
    fit a chunk into one tile."""
    spec = gen.class_dfa(91, 4095, 20, 0.3, 0.9, 40, "protein")
    d = dm.Dfa.from_spec(spec)
    info = d.info()
    assert info.i_max > 2048 and info.states_per_thread == 16
    data = gen.protein_text(92, 2 << 20)
    for P in (0, 1, 777):
        _check(dm, d, spec, data, num_chunks=P)
    _check(dm, d, spec, data, num_chunks=500, lookahead=0)   # Algorithm 2: all 4096 states


@pytest.mark.parametrize("which", ["fig6", "plain", "regex", "protein", "random_missing"])
def test_chunk_maps_equal_algorithm3(dm, which):
    """The chunk maps L_k the match kernel computes (Sec. 4.1: L_k[j] =
    delta*(j, chunk k) for j in I_k, identity elsewhere) equal the oracle's
    Algorithm 3 maps entry by entry, on the same partition."""
    import torch
    from tests._golden import dfa_from, load, symbol_map
    if which == "fig6":
        f = load("w2_fig6.txt")
        Q, syms, delta, q0, finals = dfa_from(f)
        spec = gen.DfaSpec(Q, len(syms), delta, q0, np.array(finals, np.uint32), symbol_map(syms))
        data = np.frombuffer((f["input"][0][0] * 40).encode(), dtype=np.uint8).copy()
    elif which == "plain":
        spec, data = gen.plain_dfa(1), gen.uniform_bytes(1, 1 << 20)
    elif which == "regex":
        spec, data = gen.regex_dfa(2), gen.zipf_text(2, 1 << 20)
    elif which == "protein":
        spec, data = gen.protein_dfa(3), gen.protein_text(3, 1 << 20)
    else:
        spec = gen.random_dfa(99, 40, 256, num_finals=5, missing=0.05)
        data = gen.uniform_bytes(98, 1 << 18)
    d = dm.Dfa.from_spec(spec)
    dev = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    od = oracle.Dfa.from_spec(spec)
    for P in (3, 257, 2000):
        if P > len(data):
            continue
        got, fs = d.chunk_maps(dev, num_chunks=P)
        st, efs, eacc, want = od.chunked(data, oracle.chunk_starts(len(data), P, 1), want_maps=True)
        assert st == 0 and fs == efs
        assert got.shape == want.shape
        assert np.array_equal(got.astype(np.uint32), want), (which, P)
        # with r = 2 the kernel matches fewer states; those it matches agree with Algorithm 3
        got2, fs2 = d.chunk_maps(dev, num_chunks=P, lookahead=2)
        ident = np.arange(spec.num_states + 1, dtype=np.uint32)[None, :]
        g2 = got2.astype(np.uint32)
        assert fs2 == efs
        assert np.all((g2 == want) | (g2 == ident))


def test_tuning_records_per_lookahead(dm):
    """A depth's own tuning record changes how its launches are planned, never
    their answer, and leaves the base record (lookahead 1) alone."""
    import torch
    w = gen.regex_workload(4, (3 << 20) + 77)
    d = dm.Dfa.from_spec(w.spec)
    dev = torch.from_numpy(w.data).cuda()
    want = oracle.Dfa.from_spec(w.spec).run(w.data)
    d.set_tuning(states_per_thread=8, tiles_per_cta=4, min_chunk_bytes=4096)
    d.set_tuning(states_per_thread=2, tiles_per_cta=16, min_chunk_bytes=512, lookahead=4)
    d.set_tuning(states_per_thread=16, tiles_per_cta=4, lookahead=0)
    assert (d.tuning().states_per_thread, d.tuning().tiles_per_cta) == (8, 4)
    assert (d.tuning(lookahead=4).states_per_thread, d.tuning(lookahead=4).tiles_per_cta) == (2, 16)
    assert d.tuning(lookahead=2).states_per_thread == 8       # no record of its own: the base
    assert d.plan_chunks(dev.numel(), lookahead=4) != d.plan_chunks(dev.numel(), lookahead=1)
    for r in (0, 1, 2, 4):
        assert d.match(dev, lookahead=r) == want, r
    t, ms = d.autotune(dev, lookahead=2)
    assert ms > 0 and d.tuning(lookahead=2).states_per_thread == t.states_per_thread
    assert d.tuning().states_per_thread == 8
    assert d.match(dev, lookahead=2) == want


def test_smem_table_beyond_16bit_row_offsets(dm):
    """A 32-class, 1288-state table (85 KB, row offsets above 16 bits) stays in
    shared memory: the 8-bit class stream addresses its rows without offsets."""
    spec = gen.class_dfa(93, 1288, 32, 0.02, 0.4, 12, "byte")
    d = dm.Dfa.from_spec(spec)
    info = d.info()
    assert info.placement == 0 and info.num_classes == 32 and info.state_bytes == 2
    assert 32 * 1288 * 2 > 0xFFFF
    data = gen.zipf_text(94, 5 << 20)
    for P in (0, 1, 7, 4000):
        for r in (0, 1, 3):
            _check(dm, d, spec, data, num_chunks=P, lookahead=r)


def test_lookup_probe_rates(dm):
    """The lookup-rate probe (the unit of work alone) runs on shared-memory and
    L2-placed tables and gives rates in the range the hardware allows: the
    shared-memory rate at most a little above SMs x 32 lanes x clock."""
    import torch
    props = torch.cuda.get_device_properties(0)
    d = dm.Dfa.from_spec(gen.regex_dfa(2))
    r = dm.probe_lookup_rate(d, 2048)
    peak = props.multi_processor_count * 32 * 2.07e9
    assert 0.3 * peak < r < 1.1 * peak, (r, peak)
    dl = dm.Dfa.from_spec(gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte"))
    assert dl.info().placement == 1
    rl = dm.probe_lookup_rate(dl, 512)
    assert 1e9 < rl < 1.1 * peak, rl
