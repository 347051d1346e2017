"""GPU parity of DFA groups (several DFAs on one input, the input staged once
for all of them; Sec. 5): every DFA's answer bit-exact against the oracle
(Algorithm 1), every DFA's chunk maps entry by entry against the oracle's
Algorithm 3 on the same chunk starts (Eqs. 6-7, m = 1), the launch's lookup
count against the sum of L_k |I_k| computed from the oracle's sets, bytes
outside one DFA's Sigma, empty and ragged inputs, every chains-per-thread K,
and the full-size group workload."""
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


@pytest.fixture(scope="module")
def protein_group(dm):
    specs = gen.protein_group_dfas(7)
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    return specs, dfas, dm.Group(dfas)


def _expect(specs, data):
    return [oracle.Dfa.from_spec(s).run(data) for s in specs]


def _check(g, specs, dev, data, **kw):
    got = g.match(dev, **kw)
    want = _expect(specs, data)
    for i, ((st, fs, acc), (est, efs, eacc)) in enumerate(zip(got, want)):
        assert st == est, (i, kw, st, est)
        if st == 0:
            assert (fs, acc) == (efs, eacc), (i, kw)


def test_group_answers_equal_oracle(dm, protein_group):
    import torch
    specs, _, g = protein_group
    data = gen.protein_text(71, 300_001)
    dev = torch.from_numpy(data).cuda()
    for K in (0, 1, 2, 4, 8, 16):
        for P in (0, 1, 2, 7, 64, 1000, 20_000):
            _check(g, specs, dev, data, num_chunks=P, states_per_thread=K)


def test_group_empty_and_ragged_inputs(dm, protein_group):
    import torch
    specs, _, g = protein_group
    data = gen.protein_text(72, 70_000)
    for n in (0, 1, 2, 15, 16, 17, 31, 33, 4097, 65539):
        dev = torch.from_numpy(data[:n].copy()).cuda()
        for P in (0, 1, 3, 40):
            _check(g, specs, dev, data[:n], num_chunks=P)
    # more chunks than bytes: empty chunks are entered in q0 or pass the state on
    dev = torch.from_numpy(data[:5].copy()).cuda()
    _check(g, specs, dev, data[:5], num_chunks=9)


def test_group_chunk_maps_equal_algorithm3(dm, protein_group):
    import torch
    specs, _, g = protein_group
    data = gen.protein_text(73, 40_000)
    dev = torch.from_numpy(data).cuda()
    for P, K in ((1, 0), (3, 4), (40, 1), (40, 16)):
        maps, fs = g.chunk_maps(dev, num_chunks=P, states_per_thread=K)
        starts = oracle.chunk_starts(len(data), P, 1)
        for i, s in enumerate(specs):
            st, efs, _, want = oracle.Dfa.from_spec(s).chunked(data, starts, want_maps=True)
            qe = s.num_states + 1
            assert st == 0 and fs[i] == efs
            assert np.array_equal(maps[i, :, :qe].astype(np.uint32), want), (i, P, K)


def _work(specs, data, P):
    """sum over DFAs and chunks of L_k |I_k| (chunk 0 and chunks starting at 0
    use the start set {q0}), from the oracle's initial-state sets."""
    bounds = oracle.chunk_starts(len(data), P, 1)
    starts, ends = bounds[:-1], bounds[1:]
    total = 0
    for s in specs:
        o = oracle.Dfa.from_spec(s)
        sym = s.symbol_of_byte()
        for k, (a, b) in enumerate(zip(starts, ends)):
            if k == 0 or a == 0:
                size = 1
            else:
                size = len(o.iset(int(sym[data[a - 1]])))
            total += size * (b - a)
    return total


def test_group_lookup_count(dm, protein_group):
    import torch
    specs, _, g = protein_group
    data = gen.protein_text(74, 200_000)
    dev = torch.from_numpy(data).cuda()
    for P in (1, 13, 500):
        work = torch.zeros(1, dtype=torch.int64, device="cuda")
        out = torch.zeros(12 * g.count, dtype=torch.uint8, device="cuda")
        ws = torch.empty(g.workspace_size(len(data), num_chunks=P), dtype=torch.uint8, device="cuda")
        g.match_async(dev, out, ws, num_chunks=P, work=work)
        torch.cuda.synchronize()
        assert int(work.item()) == _work(specs, data, P), P


def test_group_bytes_outside_sigma(dm):
    """A byte-classed DFA (all 256 bytes in Sigma) grouped with protein DFAs:
    a byte outside the amino-acid letters fails only the protein DFAs, also
    when it is the lookahead byte of a chunk or the first or last byte."""
    import torch
    specs = [gen.class_dfa(75, 60, 8, 0.05, 0.4, 2, "byte")] + gen.protein_group_dfas(8, (20, 90))
    g = dm.Group([dm.Dfa.from_spec(s) for s in specs])
    assert g.info().joint_classes > 21
    base = gen.protein_text(76, 50_000)
    P = 10
    starts = oracle.chunk_starts(len(base), P, 1)
    for pos in (0, 1, starts[3] - 1, starts[3], 25_000, len(base) - 1):
        x = base.copy()
        x[pos] = ord("#")
        dev = torch.from_numpy(x).cuda()
        got = g.match(dev, num_chunks=P)
        want = _expect(specs, x)
        assert want[0][0] == 0 and want[1][0] == dm.ESYMBOL
        for (st, fs, acc), (est, efs, eacc) in zip(got, want):
            assert st == est and (st != 0 or (fs, acc) == (efs, eacc)), pos
    dev = torch.from_numpy(base).cuda()
    _check(g, specs, dev, base, num_chunks=P)


def test_group_of_one_and_paper_examples(dm):
    """A group of one DFA answers as dfa_match does; the paper's Fig. 1 and
    Fig. 6 DFAs grouped on their own example strings."""
    import torch
    from tests._golden import dfa_from, load, symbol_map
    w = gen.regex_workload(2, 4 << 20)
    d = dm.Dfa.from_spec(w.spec)
    g = dm.Group([d])
    dev = torch.from_numpy(w.data).cuda()
    (st, fs, acc), = g.match(dev)
    assert (st, fs, acc) == oracle.Dfa.from_spec(w.spec).run(w.data) == d.match(dev)
    specs = []
    texts = []
    for name in ("w1_fig1.txt", "w2_fig6.txt"):
        f = load(name)
        Q, syms, delta, q0, finals = dfa_from(f)
        specs.append(gen.DfaSpec(Q, len(syms), delta, q0, np.array(finals, np.uint32), symbol_map(syms)))
        texts.append(f["input"][0][0].encode())
    g2 = dm.Group([dm.Dfa.from_spec(s) for s in specs])
    for text in texts:
        x = np.frombuffer(text, dtype=np.uint8).copy()
        dev = torch.from_numpy(x).cuda()
        for P in (1, 2, 3, 5, 12, 36):
            for n in (len(x), len(x) // 2, 1):
                _check(g2, specs, dev[:n], x[:n], num_chunks=P)


def test_group_async_reuse_and_events(dm, protein_group):
    """One workspace reused by launches on a side stream, events around the
    match kernel; every launch's results against the oracle."""
    import torch
    specs, _, g = protein_group
    xs = [gen.protein_text(77 + i, 100_000 + 333 * i) for i in range(3)]
    want = [_expect(specs, x) for x in xs]
    ws = torch.empty(max(g.workspace_size(len(x)) for x in xs), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for e in ev:
        e.record(st)    # creates the events; the library re-records them around the match kernel
    devs = [torch.from_numpy(x).cuda() for x in xs]
    for rep in range(2):
        for x, dev, w in zip(xs, devs, want):
            out = torch.zeros(12 * g.count, dtype=torch.uint8, device="cuda")
            st.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(st):
                g.match_async(dev, out, ws, stream=st, events=ev)
            st.synchronize()
            assert ev[0].elapsed_time(ev[1]) > 0
            got = dm.results_from(out)
            for (fs, acc, s_), (es, efs, eacc) in zip(got, w):
                assert s_ == es and (s_ != 0 or (fs, acc) == (efs, eacc))


def _random_group(case):
    """1-16 random DFAs over the letters a-h: each maps a random subset of them
    (at least one) onto its symbols, so some letters are outside some DFAs'
    Sigma; random sizes, missing delta entries and accepting states."""
    u = gen.unit(gen.draws(gen.key(900 + case, 1), 64))
    G = 1 + int(u[0] * 16)
    specs = []
    for i in range(G):
        Q = 1 + int(u[1 + i] ** 2 * 300)
        m = np.full(256, 0xFF, dtype=np.uint8)
        letters = [c for j, c in enumerate(b"abcdefgh") if u[17 + (i + j) % 40] < 0.85 or j == 0]
        S = 1 + int(u[20 + i] * len(letters))
        for j, c in enumerate(letters):
            m[c] = j % S
        specs.append(gen.random_dfa(1000 * case + i, Q, S, num_finals=max(1, Q // 4),
                                    missing=0.1 * u[40 + i], byte_to_symbol=m))
    return specs, u


def test_group_random(dm):
    """Random groups, inputs, chunk counts and K against the oracle."""
    import torch
    done = 0
    for case in range(30):
        specs, u = _random_group(case)
        try:
            g = dm.Group([dm.Dfa.from_spec(s) for s in specs])
        except dm.DfaError as e:          # limits of a group (sets of one chunk, ...)
            assert e.status == dm.EINVAL
            continue
        n = int(u[60] * 200_000)
        x = (gen.uniform_bytes(case, n) % 8 + ord("a")).astype(np.uint8)
        if u[61] < 0.3 and n:
            x[int(u[62] * n)] = ord("z")     # outside every DFA's Sigma
        dev = torch.from_numpy(x).cuda()
        want = _expect(specs, x)
        for P in (0, 1 + int(u[63] * 3000)):
            for K in (0, 1, 2, 4, 8, 16):
                try:
                    got = g.match(dev, num_chunks=P, states_per_thread=K)
                except dm.DfaError as e:     # K too small for one chunk's sets
                    assert e.status == dm.EINVAL and K > 0
                    continue
                assert got == want, (case, P, K)
                done += 1
    assert done > 100


def test_group_sixteen_dfas(dm):
    """The largest group: 16 DFAs, one of 2000 states (the combine stages
    the CTA maps in batches that split a CTA's 16 rows); answers and chunk maps
    against the oracle."""
    import torch
    specs = gen.protein_group_dfas(12, tuple(range(8, 68, 4))) + gen.protein_group_dfas(13, (2000,))
    assert len(specs) == 16
    g = dm.Group([dm.Dfa.from_spec(s) for s in specs])
    assert g.info().max_states_ext == 2001 and g.info().state_bytes == 2
    data = gen.protein_text(79, 500_000)
    dev = torch.from_numpy(data).cuda()
    for P in (0, 1, 5, 500):
        _check(g, specs, dev, data, num_chunks=P)
    maps, fs = g.chunk_maps(dev[:30_000], num_chunks=6)
    starts = oracle.chunk_starts(30_000, 6, 1)
    for i in (0, 7, 15):
        st, efs, _, want = oracle.Dfa.from_spec(specs[i]).chunked(data[:30_000], starts, want_maps=True)
        assert st == 0 and fs[i] == efs
        assert np.array_equal(maps[i, :, :specs[i].num_states + 1].astype(np.uint32), want), i


def test_group_host_input(dm, protein_group):
    """dfa_group_match on host input (bytes, numpy, pinned and pageable CPU
    tensors) gives the answers of device input and of the oracle; the group's
    buffers grow and are reused across calls of different sizes."""
    import torch
    specs, _, g = protein_group
    for n in (0, 1, 5_000, 3_000_001, 40_000):
        x = gen.protein_text(80 + n % 7, n)
        want = _expect(specs, x)
        assert g.match(x) == want
        assert g.match(bytes(x)) == want
        assert g.match(torch.from_numpy(x)) == want
        assert g.match(torch.from_numpy(x).pin_memory()) == want
        assert g.match(torch.from_numpy(x).cuda()) == want


def test_group_host_input_pipelined(dm, protein_group):
    """Host input of 32 MiB and more is copied in segments while the earlier
    segments are matched (continuation launches and Eq. 8 over their state
    maps): answers against the oracle, also with a byte outside Sigma at a
    segment boundary (the last byte of one segment, the first of the next)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    specs, _, g = protein_group
    n = (64 << 20) + 7                      # segments of 16, 16, 16 and 16 MiB + 7
    base = gen.protein_text(85, n)
    cases = [base]
    for pos in ((16 << 20) - 1, 32 << 20):
        x = base.copy()
        x[pos] = ord("#")
        cases.append(x)
    with ThreadPoolExecutor(len(specs)) as ex:
        for x in cases:
            want = list(ex.map(lambda s: oracle.Dfa.from_spec(s).run(x), specs))
            assert g.match(x) == want
            assert g.match(torch.from_numpy(x).pin_memory()) == want
            assert g.match(torch.from_numpy(x).cuda()) == want


def test_group_autotune(dm):
    """The tuner keeps one of the candidates as the group's default; answers
    with the tuned default equal the oracle's."""
    import torch
    specs = gen.protein_group_dfas(11, (24, 150, 400))
    g = dm.Group([dm.Dfa.from_spec(s) for s in specs])
    data = gen.protein_text(78, 3 << 20)
    dev = torch.from_numpy(data).cuda()
    K, c, ms = g.autotune(dev)
    info = g.info()
    assert K in (1, 2, 4, 8, 16) and c in (1, 2) and ms > 0
    assert (info.states_per_thread, info.ctas_per_sm) == (K, c)
    _check(g, specs, dev, data)
    _check(g, specs, dev[:77_777], data[:77_777], num_chunks=33)


def test_group_rejections(dm, protein_group):
    import torch
    _, dfas, g = protein_group
    dev = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    out = torch.zeros(12 * g.count, dtype=torch.uint8, device="cuda")
    ws = torch.empty(g.workspace_size(1000), dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DfaError) as e:                    # K not in {1, 2, 4, 8, 16}
        g.match_async(dev, out, ws, states_per_thread=3)
    assert e.value.status == dm.EINVAL
    with pytest.raises(dm.DfaError) as e:                    # workspace too small
        g.match_async(dev, out, ws[: 256], num_chunks=900)
    assert e.value.status == dm.ENOSPACE
    with pytest.raises(dm.DfaError) as e:                    # misaligned result pointer
        g.match_async(dev, out[1:], ws)
    assert e.value.status == dm.EINVAL
    with pytest.raises(dm.DfaError) as e:                    # host-only and device DFAs mixed
        dm.Group([dfas[0], dm.Dfa.from_spec(gen.protein_group_dfas(9, (30,))[0], host_only=True)])
    assert e.value.status == dm.EINVAL
    # a group of sets too large for one CTA at small K: K = 1 needs more than 512 threads
    big = [dm.Dfa.from_spec(s) for s in gen.protein_group_dfas(10, (1500, 1500))]
    gb = dm.Group(big)
    with pytest.raises(dm.DfaError) as e:
        gb.plan_chunks(1 << 20, states_per_thread=1)
    assert e.value.status == dm.EINVAL
    assert gb.plan_chunks(1 << 20) >= 1


@pytest.mark.slow
def test_group_full_size(dm):
    """The group workload the bench times: 8 protein-shaped DFAs on 1 GiB of
    protein text, every answer against the oracle (one host thread per DFA)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    specs = gen.protein_group_dfas(7)
    data = gen.protein_text(3, 1 << 30)
    g = dm.Group([dm.Dfa.from_spec(s) for s in specs])
    dev = torch.from_numpy(data).cuda()
    with ThreadPoolExecutor(len(specs)) as ex:
        want = list(ex.map(lambda s: oracle.Dfa.from_spec(s).run(data), specs))
    for K in (0, 2, 4):
        got = g.match(dev, states_per_thread=K)
        for (st, fs, acc), (est, efs, eacc) in zip(got, want):
            assert st == est and (st != 0 or (fs, acc) == (efs, eacc)), K
