"""Sec. 4.2 boundary placement on the GPU (opts.boundary_window), through the
C ABI, against the oracle:

* the chunk starts k_boundaries places equal the oracle's placement bit for
  bit (same window rule, same tie-breaks), for every workload DFA, several
  windows, multiplicities and lookahead depths;
* the set sizes the planner then charges, and the chunk maps L_k the match
  kernel computes on the placed chunks, equal the oracle's Algorithm 3 on the
  same chunks;
* the answer (final state, accept bit, status) equals Algorithm 1 on every
  entry point: async, synchronous (including the host pipeline), batched,
  allocation-free; bytes outside Sigma; empty and tiny inputs; Algorithm 2
  (which has no lookahead symbol and ignores the window).
"""
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


def _dev(data):
    import torch
    return torch.from_numpy(np.ascontiguousarray(data)).cuda()


def _workload(which):
    if which == "regex":
        return gen.regex_dfa(2), gen.zipf_text(2, (4 << 20) + 333)
    if which == "protein":
        return gen.protein_dfa(3), gen.protein_text(3, (4 << 20) + 17)
    if which == "plain":
        return gen.plain_dfa(1), gen.uniform_bytes(1, 4 << 20)
    return (gen.random_dfa(99, 40, 256, num_finals=5, missing=0.05),
            gen.uniform_bytes(98, (1 << 20) + 5))


@pytest.mark.parametrize("which", ["regex", "protein", "plain", "random_missing"])
def test_placed_starts_equal_oracle(dm, which):
    spec, data = _workload(which)
    d = dm.Dfa.from_spec(spec)
    od = oracle.Dfa.from_spec(spec)
    dev = _dev(data)
    n = len(data)
    for P, m, window in [(0, 1, 256), (1024, 1, 8), (3001, 1, 64), (97, 3, 4096), (5000, 1, 1),
                         (2, 1, 65536)]:
        P_used = d.plan_chunks(n, num_chunks=P, multiplicity=m, boundary_window=window)
        got = d.plan_starts(dev, num_chunks=P, multiplicity=m, boundary_window=window)
        want = oracle.boundary_starts(od, data, P_used, m, window)
        assert got.tolist() == want, (which, P, m, window)
        # no window: Eqs. (6)-(7), the same as dfa_partition
        plain = d.plan_starts(dev, num_chunks=P_used, multiplicity=m)
        assert plain.tolist() == oracle.chunk_starts(n, P_used, m)


@pytest.mark.parametrize("which", ["regex", "protein", "random_missing"])
def test_placed_sets_and_chunk_maps_equal_algorithm3(dm, which):
    spec, data = _workload(which)
    d = dm.Dfa.from_spec(spec)
    od = oracle.Dfa.from_spec(spec)
    dev = _dev(data[: 1 << 20])
    data = data[: 1 << 20]
    flags, _ = od.isets()
    size = flags.sum(axis=1)
    sym = od.symbols(data)
    for P, window in [(257, 512), (2000, 32)]:
        starts = oracle.boundary_starts(od, data, P, 1, window)
        sizes = d.plan_sets(dev, num_chunks=P, boundary_window=window)
        want_sizes = [1] + [int(size[sym[s - 1]]) for s in starts[1:-1]]
        assert sizes.tolist() == want_sizes
        got, fs = d.chunk_maps(dev, num_chunks=P, boundary_window=window)
        st, efs, eacc, want = od.chunked(data, starts, want_maps=True)
        assert st == 0 and fs == efs
        assert np.array_equal(got.astype(np.uint32), want), (which, P, window)
    # placement shrinks the regex-shaped work sum_k L_k |I_k| (Eq. 16's term)
    if which == "regex":
        P = 2000
        w0 = (np.diff(d.plan_starts(dev, num_chunks=P).astype(np.int64)) *
              d.plan_sets(dev, num_chunks=P).astype(np.int64)).sum()
        w1 = (np.diff(d.plan_starts(dev, num_chunks=P, boundary_window=256).astype(np.int64)) *
              d.plan_sets(dev, num_chunks=P, boundary_window=256).astype(np.int64)).sum()
        assert w1 * 3 < w0


@pytest.mark.parametrize("which", ["regex", "protein", "plain", "random_missing"])
def test_placed_answers_equal_oracle(dm, which):
    import torch
    spec, data = _workload(which)
    d = dm.Dfa.from_spec(spec)
    want = oracle.Dfa.from_spec(spec).run(data)
    dev = _dev(data)
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    for P in (0, 1, 2, 1024, 40000):
        for r in (0, 1, 2, 4):
            for window in (1, 16, 256):
                ws = torch.empty(d.workspace_size(len(data), num_chunks=P, lookahead=r,
                                                  boundary_window=window),
                                 dtype=torch.uint8, device="cuda")
                d.match_async(dev, out, ws, num_chunks=P, lookahead=r, boundary_window=window)
                torch.cuda.synchronize()
                (fs, acc, st), = dm.results_from(out)
                assert (st, fs, acc) == want, (which, P, r, window)


def test_placement_with_bytes_outside_sigma_and_tiny_inputs(dm):
    spec = gen.protein_dfa(3)
    d = dm.Dfa.from_spec(spec)
    od = oracle.Dfa.from_spec(spec)
    data = gen.protein_text(5, 1 << 20)
    for pos in (0, 4095, 524287, (1 << 20) - 1):
        bad = data.copy()
        bad[pos] = ord("#")
        for P in (0, 256):
            st, fs, acc = d.match(_dev(bad), num_chunks=P, boundary_window=128)
            assert st == oracle.ESYMBOL and st == od.run(bad)[0], pos
    for n in (0, 1, 2, 3, 7, 64, 1000):
        for P in (0, 1, 3, 16):
            got = d.match(_dev(data[:n]) if n else data[:0], num_chunks=P, boundary_window=4096)
            assert got == od.run(data[:n]), (n, P)


def test_placement_batched_pipelined_and_noalloc(dm):
    import torch
    w = gen.regex_workload(5, (6 << 20) + 12345)
    d = dm.Dfa.from_spec(w.spec)
    od = oracle.Dfa.from_spec(w.spec)
    want = od.run(w.data)
    # host pipeline: later segments are continuation map tests with placed chunks
    d.set_tuning(host_segment_bytes=(1 << 20) + 7)
    host = torch.empty(len(w.data), dtype=torch.uint8, pin_memory=True)
    host.numpy()[:] = w.data
    for r in (1, 4):
        assert d.match(host, lookahead=r, boundary_window=256) == want, r
    # batch of many lengths, two DFAs
    p = gen.protein_workload(3, 2 << 20)
    dp = dm.Dfa.from_spec(p.spec)
    lens = [0, 1, 300, 5000, 70000, 1 << 20, len(w.data)]
    tensors, dfas, expect = [], [], []
    for i, n in enumerate(lens):
        for dd, spec, src in ((d, w.spec, w.data), (dp, p.spec, p.data)):
            s = np.ascontiguousarray(src[:n])
            tensors.append(_dev(s))
            dfas.append(dd)
            st, fs, acc = oracle.Dfa.from_spec(spec).run(s)
            expect.append((fs or 0, bool(acc), st))
    for window in (0, 64, 1024):
        got = dm.match_batch(dfas, tensors, boundary_window=window)
        assert got == expect, window
    # the allocation-free entry point with placement equals the async one
    dev = _dev(w.data)
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    d.match_noalloc(dev, out, boundary_window=256)
    torch.cuda.synchronize()
    (fs, acc, st), = dm.results_from(out)
    assert (st, fs, acc) == want


def test_placed_tuning_records_and_kernel_count(dm):
    """Placed launches keep their own tuning record per depth; a record never
    set reads as the unplaced one; the launch gains one kernel (k_boundaries)."""
    w = gen.regex_workload(4, (3 << 20) + 77)
    d = dm.Dfa.from_spec(w.spec)
    dev = _dev(w.data)
    want = oracle.Dfa.from_spec(w.spec).run(w.data)
    d.set_tuning(states_per_thread=4, tiles_per_cta=8)
    assert d.tuning(boundary_window=256).states_per_thread == 4
    d.set_tuning(states_per_thread=2, tiles_per_cta=16, boundary_window=256)
    assert d.tuning(boundary_window=256).tiles_per_cta == 16
    assert d.tuning(boundary_window=1).tiles_per_cta == 16    # any window: the placed record
    assert d.tuning().tiles_per_cta == 8
    n = dev.numel()
    assert d.num_kernels(n, boundary_window=256) == d.num_kernels(n) + 1
    assert d.num_kernels(n, lookahead=0, boundary_window=256) == d.num_kernels(n, lookahead=0)
    t, ms = d.autotune(dev, boundary_window=256)
    assert ms > 0 and d.tuning(boundary_window=256).states_per_thread == t.states_per_thread
    assert d.tuning().tiles_per_cta == 8
    assert d.match(dev, boundary_window=256) == want
    with pytest.raises(dm.DfaError) as e:
        d.match(dev, boundary_window=65537)
    assert e.value.status == dm.EINVAL


def test_served_with_placement_equal_oracle(dm):
    """The serving loop plans its batches with the placement window it was given."""
    import torch
    w = gen.regex_workload(8, 2 << 20)
    d = dm.Dfa.from_spec(w.spec)
    od = oracle.Dfa.from_spec(w.spec)
    lens = [0, 5, 700, 9000, 100_000, 1 << 20, 2 << 20]
    datas = [np.ascontiguousarray(w.data[:n]) for n in lens]
    want = [od.run(x) for x in datas]
    srv = dm.Server(1 << 28, max_inflight=4, boundary_window=256)
    tickets = {}
    for rep in range(3):
        for i, x in enumerate(datas):
            host = torch.from_numpy(x).pin_memory() if len(x) else x
            tickets[srv.submit(d, host)] = i
    srv.drain(120.0)
    done = srv.poll(1024)
    assert len(done) == len(tickets)
    for c in done:
        st, fs, acc = want[tickets[c[0]]]
        assert c[3] == st
        if st == 0:
            assert (c[1], c[2]) == (fs, acc)
    with pytest.raises(dm.DfaError) as e:
        srv.set_opts(boundary_window=70000)
    assert e.value.status == dm.EINVAL
    srv.close()


@pytest.mark.parametrize("window", [0, 256])
def test_grid_waves_equal_oracle(dm, window):
    """More CTAs than fit at once (tuning grid_waves 2 or 4: the same chunks cut
    into more, smaller CTA shares, scheduled as earlier CTAs finish) give the
    same answers and the same chunks."""
    w = gen.regex_workload(6, (16 << 20) + 999)
    d = dm.Dfa.from_spec(w.spec)
    dev = _dev(w.data)
    want = oracle.Dfa.from_spec(w.spec).run(w.data)
    n = dev.numel()
    base = None
    for waves in (1, 2, 4):
        d.set_tuning(states_per_thread=2, tiles_per_cta=4, ctas_per_sm=2, grid_waves=waves,
                     boundary_window=window)
        assert d.tuning(boundary_window=window).grid_waves == waves
        P = d.plan_chunks(n, boundary_window=window)
        base = P if base is None else base
        assert P == base                      # waves do not change the chunks
        for r in (1, 4):
            assert d.match(dev, lookahead=r, boundary_window=window) == want, (waves, r)
    with pytest.raises(dm.DfaError) as e:
        d.set_tuning(grid_waves=5, boundary_window=window)
    assert e.value.status == dm.EINVAL
