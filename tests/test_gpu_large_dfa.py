"""GPU parity for DFAs with more than 4095 states (up to the ABI's limit of
65534, with q_e the 65535th state and 0xFFFF reserved), bit-exact against the
oracle (Algorithm 1) and, on small inputs, against the oracle's Algorithm 3
chunk maps entry by entry.

Large sets change the launch in three ways, each covered here:
  * a set with more chains than one CTA's threads hold at K = 16 (more than
    8192 states) runs its chains in several passes over its chunk (|Q| = 20000
    under Algorithm 3, every large DFA under Algorithm 2);
  * the running state maps of launches whose sets exceed 4096 states live in
    global memory (every DFA here under Algorithm 2, |Q| = 20000 and 65534
    under Algorithm 3);
  * above 32767 states the table holds 32-bit entries, and the segment maps of
    a test spread over several CTAs are too large to stage, so the Eq. (8)
    combine reads them in place (|Q| = 65534).
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


def _expect(spec, data):
    return oracle.Dfa.from_spec(spec).run(data)


def _check(dm, d, spec, data, **kw):
    st, fs, acc = d.match(data, **kw)
    est, efs, eacc = _expect(spec, data)
    assert st == est, (st, est, kw)
    if st == 0:
        assert (fs, acc) == (efs, eacc), kw


def _large(Q, seed):
    """Protein-lettered, shaped like the paper's PROSITE DFAs: per-class sets of
    0.2-0.9 |Q| (so I_max = 0.9 |Q|)."""
    return gen.class_dfa(seed, Q, 20, 0.2, 0.9, max(1, Q // 100), "protein")


@pytest.mark.parametrize("Q", [5000, 20000])
def test_large_dfa_algorithms_2_and_3(dm, Q):
    spec = _large(Q, 1000 + Q)
    d = dm.Dfa.from_spec(spec)
    info = d.info()
    assert info.num_states == Q and info.i_max == int(np.ceil(0.9 * Q - 1e-9))
    assert info.state_bytes == 2 and info.placement == 1
    data = gen.protein_text(7 + Q, (1 << 20) + 37)
    for P in (0, 1, 7, 300):
        _check(dm, d, spec, data, num_chunks=P)               # Algorithm 3 (r = 1)
    for P in (0, 5, 130):
        _check(dm, d, spec, data[: 200_003], num_chunks=P, lookahead=0)   # Algorithm 2
    _check(dm, d, spec, data[:1])
    _check(dm, d, spec, data[:0])
    with pytest.raises(dm.DfaError) as e:                      # Eq. 13 sets stop at 4095 states
        d.match(data[:1000], lookahead=2)
    assert e.value.status == dm.EINVAL


@pytest.mark.parametrize("Q", [5000, 20000])
def test_large_dfa_chunk_maps_equal_algorithm3(dm, Q):
    import torch
    spec = _large(Q, 2000 + Q)
    d = dm.Dfa.from_spec(spec)
    data = gen.protein_text(11 + Q, 50_000)
    dev = torch.from_numpy(data).cuda()
    od = oracle.Dfa.from_spec(spec)
    for P in (3, 40):
        got, fs = d.chunk_maps(dev, num_chunks=P)
        st, efs, eacc, want = od.chunked(data, oracle.chunk_starts(len(data), P, 1), want_maps=True)
        assert st == 0 and fs == efs
        assert np.array_equal(got.astype(np.uint32), want), (Q, P)


def test_largest_dfa_65534_states(dm):
    """The ABI's limit: 65534 user states plus q_e; 32-bit table entries; a
    random delta with missing entries (so q_e is reachable and excluded)."""
    import torch
    Q = 65534
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[ord("a"):ord("a") + 4] = np.arange(4)
    spec = gen.random_dfa(4242, Q, 4, num_finals=300, missing=0.02, byte_to_symbol=m)
    d = dm.Dfa.from_spec(spec)
    info = d.info()
    assert info.num_states_ext == 65535 and info.state_bytes == 4 and info.placement == 1
    data = (gen.uniform_bytes(43, 40_000) % 4 + ord("a")).astype(np.uint8)
    for P in (0, 1, 2, 60):
        _check(dm, d, spec, data, num_chunks=P)
    _check(dm, d, spec, data[: 3000], num_chunks=9, lookahead=0)   # Algorithm 2: 8 passes
    dev = torch.from_numpy(data[: 6000]).cuda()
    got, fs = d.chunk_maps(dev, num_chunks=4)
    st, efs, eacc, want = oracle.Dfa.from_spec(spec).chunked(
        data[: 6000], oracle.chunk_starts(6000, 4, 1), want_maps=True)
    assert st == 0 and fs == efs and np.array_equal(got.astype(np.uint32), want)
    # a byte outside Sigma is still reported
    bad = data.copy()
    bad[20_000] = ord("z")
    _check(dm, d, spec, bad)


def test_large_dfa_in_a_batch_and_async(dm):
    """A 20000-state DFA batched with the regex-shaped DFA (the launch keeps
    its running maps in global memory for every test), and the asynchronous
    entry point with a caller workspace; answers against the oracle."""
    import torch
    big = _large(20000, 77)
    small = gen.regex_dfa(2)
    db, ds = dm.Dfa.from_spec(big), dm.Dfa.from_spec(small)
    xs = [gen.protein_text(80 + i, 30_000 * (i + 1) + i) if i % 2 == 0 else
          gen.zipf_text(80 + i, 100_000 * (i + 1)) for i in range(6)]
    dev = [torch.from_numpy(x).cuda() for x in xs]
    res = dm.match_batch([db, ds, db, ds, db, ds], dev)
    for i, (fs, acc, st) in enumerate(res):
        assert (st, fs, acc) == _expect(big if i % 2 == 0 else small, xs[i]), i
    ws = torch.empty(db.workspace_size(dev[4].numel()), dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    db.match_async(dev[4], out, ws)
    torch.cuda.synchronize()
    (fs, acc, st), = dm.results_from(out)
    assert (st, fs, acc) == _expect(big, xs[4])


def test_multipass_after_other_kernels(dm):
    """Multi-pass composition marks finished map entries in shared memory;
    those marks must start cleared in every launch whatever earlier kernels
    left in shared memory.  Launches with large shared-memory use (the
    regex-shaped DFA's table and stage buffers) alternate with multi-pass
    launches of a 20000-state DFA whose CTAs hold several chunks each."""
    import torch
    big = gen.class_dfa(1020, 20000, 20, 0.2, 0.9, 200, "protein")
    data = gen.protein_text(9, 300_000)
    want = _expect(big, data)
    db = dm.Dfa.from_spec(big)
    w = gen.regex_workload(2, 32 << 20)
    dr = dm.Dfa.from_spec(w.spec)
    dev_r = torch.from_numpy(w.data).cuda()
    want_r = _expect(w.spec, w.data)
    for i in range(4):
        assert dr.match(dev_r) == want_r
        assert db.match(data) == want, i
        assert db.match(data, num_chunks=585 + 7 * i) == want, i


def test_large_dfa_placement_server_and_noalloc(dm):
    """A 20000-state DFA with Sec. 4.2 placement (the window search reads 16-bit
    set sizes), through the serving loop next to a small DFA, and through the
    allocation-free entry point, whose fixed scratch cannot hold the running maps
    of such sets (DFA_ENOSPACE, nothing launched)."""
    import torch
    big = _large(20000, 91)
    db = dm.Dfa.from_spec(big)
    data = gen.protein_text(92, 400_000)
    for w in (16, 256):
        _check(dm, db, big, data, boundary_window=w)
    small = gen.regex_dfa(2)
    ds = dm.Dfa.from_spec(small)
    xs = [gen.protein_text(93 + i, 20_000 * (i + 1)) if i % 2 == 0 else gen.zipf_text(93 + i, 50_000)
          for i in range(6)]
    srv = dm.Server(1 << 30, max_inflight=3)
    tickets = {srv.submit(db if i % 2 == 0 else ds, x): i for i, x in enumerate(xs)}
    srv.drain(120.0)
    done = srv.poll(64)
    srv.close()
    assert len(done) == len(xs)
    for c in done:
        i = tickets[c[0]]
        st, fs, acc = _expect(big if i % 2 == 0 else small, xs[i])
        assert (c[3], c[1], c[2]) == (st, fs, acc), i
    dev = torch.from_numpy(data).cuda()
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DfaError) as e:
        db.match_noalloc(dev, out)
    assert e.value.status == dm.ENOSPACE
