"""dfa_match_noalloc: the entry point for callers that cannot allocate device
memory (no cudaMalloc and no workspace of their own to pass).  It runs the same
kernels with their scratch in a fixed device array inside the library, so its
answers must equal dfa_match_async's and the oracle's (Algorithm 1), call after
call, even though every call reuses (and leaves behind) the previous call's
scratch contents.

This file is collected last so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process."""
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


def _via_async(dm, d, dev, **kw):
    import torch
    ws = torch.empty(d.workspace_size(dev.numel(), **kw), dtype=torch.uint8, device="cuda")
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    d.match_async(dev, out, ws, **kw)
    torch.cuda.synchronize()
    return dm.results_from(out)[0]


def _via_noalloc(dm, d, dev, **kw):
    import torch
    out = torch.full((12,), 0xAB, dtype=torch.uint8, device="cuda")
    d.match_noalloc(dev, out, **kw)
    torch.cuda.synchronize()
    return dm.results_from(out)[0]


def test_noalloc_matches_async_on_consecutive_calls(dm):
    import torch
    assert dm.noalloc_scratch_bytes() == 16 << 20
    regex = gen.regex_workload(2, 8 << 20)
    plain = gen.plain_workload(1)
    d_regex = dm.Dfa.from_spec(regex.spec)
    d_plain = dm.Dfa.from_spec(plain.spec)
    dev_regex = torch.from_numpy(regex.data).cuda()
    dev_plain = torch.from_numpy(plain.data).cuda()
    calls = [(d_regex, dev_regex, {}),
             (d_plain, dev_plain, {"num_chunks": plain.num_chunks}),
             (d_regex, dev_regex[: (5 << 20) + 3], {"num_chunks": 4097})]
    specs = {id(d_regex): regex.spec, id(d_plain): plain.spec}
    for d, dev, kw in calls:
        want = _via_async(dm, d, dev, **kw)
        got = _via_noalloc(dm, d, dev, **kw)
        assert got == want, (got, want, kw)          # bit-exact: final state, accept, status
        assert got[2] == dm.OK
        st, fs, acc = oracle.Dfa.from_spec(specs[id(d)]).run(dev.cpu().numpy())
        assert (got[2], got[0], got[1]) == (st, fs, acc), (got, kw)


def test_noalloc_rejects_plans_beyond_the_array(dm):
    import torch
    w = gen.regex_workload(2, 1 << 20)
    d = dm.Dfa.from_spec(w.spec)
    dev = torch.from_numpy(w.data).cuda()
    out = torch.zeros(12, dtype=torch.uint8, device="cuda")
    assert d.workspace_size(dev.numel(), num_chunks=1_000_000) > dm.noalloc_scratch_bytes()
    with pytest.raises(dm.DfaError) as e:
        d.match_noalloc(dev, out, num_chunks=1_000_000)
    assert e.value.status == dm.ENOSPACE
