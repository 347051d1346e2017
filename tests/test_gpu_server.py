"""The serving loop (dfa_server_*): continuous batching of requests that
arrive while earlier batches run.  Each result must equal the result of the
same test run alone (and the oracle's), bit-exactly; admission respects the
memory budget; batches overlap on the device."""
import time

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


def test_served_results_equal_alone(dm):
    specs = [gen.plain_dfa(1), gen.regex_dfa(2), gen.protein_dfa(3)] + gen.batch_dfas(5, 4)
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    n_req = 240
    lens = gen.batch_lengths(21, n_req, 1, 2 << 20)
    picks = gen.batch_picks(21, n_req, len(specs))
    datas = []
    for i in range(n_req):
        spec = specs[picks[i]]
        if spec.name == "plain16":
            x = gen.uniform_bytes(100 + i, int(lens[i]))
        else:
            x = gen.batch_text(100 + i, spec, int(lens[i]))
        datas.append(x)
    # one request carries a byte outside a protein DFA's alphabet
    bad = next(i for i in range(n_req) if specs[picks[i]].byte_to_symbol is not None and lens[i] > 10)
    datas[bad] = datas[bad].copy()
    datas[bad][5] = ord("Z") if ord("Z") not in gen.AMINO else ord("#")
    srv = dm.Server(64 << 20, max_inflight=4)
    tickets = {}
    done = {}
    for i in range(n_req):
        tickets[srv.submit(dfas[picks[i]], datas[i])] = i
        if i % 16 == 15:
            time.sleep(0.002)           # requests keep arriving while batches run
            for c in srv.poll():
                done[c[0]] = c
    srv.drain(120.0)
    for c in srv.poll(4096):
        done[c[0]] = c
    assert len(done) == n_req
    st = srv.stats()
    assert st.completed == n_req and st.submitted == n_req
    assert st.launches >= 2
    assert st.max_bytes_in_flight <= 64 << 20
    for t, (ticket, fs, acc, status, t_sub, t_done) in done.items():
        i = tickets[ticket]
        assert t_done >= t_sub
        est, efs, eacc = oracle.Dfa.from_spec(specs[picks[i]]).run(datas[i])
        if i == bad:
            assert status == dm.ESYMBOL and est == oracle.ESYMBOL
            continue
        assert (status, fs, acc) == (0, efs, eacc), i
        alone = dfas[picks[i]].match(datas[i])
        assert alone == (0, fs, acc)
    with pytest.raises(dm.DfaError) as e:
        srv.submit(dfas[0], np.zeros((64 << 20) + 1, dtype=np.uint8))
    assert e.value.status == dm.EBUDGET
    srv.close()


def test_batches_overlap_under_continuous_arrivals(dm):
    spec = gen.regex_dfa(2)
    d = dm.Dfa.from_spec(spec)
    # each request takes a few ms on the device; they arrive 0.5 ms apart, so
    # later batches are launched while earlier ones still run
    x = gen.zipf_text(7, 256 << 20)
    srv = dm.Server(3 << 30, max_inflight=3)
    for k in range(6):
        srv.submit(d, x)
        time.sleep(0.0005)
    srv.drain(120.0)
    res = srv.poll(64)
    assert len(res) == 6
    st = srv.stats()
    assert st.max_concurrent >= 2
    _, efs, eacc = oracle.Dfa.from_spec(spec).run(x)
    assert all((r[1], r[2], r[3]) == (efs, eacc, 0) for r in res)
    srv.close()


def test_error_paths_reported_without_a_fault(dm):
    """Failures made on the host, none on the GPU: a server budget larger than the
    device (DFA_ENOMEM from its allocation), a drain that runs out of time while
    work is still on the device (DFA_ETIMEOUT, after which the work completes and
    is right), a workspace smaller than the size query (DFA_ENOSPACE) and
    misaligned device pointers (DFA_EINVAL)."""
    import torch
    with pytest.raises(dm.DfaError) as e:
        dm.Server(1 << 50)
    assert e.value.status == dm.ENOMEM
    spec = gen.regex_dfa(2)
    d = dm.Dfa.from_spec(spec)
    x = gen.zipf_text(17, 256 << 20)
    srv = dm.Server(2 << 30, max_inflight=2)
    t = srv.submit(d, x)
    with pytest.raises(dm.DfaError) as e:
        srv.drain(1e-6)
    assert e.value.status == dm.ETIMEOUT
    srv.drain(120.0)
    done = srv.poll(8)
    srv.close()
    assert len(done) == 1 and done[0][0] == t
    assert (done[0][3], done[0][1], done[0][2]) == oracle.Dfa.from_spec(spec).run(x)
    dev = torch.from_numpy(x[: 1 << 20]).cuda()
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    need = d.workspace_size(dev.numel())
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DfaError) as e:
        d.match_async(dev, out, ws[: need - 256])
    assert e.value.status == dm.ENOSPACE
    with pytest.raises(dm.DfaError) as e:
        d.match_async(dev, out[1:], ws)           # result not 4-byte aligned
    assert e.value.status == dm.EINVAL
    big = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DfaError) as e:
        d.match_async(dev, out, big[16:])         # workspace not 256-byte aligned
    assert e.value.status == dm.EINVAL
