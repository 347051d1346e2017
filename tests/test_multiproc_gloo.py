"""The N > 1 host logic of bench.py on CPU with gloo, world size 2: every
rank gets its own seed (tests shard by rank, no data-path collective), and
the job's value is all ranks' bytes over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(2, rank)
    elapsed = [100.0, 250.0][rank]          # the second rank is the slow one
    gbs, ms_max = bench.reduce_job(dist, "cpu", 1 << 30, 10, elapsed, world)
    q.put((rank, seed, gbs, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [2, 3]                 # distinct tests per rank
    for _, _, gbs, ms_max in res:
        assert ms_max == 250.0                           # max over ranks
        assert gbs == pytest.approx((1 << 30) * 2 * 10 / 0.25 / 1e9)
