"""Host logic of bench.py's multi-rank path on CPU (gloo, world size 2): every rank
holds a replica and draws its own samples; the job time is the slowest rank's and
the rate counts all ranks' samples.  No GPU, no collective on the data path."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = 1.0 + 0.5 * rank                     # rank 1 is the slower one
    slowest = bench.max_over_ranks(seconds, world, device="cpu")
    rate = bench.job_rate(world, 128, 3, slowest)
    q.put((rank, bench.rank_seed(rank), slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank_and_count_every_sample():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0), (r1, s1, t1, v1) = out
    assert s0 != s1                                   # independent sample streams
    assert t0 == t1 == 1.5                            # both ranks see the max
    assert v0 == v1 == pytest.approx(2 * 128 * 3 / 1.5)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(1, 128, 3, 2.0) == pytest.approx(192.0)
    assert len({bench.rank_seed(r) for r in range(8)}) == 8
