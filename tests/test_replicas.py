"""Host logic of bench.py's multi-rank path on CPU (gloo, world size 2): every rank
holds a replica of the state and draws a disjoint, contiguous range of one sample
stream (one seed, Philox counters keyed by the global sample index); the job time is
the slowest rank's and the rate counts all ranks' samples.  No GPU, no collective on
the data path."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiny_state():
    import workloads as w
    from oracle.tns import GridTNS
    lat = w.square(2, 3)
    t = GridTNS(lat.grid_rc, lat.edges, w.domain_wall_bits(lat))
    for g in w.heisenberg_circuit(lat, 2, 0.2):
        t.apply_group(g, 4)
        t.bp(200, 1e-12)
    return t


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import bmps
    seconds = 1.0 + 0.5 * rank                     # rank 1 is the slower one
    slowest = bench.max_over_ranks(seconds, world, device="cpu")
    rate = bench.job_rate(world, 128, 3, slowest)
    # each rank draws its shard of two steps with the oracle sampler (the library's
    # tns_sample_range follows the same indexing); rank 0 gathers the bits
    t, B = _tiny_state(), 3
    mine = [bmps.sample(t, 8, B, bench.SAMPLING_SEED, sample_offset=bench.shard_first(rank, world, k, B))[0]
            for k in range(2)]
    bits = torch.tensor(np.concatenate(mine), dtype=torch.uint8)
    got = [torch.zeros_like(bits) for _ in range(world)] if rank == 0 else None
    dist.gather(bits, got, dst=0)
    q.put((rank, slowest, rate, [g.numpy() for g in got] if got else None))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_shard_one_stream_and_take_the_slowest_rank():
    from oracle import bmps
    import bench
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, got), (r1, t1, v1, _) = out
    assert t0 == t1 == 1.5                            # both ranks see the max
    assert v0 == v1 == pytest.approx(2 * 128 * 3 / 1.5)
    # the two ranks' samples, step by step, are the single stream's first 2 * 2 * 3 draws
    B = 3
    ref = bmps.sample(_tiny_state(), 8, 2 * 2 * B, bench.SAMPLING_SEED)[0]
    for k in range(2):
        for r in range(2):
            f = bench.shard_first(r, 2, k, B)
            assert np.array_equal(got[r][k * B:(k + 1) * B], ref[f:f + B])


def test_shards_are_disjoint_and_cover_the_stream():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(1, 128, 3, 2.0) == pytest.approx(192.0)
    for world in (1, 2, 8):
        idx = sorted(i for k in range(3) for r in range(world)
                     for i in range(bench.shard_first(r, world, k, 5), bench.shard_first(r, world, k, 5) + 5))
        assert idx == list(range(3 * world * 5))
