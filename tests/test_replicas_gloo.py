"""Multi-rank path of bench.py (independent replicas) on CPU with the gloo backend.

Every rank factors its own matrix; the only collective is the reduction of the
timed region to the slowest rank, and the reported value is the work of all
ranks over that time.  Two ranks here, each with its own (deliberately unequal)
timing; the oracle stands in for the GPU factorization so the test needs no GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import workloads
    g = workloads.prescribed_rank_matrix(64, 48, 20, 65521, seed=10 + rank)
    res = oracle.pluq(g.A, 65521)  # each rank's own replica
    local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    F = bench.field_ops(64, 48, res.rank)
    out[rank] = (res.rank == g.rank and res.rpm == g.rpm, slowest,
                 bench.whole_job_gfops(world, F, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert all(res[r][0] for r in range(world))
    assert res[0][1] == res[1][1] == 20.0
    F = 2 * 64 * 48 * 20 - (64 + 48) * 20 ** 2 + 2 * 20 ** 3 / 3
    assert np.isclose(res[0][2], world * F / 0.020 / 1e9)


def _dead_replica_main(rank, world, port, out):
    import sys
    import time
    from datetime import timedelta
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    import bench
    if rank == 1:
        out[1] = "left"
        os._exit(3)  # this replica dies between steps, before the timing reduction
    t0 = time.time()
    try:
        bench.max_over_ranks(10.0, dist, "cpu")
        out[0] = ("no error", time.time() - t0)
    except Exception as e:  # the dead peer surfaces as an error on the host
        out[0] = (type(e).__name__, time.time() - t0)


def test_dead_replica_is_reported():
    """A replica that leaves between steps: the surviving rank's timing reduction
    ends with an error within the process-group timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_dead_replica_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        alive = [p.is_alive() for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        res = dict(out)
    assert not any(alive)
    assert procs[1].exitcode == 3 and res[1] == "left"
    assert res[0][0] != "no error" and res[0][1] < 60


def _shard_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    cfg = workloads.CONFIGS["batched-4096-lru-p65521"]
    tag, ms, ns, rs = bench.batch_shard(cfg, rank)
    # each rank factors a few of its own matrices (the oracle stands in for the GPU)
    import oracle
    ok = True
    for b in range(3):
        g = workloads.prescribed_rank_matrix(int(ms[b]), int(ns[b]), int(rs[b]), cfg.p, seed=1,
                                             tag=f"{tag}:{b}")
        res = oracle.pluq(g.A, cfg.p, want_lu=False)
        ok &= res.rank == g.rank and res.rpm == g.rpm
    shapes = [None] * world
    dist.all_gather_object(shapes, (tag, ms.tolist(), ns.tolist(), rs.tolist()))
    local_ms = 5.0 + rank
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (ok, shapes, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_batched_shards_gloo():
    """The batched workload sharded over two ranks: shard 0 is the single-GPU workload
    itself, shard 1 a distinct batch of the same distribution, each rank factors its
    own matrices with no collective on the data path, and the whole-job figure takes
    all ranks' matrices over the slowest rank's time."""
    import workloads
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] and res[1][0]
    shapes = res[0][1]
    cfg = workloads.CONFIGS["batched-4096-lru-p65521"]
    ms, ns, rs = workloads.batched_shapes(cfg.count, cfg.lo, cfg.hi, seed=1)
    assert shapes[0][1:] == (ms.tolist(), ns.tolist(), rs.tolist())  # shard 0 = the workload
    assert shapes[0][0] != shapes[1][0] and shapes[0][1:] != shapes[1][1:]
    for tag, m, n, r in shapes:
        assert len(m) == cfg.count
        assert all(cfg.lo <= x <= cfg.hi for x in m + n)
        assert all(1 <= rr <= min(a, b) for rr, a, b in zip(r, m, n))
    assert res[0][2] == res[1][2] == 6.0
