"""The multi-rank path of bench.py on the CPU (gloo, world size 2): each rank solves its own
ensemble (weak scaling) and the whole-job value is the sum of the ranks' node-updates over the
slowest rank's time.  Ranks run a small oracle sample of their own ensemble as the workload."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import time

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle

    probs = bench.ensemble_problems(rank, members=4)
    t0 = time.perf_counter()
    units = 0
    for p in probs:
        oracle.run_problem(p, nsteps=5)
        units += p.N * 5
    if rank == 1:
        time.sleep(0.2)  # the slow rank sets the job time
    t = time.perf_counter() - t0
    value, tmax = bench.aggregate(t, units, world)
    out[rank] = (value, tmax, t, units, [p.N for p in probs])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    v0, tmax0, t0, u0, n0 = out[0]
    v1, tmax1, t1, u1, n1 = out[1]
    assert tmax0 == tmax1 == max(t0, t1) and t1 >= 0.2
    assert v0 == v1 == pytest.approx((u0 + u1) / max(t0, t1))
    assert n0 != n1  # each rank draws its own members (seed + rank)
