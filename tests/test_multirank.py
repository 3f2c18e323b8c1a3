"""The multi-rank path of bench.py on the CPU (gloo, world size 2).

The ensemble is one seeded batch; rank r takes members r, r + world, ... (no collective while
stepping), and the per-member results (index, sum phi, max |phi|, non-finite count) are gathered
to every rank once at the end.  The whole-job value is the sum of the ranks' node-updates over
the slowest rank's time.  On the CPU the oracle stands in for the library as each rank's solver.

Checked: the ranks' members are disjoint and their union is the single-rank batch; the gathered
records equal, bit for bit, those of one process solving the whole batch; the aggregate takes
the maximum time and the summed work."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

MEMBERS, STEPS = 8, 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _records(probs, steps):
    import oracle

    out = []
    for p in probs:
        phi = oracle.run_problem(p, nsteps=steps)
        out.append((int(p.meta["index"]), float(phi.sum()), float(np.abs(phi).max()), int((~np.isfinite(phi)).sum())))
    return out


def _worker(rank, world, port, out):
    import sys
    import time

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    probs = bench.ensemble_problems(rank, members=MEMBERS, world=world)
    t0 = time.perf_counter()
    recs = _records(probs, STEPS)
    units = sum(p.N for p in probs) * STEPS
    if rank == 1:
        time.sleep(0.2)  # the slow rank sets the job time
    t = time.perf_counter() - t0
    value, tmax = bench.aggregate(t, units, world)
    gathered = bench.gather_member_records(recs, world, device="cpu")
    out[rank] = (value, tmax, t, units, [int(p.meta["index"]) for p in probs], gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_gather_and_aggregate():
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    v0, tmax0, t0, u0, idx0, g0 = out[0]
    v1, tmax1, t1, u1, idx1, g1 = out[1]
    # a partition of the one batch
    assert set(idx0).isdisjoint(idx1) and sorted(idx0 + idx1) == list(range(MEMBERS))
    # the gathered per-member results equal one process solving the whole batch
    whole = sorted(_records(bench.ensemble_problems(0, members=MEMBERS, world=1), STEPS))
    assert g0 == g1 == whole
    # whole-job throughput: summed work over the slowest rank's time
    assert tmax0 == tmax1 == max(t0, t1) and t1 >= 0.2
    assert v0 == v1 == pytest.approx((u0 + u1) / max(t0, t1))
