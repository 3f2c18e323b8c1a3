"""The multi-rank path of bench.py with the library doing the work (two ranks, one GPU).

Each rank is a process with its own CUDA context on cuda:0; its kernels never wait on the other
rank's (no collective on the data path), so sharing one GPU is safe.  Rank r solves members r,
r + 2, ... of one seeded ensemble, FP32, on the on-chip kernel at 8 nodes a thread (the same
arithmetic whatever the packing), and the per-member records (index, sum phi, max |phi|,
non-finite count) are gathered over gloo.  They must equal, bit for bit, the records of one
process solving the whole batch with the same kernel.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MEMBERS, STEPS = 24, 60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve(probs):
    from paper_0907_1720_gb300 import lbhpde as L

    b = L.Batch(probs, precision=L.FP32_DEV)
    b.set_kernel(L.KERNEL_ONCHIP, 8)
    b.set_phi(np.concatenate([p.phi0 for p in probs])).step(STEPS)
    diag = b.diagnostics()
    b.close()
    return [(int(p.meta["index"]), float(d["sum_phi"]), float(d["max_abs_phi"]), int(d["nonfinite"]))
            for p, d in zip(probs, diag)]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    probs = bench.ensemble_problems(rank, members=MEMBERS, world=world, nodes=0)
    recs = _solve(probs)
    out[rank] = (sorted(int(p.meta["index"]) for p in probs), bench.gather_member_records(recs, world, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_the_library_match_one_process():
    import sys

    import torch.multiprocessing as mp

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_0907_1720_gb300 import build as B

    B.build()
    import bench

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    idx0, g0 = out[0]
    idx1, g1 = out[1]
    assert set(idx0).isdisjoint(idx1) and sorted(idx0 + idx1) == list(range(MEMBERS))
    whole = sorted(_solve(bench.ensemble_problems(0, members=MEMBERS, world=1, nodes=0)))
    assert g0 == g1 == whole
