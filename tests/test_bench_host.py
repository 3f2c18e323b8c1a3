"""Host-side pieces of bench.py (no GPU): the algorithmic work per node-update that the roofline
objects divide by, and the workload description both arms print."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flops_per_node_update():
    """Per moving population: Horner of degree D and the relaxation (D + 1 multiply-adds), then the
    flux-difference update (2 flops): 56 for D1Q5 degree 5, 108 for D1Q7 degree 7."""
    assert bench.flops_per_node_update(5, 5) == 56
    assert bench.flops_per_node_update(7, 7) == 108
    # real exponents, 5 rows of degree 1 (the gKdV grid): (A + 1) Dg + A + 1 multiply-adds
    assert bench.flops_per_node_update_nu(5, 4, 1) == 4 * (2 * (5 + 4 + 1) + 2) == 88
    # a single row of degree D is the polynomial case
    for D in range(0, 8):
        assert bench.flops_per_node_update_nu(5, 0, D) == bench.flops_per_node_update(5, D)


def test_bytes_per_node_update():
    assert bench.bytes_per_node_update(5, 4) == 40
    assert bench.bytes_per_node_update(7, 8) == 112


@pytest.mark.parametrize("workload", ["ensemble", "bounded", "nu_grid", "long_grid"])
def test_workload_description_is_shared(workload):
    """Both arms name the workload through workload_problems, from seeded inputs: the same
    arguments give the same description and the same problem sizes."""
    args = argparse.Namespace(workload=workload, members=64, sweep_members=32, nodes=1 << 12, kernel="auto")
    p1, n1, d1 = bench.workload_problems(args)
    p2, n2, d2 = bench.workload_problems(args)
    assert d1 == d2 and n1 == n2 and [p.N for p in p1] == [p.N for p in p2]
    assert n1 > 0 and sum(p.N for p in p1) > 0
