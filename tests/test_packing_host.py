"""The on-chip planning of the library (no GPU): resident size classes with gap filling,
resident CTA packing and window cutting, checked on random member sets by a small C++ program
(tests/pack_check.cu) that calls the library's exported host functions.

Invariants: every member placed exactly once; warp-aligned, non-overlapping thread runs within
the CTA size; at most 32 instances per CTA; 16-byte aligned coefficient offsets; only gap fillers
move up a size class; the valid nodes of a member's windows cover each of its nodes exactly
once; window depths leave the stated share of a window valid; for bounded resident instances,
the position shift puts each end's outer nodes and extrapolation node in one warp inside the CTA
(every depth 1-4 and grid size up to the CTA's 2048 nodes); for bounded members on the 16-node
kernel, contiguous thread runs, at most 32 instances and enough threads for the helper roles in
every CTA, aligned coefficient blocks, shared memory within 227 KB, and the depth-2 variant chosen
exactly when every member allows it.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_onchip_planning_invariants(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    from paper_0907_1720_gb300 import build as B
    lib = B.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "pack_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0907_1720_gb300", "csrc"),
           os.path.join(ROOT, "tests", "pack_check.cu"), "-o", exe, "-L", libdir, "-llbhpde", "-lcudart",
           "-Xlinker", "-rpath=" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout[-2000:]
