"""GB300-native lattice Boltzmann solver for high-order nonlinear PDEs (Shi, He, Guo).

The compute path is a CUDA shared library with a C ABI (``include/lbhpde.h``);
``paper_0907_1720_gb300.lbhpde`` is its thin Python binding.  Importing this
package does not load the library; ``workloads`` holds the seeded inputs.
"""
__all__ = ["lbhpde", "workloads"]
