"""GB300 (sm_103a) implementation of the coupled level-set lattice Boltzmann
method on block-structured adaptive Cartesian grids (arXiv 2601.05936).

The method runs in the CUDA library built from ``csrc/`` (C ABI in
``include/lsb.h``); ``lsb`` is its ctypes binding and ``workloads`` the seeded
input generators.  ``build.build()`` compiles the library in-tree.
"""
__all__ = ["lsb", "workloads", "build"]
