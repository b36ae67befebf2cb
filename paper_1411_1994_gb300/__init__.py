"""GB300 (sm_103a) lattice summation of Newton potentials with defects in
canonical / Tucker tensor form (Khoromskaia & Khoromskij, arXiv 1411.1994).

The compute path is the CUDA library behind the C ABI in
include/lattice_sum.h; ``lattice_sum`` is its ctypes binding (loaded on first
use) and ``workloads`` describes the seeded synthetic inputs.
"""
__all__ = ["lattice_sum", "workloads", "build"]
