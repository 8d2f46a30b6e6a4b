"""GB300 (sm_103a) coupled lattice-Boltzmann + WENO5 solver for settling-driven
gravitational instabilities (arXiv 2106.07694).

The compute path is the CUDA library liblbm_wenoc.so behind the C ABI in
include/lbm_wenoc.h; ``lbm_wenoc`` is its Python binding.
"""
from . import workloads  # noqa: F401  (no CUDA needed)

__all__ = ["workloads", "lbm_wenoc", "build"]
