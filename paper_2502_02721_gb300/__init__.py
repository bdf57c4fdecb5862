"""GB300 (sm_103a) library for the sketched inner-product-free Krylov method
sCMRH (arXiv 2502.02721): pivoted Hessenberg basis, sparse-sign sketch and
the sketched projected (Tikhonov) least-squares solve, behind the C ABI of
include/ipf.h.  This package holds the CUDA sources (csrc/), the nvcc build
(build.py) and a ctypes binding (binding.py)."""
from . import build  # noqa: F401
