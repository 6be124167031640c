"""GB300-native TENO-M (arXiv 2010.13289): FP64 characteristic TENO-M reconstruction
inside SSP-RK3 for the 1D/2D/3D Euler equations, as hand-written sm_103a CUDA behind
a C ABI (include/tenom.h).  The binding (``tenom``) loads libtenom.so lazily and
raises if it is missing: there is no CPU fallback."""
__all__ = ["problems", "tenom"]
