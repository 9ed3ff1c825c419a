"""GB300 (sm_103a) implementation of the Fourier-accelerated volume integral method
for elastoplastic contact (Frerot, Bonnet, Molinari & Anciaux, arXiv:1811.11558).

The compute path is libfvim.so (hand-written CUDA kernels behind the C ABI of
include/fvim.h); ``fvim`` is its Python binding and ``inputs`` the seeded
synthetic workloads.
"""
from . import inputs  # noqa: F401
from .fvim import Context, FvimError, lib  # noqa: F401
