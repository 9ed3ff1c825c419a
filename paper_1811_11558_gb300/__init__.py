"""GB300 (sm_103a) implementation of the Fourier-accelerated volume integral method
for elastoplastic contact (Frerot, Bonnet, Molinari & Anciaux, arXiv:1811.11558).

The compute path is libfvim.so (hand-written CUDA kernels behind the C ABI of
include/fvim.h); ``fvim`` is its Python binding and ``inputs`` the seeded
synthetic workloads.  The binding is imported on first use of ``Context``,
``FvimError`` or ``lib``, so that importing ``inputs`` alone (the input
generators that the oracle's scripts share) loads nothing of the CUDA path.
"""
_BINDING = ("Context", "FvimError", "lib")


def __getattr__(name):
    if name in _BINDING:
        from . import fvim

        return getattr(fvim, name)
    raise AttributeError("module %r has no attribute %r" % (__name__, name))


def __dir__():
    return sorted(list(globals()) + list(_BINDING))
