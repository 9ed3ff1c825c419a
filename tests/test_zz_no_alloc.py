"""The allocation-free Mindlin entry point against the context-based one.

fvim_apply_mindlin_noalloc serves callers that cannot allocate device memory while
they run; its scratch is a static device array inside the library.  This file is
collected last so that a run stopping at the first failure has run everything else.
It must pass alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}


def _noalloc():
    from paper_1811_11558_gb300 import fvim

    f = fvim.lib().fvim_apply_mindlin_noalloc
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f.restype = i
    f.argtypes = [i, i, i, ctypes.POINTER(d), d, d, d, d, i, vp, vp, i, vp, vp]
    return f


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_context_entry_point_twice(prec):
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context

    n1, n2 = 64, 32
    z = inputs.uniform_depth(13, 0.4)
    ctx = Context(n1, n2, z, 1.0, 0.8, precision=prec, E=1.0, nu=0.3)
    dt = ctx.dtype
    f = _noalloc()
    zc = np.ascontiguousarray(z, dtype=np.float64)
    zp = zc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pcode = 0 if prec == "fp32" else 1
    for call, seed in enumerate((21, 22)):
        ep = to_dev(torch, inputs.plastic_strain_field(n1, n2, z, seed=seed), dt)
        ref_u3 = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
        ref = ctx.apply_mindlin(ep, kind="stress", u3=ref_u3)
        out = torch.full(ctx.vol_shape, float("nan"), dtype=dt, device="cuda")
        u3 = torch.full(ctx.surf_shape, float("nan"), dtype=dt, device="cuda")
        rc = f(n1, n2, z.size, zp, 1.0, 0.8, 1.0, 0.3, pcode, ctypes.c_void_p(ep.data_ptr()),
               ctypes.c_void_p(out.data_ptr()), 0, ctypes.c_void_p(u3.data_ptr()), stream)
        assert rc == 0, call
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < TOL[prec], call
        assert rel_l2(u3.cpu().numpy(), ref_u3.cpu().numpy()) < TOL[prec], call


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = require_gpu()
    f = _noalloc()
    z = np.ascontiguousarray(inputs.uniform_depth(64, 0.4))
    zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # 512 x 512 x 64 needs ~400 MB of scratch: refused on the host before any device work
    a = torch.zeros((64, 6, 512, 512), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    rc = f(512, 512, 64, zp, 1.0, 1.0, 1.0, 0.3, 0, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
           0, None, None)
    assert rc == -7
