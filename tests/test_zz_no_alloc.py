"""The allocation-free Mindlin entry point against the context-based one.

fvim_apply_mindlin_noalloc serves callers that cannot allocate device memory while
they run; its scratch is a static device array inside the library.  This file is
collected last so that a run stopping at the first failure has run everything else.
It must pass alone in a fresh process and after the other tests; one case starts a
fresh process whose very first GPU call is the allocation-free entry point.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}
HERE = os.path.dirname(os.path.abspath(__file__))


def _noalloc():
    from paper_1811_11558_gb300 import fvim

    f = fvim.lib().fvim_apply_mindlin_noalloc
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    f.restype = i
    f.argtypes = [i, i, i, ctypes.POINTER(d), d, d, d, d, i, vp, vp, i, vp, vp]
    return f


def _nonuniform(nz, depth):
    """Depth nodes [0, depth] refined towards the surface (z ~ s^1.5)."""
    s = np.linspace(0.0, 1.0, nz)
    return depth * s ** 1.5


# (precision, n1, n2, nodes, output kind): stress and strain outputs, uniform and refined
# depth nodes, a small grid and the FP32 128 x 128 x 32 grid close to the scratch limit
CASES = [
    ("fp32", 64, 32, ("uniform", 13), "stress"),
    ("fp64", 64, 32, ("uniform", 13), "stress"),
    ("fp32", 64, 32, ("refined", 13), "strain"),
    ("fp64", 32, 16, ("refined", 9), "strain"),
    ("fp32", 128, 128, ("uniform", 32), "stress"),
    ("fp32", 128, 128, ("refined", 32), "strain"),
]


def _nodes(spec):
    kind, nz = spec
    return inputs.uniform_depth(nz, 0.4) if kind == "uniform" else _nonuniform(nz, 0.4)


@pytest.mark.parametrize("prec,n1,n2,nodes,kind", CASES)
def test_noalloc_matches_context_entry_point_twice(prec, n1, n2, nodes, kind):
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context

    z = _nodes(nodes)
    ctx = Context(n1, n2, z, 1.0, 0.8, precision=prec, E=1.0, nu=0.3)
    dt = ctx.dtype
    f = _noalloc()
    zc = np.ascontiguousarray(z, dtype=np.float64)
    zp = zc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pcode = 0 if prec == "fp32" else 1
    kcode = 0 if kind == "stress" else 1
    for call, seed in enumerate((21, 22)):
        ep = to_dev(torch, inputs.plastic_strain_field(n1, n2, z, seed=seed), dt)
        ref_u3 = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
        ref = ctx.apply_mindlin(ep, kind=kind, u3=ref_u3)
        out = torch.full(ctx.vol_shape, float("nan"), dtype=dt, device="cuda")
        u3 = torch.full(ctx.surf_shape, float("nan"), dtype=dt, device="cuda")
        rc = f(n1, n2, z.size, zp, 1.0, 0.8, 1.0, 0.3, pcode, ctypes.c_void_p(ep.data_ptr()),
               ctypes.c_void_p(out.data_ptr()), kcode, ctypes.c_void_p(u3.data_ptr()), stream)
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


# run in a fresh interpreter: the first call into the library on the device is the
# allocation-free one (torch only provides the input and output buffers)
_FRESH = r"""
import ctypes, sys
import numpy as np
sys.path[:0] = [{root!r}, {tests!r}]
import torch
from paper_1811_11558_gb300 import fvim, inputs
lib = fvim.lib()
f = lib.fvim_apply_mindlin_noalloc
vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
f.restype = i
f.argtypes = [i, i, i, ctypes.POINTER(d), d, d, d, d, i, vp, vp, i, vp, vp]
n1, n2 = 64, 32
z = np.ascontiguousarray(inputs.uniform_depth(9, 0.3))
zp = z.ctypes.data_as(ctypes.POINTER(d))
ep = torch.from_numpy(inputs.plastic_strain_field(n1, n2, z, seed=5).astype(np.float32)).cuda()
out = torch.full_like(ep, float("nan"))
rc = f(n1, n2, z.size, zp, 1.0, 0.8, 1.0, 0.3, 0, vp(ep.data_ptr()), vp(out.data_ptr()), 0, None, None)
assert rc == 0, rc
torch.cuda.synchronize()
ctx = fvim.Context(n1, n2, z, 1.0, 0.8, precision="fp32", E=1.0, nu=0.3)
ref = ctx.apply_mindlin(ep, kind="stress")
torch.cuda.synchronize()
a, b = out.cpu().numpy(), ref.cpu().numpy()
err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
assert err < 2e-5, err
print("ok", err)
"""


def test_noalloc_as_first_gpu_call_of_a_fresh_process():
    """A process whose first library call on the device is the allocation-free one: the
    scratch array's address is looked up on that call, and the result equals the
    context-based apply created afterwards."""
    require_gpu()
    root = os.path.dirname(HERE)
    code = _FRESH.format(root=root, tests=HERE)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "ok" in r.stdout
