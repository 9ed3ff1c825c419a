"""The grouped Mindlin apply (fvim_apply_mindlin_group): problems of uneven grid size in one
launch per pass give each problem's own apply, bit for bit under the same depth plan, and
the FP64 oracle's operator within the FP32 bar."""
import numpy as np
import pytest

from oracle import operators as op
from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3


def _refined(nz, depth):
    s = np.linspace(0.0, 1.0, nz)
    return depth * s ** 1.5


# (n1, n2, z, L1, L2): every side length the group takes, depth chunk counts 1, 2, 4, 9
# (padded to 16), 16; uniform and refined nodes; non-square cells
GROUP = [
    (64, 64, inputs.uniform_depth(16, 0.4), 1.0, 1.0),
    (128, 64, inputs.uniform_depth(33, 0.4), 1.0, 0.5),
    (64, 128, _refined(13, 0.3), 0.8, 1.0),
    (256, 256, inputs.uniform_depth(8, 0.05), 1.0, 1.0),
    (512, 512, inputs.uniform_depth(5, 0.02), 1.0, 1.0),
    (128, 256, inputs.uniform_depth(64, 0.4), 1.0, 1.0),
    (256, 64, inputs.uniform_depth(4, 0.1), 1.0, 0.7),
    (512, 128, _refined(21, 0.2), 1.0, 0.5),
]
ORACLE = (0, 1, 2)   # members small enough for the oracle


def _group(torch, cutoff):
    from paper_1811_11558_gb300 import Context

    ctxs, eps = [], []
    for i, (n1, n2, z, L1, L2) in enumerate(GROUP):
        c = Context(n1, n2, z, L1, L2, precision="fp32", E=E, nu=NU)
        c.set_plan(depth_chunk=4, fft_path="rows_cols", depth_ctas=2, depth_cutoff=cutoff)
        ctxs.append(c)
        eps.append(to_dev(torch, inputs.plastic_strain_field(n1, n2, z, seed=4100 + i), torch.float32))
    return ctxs, eps


@pytest.mark.parametrize("kind", ["stress", "strain"])
def test_group_equals_each_problem_apply_bitwise(kind):
    """With the exact chunk scan (cutoff 0) the grouped kernels run each problem's arithmetic
    of its own launch sequence (same bodies, same chunk length): equal bit for bit."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import fvim

    ctxs, eps = _group(torch, 0.0)
    outs = fvim.apply_mindlin_group(ctxs, eps, kind=kind)
    for c, e, o in zip(ctxs, eps, outs):
        ref = c.apply_mindlin(e, kind=kind)
        torch.cuda.synchronize()
        assert torch.equal(o, ref), (c.n1, c.n2, c.nz)
        assert bool(torch.isfinite(o).all())


def test_group_matches_the_oracle():
    """Members of the group against the FP64 oracle at the FP32 bar (2e-5), with the default
    cutoff of the chunk scan decided over the tiles a CTA holds."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import fvim

    ctxs, eps = _group(torch, 18.0)
    for kind in ("stress", "strain"):
        outs = fvim.apply_mindlin_group(ctxs, eps, kind=kind)
        torch.cuda.synchronize()
        errs = []
        for i in ORACLE:
            n1, n2, z, L1, L2 = GROUP[i]
            ref = op.mindlin_apply(eps[i].double().cpu().numpy(), z, L1, L2, E, NU, kind)
            errs.append(rel_l2(outs[i].double().cpu().numpy(), ref))
        print(kind, "group vs oracle", ["%.2e" % x for x in errs])
        assert max(errs) < 2e-5


def test_group_cutoff_against_exact_scan():
    """The cutoff voted over a CTA's tiles changes results only at FP32 rounding."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import fvim

    ctxs, eps = _group(torch, 0.0)
    exact = [o.clone() for o in fvim.apply_mindlin_group(ctxs, eps)]
    for c in ctxs:
        c.set_plan(depth_chunk=4, fft_path="rows_cols", depth_ctas=2, depth_cutoff=18.0)
    cut = fvim.apply_mindlin_group(ctxs, eps)
    torch.cuda.synchronize()
    errs = [rel_l2(a.double().cpu().numpy(), b.double().cpu().numpy()) for a, b in zip(cut, exact)]
    print("cutoff vs exact", ["%.1e" % x for x in errs])
    assert max(errs) < 2e-6


def test_group_in_a_cuda_graph():
    """The problem table travels as a kernel parameter: the call captures into a CUDA graph,
    and a replay on new inputs equals a direct call."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import fvim

    ctxs, eps = _group(torch, 18.0)
    outs = [torch.empty_like(e) for e in eps]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fvim.apply_mindlin_group(ctxs, eps, outs)   # first call outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fvim.apply_mindlin_group(ctxs, eps, outs)
    for i, (n1, n2, z, _, _) in enumerate(GROUP):
        eps[i].copy_(to_dev(torch, inputs.plastic_strain_field(n1, n2, z, seed=4200 + i), torch.float32))
    g.replay()
    torch.cuda.synchronize()
    direct = fvim.apply_mindlin_group(ctxs, eps)
    torch.cuda.synchronize()
    for a, b in zip(outs, direct):
        assert torch.equal(a, b)


def test_group_rejects_what_it_does_not_take():
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context, FvimError, fvim

    z8 = inputs.uniform_depth(8, 0.1)
    ok = Context(64, 64, z8, precision="fp32")
    e = torch.zeros(ok.vol_shape, device="cuda")
    bad = [
        (Context(64, 64, z8, precision="fp64"), -7),                     # FP64
        (Context(32, 64, z8, precision="fp32"), -7),                     # side below 64
        (Context(1024, 64, inputs.uniform_depth(4, 0.1), precision="fp32"), -7),   # side above 512
        (Context(64, 64, inputs.uniform_depth(65, 0.4), precision="fp32"), -7),    # Nz above 64
        (Context(81, 81, inputs.uniform_depth(4, 0.1), precision="fp32"), -7),     # odd sides
    ]
    for c, status in bad:
        x = torch.zeros(c.vol_shape, dtype=c.dtype, device="cuda")
        with pytest.raises(FvimError) as ei:
            fvim.apply_mindlin_group([ok, c], [e, x])
        assert ei.value.status == status
    with pytest.raises(FvimError) as ei:                                 # the same context twice
        fvim.apply_mindlin_group([ok, ok], [e, e.clone()])
    assert ei.value.status == -1
