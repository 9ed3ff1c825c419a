"""Tile plans of the depth kernel: every chunk length gives the oracle's operator, and the
autotuner keeps its choice per grid.

The chunk length only changes how the exact depth recursions of a mode are cut between
threads (and so the rounding order of the chunk scan), so every launchable plan must meet
the parity bar of the operators: 1e-10 in FP64, 2e-5 in FP32 (relative L2).  The grids here
are used by no other test: the tuned-plan table is process-wide.
"""
import numpy as np
import pytest

from oracle import operators as op
from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3
TOL = {"fp64": 1e-10, "fp32": 2e-5}
CHUNKS = [2, 3, 4, 5, 6, 8, 12, 16]


@pytest.mark.parametrize("n1,n2,z,prec", [
    (16, 32, inputs.uniform_depth(10, 0.3), "fp64"),
    (16, 16, np.array([0.0, 0.02, 0.05, 0.09, 0.14, 0.2, 0.27, 0.35, 0.44, 0.54, 0.65]), "fp64"),
    (64, 32, inputs.uniform_depth(23, 0.4), "fp32"),   # ragged last chunk for most lengths
    (32, 64, np.concatenate([[0.0], np.cumsum(np.linspace(0.01, 0.03, 18))]), "fp32"),
])
def test_every_chunk_length_matches_oracle(n1, n2, z, prec):
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context, FvimError

    ep = inputs.plastic_strain_field(n1, n2, z, seed=1830 + n1 + z.size)
    ref, u3_ref = op.mindlin_apply(ep, z, 1.0, 1.0, E, NU, "stress", with_surface=True)
    ctx = Context(n1, n2, z, 1.0, 1.0, precision=prec, E=E, nu=NU)
    d_ep = to_dev(torch, ep, ctx.dtype)
    u3 = torch.empty(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
    ran = []
    for C in CHUNKS + [0]:
        try:
            ctx.set_plan(C)
        except FvimError as e:
            assert e.status == -1 and C > 0
            continue
        assert ctx.plan["depth_chunk"] >= (C if C else 2)
        out = ctx.apply_mindlin(d_ep, kind="stress", u3=u3)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) < TOL[prec], C
        assert rel_l2(u3.cpu().numpy(), u3_ref) < TOL[prec], C
        ran.append(C)
    assert len(ran) >= 5
    ctx.close()


def test_set_plan_rejects_unlaunchable_chunks():
    """Nz = 64 in FP32: chunks of 2 or 3 nodes need 32 or 22 chunk threads per column,
    more than one 256-thread tile of 16 columns holds."""
    require_gpu()
    from paper_1811_11558_gb300 import Context, FvimError

    ctx = Context(32, 32, inputs.uniform_depth(64, 0.4), precision="fp32")
    for C in (2, 3):
        with pytest.raises(FvimError) as e:
            ctx.set_plan(C)
        assert e.value.status == -1
    ctx.set_plan(4)
    assert ctx.plan == {"depth_chunk": 4, "tuned": False, "timings_ms": {}}
    ctx.set_plan(0)
    assert ctx.plan["depth_chunk"] == 4      # the default rule, max(2, ceil(64 / 16))
    ctx.close()


def test_autotune_keeps_the_fastest_per_grid():
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context

    z = inputs.uniform_depth(28, 0.4)
    ctx = Context(128, 64, z, precision="fp32")
    assert not ctx.plan["tuned"]
    pl = ctx.autotune(reps=5)
    t = pl["timings_ms"]
    assert pl["tuned"] and pl["depth_chunk"] in t and len(t) >= 4
    from paper_1811_11558_gb300 import fvim

    assert sorted(t) == sorted(fvim.plan_candidates(128, 64, 28, "fp32"))
    assert all(v > 0 for v in t.values())
    # the default rule (2 here) stays unless another length is more than 2 % faster
    assert pl["depth_chunk"] == 2 or t[pl["depth_chunk"]] < 0.98 * t[2]
    assert ctx.plan["depth_chunk"] == pl["depth_chunk"]
    # a later context of the same grid starts with the tuned plan; another grid does not
    same = Context(128, 64, z, precision="fp32")
    assert same.plan == {"depth_chunk": pl["depth_chunk"], "tuned": True, "timings_ms": {}}
    other = Context(128, 64, z, precision="fp64")
    assert not other.plan["tuned"]
    # the tuned context still computes the operator (its scratch was overwritten by the timing)
    ep = inputs.plastic_strain_field(128, 64, z, seed=1831)
    a = same.apply_mindlin(to_dev(torch, ep, torch.float32))
    b = ctx.apply_mindlin(to_dev(torch, ep, torch.float32))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    for c in (ctx, same, other):
        c.close()


def test_solve_after_plan_change_recaptures_graphs():
    """Captured solver graphs hold the depth kernel's launch shape: a plan change drops them,
    and the next solve (recaptured) meets the FP32 bar against the stored FP64 solution."""
    torch = require_gpu()
    import os
    from paper_1811_11558_gb300 import Context

    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hertz_32x32x16.npz"))
    z, loads = inputs.uniform_depth(16, 0.5), [float(w) for w in g["loads"]]
    ctx = Context(32, 32, z, 1.0, 1.0, precision="fp32", E=E, nu=NU, sigma_y=float(g["sigma_y"]),
                  E_h=float(g["E_h"]))     # set_plan is per context: the process table is untouched
    h = to_dev(torch, inputs.hertz_profile(32, 32, 1.0, 1.0, 0.5), torch.float32)
    p = torch.empty(ctx.surf_shape, dtype=torch.float32, device="cuda")
    opts = ctx.default_opts(relax=float(g["relax"]), max_iter=200)
    for C in (0, 4, 3):
        ctx.set_plan(C)
        ctx.reset_state()
        ctx.solve_contact(h, loads, p, opts)
        assert rel_l2(p.cpu().numpy().astype(np.float64), g["p"]) < 2e-5, C
    ctx.close()
