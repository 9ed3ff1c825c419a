"""Tile plans of the depth kernel and in-plane FFT paths: every chunk length and every path
gives the oracle's operator, and the autotuner keeps its choice per grid.

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
        for ctas in (2, 3):
            try:
                ctx.set_plan(C, depth_ctas=ctas)
            except FvimError as e:
                assert e.status == -1 and (C > 0 or ctas == 3)
                continue
            assert ctx.plan["depth_chunk"] >= (C if C else 2)
            out = ctx.apply_mindlin(d_ep, kind="stress", u3=u3)
            torch.cuda.synchronize()
            assert rel_l2(out.cpu().numpy(), ref) < TOL[prec], (C, ctas)
            assert rel_l2(u3.cpu().numpy(), u3_ref) < TOL[prec], (C, ctas)
            ran.append((C, ctas))
    assert len(ran) >= 5
    if prec == "fp32":
        assert any(k == 3 for _, k in ran)       # the 85-register variant ran too
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
    assert ctx.plan == {"depth_chunk": 4, "depth_ctas": 2, "depth_cutoff": 18.0, "tuned": False, "timings_ms": {},
                        "fft_path": "rows_cols"}
    ctx.set_plan(4, depth_ctas=3)
    assert ctx.plan["depth_ctas"] == 3
    with pytest.raises(FvimError) as e:
        ctx.set_plan(12, depth_ctas=3)          # the shared-memory variant has no 3-CTA budget
    assert e.value.status == -1
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

    t3 = pl.get("timings_ms_3ctas", {})
    cands = fvim.plan_candidates(128, 64, 28, "fp32")
    assert sorted(t) == sorted(c for c, k in cands if k != 3) and sorted(t3) == sorted(c for c, k in cands if k == 3)
    assert all(v > 0 for v in list(t.values()) + list(t3.values()))
    # the default rule (2 here, two CTAs per SM) stays unless another shape is more than 2 % faster
    tp = (t3 if pl["depth_ctas"] == 3 else t)[pl["depth_chunk"]]
    assert (pl["depth_chunk"], pl["depth_ctas"]) == (2, 2) or tp < 0.98 * t[2]
    assert tp == min(list(t.values()) + list(t3.values())) or (pl["depth_chunk"], pl["depth_ctas"]) == (2, 2)
    assert ctx.plan["depth_chunk"] == pl["depth_chunk"] and ctx.plan["depth_ctas"] == pl["depth_ctas"]
    # a later context of the same grid starts with the tuned plan; another grid does not
    same = Context(128, 64, z, precision="fp32")
    assert same.plan == {"depth_chunk": pl["depth_chunk"], "depth_ctas": pl["depth_ctas"], "depth_cutoff": 18.0,
                         "tuned": True, "timings_ms": {}, "fft_path": "rows_cols"}
    assert "fft_apply_ms" not in pl      # only the row / column path is built for a 64-point side
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


def test_autotune_picks_an_fft_path_per_grid():
    """On a 256 x 256 FP32 grid three in-plane FFT paths are built (row and column kernels, one
    kernel per direction through L2, one cluster per plane): the tuner times whole applies with
    each, keeps the fastest (the row / column path unless another is more than 2 % faster),
    later contexts of the grid start with it, and every path gives the same operator."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context, FvimError, fvim

    z = inputs.uniform_depth(6, 0.05)
    ctx = Context(256, 256, z, precision="fp32")
    pl = ctx.autotune(reps=5)
    t = pl["fft_apply_ms"]
    assert sorted(t) == sorted(fvim.FFT_PATHS) and all(v > 0 for v in t.values())
    best = min(t, key=t.get)
    assert pl["fft_path"] == (best if t[best] < 0.98 * t["rows_cols"] else "rows_cols")
    same = Context(256, 256, z, precision="fp32")
    assert same.plan["fft_path"] == pl["fft_path"] and same.plan["tuned"]
    ep = to_dev(torch, inputs.plastic_strain_field(256, 256, z, seed=1832), torch.float32)
    outs = {}
    for path in fvim.FFT_PATHS:
        same.set_plan(pl["depth_chunk"], path, depth_ctas=pl["depth_ctas"])
        outs[path] = same.apply_mindlin(ep).cpu().numpy().astype(np.float64)
        assert same.last_kernel_count() == (5 if path == "rows_cols" else 3)
    for path in fvim.FFT_PATHS:
        assert rel_l2(outs[path], outs["rows_cols"]) < 5e-6, path
    # FP64 and direct-DFT grids have the row / column (or DFT) path only
    d = Context(64, 64, z, precision="fp64")
    with pytest.raises(FvimError) as e:
        d.set_plan(0, "l2_exchange")
    assert e.value.status == -1
    for c in (ctx, same, d):
        c.close()


def test_solve_after_fft_path_change_recaptures_graphs():
    """Captured solver graphs hold the apply's kernels: a change of FFT path drops them, and
    the recaptured FP32 solve meets the FP32 bar against the stored FP64 solution."""
    torch = require_gpu()
    import os
    from paper_1811_11558_gb300 import Context, fvim

    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hertz_32x32x16.npz"))
    # the golden grid (32 x 32) has the row / column path only; the change is exercised on the
    # operator of a 128 x 128 grid inside the same context kind
    z = inputs.uniform_depth(16, 0.5)
    ctx = Context(128, 128, z, 1.0, 1.0, precision="fp32", E=E, nu=NU, sigma_y=float(g["sigma_y"]),
                  E_h=float(g["E_h"]))
    h = to_dev(torch, inputs.hertz_profile(128, 128, 1.0, 1.0, 0.5), torch.float32)
    p = torch.empty(ctx.surf_shape, dtype=torch.float32, device="cuda")
    opts = ctx.default_opts(relax=float(g["relax"]), max_iter=200)
    loads = [float(w) for w in g["loads"]][:2]
    ps = {}
    for path in ("rows_cols", "l2_exchange", "rows_cols"):
        ctx.set_plan(0, path)
        ctx.reset_state()
        rep = ctx.solve_contact(h, loads, p, opts)
        assert rep["status"] == 0, path
        ps.setdefault(path, []).append(p.cpu().numpy().astype(np.float64))
    # same path twice: bitwise identical (graphs dropped and recaptured in between)
    assert np.array_equal(ps["rows_cols"][0], ps["rows_cols"][1])
    assert rel_l2(ps["l2_exchange"][0], ps["rows_cols"][0]) < 2e-5
    ctx.close()


def test_chunk_scan_cutoff_error_study():
    """The chunk-scan cutoff eps_co (Sec. 3.2's cutoff, restated for the exact recursion): where
    every chunk span of a tile damps by more than e^{-eps_co}, the carries come from the
    neighbouring chunks alone.  The difference from the exact scan falls with eps_co (dropped
    terms are below e^{-eps_co} of the moments), is at the FP32 rounding level at the default
    eps_co = 18, and every setting still meets the oracle bar down to eps_co = 12."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context

    n, z = 256, inputs.uniform_depth(32, 0.4)       # chunk span 2 h = 0.026: tiles with |k| > 110
    ep = inputs.plastic_strain_field(n, n, z, seed=1833)
    ref = op.mindlin_apply(ep.astype(np.float64), z, 1.0, 1.0, E, NU, "stress")
    ctx = Context(n, n, z, 1.0, 1.0, precision="fp32", E=E, nu=NU)
    d = to_dev(torch, ep, torch.float32)
    out = {}
    for eps in (0.0, 4.0, 8.0, 12.0, 18.0):
        ctx.set_plan(2, depth_cutoff=eps)
        assert ctx.plan["depth_cutoff"] == eps
        out[eps] = ctx.apply_mindlin(d).cpu().numpy().astype(np.float64)
    diff = {eps: rel_l2(out[eps], out[0.0]) for eps in (4.0, 8.0, 12.0, 18.0)}
    err = {eps: rel_l2(out[eps], ref) for eps in out}
    print("cutoff vs exact scan:", diff, "vs oracle:", err)
    assert diff[4.0] > diff[8.0] > diff[12.0] >= diff[18.0]
    assert diff[4.0] > 1e-4           # the cutoff acts on this grid
    assert diff[18.0] < 1e-6          # below the operator's FP32 rounding (3e-7 .. 1e-6)
    for eps in (0.0, 12.0, 18.0):
        assert err[eps] < TOL["fp32"], eps
    ctx.close()


def test_depth_tile_wait_expires_and_the_context_stays_usable(monkeypatch):
    """The depth kernel's tensor-copy wait is bounded: a context created with a test offset on
    the expected copy bytes (the copies complete, the barrier never does) makes every CTA give up
    after its time limit and set the status word; fvim_sync reports FVIM_ERR_TIMEOUT once, and
    the device and a fresh context compute the operator afterwards.  No copy is left in flight."""
    torch = require_gpu()
    from paper_1811_11558_gb300 import Context, FvimError

    n, z = 32, inputs.uniform_depth(8, 0.2)        # one wave of 32 CTAs: about 2 s of waiting
    ep = inputs.plastic_strain_field(n, n, z, seed=1834)
    d = to_dev(torch, ep, torch.float32)
    monkeypatch.setenv("FVIM_TEST_TMA_EXTRA", "16")
    bad = Context(n, n, z, 1.0, 1.0, precision="fp32", E=E, nu=NU)
    monkeypatch.delenv("FVIM_TEST_TMA_EXTRA")
    bad.apply_mindlin(d)
    with pytest.raises(FvimError) as e:
        bad.sync()
    assert e.value.status == -6
    bad.sync()                                     # the status was reported once and cleared
    ref = op.mindlin_apply(ep, z, 1.0, 1.0, E, NU, "stress")
    good = Context(n, n, z, 1.0, 1.0, precision="fp32", E=E, nu=NU)
    out = good.apply_mindlin(d)
    good.sync()
    assert rel_l2(out.cpu().numpy(), ref) < TOL["fp32"]
    for c in (bad, good):
        c.close()
