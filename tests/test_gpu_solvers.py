"""Parity of the CUDA solvers (through the C ABI) with the FP64 oracle.

The solvers stop at a tolerance, so converged answers are compared with a bound set by
the two stopping rules (not by rounding): FP64 runs use tight tolerances on both sides;
FP32 runs use the FP32 defaults and the bars of the FP32 path (2e-5 on the pressure and the
plastic strain where the solver tolerance allows it, 1e-4 on the contact area: on the 32 x 32
golden grids one node is 9.8e-4 of the area, so the areas are equal).
"""
import os

import numpy as np
import pytest

from oracle import contact as C
from oracle import operators as op
from oracle import tensors as T
from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

E, NU, R = 1.0, 0.3, 0.5
ES = T.e_star(E, NU)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hertz_32x32x16.npz")


def _ctx(n, z, prec, **kw):
    from paper_1811_11558_gb300 import Context

    return Context(n, n, z, 1.0, 1.0, precision=prec, E=E, nu=NU, **kw)


@pytest.mark.parametrize("prec,n", [("fp64", 64), ("fp32", 256)])
def test_elastic_contact_parity(prec, n):
    torch = require_gpu()
    z = inputs.uniform_depth(2, 0.1)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    W = 4.7916e-3
    ref, info = C.polonsky_keer(h, W, 1.0, 1.0, E, NU, tol=1e-13)
    ctx = _ctx(n, z, prec)
    dt = ctx.dtype
    p = torch.zeros(ctx.surf_shape, dtype=dt, device="cuda")
    opts = ctx.default_opts(cg_tol=1e-13) if prec == "fp64" else ctx.default_opts()
    it, err = ctx.elastic_contact(to_dev(torch, h, dt), W, p, opts)
    got = p.cpu().numpy()
    assert it > 3 and err < opts.cg_tol
    assert abs(got.sum() / (n * n) - W) < (1e-14 if prec == "fp64" else 1e-7) * 1.0
    area_ref = (ref > 0).mean()
    area = (got > 0).mean()
    if prec == "fp64":
        assert rel_l2(got, ref) < 1e-9
        assert area == area_ref
    else:
        print("elastic contact FP32 %d^2: p %.2e area %g vs %g" % (n, rel_l2(got, ref), area, area_ref))
        assert rel_l2(got, ref) < 2e-5
        assert abs(area - area_ref) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_device_cg_loop_equals_host_loop(prec, monkeypatch):
    """The contact CG as one WHILE graph (one read of its state per solve) and as host-driven
    batches of captured iterations run the same kernels: same pressure bit for bit, same
    iteration count, also with an iteration cap that stops it early and inside Algorithm 1."""
    torch = require_gpu()
    n = 64
    z = inputs.uniform_depth(4, 0.1)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    W = 4.7916e-3
    res = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("FVIM_DEVICE_CG", mode)
        ctx = _ctx(n, z, prec, sigma_y=0.05 * E / (1 - NU * NU), E_h=0.1 * E)
        dt = ctx.dtype
        hd = to_dev(torch, h, dt)
        out = []
        for cap in (500, 7):
            p = torch.zeros(ctx.surf_shape, dtype=dt, device="cuda")
            it, err = ctx.elastic_contact(hd, W, p, ctx.default_opts(cg_max_iter=cap), allow_not_converged=True)
            out.append((it, err, p.cpu().numpy()))
        p = torch.zeros(ctx.surf_shape, dtype=dt, device="cuda")
        rep = ctx.solve_contact(hd, [W / 2, W], p, ctx.default_opts(), allow_not_converged=True)
        out.append((rep["cg_iters"], rep["alg1_iters"], p.cpu().numpy()))
        res[mode] = out
        ctx.close()
    for a, b in zip(res["1"], res["0"]):
        assert a[0] == b[0] and a[1] == b[1]
        assert np.array_equal(a[2], b[2])
    assert res["1"][1][0] == 7                 # the cap ends the loop


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plasticity_parity(prec):
    torch = require_gpu()
    n, nz = 16, 8
    z = inputs.uniform_depth(nz, 0.5)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    sy, Eh = 0.05 * ES, 0.1
    dT, _ = C.polonsky_keer(h, 3.0e-3, 1.0, 1.0, E, NU, tol=1e-13)
    st = C.PlasticState(nz, n, n)
    # both sides solve to a residual of 1e-14 relative (FP64): the fixed points agree to 1e-10
    dE_ref, dep_ref, dEp_ref, info = C.plasticity_solve(dT, st, z, 1.0, 1.0, E, NU, sy, Eh, tol_rel=1e-14)
    assert dEp_ref.max() > 0
    ctx = _ctx(n, z, prec, sigma_y=sy, E_h=Eh)
    dt = ctx.dtype
    dE = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    dep = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    dEp = torch.empty(ctx.scal_shape, dtype=dt, device="cuda")
    opts = ctx.default_opts(df_tol_rel=1e-14) if prec == "fp64" else ctx.default_opts()
    it, res = ctx.plasticity_solve(to_dev(torch, dT, dt), dE, dep, dEp, opts)
    e = [rel_l2(dE.cpu().numpy(), dE_ref), rel_l2(dep.cpu().numpy(), dep_ref), rel_l2(dEp.cpu().numpy(), dEp_ref)]
    print("plasticity %s vs oracle: dE %.2e deps_p %.2e de_p %.2e" % (prec, *e))
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert e[0] < tol
    assert e[1] < 10 * tol
    assert e[2] < 10 * tol


def _golden_run(prec, **opt_kw):
    torch = require_gpu()
    g = np.load(GOLDEN)
    n, nz = 32, 16
    z = inputs.uniform_depth(nz, 0.5)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    ctx = _ctx(n, z, prec, sigma_y=float(g["sigma_y"]), E_h=float(g["E_h"]))
    dt = ctx.dtype
    p = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
    opts = ctx.default_opts(relax=float(g["relax"]), **opt_kw)
    rep = ctx.solve_contact(to_dev(torch, h, dt), list(g["loads"]), p, opts)
    epp = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    ep = torch.empty(ctx.scal_shape, dtype=dt, device="cuda")
    ctx.get_state(epp, ep, None)
    torch.cuda.synchronize()
    return g, rep, p.cpu().numpy(), epp.cpu().numpy(), ep.cpu().numpy()


def test_solve_contact_fp64_matches_oracle_hertz():
    """The plain FP64 elastic-plastic Hertz case (32 x 32 x 16, five increments to the load
    of an elastic peak pressure of 3 sigma_y): Algorithm 1 on the GPU against the oracle, both
    converged to e < 1e-12, at the FP64 bar of 1e-10."""
    g, rep, p, epp, ep = _golden_run("fp64", tol=1e-12, cg_tol=1e-14, df_tol_rel=1e-13, max_iter=600)
    print("hertz FP64 vs oracle: p %.2e e_p %.2e eps_p %.2e" % (
        rel_l2(p, g["p"]), rel_l2(ep, g["e_p"]), rel_l2(epp, g["eps_p"])))
    assert rep["status"] == 0 and rep["n_increments"] == 5
    assert rep["load_error"] < 1e-12
    assert rel_l2(p, g["p"]) < 1e-10
    assert rel_l2(ep, g["e_p"]) < 1e-10
    assert rel_l2(epp, g["eps_p"]) < 1e-10
    assert np.array_equal(np.array(rep["contact_area"]), g["areas"])


def test_solve_contact_fp32_matches_oracle_hertz():
    """The FP32 path (FP32 defaults: Algorithm-1 tolerance 1e-8) at the FP32 bars: 2e-5 on the
    pressure and the cumulated plastic strain, 1e-4 on the contact area (on 32 x 32, equal
    areas)."""
    g, rep, p, epp, ep = _golden_run("fp32", max_iter=200)
    print("hertz FP32 vs oracle: p %.2e e_p %.2e areas %s vs %s" % (
        rel_l2(p, g["p"]), rel_l2(ep, g["e_p"]), rep["contact_area"], list(g["areas"])))
    assert rep["status"] == 0
    assert rel_l2(p, g["p"]) < 2e-5
    assert rel_l2(ep, g["e_p"]) < 2e-5
    assert np.abs(np.array(rep["contact_area"]) - g["areas"]).max() <= 1e-4


EPP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "epp_hertz_32x32x8.npz")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_contact_perfectly_plastic_sweep(prec):
    """E_h = 0 (elastic-perfectly-plastic) Hertz sweep W / W_y = 2, 4, 8 on 32 x 32 x 8: the GPU
    Algorithm 1 against the oracle's stored solution."""
    torch = require_gpu()
    g = np.load(EPP)
    n, nz = 32, 8
    z = inputs.uniform_depth(nz, float(g["depth"]))
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    ctx = _ctx(n, z, prec, sigma_y=float(g["sigma_y"]), E_h=0.0)
    dt = ctx.dtype
    p = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
    kw = dict(cg_tol=1e-13, df_tol_rel=1e-11) if prec == "fp64" else {}
    opts = ctx.default_opts(relax=float(g["relax"]), max_iter=400, **kw)
    rep = ctx.solve_contact(to_dev(torch, h, dt), [float(w) for w in g["loads"]], p, opts)
    ep = torch.empty(ctx.scal_shape, dtype=dt, device="cuda")
    ctx.get_state(None, ep, None)
    torch.cuda.synchronize()
    assert rep["status"] == 0 and rep["n_increments"] == 3
    pn, epn = p.cpu().numpy(), ep.cpu().numpy()
    print("epp %s vs oracle: p %.2e e_p %.2e areas %s vs %s" % (
        prec, rel_l2(pn, g["p"]), rel_l2(epn, g["e_p"]), rep["contact_area"], list(g["areas"])))
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert rel_l2(pn, g["p"]) < tol
    assert rel_l2(epn, g["e_p"]) < (1e-10 if prec == "fp64" else 1e-4)
    assert np.abs(np.array(rep["contact_area"]) - g["areas"]).max() <= (0 if prec == "fp64" else 1e-4)


ROUGH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rough_32x32x8.npz")


def _rough_run(prec, **opt_kw):
    """The small elastic-plastic rough-surface case (self-affine 32 x 32, 8 nodes to z = 0.1,
    two increments to W = 5e-3, relaxation 0.3) through Algorithm 1 on the GPU."""
    torch = require_gpu()
    g = np.load(ROUGH)
    n, nz = 32, 8
    z = inputs.uniform_depth(nz, float(g["depth"]))
    # the stored surface is the oracle's input (the generator's FFT may round differently on
    # another machine)
    h = np.array(g["h"])
    assert np.allclose(h, inputs.self_affine_surface(n, 1.0, 0.8, 2, 4, 8, 0.1, seed=1813), rtol=0, atol=1e-12)
    ctx = _ctx(n, z, prec, sigma_y=float(g["sigma_y"]), E_h=float(g["E_h"]))
    dt = ctx.dtype
    p = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
    rep = ctx.solve_contact(to_dev(torch, h, dt), list(g["loads"]), p,
                            ctx.default_opts(relax=float(g["relax"]), **opt_kw))
    epp = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    ep = torch.empty(ctx.scal_shape, dtype=dt, device="cuda")
    ctx.get_state(epp, ep, None)
    torch.cuda.synchronize()
    return g, rep, p.cpu().numpy(), epp.cpu().numpy(), ep.cpu().numpy()


def test_rough_solve_fp64_matches_oracle():
    g, rep, p, epp, ep = _rough_run("fp64", cg_tol=1e-13, df_tol_rel=1e-11, max_iter=200)
    print("rough FP64 vs oracle: p %.2e e_p %.2e eps_p %.2e" % (
        rel_l2(p, g["p"]), rel_l2(ep, g["e_p"]), rel_l2(epp, g["eps_p"])))
    assert rep["status"] == 0 and rep["n_increments"] == 2
    assert rel_l2(p, g["p"]) < 1e-10
    assert rel_l2(ep, g["e_p"]) < 1e-10
    assert rel_l2(epp, g["eps_p"]) < 1e-10
    assert np.array_equal(np.array(rep["contact_area"]), g["areas"])


def test_rough_solve_fp32_matches_oracle():
    g, rep, p, epp, ep = _rough_run("fp32", max_iter=200)
    print("rough FP32 vs oracle: p %.2e e_p %.2e eps_p %.2e areas %s vs %s" % (
        rel_l2(p, g["p"]), rel_l2(ep, g["e_p"]), rel_l2(epp, g["eps_p"]), rep["contact_area"], list(g["areas"])))
    assert rep["status"] == 0
    assert rel_l2(p, g["p"]) < 2e-5
    assert rel_l2(ep, g["e_p"]) < 2e-5
    assert np.abs(np.array(rep["contact_area"]) - g["areas"]).max() <= 1e-4


def test_solve_contact_deterministic_and_caps():
    torch = require_gpu()
    n, nz = 16, 8
    z = inputs.uniform_depth(nz, 0.5)
    h = to_dev(torch, inputs.hertz_profile(n, n, 1.0, 1.0, R), torch.float64)
    outs = []
    for _ in range(2):
        ctx = _ctx(n, z, "fp64", sigma_y=0.05 * ES, E_h=0.1)
        p = torch.empty(ctx.surf_shape, dtype=torch.float64, device="cuda")
        ctx.solve_contact(h, [2e-3, 4e-3], p)
        outs.append(p.clone())
    assert torch.equal(outs[0], outs[1])
    # an iteration cap is reported, not hidden
    ctx = _ctx(n, z, "fp64", sigma_y=0.05 * ES, E_h=0.1)
    p = torch.empty(ctx.surf_shape, dtype=torch.float64, device="cuda")
    rep = ctx.solve_contact(h, [4e-3], p, ctx.default_opts(max_iter=1), allow_not_converged=True)
    assert rep["status"] == -5 and rep["alg1_iters"][0] == 1
    # a non-finite surface is refused with a status, the GPU stays usable
    bad = h.clone()
    bad[3, 3] = float("nan")
    from paper_1811_11558_gb300 import FvimError

    with pytest.raises(FvimError):
        ctx.elastic_contact(bad, 4e-3, torch.zeros_like(p))
    torch.cuda.synchronize()
    assert torch.isfinite(outs[0]).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_carried_relaxation_reaches_the_oracle_solution(prec):
    """Algorithm 1 with the relaxed value carried between iterations (FVIM_RELAX_CARRIED)
    converges to the same increments as the listing's order: the stored oracle solution of the
    Hertz case (written with the literal order).  The two orders stop at different iterates of
    one fixed point, each with e < 1e-12 relative to ||H0||, the norm of the whole surface, some
    10^2-10^3 times the indentation the pressure answers to: the FP64 pressures agree to about
    1e-9 (the literal GPU solve, which follows the oracle's own path, agrees to 2e-11)."""
    kw = dict(tol=1e-12, cg_tol=1e-14, df_tol_rel=1e-13, max_iter=600) if prec == "fp64" else dict(max_iter=400)
    g, rep, p, epp, ep = _golden_run(prec, relax_mode=1, **kw)
    print("hertz carried %s vs oracle: p %.2e e_p %.2e iters %s" % (prec, rel_l2(p, g["p"]), rel_l2(ep, g["e_p"]),
                                                                  rep["alg1_iters"]))
    assert rep["status"] == 0
    tol = 2e-9 if prec == "fp64" else 2e-5
    assert rel_l2(p, g["p"]) < tol
    assert rel_l2(ep, g["e_p"]) < tol
    assert np.abs(np.array(rep["contact_area"]) - g["areas"]).max() <= (0 if prec == "fp64" else 1e-4)
