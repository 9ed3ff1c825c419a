"""Parity of the CUDA operators (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over all outputs): 1e-10 for the FP64 path and 2e-5 for
the FP32 path, the bars the project states for its operators.
"""
import numpy as np
import pytest

from oracle import operators as op
from oracle import plasticity as pl
from oracle import tensors as T
from paper_1811_11558_gb300 import inputs

from gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3
TOL = {"fp64": 1e-10, "fp32": 2e-5}


def _ctx(n1, n2, z, L1, L2, prec, **kw):
    from paper_1811_11558_gb300 import Context

    return Context(n1, n2, z, L1, L2, precision=prec, E=E, nu=NU, **kw)


MINDLIN_CASES = [
    # (n1, n2, z, L1, L2, precision)
    (16, 8, inputs.uniform_depth(5, 0.3), 1.0, 0.7, "fp64"),
    (32, 32, inputs.uniform_depth(16, 0.5), 1.0, 1.0, "fp64"),          # Hertz-case grid
    (32, 16, np.array([0.0, 0.01, 0.03, 0.06, 0.1, 0.15, 0.21, 0.28, 0.36, 0.45, 0.55, 0.66, 0.8]), 1.0, 1.0, "fp64"),
    (4, 2, inputs.uniform_depth(2, 0.2), 1.0, 1.0, "fp64"),              # smallest grid, two nodes
    (64, 64, inputs.uniform_depth(16, 0.4), 1.0, 1.0, "fp32"),
    (128, 64, inputs.uniform_depth(33, 0.4), 1.0, 0.5, "fp32"),         # ragged depth chunks
    (256, 32, inputs.uniform_depth(64, 0.4), 1.0, 1.0, "fp32"),         # config-[1] depth, several tiles
    # deep grids: the depth tile narrows to fit shared memory
    (32, 16, inputs.uniform_depth(130, 0.3), 1.0, 1.0, "fp64"),
    (32, 16, inputs.uniform_depth(300, 0.5), 1.0, 1.0, "fp32"),
    # plane sizes of the whole-plane cluster FFTs (FP32); depth steps keep q h within the
    # range where the oracle's element quadrature is exact
    (256, 256, inputs.uniform_depth(4, 0.06), 1.0, 1.0, "fp32"),
    (512, 256, inputs.uniform_depth(3, 0.02), 1.0, 0.5, "fp32"),
    (256, 512, np.array([0.0, 0.004, 0.011]), 0.5, 1.0, "fp32"),
    # larger planes, non-square cells, ragged depth chunks
    (128, 128, inputs.uniform_depth(33, 0.4), 1.0, 0.6, "fp32"),
    (128, 256, np.array([0.0, 0.005, 0.012, 0.02, 0.035]), 0.7, 1.0, "fp32"),
    (512, 512, inputs.uniform_depth(3, 0.01), 1.0, 1.0, "fp32"),
    (1024, 512, inputs.uniform_depth(2, 0.004), 1.0, 0.5, "fp32"),
    # sides that are not powers of two (direct DFTs): odd grids, whose every mode is in Z^2_N,
    # and mixed ones, whose even side keeps its Nyquist row or column out of the operator
    (9, 7, inputs.uniform_depth(5, 0.3), 1.0, 0.8, "fp64"),
    (27, 27, np.array([0.0, 0.01, 0.03, 0.06, 0.1, 0.15, 0.21, 0.28]), 1.0, 1.0, "fp64"),
    (81, 81, inputs.uniform_depth(4, 0.03), 1.0, 1.0, "fp32"),
    (81, 81, inputs.uniform_depth(6, 0.05), 1.0, 1.0, "fp64"),
    (15, 32, inputs.uniform_depth(9, 0.2), 0.6, 1.0, "fp32"),
    (64, 27, inputs.uniform_depth(7, 0.1), 1.0, 0.5, "fp64"),
]

CLUSTER_PLANES = {(256, 256), (512, 512), (256, 512), (512, 256)}
FUSED_PLANES = {(128, 128), (256, 128), (128, 256), (256, 256), (512, 256), (256, 512), (512, 512),
                (1024, 512), (512, 1024), (1024, 1024)}


def _kernels(n1, n2, prec, with_u3):
    """Kernels of one Mindlin apply on the default path: rows / columns / depth / columns /
    rows, plus two for the surface displacement."""
    return 5 + (2 if with_u3 else 0)


@pytest.mark.parametrize("n1,n2,z,L1,L2,prec", MINDLIN_CASES)
@pytest.mark.parametrize("kind", ["stress", "strain"])
def test_mindlin_parity(n1, n2, z, L1, L2, prec, kind, monkeypatch):
    torch = require_gpu()
    # the default path: separate row and column kernels (direct DFTs on odd grids)
    monkeypatch.setenv("FVIM_FFT2_CLUSTER", "0")
    monkeypatch.delenv("FVIM_FFT2_FUSED", raising=False)
    ep = inputs.plastic_strain_field(n1, n2, z, seed=1812 + n1 + n2 + z.size)
    ref, u3_ref = op.mindlin_apply(ep, z, L1, L2, E, NU, kind, with_surface=True)
    ctx = _ctx(n1, n2, z, L1, L2, prec)
    dt = ctx.dtype
    d_ep = to_dev(torch, ep, dt)
    u3 = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
    out = ctx.apply_mindlin(d_ep, kind=kind, u3=u3)
    torch.cuda.synchronize()
    assert ctx.last_kernel_count() == _kernels(n1, n2, prec, True)
    assert rel_l2(out.cpu().numpy(), ref) < TOL[prec]
    assert rel_l2(u3.cpu().numpy(), u3_ref) < TOL[prec]
    # the input is not modified
    assert torch.equal(d_ep, to_dev(torch, ep, dt))


@pytest.mark.parametrize("n1,n2", sorted(FUSED_PLANES | CLUSTER_PLANES))
def test_fft_paths_agree(n1, n2, monkeypatch):
    """The one-pass 2-D FFTs through L2, the whole-plane cluster FFTs (both opt-in) in distributed shared memory and the separate row / column
    kernels compute the same operator (FP32 rounding apart), for the Mindlin stress, strain
    and surface displacement and the Boussinesq volume output."""
    torch = require_gpu()
    z = inputs.uniform_depth(5, 0.1)
    ep = to_dev(torch, inputs.plastic_strain_field(n1, n2, z, seed=77 + n1 + n2, dtype=np.float32), torch.float32)
    p = to_dev(torch, np.abs(inputs.random_field((n2, n1), seed=5)) + 0.5, torch.float32)
    paths = {"rows_cols": ({"FVIM_FFT2_CLUSTER": "0"}, 7)}
    if (n1, n2) in FUSED_PLANES:
        paths["fused"] = ({"FVIM_FFT2_FUSED": "1", "FVIM_FFT2_CLUSTER": "0"}, 5)
    if (n1, n2) in CLUSTER_PLANES:
        paths["cluster"] = ({"FVIM_FFT2_CLUSTER": "1"}, 5)
    outs = {}
    for name, (env, nk) in paths.items():
        for k in ("FVIM_FFT2_FUSED", "FVIM_FFT2_CLUSTER"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        ctx = _ctx(n1, n2, z, 1.0, 1.0, "fp32")
        u3 = torch.empty(ctx.surf_shape, dtype=torch.float32, device="cuda")
        s = ctx.apply_mindlin(ep, kind="stress", u3=u3).clone()
        assert ctx.last_kernel_count() == nk, name
        e = ctx.apply_mindlin(ep, kind="strain").clone()
        vol = torch.empty(ctx.vol_shape, dtype=torch.float32, device="cuda")
        ctx.apply_boussinesq(p, vol=vol, kind="stress")
        torch.cuda.synchronize()
        outs[name] = [x.cpu().numpy().astype(np.float64) for x in (s, e, u3, vol)]
    for name, got in outs.items():
        for a, b in zip(got, outs["rows_cols"]):
            assert rel_l2(a, b) < 5e-6, name


def test_mindlin_deterministic_and_reusable():
    torch = require_gpu()
    z = inputs.uniform_depth(20, 0.4)
    ep = inputs.plastic_strain_field(64, 32, z, seed=5)
    ctx = _ctx(64, 32, z, 1.0, 1.0, "fp32")
    d = to_dev(torch, ep, torch.float32)
    a = ctx.apply_mindlin(d).clone()
    b = ctx.apply_mindlin(d).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_mindlin_full_size_sampled_modes():
    """512 x 512 x 64 FP32 (the operator-apply workload, the launch configuration the
    benchmark times): the GPU stress is transformed back to Fourier space in FP64 and
    a random sample of modes is compared with the oracle's per-mode operator."""
    torch = require_gpu()
    n, nz = 512, 64
    z = inputs.uniform_depth(nz, 0.4)
    ep = inputs.plastic_strain_field(n, n, z, seed=1812, dtype=np.float32)
    ctx = _ctx(n, n, z, 1.0, 1.0, "fp32")
    d = to_dev(torch, ep, torch.float32)
    out = ctx.apply_mindlin(d)
    torch.cuda.synchronize()
    lam, mu = T.lame(E, NU)
    w_hat = np.fft.fft2(T.hooke6(ep.astype(np.float64), lam, mu, axis=1), axes=(-2, -1))
    s_hat = np.fft.fft2(out.cpu().numpy().astype(np.float64), axes=(-2, -1))
    rng = np.random.default_rng(0)
    k2 = rng.integers(0, n, 200)
    k1 = rng.integers(0, n, 200)
    Q1, Q2, nyq, zero = op.mode_grid(n, n, 1.0, 1.0)
    keep = ~(nyq[k2, k1] | zero[k2, k1])
    k1, k2 = k1[keep], k2[keep]
    W = np.moveaxis(T.sym6_to_full(w_hat[:, :, k2, k1], axis=1), 1, 0)  # [K, nz, 3, 3]
    Q = np.stack([Q1[k2, k1], Q2[k2, k1]], axis=1)
    H, _, _ = op.mindlin_modes(W, Q, z, E, NU)
    sig = T.hooke_full(T.sym_part(H), lam, mu) - W
    ref = np.moveaxis(T.full_to_sym6(sig, axis=-1), -1, 1)                # [K, 6, nz]... reorder below
    got = np.moveaxis(s_hat[:, :, k2, k1], 2, 0)                          # [K, nz, 6]
    ref = np.moveaxis(ref, 1, 2)                                          # [K, nz, 6]
    assert rel_l2(got, ref) < TOL["fp32"]
    # the full output is real, finite and has the free surface of Eq. fundamental_problem
    assert np.isfinite(out.cpu().numpy()).all()


BOUS_CASES = [
    (16, 8, inputs.uniform_depth(5, 0.3), 1.0, 0.7, "fp64"),
    (32, 32, np.array([0.0, 0.02, 0.05, 0.1, 0.2, 0.35, 0.5]), 1.0, 1.0, "fp64"),
    (128, 64, inputs.uniform_depth(17, 0.2), 1.0, 1.0, "fp32"),
    (256, 256, inputs.uniform_depth(3, 0.05), 1.0, 1.0, "fp32"),         # one-pass inverse FFT
    (512, 128, inputs.uniform_depth(4, 0.03), 1.0, 0.4, "fp32"),
    (27, 21, inputs.uniform_depth(6, 0.2), 1.0, 0.8, "fp64"),
    (81, 81, inputs.uniform_depth(5, 0.05), 1.0, 1.0, "fp32"),
    (32, 9, inputs.uniform_depth(4, 0.1), 1.0, 1.0, "fp64"),
]


@pytest.mark.parametrize("n1,n2,z,L1,L2,prec", BOUS_CASES)
@pytest.mark.parametrize("kind", ["stress", "strain"])
def test_boussinesq_parity(n1, n2, z, L1, L2, prec, kind, monkeypatch):
    torch = require_gpu()
    monkeypatch.setenv("FVIM_FFT2_CLUSTER", "0")
    monkeypatch.delenv("FVIM_FFT2_FUSED", raising=False)
    p = np.abs(inputs.random_field((n2, n1), seed=3 + n1)) + 0.5
    u3_ref, vol_ref = op.boussinesq_apply(p, z, L1, L2, E, NU, kind)
    ctx = _ctx(n1, n2, z, L1, L2, prec)
    dt = ctx.dtype
    u3 = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
    vol = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    ctx.apply_boussinesq(to_dev(torch, p, dt), u3=u3, vol=vol, kind=kind)
    torch.cuda.synchronize()
    assert rel_l2(u3.cpu().numpy(), u3_ref) < TOL[prec]
    assert rel_l2(vol.cpu().numpy(), vol_ref) < TOL[prec]
    # surface only (no volume output; its column pass transforms, applies the compliance and
    # transforms back in one kernel) gives the same displacement up to rounding
    u3b = torch.empty_like(u3)
    ctx.apply_boussinesq(to_dev(torch, p, dt), u3=u3b)
    torch.cuda.synchronize()
    assert rel_l2(u3b.cpu().numpy(), u3.cpu().numpy()) < (1e-14 if prec == "fp64" else 1e-6)
    assert rel_l2(u3b.cpu().numpy(), u3_ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_return_map_parity(prec):
    torch = require_gpu()
    n1, n2 = 32, 16
    z = inputs.uniform_depth(6, 0.3)
    rng = np.random.default_rng(9)
    shp = (z.size, 6, n2, n1)
    sig_n = rng.standard_normal(shp) * 0.02
    e_p = np.abs(rng.standard_normal((z.size, n2, n1))) * 0.01
    d_eps = rng.standard_normal(shp) * 0.05
    sy, Eh = 0.05, 0.1
    dep_ref, dEp_ref, _ = pl.return_map(np.moveaxis(d_eps, 1, 0), np.moveaxis(sig_n, 1, 0), e_p, E, NU, sy, Eh)
    dep_ref = np.moveaxis(dep_ref, 0, 1)
    ctx = _ctx(n1, n2, z, 1.0, 1.0, prec, sigma_y=sy, E_h=Eh)
    dt = ctx.dtype
    ctx.set_state(e_p=to_dev(torch, e_p, dt), sigma=to_dev(torch, sig_n, dt))
    d_eps_p = torch.empty(ctx.vol_shape, dtype=dt, device="cuda")
    d_ep = torch.empty(ctx.scal_shape, dtype=dt, device="cuda")
    ctx.return_map(to_dev(torch, d_eps, dt), d_eps_p, d_ep)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert rel_l2(d_eps_p.cpu().numpy(), dep_ref) < tol
    assert rel_l2(d_ep.cpu().numpy(), dEp_ref) < tol
    # the plastic/elastic decision matches the oracle's wherever it is not within rounding
    f_margin = np.abs(dEp_ref) > 1e-5
    assert np.array_equal((d_ep.cpu().numpy() > 0)[f_margin], (dEp_ref > 0)[f_margin])


def test_commit_state():
    torch = require_gpu()
    z = inputs.uniform_depth(4, 0.3)
    ctx = _ctx(8, 4, z, 1.0, 1.0, "fp64", sigma_y=0.05, E_h=0.1)
    rng = np.random.default_rng(2)
    d_eps = rng.standard_normal(ctx.vol_shape) * 0.01
    d_eps_p = rng.standard_normal(ctx.vol_shape) * 0.001
    d_ep = np.abs(rng.standard_normal(ctx.scal_shape)) * 0.001
    ctx.commit_state(*(to_dev(torch, a, torch.float64) for a in (d_eps, d_eps_p, d_ep)))
    sig = torch.empty(ctx.vol_shape, dtype=torch.float64, device="cuda")
    epp = torch.empty(ctx.vol_shape, dtype=torch.float64, device="cuda")
    ep = torch.empty(ctx.scal_shape, dtype=torch.float64, device="cuda")
    ctx.get_state(epp, ep, sig)
    torch.cuda.synchronize()
    lam, mu = T.lame(E, NU)
    assert np.allclose(sig.cpu().numpy(), T.hooke6(d_eps - d_eps_p, lam, mu, axis=1), atol=1e-15)
    assert np.allclose(epp.cpu().numpy(), d_eps_p, atol=0)
    assert np.allclose(ep.cpu().numpy(), d_ep, atol=0)


def test_argument_errors():
    torch = require_gpu()
    from paper_1811_11558_gb300 import fvim

    L = fvim.lib()
    import ctypes

    h = ctypes.c_void_p()
    z = np.array([0.0, 0.1, 0.2])
    zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.fvim_create(ctypes.byref(h), 12, 8, 3, zp, 1.0, 1.0, 0, None) == fvim.FvimError(-1, "").status
    bad = np.array([0.1, 0.2, 0.3])
    assert L.fvim_create(ctypes.byref(h), 8, 8, 3, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         1.0, 1.0, 0, None) == -1
    ctx = _ctx(8, 8, z, 1.0, 1.0, "fp32")
    d = torch.zeros(ctx.vol_shape, dtype=torch.float32, device="cuda")
    assert L.fvim_apply_mindlin(ctx._h, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()), 0, None) == -1
    assert L.fvim_apply_mindlin(ctx._h, ctypes.c_void_p(d.data_ptr()), None, 0, None) == -1
