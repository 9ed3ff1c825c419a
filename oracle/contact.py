"""Elastic contact and elastic-plastic coupling (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

polonsky_keer
    Elastic normal contact of the periodic half-space with a rigid surface h under the
    total load W (Sec. 5.1: dual problem with the load constraint Eq. total_pressure,
    solved with the constrained conjugate gradient of Polonsky & Keer 1999; the FFT
    gives u3 = K*p with K_hat = 2/(E* q), K_hat(0) = 0).  Unknown: pressure p >= 0 on the
    surface grid (force per unit area pushing into the body); gap g = u3 - h + c >= 0,
    p g = 0, dA sum p = W, the rigid shift c being the multiplier of the load.
    Iteration (the published method, in its order):
      u = K*p;  g = u - h, centred on the contact set I_c = {p > 0};
      t = g + delta (G/G_old) t on I_c, 0 elsewhere (delta = 0 after a step that found
      penetrating points outside I_c, else 1);  r = K*t centred on I_c;
      tau = <g, t>_Ic / <r, t>_Ic;  p <- max(p - tau t, 0);
      penetrating points with zero pressure get p <- -tau g;  p <- p W / (dA sum p);
      stop when dA sum |p - p_prev| / W < tol.
    Parity: pinned by the KKT conditions and the Hertz closed forms (contact radius,
    peak pressure, pressure profile) in tests/test_oracle_solvers.py.  The elastic
    contact problem is strictly convex, so p is unique for a given h: iterates are not
    compared, only the converged pressure.

algorithm1
    Sec. 5.2, Algorithm 1, literally: elastic contact with the modified surface
    H = H0 - dU_prev, pressure increment dT, plastic strain increment dE from the
    DF-SANE solve of R[dE] = dE - grad^sym M[dT] - grad^sym N[C:deps_p(dE; S)] = 0,
    surface residual displacement dU = N[C:deps_p].e3 at z = 0, error
    e = ||dU - dU_prev|| / ||H0||, relaxation, H = H0 - dU_prev, dU_prev = dU, until
    e < tol or k > N_max; then update(S).
    Readings: H0 = h - N[C:eps_p_n].e3|0 at the start of the increment (Rem.
    modified_contact); the literal order of the relaxation lines is kept by default, and the
    under-relaxation that carries the relaxed value (what the text ascribes to lambda) is
    the option relax_mode="carried".
    Parity: the converged increment is pinned by its defining equations (R = 0, contact
    KKT on the modified surface, plastic admissibility, total load); the iterates of
    the coupling loop are not compared.
"""
import numpy as np

from . import operators as op
from .plasticity import dfsane, return_map
from .tensors import lame, hooke6


def surface_conv(f, kern):
    """u = K*f with the Fourier multiplier kern (numpy FFT as the library DFT)."""
    return np.fft.ifft2(kern * np.fft.fft2(f)).real


def polonsky_keer(h, W, L1, L2, E, nu, tol=1e-12, max_iter=5000, p0=None):
    """Return (p, info) for the elastic contact of the surface h [N2, N1] under load W."""
    h = np.asarray(h, dtype=np.float64)
    N2, N1 = h.shape
    dA = L1 * L2 / (N1 * N2)
    kern = op.surface_compliance(N1, N2, L1, L2, E, nu)
    p = np.full_like(h, W / (L1 * L2)) if p0 is None else np.array(p0, dtype=np.float64)
    if p0 is not None:
        p *= W / (dA * p.sum())
    t = np.zeros_like(h)
    delta = 0.0
    G_old = 1.0
    err = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        u = surface_conv(p, kern)
        Ic = p > 0
        g = u - h
        g = g - g[Ic].mean()
        G = np.sum(g[Ic] ** 2)
        t = np.where(Ic, g + delta * (G / G_old) * t, 0.0)
        G_old = G
        r = surface_conv(t, kern)
        r = r - r[Ic].mean()
        denom = np.sum(r[Ic] * t[Ic])
        tau = np.sum(g[Ic] * t[Ic]) / denom if denom != 0 else 0.0
        p_old = p
        p = np.maximum(p - tau * t, 0.0)
        Iol = (p == 0.0) & (g < 0.0)
        if Iol.any():
            delta = 0.0
            p = np.where(Iol, p - tau * g, p)
        else:
            delta = 1.0
        p = p * (W / (dA * p.sum()))
        err = dA * np.abs(p - p_old).sum() / W
        if err < tol:
            break
    u = surface_conv(p, kern)
    Ic = p > 0
    shift = np.mean((h - u)[Ic])
    gap = u - h + shift
    return p, {"iterations": it, "error": err, "gap": gap, "area": float(Ic.mean()), "displacement": u}


class PlasticState:
    """S_n = (e_p, eps_p) of Sec. 4.2 plus sigma_n, and the last converged pressure."""

    def __init__(self, nz, n2, n1):
        self.eps_p = np.zeros((nz, 6, n2, n1))
        self.e_p = np.zeros((nz, n2, n1))
        self.sigma = np.zeros((nz, 6, n2, n1))
        self.T = np.zeros((n2, n1))


def depth_weights_trapezoid(z):
    """Trapezoid weights of the depth nodes (for the discrete L2 inner product)."""
    z = np.asarray(z, dtype=np.float64)
    w = np.zeros_like(z)
    h = np.diff(z)
    w[:-1] += 0.5 * h
    w[1:] += 0.5 * h
    return w


def l2_inner(z, dA):
    """<a, b> = sum over voxels dA w_z (a:b), shears counted twice (reading: the paper
    leaves the discrete scalar product of Sec. 4.3 unspecified)."""
    wz = depth_weights_trapezoid(z)[:, None, None] * dA
    cw = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])

    def inner(a, b):
        return float(np.sum(wz[:, None] * cw[None, :, None, None] * a * b))

    return inner


def plasticity_solve(dT, state, z, L1, L2, E, nu, sigma_y, E_h, tol_abs=1e-14, tol_rel=1e-10,
                     max_iter=500):
    """DF-SANE solve of R[dE] = dE - grad^sym M[dT] - grad^sym N[C:deps_p(dE; S)] = 0
    (Sec. 4.2 Eq. incremental_strain).  Returns (dE, deps_p, dEp, info)."""
    nz, _, n2, n1 = state.sigma.shape
    lam, mu = lame(E, nu)
    _, b = op.boussinesq_apply(dT, z, L1, L2, E, nu, "strain")

    def flow(x):
        dep, dEp, _ = return_map(np.moveaxis(x, 1, 0), np.moveaxis(state.sigma, 1, 0), state.e_p, E, nu,
                                 sigma_y, E_h)
        return np.moveaxis(dep, 0, 1), dEp

    def R(x):
        dep, _ = flow(x)
        return x - b - op.mindlin_apply(dep, z, L1, L2, E, nu, "strain")

    inner = l2_inner(z, L1 * L2 / (n1 * n2))
    x, info = dfsane(R, b.copy(), inner, tol_abs, tol_rel, max_iter)
    dep, dEp = flow(x)
    return x, dep, dEp, info


def residual_surface(eps_p, z, L1, L2, E, nu):
    """u3 = N[C:eps_p].e3 at z = 0 (mode 0 set to 0)."""
    _, u3 = op.mindlin_apply(eps_p, z, L1, L2, E, nu, "strain", with_surface=True)
    return u3


def algorithm1(W, h, state, z, L1, L2, E, nu, sigma_y, E_h, tol=1e-9, N_max=50, relax=1.0,
               cg_tol=1e-13, df_tol_rel=1e-11, relax_mode="literal"):
    """One load increment of Algorithm 1 (Sec. 5.2).  Updates ``state`` in place and
    returns (T, info).

    relax_mode "literal": the listing's order (relax, H = H0 - relaxed, then dU_prev = dU).
    relax_mode "carried": the relaxed value is kept as dU_prev (under-relaxation of the fixed
    point dU = F(H0 - dU)); the error is then the fixed-point residual ||dU - dU_prev|| / ||H0||
    against the relaxed value the modified surface was built from.  The paper's text says the
    relaxation helps convergence on large steps, which is what this form does; both give the
    same converged increment."""
    if relax_mode not in ("literal", "carried"):
        raise ValueError(relax_mode)
    H0 = np.asarray(h, dtype=np.float64) - residual_surface(state.eps_p, z, L1, L2, E, nu)
    h_norm = np.linalg.norm(H0)
    dU_prev = np.zeros_like(H0)
    T_prev = state.T
    H = H0.copy()
    e = np.inf
    k = 1
    T = dE = dep = dEp = None
    history = []
    while True:
        T, cinfo = polonsky_keer(H, W, L1, L2, E, nu, tol=cg_tol, p0=T)
        dT = T - T_prev
        dE, dep, dEp, dinfo = plasticity_solve(dT, state, z, L1, L2, E, nu, sigma_y, E_h, tol_rel=df_tol_rel)
        dU = residual_surface(dep, z, L1, L2, E, nu)
        e = np.linalg.norm(dU - dU_prev) / h_norm
        history.append((cinfo["iterations"], dinfo["iterations"], e))
        dU_prev = dU_prev + relax * (dU - dU_prev)
        H = H0 - dU_prev
        if relax_mode == "literal":
            dU_prev = dU
        k += 1
        if e < tol or k > N_max:
            break
    # update(S, dE): sigma_n += C:(dE - deps_p), e_p += de_p, eps_p += deps_p
    lam, mu = lame(E, nu)
    state.sigma = state.sigma + hooke6(dE - dep, lam, mu, axis=1)
    state.e_p = state.e_p + dEp
    state.eps_p = state.eps_p + dep
    state.T = T
    area = float(np.mean(T > 0))
    return T, {"iterations": k - 1, "error": e, "converged": e < tol, "history": history, "area": area,
               "H0": H0, "dE": dE}
