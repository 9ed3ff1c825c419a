"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these calls the CUDA path.  Each test names the passage it checks.
"""
import numpy as np
import pytest

from oracle import kernels as K
from oracle import operators as op
from oracle import plasticity as pl
from oracle import tensors as T

import navier_ode as ode

E, NU = 1.0, 0.3
LAM, MU = T.lame(E, NU)


def _fd_deriv(f, x, h, order):
    """Central finite-difference derivative of order 1 or 2 (8th-order accurate)."""
    c1 = [(1, 4 / 5), (2, -1 / 5), (3, 4 / 105), (4, -1 / 280)]
    c2 = [(1, 8 / 5), (2, -1 / 5), (3, 8 / 315), (4, -1 / 560)]
    if order == 1:
        return sum(c * (f(x + k * h) - f(x - k * h)) for k, c in c1) / h
    f0 = f(x)
    return (sum(c * (f(x + k * h) + f(x - k * h)) for k, c in c2) - 205 / 72 * f0) / h ** 2


def _navier_residual(Ufun, Q, y, h=2e-3):
    """mu (U'' - q^2 U) + (lambda+mu) grad(div U) for every column of U(y) [3, 3]."""
    q1, q2 = Q
    q2sum = q1 * q1 + q2 * q2
    U = Ufun(y)
    Up = _fd_deriv(Ufun, y, h, 1)
    Upp = _fd_deriv(Ufun, y, h, 2)
    res = np.zeros((3, 3), dtype=complex)
    for k in range(3):            # force index: displacement is U[k, :]
        u, du, ddu = U[k], Up[k], Upp[k]
        div = 1j * q1 * u[0] + 1j * q2 * u[1] + du[2]
        ddiv = 1j * q1 * du[0] + 1j * q2 * du[1] + ddu[2]
        grad_div = np.array([1j * q1 * div, 1j * q2 * div, ddiv])
        res[k] = MU * (ddu - q2sum * u) + (LAM + MU) * grad_div
    return res


QS = [(6.0, 0.0), (3.0, -4.0), (-11.0, 7.0)]


@pytest.mark.parametrize("Q", QS)
def test_kelvin_solves_navier_away_from_source_and_is_continuous(Q):
    """Eq. full_space_solution / Table 1: each column of U_inf solves N[U] = 0 for y3 != x3
    (Eq. ker(N)), U_inf is continuous at y3 = x3, and the traction jump across the
    source plane balances the point force e_k (Eq. fourier_kelvin_problem)."""
    Qa = np.array([Q], dtype=float)

    def U(t):
        return K.kelvin_displacement(Qa, MU, NU, t)[0]

    scale = np.abs(U(0.0)).max()
    for t in (-0.35, -0.1, 0.12, 0.4):
        r = _navier_residual(U, Q, t)
        assert np.abs(r).max() < 1e-7 * scale * (Q[0] ** 2 + Q[1] ** 2)
    # continuity (g1 vanishes at 0, U00 is common to both branches)
    eps = 1e-9
    assert np.allclose(U(-eps), U(eps), atol=1e-7 * scale)
    # traction jump: sigma(u) . e3 just below minus just above = -e_k (force balance)
    def trac(t, k):
        h = 1e-4
        u = U(t)[k]
        du = (U(t + h)[k] - U(t - h)[k]) / (2 * h) if abs(t) > 2 * h else None
        return u, du
    for k in range(3):
        def tau(t):
            h = 1e-5
            sgn = np.sign(t)
            # one-sided second-order derivative staying on the branch of t
            u0 = U(t)[k]
            u1 = U(t + sgn * h)[k]
            u2 = U(t + 2 * sgn * h)[k]
            du = sgn * (-3 * u0 + 4 * u1 - u2) / (2 * h)
            grad = np.zeros((3, 3), dtype=complex)
            grad[:, 0] = 1j * Q[0] * u0
            grad[:, 1] = 1j * Q[1] * u0
            grad[:, 2] = du
            eps_ = 0.5 * (grad + grad.T)
            sig = LAM * np.trace(eps_) * np.eye(3) + 2 * MU * eps_
            return sig[:, 2]
        jump = tau(1e-9) - tau(-1e-9)
        expect = np.zeros(3)
        expect[k] = -1.0
        assert np.allclose(jump, expect, atol=2e-6)


@pytest.mark.parametrize("Q", QS)
def test_boussinesq_traction_condition_and_compliance(Q):
    """Eq. B:fourier: B solves N[B] = 0 in the body, T[B^k] = e_k on the surface
    (n = -e3, so sigma . e3 = -e_k), and B_33(q, 0) = 2 / (E* q) (Sec. 5.1 footnote)."""
    Qa = np.array([Q], dtype=float)
    q = np.hypot(*Q)

    def B(y):
        return K.boussinesq_displacement(Qa, MU, NU, y)[0]

    scale = np.abs(B(0.0)).max()
    for y in (0.05, 0.2, 0.5):
        assert np.abs(_navier_residual(B, Q, y)).max() < 1e-7 * scale * q * q
    for k in range(3):
        h = 1e-5
        u0, u1, u2 = B(0.0)[k], B(h)[k], B(2 * h)[k]
        du = (-3 * u0 + 4 * u1 - u2) / (2 * h)
        grad = np.zeros((3, 3), dtype=complex)
        grad[:, 0] = 1j * Q[0] * u0
        grad[:, 1] = 1j * Q[1] * u0
        grad[:, 2] = du
        eps_ = 0.5 * (grad + grad.T)
        sig = LAM * np.trace(eps_) * np.eye(3) + 2 * MU * eps_
        expect = np.zeros(3)
        expect[k] = -1.0
        assert np.allclose(sig[:, 2], expect, atol=2e-6)
    assert abs(B(0.0)[2, 2] - 2.0 / (T.e_star(E, NU) * q)) < 1e-14 * scale


def test_jump_formula():
    """Eq. (jump): U01^+ - U01^- = (2 e3 x e3 - b I) x e3 / (mu b), independent of q."""
    Q = np.array([[5.0, 2.0], [-1.0, 9.0]])
    kel = K.kelvin_gradient_tensors(Q, MU, NU)
    J = kel[(1, +1)][0] - kel[(1, -1)][0]
    b = 4 * (1 - NU)
    e3 = np.array([0.0, 0.0, 1.0])
    expect = np.einsum("ab,c->abc", 2 * np.outer(e3, e3) - b * np.eye(3), e3) / (MU * b)
    assert np.allclose(J, expect[None], atol=1e-14)


CASES = [
    ((6.283185307179586, 0.0), np.linspace(0.0, 0.5, 7)),
    ((6.283185307179586, -12.566370614359172), np.linspace(0.0, 0.5, 9)),
    ((-37.69911184307752, 25.132741228718345), np.array([0.0, 0.01, 0.03, 0.07, 0.12, 0.2, 0.31])),
    ((150.79644737231007, 0.0), np.linspace(0.0, 0.1, 16)),
]


@pytest.mark.parametrize("Q,z", CASES)
def test_mindlin_matches_navier_ode(Q, z):
    """Thm 1 + Eq. (2gradient) + Eq. (jump) + Eq. (mindlin_B_U): the oracle's displacement
    gradient of one mode equals the independent solution of the traction-free Navier
    problem (App. B, Eq. eigenstress:ODE) for a piecewise-linear eigenstress."""
    rng = np.random.default_rng(7)
    W6 = rng.standard_normal((z.size, 6)) + 1j * rng.standard_normal((z.size, 6))
    Wf = T.sym6_to_full(W6, axis=1)
    H, u0, _ = op.mindlin_modes(Wf[None], np.array([Q]), z, E, NU)
    g, u = ode.solve_mode(Q[0], Q[1], z, W6, LAM, MU)
    assert np.abs(H[0] - g).max() < 1e-11 * np.abs(g).max()
    assert np.abs(u0[0] - u[0]).max() < 1e-11 * np.abs(u[0]).max()


@pytest.mark.parametrize("Q,z", CASES)
def test_boussinesq_matches_navier_ode(Q, z):
    """Eq. (B:fourier) and its gradient recurrence against the Navier ODE with the
    surface traction p e3 (sigma . e3 = -p e3 on the surface)."""
    P = 0.3 - 1.7j
    H, u0 = op.boussinesq_modes(np.array([P]), np.array([Q]), z, E, NU)
    g, u = ode.solve_mode(Q[0], Q[1], z, np.zeros((z.size, 6)), LAM, MU, t_applied=[0, 0, P])
    assert np.abs(H[0] - g).max() < 1e-11 * np.abs(g).max()
    assert np.abs(u0[0] - u[0]).max() < 1e-11 * np.abs(u[0]).max()


def test_planted_sign_error_is_caught(monkeypatch):
    """A plausible mistake (Kelvin kernel at +q instead of -q, Lemma 1) fails the ODE pin."""
    Q, z = CASES[1]
    rng = np.random.default_rng(3)
    W6 = rng.standard_normal((z.size, 6)) + 1j * rng.standard_normal((z.size, 6))
    g, _ = ode.solve_mode(Q[0], Q[1], z, W6, LAM, MU)
    orig = K.kelvin_gradient_tensors
    monkeypatch.setattr(K, "kelvin_gradient_tensors", lambda Qm, mu, nu: orig(-Qm, mu, nu))
    op._MODE_CACHE.clear()
    try:
        H, _, _ = op.mindlin_modes(T.sym6_to_full(W6, axis=1)[None], np.array([Q]), z, E, NU)
    finally:
        op._MODE_CACHE.clear()
    assert np.abs(H[0] - g).max() > 1e-2 * np.abs(g).max()


def _small_field(n1, n2, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nz, 6, n2, n1)) * 1e-3


@pytest.mark.parametrize("n1,n2", [(8, 6), (9, 7)])
def test_free_surface_and_real_output(n1, n2, monkeypatch):
    """Eq. (fundamental_problem): N[w] is traction free, so sigma_i3 = 0 at z = 0 for every
    resolved mode; the output spectrum of a real field is Hermitian, so its inverse DFT has
    no imaginary part (even grids, whose Nyquist modes are dropped, and odd ones)."""
    z = np.linspace(0, 0.4, 5)
    ep = _small_field(n1, n2, z.size, 1)
    imag = []
    ifft2 = np.fft.ifft2

    def spy(a, *args, **kw):
        r = ifft2(a, *args, **kw)
        imag.append(np.abs(r.imag).max() / max(np.abs(r.real).max(), 1e-300))
        return r

    monkeypatch.setattr(op.np.fft, "ifft2", spy)
    sig = op.mindlin_apply(ep, z, 1.0, 0.8, E, NU, "stress")
    monkeypatch.undo()
    assert imag and max(imag) < 1e-13
    # remove the Nyquist content (sigma = -w there) before checking the free surface
    w = T.hooke6(ep, LAM, MU, axis=1)
    Q1, Q2, nyq, zero = op.mode_grid(n1, n2, 1.0, 0.8)
    s_hat = np.fft.fft2(sig[0], axes=(-2, -1))
    s_hat[:, nyq] = 0.0
    top = np.fft.ifft2(s_hat, axes=(-2, -1)).real
    for c in (2, 3, 4):   # 33, 23, 13
        assert np.abs(top[c]).max() < 1e-12 * np.abs(w).max()


@pytest.mark.parametrize("n1,n2", [(4, 4), (5, 3)])
def test_translation_invariance_and_linearity_bruteforce(n1, n2):
    """Brute force on 4x4x3 and 5x3x3 grids (Sec. 1.3 translation invariance; Thm 1
    linearity): the operator assembled column by column from unit impulses is circulant
    in-plane and linear."""
    z = np.array([0.0, 0.1, 0.25])
    nz = z.size
    rng = np.random.default_rng(5)
    a = rng.standard_normal((nz, 6, n2, n1))
    b = rng.standard_normal((nz, 6, n2, n1))
    Na = op.mindlin_apply(a, z, 1.0, 1.0, E, NU)
    Nb = op.mindlin_apply(b, z, 1.0, 1.0, E, NU)
    Nab = op.mindlin_apply(2 * a - 3 * b, z, 1.0, 1.0, E, NU)
    assert np.abs(Nab - (2 * Na - 3 * Nb)).max() < 1e-12 * np.abs(Nab).max()
    # unit impulse at (x1, x2) = (0, 0) vs at (1, 2): outputs are rolled copies
    for c in range(6):
        for j in range(nz):
            e0 = np.zeros((nz, 6, n2, n1))
            e0[j, c, 0, 0] = 1.0
            e1 = np.zeros((nz, 6, n2, n1))
            e1[j, c, 2, 1] = 1.0
            r0 = op.mindlin_apply(e0, z, 1.0, 1.0, E, NU)
            r1 = op.mindlin_apply(e1, z, 1.0, 1.0, E, NU)
            assert np.abs(np.roll(r0, (2, 1), axis=(-2, -1)) - r1).max() < 1e-12


def test_laminate_mode_closed_form():
    """Rem. fundamental_mode (reading): a horizontally uniform eigenstrain gives the 1-D
    equilibrium solution sigma_i3 = 0, eps_ab = 0, eps_33 = w_33 / (lambda + 2 mu),
    eps_a3 = w_a3 / (2 mu), sigma_ab = lambda eps_33 delta_ab - w_ab."""
    z = np.linspace(0, 0.3, 4)
    rng = np.random.default_rng(2)
    prof = rng.standard_normal((z.size, 6))
    ep = np.broadcast_to(prof[:, :, None, None], (z.size, 6, 4, 4)).copy()
    w = T.hooke6(prof, LAM, MU, axis=1)
    sig = op.mindlin_apply(ep, z, 1.0, 1.0, E, NU, "stress")[:, :, 0, 0]
    eps = op.mindlin_apply(ep, z, 1.0, 1.0, E, NU, "strain")[:, :, 0, 0]
    e33 = w[:, 2] / (LAM + 2 * MU)
    assert np.allclose(eps[:, 2], e33, atol=1e-15)
    assert np.allclose(eps[:, 3], w[:, 3] / (2 * MU), atol=1e-15)
    assert np.allclose(eps[:, 4], w[:, 4] / (2 * MU), atol=1e-15)
    assert np.allclose(eps[:, [0, 1, 5]], 0.0, atol=1e-15)
    assert np.allclose(sig[:, 2:5], 0.0, atol=1e-14)
    assert np.allclose(sig[:, 0], LAM * e33 - w[:, 0], atol=1e-14)
    assert np.allclose(sig[:, 5], -w[:, 5], atol=1e-14)


def test_betti_reciprocity():
    """Reciprocity of the two operators (Betti): for one mode q, a pressure P at -q and an
    eigenstress w at +q satisfy  P u3[w](0) = int eps[M P](z) : w_h(z) dz,
    where the depth integral of the continuous Boussinesq strain against the
    piecewise-linear w_h is done exactly by Gauss-Legendre on every element."""
    Q = np.array([[12.0, -5.0]])
    z = np.array([0.0, 0.02, 0.05, 0.1, 0.16, 0.25])
    rng = np.random.default_rng(11)
    W6 = rng.standard_normal((z.size, 6)) + 1j * rng.standard_normal((z.size, 6))
    Wf = T.sym6_to_full(W6, axis=1)
    _, u0, _ = op.mindlin_modes(Wf[None], Q, z, E, NU)
    P = 0.8 + 0.1j
    xg, wg = np.polynomial.legendre.leggauss(30)
    total = 0.0
    for m in range(z.size - 1):
        h = z[m + 1] - z[m]
        y = z[m] + 0.5 * h * (xg + 1)
        H, _ = op.boussinesq_modes(np.array([P]), -Q, y, E, NU)
        eps_ = 0.5 * (H[0] + np.swapaxes(H[0], -1, -2))
        wl = ((z[m + 1] - y) / h)[:, None, None] * Wf[m] + ((y - z[m]) / h)[:, None, None] * Wf[m + 1]
        total += np.sum(0.5 * h * wg * np.einsum("pab,pab->p", eps_, wl))
    lhs = P * u0[0, 2]
    assert abs(lhs - total) < 1e-12 * abs(lhs)


@pytest.mark.slow
def test_mindlin_cheng_sphere():
    """Sec. 6.1: hydrostatic eigenstrain alpha T I in a ball of radius a centred at depth
    c = 2a; closed forms of Mindlin & Cheng for the surface displacement and the on-axis
    stresses outside the inclusion.  Grid 64 x 64 x 61 over ]-7.5a, 7.5a[^2 x [0, 5a]
    (coarser than the paper's 128 x 128 x 126); agreement within a few percent.

    The printed on-axis sigma_z, (6z + c)/(z + c)^4 - 2/|z - c|^3, is not zero at the
    free surface z = 0; the expression used here, (14z + 2c)/(z + c)^4 - 2/|z - c|^3, is
    the one derived in test_mindlin_cheng_on_axis_derivation from the traction-free
    nucleus solution, which reproduces the printed u_r, u_z and sigma_theta exactly."""
    a, c = 1.0, 2.0
    L = 15.0
    n = 64
    z = np.linspace(0.0, 5.0, 61)
    alphaT = 1e-3
    x = -L / 2 + np.arange(n) * L / n
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    inside = (X1[None] ** 2 + X2[None] ** 2 + (z[:, None, None] - c) ** 2) < a * a
    ep = np.zeros((z.size, 6, n, n))
    for k in range(3):
        ep[:, k] = alphaT * inside
    sig, u3 = op.mindlin_apply(ep, z, L, L, E, NU, "stress", with_surface=True)
    beta = alphaT * (1 + NU) / (1 - NU)
    i0 = n // 2
    # surface u_z along x2 = 0 relative to its value at the cell edge (mode 0 is dropped)
    r = np.abs(x)
    uz = -4 * a ** 3 / (3 * (r ** 2 + c * c) ** 1.5) * beta * (1 - NU) * c
    num = u3[i0] - u3[i0, 0]
    ref = uz - uz[0]
    centre = r < 3.0
    assert np.abs(num[centre] - ref[centre]).max() < 0.05 * np.abs(ref).max()
    # on-axis sigma_z outside the inclusion (Gibbs zone excluded)
    zz = z
    zz = np.where(np.abs(zz - c) < 1e-12, np.nan, zz)
    pref = 2 * MU * beta * a ** 3 / 3
    sz = pref * ((14 * zz + 2 * c) / (zz + c) ** 4 - 2 / np.abs(zz - c) ** 3)
    stheta = pref * ((4 * NU - 3) / (zz + c) ** 3 + 6 * c / (zz + c) ** 4 + 1 / np.abs(zz - c) ** 3)
    out = (z < 0.6) | (z > 3.5)
    ref_scale = 2 * pref / a ** 3
    assert np.abs(sig[out, 2, i0, i0] - sz[out]).max() < 0.05 * ref_scale
    # sigma_theta on the axis equals sigma_11 = sigma_22 there
    assert np.abs(sig[out, 0, i0, i0] - stheta[out]).max() < 0.05 * ref_scale


def test_return_map_consistency_and_flow():
    """Sec. 4.1: after a plastic step f_y(sigma_n+1) = sigma_y + E_h (e_p + de_p);
    tr d_eps_p = 0; de_p = sqrt(2/3) ||d_eps_p||; elastic steps have no flow."""
    rng = np.random.default_rng(4)
    n = 2000
    sig_n = rng.standard_normal((6, n)) * 0.02
    e_p = np.abs(rng.standard_normal(n)) * 0.01
    d_eps = rng.standard_normal((6, n)) * 0.05
    sy, Eh = 0.05, 0.1
    dep, dEp, sig_new = pl.return_map(d_eps, sig_n, e_p, E, NU, sy, Eh)
    plastic = dEp > 0
    assert plastic.sum() > 100 and (~plastic).sum() > 10
    fy = pl.von_mises(sig_new)
    assert np.allclose(fy[plastic], sy + Eh * (e_p[plastic] + dEp[plastic]), rtol=1e-13, atol=1e-15)
    assert np.allclose(dep[0] + dep[1] + dep[2], 0.0, atol=1e-16)
    assert np.allclose(dEp, np.sqrt(2 / 3) * T.norm6(dep, axis=0), rtol=1e-13, atol=1e-18)
    sig_tr = sig_n + T.hooke6(d_eps, LAM, MU, axis=0)
    assert np.all(pl.von_mises(sig_tr[:, ~plastic]) <= sy + Eh * e_p[~plastic] + 1e-15)
    assert np.all(dep[:, ~plastic] == 0.0)


def test_return_map_uniaxial_closed_form():
    """Uniaxial stress path (Sec. 4.1 with linear hardening): for a strain increment that
    keeps sigma_11 the only non-zero stress, de_p = (sigma_tr_eq - sigma_y)/(3 mu + E_h)
    with sigma_tr_eq = |sigma_11 trial| (von Mises of a uniaxial deviator)."""
    s11 = 0.2
    d_eps = np.zeros((6, 1))
    # strain that produces sigma = (s11, 0, 0, ...) elastically
    d_eps[0] = s11 / E
    d_eps[1] = d_eps[2] = -NU * s11 / E
    dep, dEp, sig_new = pl.return_map(d_eps, np.zeros((6, 1)), np.zeros(1), E, NU, 0.05, 0.1)
    assert abs(dEp[0] - (s11 - 0.05) / (3 * MU + 0.1)) < 1e-15
    assert abs(dep[0, 0] - dEp[0]) < 1e-15 and abs(dep[1, 0] + 0.5 * dEp[0]) < 1e-15


@pytest.mark.slow
def test_mindlin_cheng_on_axis_derivation():
    """Sec. 6.1 closed forms, re-derived: a centre of dilatation of strength C = beta a^3/3
    at depth c in the half-space, written as a Papkovich-Neuber field
        u = 4(1-nu) psi - grad(x.psi + chi), psi = (0, 0, k1 d_z(1/R2) + k2/R2),
        chi = C/R1 + k3/R2 + k4 c d_z(1/R2)
    (R1, R2 distances to the source and its mirror image), with k1..k4 fixed by the
    traction-free surface.  The result reproduces the printed u_r, u_z and sigma_theta,
    and gives the on-axis sigma_z used in test_mindlin_cheng_sphere."""
    sp = pytest.importorskip("sympy")
    x, y, z, c, nu, C, mu = sp.symbols("x y z c nu C mu", positive=True)
    k = sp.symbols("k1:5")
    R1 = sp.sqrt(x ** 2 + y ** 2 + (z - c) ** 2)
    R2 = sp.sqrt(x ** 2 + y ** 2 + (z + c) ** 2)
    psi3 = k[0] * sp.diff(1 / R2, z) + k[1] / R2
    chi = C / R1 + k[2] / R2 + k[3] * c * sp.diff(1 / R2, z)
    X = [x, y, z]
    phi = z * psi3 + chi
    u = [-sp.diff(phi, v) for v in X]
    u[2] += 4 * (1 - nu) * psi3
    lam = 2 * mu * nu / (1 - 2 * nu)
    eps = [[(sp.diff(u[i], X[j]) + sp.diff(u[j], X[i])) / 2 for j in range(3)] for i in range(3)]
    tr = eps[0][0] + eps[1][1] + eps[2][2]
    sig = [[lam * tr * (1 if i == j else 0) + 2 * mu * eps[i][j] for j in range(3)] for i in range(3)]
    eqs = []
    for (i, j) in ((0, 2), (2, 2)):
        e = sig[i][j].subs(z, 0)
        for xv in (sp.Rational(1, 3), sp.Rational(1, 2), 1, 2, 3):
            eqs.append(sp.simplify(e.subs({x: xv, y: 0, c: 1})))
    sol = sp.solve(eqs, list(k), dict=True)[0]
    uz0 = sp.simplify(u[2].subs(sol).subs(z, 0))
    ux0 = sp.simplify(u[0].subs(sol).subs(z, 0))
    assert sp.simplify(uz0 + 4 * C * (1 - nu) * c / (x ** 2 + y ** 2 + c ** 2) ** sp.Rational(3, 2)) == 0
    assert sp.simplify(ux0 - 4 * C * (1 - nu) * x / (x ** 2 + y ** 2 + c ** 2) ** sp.Rational(3, 2)) == 0
    zz = sp.Symbol("zz", positive=True)
    s33 = sig[2][2].subs(sol).subs({x: 0, y: 0})
    s11 = sig[0][0].subs(sol).subs({x: 0, y: 0})
    vals = {c: 2, nu: sp.Rational(3, 10), mu: sp.Rational(5, 13), C: 1}
    for zv in (sp.Rational(1, 4), sp.Rational(3, 2), sp.Rational(7, 2), 5):
        cv = 2
        s33v = float(s33.subs(vals).subs(z, zv)) / (2 * float(vals[mu]))
        s11v = float(s11.subs(vals).subs(z, zv)) / (2 * float(vals[mu]))
        zf = float(zv)
        e33 = (14 * zf + 2 * cv) / (zf + cv) ** 4 - 2 / abs(zf - cv) ** 3
        e11 = (4 * 0.3 - 3) / (zf + cv) ** 3 + 6 * cv / (zf + cv) ** 4 + 1 / abs(zf - cv) ** 3
        assert abs(s33v - e33) < 1e-12
        assert abs(s11v - e11) < 1e-12


# Real-space single-mode pins on a non-square cell (Sec. 3.1 periodic cell and DFT, Thm 1).
# The whole apply (DFT of the nodal values, mode grid, per-mode operator, inverse DFT and
# its 1/(N1 N2)) is driven with a field that holds one in-plane mode, and the real-space
# output is compared, node by node, with the independent Navier-ODE solve of that mode.
# N1 != N2 and L1 != L2, so pairing k1 with L2 (or k2 with L1), a wrong DFT normalisation,
# a missing conjugate mode or a transposed axis each change the result by O(1).
SM_GRID = dict(n1=8, n2=6, L1=1.3, L2=0.7)
SM_Z = np.array([0.0, 0.04, 0.1, 0.19, 0.3])
SM_MODES = [(1, 0), (0, 1), (2, -1)]


def _single_mode_case(k1, k2, seed):
    n1, n2, L1, L2 = SM_GRID["n1"], SM_GRID["n2"], SM_GRID["L1"], SM_GRID["L2"]
    q1, q2 = 2 * np.pi * k1 / L1, 2 * np.pi * k2 / L2
    x1 = np.arange(n1) * L1 / n1
    x2 = np.arange(n2) * L2 / n2
    phase = np.exp(1j * (q2 * x2[:, None] + q1 * x1[None, :]))   # [N2, N1]
    rng = np.random.default_rng(seed)
    c6 = (rng.standard_normal((SM_Z.size, 6)) + 1j * rng.standard_normal((SM_Z.size, 6))) * 1e-3
    eps_p = (c6[:, :, None, None] * phase[None, None]).real        # [Nz, 6, N2, N1]
    return q1, q2, phase, c6, eps_p


def _hooke6_c(e6):
    """lambda tr(e) I + 2 mu e on six stored components (last axis)."""
    w = 2 * MU * e6
    w[..., :3] += LAM * (e6[..., 0] + e6[..., 1] + e6[..., 2])[..., None]
    return w


def _grad_to_strain6(g):
    """sym(grad u) of [.., 3, 3] gradients as six stored components."""
    pairs = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    return np.stack([0.5 * (g[..., i, j] + g[..., j, i]) for i, j in pairs], axis=-1)


def _single_mode_mindlin_error(k1, k2, seed=11):
    n1, n2, L1, L2 = SM_GRID["n1"], SM_GRID["n2"], SM_GRID["L1"], SM_GRID["L2"]
    q1, q2, phase, c6, eps_p = _single_mode_case(k1, k2, seed)
    w6 = _hooke6_c(c6)
    g, u = ode.solve_mode(q1, q2, SM_Z, w6, LAM, MU)
    e6 = _grad_to_strain6(g)                                        # [Nz, 6]
    s6 = _hooke6_c(e6) - w6
    want_e = (e6[:, :, None, None] * phase[None, None]).real
    want_s = (s6[:, :, None, None] * phase[None, None]).real
    want_u3 = (u[0, 2] * phase).real
    got_e = op.mindlin_apply(eps_p, SM_Z, L1, L2, E, NU, "strain")
    got_s, got_u3 = op.mindlin_apply(eps_p, SM_Z, L1, L2, E, NU, "stress", with_surface=True)
    return (np.abs(got_e - want_e).max() / np.abs(want_e).max(),
            np.abs(got_s - want_s).max() / np.abs(want_s).max(),
            np.abs(got_u3 - want_u3).max() / np.abs(want_u3).max())


@pytest.mark.parametrize("k1,k2", SM_MODES)
def test_single_mode_real_space_mindlin_non_square_cell(k1, k2):
    """Sec. 3.1 (cell ]-L1/2, L1/2[ x ]-L2/2, L2/2[, modes q = 2 pi (k1/L1, k2/L2), DFT of
    the nodal values) with Thm 1: a one-mode plastic strain on an 8x6 grid of a 1.3 x 0.7
    cell gives, at every voxel, the strain, the stress sigma = C:eps - w and the surface u3
    of the Navier-ODE solution of that mode (App. B), to 1e-11."""
    err = _single_mode_mindlin_error(k1, k2)
    assert max(err) < 1e-11, err


@pytest.mark.parametrize("k1,k2", SM_MODES)
def test_single_mode_real_space_boussinesq_non_square_cell(k1, k2):
    """Eq. (M:conv) and Eq. (B:fourier) on the same non-square cell: a one-mode surface
    pressure gives the Navier-ODE strain at every node and the surface u3, to 1e-11."""
    n1, n2, L1, L2 = SM_GRID["n1"], SM_GRID["n2"], SM_GRID["L1"], SM_GRID["L2"]
    q1, q2 = 2 * np.pi * k1 / L1, 2 * np.pi * k2 / L2
    x1 = np.arange(n1) * L1 / n1
    x2 = np.arange(n2) * L2 / n2
    phase = np.exp(1j * (q2 * x2[:, None] + q1 * x1[None, :]))
    P = 0.4 - 0.9j
    p = (P * phase).real
    g, u = ode.solve_mode(q1, q2, SM_Z, np.zeros((SM_Z.size, 6)), LAM, MU, t_applied=[0, 0, P])
    e6 = _grad_to_strain6(g)
    want_e = (e6[:, :, None, None] * phase[None, None]).real
    want_u3 = (u[0, 2] * phase).real
    got_u3, got_e = op.boussinesq_apply(p, SM_Z, L1, L2, E, NU, "strain")
    assert np.abs(got_e - want_e).max() < 1e-11 * np.abs(want_e).max()
    assert np.abs(got_u3 - want_u3).max() < 1e-11 * np.abs(want_u3).max()


def test_planted_cell_length_swap_is_caught(monkeypatch):
    """A plausible mistake in the mode grid (k1 paired with L2 and k2 with L1) fails the
    real-space single-mode pin above by O(1) on every mode it changes."""
    orig = op.mode_grid
    monkeypatch.setattr(op, "mode_grid", lambda N1, N2, L1, L2: orig(N1, N2, L2, L1))
    op._MODE_CACHE.clear()
    try:
        for k1, k2 in SM_MODES:
            assert max(_single_mode_mindlin_error(k1, k2)) > 1e-2
    finally:
        op._MODE_CACHE.clear()


def test_planted_dft_normalisation_error_is_caught(monkeypatch):
    """A plausible mistake in the DFT assembly (the inverse transform's 1/(N1 N2) dropped,
    or applied twice) fails the real-space single-mode pin."""
    ifft2 = np.fft.ifft2
    n = SM_GRID["n1"] * SM_GRID["n2"]
    for f in (n, 1.0 / n):
        monkeypatch.setattr(op.np.fft, "ifft2", lambda a, *args, _f=f, **kw: ifft2(a, *args, **kw) * _f)
        try:
            assert max(_single_mode_mindlin_error(1, 0)) > 1e-2
        finally:
            monkeypatch.undo()
