"""Discretised Mindlin and Boussinesq operators (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Method (the paper's, in its order; no blocking, fusion or cutoff):

1. Eigenstress w = C:eps_p per voxel (Sec. 4.2: the operator is applied to C:eps_p).
2. DFT of the nodal values of every layer, w_j(k) = DFT[w|X] (Eq. dft), unnormalised,
   with numpy's FFT as the library DFT.
3. For every mode k in Z^2_N (strict inequalities, Sec. 3.1: Nyquist modes excluded)
   and q = 2 pi (k1/L1, k2/L2), the displacement gradient at every depth node x3^i is
   the depth integral of the Fourier-space kernel against the piecewise-linear
   interpolant w_h(k, y3) = sum_j w_j(k) phi_j(y3) (Eq. full_discrete_convolution with
   Lagrange elements of degree 1).  Every element integral of the simpler form
   int g_n(q(y3 - x3^i)) phi_j(y3) dy3 (Eq. typical_integral) is computed by dense
   32-point Gauss-Legendre quadrature, for all N3 x N3 pairs (no cutoff).
   * Kelvin part: Eq. (2gradient), with the kernel evaluated at -q (Lemma 1, Thm 1),
     regular part from the second-order tensors of Eq. (recurrence), plus the jump
     term of Eq. (jump).
   * Image part (Eq. mindlin_B_U): the full-space field of the eigenstress leaves the
     traction T_inf = sigma_inf(0+) . n on the surface; the Boussinesq-Cerruti field
     of the cancelling traction -T_inf is added, evaluated at the field depth.
   * Mode k = 0: horizontally uniform (laminate) solution of the periodic half-space.
   * Nyquist modes: no operator contribution (they are not in Z^2_N).
4. sigma = C:grad^sym N[w] - w (Sec. 6.1), or the strain grad^sym N[w]; inverse DFT.

Readings of the paper where it is silent or garbled:
* no 1/(4 pi^2) factor in front of the Fourier series (Thm 1 / App. B garble);
* every Delta of the Kelvin kernel is taken at -q, the Boussinesq kernel of the image
  term at +q (the standard convolution of a surface traction with B);
* the image term is the superposition N[w] = N_inf[w] + M[-T_inf] (Eq. mindlin_B_U);
* linear elements; w_h = 0 below the last node; the jump term uses the nodal w_i,
  also at the first and last nodes (limits taken from inside the layer);
* k = 0: sigma_i3 = 0, eps_ab = 0, eps_a3 = w_a3/(2 mu), eps_33 = w_33/(lambda+2 mu);
  the surface displacement of mode 0 is set to 0 (Rem. fundamental_mode);
* Nyquist modes: grad N[w] = 0, so sigma = -w there.

Parity: every mode is pinned against an independent solve of the Navier ODE with the
traction-free condition (tests/test_oracle_pins.py::test_mindlin_matches_navier_ode),
the free-surface and equilibrium conditions, brute-force translation invariance and
linearity, Betti reciprocity against the Boussinesq operator, and the Mindlin-Cheng
closed forms of Sec. 6.1.
"""
import numpy as np

from . import kernels as K
from .tensors import lame, hooke_full, sym_part, sym6_to_full, full_to_sym6, hooke6

GL_POINTS = 32
_MAX_QH = 25.0  # 32-point Gauss-Legendre is exact to round-off for q*h up to this


def mode_grid(N1, N2, L1, L2):
    """Signed integer modes (numpy FFT order) and the wavevectors q = 2 pi k / L."""
    k1 = np.fft.fftfreq(N1, 1.0 / N1)
    k2 = np.fft.fftfreq(N2, 1.0 / N2)
    K2, K1 = np.meshgrid(k2, k1, indexing="ij")
    Q1 = 2.0 * np.pi * K1 / L1
    Q2 = 2.0 * np.pi * K2 / L2
    nyq = np.zeros_like(K1, dtype=bool)
    if N1 % 2 == 0:
        nyq |= np.abs(K1) == N1 // 2
    if N2 % 2 == 0:
        nyq |= np.abs(K2) == N2 // 2
    zero = (K1 == 0) & (K2 == 0)
    return Q1, Q2, nyq, zero


def depth_weights(q, z):
    """Element-integral weights of the piecewise-linear interpolant (Sec. 3.2).

    Returns dict (n, sign) -> Lambda [K, Nz, Nz] with
        Lambda[k, i, j] = sum over elements E_m on the ``sign`` side of x3^i of
                          int_{E_m} g_n^sign(q_k (y - z_i)) phi_j(y) dy,
    the - branch for elements above the node (y < z_i), + for elements below.
    Computed with 32-point Gauss-Legendre on every element.
    """
    q = np.asarray(q, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    Nz = z.size
    xg, wg = np.polynomial.legendre.leggauss(GL_POINTS)
    h = np.diff(z)
    if h.size and float(np.max(q)) * float(np.max(h)) > _MAX_QH:
        raise ValueError("q*h beyond the range where the oracle quadrature is exact")
    zc = 0.5 * (z[:-1] + z[1:])
    e = 0.5 * h
    y = zc[:, None] + e[:, None] * xg[None, :]          # [E, P]
    wq = e[:, None] * wg[None, :]                         # [E, P]
    phiL = (z[1:, None] - y) / h[:, None]
    phiR = (y - z[:-1, None]) / h[:, None]
    above = z[None, 1:] <= z[:, None]                     # [Nz(i), E(m)]: element above node i
    below = z[None, :-1] >= z[:, None]
    out = {}
    t = q[:, None, None, None] * (y[None, None, :, :] - z[None, :, None, None])  # [K, Nz, E, P]
    for sign, mask in ((-1, above), (+1, below)):
        ts = np.where(mask[None, :, :, None], t, 0.0)
        base = K.g0(ts, sign) * wq[None, None]
        for n in (0, 1):
            G = base if n == 0 else ts * base
            AL = np.einsum("kimp,mp->kim", G, phiL) * mask[None]
            AR = np.einsum("kimp,mp->kim", G, phiR) * mask[None]
            Lam = np.zeros((q.size, Nz, Nz))
            Lam[:, :, :-1] += AL
            Lam[:, :, 1:] += AR
            out[(n, sign)] = Lam
    return out


def _chunks(Kn, Nz):
    per = max(1, int(8.0e7 // max(1, Nz * max(Nz - 1, 1) * GL_POINTS * 8)))
    return [slice(s, min(Kn, s + per)) for s in range(0, Kn, per)]


_MODE_CACHE = {}


def _mode_data(Q, z, mu, nu):
    """Kelvin tensors at -q (Lemma 1), depth weights and Boussinesq tensors at +q for a
    batch of modes; memoised per (modes, nodes, material) since repeated applies on one
    grid (the solvers) use the same values."""
    key = (Q.tobytes(), np.asarray(z, dtype=np.float64).tobytes(), float(mu), float(nu))
    hit = _MODE_CACHE.get(key)
    if hit is None:
        q = np.hypot(Q[:, 0], Q[:, 1])
        hit = (K.kelvin_gradient_tensors(-Q, mu, nu), depth_weights(q, z), K.boussinesq_gradient_tensors(Q, mu, nu))
        if len(_MODE_CACHE) > 64:
            _MODE_CACHE.clear()
        _MODE_CACHE[key] = hit
    return hit


def mindlin_modes(W, Q, z, E, nu):
    """Mindlin operator for a batch of non-zero modes.

    W: [K, Nz, 3, 3] complex nodal Fourier coefficients w_j(k) of the eigenstress.
    Q: [K, 2] wavevectors q = 2 pi kbar (all |q| > 0).
    Returns (H, u0, t):
      H  [K, Nz, 3, 3]  displacement gradient grad N[w](k, x3^i)  ((H)_am = d_m u_a)
      u0 [K, 3]         surface displacement N[w](k, 0)
      t  [K, 3]         traction sigma_inf(0+) . e3 cancelled by the image term
    """
    lam, mu = lame(E, nu)
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    W = np.asarray(W, dtype=np.complex128)
    q = np.hypot(Q[:, 0], Q[:, 1])
    kel, Lw, bou = _mode_data(Q, z, mu, nu)
    M = {key: np.einsum("kij,kjab->kiab", Lw[key], W, optimize=True) for key in Lw}
    # Eq. (2gradient): - int grad^2 U(-q, y3 - x3) : w(y3) dy3, both branches
    G = np.zeros(W.shape, dtype=np.complex128)
    for s in (-1, +1):
        U02, U12 = kel[(2, s)]
        G -= q[:, None, None, None] * (
            np.einsum("kabcd,kibc->kiad", U02, M[(0, s)], optimize=True)
            + np.einsum("kabcd,kibc->kiad", U12, M[(1, s)], optimize=True)
        )
    # jump term of Eq. (jump): - ([[grad U]] : w(x3)) x e3, [[grad U]] = U01^+ - U01^-
    J = kel[(1, +1)][0] - kel[(1, -1)][0]
    G[..., :, 2] -= np.einsum("kabc,kibc->kia", J, W)
    # full-space displacement at the surface (only the + branch: all sources below)
    U01p, U11p = kel[(1, +1)]
    uinf0 = np.einsum("kabc,kbc->ka", U01p, M[(0, +1)][:, 0]) + np.einsum("kabc,kbc->ka", U11p, M[(1, +1)][:, 0])
    # image term (Eq. mindlin_B_U): cancel the surface traction of the full-space field
    sig0 = hooke_full(sym_part(G[:, 0]), lam, mu) - W[:, 0]
    t = sig0[:, :, 2]                                    # applied traction -T_inf = sigma . e3
    B00, B10 = bou[0]
    B01, B11 = bou[1]
    zq = q[:, None] * np.asarray(z)[None, :]             # [K, Nz]
    Pg = np.einsum("kf,kfam->kam", t, B01)
    Qg = np.einsum("kf,kfam->kam", t, B11)
    H = G + np.exp(-zq)[..., None, None] * (Pg[:, None] + zq[..., None, None] * Qg[:, None])
    u0 = uinf0 + np.einsum("kf,kfa->ka", t, B00) / q[:, None]
    return H, u0, t


def laminate_mindlin(W0, E, nu):
    """Mode k = 0 of the Mindlin operator: grad u of the horizontally uniform solution.

    sigma_i3 = 0 through the depth (equilibrium + free surface), eps_ab = 0 (periodic),
    so eps_a3 = w_a3 / (2 mu) and eps_33 = w_33 / (lambda + 2 mu).  W0: [Nz, 3, 3].
    Returned as a symmetric displacement-gradient-like tensor (only its sym part is used).
    """
    lam, mu = lame(E, nu)
    H = np.zeros_like(W0, dtype=np.complex128)
    H[:, 0, 2] = H[:, 2, 0] = W0[:, 0, 2] / (2.0 * mu)
    H[:, 1, 2] = H[:, 2, 1] = W0[:, 1, 2] / (2.0 * mu)
    H[:, 2, 2] = W0[:, 2, 2] / (lam + 2.0 * mu)
    return H


def mindlin_apply(eps_p, z, L1, L2, E, nu, out_kind="stress", with_surface=False):
    """Apply the discretised Mindlin operator to a plastic strain field.

    eps_p: [Nz, 6, N2, N1] real (x1 fastest).  Returns out [Nz, 6, N2, N1]:
    sigma = C:grad^sym N[C:eps_p] - C:eps_p ("stress") or grad^sym N[C:eps_p]
    ("strain"); with_surface=True also returns the surface displacement u3 [N2, N1].
    """
    lam, mu = lame(E, nu)
    eps_p = np.asarray(eps_p, dtype=np.float64)
    Nz, _, N2, N1 = eps_p.shape
    w = hooke6(eps_p, lam, mu, axis=1)                               # step 1
    w_hat = np.fft.fft2(w, axes=(-2, -1))                             # step 2
    W = np.moveaxis(sym6_to_full(w_hat, axis=1), 0, -3)               # [N2, N1, Nz, 3, 3]
    Q1, Q2, nyq, zero = mode_grid(N1, N2, L1, L2)
    H = np.zeros_like(W)
    u0 = np.zeros((N2, N1, 3), dtype=np.complex128)
    sel = ~(nyq | zero)
    idx = np.argwhere(sel)
    Wk = W[sel]
    Qk = np.stack([Q1[sel], Q2[sel]], axis=1)
    Hk = np.empty_like(Wk)
    uk = np.empty((Wk.shape[0], 3), dtype=np.complex128)
    for sl in _chunks(Wk.shape[0], Nz):                               # step 3 (k != 0)
        Hk[sl], uk[sl], _ = mindlin_modes(Wk[sl], Qk[sl], z, E, nu)
    H[idx[:, 0], idx[:, 1]] = Hk
    u0[idx[:, 0], idx[:, 1]] = uk
    H[0, 0] = laminate_mindlin(W[0, 0], E, nu)                        # k = 0
    eps_hat = sym_part(H)                                             # Nyquist stays 0
    if out_kind == "stress":
        out_hat = hooke_full(eps_hat, lam, mu) - W                    # step 4
    elif out_kind == "strain":
        out_hat = eps_hat
    else:
        raise ValueError(out_kind)
    out6 = full_to_sym6(np.moveaxis(out_hat, -3, 0), axis=1)          # [Nz, 6, N2, N1]
    out = np.fft.ifft2(out6, axes=(-2, -1))
    if not with_surface:
        return out.real
    u3 = np.fft.ifft2(u0[..., 2]).real
    return out.real, u3


def boussinesq_modes(P, Q, z, E, nu):
    """Boussinesq operator for a batch of non-zero modes of a normal surface pressure.

    P: [K] complex pressure coefficients (force p e3 per unit area pushing into the body,
    sigma . e3 = -p e3 on the surface).  Returns (H [K, Nz, 3, 3], u0 [K, 3]).
    """
    lam, mu = lame(E, nu)
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    q = np.hypot(Q[:, 0], Q[:, 1])
    bou = K.boussinesq_gradient_tensors(Q, mu, nu)
    B00, B10 = bou[0]
    B01, B11 = bou[1]
    t = np.zeros((Q.shape[0], 3), dtype=np.complex128)
    t[:, 2] = P
    zq = q[:, None] * np.asarray(z)[None, :]
    Pg = np.einsum("kf,kfam->kam", t, B01)
    Qg = np.einsum("kf,kfam->kam", t, B11)
    H = np.exp(-zq)[..., None, None] * (Pg[:, None] + zq[..., None, None] * Qg[:, None])
    u0 = np.einsum("kf,kfa->ka", t, B00) / q[:, None]
    return H, u0


def boussinesq_apply(p, z, L1, L2, E, nu, out_kind="stress"):
    """Apply the discretised Boussinesq operator to a surface pressure p [N2, N1].

    Returns (u3 [N2, N1], vol [Nz, 6, N2, N1]): the surface normal displacement
    M[p].e3 (mode 0 set to 0, Rem. fundamental_mode) and sigma = C:grad^sym M[p]
    ("stress") or grad^sym M[p] ("strain") at every node.
    Mode 0 (uniform pressure pbar): eps_33 = -pbar/(lambda+2mu), all other strains 0.
    """
    lam, mu = lame(E, nu)
    p = np.asarray(p, dtype=np.float64)
    N2, N1 = p.shape
    Nz = len(z)
    p_hat = np.fft.fft2(p)
    Q1, Q2, nyq, zero = mode_grid(N1, N2, L1, L2)
    sel = ~(nyq | zero)
    H = np.zeros((N2, N1, Nz, 3, 3), dtype=np.complex128)
    u0 = np.zeros((N2, N1, 3), dtype=np.complex128)
    Qk = np.stack([Q1[sel], Q2[sel]], axis=1)
    Hk, uk = boussinesq_modes(p_hat[sel], Qk, z, E, nu)
    H[sel] = Hk
    u0[sel] = uk
    H[0, 0, :, 2, 2] = -p_hat[0, 0] / (lam + 2.0 * mu)
    eps_hat = sym_part(H)
    out_hat = hooke_full(eps_hat, lam, mu) if out_kind == "stress" else eps_hat
    out6 = full_to_sym6(np.moveaxis(out_hat, -3, 0), axis=1)
    vol = np.fft.ifft2(out6, axes=(-2, -1)).real
    u3 = np.fft.ifft2(u0[..., 2]).real
    return u3, vol


def surface_compliance(N1, N2, L1, L2, E, nu):
    """Fourier multiplier of the surface normal displacement under normal pressure:
    u3_hat = 2 p_hat / (E* q) (B33(q, 0), Eq. B:fourier), 0 at k = 0 and Nyquist."""
    Q1, Q2, nyq, zero = mode_grid(N1, N2, L1, L2)
    Qk = np.stack([Q1.ravel(), Q2.ravel()], axis=1)
    keep = ~(nyq | zero).ravel()
    lam, mu = lame(E, nu)
    kern = np.zeros(N1 * N2)
    B00, _ = K.boussinesq_coefficients(Qk[keep], mu, nu)
    q = np.hypot(Qk[keep, 0], Qk[keep, 1])
    kern[keep] = (B00[:, 2, 2] / q).real
    return kern.reshape(N2, N1)
