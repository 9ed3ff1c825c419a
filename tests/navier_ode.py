"""Independent per-mode solver of the half-space eigenstress problem (test helper).

Used to pin the oracle's Mindlin and Boussinesq operators against the PDE itself,
without any of the paper's fundamental solutions.  For one in-plane Fourier mode
exp(i q.x) the problem of App. B, Eq. (eigenstress:ODE) reads, with the traction
vector tau = sigma . e3 = (sigma_13, sigma_23, sigma_33) and sigma = C:eps - w:

    div sigma = 0            for z > 0,
    tau(0)    = -t_applied   (0 for the Mindlin problem, p e3 for a pressure p),
    u -> 0                   as z -> infinity.

Written as the first-order system X' = A X + F w(z) in X = (u, tau), with the
eigenstress w piecewise linear between the depth nodes and zero below the last one.
Each element is integrated exactly with the matrix exponential of an augmented
system; the nodal states are coupled by multiple shooting (well conditioned for
any q*h the tests use); the radiation condition at the last node keeps X in the
decaying generalised eigenspace ker((A + qI)^2).
"""
import numpy as np
import scipy.linalg as sla

SYM_IJ = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def _rhs(q1, q2, lam, mu, X, w):
    """d/dz of X = (u, tau) for the mode exp(i(q1 x1 + q2 x2)); w is a full 3x3 tensor."""
    iq = np.array([1j * q1, 1j * q2])
    u = X[:3]
    tau = X[3:]
    du = np.zeros(3, dtype=np.complex128)
    # tau_a = mu (i q_a u3 + u_a') - w_a3 ; tau_3 = lam tr eps + 2 mu u3' - w_33
    du[0] = (tau[0] + w[0, 2]) / mu - iq[0] * u[2]
    du[1] = (tau[1] + w[1, 2]) / mu - iq[1] * u[2]
    du[2] = (tau[2] + w[2, 2] - lam * (iq[0] * u[0] + iq[1] * u[1])) / (lam + 2 * mu)
    tr = iq[0] * u[0] + iq[1] * u[1] + du[2]
    dtau = np.zeros(3, dtype=np.complex128)
    for b in range(2):
        s = 0.0
        for a in range(2):
            sig_ba = (lam * tr if a == b else 0.0) + mu * (iq[a] * u[b] + iq[b] * u[a]) - w[b, a]
            s = s + iq[a] * sig_ba
        dtau[b] = -s
    dtau[2] = -(iq[0] * tau[0] + iq[1] * tau[1])
    return np.concatenate([du, dtau])


def _system(q1, q2, lam, mu):
    A = np.zeros((6, 6), dtype=np.complex128)
    F = np.zeros((6, 6), dtype=np.complex128)
    for c in range(6):
        e = np.zeros(6, dtype=np.complex128)
        e[c] = 1.0
        A[:, c] = _rhs(q1, q2, lam, mu, e, np.zeros((3, 3)))
        w = np.zeros((3, 3), dtype=np.complex128)
        i, j = SYM_IJ[c]
        w[i, j] = w[j, i] = 1.0
        F[:, c] = _rhs(q1, q2, lam, mu, np.zeros(6), w)
    return A, F


def _full(w6):
    w = np.zeros((3, 3), dtype=np.complex128)
    for c, (i, j) in enumerate(SYM_IJ):
        w[i, j] = w[j, i] = w6[c]
    return w


def solve_mode(q1, q2, z, w6_nodes, lam, mu, t_applied=None):
    """Nodal displacement gradients of one mode.

    w6_nodes: [Nz, 6] complex eigenstress Fourier coefficients at the nodes z.
    t_applied: applied surface traction (force on the body per unit area), or None.
    Returns (grad [Nz, 3, 3] with grad[a, m] = d_m u_a, u [Nz, 3]).
    """
    z = np.asarray(z, dtype=np.float64)
    Nz = z.size
    q = np.hypot(q1, q2)
    A, F = _system(q1, q2, lam, mu)
    n = 6 * Nz
    Mat = np.zeros((n, n), dtype=np.complex128)
    rhs = np.zeros(n, dtype=np.complex128)
    row = 0
    Z6 = np.zeros((6, 6))
    for m in range(Nz - 1):
        h = z[m + 1] - z[m]
        Aug = np.block([[A, F, Z6], [Z6, Z6, np.eye(6)], [Z6, Z6, Z6]])
        E = sla.expm(Aug * h)
        Phi = E[:6, :6]
        s = (w6_nodes[m + 1] - w6_nodes[m]) / h
        part = E[:6, 6:12] @ w6_nodes[m] + E[:6, 12:18] @ s
        # X_{m+1} - Phi X_m = part
        Mat[row:row + 6, 6 * (m + 1):6 * (m + 2)] = np.eye(6)
        Mat[row:row + 6, 6 * m:6 * m + 6] = -Phi
        rhs[row:row + 6] = part
        row += 6
    # traction at the surface: sigma . n = t_applied with n = -e3  =>  tau(0) = -t_applied
    Mat[row:row + 3, 3:6] = np.eye(3)
    if t_applied is not None:
        rhs[row:row + 3] = -np.asarray(t_applied)
    row += 3
    # below the last node w = 0 and the state must decay: (A + q I)^2 X = 0 there.
    # The eigenstress jumps to zero at the last node, tau stays continuous.
    Pd = (A + q * np.eye(6)) @ (A + q * np.eye(6))
    U, S, Vh = np.linalg.svd(Pd)
    C = U[:, :3].conj().T @ Pd
    Mat[row:row + 3, 6 * (Nz - 1):6 * Nz] = C
    row += 3
    X = np.linalg.solve(Mat, rhs).reshape(Nz, 6)
    grad = np.zeros((Nz, 3, 3), dtype=np.complex128)
    for i in range(Nz):
        d = _rhs(q1, q2, lam, mu, X[i], _full(w6_nodes[i]))
        u = X[i, :3]
        grad[i, :, 0] = 1j * q1 * u
        grad[i, :, 1] = 1j * q2 * u
        grad[i, :, 2] = d[:3]
    return grad, X[:, :3]
