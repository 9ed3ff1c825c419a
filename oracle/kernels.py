"""Fundamental solutions in partial Fourier space (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Everything here is a direct transcription of Sec. 2.2 of the paper:

* Delta(q) = (i q1/q, i q2/q, 0), Delta^{+-} = e3 -+ Delta, b = 4(1 - nu)  (Table 1)
* Kelvin:  U00^{+-} = (b I + Delta x Delta - e3 x e3) / (2 mu b),
           U10^{-}  = -(Delta^- x Delta^-) / (2 mu b),
           U10^{+}  = +(Delta^+ x Delta^+) / (2 mu b)                      (Table 1)
  U_infty^{+-}(q, x3, y3) = [U00 g0^{+-}(q(y3-x3)) + U10 g1^{+-}(q(y3-x3))] / q
                                                        (Eq. full_space_solution)
* Boussinesq-Cerruti: B00 = (2 I + (1-2nu) Delta^+ x Delta^- + Delta x Delta - e3 x e3)/(2 mu),
  B10 = Delta^+ x Delta^+ / (2 mu), B(q, y3) = [B00 g0^+(q y3) + B10 g1^+(q y3)] / q
                                                        (Eq. B:fourier, Eq. B:1_0)
* gradient recurrence, derivative index appended last (Eq. recurrence):
  U0n = -+ U0(n-1) x Delta^{+-} + U1(n-1) x e3,   U1n = -+ U1(n-1) x Delta^{+-},
  and the n-th gradient carries the factor q^(n-1).
* g0^{+-}(z) = exp(-+ z), g1^{+-}(z) = z exp(-+ z)                         (Table 1)

Tensor index convention: U = e_k x U^k, so U[..., k, i] is component i of the
displacement created by a force along e_k; gradients append indices to the right
((grad u)_ij = d_j u_i, Sec. 1).

All functions are vectorised over a leading batch of wavevectors Q (shape [K, 2],
all |Q| > 0).  The caller chooses whether a kernel is evaluated at +q or -q.
Parity: pinned in tests/test_oracle_pins.py (Navier ODE in y3 for every column,
Kelvin continuity and jump, Boussinesq traction condition and the 2/(E* q)
surface compliance, jump formula Eq. jump).
"""
import numpy as np

E3 = np.array([0.0, 0.0, 1.0])


def delta_vectors(Q):
    """Delta(Q), Delta^+(Q), Delta^-(Q) for a batch of wavevectors Q [K, 2] (Table 1)."""
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    q = np.hypot(Q[:, 0], Q[:, 1])
    D = np.zeros((Q.shape[0], 3), dtype=np.complex128)
    D[:, 0] = 1j * Q[:, 0] / q
    D[:, 1] = 1j * Q[:, 1] / q
    Dp = E3[None, :] - D
    Dm = E3[None, :] + D
    return q, D, Dp, Dm


def _outer(a, b):
    return a[..., :, None] * b[..., None, :]


def kelvin_coefficients(Q, mu, nu):
    """Return (U00, U10p, U10m), each [K, 3, 3] complex (Table 1)."""
    q, D, Dp, Dm = delta_vectors(Q)
    b = 4.0 * (1.0 - nu)
    I = np.eye(3)[None]
    U00 = (b * I + _outer(D, D) - _outer(E3, E3)[None]) / (2.0 * mu * b)
    U10p = _outer(Dp, Dp) / (2.0 * mu * b)
    U10m = -_outer(Dm, Dm) / (2.0 * mu * b)
    return U00, U10p, U10m


def boussinesq_coefficients(Q, mu, nu):
    """Return (B00, B10), each [K, 3, 3] complex (Eq. B:fourier, Eq. B:1_0)."""
    q, D, Dp, Dm = delta_vectors(Q)
    I = np.eye(3)[None]
    B00 = (2.0 * I + (1.0 - 2.0 * nu) * _outer(Dp, Dm) + _outer(D, D) - _outer(E3, E3)[None]) / (2.0 * mu)
    B10 = _outer(Dp, Dp) / (2.0 * mu)
    return B00, B10


def recurrence_step(U0, U1, sign, Q):
    """One step of Eq. (recurrence) for branch ``sign`` (+1 or -1).

    U0, U1: [K, 3, ...] tensors of order n-1; returns the order-n pair with the
    new derivative index appended last:
        U0n = -sign * U0 x Delta^sign + U1 x e3,   U1n = -sign * U1 x Delta^sign.
    """
    q, D, Dp, Dm = delta_vectors(Q)
    Ds = Dp if sign > 0 else Dm
    shape = (U0.shape[0],) + (1,) * (U0.ndim - 1) + (3,)
    Ds_b = Ds.reshape(shape)
    e3_b = E3.reshape((1,) * U0.ndim + (3,))
    U0n = -sign * U0[..., None] * Ds_b + U1[..., None] * e3_b
    U1n = -sign * U1[..., None] * Ds_b
    return U0n, U1n


def g0(z, sign):
    """g0^{sign}(z) = exp(-sign z) (Table 1)."""
    return np.exp(-sign * z)


def g1(z, sign):
    """g1^{sign}(z) = z exp(-sign z) (Table 1)."""
    return z * np.exp(-sign * z)


def kelvin_gradient_tensors(Q, mu, nu):
    """Kelvin tensors of orders 0, 1, 2 for both branches.

    Returns dict with keys (n, sign) -> (U0n, U1n); U0n/U1n have n+2 tensor indices.
    The n-th gradient of U_infty^{sign} is q^(n-1) [U0n g0 + U1n g1].
    """
    U00, U10p, U10m = kelvin_coefficients(Q, mu, nu)
    out = {(0, +1): (U00, U10p), (0, -1): (U00, U10m)}
    for s in (+1, -1):
        a, b = out[(0, s)]
        for n in (1, 2):
            a, b = recurrence_step(a, b, s, Q)
            out[(n, s)] = (a, b)
    return out


def boussinesq_gradient_tensors(Q, mu, nu):
    """Boussinesq tensors of orders 0 and 1 (+ branch only: decay as y3 -> infinity).

    The n-th gradient of B is q^(n-1) [B0n g0^+ + B1n g1^+].
    """
    B00, B10 = boussinesq_coefficients(Q, mu, nu)
    B01, B11 = recurrence_step(B00, B10, +1, Q)
    return {0: (B00, B10), 1: (B01, B11)}


def kelvin_displacement(Q, mu, nu, t):
    """Kelvin displacement U_infty(Q, x3, y3) for t = y3 - x3 (scalar or [K]); [K,3,3]."""
    q = np.hypot(np.atleast_2d(Q)[:, 0], np.atleast_2d(Q)[:, 1])
    U00, U10p, U10m = kelvin_coefficients(Q, mu, nu)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), q.shape)
    s = np.where(t >= 0, 1.0, -1.0)
    U10 = np.where((s > 0)[:, None, None], U10p, U10m)
    z = q * t
    return (U00 * g0(z, s)[:, None, None] + U10 * g1(z, s)[:, None, None]) / q[:, None, None]


def boussinesq_displacement(Q, mu, nu, y3):
    """Boussinesq-Cerruti displacement B(Q, y3) [K,3,3] (Eq. B:fourier)."""
    q = np.hypot(np.atleast_2d(Q)[:, 0], np.atleast_2d(Q)[:, 1])
    B00, B10 = boussinesq_coefficients(Q, mu, nu)
    z = q * np.broadcast_to(np.asarray(y3, dtype=np.float64), q.shape)
    return (B00 * g0(z, 1)[:, None, None] + B10 * g1(z, 1)[:, None, None]) / q[:, None, None]
