"""Symmetric second-order tensors and isotropic elasticity (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Storage convention (shared by the whole project as an *interface*, not as code):
six TENSOR components in the order (11, 22, 33, 23, 13, 12); shears are tensor
shears eps_ij, not engineering gamma = 2 eps_ij.

Elasticity: Sec. 1, Eq. (sigma) sigma = C:(eps - eps_p); isotropic C with the
Lame constants lambda, mu; c = (lambda+mu)/mu = 1/(1-2 nu) (Sec. 2.2).
Parity: pinned by the closed forms in tests/test_oracle_pins.py (Hooke round trip,
deviator trace, Lame relations).
"""
import numpy as np

# (i, j) index pairs of the six stored components
SYM_IJ = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def lame(E, nu):
    """Lame constants (lambda, mu) of an isotropic solid from E and nu."""
    mu = E / (2.0 * (1.0 + nu))
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    return lam, mu


def e_star(E, nu):
    """Hertz modulus E* = E / (1 - nu^2) (Sec. 6.2)."""
    return E / (1.0 - nu * nu)


def sym6_to_full(a6, axis=0):
    """Six stored components along ``axis`` -> full 3x3 tensor in the last two axes."""
    a6 = np.moveaxis(np.asarray(a6), axis, -1)
    out = np.empty(a6.shape[:-1] + (3, 3), dtype=a6.dtype)
    for c, (i, j) in enumerate(SYM_IJ):
        out[..., i, j] = a6[..., c]
        out[..., j, i] = a6[..., c]
    return out


def full_to_sym6(a, axis=0):
    """Full 3x3 tensor (last two axes) -> six stored components placed at ``axis``."""
    a = np.asarray(a)
    out = np.stack([0.5 * (a[..., i, j] + a[..., j, i]) for (i, j) in SYM_IJ], axis=-1)
    return np.moveaxis(out, -1, axis)


def hooke_full(eps, lam, mu):
    """C:eps = lambda tr(eps) I + 2 mu eps for full tensors in the last two axes."""
    tr = np.trace(eps, axis1=-2, axis2=-1)
    return lam * tr[..., None, None] * np.eye(3) + 2.0 * mu * eps


def hooke6(eps6, lam, mu, axis=0):
    """C:eps in six-component storage (components along ``axis``)."""
    e = np.moveaxis(np.asarray(eps6), axis, 0)
    tr = e[0] + e[1] + e[2]
    out = 2.0 * mu * e
    out[0:3] = out[0:3] + lam * tr
    return np.moveaxis(out, 0, axis)


def sym_part(a):
    """Symmetric part of a full tensor (last two axes)."""
    return 0.5 * (a + np.swapaxes(a, -1, -2))


def deviator6(s6, axis=0):
    """s = sigma - tr(sigma)/3 I in six-component storage."""
    s = np.array(np.moveaxis(np.asarray(s6), axis, 0), dtype=np.float64, copy=True)
    m = (s[0] + s[1] + s[2]) / 3.0
    s[0:3] -= m
    return np.moveaxis(s, 0, axis)


def norm6(a6, axis=0):
    """Frobenius norm ||a|| = sqrt(a:a); the three shears count twice."""
    a = np.moveaxis(np.asarray(a6), axis, 0)
    return np.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2 + 2.0 * (a[3] ** 2 + a[4] ** 2 + a[5] ** 2))


def ddot6(a6, b6, axis=0):
    """a:b with the three shears counted twice."""
    a = np.moveaxis(np.asarray(a6), axis, 0)
    b = np.moveaxis(np.asarray(b6), axis, 0)
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + 2.0 * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5])
