"""J2 plasticity with linear isotropic hardening (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.1 of the paper: von Mises yield function f_y(sigma) = sqrt(3/2) ||s||, s the
deviator; cumulated plastic strain e_p = sqrt(2/3) int ||d eps_p||; plasticity
conditions f_y - f_h <= 0, (f_y - f_h) de_p = 0; associated flow
d eps_p = 3 de_p / (2 f_y) s; linear hardening f_h(e_p) = sigma_y + E_h e_p.

return_map: the backward-Euler (radial return) increment for one strain increment,
in closed form for linear hardening (no iteration):
    sigma_tr = sigma_n + C:d_eps,  f = f_y(sigma_tr) - f_h(e_p)
    f <= 0: d_eps_p = 0, de_p = 0
    f  > 0: de_p = f / (3 mu + E_h),  d_eps_p = 3/2 de_p s_tr / f_y(sigma_tr)
The state S_n of Sec. 4.2 lists (e_p, eps_p); the trial stress needs sigma_n too, so
the state carried here is (sigma_n, e_p) (reading: the paper is silent).
Parity: pinned by consistency (f_y(sigma_n+1) = f_h(e_p + de_p) when plastic),
elastic unloading, plastic incompressibility, de_p = sqrt(2/3)||d eps_p|| and the
uniaxial closed form (tests/test_oracle_pins.py).
"""
import numpy as np

from .tensors import lame, hooke6, deviator6, norm6


def return_map(d_eps, sigma_n, e_p, E, nu, sigma_y, E_h):
    """Radial return for a field of voxels.

    d_eps, sigma_n: [6, ...] (six stored components first); e_p: [...].
    Returns (d_eps_p [6, ...], de_p [...], sigma_new [6, ...]).
    """
    lam, mu = lame(E, nu)
    d_eps = np.asarray(d_eps, dtype=np.float64)
    sig_tr = np.asarray(sigma_n, dtype=np.float64) + hooke6(d_eps, lam, mu, axis=0)
    s = deviator6(sig_tr, axis=0)
    fy = np.sqrt(1.5) * norm6(s, axis=0)
    f = fy - (sigma_y + E_h * np.asarray(e_p, dtype=np.float64))
    plastic = f > 0.0
    de_p = np.where(plastic, f / (3.0 * mu + E_h), 0.0)
    safe_fy = np.where(plastic, fy, 1.0)
    d_eps_p = np.where(plastic[None], 1.5 * (de_p / safe_fy)[None] * s, 0.0)
    sigma_new = sig_tr - hooke6(d_eps_p, lam, mu, axis=0)
    return d_eps_p, de_p, sigma_new


def von_mises(sig6):
    """f_y(sigma) = sqrt(3/2) ||dev sigma|| (Sec. 4.1)."""
    return np.sqrt(1.5) * norm6(deviator6(sig6, axis=0), axis=0)
