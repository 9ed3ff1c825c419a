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


def dfsane(F, x0, inner, tol_abs, tol_rel, max_iter, M=10, gamma=1e-4, sigma_min=1e-10, sigma_max=1e10,
           tau_min=0.1, tau_max=0.5, max_backtrack=60):
    """Derivative-free spectral residual method (DF-SANE) of La Cruz, Martinez & Raydan
    (2006), the published algorithm used in Sec. 4.3:
        d_k = -sigma_k F(x_k),  sigma_k = <s, s> / <s, y>  (s = x_k - x_{k-1},
        y = F(x_k) - F(x_{k-1})), safeguarded into [sigma_min, sigma_max];
        nonmonotone line search on f = ||F||^2, trying x + alpha d and x - alpha d:
        accept when f(x +- alpha d) <= max(last M values of f) + eta_k - gamma alpha^2 f(x_k),
        eta_k = ||F(x_0)|| / (1 + k)^2, otherwise shrink alpha by the safeguarded
        quadratic model into [tau_min alpha, tau_max alpha].
    Published defaults (the paper gives none).  Stops when ||F|| <= tol_abs + tol_rel ||F(x_0)||.
    Returns (x, info)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    Fx = F(x)
    f = inner(Fx, Fx)
    nF0 = np.sqrt(f)
    hist = [f]
    sigma = 1.0
    evals = 1
    k = 0
    for k in range(max_iter):
        if np.sqrt(f) <= tol_abs + tol_rel * nF0:
            return x, {"iterations": k, "residual": np.sqrt(f), "residual0": nF0, "evals": evals,
                       "converged": True}
        d = -sigma * Fx
        fmax = max(hist[-M:])
        eta = nF0 / (1.0 + k) ** 2
        ap = am = 1.0
        xn = Fn = fn = None
        for _ in range(max_backtrack):
            xp = x + ap * d
            Fp = F(xp)
            evals += 1
            fp = inner(Fp, Fp)
            if fp <= fmax + eta - gamma * ap * ap * f:
                xn, Fn, fn = xp, Fp, fp
                break
            xm = x - am * d
            Fm = F(xm)
            evals += 1
            fm = inner(Fm, Fm)
            if fm <= fmax + eta - gamma * am * am * f:
                xn, Fn, fn = xm, Fm, fm
                break
            ap = min(max(ap * ap * f / (fp + (2.0 * ap - 1.0) * f), tau_min * ap), tau_max * ap)
            am = min(max(am * am * f / (fm + (2.0 * am - 1.0) * f), tau_min * am), tau_max * am)
        if xn is None:
            break
        s = xn - x
        y = Fn - Fx
        sy = inner(s, y)
        ss = inner(s, s)
        sigma = ss / sy if sy != 0.0 else np.inf
        if not (sigma_min <= abs(sigma) <= sigma_max):
            nf = np.sqrt(fn)
            sigma = 1.0 if nf > 1.0 else (1.0 / nf if nf >= 1e-5 else 1e5)
        x, Fx, f = xn, Fn, fn
        hist.append(f)
    return x, {"iterations": k, "residual": np.sqrt(f), "residual0": nF0, "evals": evals,
               "converged": bool(np.sqrt(f) <= tol_abs + tol_rel * nF0)}
