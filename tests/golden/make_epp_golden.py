"""Write the oracle's solution of an elastic-perfectly-plastic Hertz load sweep to
epp_hertz_32x32x8.npz.

Case (the perfectly plastic limit E_h = 0 of the Hertz problem, in the spirit of the paper's
elastic-perfectly-plastic comparison of App. C.2, on a power-of-two grid): rigid paraboloid
R = 0.5 on the periodic half-space, cell 1 x 1, 32 x 32 surface points, 8 uniform depth nodes
to z = 0.25, E = 1, nu = 0.3, sigma_y = 0.05 E*, E_h = 0.  Loads W / W_y = 2, 4, 8 applied as
three increments, with W_y the onset load of yield of the elastic Hertz solution: the peak
pressure p0 = 1.6 sigma_y at onset for nu = 0.3, a_y = pi R p0 / (2 E*), W_y = 2 pi a_y^2 p0 / 3.
Algorithm 1 (Sec. 5.2) with tol 1e-9 and relaxation 0.5; contact CG to 1e-13, DF-SANE to 1e-11.
Only the oracle is called.  Run from the repository root:
    python tests/golden/make_epp_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import contact as C  # noqa: E402
from oracle import tensors as T  # noqa: E402
from paper_1811_11558_gb300 import inputs  # noqa: E402

E, NU, R = 1.0, 0.3, 0.5
RELAX = 0.5
N, NZ, DEPTH = 32, 8, 0.25
RATIOS = (2.0, 4.0, 8.0)


def case():
    es = T.e_star(E, NU)
    sy = 0.05 * es
    p0 = 1.6 * sy
    a = np.pi * R * p0 / (2.0 * es)
    wy = 2.0 * np.pi * a * a * p0 / 3.0
    return dict(sigma_y=sy, E_h=0.0, W_y=wy, loads=np.array([r * wy for r in RATIOS]))


def main():
    c = case()
    z = inputs.uniform_depth(NZ, DEPTH)
    h = inputs.hertz_profile(N, N, 1.0, 1.0, R)
    st = C.PlasticState(NZ, N, N)
    iters, areas = [], []
    for W in c["loads"]:
        t0 = time.time()
        Tn, info = C.algorithm1(W, h, st, z, 1.0, 1.0, E, NU, c["sigma_y"], 0.0, tol=1e-9, N_max=400,
                                relax=RELAX, cg_tol=1e-13, df_tol_rel=1e-11)
        assert info["converged"]
        iters.append(info["iterations"])
        areas.append(info["area"])
        print("W/W_y=%.1f iterations=%d area=%.6f max p/sigma_y=%.4f max e_p=%.5f (%.0f s)"
              % (W / c["W_y"], info["iterations"], info["area"], Tn.max() / c["sigma_y"], st.e_p.max(),
                 time.time() - t0))
    np.savez_compressed(os.path.join(HERE, "epp_hertz_32x32x8.npz"), p=st.T, e_p=st.e_p, eps_p=st.eps_p,
                        sigma=st.sigma, loads=c["loads"], W_y=c["W_y"], sigma_y=c["sigma_y"], E_h=0.0,
                        relax=RELAX, depth=DEPTH, iterations=np.array(iters), areas=np.array(areas))


if __name__ == "__main__":
    main()
