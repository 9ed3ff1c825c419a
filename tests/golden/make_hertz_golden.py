"""Write the oracle's solution of the elastic-plastic Hertz case to hertz_32x32x16.npz.

Case (the plain FP64 workload): rigid paraboloid R = 0.5 on the periodic half-space,
cell 1 x 1, 32 x 32 surface points, 16 uniform depth nodes to z = 0.5, E = 1, nu = 0.3,
sigma_y = 0.05 E*, E_h = 0.1 E, five equal load increments up to the load at which the
elastic Hertz peak pressure is 3 sigma_y (W_max = 2 pi a^2 p0 / 3, a = pi R p0 / (2 E*)).
Algorithm 1 (Sec. 5.2) with tol 1e-12 and relaxation lambda = 0.5 (with lambda = 1 the coupling
oscillates from the third increment on and never reaches the tolerance; the paper leaves
lambda to the user); contact CG to 1e-15, DF-SANE to 1e-13.  The tolerances are three orders
tighter than the paper's 1e-9 so that the stored solution is converged well below the FP64
parity bar of 1e-10 (every increment reaches e < 1e-12 in 46-81 coupling iterations).
Only the oracle is called.  Run from the repository root:
    python tests/golden/make_hertz_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import contact as C  # noqa: E402
from oracle import tensors as T  # noqa: E402
from paper_1811_11558_gb300 import inputs  # noqa: E402

E, NU, R = 1.0, 0.3, 0.5
RELAX = 0.5
N, NZ, DEPTH, NINC = 32, 16, 0.5, 5


def case():
    es = T.e_star(E, NU)
    sy = 0.05 * es
    p0 = 3.0 * sy
    a = np.pi * R * p0 / (2.0 * es)
    wmax = 2.0 * np.pi * a * a * p0 / 3.0
    loads = [wmax * (k + 1) / NINC for k in range(NINC)]
    return dict(E=E, nu=NU, sigma_y=sy, E_h=0.1 * E, R=R, n=N, nz=NZ, depth=DEPTH, loads=np.array(loads))


def main():
    c = case()
    z = inputs.uniform_depth(NZ, DEPTH)
    h = inputs.hertz_profile(N, N, 1.0, 1.0, R)
    st = C.PlasticState(NZ, N, N)
    iters, areas = [], []
    for W in c["loads"]:
        Tn, info = C.algorithm1(W, h, st, z, 1.0, 1.0, E, NU, c["sigma_y"], c["E_h"], tol=1e-12, N_max=600,
                                relax=RELAX, cg_tol=1e-15, df_tol_rel=1e-13)
        assert info["converged"]
        iters.append(info["iterations"])
        areas.append(info["area"])
        print("W=%.6e iterations=%d area=%.6f max e_p=%.5f" % (W, info["iterations"], info["area"], st.e_p.max()))
    np.savez_compressed(os.path.join(HERE, "hertz_32x32x16.npz"), p=st.T, e_p=st.e_p, eps_p=st.eps_p,
                        sigma=st.sigma, loads=c["loads"], sigma_y=c["sigma_y"], E_h=c["E_h"], relax=RELAX,
                        iterations=np.array(iters), areas=np.array(areas))


if __name__ == "__main__":
    main()
