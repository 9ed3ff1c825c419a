"""Write the oracle's solution of a small elastic-plastic rough-surface case to rough_32x32x8.npz.

Case: seeded self-affine surface 32 x 32 (H = 0.8, flat PSD for 2 <= |k| < 4, power law to
k_s = 8, rms slope 0.1, PCG64 seed 1813) on the periodic half-space, cell 1 x 1, 8 uniform
depth nodes to z = 0.1, E = 1, nu = 0.3, sigma_y = 0.05 E*, E_h = 0.1 E, two equal load
increments to W = 5e-3 (contact fraction 7.6 % then 14 %, plastic strain up to 2.5 %).
Algorithm 1 (Sec. 5.2) with tol 1e-9 and relaxation lambda = 0.3 (the paper's value for rough
surfaces, App. C.3); contact CG to 1e-13, DF-SANE to 1e-11.
Only the oracle is called.  Run from the repository root:
    python tests/golden/make_rough_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import contact as C  # noqa: E402
from oracle import tensors as T  # noqa: E402
from paper_1811_11558_gb300 import inputs  # noqa: E402

E, NU = 1.0, 0.3
RELAX = 0.3
N, NZ, DEPTH, NINC, WMAX, SEED = 32, 8, 0.1, 2, 5e-3, 1813


def main():
    es = T.e_star(E, NU)
    sy, Eh = 0.05 * es, 0.1 * E
    loads = np.array([WMAX * (k + 1) / NINC for k in range(NINC)])
    z = inputs.uniform_depth(NZ, DEPTH)
    h = inputs.self_affine_surface(N, 1.0, 0.8, 2, 4, 8, 0.1, seed=SEED)
    st = C.PlasticState(NZ, N, N)
    iters, areas = [], []
    for W in loads:
        Tn, info = C.algorithm1(W, h, st, z, 1.0, 1.0, E, NU, sy, Eh, tol=1e-9, N_max=400, relax=RELAX,
                                cg_tol=1e-13, df_tol_rel=1e-11)
        assert info["converged"]
        iters.append(info["iterations"])
        areas.append(info["area"])
        print("W=%.6e iterations=%d area=%.6f max e_p=%.5f" % (W, info["iterations"], info["area"], st.e_p.max()))
    np.savez_compressed(os.path.join(HERE, "rough_32x32x8.npz"), h=h, p=st.T, e_p=st.e_p, eps_p=st.eps_p,
                        sigma=st.sigma, loads=loads, sigma_y=sy, E_h=Eh, relax=RELAX, depth=DEPTH,
                        iterations=np.array(iters), areas=np.array(areas))


if __name__ == "__main__":
    main()
