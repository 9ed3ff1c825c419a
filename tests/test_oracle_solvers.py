"""Pins of the oracle's solvers (Polonsky-Keer CG, DF-SANE, Algorithm 1).

Iterates are never compared; the converged answers are checked against closed forms and
against the equations that define them.
"""
import numpy as np
import pytest

from oracle import contact as C
from oracle import operators as op
from oracle import plasticity as pl
from oracle import tensors as T
from paper_1811_11558_gb300 import inputs

E, NU = 1.0, 0.3
LAM, MU = T.lame(E, NU)
ES = T.e_star(E, NU)
R = 0.5


def _hertz(W):
    a = (3 * W * R / (4 * ES)) ** (1 / 3)
    return a, 3 * W / (2 * np.pi * a * a)


def test_polonsky_keer_kkt_and_load():
    """Sec. 5.1: p >= 0, gap >= 0, p gap = 0 and dA sum p = W at convergence."""
    n = 64
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    W = 4.7916e-3
    p, info = C.polonsky_keer(h, W, 1.0, 1.0, E, NU, tol=1e-13)
    dA = 1.0 / (n * n)
    assert info["error"] < 1e-13
    assert p.min() >= 0.0
    assert abs(dA * p.sum() - W) < 1e-14
    scale = np.abs(h).max()
    assert info["gap"].min() > -1e-12 * scale
    assert np.abs(p * info["gap"]).max() < 1e-12 * scale * p.max()


def test_polonsky_keer_hertz_converges_with_grid():
    """Hertz: a = (3PR/(4E*))^(1/3), p0 = 3P/(2 pi a^2), p(r) = p0 sqrt(1 - r^2/a^2);
    the periodic discrete solution approaches them as the grid is refined."""
    W = 4.7916e-3
    a_ref, p0_ref = _hertz(W)
    errs = []
    for n in (64, 128):
        h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
        p, info = C.polonsky_keer(h, W, 1.0, 1.0, E, NU, tol=1e-12)
        a_num = np.sqrt(info["area"] / np.pi)
        errs.append(abs(a_num - a_ref) / a_ref)
        assert abs(p.max() - p0_ref) / p0_ref < 0.01
        x = -0.5 + np.arange(n) / n
        r = np.abs(x)
        inside = r < 0.8 * a_ref
        prof = p0_ref * np.sqrt(np.clip(1 - r[inside] ** 2 / a_ref ** 2, 0, None))
        assert np.abs(p[n // 2, inside] - prof).max() < 0.02 * p0_ref
    assert errs[1] < errs[0] and errs[1] < 0.01


def test_hertz_subsurface_stress_and_onset_of_yield():
    """Sec. 6.2: at the load W_y = pi^3 R^2 p_y^3 / (6 E*^2) with p_y = 1.6 sigma_y the peak
    Hertz pressure is p_y, a_y = sqrt(3 W_y / (2 pi p_y)), and the maximum von Mises stress of
    the Boussinesq field of the contact pressure reaches sigma_y (within the grid error);
    on the axis sigma_z = -p0 / (1 + z^2/a^2)."""
    sy = 0.05 * ES
    py = 1.6 * sy
    Wy = np.pi ** 3 * R ** 2 * py ** 3 / (6 * ES ** 2)
    ay = np.sqrt(3 * Wy / (2 * np.pi * py))
    a_ref, p0_ref = _hertz(Wy)
    assert abs(a_ref - ay) < 1e-12 and abs(p0_ref - py) < 1e-12
    n = 128
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    p, _ = C.polonsky_keer(h, Wy, 1.0, 1.0, E, NU, tol=1e-12)
    z = np.linspace(0.0, 3 * ay, 49)
    _, sig = op.boussinesq_apply(p, z, 1.0, 1.0, E, NU, "stress")
    vm = pl.von_mises(np.moveaxis(sig, 1, 0))
    assert abs(vm.max() - sy) / sy < 0.03
    axis = sig[:, 2, n // 2, n // 2]
    ref = -p0_ref / (1 + z ** 2 / ay ** 2)
    assert np.abs(axis - ref).max() < 0.03 * p0_ref


def test_dfsane_elastic_is_the_predictor():
    """Without yield the residual is R[x] = x - grad^sym M[dT]: DF-SANE stops after one
    step at the elastic predictor (Sec. 4.2 with deps_p = 0)."""
    n, nz = 8, 5
    z = inputs.uniform_depth(nz, 0.3)
    st = C.PlasticState(nz, n, n)
    dT = np.abs(inputs.random_field((n, n), seed=4)) * 1e-3
    dE, dep, dEp, info = C.plasticity_solve(dT, st, z, 1.0, 1.0, E, NU, 1e9, 0.0)
    _, b = op.boussinesq_apply(dT, z, 1.0, 1.0, E, NU, "strain")
    assert info["iterations"] == 0
    assert np.abs(dE - b).max() == 0.0 and not dep.any()


def test_dfsane_uniaxial_strain_closed_form():
    """A uniform pressure pbar (mode 0 only) loads every layer in uniaxial strain.  With
    linear hardening the increment from the virgin state has the closed form
    deps_p = k (1/2, 1/2, -1, 0, 0, 0) with
        k = (2 mu pbar/(lambda + 2 mu) - sigma_y) / (3 mu - 4 mu^2/(lambda + 2 mu) + E_h),
    which the DF-SANE fixed point of Eq. incremental_strain must reproduce at every voxel."""
    n, nz = 4, 4
    z = inputs.uniform_depth(nz, 0.2)
    sy, Eh = 0.05, 0.1
    pbar = 0.2
    st = C.PlasticState(nz, n, n)
    dT = np.full((n, n), pbar)
    dE, dep, dEp, info = C.plasticity_solve(dT, st, z, 1.0, 1.0, E, NU, sy, Eh, tol_rel=1e-13)
    assert info["converged"]
    k = (2 * MU * pbar / (LAM + 2 * MU) - sy) / (3 * MU - 4 * MU ** 2 / (LAM + 2 * MU) + Eh)
    assert k > 0
    expect = np.array([0.5, 0.5, -1.0, 0, 0, 0]) * k
    assert np.abs(dep - expect[None, :, None, None]).max() < 1e-11 * k
    assert np.abs(dEp - k).max() < 1e-11 * k


@pytest.mark.slow
def test_algorithm1_increment_satisfies_its_equations():
    """Sec. 5.2: a converged increment of Algorithm 1 carries the load W, its pressure is
    the elastic-contact solution on the modified surface H0 - dU (KKT), the plastic
    strain increment is the fixed point of Eq. incremental_strain and the updated stress
    is plastically admissible (f_y <= f_h)."""
    n, nz = 16, 8
    z = inputs.uniform_depth(nz, 0.5)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    sy, Eh = 0.05 * ES, 0.1
    st = C.PlasticState(nz, n, n)
    for k in (1, 2, 3):
        W = k * 4.7916e-3 / 3
        sigma_before = st.sigma.copy()
        e_p_before = st.e_p.copy()
        T_prev = st.T.copy()
        prev = C.PlasticState(nz, n, n)
        prev.sigma, prev.e_p = sigma_before, e_p_before
        eps_p_before = st.eps_p.copy()
        Tn, info = C.algorithm1(W, h, st, z, 1.0, 1.0, E, NU, sy, Eh, tol=1e-9, N_max=200)
        assert info["converged"]
        dA = 1.0 / (n * n)
        assert abs(dA * Tn.sum() - W) < 1e-13
        dep_total = st.eps_p - eps_p_before
        dU = C.residual_surface(dep_total, z, 1.0, 1.0, E, NU)
        p_chk, cinfo = C.polonsky_keer(info["H0"] - dU, W, 1.0, 1.0, E, NU, tol=1e-13)
        assert np.abs(p_chk - Tn).max() < 1e-6 * Tn.max()
        # the fixed point of the plastic residual for dT = T - T_prev
        dE = info["dE"]
        _, b = op.boussinesq_apply(Tn - T_prev, z, 1.0, 1.0, E, NU, "strain")
        dep, _, _ = pl.return_map(np.moveaxis(dE, 1, 0), np.moveaxis(sigma_before, 1, 0), e_p_before, E, NU, sy, Eh)
        res = dE - b - op.mindlin_apply(np.moveaxis(dep, 0, 1), z, 1.0, 1.0, E, NU, "strain")
        assert np.abs(res).max() < 1e-8 * np.abs(dE).max()
        fy = pl.von_mises(np.moveaxis(st.sigma, 1, 0))
        assert (fy - (sy + Eh * st.e_p)).max() < 1e-12
    assert st.e_p.max() > 0   # the last load is well beyond the onset of yield


def test_relaxation_does_not_change_the_converged_increment():
    """The relaxation factor of Algorithm 1 only changes the path, not the converged
    increment (the coupled problem has one solution for a given load)."""
    n, nz = 8, 5
    z = inputs.uniform_depth(nz, 0.5)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.25)
    sy, Eh = 0.03, 0.2
    outs = []
    for relax in (1.0, 0.5):
        st = C.PlasticState(nz, n, n)
        Tn, info = C.algorithm1(6e-3, h, st, z, 1.0, 1.0, E, NU, sy, Eh, tol=1e-11, N_max=200, relax=relax)
        assert info["converged"]
        outs.append((Tn, st.eps_p))
    assert st.e_p.max() > 0
    assert np.abs(outs[0][0] - outs[1][0]).max() < 1e-7 * outs[0][0].max()
    assert np.abs(outs[0][1] - outs[1][1]).max() < 1e-7 * np.abs(outs[0][1]).max()


def test_carried_relaxation_reaches_the_same_increment():
    """Algorithm 1 with the relaxed value carried between iterations (relax_mode "carried")
    converges to the increment of the listing's order: the coupled problem has one solution
    for a given load, the relaxation only changes the path."""
    n, nz = 8, 5
    z = inputs.uniform_depth(nz, 0.5)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.25)
    sy, Eh = 0.03, 0.2
    outs = []
    for mode, relax in (("literal", 1.0), ("carried", 0.5), ("carried", 0.2)):
        st = C.PlasticState(nz, n, n)
        Tn, info = C.algorithm1(6e-3, h, st, z, 1.0, 1.0, E, NU, sy, Eh, tol=1e-11, N_max=400, relax=relax,
                                relax_mode=mode)
        assert info["converged"], (mode, relax)
        outs.append((Tn, st.eps_p))
    for Tn, ep in outs[1:]:
        assert np.abs(Tn - outs[0][0]).max() < 1e-7 * outs[0][0].max()
        assert np.abs(ep - outs[0][1]).max() < 1e-7 * np.abs(outs[0][1]).max()


@pytest.mark.parametrize("a", [0.8, 1.2, 1.6, 3.0])
def test_relaxation_orders_on_a_linear_coupling(a):
    """The two relaxation orders on the scalar model of one coupled increment: the residual
    displacement x of the plastic flow lowers the modified surface H = H0 - r, which lowers the
    flow, x = 1 - a (H0 - H), a the gain of that feedback (large on rough surfaces with a few
    heavily loaded asperities).  The listing's order, x_{k+1} = 1 - a ((1 - lambda) x_{k-1} +
    lambda x_k), converges only when a (1 - lambda) < 1 (the product of its characteristic roots);
    the carried one, r_k = r_{k-1} + lambda (x_k - r_{k-1}), whenever |1 - lambda (1 + a)| < 1.
    The iteration is the one written in oracle.contact.algorithm1, with the two inner solves
    replaced by this linear response."""
    lam = 0.3

    def run(mode):
        x_prev, H, H0, errs = 0.0, 1.0, 1.0, []
        for _ in range(400):
            x = 1.0 - a * (H0 - H)        # F: more residual displacement, less flow
            e = abs(x - x_prev)
            errs.append(e)
            r = x_prev + lam * (x - x_prev)
            H = H0 - r
            x_prev = x if mode == "literal" else r
        return errs

    lit, car = run("literal"), run("carried")
    assert car[-1] < 1e-12                       # carried: |1 - 0.3 (1 + a)| < 1 for every a here
    if a * (1 - lam) < 1:
        assert lit[-1] < 1e-6
    else:
        assert lit[-1] > 1e-3                     # literal: stalls or grows once a (1 - lambda) >= 1
