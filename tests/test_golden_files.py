"""The stored Algorithm-1 solutions satisfy the equations that define them.

The golden files are written by the oracle (tests/golden/make_*_golden.py); these checks do
not call the oracle: they restate, on the stored arrays, the total-load constraint and the
positivity of the pressure (Sec. 5.1), the plastic incompressibility of eps_p and the yield
admissibility of the stress state (Sec. 4.1), in a few lines of numpy.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
E, NU = 1.0, 0.3


def _von_mises(sig):
    s = np.array(sig, dtype=np.float64)
    m = (s[:, 0] + s[:, 1] + s[:, 2]) / 3.0
    for k in range(3):
        s[:, k] -= m
    return np.sqrt(1.5 * (s[:, 0] ** 2 + s[:, 1] ** 2 + s[:, 2] ** 2 + 2 * (s[:, 3] ** 2 + s[:, 4] ** 2 + s[:, 5] ** 2)))


@pytest.mark.parametrize("name", ["hertz_32x32x16.npz", "rough_32x32x8.npz", "epp_hertz_32x32x8.npz"])
def test_golden_solution_is_admissible(name):
    g = np.load(os.path.join(GOLDEN, name))
    p, ep, epp, sig = g["p"], g["e_p"], g["eps_p"], g["sigma"]
    n2, n1 = p.shape
    dA = 1.0 / (n1 * n2)
    W = float(g["loads"][-1])
    # total load and unilateral contact
    assert abs(p.sum() * dA - W) < 1e-10 * W
    assert (p >= 0).all()
    assert abs((p > 0).mean() - g["areas"][-1]) == 0
    # plastic flow is isochoric, cumulated plastic strain is non-negative
    assert np.abs(epp[:, 0] + epp[:, 1] + epp[:, 2]).max() < 1e-12
    assert (ep >= -1e-15).all() and ep.max() > 0
    # the stress state lies inside the current yield surface (to the solver tolerance)
    fy = float(g["sigma_y"]) + float(g["E_h"]) * ep
    assert (_von_mises(sig) <= fy * (1 + 1e-6)).all()
    # the last increment loaded some points plastically: there the state is on the yield
    # surface (a point that flowed earlier may have unloaded elastically since, so the most
    # strained point need not be)
    vm = _von_mises(sig)
    i = np.unravel_index(np.argmax(vm / fy), ep.shape)
    assert ep[i] > 0 and abs(vm[i] - fy[i]) < 1e-6 * fy[i]


def test_perfectly_plastic_sweep_flattens_the_contact():
    """E_h = 0: plastic flow caps the contact pressure below the elastic Hertz peak of the same
    load and widens the contact beyond the elastic Hertz area (closed forms, Sec. 6.2)."""
    g = np.load(os.path.join(GOLDEN, "epp_hertz_32x32x8.npz"))
    es = E / (1 - NU * NU)
    R = 0.5
    W = float(g["loads"][-1])
    a = (3 * W * R / (4 * es)) ** (1.0 / 3.0)
    p0 = 3 * W / (2 * np.pi * a * a)
    p = g["p"]
    assert p.max() < 0.75 * p0
    assert float(g["areas"][-1]) > 1.2 * np.pi * a * a
    # the peak pressure grows with the load, but far less than the elastic W^(1/3)
    assert float(g["E_h"]) == 0.0 and p.max() < 3.0 * float(g["sigma_y"])
