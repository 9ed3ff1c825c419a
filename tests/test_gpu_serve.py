"""Served solves: results are independent of the mix, requests overlap on the device."""
import numpy as np
import pytest

from oracle import tensors as T
from paper_1811_11558_gb300 import inputs

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

E, NU = 1.0, 0.3
ES = T.e_star(E, NU)


def _requests(prec):
    from paper_1811_11558_gb300.serve import Request

    reqs = []
    rng = np.random.default_rng(1815)
    for i in range(6):
        n = (16, 32)[i % 2]
        nz = (8, 12)[(i // 2) % 2]
        z = inputs.uniform_depth(nz, 0.5)
        if i % 3 == 2:
            h = inputs.self_affine_surface(n, 1.0, 0.8, 2, 4, n // 4, 0.1, seed=1813 + i)
            wmax = 2e-3
        else:
            h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.5)
            wmax = 4e-3 * float(rng.uniform(0.5, 1.0))
        loads = [wmax * (k + 1) / 3 for k in range(3)]
        reqs.append(Request(i, n, z, h, loads, precision=prec, sigma_y=0.05 * ES, E_h=0.1, opts={"max_iter": 200}))
    return reqs


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_result_alone_equals_result_in_the_mix(prec):
    require_gpu()
    from paper_1811_11558_gb300.serve import Server

    reqs = _requests(prec)
    alone = [Server(slots=1).solve(r) for r in reqs[:2]]
    mix, wall = Server(slots=4).run(reqs)
    for a, m in zip(alone, mix[:2]):
        assert np.array_equal(a.pressure, m.pressure)
        assert a.report["alg1_iters"] == m.report["alg1_iters"]
    for m in mix:
        assert m.report["n_increments"] == 3
        assert abs(m.pressure.sum() / m.pressure.size - m_load(reqs[m.rid])) < 1e-6 * m_load(reqs[m.rid])


def m_load(r):
    return r.loads[-1] / (r.L * r.L)


def test_budget_refuses_oversized_request():
    require_gpu()
    from paper_1811_11558_gb300.serve import Server

    r = _requests("fp32")[0]
    with pytest.raises(ValueError):
        Server(slots=2, hbm_budget=1024).solve(r)


def test_new_shapes_arriving_while_others_capture_graphs():
    """Twelve requests of twelve different shapes on eight slots: contexts are created (device
    allocations, fills on the legacy stream) while other requests capture and replay their
    solver graphs.  Every request completes and gives the bits it gives alone."""
    require_gpu()
    from paper_1811_11558_gb300.serve import Request, Server

    reqs = []
    for i in range(12):
        n = (16, 32)[i % 2]
        z = inputs.uniform_depth(6 + i, 0.3)
        h = inputs.self_affine_surface(n, 1.0, 0.8, 2, 4, n // 4, 0.1, seed=1900 + i)
        reqs.append(Request(i, n, z, h, [1e-3, 2e-3], precision="fp32", sigma_y=0.05 * ES, E_h=0.1,
                            opts={"max_iter": 60, "relax": 0.3}))
    mix, _ = Server(slots=8).run(reqs)
    alone = [Server(slots=1).solve(r) for r in reqs]
    for a, m in zip(alone, mix):
        assert m is not None and m.report["n_increments"] == 2
        assert np.array_equal(a.pressure, m.pressure)


def test_prepared_pool_runs_tuned_plans_alone_and_in_the_mix():
    """Server.prepare tunes the depth kernel's tile plan once per shape before serving; every
    later context of that grid starts with the tuned plan, so a request gives the same bits
    alone (fresh server, fresh contexts) and in the mix."""
    require_gpu()
    from paper_1811_11558_gb300.serve import Request, Server

    reqs = []
    for i, (n, nz) in enumerate([(64, 10), (64, 14), (32, 9), (64, 10), (32, 9), (64, 14)]):
        z = inputs.uniform_depth(nz, 0.5)
        h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.5)
        reqs.append(Request(i, n, z, h, [1e-3 * (1 + i % 3), 3e-3], precision="fp32", sigma_y=0.05 * ES,
                            E_h=0.1, opts={"max_iter": 100}))
    srv = Server(slots=4)
    plans = srv.prepare(reqs, reps=3)
    assert len(plans) == 3 and all(p["tuned"] for p in plans.values())
    mix, _ = srv.run(reqs)
    alone = [Server(slots=1).solve(r) for r in reqs[:3]]
    for a, m in zip(alone, mix[:3]):
        assert np.array_equal(a.pressure, m.pressure)
        assert a.report["alg1_iters"] == m.report["alg1_iters"]
