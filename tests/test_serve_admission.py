"""Host logic of the request server: admission by slots and HBM budget, FIFO order."""
import threading
import time

import pytest

from paper_1811_11558_gb300.serve import Admission, percentiles, poisson_arrivals


def _run(adm, jobs):
    """jobs: list of (footprint, hold seconds); returns admission order and peak usage."""
    order = []
    peak = {"active": 0, "used": 0}
    lock = threading.Lock()

    def work(i, fp, hold):
        adm.admit(fp)
        with lock:
            order.append(i)
            peak["active"] = max(peak["active"], adm.active)
            peak["used"] = max(peak["used"], adm.used)
        time.sleep(hold)
        adm.release(fp)

    ths = []
    for i, (fp, hold) in enumerate(jobs):
        th = threading.Thread(target=work, args=(i, fp, hold))
        th.start()
        ths.append(th)
        time.sleep(0.005)
    for th in ths:
        th.join()
    return order, peak


def test_slots_bound_concurrency_and_order_is_fifo():
    adm = Admission(slots=2, budget_bytes=10 ** 12)
    order, peak = _run(adm, [(1, 0.05)] * 6)
    assert peak["active"] <= 2
    assert order == list(range(6))
    assert adm.active == 0 and adm.used == 0


def test_budget_bounds_memory():
    adm = Admission(slots=8, budget_bytes=100)
    order, peak = _run(adm, [(60, 0.05), (30, 0.05), (50, 0.05), (10, 0.05)])
    assert peak["used"] <= 100
    # FIFO: the 50-byte request waits for memory and the 10-byte one does not overtake it
    assert order == [0, 1, 2, 3]


def test_request_larger_than_budget_is_refused():
    adm = Admission(slots=1, budget_bytes=10)
    with pytest.raises(ValueError):
        adm.admit(11)


def test_percentiles_and_arrivals():
    p = percentiles(list(range(1, 101)))
    assert p[50] == pytest.approx(50.5) and p[99] == pytest.approx(99.01)
    a = poisson_arrivals(1000, 50.0, seed=1)
    assert (a[1:] >= a[:-1]).all() and abs(a[-1] / 1000 - 1 / 50.0) < 0.1 / 50.0 * 3
