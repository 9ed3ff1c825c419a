"""The bench's synthetic workloads are seeded and have the stated shapes (no GPU needed)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

E, NU = 1.0, 0.3


def test_uneven_batch_is_seeded_and_spans_the_stated_mix():
    a = bench.batch_problems()
    b = bench.batch_problems()
    assert len(a) == 64
    for p, q in zip(a, b):
        assert (p["n"], p["nz"], p["rough"]) == (q["n"], q["nz"], q["rough"])
        assert np.array_equal(p["h"], q["h"]) and p["loads"] == q["loads"]
    assert {p["n"] for p in a} == {64, 128, 256, 512}
    assert {p["nz"] for p in a} == {8, 16, 32}
    assert 16 < sum(p["rough"] for p in a) < 48
    es = E / (1 - NU * NU)
    for p in a:
        n, h, z = p["n"], p["h"], p["z"]
        assert h.shape == (n, n) and z[0] == 0.0 and z.size == p["nz"]
        # five equal increments; the total load lies in the decade below the 10 % area load
        loads = np.array(p["loads"])
        assert np.allclose(np.diff(loads), loads[0])
        if p["rough"]:
            w10 = 0.1 * es * 0.1 / 2.0
            assert abs(z[-1] - 0.05) < 1e-12 and abs(h.mean()) < 1e-12
        else:
            w10 = 4.0 * es * np.sqrt(0.1 / np.pi) ** 3 / (3.0 * 0.5)
            assert abs(z[-1] - 0.5) < 1e-12
        assert 0.1 * w10 * (1 - 1e-12) <= loads[-1] <= w10 * (1 + 1e-12)


def test_rough_surfaces_of_the_batch_have_the_stated_slope():
    """Spectral rms slope sqrt(mean |grad h|^2) = 0.1 for the self-affine surfaces among the first
    twelve problems."""
    for p in bench.batch_problems()[:12]:
        if not p["rough"]:
            continue
        n, h = p["n"], p["h"]
        k = np.fft.fftfreq(n, 1.0 / n)
        K2, K1 = np.meshgrid(k, k, indexing="ij")
        g = np.fft.fft2(h)
        slope = np.sqrt(np.sum(((2 * np.pi) ** 2) * (K1 ** 2 + K2 ** 2) * np.abs(g) ** 2)) / (n * n)
        assert abs(slope - 0.1) < 1e-9
