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


def test_reference_arm_line_keeps_the_contract():
    """`bench.py --impl reference` (the oracle on the host cores, no GPU) prints one JSON line
    with the GPU arm's metric and unit, a measured step time that the run can account for, and
    the extrapolated one-core apply time beside it."""
    import json
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert 0 < d["ms_per_step"] < 600e3
    assert d["ms_per_apply_one_core_extrapolated"] > d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_batch_runs_every_problem_with_the_carried_relaxation():
    for pb in bench.batch_problems(64, 1814):
        assert pb["relax_mode"] == 1
        assert pb["relax"] == (0.3 if pb["rough"] else 0.5)
