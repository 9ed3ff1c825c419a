"""The C ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fvim_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1811_11558_gb300 import build, fvim

    if not os.path.exists(fvim.LIB_PATH):
        build.build()
    L = ctypes.CDLL(fvim.LIB_PATH)
    names = _declared()
    assert "fvim_apply_mindlin" in names and len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_strerror_without_gpu():
    from paper_1811_11558_gb300 import fvim

    assert fvim.strerror(0) == "ok"
    assert fvim.strerror(-5) == "not converged"


def test_create_rejects_bad_grid_without_launching():
    """Argument errors are found on the host before anything touches the GPU."""
    from paper_1811_11558_gb300 import fvim
    import numpy as np

    L = fvim.lib()
    h = ctypes.c_void_p()
    z = np.array([0.0, 0.1])
    zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.fvim_create(ctypes.byref(h), 6, 8, 2, zp, 1.0, 1.0, 0, None) == -1      # even, not a power of 2
    assert L.fvim_create(ctypes.byref(h), 81, 512, 2, zp, 1.0, 1.0, 0, None) == -1   # odd side with a 512 side
    assert L.fvim_create(ctypes.byref(h), 257, 9, 2, zp, 1.0, 1.0, 0, None) == -1    # odd side beyond 255
    assert L.fvim_create(ctypes.byref(h), 1, 9, 2, zp, 1.0, 1.0, 0, None) == -1      # a single point
    assert L.fvim_create(ctypes.byref(h), 8, 8, 1, zp, 1.0, 1.0, 0, None) == -1      # one node
    assert L.fvim_create(ctypes.byref(h), 8, 8, 2, zp, -1.0, 1.0, 0, None) == -1     # bad cell
    assert L.fvim_create(ctypes.byref(h), 8, 8, 2, zp, 1.0, 1.0, 7, None) == -1      # bad precision
    assert L.fvim_apply_mindlin(None, None, None, 0, None) == -1


def test_group_apply_checks_arguments_without_gpu():
    """The grouped apply refuses a bad group size or NULL arrays on the host."""
    from paper_1811_11558_gb300 import fvim

    L = fvim.lib()
    arr = (ctypes.c_void_p * 65)()
    f = L.fvim_apply_mindlin_group
    assert f(None, 1, arr, arr, 0, None) == -1
    assert f(arr, 0, arr, arr, 0, None) == -1
    assert f(arr, 65, arr, arr, 0, None) == -1
    assert f(arr, 1, arr, arr, 0, None) == -1        # NULL context
    assert f(arr, 1, arr, arr, 7, None) == -1        # bad output kind
    assert fvim.GROUP_MAX == 64


def test_product_path_does_not_import_oracle():
    """The product package never names the CPU oracle (no fallback)."""
    pkg = os.path.join(ROOT, "paper_1811_11558_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f


def test_input_generators_load_nothing_of_the_cuda_path():
    """The oracle's golden-value scripts import the seeded input generators only: importing
    them loads neither the ctypes binding nor libfvim.so."""
    import subprocess
    import sys

    code = ("import sys; sys.path.insert(0, %r); import paper_1811_11558_gb300.inputs; "
            "print(any(m.endswith('.fvim') for m in sys.modules))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "False"


def test_plan_entry_points_check_arguments_without_gpu():
    from paper_1811_11558_gb300 import fvim

    L = fvim.lib()
    pl = fvim.Plan()
    assert L.fvim_autotune(None, 10, ctypes.byref(pl)) == -1
    assert L.fvim_get_plan(None, ctypes.byref(pl)) == -1
    assert L.fvim_set_plan(None, ctypes.byref(pl)) == -1


def test_plan_candidates_follow_the_launch_limits():
    """Host-only query of the chunk lengths the tuner times: a chunk length is launchable when
    the chunk threads of a 16-column tile fit one 256-thread block and the tile fits in shared
    memory; the default rule max(2, ceil(Nz / 16)) is always among them."""
    import pytest
    from paper_1811_11558_gb300 import fvim

    for n, nz, prec in [(512, 64, "fp32"), (512, 32, "fp32"), (64, 8, "fp32"), (128, 28, "fp64"),
                        (32, 300, "fp32"), (32, 300, "fp64"), (4, 2, "fp64")]:
        c = fvim.plan_candidates(n, n, nz, prec)
        chunks = [x for x, _ in c]
        assert (max(2, -(-nz // 16)), 2 if prec == "fp32" and n >= 32 and nz <= 64 else 0) in c
        assert all(2 <= x <= nz for x in chunks) and len(set(c)) == len(c)
        # FP64 and deep grids: the shared-memory variant (no register budget); FP32 registers: 2 or 3
        assert all(k == 0 for _, k in c) if prec == "fp64" else all(k in (0, 2, 3) for _, k in c)
    # Nz = 64 in FP32: 2 and 3 nodes per chunk would need 32 and 22 chunk threads per column; the
    # register variant of chunk lengths 4..8 also builds for three CTAs per SM (85 registers)
    assert fvim.plan_candidates(512, 512, 64, "fp32") == [(4, 2), (6, 2), (8, 2), (12, 0), (16, 0),
                                                          (4, 3), (6, 3), (8, 3)]
    assert fvim.plan_candidates(64, 64, 8, "fp32") == [(2, 2), (3, 2), (4, 2), (6, 2), (8, 2),
                                                       (4, 3), (6, 3), (8, 3)]
    with pytest.raises(fvim.FvimError):
        fvim.plan_candidates(6, 8, 8)
    with pytest.raises(fvim.FvimError):
        fvim.plan_candidates(8, 8, 1)


def test_no_cpu_fallback():
    """Without a CUDA device the binding refuses to build a context, and it never accepts host
    tensors as device buffers: there is no CPU path to fall back on."""
    import numpy as np
    import pytest
    torch = pytest.importorskip("torch")
    from paper_1811_11558_gb300 import fvim

    with pytest.raises(TypeError):
        fvim._ptr(torch.zeros(3), torch.float32, (3,), "x")
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            fvim.Context(8, 8, np.array([0.0, 0.1]))
