"""Thin Python binding of libfvim (include/fvim.h): argument marshalling only.

Every step of every operator runs in the CUDA kernels of libfvim.so; this module
checks tensor shapes, dtypes and devices, passes raw device pointers and the
current torch CUDA stream, and turns status codes into exceptions.  There is no
CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfvim.so")

FVIM_FP32 = 0
FVIM_FP64 = 1
FVIM_STRESS = 0
FVIM_STRAIN = 1

_lib = None


MAX_INCREMENTS = 64


class Opts(ctypes.Structure):
    """fvim_opts (include/fvim.h)."""
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("relax", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int), ("df_tol_abs", ctypes.c_double),
                ("df_tol_rel", ctypes.c_double), ("df_max_iter", ctypes.c_int), ("relax_mode", ctypes.c_int)]


class Report(ctypes.Structure):
    """fvim_report (include/fvim.h)."""
    _fields_ = [("status", ctypes.c_int), ("n_increments", ctypes.c_int),
                ("alg1_iters", ctypes.c_int * MAX_INCREMENTS), ("alg1_error", ctypes.c_double * MAX_INCREMENTS),
                ("contact_area", ctypes.c_double * MAX_INCREMENTS), ("load_error", ctypes.c_double),
                ("cg_iters", ctypes.c_long), ("df_iters", ctypes.c_long), ("residual_evals", ctypes.c_long),
                ("mindlin_applies", ctypes.c_long)]

    def as_dict(self):
        n = self.n_increments
        return {"status": self.status, "n_increments": n, "alg1_iters": list(self.alg1_iters[:n]),
                "alg1_error": list(self.alg1_error[:n]), "contact_area": list(self.contact_area[:n]),
                "load_error": self.load_error, "cg_iters": self.cg_iters, "df_iters": self.df_iters,
                "residual_evals": self.residual_evals, "mindlin_applies": self.mindlin_applies}


PLAN_MAX_CAND = 16
FFT_PATHS = ("rows_cols", "l2_exchange", "cluster")   # FVIM_FFT_ROWCOL, FVIM_FFT_L2, FVIM_FFT_CLUSTER


class Plan(ctypes.Structure):
    """fvim_plan (include/fvim.h)."""
    _fields_ = [("depth_chunk", ctypes.c_int), ("tuned", ctypes.c_int), ("n_cand", ctypes.c_int),
                ("cand", ctypes.c_int * PLAN_MAX_CAND), ("cand_ctas", ctypes.c_int * PLAN_MAX_CAND),
                ("cand_ms", ctypes.c_float * PLAN_MAX_CAND), ("depth_ctas", ctypes.c_int),
                ("depth_cutoff", ctypes.c_float), ("fft_path", ctypes.c_int),
                ("fft_ms", ctypes.c_float * len(FFT_PATHS))]

    def as_dict(self):
        """timings_ms: chunk length -> ms with the default register budget; timings_ms_3ctas:
        the same with three CTAs per SM (85 registers), where built."""
        n = self.n_cand
        d = {"depth_chunk": self.depth_chunk, "depth_ctas": self.depth_ctas,
             "depth_cutoff": round(float(self.depth_cutoff), 6), "tuned": bool(self.tuned),
             "timings_ms": {int(self.cand[i]): float(self.cand_ms[i]) for i in range(n) if self.cand_ctas[i] != 3},
             "fft_path": FFT_PATHS[self.fft_path]}
        t3 = {int(self.cand[i]): float(self.cand_ms[i]) for i in range(n) if self.cand_ctas[i] == 3}
        if t3:
            d["timings_ms_3ctas"] = t3
        if any(self.fft_ms[i] > 0 for i in range(len(FFT_PATHS))):
            d["fft_apply_ms"] = {FFT_PATHS[i]: float(self.fft_ms[i]) for i in range(len(FFT_PATHS))
                                 if self.fft_ms[i] > 0}
        return d


def plan_candidates(n1, n2, nz, precision="fp32"):
    """Depth-kernel launch shapes the tuner times on this grid, as (chunk length, CTAs per SM)
    pairs (host computation only)."""
    buf = (ctypes.c_int * PLAN_MAX_CAND)()
    ctas = (ctypes.c_int * PLAN_MAX_CAND)()
    prec = FVIM_FP32 if precision == "fp32" else FVIM_FP64
    n = lib().fvim_plan_candidates(int(n1), int(n2), int(nz), prec, buf, ctas, PLAN_MAX_CAND)
    _check(n if n < 0 else 0, "fvim_plan_candidates")
    return list(zip(buf[:n], ctas[:n]))


class FvimError(RuntimeError):
    def __init__(self, status, what):
        msg = "%s failed: %s (status %d)" % (what, strerror(status), status)
        if status == -3:
            msg += ": " + lib().fvim_last_cuda_error().decode()
        super().__init__(msg)
        self.status = status


def lib():
    """Load libfvim.so (built by paper_1811_11558_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfvim.so not built (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "fvim_create": (i, [ctypes.POINTER(vp), i, i, i, ctypes.POINTER(d), d, d, i, vp]),
        "fvim_set_material": (i, [vp, d, d, d, d]),
        "fvim_set_stream": (i, [vp, vp]),
        "fvim_apply_mindlin": (i, [vp, vp, vp, i, vp]),
        "fvim_apply_mindlin_group": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]),
        "fvim_apply_boussinesq": (i, [vp, vp, vp, vp, i]),
        "fvim_return_map": (i, [vp, vp, vp, vp]),
        "fvim_commit_state": (i, [vp, vp, vp, vp]),
        "fvim_get_state": (i, [vp, vp, vp, vp]),
        "fvim_set_state": (i, [vp, vp, vp, vp]),
        "fvim_sync": (i, [vp]),
        "fvim_destroy": (i, [vp]),
        "fvim_strerror": (ctypes.c_char_p, [i]),
        "fvim_last_cuda_error": (ctypes.c_char_p, []),
        "fvim_last_kernel_count": (i, [vp]),
        "fvim_profile_enable": (i, [vp, i]),
        "fvim_profile_read": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(i), i]),
        "fvim_profile_name": (ctypes.c_char_p, [i]),
        "fvim_default_opts": (i, [vp, ctypes.POINTER(Opts)]),
        "fvim_elastic_contact": (i, [vp, vp, d, vp, ctypes.POINTER(Opts), ctypes.POINTER(i), ctypes.POINTER(d)]),
        "fvim_plasticity_solve": (i, [vp, vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(i),
                                      ctypes.POINTER(d)]),
        "fvim_solve_contact": (i, [vp, vp, ctypes.POINTER(d), i, ctypes.POINTER(Opts), vp, ctypes.POINTER(Report)]),
        "fvim_reset_state": (i, [vp]),
        "fvim_footprint": (ctypes.c_size_t, [i, i, i, i]),
        "fvim_autotune": (i, [vp, i, ctypes.POINTER(Plan)]),
        "fvim_get_plan": (i, [vp, ctypes.POINTER(Plan)]),
        "fvim_plan_candidates": (i, [i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), i]),
        "fvim_set_plan": (i, [vp, ctypes.POINTER(Plan)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(status):
    return lib().fvim_strerror(int(status)).decode()


def _check(status, what):
    if status != 0:
        raise FvimError(status, what)


def _ptr(t, dtype, shape, name):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


GROUP_MAX = 64


def apply_mindlin_group(contexts, eps_list, out_list=None, kind="stress"):
    """fvim_apply_mindlin_group: the Mindlin apply of up to GROUP_MAX FP32 contexts of uneven
    grid size (power-of-two sides 64..512, 4..64 depth nodes) in one launch per pass, on torch's
    current stream.  eps_list[i] and out_list[i] have contexts[i].vol_shape; returns out_list."""
    import torch

    n = len(contexts)
    if n != len(eps_list) or (out_list is not None and n != len(out_list)):
        raise ValueError("one input and one output per context")
    if out_list is None:
        out_list = [torch.empty(c.vol_shape, dtype=c.dtype, device=e.device) for c, e in zip(contexts, eps_list)]
    k = FVIM_STRESS if kind == "stress" else FVIM_STRAIN
    arr = ctypes.c_void_p * max(n, 1)
    hs = arr(*[c._h.value for c in contexts])
    ins = arr(*[_ptr(e, c.dtype, c.vol_shape, "eps_p").value for c, e in zip(contexts, eps_list)])
    outs = arr(*[_ptr(o, c.dtype, c.vol_shape, "out").value for c, o in zip(contexts, out_list)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(lib().fvim_apply_mindlin_group(hs, n, ins, outs, k, stream), "fvim_apply_mindlin_group")
    return out_list


class Context:
    """One periodic half-space grid with its material, precision and plastic state.

    n1, n2: in-plane points (powers of two); z: depth nodes (z[0] = 0, increasing);
    L1, L2: cell lengths; precision: "fp32" or "fp64".
    """

    def __init__(self, n1, n2, z, L1=1.0, L2=1.0, precision="fp32", E=1.0, nu=0.3,
                 sigma_y=math.inf, E_h=0.0):
        import torch

        self.n1, self.n2 = int(n1), int(n2)
        z = np.ascontiguousarray(np.asarray(z, dtype=np.float64))
        self.z = z
        self.nz = int(z.size)
        self.L1, self.L2 = float(L1), float(L2)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        prec = FVIM_FP32 if precision == "fp32" else FVIM_FP64
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        torch.cuda.init()
        self._h = ctypes.c_void_p()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _check(lib().fvim_create(ctypes.byref(self._h), self.n1, self.n2, self.nz,
                                 z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 self.L1, self.L2, prec, stream), "fvim_create")
        self.set_material(E, nu, sigma_y, E_h)

    # -- plumbing -----------------------------------------------------------------
    def _stream(self):
        import torch

        _check(lib().fvim_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "fvim_set_stream")

    @property
    def vol_shape(self):
        return (self.nz, 6, self.n2, self.n1)

    @property
    def surf_shape(self):
        return (self.n2, self.n1)

    @property
    def scal_shape(self):
        return (self.nz, self.n2, self.n1)

    def profile(self, on=True):
        """Bracket every kernel launch with CUDA events on the context's stream."""
        _check(lib().fvim_profile_enable(self._h, 1 if on else 0), "fvim_profile_enable")

    def profile_read(self):
        """{kernel kind: (total ms, launches)} since the last read (synchronises)."""
        n = 16
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        _check(lib().fvim_profile_read(self._h, ms, cnt, n), "fvim_profile_read")
        out = {}
        for s in range(n):
            name = lib().fvim_profile_name(s)
            if name is None:
                break
            if cnt[s]:
                out[name.decode()] = (ms[s], cnt[s])
        return out

    def autotune(self, reps=20):
        """Time the depth kernel's chunk lengths and then whole applies with each in-plane FFT
        path built for this grid (on the current stream), and keep the fastest for this
        context and later ones of the same grid; returns the plan."""
        pl = Plan()
        self._stream()
        _check(lib().fvim_autotune(self._h, int(reps), ctypes.byref(pl)), "fvim_autotune")
        return pl.as_dict()

    @property
    def plan(self):
        pl = Plan()
        _check(lib().fvim_get_plan(self._h, ctypes.byref(pl)), "fvim_get_plan")
        return pl.as_dict()

    def set_plan(self, depth_chunk=0, fft_path="rows_cols", depth_ctas=2, depth_cutoff=18.0):
        """Force the depth chunk length (0: the default rule), the depth kernel's register budget
        (CTAs per SM: 2, or 3 where built), its chunk-scan cutoff eps_co (0: exact scan) and the
        in-plane FFT path (one of FFT_PATHS) on this context."""
        pl = Plan()
        pl.depth_chunk = int(depth_chunk)
        pl.depth_ctas = int(depth_ctas)
        pl.depth_cutoff = float(depth_cutoff)
        pl.fft_path = FFT_PATHS.index(fft_path)
        _check(lib().fvim_set_plan(self._h, ctypes.byref(pl)), "fvim_set_plan")

    def last_kernel_count(self):
        return lib().fvim_last_kernel_count(self._h)

    def close(self):
        if self._h:
            lib().fvim_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ----------------------------------------------------------------------
    def set_material(self, E, nu, sigma_y=math.inf, E_h=0.0):
        self.E, self.nu, self.sigma_y, self.E_h = float(E), float(nu), float(sigma_y), float(E_h)
        sy = self.sigma_y if math.isfinite(self.sigma_y) else 1e300
        _check(lib().fvim_set_material(self._h, self.E, self.nu, sy, self.E_h), "fvim_set_material")

    def apply_mindlin(self, eps_p, out=None, kind="stress", u3=None):
        import torch

        if out is None:
            out = torch.empty(self.vol_shape, dtype=self.dtype, device=eps_p.device)
        k = FVIM_STRESS if kind == "stress" else FVIM_STRAIN
        a = _ptr(eps_p, self.dtype, self.vol_shape, "eps_p")
        b = _ptr(out, self.dtype, self.vol_shape, "out")
        c = _ptr(u3, self.dtype, self.surf_shape, "u3")
        self._stream()
        _check(lib().fvim_apply_mindlin(self._h, a, b, k, c), "fvim_apply_mindlin")
        return out

    def apply_boussinesq(self, p, u3=None, vol=None, kind="stress"):
        k = FVIM_STRESS if kind == "stress" else FVIM_STRAIN
        a = _ptr(p, self.dtype, self.surf_shape, "p")
        b = _ptr(u3, self.dtype, self.surf_shape, "u3")
        c = _ptr(vol, self.dtype, self.vol_shape, "vol")
        self._stream()
        _check(lib().fvim_apply_boussinesq(self._h, a, b, c, k), "fvim_apply_boussinesq")
        return u3, vol

    def return_map(self, d_eps, d_eps_p, d_ep=None):
        a = _ptr(d_eps, self.dtype, self.vol_shape, "d_eps")
        b = _ptr(d_eps_p, self.dtype, self.vol_shape, "d_eps_p")
        c = _ptr(d_ep, self.dtype, self.scal_shape, "d_ep")
        self._stream()
        _check(lib().fvim_return_map(self._h, a, b, c), "fvim_return_map")
        return d_eps_p, d_ep

    def commit_state(self, d_eps, d_eps_p, d_ep):
        a = _ptr(d_eps, self.dtype, self.vol_shape, "d_eps")
        b = _ptr(d_eps_p, self.dtype, self.vol_shape, "d_eps_p")
        c = _ptr(d_ep, self.dtype, self.scal_shape, "d_ep")
        self._stream()
        _check(lib().fvim_commit_state(self._h, a, b, c), "fvim_commit_state")

    def get_state(self, eps_p=None, e_p=None, sigma=None):
        a = _ptr(eps_p, self.dtype, self.vol_shape, "eps_p")
        b = _ptr(e_p, self.dtype, self.scal_shape, "e_p")
        c = _ptr(sigma, self.dtype, self.vol_shape, "sigma")
        self._stream()
        _check(lib().fvim_get_state(self._h, a, b, c), "fvim_get_state")

    def set_state(self, eps_p=None, e_p=None, sigma=None):
        a = _ptr(eps_p, self.dtype, self.vol_shape, "eps_p")
        b = _ptr(e_p, self.dtype, self.scal_shape, "e_p")
        c = _ptr(sigma, self.dtype, self.vol_shape, "sigma")
        self._stream()
        _check(lib().fvim_set_state(self._h, a, b, c), "fvim_set_state")

    def sync(self):
        _check(lib().fvim_sync(self._h), "fvim_sync")

    def reset_state(self):
        self._stream()
        _check(lib().fvim_reset_state(self._h), "fvim_reset_state")

    # -- solvers ------------------------------------------------------------------
    def default_opts(self, **kw):
        o = Opts()
        _check(lib().fvim_default_opts(self._h, ctypes.byref(o)), "fvim_default_opts")
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def elastic_contact(self, h, W, p, opts=None, allow_not_converged=False):
        """Polonsky-Keer contact under load W; p: initial guess in, pressure out."""
        o = opts or self.default_opts()
        a = _ptr(h, self.dtype, self.surf_shape, "h")
        b = _ptr(p, self.dtype, self.surf_shape, "p")
        it = ctypes.c_int()
        err = ctypes.c_double()
        self._stream()
        st = lib().fvim_elastic_contact(self._h, a, float(W), b, ctypes.byref(o), ctypes.byref(it), ctypes.byref(err))
        if st != 0 and not (allow_not_converged and st == -5):
            raise FvimError(st, "fvim_elastic_contact")
        return it.value, err.value

    def plasticity_solve(self, dT, dE, deps_p=None, dep=None, opts=None):
        o = opts or self.default_opts()
        a = _ptr(dT, self.dtype, self.surf_shape, "dT")
        b = _ptr(dE, self.dtype, self.vol_shape, "dE")
        c = _ptr(deps_p, self.dtype, self.vol_shape, "deps_p")
        e = _ptr(dep, self.dtype, self.scal_shape, "dep")
        it = ctypes.c_int()
        res = ctypes.c_double()
        self._stream()
        _check(lib().fvim_plasticity_solve(self._h, a, b, c, e, ctypes.byref(o), ctypes.byref(it),
                                           ctypes.byref(res)), "fvim_plasticity_solve")
        return it.value, res.value

    def solve_contact(self, h, loads, p_out=None, opts=None, allow_not_converged=False):
        """Algorithm 1 over the load increments; returns the report as a dict."""
        o = opts or self.default_opts()
        a = _ptr(h, self.dtype, self.surf_shape, "h")
        b = _ptr(p_out, self.dtype, self.surf_shape, "p_out")
        L = (ctypes.c_double * len(loads))(*[float(x) for x in loads])
        rep = Report()
        self._stream()
        st = lib().fvim_solve_contact(self._h, a, L, len(loads), ctypes.byref(o), b, ctypes.byref(rep))
        if st != 0 and not (allow_not_converged and st == -5):
            raise FvimError(st, "fvim_solve_contact")
        return rep.as_dict()
