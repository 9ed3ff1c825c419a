"""Benchmark of the Mindlin-operator apply on the 512 x 512 x 64 operator workload.

One step = one apply of the discretised Mindlin operator (plastic strain -> stress,
all six components on every voxel: eigenstress, forward in-plane FFT, per-mode depth
operator, inverse FFT with the stress epilogue) on a seeded random plastic-strain
field (i.i.d. N(0, 1e-3^2) per voxel and component times exp(-z/0.1)), FP32, inputs
resident in HBM (402.7 MB in, 402.7 MB out: larger than the 129 MB L2, so no flush
is needed between steps).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead
(a bounded sample of the same workload, extrapolated to a full apply).
Multi-GPU (torchrun): one independent replica per rank ("replicas only"), value is
the sum of voxels over ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N1 = N2 = 512
NZ = 64
DEPTH = 0.4
E, NU = 1.0, 0.3
SEED = 1812
METRIC = "Mindlin-apply voxels/s"
UNIT = "voxel/s"
WORKLOAD = "mindlin_apply_512x512x64_fp32"
# algorithmic bytes per voxel of one kernel pass: read 6 FP32 values, write 6 FP32 values
# (each kernel of the apply reads and writes the whole field once; the apply as a whole
# needs the same 48 B/voxel)
ALG_BYTES_PER_VOXEL = 48.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """SM clock and clock-event (throttle) reasons during the timed region: read through NVML
    (read-only queries, one sample per millisecond from a host thread) where the library
    loads, else nvidia-smi every 100 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of NVML's public API
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
            "hw_power_brake_slowdown": 0x80}

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None
        self.nvml = None
        self.thread = None
        self.samples = []

    def _nvml_open(self):
        import ctypes

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(h)) != 0:
            return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx))  # NVML_CLOCK_SM
        return lib, h, reasons, mx.value

    def _poll(self):
        import ctypes

        lib, h, reasons, _ = self.nvml
        sm, r = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(sm)) == 0 and \
                    reasons(h, ctypes.byref(r)) == 0:
                self.samples.append((sm.value, r.value))
            time.sleep(0.001)

    def start(self):
        import threading

        try:
            self.nvml = self._nvml_open()
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.stop_flag = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            t_end = time.perf_counter() + 0.5
            while not self.samples and self.thread.is_alive() and time.perf_counter() < t_end:
                time.sleep(0.001)  # the first sample before the region
            self.samples.clear()
            return
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            if not self.samples:
                return None
            sm = [a for a, _ in self.samples]
            reasons = sorted(nm for nm, bit in self.BITS.items() if any(b & bit for _, b in self.samples))
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(self.nvml[3]), "reasons": reasons,
                    "samples": len(sm), "source": "nvml, 1 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 100 ms"}


def max_over_ranks(x, dist=None, device="cpu"):
    """Slowest rank's value (the timing of a replica run is the slowest replica's)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, steps, ms_max, world):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_gpu(args):
    import torch

    from paper_1811_11558_gb300 import Context, fvim, inputs

    ws, rank, local = _dist()
    if not os.path.exists(fvim.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    z = inputs.uniform_depth(NZ, DEPTH)
    ep = inputs.plastic_strain_field(N1, N2, z, seed=SEED + rank, dtype=np.float32)
    vox = N1 * N2 * NZ
    ctx = Context(N1, N2, z, 1.0, 1.0, precision="fp32", E=E, nu=NU)
    plan = ctx.autotune(reps=20)       # the depth kernel's tile plan for this grid
    d_in = torch.from_numpy(ep).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # --- device-resident timing -------------------------------------------------------
    for _ in range(args.warmup):
        ctx.apply_mindlin(d_in, d_out)
    kernels_per_step = ctx.last_kernel_count()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        ctx.apply_mindlin(d_in, d_out)
    t1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1)
    ms_max = max_over_ranks(ms, pg, "cuda")
    value = replica_throughput(vox, args.steps, ms_max, ws)

    # --- the same K steps again with one event between consecutive applies: median and
    # p99 of the duration of one apply
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    evs[0].record(stream)
    for i in range(args.steps):
        ctx.apply_mindlin(d_in, d_out)
        evs[i + 1].record(stream)
    barrier()
    per_apply = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)])
    apply_ms = {"median": round(float(np.median(per_apply)), 5), "p99": round(float(np.percentile(per_apply, 99)), 5)}

    # --- the same K steps again with every kernel bracketed by CUDA events on the
    # launching stream (recorded live by the library): per-kernel durations for the roofline
    ctx.profile_read()
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    for _ in range(args.steps):
        ctx.apply_mindlin(d_in, d_out)
    barrier()
    prof = ctx.profile_read()
    ctx.profile(False)

    # --- end to end through the same C-ABI call with host buffers -------------------
    # every step copies its input from pinned host memory, applies the operator and copies
    # the stress back.  Three streams form a pipeline over three buffer slots: the upload of
    # step i+1, the apply of step i and the download of step i-1 run at the same time (the
    # link carries both directions at once); events order each slot's reuse.
    h_in = torch.from_numpy(ep).pin_memory()
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    NS = 3
    d_ins = [d_in] + [torch.empty_like(d_in) for _ in range(NS - 1)]
    d_outs = [d_out] + [torch.empty_like(d_out) for _ in range(NS - 1)]
    h_outs = [torch.empty(h_in.shape, dtype=torch.float32).pin_memory() for _ in range(NS)]
    ev_in = [torch.cuda.Event() for _ in range(NS)]
    ev_cmp = [torch.cuda.Event() for _ in range(NS)]
    ev_out = [torch.cuda.Event() for _ in range(NS)]
    used = [False] * NS

    def e2e_step(i):
        j = i % NS
        with torch.cuda.stream(s_in):
            if used[j]:
                s_in.wait_event(ev_cmp[j])          # the apply of step i-3 has read d_ins[j]
            d_ins[j].copy_(h_in, non_blocking=True)
            ev_in[j].record(s_in)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev_in[j])
            if used[j]:
                s_cmp.wait_event(ev_out[j])         # the download of step i-3 has read d_outs[j]
            ctx.apply_mindlin(d_ins[j], d_outs[j])
            ev_cmp[j].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_cmp[j])
            h_outs[j].copy_(d_outs[j], non_blocking=True)
            ev_out[j].record(s_out)
        used[j] = True

    for i in range(max(NS, args.warmup // 2)):
        e2e_step(i)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    s_cmp.wait_event(e0)
    s_out.wait_event(e0)
    for i in range(args.steps):
        e2e_step(i)
    e1 = torch.cuda.Event(enable_timing=True)
    e1.record(s_out)
    barrier()
    ems = e0.elapsed_time(e1)
    e2e_value = replica_throughput(vox, args.steps, max_over_ranks(ems, pg, "cuda"), ws)
    assert all(np.isfinite(h[0, 0, :4, :4].numpy()).all() for h in h_outs)
    h_out = h_outs[0]

    # --- roofline of the dominant kernel ---------------------------------------------
    peak, peak_kind = _peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    avg_ms = dom_ms / dom_n
    alg_bytes = ALG_BYTES_PER_VOXEL * vox
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    roofline = {
        "bound": "hbm",
        "kernel": dom_name,
        "achieved": round(achieved, 1),
        "peak": peak,
        "peak_kind": peak_kind,
        "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": TRAFFIC_BYTES.get(dom_name) if (plan["depth_chunk"], plan["depth_ctas"]) == TRAFFIC_DEPTH_PLAN or
        dom_name != "mindlin_depth" else None,
        "alg_bytes": alg_bytes,
        "avg_launch_ms": round(avg_ms, 5),
    }
    kernel_ms = {k: round(v[0] / v[1], 5) for k, v in prof.items()}
    # every kernel of the apply moves the whole field once (48 B per voxel): its fraction of the
    # measured copy bandwidth
    kernel_frac = {k: round(alg_bytes / (v[0] / v[1] / 1e3) / 1e9 / peak, 4) for k, v in prof.items()}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n1": N1, "n2": N2, "nz": NZ, "depth": DEPTH, "output": "stress",
                   "voxels": vox, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs (402.7 MB) larger than L2, no flush"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h_in.numel() * 4),
                "d2h_bytes_per_step": int(h_out.numel() * 4),
                "pipeline": "pinned host -> device, apply, device -> pinned host every step; upload, "
                            "apply and download on three streams over three buffer slots"},
        "gpu_launches": kernels_per_step * args.steps,
        "apply_ms": apply_ms,
        "kernel_ms": kernel_ms,
        "kernel_hbm_frac": kernel_frac,
        "tile_plan": plan,
        "roofline": roofline,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_solves:
        line["solves"] = solve_metrics()
        line["solves"]["rough"] = rough_metrics()
        line["solves"]["stream"] = stream_metrics()
        line["solves"]["batch"] = batch_metrics()
        line["solves"]["epp_sweep"] = epp_metrics()
        line["scaling_sweep"] = scaling_metrics()
        line["group_apply"] = group_metrics()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def hertz_case():
    """Elastic-plastic Hertz contact: rigid paraboloid R = 0.5 in a unit cell, 32 x 32 surface
    points, 16 uniform depth nodes to z = 0.5, E = 1, nu = 0.3, sigma_y = 0.05 E*, E_h = 0.1 E,
    five equal increments up to the load of an elastic Hertz peak pressure of 3 sigma_y."""
    from paper_1811_11558_gb300 import inputs

    es = E / (1 - NU * NU)
    sy = 0.05 * es
    p0 = 3 * sy
    a = np.pi * 0.5 * p0 / (2 * es)
    wmax = 2 * np.pi * a * a * p0 / 3
    return dict(n=32, z=inputs.uniform_depth(16, 0.5), h=inputs.hertz_profile(32, 32, 1.0, 1.0, 0.5),
                loads=[wmax * (k + 1) / 5 for k in range(5)], sigma_y=sy, E_h=0.1 * E)


def solve_metrics(repeats=3, served=32, slots=16):
    """Contact solves/s of Algorithm 1 (relaxation 0.5) on the Hertz case: FP64 and FP32 one
    solve at a time, and FP32 served (requests admitted as slots free up, solves overlapping on
    the device), with p50/p99 latency and the FP32 error against the FP64 solution; first with
    the listing's relaxation order, then (``relax_carried``) with the relaxed value carried
    between coupling iterations."""
    import torch

    from paper_1811_11558_gb300 import Context
    from paper_1811_11558_gb300.serve import Request, Server, percentiles

    c = hertz_case()

    def run(mode):
        out = {"workload": "hertz_32x32x16_5inc", "relax": 0.5, "relax_mode": ("literal", "carried")[mode]}
        press = {}
        for prec in ("fp64", "fp32"):
            ctx = Context(c["n"], c["n"], c["z"], 1.0, 1.0, precision=prec, E=E, nu=NU, sigma_y=c["sigma_y"],
                          E_h=c["E_h"])
            ctx.autotune()
            h = torch.from_numpy(c["h"]).to("cuda", ctx.dtype)
            p = torch.empty(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
            opts = ctx.default_opts(relax=0.5, max_iter=400, relax_mode=mode)
            times, rep = [], None
            for r in range(repeats + 1):
                ctx.reset_state()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = ctx.solve_contact(h, c["loads"], p, opts)
                times.append(time.perf_counter() - t0)
            t = float(np.median(times[1:]))
            press[prec] = p.cpu().numpy().astype(np.float64)
            out[prec + "_plain"] = {"solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t, "tol": opts.tol,
                                    "alg1_iters": rep["alg1_iters"], "contact_area": rep["contact_area"][-1]}
            ctx.close()
        srv = Server(slots=slots)
        reqs = [Request(i, c["n"], c["z"], c["h"], c["loads"], precision="fp32", E=E, nu=NU, sigma_y=c["sigma_y"],
                        E_h=c["E_h"], opts={"relax": 0.5, "max_iter": 400, "relax_mode": mode})
                for i in range(served)]
        srv.prepare(reqs[:1])                       # the grid's tuned tile plan
        srv.run(reqs[:slots])                       # warm the context pool
        res, wall = srv.run(reqs)
        lat = percentiles([r.latency for r in res])
        out["fp32_served"] = {"solves_per_s": served / wall, "slots": slots, "requests": served,
                              "p50_ms": 1e3 * lat[50], "p99_ms": 1e3 * lat[99], "arrivals": "all at t = 0"}
        out["fp32_vs_fp64"] = {
            "pressure_rel_l2": float(np.linalg.norm(press["fp32"] - press["fp64"]) / np.linalg.norm(press["fp64"])),
            "area_diff": float(abs((press["fp32"] > 0).mean() - (press["fp64"] > 0).mean()))}
        out["served_over_fp64_plain"] = out["fp32_served"]["solves_per_s"] / out["fp64_plain"]["solves_per_s"]
        return out

    out = run(0)
    out["relax_carried"] = run(1)
    return out


def rough_metrics(n=1024, nz=32, depth=0.05, seed=1813, n_inc=10, cap=120):
    """Algorithm 1 on a rough surface, FP32: seeded self-affine surface n x n (H = 0.8, flat PSD
    for 4 <= |k| < 8, power law to k_s = 64, rms slope 0.1), nz uniform nodes to the given
    depth, sigma_y = 0.05 E*, E_h = 0.1 E, relaxation 0.3.  (a) the paper's rough-surface load
    W = 1e-3 E x rms slope in five increments (Algorithm 1 in the listing's order, tolerance
    1e-6), and the same with the relaxed value carried between coupling iterations; (b) the load of a 10 % elastic contact fraction, ramped in n_inc equal increments (the
    paper's remedy for the coupling's slow convergence on rough surfaces: small load steps),
    Algorithm 1 with the relaxed value carried between iterations (relax_mode 1), tolerance 1e-7,
    capped at ``cap`` iterations per increment.  Both are timed as whole solves; the status says whether every increment
    reached the tolerance."""
    import torch

    from paper_1811_11558_gb300 import Context, inputs

    es = E / (1 - NU * NU)
    z = inputs.uniform_depth(nz, depth)
    h = inputs.self_affine_surface(n, 1.0, 0.8, 4, 8, 64, 0.1, seed=seed)
    ctx = Context(n, n, z, 1.0, 1.0, precision="fp32", E=E, nu=NU, sigma_y=0.05 * es, E_h=0.1 * E)
    ctx.autotune()
    hd = torch.from_numpy(h).to("cuda", torch.float32)
    p = torch.zeros(ctx.surf_shape, dtype=torch.float32, device="cuda")
    out = {"workload": "rough_%dx%dx%d_fp32" % (n, n, nz), "depth": depth, "seed": seed}
    W = 1e-3 * E * 0.1
    # FP32: the coupling error floors near 1e-7..1e-6 once the plastic zone is large (the inner
    # DF-SANE solves stop at the FP32 rounding floor of the residual), so 1e-6 here
    opts = ctx.default_opts(relax=0.3, max_iter=cap, tol=1e-6)
    ctx.reset_state()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve_contact(hd, [W * (k + 1) / 5 for k in range(5)], p, opts, allow_not_converged=True)
    t = time.perf_counter() - t0
    out["paper_load"] = {"W": W, "increments": 5, "relax": 0.3, "tol": opts.tol, "status": rep["status"],
                         "solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t, "alg1_iters": rep["alg1_iters"],
                         "alg1_error": rep["alg1_error"], "contact_area": rep["contact_area"][-1],
                         "residual_evals": rep["residual_evals"], "cg_iters": rep["cg_iters"]}
    # the same solve with the relaxed value carried between coupling iterations
    optc = ctx.default_opts(relax=0.3, max_iter=cap, tol=1e-6, relax_mode=1)
    ctx.reset_state()
    p.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve_contact(hd, [W * (k + 1) / 5 for k in range(5)], p, optc, allow_not_converged=True)
    t = time.perf_counter() - t0
    out["paper_load_carried"] = {"W": W, "increments": 5, "relax": 0.3, "relax_mode": "carried", "tol": optc.tol,
                                 "status": rep["status"], "solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t,
                                 "alg1_iters": rep["alg1_iters"], "alg1_error": rep["alg1_error"],
                                 "contact_area": rep["contact_area"][-1]}
    # load of a 10 % elastic contact fraction (area ~ linear in the load at small fractions)
    p.zero_()
    ctx.elastic_contact(hd, 5e-3, p, ctx.default_opts())
    W10 = 5e-3 * 0.1 / float((p > 0).double().mean())
    # with the listing's update order the coupling stalls near 1e-5..1e-3 on this load in FP32
    # and FP64 alike; the relaxed value carried between iterations converges in ~21 per increment
    opts10 = ctx.default_opts(relax=0.3, max_iter=cap, tol=1e-7, relax_mode=1)
    ctx.reset_state()
    p.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve_contact(hd, [W10 * (k + 1) / n_inc for k in range(n_inc)], p, opts10, allow_not_converged=True)
    t = time.perf_counter() - t0
    its = sum(rep["alg1_iters"])
    out["area_10pct"] = {"W": W10, "increments": n_inc, "relax": 0.3, "relax_mode": "carried", "tol": opts10.tol,
                         "alg1_cap": cap,
                         "status": rep["status"], "converged_increments": sum(
                             1 for e in rep["alg1_error"] if e < opts10.tol),
                         "solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t, "ms_per_alg1_iter": 1e3 * t / its,
                         "alg1_iters": rep["alg1_iters"], "alg1_error": rep["alg1_error"],
                         "contact_area": rep["contact_area"][-1]}
    ctx.close()
    return out


def epp_loads():
    """W / W_y of the paper's elastic-perfectly-plastic Hertz sweep (App. C.2): 20 values
    spread evenly over [0.9, 15.5] together with 1, 2.1, 6.4 and 15.5, sorted (monotonic
    loading), without the repeated 15.5."""
    return sorted(set(np.round(np.linspace(0.9, 15.5, 20), 12).tolist()) | {1.0, 2.1, 6.4, 15.5})


def epp_metrics(n=81, nz=32, a_y_over_L=0.05, relax=0.5, cap=200, n64=4):
    """Elastic-perfectly-plastic Hertz load sweep at the paper's discretisation (App. C.2): cell
    [0, 20 R / 3]^2 x [0, 10 R / 3] with L = 1 (R = 0.15, depth 0.5), N = (81, 81, 32), nu = 0.3,
    E_h = 0, W / W_y over epp_loads() one increment each (the state carries over), relaxation
    0.5.  The paper leaves sigma_y free (normalised results do not depend on it); here it is set
    so that the onset contact radius a_y = pi R p_y / (2 E*) (p_y = 1.6 sigma_y) is a_y_over_L
    of the cell.  The whole sweep runs in FP32 (Algorithm 1 to 1e-7: with E_h = 0 the FP32 coupling
    error stalls between 1e-8 and 1e-6 on the heavier loads); plain FP64 (Algorithm 1 to 1e-9,
    the paper's tolerance) runs the first n64 loads, and the two
    pressures and contact areas are compared after that load.  Reports per load the peak
    pressure over sigma_y, the contact radius over a_y (from the contact area), the peak
    plastic strain and the coupling iterations."""
    import torch

    from paper_1811_11558_gb300 import Context, inputs

    es = E / (1 - NU * NU)
    R = 0.15
    a_y = a_y_over_L
    p_y = 2 * es * a_y / (np.pi * R)
    sy = p_y / 1.6
    w_y = np.pi ** 3 * R ** 2 * p_y ** 3 / (6 * es ** 2)
    loads = epp_loads()
    z = inputs.uniform_depth(nz, 10 * R / 3)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, R)
    out = {"workload": "epp_hertz_%dx%dx%d" % (n, n, nz), "W_over_W_y": loads, "relax": relax, "R": R,
           "sigma_y_over_E_star": sy / es, "a_y": a_y, "W_y": w_y}
    press = {}
    for prec, nl in (("fp32", len(loads)), ("fp64", n64)):
        ctx = Context(n, n, z, 1.0, 1.0, precision=prec, E=E, nu=NU, sigma_y=sy, E_h=0.0)
        ctx.autotune()
        hd = torch.from_numpy(h).to("cuda", ctx.dtype)
        p = torch.zeros(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
        opts = ctx.default_opts(relax=relax, max_iter=cap, **({"tol": 1e-7} if prec == "fp32" else {}))
        rows = []
        ep = torch.empty(ctx.scal_shape, dtype=ctx.dtype, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, r in enumerate(loads[:nl]):   # one increment per call (the state carries over)
            rep = ctx.solve_contact(hd, [r * w_y], p, opts, allow_not_converged=True)
            ctx.get_state(None, ep, None)
            area = rep["contact_area"][-1]
            rows.append({"W_over_W_y": r, "p_max_over_sigma_y": float(p.max()) / sy,
                         "a_over_a_y": float(np.sqrt(area / np.pi)) / a_y, "e_p_max": float(ep.max()),
                         "alg1_iters": rep["alg1_iters"][-1], "alg1_error": rep["alg1_error"][-1],
                         "status": rep["status"]})
            if k + 1 == n64:
                press[prec] = p.cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        out[prec] = {"ms": 1e3 * (time.perf_counter() - t0), "loads": nl, "tol": opts.tol,
                     "converged": sum(1 for q in rows if q["status"] == 0), "increments": rows}
        ctx.close()
    out["fp32_vs_fp64_at_load"] = loads[n64 - 1]
    out["fp32_vs_fp64_pressure_rel_l2"] = float(np.linalg.norm(press["fp32"] - press["fp64"]) /
                                                np.linalg.norm(press["fp64"]))
    out["fp32_vs_fp64_area_diff"] = abs(float((press["fp32"] > 0).mean()) - float((press["fp64"] > 0).mean()))
    return out


def batch_problems(n_prob=64, seed=1814):
    """Uneven elastic-plastic contact problems: grids n^2 with n drawn from {64, 128, 256, 512},
    nz from {8, 16, 32}; half paraboloids (R = 0.5, depth 0.5), half seeded self-affine surfaces
    (H uniform in [0.6, 0.9], flat PSD for 4 <= |k| < 8, power law to k_s = max(8, n / 16),
    rms slope 0.1, depth 0.05); total load log-uniform over the decade below the load of a 10 %
    elastic contact fraction (Hertz: pi a^2 = 0.1, W = 4 E* a^3 / (3 R); rough: mean pressure
    0.1 E* slope / 2), five increments (Hertz) or ten (rough); sigma_y = 0.05 E*, E_h = 0.1 E;
    Algorithm 1 with the relaxed value carried between iterations (relax_mode 1: the listing's
    order stalls on rough loads and needs two to three times the iterations on Hertz loads) at
    relaxation 0.5 (Hertz) and 0.3 (rough)."""
    from paper_1811_11558_gb300 import inputs

    rng = np.random.Generator(np.random.PCG64(seed))
    es = E / (1 - NU * NU)
    probs = []
    for i in range(n_prob):
        n = int(2 ** rng.integers(6, 10))
        nz = int(rng.choice([8, 16, 32]))
        rough = bool(rng.integers(0, 2))
        u = float(rng.uniform(-1.0, 0.0))
        if rough:
            hurst = float(rng.uniform(0.6, 0.9))
            h = inputs.self_affine_surface(n, 1.0, hurst, 4, 8, max(8, n // 16), 0.1, seed=seed + 1 + i)
            z = inputs.uniform_depth(nz, 0.05)
            w10 = 0.1 * es * 0.1 / 2.0
            relax, mode = 0.3, 1
        else:
            h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.5)
            z = inputs.uniform_depth(nz, 0.5)
            a = np.sqrt(0.1 / np.pi)
            w10 = 4.0 * es * a ** 3 / (3.0 * 0.5)
            relax, mode = 0.5, 1
        W = w10 * 10.0 ** u
        ninc = 10 if rough else 5   # small load steps on rough surfaces (the paper's remedy)
        probs.append({"n": n, "nz": nz, "rough": rough, "z": z, "h": h,
                      "loads": [W * (k + 1) / ninc for k in range(ninc)], "relax": relax, "relax_mode": mode})
    return probs


def batch_metrics(n_prob=64, slots=16, seed=1814, max_iter=80, n64=4):
    """Batched uneven solves: n_prob problems (batch_problems) submitted at once to the
    server (slots contexts, one stream and one set of captured graphs each, FP32 operators,
    FP64 reductions), aggregate solves/s and per-problem latency; plain FP64 and FP32 one at a
    time on the first n64 problems of the smallest grid, with the FP32 pressure error."""
    import torch

    from paper_1811_11558_gb300 import Context
    from paper_1811_11558_gb300.serve import Request, Server, percentiles

    es = E / (1 - NU * NU)
    probs = batch_problems(n_prob, seed)

    def req(i, pb, prec="fp32"):
        return Request(i, pb["n"], pb["z"], pb["h"], pb["loads"], precision=prec, E=E, nu=NU, sigma_y=0.05 * es,
                       E_h=0.1 * E, opts={"relax": pb["relax"], "relax_mode": pb["relax_mode"],
                                                         "max_iter": max_iter})

    srv = Server(slots=slots)
    t0 = time.perf_counter()
    plans = srv.prepare([req(i, pb) for i, pb in enumerate(probs)])   # one tuned context per shape
    prep_s = time.perf_counter() - t0
    seen, warm = set(), []
    for i, pb in enumerate(probs):          # one request per shape warms the context pool
        key = (pb["n"], pb["nz"], pb["rough"])
        if key not in seen:
            seen.add(key)
            warm.append(req(i, pb))
    srv.run(warm)
    res, wall = srv.run([req(i, pb) for i, pb in enumerate(probs)])
    lat = percentiles([r.latency for r in res])
    conv = sum(1 for r in res if r.report.get("status", 0) == 0)
    small = [i for i, pb in enumerate(probs) if pb["n"] == min(q["n"] for q in probs)][:n64]
    t = {"fp64": [], "fp32": []}
    err, darea = [], []
    for i in small:
        pb = probs[i]
        press = {}
        for prec in ("fp64", "fp32"):
            ctx = Context(pb["n"], pb["n"], pb["z"], 1.0, 1.0, precision=prec, E=E, nu=NU, sigma_y=0.05 * es,
                          E_h=0.1 * E)
            ctx.autotune()
            hd = torch.from_numpy(np.ascontiguousarray(pb["h"])).to("cuda", ctx.dtype)
            p = torch.empty(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_contact(hd, pb["loads"], p, ctx.default_opts(relax=pb["relax"], relax_mode=pb["relax_mode"],
                                                                    max_iter=max_iter),
                              allow_not_converged=True)
            t[prec].append(time.perf_counter() - t0)
            press[prec] = p.cpu().numpy().astype(np.float64)
            ctx.close()
        err.append(float(np.linalg.norm(press["fp32"] - press["fp64"]) / np.linalg.norm(press["fp64"])))
        darea.append(abs(float((press["fp32"] > 0).mean()) - float((press["fp64"] > 0).mean())))
    return {"workload": "batch_%d_uneven" % n_prob, "grids": sorted({pb["n"] for pb in probs}),
            "nz": sorted({pb["nz"] for pb in probs}), "rough": sum(pb["rough"] for pb in probs),
            "slots": slots, "alg1_cap": max_iter, "converged": conv, "unconverged": n_prob - conv,
            "unconverged_problems": [{"i": i, "n": pb["n"], "nz": pb["nz"], "rough": pb["rough"],
                                      "iters": r.report.get("alg1_iters"), "errors": r.report.get("alg1_error")}
                                     for i, (pb, r) in enumerate(zip(probs, res))
                                     if r.report.get("status", 0) != 0],
            "tile_plans": {"shapes": len(plans), "tuning_s": prep_s,
                           "depth_chunk": sorted({(p["n"], p["nz"], p["depth_chunk"]) for p in plans.values()})},
            "fp32_served": {"solves_per_s": conv / wall, "counted": "converged solves only", "wall_s": wall,
                            "all_solves_per_s": n_prob / wall, "p50_ms": 1e3 * lat[50], "p99_ms": 1e3 * lat[99],
                            "arrivals": "all at t = 0"},
            "sample_n%d" % probs[small[0]]["n"] if small else "sample": {
                "problems": small, "fp64_plain_ms": [1e3 * x for x in t["fp64"]],
                "fp32_plain_ms": [1e3 * x for x in t["fp32"]], "fp32_vs_fp64_pressure_rel_l2": err,
                "fp32_vs_fp64_area_diff": darea},
            "per_problem": [{"n": pb["n"], "nz": pb["nz"], "rough": pb["rough"], "ms": 1e3 * (r.finished - r.admitted),
                             "status": r.report.get("status", 0), "iters": r.report.get("alg1_iters")}
                            for pb, r in zip(probs, res)]}


def stream_metrics(n_req=8, slots=8, seed=1815, n_inc=3, n64_max=256):
    """Served request stream, FP32 vs plain FP64: requests with grids n^2, n drawn uniformly in
    log2 from {128, 256, 512, 1024}, nz = round(16 x 4^U) in [16, 64] (U uniform), seeded
    self-affine surfaces (H 0.8, rms slope 0.1, depth 0.05), load ramps of n_inc increments to
    the paper's rough-surface load, relaxation 0.3, the default tolerances of each precision
    (Algorithm 1: 1e-8 FP32, 1e-9 FP64).
    Passes: every request alone, one at a time (the single-stream capacity and each request's
    FP32 plain time); Poisson arrivals at 0.7 x that capacity; all requests at t = 0 (saturated).
    p50 / p99 latency from arrival to result.  Plain FP64 solves the requests of grids up to
    n64_max one at a time (a stated subsample: a 1024^2 x 64 FP64 solve takes minutes); its
    per-request time, and the pressure error and contact-area difference of the FP32 result, are
    reported beside the FP32 plain time of the same request."""
    import torch

    from paper_1811_11558_gb300 import Context, inputs
    from paper_1811_11558_gb300.serve import Request, Server, percentiles, poisson_arrivals

    rng = np.random.Generator(np.random.PCG64(seed))
    es = E / (1 - NU * NU)
    W = 1e-3 * E * 0.1
    specs = []
    for i in range(n_req):
        n = int(2 ** rng.integers(7, 11))
        nz = int(round(16 * 4 ** rng.uniform(0, 1)))
        specs.append((i, n, nz))

    def make(i, n, nz, arrival=0.0):
        z = inputs.uniform_depth(nz, 0.05)
        h = inputs.self_affine_surface(n, 1.0, 0.8, 4, 8, min(64, n // 4), 0.1, seed=seed + 1 + i)
        return Request(i, n, z, h, [W * (k + 1) / n_inc for k in range(n_inc)], precision="fp32", E=E, nu=NU,
                       sigma_y=0.05 * es, E_h=0.1 * E, opts={"relax": 0.3, "max_iter": 150}, arrival=arrival)

    srv = Server(slots=slots)
    srv.prepare([make(*sp) for sp in specs])            # tuned tile plan per shape
    seen, warm = set(), []
    for sp in specs:                                    # one request per shape warms the pool
        if (sp[1], sp[2]) not in seen:
            seen.add((sp[1], sp[2]))
            warm.append(make(*sp))
    srv.run(warm)
    # single stream: one request at a time
    t0 = time.perf_counter()
    one = [srv.solve(make(*sp)) for sp in specs]
    t_one = time.perf_counter() - t0
    cap = n_req / t_one
    res, wall = srv.run([make(*sp, arrival=float(a)) for sp, a in zip(specs, poisson_arrivals(n_req, 0.7 * cap, seed))])
    lat = percentiles([r.latency for r in res])
    sat, swall = srv.run([make(*sp) for sp in specs])
    slat = percentiles([r.latency for r in sat])
    conv = {"poisson": sum(1 for r in res if r.report.get("status", 0) == 0),
            "saturated": sum(1 for r in sat if r.report.get("status", 0) == 0)}
    # plain FP64 on the subsample, one at a time
    sub = []
    for sp, o in zip(specs, one):
        i, n, nz = sp
        if n > n64_max:
            continue
        r = make(*sp)
        ctx = Context(n, n, r.z, 1.0, 1.0, precision="fp64", E=E, nu=NU, sigma_y=r.sigma_y, E_h=r.E_h)
        ctx.autotune()
        hd = torch.from_numpy(np.ascontiguousarray(r.h)).to("cuda", torch.float64)
        p = torch.zeros(ctx.surf_shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.solve_contact(hd, r.loads, p, ctx.default_opts(relax=0.3, max_iter=150), allow_not_converged=True)
        t64 = time.perf_counter() - t0
        p64 = p.cpu().numpy()
        ctx.close()
        p32 = o.pressure.astype(np.float64)
        sub.append({"i": i, "n": n, "nz": nz, "fp64_plain_ms": 1e3 * t64, "fp32_plain_ms": 1e3 * (o.finished - o.admitted),
                    "fp64_status": rep["status"], "fp32_status": o.report.get("status", 0),
                    "fp32_vs_fp64_pressure_rel_l2": float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64)),
                    "fp32_vs_fp64_area_diff": abs(float((p32 > 0).mean()) - float((p64 > 0).mean()))})
    t64s = sum(x["fp64_plain_ms"] for x in sub)
    t32s = sum(x["fp32_plain_ms"] for x in sub)
    return {"workload": "rough_stream_%dreq" % n_req, "requests": [{"i": i, "n": n, "nz": nz} for i, n, nz in specs],
            "increments": n_inc, "slots": slots, "converged": conv,
            "single_stream_fp32_solves_per_s": cap, "arrival_rate_per_s": 0.7 * cap,
            "fp32_served_poisson": {"solves_per_s": conv["poisson"] / wall, "p50_ms": 1e3 * lat[50],
                                    "p99_ms": 1e3 * lat[99]},
            "fp32_served_saturated": {"solves_per_s": conv["saturated"] / swall, "p50_ms": 1e3 * slat[50],
                                      "p99_ms": 1e3 * slat[99]},
            "fp64_plain_subsample": {"grids_up_to": n64_max, "requests": sub,
                                     "fp64_over_fp32_plain_time": (t64s / t32s) if t32s > 0 else None}}


def group_metrics(n_prob=64, seed=1814, reps=10):
    """The operator work of the uneven batch in one launch per pass: the Mindlin apply (stress
    output) of the n_prob problems of batch_problems (grids 64^2..512^2, Nz 8..32, their own
    depth nodes and cells, FP32, seeded plastic-strain fields) through
    fvim_apply_mindlin_group, five launches for all problems, replayed from a CUDA graph;
    beside it the same applies issued problem by problem (five launches each) replayed from
    one CUDA graph, every context on the same depth plan (chunk length 4, row / column FFTs).
    The problems' fields (several GB) are far larger than L2, so no flush is needed between
    replays.  CUDA events on the replay stream; 48 B per voxel (eps_p read, stress written) is
    the algorithmic traffic of an apply."""
    import torch

    from paper_1811_11558_gb300 import Context, fvim, inputs

    peak, peak_kind = _peaks()
    probs = batch_problems(n_prob, seed)
    ctxs, eps, outs = [], [], []
    for i, pb in enumerate(probs):
        c = Context(pb["n"], pb["n"], pb["z"], 1.0, 1.0, precision="fp32", E=E, nu=NU)
        c.set_plan(depth_chunk=4, fft_path="rows_cols", depth_ctas=2)
        ctxs.append(c)
        eps.append(torch.from_numpy(inputs.plastic_strain_field(pb["n"], pb["n"], pb["z"], seed=seed + 100 + i,
                                                                dtype=np.float32)).to("cuda"))
        outs.append(torch.empty_like(eps[-1]))
    vox = sum(c.n1 * c.n2 * c.nz for c in ctxs)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                 # first calls outside any capture
        fvim.apply_mindlin_group(ctxs, eps, outs)
        for c, e, o in zip(ctxs, eps, outs):
            c.apply_mindlin(e, o)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g_grp, g_seq = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_grp, capture_error_mode="thread_local"):
        fvim.apply_mindlin_group(ctxs, eps, outs)
    with torch.cuda.graph(g_seq, capture_error_mode="thread_local"):
        for c, e, o in zip(ctxs, eps, outs):
            c.apply_mindlin(e, o)

    def timed(g):
        for _ in range(3):
            g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_seq = timed(g_seq)
    ref = [o.clone() for o in outs]
    t_grp = timed(g_grp)
    diff = max(float((o - r).norm() / r.norm()) for o, r in zip(outs, ref))
    for c in ctxs:
        c.close()
    shapes = sorted({(c.n1, c.nz) for c in ctxs})
    return {"workload": "group_%d_uneven_mindlin_fp32" % n_prob, "problems": n_prob, "shapes": len(shapes),
            "voxels": vox, "l2": "inputs larger than L2 (%.1f GB per apply)" % (vox * 48e-9),
            "group": {"ms": t_grp, "voxels_per_s": vox / (t_grp * 1e-3), "launches": 5,
                      "hbm_frac": vox * ALG_BYTES_PER_VOXEL / (t_grp * 1e-3) / (peak * 1e9), "peak": peak_kind},
            "per_problem_graph": {"ms": t_seq, "voxels_per_s": vox / (t_seq * 1e-3), "launches": 5 * n_prob},
            "group_speedup": t_seq / t_grp,
            "group_vs_per_problem_rel_l2_max": diff}


def scaling_metrics(sizes=(4, 8, 16, 32, 64, 128), reps=20):
    """Mindlin-apply time and device memory on N x N x N grids (the paper's VIM complexity
    sweep, App. C.4, whose reference time T0 = 1.41 ms and memory 1.27 GB at 2^21 nodes were
    measured on a CPU node), FP32 and FP64, CUDA events, inputs resident.

    Memory: ``apply_bytes`` is what one apply touches on the device (input eps_p, output
    sigma, the context's half-spectrum scratch with its Nyquist side array, twiddles and depth
    nodes); ``context_bytes`` is the device memory the context itself took when it was
    created (its scratch plus the plastic state it keeps for the solvers), measured with
    cudaMemGetInfo around the creation."""
    import torch

    from paper_1811_11558_gb300 import Context, inputs

    out = {"workload": "mindlin_apply_cube_sweep", "paper_T0_ms_cpu": 1.41, "paper_memory_gb_128": 1.27,
           "ms": {}, "apply_bytes": {}, "context_bytes": {}}
    for prec in ("fp32", "fp64"):
        es = 4 if prec == "fp32" else 8
        for n in sizes:
            z = inputs.uniform_depth(n, 1.0)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            ctx = Context(n, n, z, 1.0, 1.0, precision=prec, E=E, nu=NU)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            ctx.autotune()
            ep = torch.from_numpy(inputs.plastic_strain_field(n, n, z, seed=n)).to("cuda", ctx.dtype)
            o = torch.empty_like(ep)
            for _ in range(3):
                ctx.apply_mindlin(ep, o)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(reps):
                ctx.apply_mindlin(ep, o)
            e.record()
            torch.cuda.synchronize()
            key = "%s_%d" % (prec, n)
            out["ms"][key] = s.elapsed_time(e) / reps
            vol = 6 * n * n * n * es
            spec = n * 6 * n * (n // 2) * 2 * es + n * 6 * n * es
            out["apply_bytes"][key] = int(2 * vol + spec + 2 * n * 2 * es + n * es)
            out["context_bytes"][key] = int(free0 - free1)
            ctx.close()
    return out


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of each kernel on this
# workload, from one capture of the current kernels (profiles/ summaries); a kernel missing
# here, or changed since its capture, reports null.
TRAFFIC_DEPTH_PLAN = (4, 2)  # depth tile plan of that capture (chunk length, CTAs per SM)
TRAFFIC_BYTES = {"rows_fwd6": 755.3e6, "cols_fwd": 744.3e6, "mindlin_depth": 743.9e6, "cols_inv": 744.3e6,
                 "rows_inv6": 756.2e6}




def _oracle_job(planes, modes, seed):
    """One bounded sample of the FP64 oracle's Mindlin apply on the operator workload.

    Hooke's law and forward and inverse DFT of ``planes`` (layer, component) planes of a
    plastic strain field drawn like the workload's (first layers of the depth envelope), and
    the per-mode depth operator on ``modes`` random resolved modes of the 512 x 512 grid.
    Returns the two measured times and the number of modes kept; input generation is not
    timed.
    """
    from oracle import operators as op
    from oracle import tensors as T
    from paper_1811_11558_gb300 import inputs

    z = inputs.uniform_depth(NZ, DEPTH)
    nl = -(-planes // 6)
    ep = inputs.plastic_strain_field(N1, N2, z[:nl], seed=seed)
    lam, mu = T.lame(E, NU)
    rng = np.random.default_rng(seed)
    Q1, Q2, nyq, zero = op.mode_grid(N1, N2, 1.0, 1.0)
    k2 = rng.integers(0, N2, modes)
    k1 = rng.integers(0, N1, modes)
    keep = ~(nyq[k2, k1] | zero[k2, k1])
    k1, k2 = k1[keep], k2[keep]
    W = (rng.standard_normal((k1.size, NZ, 3, 3)) + 1j * rng.standard_normal((k1.size, NZ, 3, 3))) * 1e-3
    W = 0.5 * (W + np.swapaxes(W, -1, -2))
    Q = np.stack([Q1[k2, k1], Q2[k2, k1]], axis=1)
    t0 = time.perf_counter()
    w = T.hooke6(ep, lam, mu, axis=1).reshape(nl * 6, N2, N1)[:planes]
    back = np.fft.ifft2(np.fft.fft2(w, axes=(-2, -1)), axes=(-2, -1)).real
    t_fft = time.perf_counter() - t0
    assert back.shape == w.shape
    op._MODE_CACHE.clear()
    t1 = time.perf_counter()
    op.mindlin_modes(W, Q, z, E, NU)
    t_modes = time.perf_counter() - t1
    return t_fft, t_modes, int(k1.size)


def _oracle_worker(inq, outq):
    """Spawned worker: runs oracle sample jobs until it receives None."""
    outq.put("ready")
    while True:
        job = inq.get()
        if job is None:
            return
        outq.put(_oracle_job(*job))


# one BLAS / OpenMP thread per worker process, so that "cores" counts processes
_ONE_THREAD_ENV = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                    "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")}


class OracleWorkers:
    """A set of spawned single-threaded processes that run oracle sample jobs at the same time
    (spawned, never forked: the parent may hold a CUDA context)."""

    def __init__(self, n):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in _ONE_THREAD_ENV}
        os.environ.update(_ONE_THREAD_ENV)
        try:
            self.q = [(ctx.Queue(), ctx.Queue()) for _ in range(n)]
            self.p = [ctx.Process(target=_oracle_worker, args=qq, daemon=True) for qq in self.q]
            for p in self.p:
                p.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for _, outq in self.q:
            assert outq.get(timeout=600) == "ready"

    def run(self, jobs):
        """One job per worker (len(jobs) <= workers), all started together."""
        for (inq, _), job in zip(self.q, jobs):
            inq.put(job)
        return [outq.get(timeout=1800) for (_, outq), _ in zip(self.q, jobs)]

    def close(self):
        for inq, _ in self.q:
            inq.put(None)
        for p in self.p:
            p.join(timeout=60)


def _full_apply_s(t_fft, t_modes, planes, kept):
    """Extrapolation of one sample to a whole apply: 384 planes each way, 131 072 modes."""
    return t_fft * (NZ * 6) / planes + t_modes * (N1 * (N2 // 2)) / kept


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(planes=12, modes=160, seed=SEED, workers=None):
    """Time the FP64 oracle on the host cores: one single-threaded process alone (the 1-core
    figure), then one single-threaded process per core, all at once, each on its own sample
    (the all-core figure); every sample is extrapolated to a whole apply (_full_apply_s)."""
    n = host_cores()
    own = workers is None
    w = workers or OracleWorkers(n)
    try:
        t1 = w.run([(planes, modes, seed)])[0]
        one = _full_apply_s(t1[0], t1[1], planes, t1[2])
        res = w.run([(planes, modes, seed + 1 + i) for i in range(n)])
        each = [_full_apply_s(r[0], r[1], planes, r[2]) for r in res]
    finally:
        if own:
            w.close()
    vox = N1 * N2 * NZ
    return {
        "value": n * vox / float(np.mean(each)),
        "unit": UNIT,
        "cores": n,
        "nproc": n,
        "kind": "oracle",
        "one_core": {"value": vox / one, "unit": UNIT, "cores": 1},
        "sample": "FP64 oracle (numpy, one BLAS thread per process): per process Hooke + DFT of %d of 384 "
                  "planes each way + per-mode depth quadrature on %d random modes, extrapolated to one "
                  "512x512x64 apply (%.0f s on one core alone); all-core = %d such processes at once"
                  % (planes, modes, one, n),
    }


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # each step runs one all-core sample of the oracle (a bounded part of one apply per core);
    # the sample shrinks with the step count so that the whole run stays within a few minutes
    nsteps = args.warmup + args.steps
    planes, modes = (12, 96) if nsteps <= 40 else (6, 32)
    n = host_cores()
    w = OracleWorkers(n)
    vals, walls, ext = [], [], []
    try:
        for i in range(nsteps):
            t0 = time.perf_counter()
            res = w.run([(planes, modes, SEED + 1000 * i + j) for j in range(n)])
            wall = time.perf_counter() - t0
            each = [_full_apply_s(r[0], r[1], planes, r[2]) for r in res]
            if i >= args.warmup:
                vals.append(n * N1 * N2 * NZ / float(np.mean(each)))
                walls.append(wall)
                ext.append(float(np.mean(each)))
    finally:
        w.close()
    value = float(np.median(vals))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "impl": "reference",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        # a step is the bounded sample below (its wall time); the throughput is that of whole
        # applies, extrapolated from each process's sample
        "ms_per_step": 1e3 * float(np.median(walls)),
        "ms_per_apply_one_core_extrapolated": 1e3 * float(np.median(ext)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n1": N1, "n2": N2, "nz": NZ, "depth": DEPTH, "output": "stress",
                   "voxels": N1 * N2 * NZ},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "nproc": n, "kind": "oracle",
                         "sample": "per step: %d single-threaded processes at once, each FP64 oracle Hooke + DFT "
                                   "of %d of 384 planes each way + depth quadrature on %d random modes, "
                                   "extrapolated to one full apply" % (n, planes, modes)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fvim", choices=["fvim", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solves", action="store_true", help="skip the contact-solve metrics")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
