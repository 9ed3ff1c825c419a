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
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
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
                "samples": len(sm)}


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
        "traffic": TRAFFIC_BYTES.get(dom_name) if plan["depth_chunk"] == TRAFFIC_DEPTH_CHUNK or
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
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sample_modes=256, sample_planes=None)
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
    the device), with p50/p99 latency and the FP32 error against the FP64 solution."""
    import torch

    from paper_1811_11558_gb300 import Context
    from paper_1811_11558_gb300.serve import Request, Server, percentiles

    c = hertz_case()
    out = {"workload": "hertz_32x32x16_5inc", "relax": 0.5}
    press = {}
    for prec in ("fp64", "fp32"):
        ctx = Context(c["n"], c["n"], c["z"], 1.0, 1.0, precision=prec, E=E, nu=NU, sigma_y=c["sigma_y"],
                      E_h=c["E_h"])
        ctx.autotune()
        h = torch.from_numpy(c["h"]).to("cuda", ctx.dtype)
        p = torch.empty(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
        opts = ctx.default_opts(relax=0.5, max_iter=400)
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
                    E_h=c["E_h"], opts={"relax": 0.5, "max_iter": 400}) for i in range(served)]
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


def rough_metrics(n=1024, nz=32, depth=0.05, seed=1813):
    """Algorithm 1 on a rough surface, FP32: seeded self-affine surface n x n (H = 0.8, flat PSD
    for 4 <= |k| < 8, power law to k_s = 64, rms slope 0.1), nz uniform nodes to the given
    depth, sigma_y = 0.05 E*, E_h = 0.1 E.  (a) the paper's rough-surface load W = 1e-3 E x rms
    slope in five increments, relaxation 0.3: a converged solve; (b) the load of a 10 % elastic
    contact fraction, where Algorithm 1 does not reach the tolerance: a fixed budget of 20
    coupling iterations on each of two increments, timed per coupling iteration."""
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
    opts = ctx.default_opts(relax=0.3, max_iter=100, tol=1e-6)
    ctx.reset_state()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve_contact(hd, [W * (k + 1) / 5 for k in range(5)], p, opts, allow_not_converged=True)
    t = time.perf_counter() - t0
    out["paper_load"] = {"W": W, "increments": 5, "relax": 0.3, "tol": opts.tol, "status": rep["status"],
                         "solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t, "alg1_iters": rep["alg1_iters"],
                         "alg1_error": rep["alg1_error"], "contact_area": rep["contact_area"][-1],
                         "residual_evals": rep["residual_evals"], "cg_iters": rep["cg_iters"]}
    # load of a 10 % elastic contact fraction (area ~ linear in the load at small fractions)
    p.zero_()
    ctx.elastic_contact(hd, 5e-3, p, ctx.default_opts())
    W10 = 5e-3 * 0.1 / float((p > 0).double().mean())
    ctx.reset_state()
    opts = ctx.default_opts(relax=0.3, max_iter=20, tol=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.solve_contact(hd, [W10 / 2, W10], p, opts, allow_not_converged=True)
    t = time.perf_counter() - t0
    its = sum(rep["alg1_iters"][:2])
    out["area_10pct"] = {"W": W10, "increments": 2, "relax": 0.3, "alg1_cap": 20, "status": rep["status"],
                         "ms_per_alg1_iter": 1e3 * t / its, "alg1_error": rep["alg1_error"],
                         "contact_area": rep["contact_area"][-1],
                         "note": "Algorithm 1 stalls near 1e-2 on this load (the paper notes it is not robust on "
                                 "rough surfaces); timed on a fixed budget"}
    ctx.close()
    return out


def epp_metrics(n=128, nz=32, depth=0.25, ratios=(2.0, 3.0, 4.0)):
    """Elastic-perfectly-plastic Hertz load sweep (E_h = 0; the paper's App. C.2 comparison is
    elastic-perfectly-plastic, on an 81 x 81 x 32 grid): paraboloid R = 0.5 on n x n, nz nodes to
    the given depth, sigma_y = 0.05 E*, increments at W / W_y = ratios with W_y the elastic onset
    load (p0 = 1.6 sigma_y).  FP32 and FP64 one solve each (tuned plans), with the peak pressure,
    contact area and peak plastic strain of every increment, for both.  (At W / W_y = 8 on this
    grid Algorithm 1 with relaxation 0.5 does not converge in either precision.)"""
    import torch

    from paper_1811_11558_gb300 import Context, inputs

    es = E / (1 - NU * NU)
    sy = 0.05 * es
    a_y = np.pi * 0.5 * 1.6 * sy / (2 * es)
    w_y = 2 * np.pi * a_y ** 2 * 1.6 * sy / 3
    z = inputs.uniform_depth(nz, depth)
    h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.5)
    out = {"workload": "epp_hertz_%dx%dx%d" % (n, n, nz), "W_over_W_y": list(ratios), "relax": 0.5}
    press = {}
    for prec in ("fp32", "fp64"):
        ctx = Context(n, n, z, 1.0, 1.0, precision=prec, E=E, nu=NU, sigma_y=sy, E_h=0.0)
        ctx.autotune()
        hd = torch.from_numpy(h).to("cuda", ctx.dtype)
        p = torch.empty(ctx.surf_shape, dtype=ctx.dtype, device="cuda")
        opts = ctx.default_opts(relax=0.5, max_iter=150)
        rows = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in ratios:     # one increment per call (the state carries over), to read each state
            rep = ctx.solve_contact(hd, [r * w_y], p, opts, allow_not_converged=True)
            ep = torch.empty(ctx.scal_shape, dtype=ctx.dtype, device="cuda")
            ctx.get_state(None, ep, None)
            rows.append({"W_over_W_y": r, "p_max_over_sigma_y": float(p.max()) / sy,
                         "area": rep["contact_area"][-1], "e_p_max": float(ep.max()),
                         "alg1_iters": rep["alg1_iters"][-1], "status": rep["status"]})
        torch.cuda.synchronize()
        out[prec] = {"ms_per_sweep": 1e3 * (time.perf_counter() - t0), "increments": rows}
        press[prec] = p.cpu().numpy().astype(np.float64)
        ctx.close()
    out["fp32_vs_fp64_pressure_rel_l2"] = float(np.linalg.norm(press["fp32"] - press["fp64"]) /
                                                np.linalg.norm(press["fp64"]))
    return out


def batch_problems(n_prob=64, seed=1814):
    """Uneven elastic-plastic contact problems: grids n^2 with n drawn from {64, 128, 256, 512},
    nz from {8, 16, 32}; half paraboloids (R = 0.5, depth 0.5), half seeded self-affine surfaces
    (H uniform in [0.6, 0.9], flat PSD for 4 <= |k| < 8, power law to k_s = max(8, n / 16),
    rms slope 0.1, depth 0.05); total load log-uniform over the decade below the load of a 10 %
    elastic contact fraction (Hertz: pi a^2 = 0.1, W = 4 E* a^3 / (3 R); rough: mean pressure
    0.1 E* slope / 2), five increments; sigma_y = 0.05 E*, E_h = 0.1 E."""
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
            relax = 0.3
        else:
            h = inputs.hertz_profile(n, n, 1.0, 1.0, 0.5)
            z = inputs.uniform_depth(nz, 0.5)
            a = np.sqrt(0.1 / np.pi)
            w10 = 4.0 * es * a ** 3 / (3.0 * 0.5)
            relax = 0.5
        W = w10 * 10.0 ** u
        probs.append({"n": n, "nz": nz, "rough": rough, "z": z, "h": h, "loads": [W * (k + 1) / 5 for k in range(5)],
                      "relax": relax})
    return probs


def batch_metrics(n_prob=64, slots=16, seed=1814, max_iter=60, n64=4):
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
                       E_h=0.1 * E, opts={"relax": pb["relax"], "max_iter": max_iter, "tol": 1e-6})

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
    err = []
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
            ctx.solve_contact(hd, pb["loads"], p, ctx.default_opts(relax=pb["relax"], max_iter=max_iter,
                                                                   **({"tol": 1e-6} if prec == "fp32" else {})),
                              allow_not_converged=True)
            t[prec].append(time.perf_counter() - t0)
            press[prec] = p.cpu().numpy().astype(np.float64)
            ctx.close()
        err.append(float(np.linalg.norm(press["fp32"] - press["fp64"]) / np.linalg.norm(press["fp64"])))
    return {"workload": "batch_%d_uneven" % n_prob, "grids": sorted({pb["n"] for pb in probs}),
            "nz": sorted({pb["nz"] for pb in probs}), "rough": sum(pb["rough"] for pb in probs),
            "slots": slots, "alg1_cap": max_iter, "converged": conv,
            "tile_plans": {"shapes": len(plans), "tuning_s": prep_s,
                           "depth_chunk": sorted({(p["n"], p["nz"], p["depth_chunk"]) for p in plans.values()})},
            "fp32_served": {"solves_per_s": n_prob / wall, "wall_s": wall, "p50_ms": 1e3 * lat[50],
                            "p99_ms": 1e3 * lat[99], "arrivals": "all at t = 0"},
            "sample_n%d" % probs[small[0]]["n"] if small else "sample": {
                "problems": small, "fp64_plain_ms": [1e3 * x for x in t["fp64"]],
                "fp32_plain_ms": [1e3 * x for x in t["fp32"]], "fp32_vs_fp64_pressure_rel_l2": err},
            "per_problem": [{"n": pb["n"], "nz": pb["nz"], "rough": pb["rough"], "ms": 1e3 * (r.finished - r.admitted),
                             "status": r.report.get("status", 0), "iters": r.report.get("alg1_iters")}
                            for pb, r in zip(probs, res)]}


def stream_metrics(n_req=12, slots=8, seed=1815, rate_sweep=(0.4, 1.0, 1.5)):
    """Served request stream, FP32 vs plain FP64: requests with grids drawn uniformly in log2
    from {128, 256}, nz = round(16 x 2^U) in [16, 32], seeded self-affine surfaces (H 0.8, rms
    slope 0.1), five-increment ramps to the paper's rough-surface load; Poisson arrivals at
    0.7 x the single-stream FP32 capacity, then swept over rate_sweep x that capacity; p50 / p99
    latency from arrival to result.  The FP64
    baseline solves the first four requests one at a time; its solves/s is the mix's mean
    service time per size class applied to the whole stream."""
    import torch

    from paper_1811_11558_gb300 import inputs
    from paper_1811_11558_gb300.serve import Request, Server, percentiles, poisson_arrivals

    rng = np.random.Generator(np.random.PCG64(seed))
    es = E / (1 - NU * NU)
    reqs = []
    for i in range(n_req):
        n = int(2 ** rng.integers(7, 9))
        nz = int(round(16 * 2 ** rng.uniform(0, 1)))
        z = inputs.uniform_depth(nz, 0.05)
        h = inputs.self_affine_surface(n, 1.0, 0.8, 4, 8, min(64, n // 4), 0.1, seed=seed + 1 + i)
        reqs.append(Request(i, n, z, h, [1e-4 * (k + 1) / 5 for k in range(5)], precision="fp32", E=E, nu=NU,
                            sigma_y=0.05 * es, E_h=0.1 * E, opts={"relax": 0.3, "max_iter": 100, "tol": 1e-6}))
    srv = Server(slots=slots)
    srv.prepare(reqs)                                   # tuned tile plan per shape
    srv.run(reqs[:4])                                   # warm the context pool
    # single-stream capacity: one request at a time
    t0 = time.perf_counter()
    one = [srv.solve(r) for r in reqs[:4]]
    cap = 4 / (time.perf_counter() - t0)
    rate = 0.7 * cap
    arr = poisson_arrivals(n_req, rate, seed)
    for r, a in zip(reqs, arr):
        r.arrival = float(a)
    res, wall = srv.run(reqs)
    lat = percentiles([r.latency for r in res])
    def fresh(arrivals):
        return [Request(r.rid, r.n, r.z, r.h, r.loads, precision="fp32", E=E, nu=NU, sigma_y=r.sigma_y,
                        E_h=r.E_h, opts=r.opts, arrival=float(a)) for r, a in zip(reqs, arrivals)]

    sat, swall = srv.run(fresh(np.zeros(n_req)))
    # the arrival rate swept as a multiple of the single-stream capacity
    sweep = []
    for f in rate_sweep:
        rs, rw = srv.run(fresh(poisson_arrivals(n_req, f * cap, seed + 1)))
        lt = percentiles([r.latency for r in rs])
        sweep.append({"rate_over_capacity": f, "arrival_rate_per_s": f * cap, "solves_per_s": n_req / rw,
                      "p50_ms": 1e3 * lt[50], "p99_ms": 1e3 * lt[99]})
    # plain FP64, one request at a time
    from paper_1811_11558_gb300 import Context

    t64 = {}
    p64 = []
    for r in reqs[:4]:
        ctx = Context(r.n, r.n, r.z, 1.0, 1.0, precision="fp64", E=E, nu=NU, sigma_y=r.sigma_y, E_h=r.E_h)
        ctx.autotune()
        hd = torch.from_numpy(np.ascontiguousarray(r.h)).to("cuda", torch.float64)
        p = torch.empty(ctx.surf_shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_contact(hd, r.loads, p, ctx.default_opts(relax=0.3, max_iter=100), allow_not_converged=True)
        t64.setdefault(r.n, []).append(time.perf_counter() - t0)
        p64.append(p.cpu().numpy())
        ctx.close()
    mean64 = {k: float(np.mean(v)) for k, v in t64.items()}
    est64 = sum(mean64.get(r.n, max(mean64.values())) for r in reqs)
    err = [float(np.linalg.norm(one[i].pressure.astype(np.float64) - p64[i]) / np.linalg.norm(p64[i]))
           for i in range(4)]
    return {"workload": "rough_stream_%dreq" % n_req, "grids": sorted({r.n for r in reqs}),
            "nz": sorted({int(np.asarray(r.z).size) for r in reqs}), "slots": slots,
            "single_stream_fp32_solves_per_s": cap, "arrival_rate_per_s": rate,
            "fp32_served_poisson": {"solves_per_s": n_req / wall, "p50_ms": 1e3 * lat[50], "p99_ms": 1e3 * lat[99]},
            "fp32_served_rate_sweep": sweep,
            "fp32_served_saturated": {"solves_per_s": n_req / swall,
                                      "p50_ms": 1e3 * percentiles([r.latency for r in sat])[50],
                                      "p99_ms": 1e3 * percentiles([r.latency for r in sat])[99]},
            "fp64_plain": {"solves_per_s": n_req / est64, "measured_requests": 4,
                           "mean_s_by_grid": {str(k): v for k, v in mean64.items()}},
            "fp32_vs_fp64_pressure_rel_l2": err,
            "served_saturated_over_fp64_plain": (n_req / swall) / (n_req / est64)}


def scaling_metrics(sizes=(16, 32, 64, 128), reps=20):
    """Mindlin-apply time on N x N x N grids (the paper's VIM complexity sweep, App. C.4, whose
    reference time T0 = 1.41 ms was measured on a CPU node), FP32 and FP64, CUDA events,
    inputs resident."""
    import torch

    from paper_1811_11558_gb300 import Context, inputs

    out = {"workload": "mindlin_apply_cube_sweep", "paper_T0_ms_cpu": 1.41, "ms": {}}
    for prec in ("fp32", "fp64"):
        for n in sizes:
            z = inputs.uniform_depth(n, 1.0)
            ctx = Context(n, n, z, 1.0, 1.0, precision=prec, E=E, nu=NU)
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
            out["ms"]["%s_%d" % (prec, n)] = s.elapsed_time(e) / reps
            ctx.close()
    return out


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of each kernel on this
# workload, from one capture of the current kernels (profiles/ summaries); a kernel missing
# here, or changed since its capture (rows_inv6: smaller CTAs), reports null.
TRAFFIC_DEPTH_CHUNK = 4     # depth tile plan of that capture
TRAFFIC_BYTES = {"rows_fwd6": 755.1e6, "cols_fwd": 744.2e6, "mindlin_depth": 743.9e6, "cols_inv": 744.4e6,
                 "rows_inv6": None}


def _operator_input(seed=SEED):
    """The operator workload's plastic strain field (seeded), generated once per process."""
    from paper_1811_11558_gb300 import inputs

    key = ("ep", seed)
    if key not in _INPUT_CACHE:
        z = inputs.uniform_depth(NZ, DEPTH)
        _INPUT_CACHE[key] = (z, inputs.plastic_strain_field(N1, N2, z, seed=seed))
    return _INPUT_CACHE[key]


_INPUT_CACHE = {}


def cpu_baseline(sample_modes=256, sample_planes=None, seed=SEED):
    """Time the FP64 oracle on a bounded sample of the operator workload.

    Sample: the oracle's Hooke's law and forward and inverse DFT of ``sample_planes`` of the
    384 (layer, component) planes (all of them when None) plus its per-mode depth operator
    on ``sample_modes`` random modes (drawn with ``seed``); both are scaled to one full apply
    (384 planes each way, 131 072 resolved modes).  Input generation is not timed.
    """
    from oracle import operators as op
    from oracle import tensors as T

    z, ep = _operator_input()
    lam, mu = T.lame(E, NU)
    planes = NZ * 6
    npl = planes if sample_planes is None else int(sample_planes)
    nl = -(-npl // 6)  # layers that hold the sampled planes
    t0 = time.perf_counter()
    w = T.hooke6(ep[:nl], lam, mu, axis=1).reshape(nl * 6, N2, N1)[:npl]
    wh = np.fft.fft2(w, axes=(-2, -1))
    back = np.fft.ifft2(wh, axes=(-2, -1)).real
    t_fft = (time.perf_counter() - t0) * planes / npl
    assert back.shape == w.shape
    rng = np.random.default_rng(seed)
    k2 = rng.integers(0, N2, sample_modes)
    k1 = rng.integers(0, N1, sample_modes)
    Q1, Q2, nyq, zero = op.mode_grid(N1, N2, 1.0, 1.0)
    keep = ~(nyq[k2, k1] | zero[k2, k1])
    k1, k2 = k1[keep], k2[keep]
    W = (rng.standard_normal((k1.size, NZ, 3, 3)) + 1j * rng.standard_normal((k1.size, NZ, 3, 3))) * 1e-3
    W = 0.5 * (W + np.swapaxes(W, -1, -2))
    Q = np.stack([Q1[k2, k1], Q2[k2, k1]], axis=1)
    t1 = time.perf_counter()
    op.mindlin_modes(W, Q, z, E, NU)
    t_modes = (time.perf_counter() - t1) * (N1 * (N2 // 2)) / k1.size
    total = t_fft + t_modes
    return {
        "value": N1 * N2 * NZ / total,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "sample": "FP64 oracle: Hooke + DFT of %d of 384 planes each way + per-mode depth quadrature on %d random "
                  "modes, scaled to one 512x512x64 apply (%.1f s extrapolated)" % (npl, k1.size, total),
    }


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # each step samples a bounded part of one apply; the sample shrinks with the step count so
    # that the whole run stays within a few minutes
    nsteps = args.warmup + args.steps
    planes, modes = (4, 16) if nsteps <= 60 else (1, 4)
    _operator_input()
    t = []
    for i in range(nsteps):
        cb = cpu_baseline(sample_modes=modes, sample_planes=planes, seed=SEED + i)
        if i >= args.warmup:
            t.append(cb["value"])
    value = float(np.median(t))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "impl": "reference",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * N1 * N2 * NZ / value,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n1": N1, "n2": N2, "nz": NZ, "depth": DEPTH, "output": "stress",
                   "voxels": N1 * N2 * NZ},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: FP64 oracle Hooke + DFT of %d of 384 planes each way + depth "
                                   "quadrature on <=%d random modes, scaled to one full apply" % (planes, modes)},
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
