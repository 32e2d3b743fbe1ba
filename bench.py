#!/usr/bin/env python
"""MOT-JVIE time-marching throughput on B300 (one JSON line on stdout).

Workload (default): 64x64x64 dielectric cube, eps_r uniform in [1.5, 6.0] per
8^3 block (seeded), dt = 8 dt_CFL, x-polarised modulated-Gaussian plane wave
along +z, mixed FP32/FP64 arithmetic.  One step = one full MOT step (Eq. 3):
incident field + history sum over ell lags, TFQMR solve of Z0 J_n = b_n with
FP64 refinement, and the history-ring update.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
timed region is bracketed by a barrier and the max over ranks is taken.
--impl reference times the FP64 CPU oracle (direct products) on the host.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MOT steps/s, Z0 FFT-matvec HBM GB/s (FP32 vs FP64), p50/p99 latency"
UNIT = "steps/s"
GRAPH_MODES = {"step": 1, "loop": 0, "none": 2}  # mot_options.graph values


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    except OSError:
        return 6400.0, "fallback"


# ---------------------------------------------------------------- distributed glue
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, v: float, device=None) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


# ---------------------------------------------------------------- workloads
def workload(name: str):
    from paper_2607_28309_b300 import synthetic

    try:
        return synthetic.workload(name)
    except ValueError as e:
        raise SystemExit(str(e))


def describe(w, precision):
    Nx, Ny, Nz = w["N"]
    return {"workload": f"{w['name']}: {Nx}x{Ny}x{Nz} voxels, {3 * Nx * Ny * Nz * len(w['exc'])} unknowns, "
                        f"alpha {w['alpha']:g} (dt = {w['alpha']:g} dt_CFL), {len(w['exc'])} plane wave(s), "
                        f"{precision} arithmetic",
            "nrhs": len(w["exc"]), "alpha": w["alpha"], "grid": list(w["N"]), "precision": precision}


# ---------------------------------------------------------------- oracle timing (CPU)
def nnz_per_lag(N, rho, ell):
    """exact nonzero count of Z_k on the grid (3 diagonal + mixed entries per
    offset in the causal support ((k-2) rho, (k+1) rho) of the lag tables)"""
    import numpy as np

    ax = [np.arange(-(n - 1), n) for n in N]
    dz, dy, dx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    lo = np.sqrt(np.maximum(np.abs(dx) - 1, 0) ** 2 + np.maximum(np.abs(dy) - 1, 0) ** 2
                 + np.maximum(np.abs(dz) - 1, 0) ** 2)
    hi = np.sqrt((np.abs(dx) + 1) ** 2 + (np.abs(dy) + 1) ** 2 + (np.abs(dz) + 1) ** 2)
    w = ((N[0] - np.abs(dx)) * (N[1] - np.abs(dy)) * (N[2] - np.abs(dz))).astype(np.float64)
    mixed = 2 * ((dx != 0) & (dy != 0)) + 2 * ((dx != 0) & (dz != 0)) + 2 * ((dy != 0) & (dz != 0))
    wt = w * (3 + mixed)
    return [float(np.sum(wt[(lo < (k + 1) * rho) & (hi > (k - 2) * rho)])) for k in range(ell + 1)]


def oracle_sample(w, mvps_per_step: float, rows: int = 2048, seed: int = 0):
    """Time the oracle's direct Z0 product on `rows` sampled rows of the full
    workload and scale by the exact nonzero count of one direct MOT step
    (history sum over all lags + mvps_per_step present-time products)."""
    import numpy as np

    import oracle

    N, eps, alpha = w["N"], w["eps"], w["alpha"]
    rho = alpha / math.sqrt(3.0)
    ell = oracle.history_length(N, rho)
    R = oracle.table_extent(0, rho, N)
    g = oracle.lag_table(0, rho, R)
    rng = np.random.default_rng(seed)
    nv = int(np.prod(N))
    x = rng.standard_normal((3, N[2], N[1], N[0]))
    rp = rng.integers(0, 3, rows)
    rm = rng.integers(0, nv, rows)
    t0 = time.perf_counter()
    oracle.Zk_rows(0, N, eps, R, g, x, rp, rm)
    dt = time.perf_counter() - t0
    nnz = nnz_per_lag(N, rho, ell)
    row_nnz0 = nnz[0] / (3.0 * nv)            # average entries of a Z0 row
    entries_per_s = rows * row_nnz0 / dt
    step_entries = sum(nnz[1:]) * len(w["exc"]) + mvps_per_step * nnz[0] * len(w["exc"])
    return {"steps_per_s": entries_per_s / step_entries, "seconds": dt, "rows": rows,
            "entries_per_s": entries_per_s, "step_entries": step_entries, "cores": os.cpu_count()}


# ---------------------------------------------------------------- roofline bookkeeping
KERNEL_NAMES = {
    "z_green": "k_z_green_r (present-time z pass)",
    "z_history": "k_hist_acc + k_col_r (history sum and its inverse z pass)",
    "fwd_half": "k_xy_forward_r<SrcHalfA> (forward xy pass of Z0 y2 + first TFQMR half step)",
    "fwd_y1": "k_xy_forward_r<SrcY1> (forward xy pass of Z0 y1)",
    "fwd_plain": "k_xy_forward_r<SrcPlain> (forward xy pass, stored input)",
    "fwd_ring": "k_xy_forward_r<SrcPlain<double>> (ring push, Mh grid)",
    "inv_half": "k_xy_inverse_r<EpiHalfB> (inverse xy pass of Z0 y2 + second TFQMR half step)",
    "inv_v": "k_xy_inverse_r<EpiV> (inverse xy pass of Z0 y1 + v update)",
    "inv_z0": "k_xy_inverse_r<EpiZ0> (inverse xy pass, Z0 epilogue)",
    "inv_residual": "k_xy_inverse_r<EpiResidual> (inverse xy pass, FP64 residual)",
    "inv_history": "k_xy_inverse_r<EpiHistory> (inverse xy pass of the history sum, Mh grid)",
}


def kernel_bytes(info, N, B, prec, lags):
    """Algorithmic bytes of one launch of each timed kernel class: every array
    the kernel must read or write once, nothing for re-reads.  lags: the
    history lag count of each timed step (for the history z pass)."""
    nv = N[0] * N[1] * N[2]
    cs = 8 if prec == 1 else 16          # complex element of the FFT precision (MOT_MIXED = 1)
    rs = cs // 2                         # real element of the solve precision
    M0, Mh = list(info.M0), list(info.Mh)
    H0, Hh = M0[0] // 2 + 1, Mh[0] // 2 + 1
    K0 = [m // 2 + 1 for m in M0]
    Kh = [m // 2 + 1 for m in Mh]
    vec = B * 3 * nv * rs                # one solver vector
    vec64 = B * 3 * nv * 8               # one FP64 vector (J, b, residual)
    pl0 = B * 3 * N[2] * M0[1] * H0 * cs  # the product's (z, ky, kx) planes
    plh = B * 3 * N[2] * Mh[1] * Hh * cs
    eps = nv * rs
    slot = B * 3 * Mh[2] * Mh[1] * Hh * cs
    lam_h = 6 * Kh[2] * Kh[1] * Hh * rs
    zh = sum(L * (slot + lam_h) + plh for L in lags) / max(len(lags), 1)
    return {
        "z_green": 2 * pl0 + 6 * K0[2] * K0[1] * H0 * rs,
        "z_history": zh,
        "fwd_half": 10 * vec + pl0,      # read d, y1, w, Ay1, v, x; write x, w, d, y2; write planes
        "fwd_y1": 3 * vec + pl0,         # read w, y2; write y1; write planes
        "fwd_plain": vec64 + pl0,        # the FP64 J of the residual product
        "fwd_ring": vec64 + plh,
        "inv_half": pl0 + eps + 9 * vec,  # read planes, eps, y2, d, w, r*, x; write Ay2, w, d, x
        "inv_v": pl0 + eps + 6 * vec,     # read planes, eps, y1, Ay2, v, r*; write Ay1, v
        "inv_z0": pl0 + eps + 2 * vec,
        "inv_residual": pl0 + nv * 8 + 3 * vec64,
        "inv_history": plh + nv * 8 + B * nv * 8 + 2 * vec64,
    }


# the headers that hold the kernels (host-only sources such as the server are left out)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2607_28309_b300", "csrc", f)
                  for f in ("common.cuh", "fft.cuh", "krylov.cuh", "spectral.cuh")]


def kernel_digest():
    """sha256 of the kernel headers, first 16 hex digits."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(cls):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload, if one exists and was taken from the current kernel sources
    (its recorded kernel digest matches); else None."""
    digest = kernel_digest()
    path = os.path.join(ROOT, "profiles", f"{cls}_cube64_a8.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("csrc digest") != digest:
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- native arm
def native(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2607_28309_b300 as mot
    from paper_2607_28309_b300 import build as mbuild

    mbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = workload(args.workload)
    prec = mot.MOT_MIXED if args.precision == "mixed" else mot.MOT_FP64
    N = w["N"]
    nv = int(np.prod(N))
    B = len(w["exc"])
    ctx = mot.mot_ctx_create(local, stream.cuda_stream)
    gopt = mot.default_options(graph=GRAPH_MODES[args.graph_mode])
    t_setup = time.perf_counter()
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], gopt)
    run = mot.mot_run_create(prob, w["exc"], prec)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    info = mot.mot_problem_info_get(prob)
    st = (mot.mot_step_stats * 1)()
    for _ in range(args.warmup):
        mot.mot_run_step(run, 1, None, st, allow_notconv=True)
    torch.cuda.synchronize()
    barrier(ws)
    K = args.steps
    sts = (mot.mot_step_stats * K)()
    l0 = mot.mot_kernel_launches()
    e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        e_all0.record(stream)
        # K steps in one call; the library records CUDA events around each step
        mot.mot_run_step(run, K, None, sts, allow_notconv=True)
        e_all1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = mot.mot_kernel_launches() - l0
    stats = [(s.iters, s.sweeps, s.relres, s.mvps, s.ms_zhist, s.ms_zgreen, s.ms_history, s.ms_solve, s.ms_push)
             for s in sts]
    barrier(ws)
    elapsed = e_all0.elapsed_time(e_all1) / 1e3
    elapsed_max = max_over_ranks(ws, elapsed, dev)
    lat = sorted(s[6] + s[7] + s[8] for s in stats)
    clocks = clk.summary()

    # ---- kernel timing region: the same workload host-driven without CUDA
    # graphs, with CUDA events around the history z pass and every Z0 spectral
    # z pass (kernels inside CUDA graphs cannot be bracketed by events)
    kopt = mot.default_options(timing=1, graph=2)
    kprob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], kopt)
    krun = mot.mot_run_create(kprob, w["exc"], prec)
    kst = (mot.mot_step_stats * 1)()
    # warm up past the history length, so the timed steps sum all ell lags as
    # the timed region's steps do
    for _ in range(max(args.warmup, info.ell + 1)):
        mot.mot_run_step(krun, 1, None, kst, allow_notconv=True)
    kstats = []
    ktimes = {}  # class -> [launches, total ms] over the timed steps
    for _ in range(max(5, min(K, 10))):
        mot.mot_run_step(krun, 1, None, kst, allow_notconv=True)
        s = kst[0]
        kstats.append((s.iters, s.sweeps, s.relres, s.mvps, s.ms_zhist, s.ms_zgreen, s.ms_history, s.ms_solve, s.ms_push))
        for name, (n, ms) in mot.mot_run_kernel_times(krun).items():
            acc = ktimes.setdefault(name, [0, 0.0])
            acc[0] += n
            acc[1] += n * ms
    k_n0 = mot.mot_run_step_index(krun) - len(kstats)
    mot.mot_run_destroy(krun)
    mot.mot_problem_destroy(kprob)

    # ---- roofline of the dominant kernel (algorithmic bytes / event time)
    peak, peak_kind = _peaks()
    nsteps_k = len(kstats)
    kb = kernel_bytes(info, N, B, prec, [min(n, info.ell) for n in range(k_n0, k_n0 + nsteps_k)])
    per_kernel = {}
    for name, (n, tot) in ktimes.items():
        if n == 0:
            continue
        mean_ms = tot / n
        alg = kb[name]
        per_kernel[name] = {"launches_per_step": n / nsteps_k, "ms_per_launch": mean_ms,
                            "ms_per_step": tot / nsteps_k, "alg_bytes_per_launch": alg,
                            "GBps": alg / (mean_ms / 1e3) / 1e9, "frac": alg / (mean_ms / 1e3) / 1e9 / peak}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_per_step"])
    d = per_kernel[dom]
    roofline = {"kernel": KERNEL_NAMES[dom], "bound": "hbm", "achieved": d["GBps"], "peak": peak, "unit": "GB/s",
                "frac": d["frac"], "traffic": profiled_traffic(dom), "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "launch_ms": d["ms_per_launch"], "kernel_ms_per_step": d["ms_per_step"],
                "alg_bytes_per_launch": d["alg_bytes_per_launch"],
                "timing": "CUDA events around every launch in a host-driven (no-graph) run of the same workload, "
                          "after ell+1 warm-up steps (full history)",
                "kernels": per_kernel}
    mvps = sum(s[3] for s in stats)
    cs = 8 if prec == mot.MOT_MIXED else 16  # complex element of the FFT precision
    M0, Mh = list(info.M0), list(info.Mh)
    Hh = Mh[0] // 2 + 1
    K0 = [m // 2 + 1 for m in M0]
    ell = info.ell

    # ---- Z0 product alone (FP32 and FP64), L2 flushed between calls
    mvp = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for name, dt_, tdt in (("fp32", mot.MOT_F32, torch.float32), ("fp64", mot.MOT_F64, torch.float64)):
        x = torch.randn(B, 3, nv, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            mot.mot_apply_Z0(prob, x, y, B, dt_)
        ts = []
        for _ in range(20):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mot.mot_apply_Z0(prob, x, y, B, dt_)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        es = x.element_size()
        alg = B * 3 * nv * es * 2 + nv * 8 + 6 * K0[0] * K0[1] * K0[2] * es
        t = statistics.median(ts) / 1e3
        mvp[name] = {"us": t * 1e6, "alg_bytes": alg, "GBps": alg / t / 1e9, "frac_of_peak": alg / t / 1e9 / peak}
    # cuFFT (torch.fft) comparison product on the same padded grid, timed only
    try:
        mvp["cufft_fp32"] = cufft_baseline(mot, prob, w, dev, stream, flush)
    except Exception as e:  # comparison baseline only
        mvp["cufft_fp32"] = {"error": str(e)[:200]}

    # ---- the plain FP64 form and a 16-excitation batch on the same GPU
    compare = {}
    for label, wl, pr_, steps_c in (("fp64", w, mot.MOT_FP64, 10),
                                    ("mixed_batch16", workload("cube64_b16"), mot.MOT_MIXED, 10)):
        try:
            pb = mot.mot_problem_create(ctx, wl["N"], wl["h"], wl["eps"], wl["alpha"], gopt)
            rb = mot.mot_run_create(pb, wl["exc"], pr_)
            # past the history length: the timed steps sum all ell lags
            mot.mot_run_step(rb, max(3, mot.mot_problem_info_get(pb).ell + 1), None, None, allow_notconv=True)
            torch.cuda.synchronize()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mot.mot_run_step(rb, steps_c, None, None, allow_notconv=True)
            b_.record(stream)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b_) / 1e3
            compare[label] = {"steps_per_s": steps_c / sec, "nrhs": len(wl["exc"]),
                              "rhs_steps_per_s": steps_c * len(wl["exc"]) / sec, "steps": steps_c,
                              "after_steps": mot.mot_run_step_index(rb) - steps_c}
            mot.mot_run_destroy(rb)
            mot.mot_problem_destroy(pb)
        except Exception as e:  # reported, not fatal
            compare[label] = {"error": str(e)[:200]}

    # ---- the Z0 product alone on the 60%-of-HBM target workloads: the
    # 16-excitation cube (72^3 grid) and the 256x256x80 pillar array
    targets = {}
    if not args.no_targets:
        from paper_2607_28309_b300 import mvp_bench

        for label, wl, nr, dtn in (("cube64_b16_f32", "cube64_b16", 16, "f32"), ("pillars8x8_f32", "pillars8x8", 1, "f32"),
                                   ("cube64_b16_f64", "cube64_b16", 16, "f64"), ("pillars8x8_f64", "pillars8x8", 1, "f64")):
            try:
                r_ = mvp_bench.run(wl, nr, dtn, warmup=3, reps=10, device=local)
                targets[label] = {k: r_[k] for k in ("us_median", "alg_bytes", "pass_bytes", "alg_GBps", "pass_GBps",
                                                     "pass_frac", "M0", "nrhs") if k in r_}
            except Exception as e:  # reported, not fatal
                targets[label] = {"error": str(e)[:200]}

    # ---- e2e: public API from host buffers, one call per step with a host J_n
    e2e = end_to_end(mot, ctx, w, prec, K, stream, gopt)

    mot.mot_run_destroy(run)
    mot.mot_problem_destroy(prob)
    mot.mot_ctx_destroy(ctx)

    iters = [s[0] for s in stats]
    res = {
        "metric": METRIC, "value": K * ws / elapsed_max, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": elapsed_max / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == mot.MOT_MIXED else "f64",
        "data": "synthetic (seeded SplitMix64 permittivity blocks, analytic plane-wave pulse)",
        "config": dict(describe(w, args.precision), graph_mode=args.graph_mode, l2="inputs larger than L2: each step reads the "
                       f"{ell}-slot history ring ({ell * B * 3 * Mh[2] * Mh[1] * Hh * cs / 1e9:.2f} GB)",
                       parallelism=f"replicas{ws}", ell=ell, M0=M0, Mh=Mh),
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                       "mean": statistics.mean(lat)},
        "tfqmr_iters_per_step": statistics.mean(iters), "mvps_per_step": mvps / K,
        "relres_max": max(s[2] for s in stats),
        "step_device_ms": statistics.mean(s[7] for s in stats),
        "same_gpu": compare,
        "setup_s": t_setup,
        "z0_mvp": mvp, "z0_mvp_targets": targets, "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
    }
    return res, w, mvps / K


def cufft_baseline(mot, prob, w, dev, stream, flush):
    """Z0 product through torch.fft (cuFFT) on the same M0 grid: timed only."""
    import numpy as np
    import torch

    info = mot.mot_problem_info_get(prob)
    N = w["N"]
    M0 = list(info.M0)
    (Rx, Ry, Rz), g = mot.mot_kernel_table(prob, 0)
    emb = np.zeros((6, M0[2], M0[1], M0[0]))
    for dz in range(-Rz, Rz + 1):
        for dy in range(-Ry, Ry + 1):
            for dx in range(-Rx, Rx + 1):
                emb[:, dz % M0[2], dy % M0[1], dx % M0[0]] = g[:, dz + Rz, dy + Ry, dx + Rx]
    lam = torch.fft.rfftn(torch.from_numpy(emb).to(dev), dim=(1, 2, 3)).real.float() / 1.0
    idx = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    eps = torch.from_numpy(np.ascontiguousarray(w["eps"])).to(dev, torch.float32)
    x = torch.randn(3, N[2], N[1], N[0], device=dev)

    def apply():
        X = torch.fft.rfftn(x, s=(M0[2], M0[1], M0[0]), dim=(1, 2, 3))
        Y = torch.stack([sum(lam[idx[p][q]] * X[q] for q in range(3)) for p in range(3)])
        G = torch.fft.irfftn(Y, s=(M0[2], M0[1], M0[0]), dim=(1, 2, 3))[:, :N[2], :N[1], :N[0]]
        return eps * 0.5 * x - (eps - 1.0) * G

    for _ in range(3):
        apply()
    ts = []
    for _ in range(20):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        apply()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return {"us": statistics.median(ts) * 1e3}


def end_to_end(mot, ctx, w, prec, K, stream, opt):
    """steps/s through the public C-ABI from host buffers: problem and run
    creation (host eps_r and plane waves copied in) plus K steps, each step
    copying J_n back to pinned host memory."""
    import numpy as np
    import torch

    N = w["N"]
    nv = int(np.prod(N))
    B = len(w["exc"])
    Jh = torch.empty((1, B, 3, nv), dtype=torch.float64).pin_memory()
    Jn = Jh.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], opt)
    run = mot.mot_run_create(prob, w["exc"], prec)
    t1 = time.perf_counter()
    for _ in range(K):
        mot.mot_run_step(run, 1, Jn, allow_notconv=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    mot.mot_run_destroy(run)
    mot.mot_problem_destroy(prob)
    h2d = nv * 8 + B * 80
    return {"value": K / (t2 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": B * 3 * nv * 8, "setup_s": t1 - t0, "steady_steps_per_s": K / (t2 - t1),
            "note": "timed region = problem + run creation from host buffers (eps_r, plane waves) and K steps, "
                    "each returning J_n to pinned host memory; the incident field is generated on the device"}


# ---------------------------------------------------------------- reference arm
def reference(args, ws, rank):
    if rank != 0:
        return None
    w = workload(args.workload)
    mvps = 2 * 12 + 3  # present-time products per step of the direct method (TFQMR, 12 iterations)
    vals = []
    for i in range(args.warmup + args.steps):
        s = oracle_sample(w, mvps, rows=16384, seed=i)
        if i >= args.warmup:
            vals.append(s)
    v = statistics.mean(x["steps_per_s"] for x in vals)
    sample = (f"{len(vals)} steps, each 16384 sampled rows of the oracle's direct Z0 product at the full "
              f"{w['N'][0]}x{w['N'][1]}x{w['N'][2]} size, scaled by the exact nonzero count of one direct MOT step "
              f"(history over all lags + {mvps} present-time products)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, "fp64 (oracle)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cube64_a8")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-targets", action="store_true", help="skip the Z0 product timings on cube64_b16 and pillars8x8")
    ap.add_argument("--graph-mode", default="step", choices=list(GRAPH_MODES),
                    help="step: one CUDA graph per MOT step (default); loop: host-driven steps, one graph per TFQMR "
                         "loop; none: no CUDA graphs (for per-kernel profilers)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        out = reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    res, w, mvps = native(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            s = oracle_sample(w, mvps, rows=4194304)
            res["cpu_baseline"] = {"value": s["steps_per_s"], "unit": UNIT, "cores": s["cores"], "kind": "oracle",
                                   "sample": f"4194304 sampled rows of the oracle's direct Z0 product at full size "
                                             f"({s['seconds']:.1f} s), scaled by the exact nonzero count of one "
                                             f"direct MOT step ({s['step_entries']:.3g} entries: history over all "
                                             f"lags + {mvps:.1f} present-time products)"}
        print(json.dumps(res))


if __name__ == "__main__":
    main()
