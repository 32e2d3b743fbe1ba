#!/usr/bin/env python
"""MOT-JVIE time-marching throughput on B300 (one JSON line on stdout).

Workload (default, `pillars8x8`): 8x8 array of two-layer dielectric cylinders
(eps_r 3.5 / 6.0, background 1) on a 256x256x80 voxel grid (15.7 M unknowns),
dt = 8 dt_CFL, x-polarised modulated-Gaussian plane wave along -z, mixed
FP32/FP64 arithmetic, a 200-step run.  One step = one full MOT step (Eq. 3):
incident field + history sum over ell lags, TFQMR solve of Z0 J_n = b_n with
FP64 refinement, and the history-ring update.  The timed region is steps
W .. W+K-1 of one run (defaults W = 5, K = 195: the whole 200-step run).

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


def product_flops(M0, B):
    """Flops of one Z0 product (SURVEY-style count): 6 real 3-D FFTs of
    2.5 M log2 M flops each per right-hand side (3 forward, 3 inverse, M = the
    padded grid's point count) plus 36 flops per half-spectrum frequency for the
    3x3 multiply."""
    M = M0[0] * M0[1] * M0[2]
    nf = M0[2] * M0[1] * (M0[0] // 2 + 1)
    return B * (6 * 2.5 * M * math.log2(M) + 36 * nf)


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
    "z_history": "k_hist_acc + k_col_r (lag 1 onto the step's partial history sum, inverse z pass)",
    "hist_side": "k_hist_block + k_hist_acc (time-blocked history: block pass at a block start, near lags 2..)",
    "fwd_half": "k_xy_forward_r<SrcHalfA> (forward xy pass of Z0 y2 + first TFQMR half step)",
    "fwd_y1": "k_xy_forward_r<SrcY1> (forward xy pass of Z0 y1)",
    "fwd_plain": "k_xy_forward_r<SrcPlain> (forward xy pass, stored input)",
    "fwd_ring": "k_xy_forward_r<SrcPlain<double>> (ring push, Mh grid)",
    "inv_half": "k_xy_inverse_r<EpiHalfB> (inverse xy pass of Z0 y2 + second TFQMR half step)",
    "inv_v": "k_xy_inverse_r<EpiV> (inverse xy pass of Z0 y1 + v update)",
    "inv_z0": "k_xy_inverse_r<EpiZ0> (inverse xy pass, Z0 epilogue)",
    "inv_residual": "k_xy_inverse_r<EpiResidual> (inverse xy pass, FP64 residual)",
    "inv_history": "k_xy_inverse_r<EpiHistory> (inverse xy pass of the history sum, Mh grid)",
    "row_fwd": "k_x_forward_r + k_col_r (forward row and column passes, planes too large for shared memory)",
    "row_inv": "k_col_r + k_x_inverse_r<EpiZ0> (inverse column and row passes with the Z0 epilogue)",
    "vec": "k_tfqmr_half_a / half_b / y1 / v (TFQMR vector updates of the row-pass path)",
}


def kernel_bytes(info, N, B, prec, steps, TB=None, spread=None):
    """Algorithmic bytes of one launch of each timed kernel class: every array
    the kernel must read or write once, nothing for re-reads.  steps: the
    indices of the timed steps (the history classes depend on them); TB: the
    time block of the history (8 in the mixed path, 4 in FP64)."""
    if TB is None:
        TB = 8 if prec == 1 else 4
    if spread is None:  # the library's schedule of the time-blocked pass
        spread = os.environ.get("MOTJVIE_HIST_SPREAD", "0") not in ("", "0")
    ell = info.ell
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

    def lags(u_lo, u_hi):
        """Lambda_k read by a block-pass part over inputs of age u in [u_lo, u_hi):
        k = u + 2 + t for t < TB, k <= ell"""
        return max(0, min(ell, u_hi + TB) - (u_lo + 2) + 1) if u_hi > u_lo else 0

    def side(m):
        """the time-blocked history work that prepares step m (t = m mod TB).
        Whole-pass schedule (default): at a block start one pass over the inputs
        within ell (read once for the block's TB steps), Lambda_2.. read once, TB
        partial sums written.  Spread schedule: at a block start the recent part
        of the block (inputs of age u < TB, its Lambda_k, the TB partial sums
        read and written), every step one chunk of TB of the next block's old
        part (inputs u >= TB, their Lambda_k, the partial sums written).  Both:
        the near accumulation of lags 2..t+1 onto the step's partial sum (read
        and written)."""
        t = m % TB
        m0 = m - t
        b = 0
        if not spread:
            if t == 0:
                U = max(0, min(ell - 1, m - 1))
                b += U * slot + min(ell - 1, U + TB) * lam_h + TB * slot
            near = max(0, min(t + 1, m, ell) - 1)
            if near:
                b += near * (slot + lam_h) + 2 * slot
            return b
        if t == 0:
            U = max(0, min(ell - 1, m0 - 1))
            R = min(TB, U)
            b += R * slot + lags(0, R) * lam_h + 2 * TB * slot
        U1 = max(0, min(ell - 1, m0 + TB - 1))
        nu = max(0, U1 - TB)
        b += (nu * slot + lags(TB, U1) * lam_h + TB * slot) / TB
        near = max(0, min(t + 1, m, ell) - 1)
        if near:
            b += near * (slot + lam_h) + 2 * slot
        return b

    nsteps = max(len(steps), 1)
    # the critical path: lag 1 onto the step's partial sum, inverse z pass of the Nz kept planes
    zh = sum((2 * slot + lam_h if m >= 1 else slot) + plh for m in steps) / nsteps
    hside = sum(side(m) for m in steps) / nsteps
    return {
        "z_green": 2 * pl0 + 6 * K0[2] * K0[1] * H0 * rs,
        "z_history": zh,
        "hist_side": hside,
        "fwd_half": 10 * vec + pl0,      # read d, y1, w, Ay1, v, x; write x, w, d, y2; write planes
        "fwd_y1": 3 * vec + pl0,         # read w, y2; write y1; write planes
        "fwd_plain": vec64 + pl0,        # the FP64 J of the residual product
        "fwd_ring": vec64 + plh,
        "inv_half": pl0 + eps + 9 * vec,  # read planes, eps, y2, d, w, r*, x; write Ay2, w, d, x
        "inv_v": pl0 + eps + 6 * vec,     # read planes, eps, y1, Ay2, v, r*; write Ay1, v
        "inv_z0": pl0 + eps + 2 * vec,
        "inv_residual": pl0 + nv * 8 + 3 * vec64,
        "inv_history": plh + nv * 8 + B * nv * 8 + 2 * vec64,
        # planes too large for shared memory: row + column passes of one product
        "row_fwd": vec + pl0,              # read the input vector, write the planes
        "row_inv": pl0 + eps + 2 * vec,    # read planes, eps and x, write y (plain epilogue)
        # TFQMR vector kernels: half_a 10, half_b 9, y1 3, v 5 vectors -> mean per launch
        "vec": 6.75 * vec,
    }


# the headers that hold the kernels (host-only sources such as the server are left out)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2607_28309_b300", "csrc", f)
                  for f in ("common.cuh", "dfloat.cuh", "fft.cuh", "krylov.cuh", "spectral.cuh")]


def kernel_digest():
    """sha256 of the kernel headers, first 16 hex digits."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(cls, wname="cube64_a8"):
    """DRAM bytes per launch from the committed ncu summary of this kernel class
    on this workload (profiles/<class>_<workload>.md), if one exists and was
    taken from the current kernel sources (its recorded kernel digest matches);
    else None."""
    digest = kernel_digest()
    path = os.path.join(ROOT, "profiles", f"{cls}_{wname}.md")
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
def _events_ms(stream, fn):
    import torch

    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


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
    K = args.steps

    # ---- e2e, cold: the first problem of this process (no quadrature cached,
    # no schedule tuned), created from host buffers, K + W steps each returning
    # J_n to pinned host memory; then the same again warm
    e2e_cold = end_to_end(mot, ctx, w, prec, args.warmup + K, stream, gopt)
    e2e_warm = end_to_end(mot, ctx, w, prec, args.warmup + K, stream, gopt)

    # ---- the timed run: W warm-up steps, K timed steps in one call
    t_setup = time.perf_counter()
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], gopt)
    run = mot.mot_run_create(prob, w["exc"], prec)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    info = mot.mot_problem_info_get(prob)
    ell = info.ell
    st = (mot.mot_step_stats * 1)()
    for _ in range(args.warmup):
        mot.mot_run_step(run, 1, None, st, allow_notconv=True)
    torch.cuda.synchronize()
    barrier(ws)
    sts = (mot.mot_step_stats * K)()
    l0 = mot.mot_kernel_launches()
    e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" restricts a launch list to it
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
    # steady state: past the history length every step sums all ell lags
    n_now = mot.mot_run_step_index(run)
    if n_now < ell + 1:
        mot.mot_run_step(run, ell + 1 - n_now, None, None, allow_notconv=True)
    S_steady = 20
    ms_steady = _events_ms(stream, lambda: mot.mot_run_step(run, S_steady, None, None, allow_notconv=True))
    steady = {"steps_per_s": S_steady / (ms_steady / 1e3), "steps": S_steady,
              "after_steps": mot.mot_run_step_index(run) - S_steady}
    schedule = mot.mot_problem_schedule(prob, B, mot.MOT_F32 if prec == mot.MOT_MIXED else mot.MOT_F64)
    mot.mot_run_destroy(run)

    # ---- kernel timing region: the same workload host-driven without CUDA
    # graphs, with CUDA events around every launch of the timed classes
    # (kernels inside CUDA graphs cannot be bracketed by events)
    kopt = mot.default_options(timing=1, graph=2)
    kprob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], kopt)
    krun = mot.mot_run_create(kprob, w["exc"], prec)
    kst = (mot.mot_step_stats * 1)()
    # warm up past the history length, so the timed steps sum all ell lags
    mot.mot_run_step(krun, max(args.warmup, ell + 1), None, None, allow_notconv=True)
    kstats = []
    ktimes = {}  # class -> [launches, total ms] over the timed steps
    for _ in range(8):  # one whole time block of the history
        mot.mot_run_step(krun, 1, None, kst, allow_notconv=True)
        s = kst[0]
        kstats.append((s.iters, s.sweeps, s.relres, s.mvps))
        for name, (n, ms) in mot.mot_run_kernel_times(krun).items():
            acc = ktimes.setdefault(name, [0, 0.0])
            acc[0] += n
            acc[1] += n * ms
    k_n0 = mot.mot_run_step_index(krun) - len(kstats)
    # the mixed march's currents at a step past the history length, for its
    # relative L2 error against the FP64 march below
    n_cmp = ell + 1 + 10 + 3  # past the FP64 run's timed steps below
    if mot.mot_run_step_index(krun) < n_cmp:
        mot.mot_run_step(krun, n_cmp - mot.mot_run_step_index(krun), None, None, allow_notconv=True)
    J_mixed = None
    if prec == mot.MOT_MIXED:
        J_mixed = torch.empty(B * 3 * nv, dtype=torch.float64, device=dev)
        src = mot.mot_run_current_device(krun)
        torch.cuda.synchronize()
        J_mixed.copy_(_dev_view(src, B * 3 * nv, dev))
    mot.mot_run_destroy(krun)
    mot.mot_problem_destroy(kprob)

    # ---- roofline of the dominant kernel class (algorithmic bytes / event time)
    peak, peak_kind = _peaks()
    nsteps_k = len(kstats)
    kb = kernel_bytes(info, N, B, prec, list(range(k_n0, k_n0 + nsteps_k)))
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
    roofline = {"kernel": KERNEL_NAMES[dom], "class": dom, "bound": "hbm", "achieved": d["GBps"], "peak": peak,
                "unit": "GB/s", "frac": d["frac"], "traffic": profiled_traffic(dom, w["name"]),
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "launch_ms": d["ms_per_launch"], "kernel_ms_per_step": d["ms_per_step"],
                "alg_bytes_per_launch": d["alg_bytes_per_launch"],
                "timing": "CUDA events on the library's stream around every launch of each class in a host-driven "
                          "(no-graph) run of the same workload, after ell+1 warm-up steps (full history)",
                "kernels": per_kernel}
    mvps = sum(s[3] for s in stats)
    M0, Mh = list(info.M0), list(info.Mh)
    Hh = Mh[0] // 2 + 1
    K0 = [m // 2 + 1 for m in M0]
    cs = 8 if prec == mot.MOT_MIXED else 16

    # ---- Z0 product alone (FP32 and FP64), L2 flushed between calls, beside
    # the cuFFT comparison product and the FMA peaks of this GPU
    fma = {}
    for name, dt_ in (("fp64", mot.MOT_F64), ("fp32", mot.MOT_F32)):
        f, ms = mot.mot_fma_peak(local, dt_)
        fma[name] = {"tflops": f / 1e12, "ms": ms}
    mvp = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lam_full = cufft_lambda(mot, prob, M0)
    keep64 = None
    for name, dt_, tdt in (("fp32", mot.MOT_F32, torch.float32), ("fp64", mot.MOT_F64, torch.float64),
                           ("fp64_double_float", mot.MOT_F64DF, torch.float64)):
        if name == "fp64_double_float" and keep64 is not None:
            x = keep64[0]  # the FP64 product's input: its output is the reference
        else:
            x = torch.randn(B, 3, nv, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            mot.mot_apply_Z0(prob, x, y, B, dt_)
        ts = []
        for _ in range(20):
            flush.zero_()
            ts.append(_events_ms(stream, lambda: mot.mot_apply_Z0(prob, x, y, B, dt_)))
        es = x.element_size()
        alg = B * 3 * nv * es * 2 + nv * es + 6 * K0[0] * K0[1] * K0[2] * es
        t = statistics.median(ts) / 1e3
        flops = product_flops(M0, B)
        mvp[name] = {"us": t * 1e6, "alg_bytes": alg, "GBps": alg / t / 1e9, "frac_of_hbm": alg / t / 1e9 / peak,
                     "flops": flops, "tflops": flops / t / 1e12}
        if name == "fp64_double_float":
            # FP64 vectors, FFTs in double-float (FP32 pairs) on the FP32 pipe
            mvp[name]["what"] = "FP64 in and out; FFTs and spectral multiply in double-float (FP32 pairs)"
            if keep64 is not None:
                mvp[name]["rel_l2_vs_fp64"] = float(torch.linalg.vector_norm(y - keep64[1]) /
                                                    torch.linalg.vector_norm(keep64[1]))
                mvp[name]["speedup_over_fp64"] = mvp["fp64"]["us"] / mvp[name]["us"]
            del x, y
            continue
        mvp[name]["frac_of_fma_peak"] = flops / t / 1e12 / fma[name]["tflops"]
        mvp[name]["schedule"] = mot.mot_problem_schedule(prob, B, dt_)
        try:  # cuFFT comparison product on the same M0 grid, timed only
            cf = CufftCompare(local, stream, N, M0, B, name == "fp64", lam_full, w["eps"])
            yc = torch.empty_like(x)
            for _ in range(3):
                cf.apply(x, yc)
            tc = []
            for _ in range(20):
                flush.zero_()
                tc.append(_events_ms(stream, lambda: cf.apply(x, yc)))
            rel = float(torch.linalg.vector_norm((yc - y).double()) / torch.linalg.vector_norm(y.double()))
            mvp["cufft_" + name] = {"us": statistics.median(tc) * 1e3, "rel_l2_vs_library": rel,
                                    "how": "cuFFT R2C/C2R plans over all 3 x nrhs components of the zero-padded M0 "
                                           "grid + one fused 3x3 multiply kernel + pad and epilogue kernels"}
            cf.close()
        except Exception as e:  # comparison baseline only
            mvp["cufft_" + name] = {"error": str(e)[:200]}
        if name == "fp64":
            keep64 = (x, y)
        del x, y
    keep64 = None
    mot.mot_problem_destroy(prob)

    # ---- the plain FP64 form of the same workload on the same GPU (steady
    # state), and the mixed march's relative L2 error against it
    compare = {}
    if prec == mot.MOT_MIXED and not args.no_fp64:
        try:
            pb = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], gopt)
            rb = mot.mot_run_create(pb, w["exc"], mot.MOT_FP64)
            mot.mot_run_step(rb, ell + 1, None, None, allow_notconv=True)
            S64 = 10
            ms64 = _events_ms(stream, lambda: mot.mot_run_step(rb, S64, None, None, allow_notconv=True))
            compare["fp64"] = {"steps_per_s": S64 / (ms64 / 1e3), "steps": S64,
                               "after_steps": mot.mot_run_step_index(rb) - S64,
                               "speedup_mixed_over_fp64": steady["steps_per_s"] / (S64 / (ms64 / 1e3))}
            n64 = mot.mot_run_step_index(rb)
            if n64 < n_cmp:
                mot.mot_run_step(rb, n_cmp - n64, None, None, allow_notconv=True)
            J64 = None
            if mot.mot_run_step_index(rb) == n_cmp:
                src = mot.mot_run_current_device(rb)
                torch.cuda.synchronize()
                J64 = _dev_view(src, B * 3 * nv, dev).clone()
                if J_mixed is not None:
                    compare["mixed_rel_l2_vs_fp64"] = {
                        "step": n_cmp,
                        "value": float(torch.linalg.vector_norm(J_mixed - J64) / torch.linalg.vector_norm(J64))}
            mot.mot_run_destroy(rb)
            mot.mot_problem_destroy(pb)
            # the FP64-accuracy march built on double-float products (FP32 inner
            # solves refined to 1e-11 against double-float residuals, history in
            # double-float), its error against the FP64 march at the same step
            pb = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], gopt)
            rb = mot.mot_run_create(pb, w["exc"], mot.MOT_FP64DF)
            mot.mot_run_step(rb, ell + 1, None, None, allow_notconv=True)
            msdf = _events_ms(stream, lambda: mot.mot_run_step(rb, S64, None, None, allow_notconv=True))
            compare["fp64_double_float"] = {
                "steps_per_s": S64 / (msdf / 1e3), "steps": S64, "after_steps": mot.mot_run_step_index(rb) - S64,
                "speedup_over_fp64": ms64 / msdf,
                "what": "MOT_FP64DF: FP32 inner TFQMR refined to 1e-11 against double-float (FP32-pair) residual "
                        "products; history ring, spectra and sum in double-float; J in FP64"}
            ndf = mot.mot_run_step_index(rb)
            if ndf < n_cmp:
                mot.mot_run_step(rb, n_cmp - ndf, None, None, allow_notconv=True)
            if mot.mot_run_step_index(rb) == n_cmp and J64 is not None:
                src = mot.mot_run_current_device(rb)
                torch.cuda.synchronize()
                Jdf = _dev_view(src, B * 3 * nv, dev)
                compare["fp64_double_float"]["rel_l2_vs_fp64"] = {
                    "step": n_cmp, "value": float(torch.linalg.vector_norm(Jdf - J64) / torch.linalg.vector_norm(J64))}
            mot.mot_run_destroy(rb)
            mot.mot_problem_destroy(pb)
            del J64
        except Exception as e:  # reported, not fatal
            compare.setdefault("fp64", {})["error"] = str(e)[:200]

    # ---- other workloads on the same GPU, mixed, steady state
    extra = {}
    if not args.no_extra:
        for label in [x for x in ("cube64_a8", "cube64_b16") if x != w["name"].split("_a")[0]]:
            try:
                wl = workload(label)
                pb = mot.mot_problem_create(ctx, wl["N"], wl["h"], wl["eps"], wl["alpha"], gopt)
                rb = mot.mot_run_create(pb, wl["exc"], mot.MOT_MIXED)
                mot.mot_run_step(rb, mot.mot_problem_info_get(pb).ell + 1, None, None, allow_notconv=True)
                Sx = 100 if len(wl["exc"]) == 1 else 20
                msx = _events_ms(stream, lambda: mot.mot_run_step(rb, Sx, None, None, allow_notconv=True))
                extra[label] = {"steps_per_s": Sx / (msx / 1e3), "nrhs": len(wl["exc"]),
                                "rhs_steps_per_s": Sx * len(wl["exc"]) / (msx / 1e3), "steps": Sx,
                                "after_steps": mot.mot_run_step_index(rb) - Sx, "grid": list(wl["N"]),
                                "alpha": wl["alpha"]}
                mot.mot_run_destroy(rb)
                mot.mot_problem_destroy(pb)
            except Exception as e:  # reported, not fatal
                extra[label] = {"error": str(e)[:200]}

    # ---- direct product (sum over the lag-0 support) against the FFT product, by
    # time-step size: the alpha crossover on the 64^3 cube (FP32, L2 flushed)
    crossover = {}
    if not args.no_extra:
        try:
            from paper_2607_28309_b300 import synthetic as syn

            for a in (1.0, 2.0, 4.0, 8.0, 16.0):
                wc = syn.cube64(a)
                pc = mot.mot_problem_create(ctx, wc["N"], wc["h"], wc["eps"], wc["alpha"], gopt)
                nvc = int(np.prod(wc["N"]))
                row = {"r0": mot.mot_problem_info_get(pc).r0}
                for pn, dtc, tdt in (("fp32", mot.MOT_F32, torch.float32), ("fp64", mot.MOT_F64, torch.float64)):
                    xc = torch.randn(1, 3, nvc, dtype=tdt, device=dev)
                    yf, yd = torch.empty_like(xc), torch.empty_like(xc)
                    for nm, fn in (("fft_us", lambda: mot.mot_apply_Z0(pc, xc, yf, 1, dtc)),
                                   ("direct_us", lambda: mot.mot_apply_Z0_direct(pc, xc, yd, 1, dtc))):
                        for _ in range(3):
                            fn()
                        tt = []
                        for _ in range(10 if (nm == "fft_us" or a <= 8) else 3):
                            flush.zero_()
                            tt.append(_events_ms(stream, fn))
                        row[f"{pn}_{nm}"] = statistics.median(tt) * 1e3
                    row[f"{pn}_rel_l2_direct_vs_fft"] = float(torch.linalg.vector_norm(yd - yf) /
                                                              torch.linalg.vector_norm(yf))
                crossover[f"alpha{int(a)}"] = row
                mot.mot_problem_destroy(pc)
        except Exception as e:  # reported, not fatal
            crossover["error"] = str(e)[:200]

    # ---- the Z0 product alone on the 60%-of-HBM target workloads
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

    # ---- serving: a Poisson stream of runs of mixed size through the server
    serving = {}
    if args.serve_runs > 0:
        try:
            serving = serve_stream(mot, ctx, args.serve_runs, args.serve_steps_scale, args.serve_slots)
        except Exception as e:  # reported, not fatal
            serving = {"error": str(e)[:300]}

    mot.mot_ctx_destroy(ctx)

    iters = [s[0] for s in stats]
    e2e = dict(e2e_warm)
    e2e["cold"] = e2e_cold
    e2e["note"] = ("value: problem + run creation from host buffers (eps_r, plane waves) and W + K steps through the "
                   "C ABI, each step's J_n returned to pinned host memory (calls of 8 steps), with the quadrature cache and tuned schedules "
                   "of this process warm; cold: the same as the process's first problem (tables and schedule computed)")
    res = {
        "metric": METRIC, "value": K * ws / elapsed_max, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": elapsed_max / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == mot.MOT_MIXED else "f64",
        "data": "synthetic (seeded SplitMix64 permittivity blocks / analytic pillar geometry, analytic plane-wave pulse)",
        "config": dict(describe(w, args.precision), graph_mode=args.graph_mode,
                       timed_steps=f"steps {args.warmup}..{args.warmup + K - 1} of one run",
                       l2=f"inputs larger than L2: each step reads the {ell}-slot history ring "
                          f"({ell * B * 3 * Mh[2] * Mh[1] * Hh * cs / 1e9:.2f} GB)",
                       parallelism=f"replicas{ws}", ell=ell, M0=M0, Mh=Mh),
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                       "mean": statistics.mean(lat), "what": "per step, CUDA events around each step's graph launch"},
        "tfqmr_iters_per_step": statistics.mean(iters), "mvps_per_step": mvps / K,
        "relres_max": max(s[2] for s in stats),
        "steady_state": steady, "setup_s": t_setup, "schedule": schedule,
        "same_gpu": compare, "other_workloads": extra, "fma_peak": fma,
        "z0_mvp": mvp, "z0_mvp_targets": targets, "z0_crossover": crossover, "serving": serving,
        "roofline": roofline, "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    return res, w, mvps / K


def serve_requests(nruns: int, steps_scale: float, seed: int = 5):
    """The serving recipe: 50 % cubes with edge in {24, 32, ..., 96} (eps_r U[1.5, 6] per
    4^3 block), 50 % n x n pillar arrays, n in {2, 3, 4} (32n x 32n x 80, layer eps_r
    U[1.5, 6] per pillar); alpha in {4, 8, 16}; steps U{100..300} times steps_scale;
    mixed precision; one plane wave along +z (cubes) or -z (pillars)."""
    import numpy as np

    from paper_2607_28309_b300 import synthetic

    u = synthetic.splitmix64(seed, 8 * nruns)
    out = []
    for i in range(nruns):
        a = u[8 * i: 8 * i + 8]
        alpha = (4.0, 8.0, 16.0)[int(a[1] * 3)]
        steps = max(3, int(round((100 + int(a[2] * 201)) * steps_scale)))
        if a[0] < 0.5:
            edge = 24 + 8 * int(a[3] * 10)
            N = (edge, edge, edge)
            eps = synthetic.block_eps(N, 4, 1.5, 6.0, seed * 100003 + i)
            exc = [synthetic.pulse(steps, alpha)]
            kind = f"cube{edge}"
        else:
            n = 2 + int(a[3] * 3)
            le = synthetic.splitmix64(seed * 7919 + i, 2 * n * n)
            layers = [(1.5 + 4.5 * le[2 * k], 1.5 + 4.5 * le[2 * k + 1]) for k in range(n * n)]
            eps = synthetic.pillar_eps(n, n, layer_eps=layers)
            N = (32 * n, 32 * n, 80)
            exc = [synthetic.pulse(steps, alpha, khat=(0.0, 0.0, -1.0))]
            kind = f"pillars{n}x{n}"
        out.append({"N": N, "eps": np.ascontiguousarray(eps), "alpha": alpha, "steps": steps, "exc": exc,
                    "kind": kind, "t_gap": float(-math.log(max(a[4], 1e-12)))})
    return out


def serve_stream(mot, ctx, nruns: int, steps_scale: float, slots: int):
    """Serve the recipe's runs through mot_server_*: calibrate the sustainable rate
    (runs served one at a time), then submit the stream with Poisson arrivals at
    0.8 x that rate into a server with `slots` slots; per-run and per-step latency
    percentiles and the aggregate MOT steps/s."""
    import threading

    reqs = serve_requests(nruns, steps_scale)
    h = 10e-9
    # calibration: the first few requests alone, one after the other
    ncal = min(6, nruns)
    srv = mot.mot_server_create(ctx, 0, 1)
    t0 = time.perf_counter()
    cal = []
    for q in reqs[:ncal]:
        tk = mot.mot_server_submit(srv, q["N"], h, q["eps"], q["alpha"], q["exc"], q["steps"])
        cal.append(mot.mot_server_wait(srv, tk, 600.0))
    cal_s = time.perf_counter() - t0
    mot.mot_server_destroy(srv)
    mean_run_s = statistics.mean(r.run_ms for r in cal) / 1e3
    rate = 0.8 / max(mean_run_s, 1e-6)  # runs per second
    srv = mot.mot_server_create(ctx, 0, slots)
    tickets = [None] * nruns
    sub_err = []

    def submitter():
        t = time.perf_counter()
        for i, q in enumerate(reqs):
            t += q["t_gap"] / rate
            dt = t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            try:
                tickets[i] = mot.mot_server_submit(srv, q["N"], h, q["eps"], q["alpha"], q["exc"], q["steps"])
            except Exception as e:  # recorded
                sub_err.append(str(e)[:100])

    t_start = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    res = []
    for i in range(nruns):
        while tickets[i] is None and th.is_alive():
            time.sleep(0.001)
        if tickets[i] is None:
            continue
        res.append((reqs[i], mot.mot_server_wait(srv, tickets[i], 3600.0)))
    th.join()
    wall = time.perf_counter() - t_start
    mot.mot_server_destroy(srv)
    ok = [(q, r) for q, r in res if r.status == 0]
    steps = sum(r.steps for _, r in ok)
    run_lat = sorted((r.queue_ms + r.run_ms) for _, r in ok)
    step50 = sorted(r.step_p50_ms for _, r in ok)
    step99 = sorted(r.step_p99_ms for _, r in ok)

    def pct(v, q):
        return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None

    kinds = {}
    for q, _ in ok:
        kinds[q["kind"]] = kinds.get(q["kind"], 0) + 1
    return {"runs": nruns, "completed": len(ok), "failed": len(res) - len(ok), "submit_errors": sub_err[:3],
            "slots": slots, "steps_scale": steps_scale, "arrival_rate_runs_per_s": rate,
            "calibration": {"runs": ncal, "mean_run_s": mean_run_s, "wall_s": cal_s},
            "aggregate_steps_per_s": steps / wall, "steps": steps, "wall_s": wall,
            "run_latency_ms": {"p50": pct(run_lat, 0.5), "p99": pct(run_lat, 0.99)},
            "step_latency_ms": {"p50_of_run_p50": pct(step50, 0.5), "p99_of_run_p99": pct(step99, 0.99)},
            "mix": kinds,
            "recipe": "cubes 24^3..96^3 (eps U[1.5,6] per 4^3) and 2x2..4x4 pillar arrays (32n x 32n x 80, layer eps "
                      "U[1.5,6] per pillar), alpha in {4,8,16}, steps U{100..300} x steps_scale, mixed; Poisson "
                      "arrivals at 0.8 x the rate of runs served one at a time (seed 5)"}


def _dev_view(ptr, n, dev):
    """A float64 torch view of n doubles at device address ptr (borrowed)."""
    import torch

    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_Arr(), device=dev)


def cufft_lambda(mot, prob, M0):
    """The real spectrum [6][Mz][My][Mx/2+1] of the circulant lag-0 table on the
    M0 grid, 1/(Mx My Mz) folded in (for the cuFFT comparison product)."""
    import numpy as np

    (Rx, Ry, Rz), g = mot.mot_kernel_table(prob, 0)
    emb = np.zeros((6, M0[2], M0[1], M0[0]))
    for dz in range(-Rz, Rz + 1):
        for dy in range(-Ry, Ry + 1):
            emb[:, dz % M0[2], dy % M0[1], np.arange(-Rx, Rx + 1) % M0[0]] = g[:, dz + Rz, dy + Ry, :]
    lam = np.fft.rfftn(emb, axes=(1, 2, 3)).real / float(M0[0] * M0[1] * M0[2])
    return np.ascontiguousarray(lam)


class CufftCompare:
    """ctypes handle of libmotcufft.so (the cuFFT comparison product)."""

    def __init__(self, device, stream, N, M0, nrhs, fp64, lam, eps):
        import ctypes

        import numpy as np

        from paper_2607_28309_b300 import build as mbuild

        self.L = ctypes.CDLL(mbuild.build_cufft_compare())
        P = ctypes.c_void_p
        self.L.mcf_create.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.POINTER(P)]
        self.L.mcf_apply.argtypes = [P, P, P]
        self.L.mcf_destroy.argtypes = [P]
        self.L.mcf_last_error.restype = ctypes.c_char_p
        n = (ctypes.c_int32 * 3)(*N)
        m = (ctypes.c_int32 * 3)(*M0)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        self.h = P()
        rc = self.L.mcf_create(int(device), P(stream.cuda_stream), n, m, int(nrhs), int(bool(fp64)),
                               lam.ctypes.data_as(P), eps.ctypes.data_as(P), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError("mcf_create: " + self.L.mcf_last_error().decode())

    def apply(self, x, y):
        import ctypes

        if self.L.mcf_apply(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())) != 0:
            raise RuntimeError("mcf_apply: " + self.L.mcf_last_error().decode())

    def close(self):
        self.L.mcf_destroy(self.h)


E2E_CHUNK = 8  # steps per mot_run_step call of the end-to-end leg


def end_to_end(mot, ctx, w, prec, K, stream, opt):
    """steps/s through the public C-ABI from host buffers: problem and run
    creation (host eps_r and plane waves copied in) plus K steps, every step's
    J_n copied back to pinned host memory (calls of E2E_CHUNK steps into one
    pinned buffer of E2E_CHUNK currents, so the library overlaps each step's
    copy with the next step)."""
    import numpy as np
    import torch

    N = w["N"]
    nv = int(np.prod(N))
    B = len(w["exc"])
    Jh = torch.empty((E2E_CHUNK, B, 3, nv), dtype=torch.float64).pin_memory()
    Jn = Jh.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"], opt)
    run = mot.mot_run_create(prob, w["exc"], prec)
    t1 = time.perf_counter()
    done = 0
    while done < K:
        c = min(E2E_CHUNK, K - done)
        mot.mot_run_step(run, c, Jn[:c], allow_notconv=True)
        done += c
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    mot.mot_run_destroy(run)
    mot.mot_problem_destroy(prob)
    h2d = nv * 8 + B * 80
    return {"value": K / (t2 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": B * 3 * nv * 8, "setup_s": t1 - t0, "steady_steps_per_s": K / (t2 - t1),
            "steps": K}


# ---------------------------------------------------------------- reference arm
def reference(args, ws, rank):
    if rank != 0:
        return None
    w = workload(args.workload)
    mvps = 2 * 12 + 3  # present-time products per step of the direct method (TFQMR, 12 iterations)
    vals = []
    t0 = time.perf_counter()
    for i in range(args.warmup + args.steps):
        s = oracle_sample(w, mvps, rows=16384, seed=i)
        if i >= args.warmup:
            vals.append(s)
    wall = time.perf_counter() - t0
    v = statistics.mean(x["steps_per_s"] for x in vals)
    sample = (f"{len(vals)} timed samples (after {args.warmup} warm-up samples), each 16384 sampled rows of the "
              f"oracle's direct Z0 product at the full {w['N'][0]}x{w['N'][1]}x{w['N'][2]} size; value = the full "
              f"direct MOT step rate extrapolated from the samples by the exact nonzero count of one step (history over "
              f"all lags + {mvps} present-time products)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, args.precision),
            "extrapolated": True,
            "timing": {"sample_ms_per_step": 1e3 * statistics.mean(x["seconds"] for x in vals),
                       "wall_s": wall,
                       "note": "each timed step is a bounded sample of the workload's direct step; ms_per_step is the "
                               "full step's time extrapolated from it, not a wall time"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def oracle_march_sample(nsteps: int = 20):
    """The oracle's real march on the 16^3 cube (alpha 4): problem set-up
    (tables, sparse LU of Z0) and nsteps steps, each timed; steady = the steps
    at and past the history length (every lag summed)."""
    import oracle
    from paper_2607_28309_b300 import synthetic

    w = synthetic.cube16()
    t0 = time.perf_counter()
    P = oracle.Problem(w["N"], w["h"], w["eps"], w["alpha"])
    import numpy as np

    Nx, Ny, Nz = w["N"]
    P.solve_Z0(np.zeros((3, Nz, Ny, Nx)))  # factorise
    t_setup = time.perf_counter() - t0
    J = np.zeros((nsteps, 3, Nz, Ny, Nx))
    ts = []
    for n in range(nsteps):
        a = time.perf_counter()
        J[n] = P.solve_Z0(P.rhs(n, w["exc"][0], J))
        ts.append(time.perf_counter() - a)
    steady = ts[P.ell:] if len(ts) > P.ell else ts[-1:]
    return {"workload": "cube16_a4 (16^3, alpha 4, FP64, exact LU solve per step)", "ell": P.ell,
            "setup_s": t_setup, "steps": nsteps, "march_s": sum(ts), "steps_per_s_over_march": nsteps / sum(ts),
            "steady_steps_per_s": len(steady) / sum(steady)}


_ONE_THREAD = r"""
import json, time, sys, numpy as np
sys.path.insert(0, %r)
import oracle
from paper_2607_28309_b300 import synthetic
w = synthetic.cube16()
t0 = time.perf_counter()
P = oracle.Problem(w["N"], w["h"], w["eps"], w["alpha"])
Nx, Ny, Nz = w["N"]
P.solve_Z0(np.zeros((3, Nz, Ny, Nx)))
ts = time.perf_counter() - t0
rng = np.random.default_rng(0)
J = rng.standard_normal((P.ell + 1, 3, Nz, Ny, Nx))
a = time.perf_counter()
P.solve_Z0(P.rhs(P.ell, w["exc"][0], J))
print(json.dumps({"setup_s": ts, "step_s": time.perf_counter() - a}))
"""


def oracle_one_thread():
    """One full-history step of the oracle's cube16 march on one thread
    (OMP_NUM_THREADS=1, the paper's single-thread methodology), in a child
    process so the thread count takes effect."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", _ONE_THREAD % ROOT], env=env, capture_output=True, text=True,
                         timeout=600)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    d["steps_per_s"] = 1.0 / d["step_s"]
    d["workload"] = "cube16_a4, one step at the full history length (ell lags), 1 thread"
    return d


def cpu_baseline(w, mvps):
    """The oracle as it stands on this host's cores: (i) sampled rows of its
    direct Z0 product on the benchmarked workload, scaled to that workload's
    MOT step (bounded to ~10 s of CPU work); (ii) its real march on the 16^3
    cube, all cores; (iii) one full-history step of that march on one thread."""
    s = oracle_sample(w, mvps, rows=1 << 18)
    rows = int(min(1 << 24, max(1 << 18, (1 << 18) * 10.0 / max(s["seconds"], 1e-3))))
    s = oracle_sample(w, mvps, rows=rows)
    out = {"value": s["steps_per_s"], "unit": UNIT, "cores": s["cores"], "kind": "oracle",
           "sample": f"{rows} sampled rows of the oracle's direct Z0 product at full size ({s['seconds']:.1f} s on "
                     f"{s['cores']} cores), scaled by the exact nonzero count of one direct MOT step "
                     f"({s['step_entries']:.3g} entries: history over all lags + {mvps:.1f} present-time products)"}
    try:
        out["march_cube16"] = oracle_march_sample()
    except Exception as e:  # reported, not fatal
        out["march_cube16"] = {"error": str(e)[:200]}
    try:
        out["one_thread_cube16"] = oracle_one_thread()
    except Exception as e:  # reported, not fatal
        out["one_thread_cube16"] = {"error": str(e)[:200]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=195)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="pillars8x8")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-targets", action="store_true", help="skip the Z0 product timings on cube64_b16 and pillars8x8")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 form of the workload")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (cube64_a8, cube64_b16)")
    ap.add_argument("--serve-runs", type=int, default=48, help="runs of the serving stream (0: skip; recipe: 256)")
    ap.add_argument("--serve-steps-scale", type=float, default=0.25,
                    help="fraction of the recipe's 100..300 steps per run (recipe: 1)")
    ap.add_argument("--serve-slots", type=int, default=8, help="server slots (runs on the GPU at once)")
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
            res["cpu_baseline"] = cpu_baseline(w, mvps)
        print(json.dumps(res))


if __name__ == "__main__":
    main()
