"""Timing of the Z0 product alone (Eq. 11-12) on the synthetic workloads.

    python -m paper_2607_28309_b300.mvp_bench --workload pillars8x8 --dtype f32
    python -m paper_2607_28309_b300.mvp_bench --workload cube64_b16 --nrhs 16 --kernels

Creates the problem (lag-0 table and Lambda0 on the device) and applies
y = Z0 x through mot_apply_Z0 to seeded random device vectors: W untimed
calls, then R calls timed with CUDA events on the library's stream, each after
writing a 256 MB buffer so that L2 (126 MB) holds none of the inputs.  Prints
one JSON line: median time, the algorithmic bytes of one product (read x,
eps_r and the Lambda0 octant, write y) and the bytes the passes move through
HBM when no intermediate stays in L2 (for the 60%-of-HBM target), as GB/s and
fractions of the measured copy bandwidth.  --kernels adds each kernel's share
(torch.profiler over the timed calls).
"""
import argparse
import json
import os
import statistics


def pass_bytes(info, N, B, es):
    """Bytes the product's passes move through HBM: every pass reads and
    writes its whole operand (es: real element size of the precision)."""
    nv = N[0] * N[1] * N[2]
    M0 = list(info.M0)
    H0 = M0[0] // 2 + 1
    cs = 2 * es
    vec = B * 3 * nv * es
    rows = B * 3 * N[2] * N[1] * H0 * cs      # after the x pass
    planes = B * 3 * N[2] * M0[1] * H0 * cs    # after the y pass
    lam = 6 * (M0[2] // 2 + 1) * (M0[1] // 2 + 1) * H0 * es
    eps = nv * es
    plane_fit = info_plane_fits(info, N, es)
    if plane_fit:  # xy forward, z pass, xy inverse
        return (vec + planes) + (2 * planes + lam) + (planes + eps + 2 * vec)
    # x forward, y forward, z pass, y inverse, x inverse
    return (vec + rows) + (rows + planes) + (2 * planes + lam) + (planes + rows) + (rows + eps + 2 * vec)


def info_plane_fits(info, N, es):
    """Mirror of the library's choice: a whole (x, y) plane in 200 KB of shared memory."""
    Mx, My = info.M0[0], info.M0[1]
    H = Mx // 2 + 1
    return (Mx + My + 2 * My * H + 2 * ((N[1] + 1) // 2) * Mx) * 2 * es <= 200 * 1024


def run(workload="cube64_a8", nrhs=None, dtype="f32", warmup=3, reps=20, kernels=False, device=0):
    import numpy as np
    import torch

    import paper_2607_28309_b300 as mot
    from paper_2607_28309_b300 import build, synthetic

    build.build()
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream()
    w = synthetic.workload(workload)
    B = int(nrhs or len(w["exc"]))
    N = w["N"]
    nv = int(np.prod(N))
    dt, tdt, es = {"f32": (mot.MOT_F32, torch.float32, 4), "f64": (mot.MOT_F64, torch.float64, 8),
                   "f64df": (mot.MOT_F64DF, torch.float64, 8)}[dtype]
    ctx = mot.mot_ctx_create(device, stream.cuda_stream)
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"])
    try:
        info = mot.mot_problem_info_get(prob)
        gen = torch.Generator(device="cuda").manual_seed(11)
        x = torch.randn(B, 3, nv, dtype=tdt, device="cuda", generator=gen)
        y = torch.empty_like(x)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        for _ in range(warmup):
            mot.mot_apply_Z0(prob, x, y, B, dt)
        torch.cuda.synchronize()
        ts = []
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" selects these products
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mot.mot_apply_Z0(prob, x, y, B, dt)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        torch.cuda.nvtx.range_pop()
        us = statistics.median(ts)
        K0 = [m // 2 + 1 for m in info.M0]
        alg = 2 * B * 3 * nv * es + nv * es + 6 * K0[0] * K0[1] * K0[2] * es
        passes = pass_bytes(info, N, B, es)
        peak = None
        pk = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
        if os.path.exists(pk):
            with open(pk) as f:
                peak = json.load(f).get("hbm_gbs")
        out = {"workload": workload, "grid": list(N), "M0": list(info.M0), "nrhs": B, "dtype": dtype,
               "us_median": us, "us_min": min(ts), "reps": reps, "alg_bytes": alg, "pass_bytes": passes,
               "alg_GBps": alg / us / 1e3, "pass_GBps": passes / us / 1e3, "peak_GBps": peak,
               "plane_passes": info_plane_fits(info, N, es)}
        if peak:
            out["alg_frac"] = out["alg_GBps"] / peak
            out["pass_frac"] = out["pass_GBps"] / peak
        if dtype == "f64df":  # the double-float product against the FP64 one
            y64 = torch.empty_like(x)
            mot.mot_apply_Z0(prob, x, y64, B, mot.MOT_F64)
            torch.cuda.synchronize()
            out["rel_l2_vs_f64"] = float(torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64))
        if kernels:
            from torch.profiler import ProfilerActivity, profile

            with profile(activities=[ProfilerActivity.CUDA]) as pr:
                for _ in range(reps):
                    mot.mot_apply_Z0(prob, x, y, B, dt)
                torch.cuda.synchronize()
            agg = {}
            for e in pr.events():
                if e.device_type == torch.autograd.DeviceType.CUDA:
                    k = e.name.split("(")[0]
                    n, t = agg.get(k, (0, 0.0))
                    agg[k] = (n + 1, t + e.device_time_total)
            out["kernels_us_per_product"] = {k: t / reps for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])}
        return out
    finally:
        mot.mot_problem_destroy(prob)
        mot.mot_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="cube64_a8")
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides (default: the workload's plane waves)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "f64df"])
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--kernels", action="store_true")
    a = ap.parse_args()
    print(json.dumps(run(a.workload, a.nrhs, a.dtype, a.warmup, a.reps, a.kernels)))


if __name__ == "__main__":
    main()
