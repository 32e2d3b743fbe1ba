"""Full-size step-equation parity (Eq. 3) of the whole march, at the sizes and in the
launch configuration the bench runs.

The oracle cannot march a 64^3 grid (its direct history is O(n^2) per step), but it
can evaluate Eq. 3 on sampled rows: for a step n past the history length,

    res_n(p, m) = sum_{k=0..ell} (Z_k J_{n-k})(p, m) - E^i_n(p, m)

with the oracle's own lag tables, its direct row-sampled product and its incident
field, fed the currents the GPU march produced.  A march whose fused TFQMR kernels,
history accumulation, ring push, incident term or epilogues were wrong anywhere
leaves a residual of the order of the rows themselves; a correct one leaves the
solver's tolerance (FP64 path: TFQMR to 1e-11; mixed path: FP32 FFT, history and
inner solve with an FP64 residual, within 1e-5).  The mixed march's relative L2
difference from the FP64 march is also checked and printed per step (the mixed
path's stated error, relative to the FP64 path).
"""
import math

import numpy as np
import pytest

import paper_2607_28309_b300 as mot
from paper_2607_28309_b300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROWS_PER_STEP = 256


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2607_28309_b300 import build

    build.build()
    c = mot.mot_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    torch.cuda.synchronize()
    mot.mot_ctx_destroy(c)


def _march(ctx, w, precision, nsteps, keep):
    """Currents J[n][b][3][nv] for the right-hand sides in `keep`.  Steps go in calls
    of as many steps as ~200 MB of host output holds (all of them for one plane
    wave), so that the step graph's overlapped history branch runs as in the bench."""
    N = w["N"]
    nv = int(np.prod(N))
    nrhs = len(w["exc"])
    prob = mot.mot_problem_create(ctx, N, w["h"], w["eps"], w["alpha"])
    try:
        info = mot.mot_problem_info_get(prob)
        run = mot.mot_run_create(prob, w["exc"], precision)
        try:
            out = np.zeros((nsteps, len(keep), 3, nv))
            chunk = max(1, min(nsteps, int(2e8 // (nrhs * 3 * nv * 8))))
            buf = np.zeros((chunk, nrhs, 3, nv))
            n = 0
            while n < nsteps:
                c = min(chunk, nsteps - n)
                mot.mot_run_step(run, c, buf[:c])
                out[n:n + c] = buf[:c][:, keep]
                n += c
        finally:
            mot.mot_run_destroy(run)
    finally:
        mot.mot_problem_destroy(prob)
    return out, int(info.ell)


def _step_residuals(orc, w, tables, J, keep, steps, rng, rows=ROWS_PER_STEP, pool=None):
    """Relative L2 of res_n over `rows` sampled rows (voxels drawn from `pool`, all
    voxels if None), per step in `steps`."""
    N, eps, h = w["N"], w["eps"], w["h"]
    nv = int(np.prod(N))
    dt = w["alpha"] * synthetic.dt_cfl(h)
    out = []
    for n in steps:
        b_sel = rng.integers(0, len(keep), rows)
        p_sel = rng.integers(0, 3, rows)
        m_sel = rng.integers(0, nv, rows) if pool is None else rng.choice(pool, rows)
        lhs = np.zeros(rows)
        rhs = np.zeros(rows)
        lhs0 = np.zeros(rows)
        for bi in np.unique(b_sel):
            sel = b_sel == bi
            pw = w["exc"][keep[bi]]
            inc = orc.incident(N, h, eps, pw, n * dt).reshape(3, nv)
            rhs[sel] = inc[p_sel[sel], m_sel[sel]]
            for k, (R, g) in enumerate(tables):
                if n - k < 0:
                    break
                x = J[n - k, bi].reshape(3, N[2], N[1], N[0])
                v = orc.Zk_rows(k, N, eps, R, g, x, p_sel[sel], m_sel[sel])
                lhs[sel] += v
                if k == 0:
                    lhs0[sel] = v
        scale = max(np.linalg.norm(lhs0), np.linalg.norm(rhs))
        assert scale > 0
        out.append(float(np.linalg.norm(lhs - rhs) / scale))
    return out


@pytest.mark.parametrize("which", ["cube64_a8", "cube64_b16"])
def test_step_equation_at_full_size(ctx, orc, which):
    w = synthetic.workload(which)
    N = w["N"]
    rho = w["alpha"] / math.sqrt(3)
    ell = orc.history_length(N, rho)
    nsteps = ell + 3
    # right-hand sides checked: one plane wave, or four of the sixteen oblique ones
    keep = [0] if len(w["exc"]) == 1 else [0, 5, 10, 15]
    tables = orc.lag_tables(N, rho, ell)
    # the pulse's peak (incident term large) and past the history length (ring wrapped)
    steps = [12, ell, ell + 2]
    rng = np.random.default_rng(2024)

    J64, ell_lib = _march(ctx, w, mot.MOT_FP64, nsteps, keep)
    assert ell_lib == ell
    assert np.abs(J64[-1]).max() > 0
    r64 = _step_residuals(orc, w, tables, J64, keep, steps, rng)
    print(f"{which} FP64 step-equation residuals", r64)
    assert max(r64) <= 1e-9, r64

    J32, _ = _march(ctx, w, mot.MOT_MIXED, nsteps, keep)
    r32 = _step_residuals(orc, w, tables, J32, keep, steps, rng)
    print(f"{which} mixed step-equation residuals", r32)
    assert max(r32) <= 1e-5, r32

    if which == "cube64_a8":
        # the double-float refined march holds the FP64 path's residual
        Jdf, _ = _march(ctx, w, mot.MOT_FP64DF, nsteps, keep)
        rdf = _step_residuals(orc, w, tables, Jdf, keep, steps, rng)
        print(f"{which} double-float step-equation residuals", rdf)
        assert max(rdf) <= 1e-9, rdf
        ddf = np.linalg.norm((Jdf - J64).reshape(nsteps, -1), axis=1).max()
        print(f"{which} double-float vs FP64 march: max relative L2 per step",
              ddf / np.linalg.norm(J64.reshape(nsteps, -1), axis=1).max())

    # the mixed path's relative L2 error against the FP64 path, per step
    d = J32.reshape(nsteps, -1) - J64.reshape(nsteps, -1)
    scale = np.linalg.norm(J64.reshape(nsteps, -1), axis=1).max()
    rel = np.linalg.norm(d, axis=1) / scale
    print(f"{which} mixed vs FP64 relative L2 per step: max {rel.max():.3e}, last {rel[-1]:.3e}")
    assert rel.max() <= 1e-5, rel.max()


def test_step_equation_on_the_pillar_array(ctx, orc):
    """The same check on the 256 x 256 x 80 pillar array at alpha 8 (15.7 M
    unknowns; 270-point present-time FFTs, 512 x 512 x 160 history grid, the
    bench's compiled shapes), over the first 14 steps: the time-blocked history's
    block pass (step 8 opens the second block) and its near-lag accumulations
    (steps 10, 13).  A pulse of a 40-step window puts its peak inside those steps;
    the oracle needs the lag tables 0..13 only.  Rows are sampled in the pillars
    (eps_r > 1): outside them the contrast, the current and the row vanish."""
    w = dict(synthetic.workload("pillars8x8"))
    w["exc"] = [synthetic.pulse(40, w["alpha"], w["h"], khat=(0.0, 0.0, -1.0))]
    N = w["N"]
    rho = w["alpha"] / math.sqrt(3)
    nsteps = 14
    tables = [(orc.table_extent(k, rho, N), None) for k in range(nsteps)]
    tables = [(R, orc.lag_table(k, rho, R)) for k, (R, _) in enumerate(tables)]
    steps = [8, 10, 13]
    pool = np.flatnonzero(np.asarray(w["eps"]).reshape(-1) > 1.0)
    J64, ell = _march(ctx, w, mot.MOT_FP64, nsteps, [0])
    assert ell > nsteps
    assert np.abs(J64[-1]).max() > 0
    r64 = _step_residuals(orc, w, tables, J64, [0], steps, np.random.default_rng(77), rows=96, pool=pool)
    print("pillars8x8 FP64 step-equation residuals", r64)
    assert max(r64) <= 1e-9, r64
    J32, _ = _march(ctx, w, mot.MOT_MIXED, nsteps, [0])
    r32 = _step_residuals(orc, w, tables, J32, [0], steps, np.random.default_rng(77), rows=96, pool=pool)
    print("pillars8x8 mixed step-equation residuals", r32)
    assert max(r32) <= 1e-5, r32
    d = J32.reshape(nsteps, -1) - J64.reshape(nsteps, -1)
    rel = np.linalg.norm(d, axis=1) / np.linalg.norm(J64.reshape(nsteps, -1), axis=1).max()
    print(f"pillars8x8 mixed vs FP64 relative L2 per step: max {rel.max():.3e}")
    assert rel.max() <= 1e-5, rel.max()
