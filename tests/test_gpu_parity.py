"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 unless stated):
- FP64 Z0 FFT product vs the oracle's direct product:            1e-10
- FP32 Z0 FFT product vs the oracle:                             1e-5 (measured value reported)
- double-float (FP32-pair) Z0 product vs the oracle with the oracle's
  table loaded, and vs the FP64 product at full size:              1e-13
- library lag tables vs the oracle's tables:                      1e-12 absolute
- FP64 march vs the oracle march (exact solve), per step, scaled
  by max_n ||J_n||:                                                1e-9
- mixed FP32/FP64 march vs the oracle, same scaling:               1e-5
- double-float refined march (FP32 inner solves, double-float
  residual and history) vs the oracle, same scaling:              1e-9
"""
import math

import numpy as np
import pytest

import paper_2607_28309_b300 as mot
from paper_2607_28309_b300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _apply(prob, x_np, nrhs, dtype):
    tdt = torch.float32 if dtype == mot.MOT_F32 else torch.float64
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to("cuda", tdt)
    y = torch.empty_like(x)
    mot.mot_apply_Z0(prob, x, y, nrhs, dtype)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


GRIDS = [((5, 6, 7), 4.0), ((12, 12, 12), 8.0), ((16, 9, 11), 16.0), ((20, 20, 20), 1.0), ((1, 1, 1), 4.0),
         ((1, 2, 3), 8.0), ((3, 17, 2), 2.0), ((33, 8, 10), 4.0)]


@pytest.mark.parametrize("N,alpha", GRIDS)
def test_z0_fft_product_matches_direct(ctx, orc, N, alpha):
    rng = np.random.default_rng(sum(N) + int(alpha))
    eps = rng.uniform(1.0, 6.0, size=N[::-1])
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
    try:
        rho = alpha / math.sqrt(3)
        R = orc.table_extent(0, rho, N)
        g = orc.lag_table(0, rho, R)
        # the library's own table equals the oracle's
        Rl, gl = mot.mot_kernel_table(prob, 0)
        assert tuple(Rl) == tuple(R)
        assert np.abs(gl - g).max() <= 1e-12
        for nrhs in (1, 2):
            x = rng.standard_normal((nrhs, 3) + N[::-1])
            ref = np.stack([orc.Zk_apply(0, N, eps, R, g, x[b]) for b in range(nrhs)])
            y64 = _apply(prob, x, nrhs, mot.MOT_F64)
            assert _rel(y64, ref) <= 1e-10
            y32 = _apply(prob, x, nrhs, mot.MOT_F32)
            assert _rel(y32, ref) <= 1e-5
        # the same product with the oracle's table loaded into the FFT path: what is
        # left is the FFT's rounding, FP64 and double-float (FP32 pairs, the
        # FP64-accuracy product of a GPU with a slow FP64 pipe; target 1e-13)
        mot.mot_set_kernel_table(prob, 0, g, R)
        x = rng.standard_normal((2, 3) + N[::-1])
        ref = np.stack([orc.Zk_apply(0, N, eps, R, g, x[b]) for b in range(2)])
        e64 = _rel(_apply(prob, x, 2, mot.MOT_F64), ref)
        edf = _rel(_apply(prob, x, 2, mot.MOT_F64DF), ref)
        print(f"{N} alpha {alpha}: FP64 {e64:.2e}, double-float {edf:.2e}")
        assert e64 <= 1e-10
        assert edf <= 1e-13
    finally:
        mot.mot_problem_destroy(prob)


def _march_pair(ctx, orc, N, eps, alpha, exc, steps, precision, opt=None):
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha, opt)
    try:
        run = mot.mot_run_create(prob, exc, precision)
        try:
            nv = int(np.prod(N))
            J = np.zeros((steps, len(exc), 3, nv))
            mot.mot_run_step(run, steps, J)
        finally:
            mot.mot_run_destroy(run)
    finally:
        mot.mot_problem_destroy(prob)
    return J


def _mot_errors(Jg, Jo):
    steps = Jo.shape[0]
    Jo = Jo.reshape(steps, -1)
    Jg = Jg.reshape(steps, -1)
    scale = np.linalg.norm(Jo, axis=1).max()
    return np.linalg.norm(Jg - Jo, axis=1) / scale


def test_mot_small_fp64_and_mixed(ctx, orc):
    N = (6, 5, 7)
    eps = synthetic.block_eps(N, 2, 2.0, 4.0, 21)
    alpha, steps = 4.0, 30
    exc = [synthetic.pulse(steps, alpha), synthetic.pulse(steps, alpha, pol=(0.0, 1.0, 0.0))]
    P = orc.Problem(N, 10e-9, eps, alpha)
    Jo = P.march(exc, steps)
    e64 = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_FP64), Jo)
    assert e64.max() <= 1e-9, e64.max()
    e32 = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_MIXED), Jo)
    assert e32.max() <= 1e-5, e32.max()
    edf = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_FP64DF), Jo)
    print("FP64 / mixed / double-float march errors", e64.max(), e32.max(), edf.max())
    assert edf.max() <= 1e-9, edf.max()


@pytest.mark.parametrize("guess", [0, 1, 2])
def test_march_initial_guesses(ctx, orc, guess):
    """Every initial guess of the step's solve (J_{n-1}; its linear and its
    quadratic extrapolation) reaches the oracle's march: the guess moves the
    solver's starting point only."""
    N = (7, 6, 5)
    eps = synthetic.block_eps(N, 2, 1.5, 5.0, 33)
    alpha, steps = 4.0, 24
    exc = [synthetic.pulse(steps, alpha)]
    Jo = orc.Problem(N, 10e-9, eps, alpha).march(exc, steps)
    for prec, tol in ((mot.MOT_FP64, 1e-9), (mot.MOT_MIXED, 1e-5)):
        e = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, prec, mot.default_options(guess=guess)), Jo)
        assert e.max() <= tol, (guess, prec, e.max())


def test_mot_oblique_batch(ctx, orc):
    N = (8, 8, 8)
    eps = synthetic.block_eps(N, 4, 2.0, 4.0, 4)
    alpha, steps = 8.0, 16
    exc = synthetic.oblique_set(steps, alpha, angles_deg=(0, 30, 70))
    Jo = orc.Problem(N, 10e-9, eps, alpha).march(exc, steps)
    e64 = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_FP64), Jo)
    assert e64.max() <= 1e-9, e64.max()
    edf = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_FP64DF), Jo)
    assert edf.max() <= 1e-9, edf.max()


def test_step_drivers_agree(ctx, orc):
    """The three step drivers (one CUDA graph per step, host-driven steps with a
    graph per TFQMR loop, no graphs at all) run the same kernels on the same
    data and take the same convergence decisions."""
    N = (9, 7, 8)
    eps = synthetic.block_eps(N, 3, 2.0, 5.0, 8)
    alpha, steps = 8.0, 14
    exc = [synthetic.pulse(steps, alpha)]
    Jo = orc.Problem(N, 10e-9, eps, alpha).march(exc, steps)
    for precision, tol in ((mot.MOT_FP64, 1e-9), (mot.MOT_MIXED, 1e-5), (mot.MOT_FP64DF, 1e-9)):
        J = {g: _march_pair(ctx, orc, N, eps, alpha, exc, steps, precision, mot.default_options(graph=g))
             for g in (0, 1, 2)}
        for g in (0, 1, 2):
            assert _mot_errors(J[g], Jo).max() <= tol, (precision, g)
        assert np.array_equal(J[0], J[2]), precision
        assert _mot_errors(J[1], J[0]).max() <= 1e-12, precision


def test_steps_in_several_calls_match_one_call(ctx):
    """The step graph takes each step's lags 2.. history partial sum from the
    previous step (computed beside its solve); the first graph step of every
    mot_run_step call computes it in front.  Any split of a march into calls
    gives the same currents bit for bit, past the history length."""
    N = (9, 7, 8)
    eps = synthetic.block_eps(N, 3, 2.0, 5.0, 8)
    alpha, steps = 8.0, 16
    exc = [synthetic.pulse(steps, alpha)]
    nv = int(np.prod(N))
    for precision in (mot.MOT_FP64, mot.MOT_MIXED, mot.MOT_FP64DF):
        prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
        try:
            J = {}
            for split in ((steps,), (1, 4, 2, 9), (3, 1, 1, 11)):
                run = mot.mot_run_create(prob, exc, precision)
                try:
                    Js, k = np.zeros((steps, 1, 3, nv)), 0
                    for c in split:
                        mot.mot_run_step(run, c, Js[k:k + c])
                        k += c
                finally:
                    mot.mot_run_destroy(run)
                J[split] = Js
            ref = J[(steps,)]
            assert np.abs(ref[-1]).max() > 0
            for split, Js in J.items():
                assert np.array_equal(Js, ref), (precision, split)
        finally:
            mot.mot_problem_destroy(prob)


def test_zero_contrast_gives_zero_current(ctx):
    N = (7, 6, 5)
    J = _march_pair(ctx, None, N, np.ones(N[::-1]), 4.0, [synthetic.pulse(20, 4.0)], 20, mot.MOT_FP64)
    assert np.all(J == 0.0)
    J = _march_pair(ctx, None, N, np.ones(N[::-1]), 4.0, [synthetic.pulse(20, 4.0)], 20, mot.MOT_MIXED)
    assert np.all(J == 0.0)


def test_cube16_full_march(ctx, orc):
    """16^3 cube, eps_r U[2,4] per 4^3 block, alpha 4, 100 steps: FP64 and mixed."""
    w = synthetic.cube16()
    P = orc.Problem(w["N"], w["h"], w["eps"], w["alpha"])
    Jo = P.march(w["exc"], w["steps"])
    e64 = _mot_errors(_march_pair(ctx, orc, w["N"], w["eps"], w["alpha"], w["exc"], w["steps"], mot.MOT_FP64), Jo)
    assert e64.max() <= 1e-9, e64.max()
    e32 = _mot_errors(_march_pair(ctx, orc, w["N"], w["eps"], w["alpha"], w["exc"], w["steps"], mot.MOT_MIXED), Jo)
    assert e32.max() <= 1e-5, e32.max()


@pytest.mark.parametrize("which", ["cube64_a8", "cube64_a16", "pillars8x8", "cube64_b16"])
def test_full_size_product_sampled_rows(ctx, orc, which):
    """Z0 product at the full workload sizes (the bench's launch configuration),
    1024 rows checked one by one against the oracle's direct sum."""
    if which == "cube64_a8":
        w = synthetic.cube64(8.0)
    elif which == "cube64_a16":
        w = synthetic.cube64(16.0)
    elif which == "pillars8x8":
        w = synthetic.pillars8x8()
    else:
        w = synthetic.cube64_batch16()
    N, eps, alpha = w["N"], w["eps"], w["alpha"]
    nrhs = len(w["exc"])
    rng = np.random.default_rng(123)
    nv = int(np.prod(N))
    x = rng.standard_normal((nrhs, 3, nv))
    prob = mot.mot_problem_create(ctx, N, w["h"], eps, alpha)
    try:
        rho = alpha / math.sqrt(3)
        R = orc.table_extent(0, rho, N)
        g = orc.lag_table(0, rho, R)
        y64 = _apply(prob, x, nrhs, mot.MOT_F64)
        y32 = _apply(prob, x, nrhs, mot.MOT_F32)
        ydf = _apply(prob, x, nrhs, mot.MOT_F64DF)
    finally:
        mot.mot_problem_destroy(prob)
    # double-float against FP64 on every element (the same tables): 1e-13
    edf = _rel(ydf, y64)
    print(f"{which}: double-float vs FP64 product {edf:.2e}")
    assert edf <= 1e-13
    bsel = rng.integers(0, nrhs, 1024)
    psel = rng.integers(0, 3, 1024)
    msel = rng.integers(0, nv, 1024)
    ref = np.empty(1024)
    for b in np.unique(bsel):
        sel = bsel == b
        ref[sel] = orc.Zk_rows(0, N, eps, R, g, x[b].reshape(3, N[2], N[1], N[0]), psel[sel], msel[sel])
    got64 = y64[bsel, psel, msel]
    got32 = y32[bsel, psel, msel]
    assert _rel(got64, ref) <= 1e-10
    assert _rel(got32, ref) <= 1e-5


@pytest.mark.parametrize("N,alpha", [((5, 6, 7), 1.0), ((12, 12, 12), 4.0), ((16, 9, 11), 8.0), ((20, 13, 9), 16.0),
                                     ((1, 1, 1), 4.0), ((33, 8, 10), 2.0)])
def test_direct_product_matches_oracle(ctx, orc, N, alpha):
    """The GPU direct product (sum over the lag-0 support, the paper's direct
    MVP) against the oracle's direct product on ragged grids, and against the
    FFT product: FP64 1e-12, FP32 1e-5 relative L2."""
    rng = np.random.default_rng(7 + sum(N) + int(alpha))
    eps = rng.uniform(1.0, 6.0, size=N[::-1])
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
    try:
        rho = alpha / math.sqrt(3)
        R = orc.table_extent(0, rho, N)
        g = orc.lag_table(0, rho, R)
        for nrhs in (1, 3):
            x = rng.standard_normal((nrhs, 3) + N[::-1])
            ref = np.stack([orc.Zk_apply(0, N, eps, R, g, x[b]) for b in range(nrhs)])
            for dt, tdt, tol in ((mot.MOT_F64, torch.float64, 1e-12), (mot.MOT_F32, torch.float32, 1e-5)):
                xt = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt)
                yd = torch.full_like(xt, float("nan"))
                mot.mot_apply_Z0_direct(prob, xt, yd, nrhs, dt)
                torch.cuda.synchronize()
                got = yd.double().cpu().numpy()
                assert np.isfinite(got).all()
                assert _rel(got, ref) <= tol, (dt, _rel(got, ref))
                yf = torch.empty_like(xt)
                mot.mot_apply_Z0(prob, xt, yf, nrhs, dt)
                torch.cuda.synchronize()
                assert _rel(got, yf.double().cpu().numpy()) <= (1e-10 if dt == mot.MOT_F64 else 2e-5)
    finally:
        mot.mot_problem_destroy(prob)


def test_delta_regularised_product_and_march(ctx, orc):
    """The delta-regularised MOT (Sec. II; the shift on the present-time matrix
    only): the FFT and direct Z0 products against the oracle's Z0 + delta I, and
    the FP64 and mixed marches against the oracle's march with the same shift
    (tolerances as for delta = 0)."""
    N, alpha, delta, steps = (7, 6, 5), 4.0, 0.35, 24
    eps = synthetic.block_eps(N, 2, 2.0, 5.0, 9)
    P = orc.Problem(N, 10e-9, eps, alpha, delta=delta)
    opt = mot.default_options(delta=delta)
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha, opt)
    try:
        rng = np.random.default_rng(11)
        x = rng.standard_normal((2, 3) + N[::-1])
        ref = np.stack([P.apply(0, x[b]) for b in range(2)])
        for dt, tdt, tol in ((mot.MOT_F64, torch.float64, 1e-10), (mot.MOT_F32, torch.float32, 1e-5)):
            assert _rel(_apply(prob, x, 2, dt), ref) <= tol
            xt = torch.from_numpy(np.ascontiguousarray(x)).to("cuda", tdt)
            yd = torch.empty_like(xt)
            mot.mot_apply_Z0_direct(prob, xt, yd, 2, dt)
            torch.cuda.synchronize()
            assert _rel(yd.double().cpu().numpy(), ref) <= tol
    finally:
        mot.mot_problem_destroy(prob)
    exc = [synthetic.pulse(steps, alpha)]
    Jo = P.march(exc, steps)
    e64 = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_FP64, opt), Jo)
    assert e64.max() <= 1e-9, e64.max()
    e32 = _mot_errors(_march_pair(ctx, orc, N, eps, alpha, exc, steps, mot.MOT_MIXED, opt), Jo)
    assert e32.max() <= 1e-5, e32.max()
    # the shift is not dropped: the unshifted march differs
    J0 = orc.Problem(N, 10e-9, eps, alpha).march(exc, steps)
    assert _mot_errors(J0, Jo).max() > 1e-3


_SPREAD_SCRIPT = r'''
import sys, numpy as np, torch
import paper_2607_28309_b300 as mot
from paper_2607_28309_b300 import synthetic
N = (9, 7, 8)
eps = synthetic.block_eps(N, 3, 2.0, 5.0, 8)
alpha, steps = 8.0, 30
ctx = mot.mot_ctx_create(0, torch.cuda.current_stream().cuda_stream)
prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
out = {}
for prec in (mot.MOT_FP64, mot.MOT_MIXED):
    run = mot.mot_run_create(prob, [synthetic.pulse(steps, alpha)], prec)
    J = np.zeros((steps, 1, 3, int(np.prod(N))))
    mot.mot_run_step(run, 11, J[:11])
    mot.mot_run_step(run, steps - 11, J[11:])
    mot.mot_run_destroy(run)
    out[str(prec)] = J
mot.mot_problem_destroy(prob)
mot.mot_ctx_destroy(ctx)
np.savez(sys.argv[1], **out)
'''


def test_spread_history_schedule_matches_whole_pass(tmp_path):
    """The spread schedule of the time-blocked history (the old part in chunks
    beside the previous block's steps, the recent part at the block start;
    MOTJVIE_HIST_SPREAD=1, read once per process) sums the same terms in another
    order: its march equals the whole-pass march to rounding, FP64 and mixed,
    past two time blocks and across a split of the march into calls."""
    import os
    import subprocess
    import sys

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    script = tmp_path / "march.py"
    script.write_text(_SPREAD_SCRIPT)
    res = {}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for spread in ("0", "1"):
        env = dict(os.environ, MOTJVIE_HIST_SPREAD=spread,
                   PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
        outp = tmp_path / f"J{spread}.npz"
        subprocess.run([sys.executable, str(script), str(outp)], check=True, env=env, timeout=600, cwd=root)
        res[spread] = np.load(outp)
    for prec, tol in ((str(mot.MOT_FP64), 1e-12), (str(mot.MOT_MIXED), 1e-6)):
        a, b = res["0"][prec], res["1"][prec]
        assert np.abs(a[-1]).max() > 0
        assert _mot_errors(b, a).max() <= tol, (prec, _mot_errors(b, a).max())
