"""Error behaviour of the C ABI that needs a device context: argument validation
of mot_problem_create / mot_run_create (eps_r finite and >= 1, khat and the
polarisation orthogonal unit vectors, sigma > 0, Sec. II and Eq. 7-8), and
MOT_ENOTCONV when a step's solve is cut off by the iteration cap (the march goes
on and the currents of every step are still returned)."""
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


def _status(f, *a, **k):
    with pytest.raises(mot.MotError) as e:
        f(*a, **k)
    return e.value.status


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), 0.5, -2.0])
def test_problem_rejects_bad_permittivity(ctx, bad):
    N = (4, 3, 5)
    eps = np.full(N[::-1], 2.0)
    eps[1, 2, 3] = bad
    assert _status(mot.mot_problem_create, ctx, N, 10e-9, eps, 4.0) == mot.MOT_EINVAL
    assert "eps_r" in mot.mot_last_error()


@pytest.mark.parametrize("h,alpha", [(0.0, 4.0), (-1e-9, 4.0), (float("nan"), 4.0), (10e-9, 0.0), (10e-9, -1.0),
                                     (10e-9, float("inf"))])
def test_problem_rejects_bad_step_or_spacing(ctx, h, alpha):
    N = (4, 3, 5)
    assert _status(mot.mot_problem_create, ctx, N, h, np.full(N[::-1], 2.0), alpha) == mot.MOT_EINVAL


@pytest.mark.parametrize("delta", [float("nan"), float("inf")])
def test_problem_rejects_non_finite_delta(ctx, delta):
    N = (4, 3, 5)
    opt = mot.default_options(delta=delta)
    assert _status(mot.mot_problem_create, ctx, N, 10e-9, np.full(N[::-1], 2.0), 4.0, opt) == mot.MOT_EINVAL
    assert "delta" in mot.mot_last_error()


def test_bad_precision_and_dtype_are_refused(ctx):
    N = (4, 3, 5)
    prob = mot.mot_problem_create(ctx, N, 10e-9, np.full(N[::-1], 2.0), 4.0)
    try:
        for bad in (-1, 3):
            assert _status(mot.mot_run_create, prob, [synthetic.pulse(8, 4.0)], bad) == mot.MOT_EINVAL
            x = torch.zeros(3 * int(np.prod(N)), dtype=torch.float64, device="cuda")
            y = torch.zeros_like(x)
            assert _status(mot.mot_apply_Z0, prob, x, y, 1, bad) == mot.MOT_EINVAL
            assert _status(mot.mot_apply_Z0_static, prob, x, y, 1, bad) == mot.MOT_EINVAL
    finally:
        mot.mot_problem_destroy(prob)


def test_run_rejects_bad_plane_waves(ctx):
    N = (5, 4, 3)
    prob = mot.mot_problem_create(ctx, N, 10e-9, np.full(N[::-1], 3.0), 4.0)
    try:
        good = synthetic.pulse(10, 4.0)
        cases = [
            dict(good, khat=(0.0, 0.0, 2.0)),                     # not a unit vector
            dict(good, khat=(0.0, 0.6, 0.6)),                     # not a unit vector
            dict(good, pol=(1.0, 1.0, 0.0)),                      # not a unit vector
            dict(good, pol=(0.0, 0.0, 1.0)),                      # parallel to khat
            dict(good, pol=(math.sqrt(0.5), 0.0, math.sqrt(0.5))),  # not orthogonal to khat
            dict(good, sigma=0.0),
            dict(good, sigma=-1e-15),
            dict(good, t0=float("nan")),
        ]
        for pw in cases:
            assert _status(mot.mot_run_create, prob, [good, pw], mot.MOT_MIXED) == mot.MOT_EINVAL, pw
        # the good wave alone is accepted
        run = mot.mot_run_create(prob, [good], mot.MOT_MIXED)
        mot.mot_run_destroy(run)
    finally:
        mot.mot_problem_destroy(prob)


@pytest.mark.parametrize("precision", [mot.MOT_FP64, mot.MOT_MIXED, mot.MOT_FP64DF])
@pytest.mark.parametrize("graph", [0, 1, 2])
def test_iteration_cap_gives_notconv(ctx, precision, graph):
    N = (8, 7, 6)
    eps = synthetic.block_eps(N, 2, 4.0, 12.0, 3)
    steps = 8
    opt = mot.default_options(maxit=1, max_refine=1, graph=graph)
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, 8.0, opt)
    try:
        run = mot.mot_run_create(prob, [synthetic.pulse(steps, 8.0)], precision)
        try:
            J = np.zeros((steps, 1, 3, int(np.prod(N))))
            stats = (mot.mot_step_stats * steps)()
            st = mot.mot_run_step(run, steps, J, stats, allow_notconv=True)
            assert st == mot.MOT_ENOTCONV
            assert "tolerance" in mot.mot_last_error()
            # every step ran and returned its currents; the pulse drives them
            assert mot.mot_run_step_index(run) == steps
            assert np.abs(J[steps // 2]).max() > 0
            assert max(s.relres for s in stats) > 1e-8
        finally:
            mot.mot_run_destroy(run)
    finally:
        mot.mot_problem_destroy(prob)
