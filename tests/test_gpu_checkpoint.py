"""Checkpoint and resume of a march (mot_run_save / mot_run_load).

A run marched n1 steps, saved, and resumed from the file in a fresh run must
produce the same currents for the following steps as the uninterrupted run
(the state that carries over is J_{n-1}, J_{n-2} (and J_{n-3} for the quadratic
guess), the history ring and the
step index; everything else is rebuilt).  The uninterrupted run continues in
graph mode while the resumed one takes its first step host-driven, so the
comparison allows the drivers' rounding difference (1e-12 relative).
"""
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
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return float(np.linalg.norm(a - b, axis=1).max() / max(np.linalg.norm(b, axis=1).max(), 1e-300))


@pytest.mark.parametrize("precision", [mot.MOT_FP64, mot.MOT_MIXED, mot.MOT_FP64DF])
def test_resume_matches_uninterrupted(ctx, tmp_path, precision):
    N = (10, 9, 8)
    eps = synthetic.block_eps(N, 3, 2.0, 5.0, 3)
    alpha, steps, n1 = 8.0, 12, 5
    exc = synthetic.oblique_set(steps, alpha, angles_deg=(0, 40))
    nv = int(np.prod(N))
    path = tmp_path / "run.ckpt"
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
    try:
        run = mot.mot_run_create(prob, exc, precision)
        try:
            J = np.zeros((steps, len(exc), 3, nv))
            mot.mot_run_step(run, n1, J[:n1])
            mot.mot_run_save(run, path)
            mot.mot_run_step(run, steps - n1, J[n1:])
        finally:
            mot.mot_run_destroy(run)
        assert np.abs(J[n1:]).max() > 0
        run2 = mot.mot_run_load(prob, path)
        try:
            assert mot.mot_run_step_index(run2) == n1
            J2 = np.zeros((steps - n1, len(exc), 3, nv))
            mot.mot_run_step(run2, steps - n1, J2)
            assert mot.mot_run_step_index(run2) == steps
        finally:
            mot.mot_run_destroy(run2)
        assert _rel(J2, J[n1:]) <= 1e-12
    finally:
        mot.mot_problem_destroy(prob)


def test_checkpoint_of_another_problem_is_refused(ctx, tmp_path):
    N = (6, 6, 6)
    eps = synthetic.block_eps(N, 3, 2.0, 4.0, 9)
    path = tmp_path / "a.ckpt"
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, 4.0)
    other = mot.mot_problem_create(ctx, N, 10e-9, eps * 1.01, 4.0)
    try:
        run = mot.mot_run_create(prob, [synthetic.pulse(8, 4.0)], mot.MOT_MIXED)
        mot.mot_run_step(run, 2)
        mot.mot_run_save(run, path)
        mot.mot_run_destroy(run)
        with pytest.raises(mot.MotError) as e:
            mot.mot_run_load(other, path)
        assert e.value.status == mot.MOT_EINVAL
        # a truncated file is refused too
        data = path.read_bytes()
        bad = tmp_path / "bad.ckpt"
        bad.write_bytes(data[: len(data) // 2])
        with pytest.raises(mot.MotError) as e:
            mot.mot_run_load(prob, bad)
        assert e.value.status == mot.MOT_EINVAL
    finally:
        mot.mot_problem_destroy(other)
        mot.mot_problem_destroy(prob)


@pytest.mark.parametrize("g_save,g_load", [(2, 1), (1, 2), (0, 2)])
def test_resume_with_another_initial_guess(ctx, tmp_path, g_save, g_load):
    """A checkpoint of a run with one initial-guess rule loads into a problem
    with another: J_{n-3} (kept by guess 2) is skipped when not needed and
    taken as J_{n-2} when missing.  Only the solver's starting points differ,
    so the resumed FP64 march agrees with the uninterrupted one to the solver
    tolerance."""
    N = (8, 7, 6)
    eps = synthetic.block_eps(N, 2, 2.0, 5.0, 8)
    alpha, steps, n1 = 8.0, 10, 4
    exc = [synthetic.pulse(steps, alpha)]
    nv = int(np.prod(N))
    path = tmp_path / "run.ckpt"
    p1 = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha, mot.default_options(guess=g_save))
    p2 = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha, mot.default_options(guess=g_load))
    try:
        run = mot.mot_run_create(p1, exc, mot.MOT_FP64)
        try:
            J = np.zeros((steps, 1, 3, nv))
            mot.mot_run_step(run, n1, J[:n1])
            mot.mot_run_save(run, path)
            mot.mot_run_step(run, steps - n1, J[n1:])
        finally:
            mot.mot_run_destroy(run)
        run2 = mot.mot_run_load(p2, path)
        try:
            J2 = np.zeros((steps - n1, 1, 3, nv))
            mot.mot_run_step(run2, steps - n1, J2)
        finally:
            mot.mot_run_destroy(run2)
        assert np.abs(J[n1:]).max() > 0
        assert _rel(J2, J[n1:]) <= 1e-9
    finally:
        mot.mot_problem_destroy(p2)
        mot.mot_problem_destroy(p1)
