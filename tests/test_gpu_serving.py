"""Serving: runs of different sizes admitted into a running server (continuous
batching) give the same currents as each run alone; admission respects the
memory budget; waits are bounded by their timeout.

Tolerance: the server runs the same kernels and step drivers as a run alone
(first step host-driven, then one CUDA graph per step), so the results agree
to 1e-12 relative (they are normally bit-identical).
"""
import time

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


SPECS = [  # grid, alpha, precision, steps, plane waves
    ((8, 8, 8), 4.0, mot.MOT_MIXED, 12, 1),
    ((12, 10, 9), 8.0, mot.MOT_MIXED, 10, 2),
    ((6, 7, 8), 16.0, mot.MOT_FP64, 8, 1),
    ((16, 16, 16), 8.0, mot.MOT_MIXED, 10, 1),
    ((10, 10, 10), 4.0, mot.MOT_FP64, 14, 2),
]


def _inputs(i, N, alpha, steps, nexc):
    eps = synthetic.block_eps(N, 2, 1.5, 6.0, 40 + i)
    exc = synthetic.oblique_set(steps, alpha, angles_deg=(0, 30))[:nexc] if nexc > 1 else [synthetic.pulse(steps, alpha)]
    return eps, exc


def _alone(ctx, N, eps, alpha, exc, prec, steps):
    nv = int(np.prod(N))
    prob = mot.mot_problem_create(ctx, N, 10e-9, eps, alpha)
    try:
        run = mot.mot_run_create(prob, exc, prec)
        try:
            J = np.zeros((steps, len(exc), 3, nv))
            mot.mot_run_step(run, steps, J)
        finally:
            mot.mot_run_destroy(run)
    finally:
        mot.mot_problem_destroy(prob)
    return J[-1]


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_runs_alone_and_in_the_mix_agree(ctx):
    inputs = [_inputs(i, N, a, s, ne) for i, (N, a, p, s, ne) in enumerate(SPECS)]
    alone = [_alone(ctx, N, eps, a, exc, p, s) for (N, a, p, s, ne), (eps, exc) in zip(SPECS, inputs)]
    srv = mot.mot_server_create(ctx, 0, 3)
    try:
        outs, tickets = [], []
        for i, ((N, a, p, s, ne), (eps, exc)) in enumerate(zip(SPECS, inputs)):
            out = np.zeros((ne, 3, int(np.prod(N))))
            tickets.append(mot.mot_server_submit(srv, N, 10e-9, eps, a, exc, s, p, J_final=out))
            outs.append(out)
            if i == 2:
                time.sleep(0.05)  # the last two arrive while the first three are on the GPU
        results = [mot.mot_server_wait(srv, t, 120.0) for t in tickets]
    finally:
        mot.mot_server_destroy(srv)
    for (N, a, p, s, ne), res, out, ref in zip(SPECS, results, outs, alone):
        assert res.status == mot.MOT_OK
        assert res.steps == s
        assert np.abs(ref).max() > 0
        assert _rel(out, ref) <= 1e-12
        assert res.run_ms > 0 and res.step_p99_ms >= res.step_p50_ms > 0
        assert res.device_bytes > 0


def test_admission_budget_and_bounded_wait(ctx):
    N, a, p, s, ne = (6, 6, 6), 4.0, mot.MOT_MIXED, 6, 1
    eps, exc = _inputs(0, N, a, s, ne)
    # a budget no run fits in: the request completes with MOT_ENOMEM
    srv = mot.mot_server_create(ctx, 1 << 20, 1)
    try:
        t = mot.mot_server_submit(srv, N, 10e-9, eps, a, exc, s, p)
        assert mot.mot_server_wait(srv, t, 30.0).status == mot.MOT_ENOMEM
    finally:
        mot.mot_server_destroy(srv)
    # a zero timeout on a run that cannot have finished yet returns MOT_ETIMEOUT
    srv = mot.mot_server_create(ctx, 0, 1)
    try:
        N2 = (24, 24, 24)
        eps2 = synthetic.block_eps(N2, 4, 1.5, 6.0, 77)
        t = mot.mot_server_submit(srv, N2, 10e-9, eps2, 8.0, [synthetic.pulse(40, 8.0)], 40, mot.MOT_MIXED)
        with pytest.raises(mot.MotError) as e:
            mot.mot_server_wait(srv, t, 0.0)
        assert e.value.status == mot.MOT_ETIMEOUT
        res = mot.mot_server_wait(srv, t, 120.0)
        assert res.status == mot.MOT_OK and res.steps == 40
        with pytest.raises(mot.MotError) as e:  # collected tickets are released
            mot.mot_server_wait(srv, t, 0.0)
        assert e.value.status == mot.MOT_EINVAL
    finally:
        mot.mot_server_destroy(srv)


def test_problems_of_one_step_and_grid_share_history_spectra(ctx):
    """Two problems with the same grid and time step (different eps_r) hold one
    copy of the history spectra Lambda_k on the device (they do not depend on
    eps_r): the second run costs less device memory by about that size, and
    each run's currents equal the run alone."""
    N, alpha, steps = (64, 64, 48), 8.0, 12  # spectra ~130 MB: well above the allocation granularity
    exc = [synthetic.pulse(steps, alpha)]
    eps_a = synthetic.block_eps(N, 4, 1.5, 6.0, 91)
    eps_b = synthetic.block_eps(N, 4, 1.5, 6.0, 92)
    alone_b = _alone(ctx, N, eps_b, alpha, exc, mot.MOT_MIXED, steps)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pa = mot.mot_problem_create(ctx, N, 10e-9, eps_a, alpha)
    ra = mot.mot_run_create(pa, exc, mot.MOT_MIXED)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    pb = mot.mot_problem_create(ctx, N, 10e-9, eps_b, alpha)
    rb = mot.mot_run_create(pb, exc, mot.MOT_MIXED)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    try:
        info = mot.mot_problem_info_get(pb)
        Kh = [m // 2 + 1 for m in info.Mh]
        spectra = (info.ell + 1) * 6 * Kh[0] * Kh[1] * Kh[2] * 4
        used_a, used_b = free0 - free1, free1 - free2
        assert used_a - used_b >= 0.9 * spectra, (used_a, used_b, spectra)
        nv = int(np.prod(N))
        J = np.zeros((steps, 1, 3, nv))
        mot.mot_run_step(rb, steps, J)
        assert np.abs(J[-1] - alone_b).max() <= 1e-12 * np.abs(alone_b).max()
        # the first problem goes; the second keeps the shared spectra
        mot.mot_run_destroy(ra)
        mot.mot_problem_destroy(pa)
        ra = pa = None
        J2 = np.zeros((2, 1, 3, nv))
        mot.mot_run_step(rb, 2, J2)
        assert np.isfinite(J2).all() and np.abs(J2).max() > 0
    finally:
        if ra is not None:
            mot.mot_run_destroy(ra)
        if pa is not None:
            mot.mot_problem_destroy(pa)
        mot.mot_run_destroy(rb)
        mot.mot_problem_destroy(pb)
