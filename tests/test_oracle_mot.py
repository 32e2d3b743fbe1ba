"""Pins of the oracle's products and of its marching-on-in-time recursion (Eq. 3).

- matrix-free direct products equal explicitly assembled dense matrices whose
  entries are written out with plain loops (also with a random table that has
  no d -> -d symmetry, so that a reversed offset cannot hide);
- X^{-1} Z0 is symmetric (Z0 = D - X G with G symmetric, Eq. 10);
- zero contrast (eps_r = 1) gives exactly zero current;
- linearity in the excitation;
- one voxel driven slowly obeys Clausius-Mossotti, J -> 3(eps-1)/(eps+2) eps0 dE/dt,
  and its recursion has all characteristic roots inside the unit circle;
- refinement of dt at fixed physical time converges.
"""
import math

import numpy as np
import pytest

from paper_2607_28309_b300 import synthetic


def _dense_by_loops(orc, k, N, eps, R, g):
    Nx, Ny, Nz = N
    n = Nx * Ny * Nz
    comp = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    Z = np.zeros((3 * n, 3 * n))
    Tk = orc.temporal(k)
    for mz in range(Nz):
        for my in range(Ny):
            for mx in range(Nx):
                m = (mz * Ny + my) * Nx + mx
                e = eps[mz, my, mx]
                for sz in range(Nz):
                    for sy in range(Ny):
                        for sx in range(Nx):
                            s = (sz * Ny + sy) * Nx + sx
                            d = (mx - sx, my - sy, mz - sz)
                            if abs(d[0]) > R[0] or abs(d[1]) > R[1] or abs(d[2]) > R[2]:
                                continue
                            for p in range(3):
                                for q in range(3):
                                    Z[p * n + m, q * n + s] -= (e - 1) * g[comp[p][q], d[2] + R[2], d[1] + R[1], d[0] + R[0]]
                for p in range(3):
                    Z[p * n + m, p * n + m] += e * Tk
    return Z


def test_direct_product_equals_dense(orc):
    rng = np.random.default_rng(11)
    N = (3, 2, 4)
    eps = rng.uniform(1.5, 5, size=N[::-1])
    rho = orc.rho_of_alpha(4)
    for k in (0, 1, 2):
        R = orc.table_extent(k, rho, N)
        g = orc.lag_table(k, rho, R)
        for table in (g, rng.standard_normal(g.shape)):
            Z = _dense_by_loops(orc, k, N, eps, R, table)
            x = rng.standard_normal((3,) + N[::-1])
            y = orc.Zk_apply(k, N, eps, R, table, x)
            assert np.allclose(y.ravel(), Z @ x.ravel(), rtol=0, atol=1e-13 * np.abs(Z).max() * np.abs(x).max() * 30)
            # the sparse assembly used for the oracle's solve is the same matrix
            assert np.allclose(orc.assemble_Zk(k, N, eps, R, table, dense=True), Z, atol=1e-15)


def test_contrast_scaled_Z0_is_symmetric(orc):
    rng = np.random.default_rng(5)
    N = (3, 3, 3)
    eps = rng.uniform(2, 4, size=N[::-1])
    rho = orc.rho_of_alpha(8)
    R = orc.table_extent(0, rho, N)
    Z = orc.assemble_Zk(0, N, eps, R, orc.lag_table(0, rho, R), dense=True)
    X = np.tile((eps - 1).ravel(), 3)
    S = Z / X[:, None]
    assert np.allclose(S, S.T, atol=1e-14)


def _cube(orc, N, alpha, eps, nsteps, pws):
    P = orc.Problem(N, 10e-9, eps, alpha)
    return P, P.march(pws, nsteps)


def test_zero_contrast_gives_zero_current(orc):
    N = (4, 4, 4)
    pw = synthetic.pulse(30, 4, 10e-9)
    P, J = _cube(orc, N, 4, np.ones(N[::-1]), 30, [pw])
    assert np.all(J == 0.0)


def test_linearity(orc):
    N = (4, 3, 5)
    rng = np.random.default_rng(2)
    eps = rng.uniform(2, 4, size=N[::-1])
    h = 10e-9
    base = synthetic.pulse(40, 4, h)
    px = dict(base, pol=(1.0, 0.0, 0.0))
    py = dict(base, pol=(0.0, 1.0, 0.0))
    pxy = dict(base, pol=(1 / math.sqrt(2), 1 / math.sqrt(2), 0.0), E0=math.sqrt(2))
    P = orc.Problem(N, h, eps, 4)
    J = P.march([px, py, pxy], 40)
    ref = J[:, 0] + J[:, 1]
    assert np.abs(J[:, 2] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("alpha", [1, 4, 16])
def test_single_voxel_recursion_roots(orc, alpha):
    rho = orc.rho_of_alpha(alpha)
    for eps in (1.5, 4.0, 12.0, 36.0):
        Z = []
        k = 0
        while k < 2 or orc.in_support(k, rho, (0, 0, 0)):
            Z.append(eps * orc.temporal(k) - (eps - 1) * orc.g_raw(k, rho, (0, 0, 0))[0])
            k += 1
        assert abs(sum(Z) - (eps + 2) / 3) < 1e-14 * eps
        assert np.abs(np.roots(Z)).max() < 1.0


def test_single_voxel_clausius_mossotti(orc):
    h, alpha, eps = 10e-9, 2.0, 5.0
    errs = []
    for nsteps in (400, 800):
        pw = synthetic.pulse(nsteps, alpha, h)
        P = orc.Problem((1, 1, 1), h, np.full((1, 1, 1), eps), alpha)
        J = P.march([pw], nsteps)[:, 0, 0, 0, 0, 0]
        b = np.array([orc.incident((1, 1, 1), h, np.full((1, 1, 1), eps), pw, n * P.dt)[0, 0, 0, 0] for n in range(nsteps)])
        cm = 3.0 / (eps + 2.0) * b  # b already carries (eps-1) eps0 dE/dt
        errs.append(np.abs(J - cm).max() / np.abs(cm).max())
    # the deviation is first order in dt/sigma (the pulse width grows with nsteps)
    assert errs[0] < 0.1 and errs[1] < 0.55 * errs[0]


def test_time_step_refinement_converges(orc):
    N = (3, 3, 3)
    rng = np.random.default_rng(9)
    eps = rng.uniform(2, 4, size=N[::-1])
    h = 10e-9
    T_steps_cfl = 160  # fixed physical window of 160 dt_CFL
    traces = {}
    for alpha in (8, 4, 2, 1):
        n = T_steps_cfl // alpha
        pw = synthetic.pulse(n, alpha, h)
        P = orc.Problem(N, h, eps, alpha)
        J = P.march([pw], n)[:, 0]
        traces[alpha] = J[:: 8 // alpha][: T_steps_cfl // 8]  # samples every 8 dt_CFL
    e84 = np.abs(traces[8] - traces[4]).max()
    e42 = np.abs(traces[4] - traces[2]).max()
    e21 = np.abs(traces[2] - traces[1]).max()
    assert e84 > e42 > e21


@pytest.mark.parametrize("alpha,delta", [(2.0, 0.3), (8.0, 0.05), (4.0, 5.0)])
def test_delta_regularised_single_voxel_recursion(orc, alpha, delta):
    """Sec. II's delta-regularised MOT with the shift on the present-time matrix
    only (Z0 + delta I, no shift on the history lags): on one voxel the march is a
    scalar recursion (Z_0 + delta) J_n = b_n - sum_k Z_k J_{n-k}, with Z_k =
    eps T(k) - (eps - 1) g_k(0)_xx written out here from the temporal and kernel
    entries, independently of the oracle's product and solve."""
    h, eps, nsteps = 10e-9, 4.0, 60
    pw = synthetic.pulse(nsteps, alpha, h)
    P = orc.Problem((1, 1, 1), h, np.full((1, 1, 1), eps), alpha, delta=delta)
    J = P.march([pw], nsteps)[:, 0, 0, 0, 0, 0]
    rho = orc.rho_of_alpha(alpha)
    Z = []
    k = 0
    while k < 2 or orc.in_support(k, rho, (0, 0, 0)):
        Z.append(eps * orc.temporal(k) - (eps - 1) * orc.g_raw(k, rho, (0, 0, 0))[0])
        k += 1
    ref = np.zeros(nsteps)
    for n in range(nsteps):
        b = orc.incident((1, 1, 1), h, np.full((1, 1, 1), eps), pw, n * P.dt)[0, 0, 0, 0]
        hist = sum(Z[k] * ref[n - k] for k in range(1, min(n, len(Z) - 1) + 1))
        ref[n] = (b - hist) / (Z[0] + delta)
    assert np.abs(J - ref).max() <= 1e-12 * np.abs(ref).max()
    # the shift changes the answer (it is not silently dropped)
    J0 = orc.Problem((1, 1, 1), h, np.full((1, 1, 1), eps), alpha).march([pw], nsteps)[:, 0, 0, 0, 0, 0]
    assert np.abs(J - J0).max() > 1e-3 * np.abs(J0).max()
