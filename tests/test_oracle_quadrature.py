"""Pins of the oracle's quadrature building blocks against independent routines.

Each check compares an oracle piece with something it does not share code with:
numpy's Gauss-Legendre rule, brute-force angular sampling, and scipy's adaptive
QUADPACK cubature of the defining 2-D / 3-D integrals (Galerkin weight of the
piecewise-constant voxel basis, Sec. II; kernel B2(k+1-R/rho)/(4 pi R)).
"""
import math

import numpy as np
import pytest


def test_gauss_legendre_matches_numpy(orc):
    for n in (1, 2, 5, 20, 40, 64):
        x, w = orc.gauss_legendre(n)
        X, W = np.polynomial.legendre.leggauss(n)
        o = np.argsort(x)
        assert np.allclose(x[o], X, atol=2e-16 * n, rtol=0)
        assert np.allclose(w[o], W, atol=5e-15, rtol=0)


def test_bspline2_closed_forms(orc):
    # T(0) = T(dt) = 1/2, T(k dt) = 0 for k >= 2 (quadratic spline, p = 2, Sec. II)
    assert orc.temporal(0) == 0.5 and orc.temporal(1) == 0.5
    assert all(orc.temporal(k) == 0.0 for k in range(2, 6))
    # partition of unity of the shifted splines and unit integral
    for u in np.linspace(-0.3, 0.99, 17):
        assert abs(sum(orc.bspline2(u + j) for j in range(-3, 6)) - 1.0) < 1e-15
    x, w = np.polynomial.legendre.leggauss(8)
    tot = sum(0.5 * wi * orc.bspline2(a + 0.5 * (xi + 1)) for a in (0, 1, 2) for xi, wi in zip(x, w))
    assert abs(tot - 1.0) < 1e-15


def _brute_angle(t, a, b, n=1_000_000):
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    lam = lambda x: np.maximum(1 - np.abs(x), 0)
    dl = lambda x: np.where((x > -1) & (x < 0), 1.0, np.where((x > 0) & (x < 1), -1.0, 0.0))
    u, v = t * np.cos(th) - a, t * np.sin(th) - b
    return (lam(u) * lam(v)).mean() * 2 * np.pi, (dl(u) * dl(v)).mean() * 2 * np.pi


def test_angular_integrals_brute_force(orc):
    rng = np.random.default_rng(7)
    for _ in range(8):
        t = rng.uniform(0.05, 4.5)
        a, b = (int(v) for v in rng.integers(-3, 4, size=2))
        bt, bq = _brute_angle(t, a, b)
        assert abs(orc.ang_tent(t, a, b) - bt) < 1e-9
        assert abs(orc.ang_quad(t, a, b) - bq) < 2e-5  # midpoint rule on a step function


def _K(orc, k, rho, R):
    return orc.bspline2(k + 1 - R / rho) / (4 * math.pi * R)


def _face_bf(orc, k, rho, c, a, b):
    from scipy import integrate

    tot = 0.0
    for i in (a - 1, a):
        for j in (b - 1, b):
            f = lambda v, u: _K(orc, k, rho, math.sqrt(c * c + u * u + v * v)) * max(1 - abs(u - a), 0) * max(1 - abs(v - b), 0)
            tot += integrate.dblquad(f, i, i + 1, j, j + 1, epsabs=1e-13, epsrel=1e-12)[0]
    return tot


@pytest.mark.parametrize("k,c,a,b", [(0, 1, 0, 0), (0, 0, 1, 1), (0, 2, 1, 0), (1, 1, 2, 1), (2, 3, 2, 1), (0, 0, 0, 0)])
def test_face_integral_vs_quadpack(orc, k, c, a, b):
    rho = 4 / math.sqrt(3)
    assert abs(orc.face(k, rho, c, a, b) - _face_bf(orc, k, rho, c, a, b)) < 1e-12


def _box_bf(orc, k, rho, dp, dq, dr):
    from scipy import integrate

    dl = lambda x: 1.0 if -1 < x < 0 else (-1.0 if 0 < x < 1 else 0.0)
    tot = 0.0
    for i in (dp - 1, dp):
        for j in (dq - 1, dq):
            for l in (dr - 1, dr):
                sg = dl(i + 0.5 - dp) * dl(j + 0.5 - dq)
                f = lambda z, y, x: _K(orc, k, rho, math.sqrt(x * x + y * y + z * z)) * max(1 - abs(z - dr), 0)
                tot += sg * integrate.tplquad(f, i, i + 1, j, j + 1, l, l + 1, epsabs=1e-12, epsrel=1e-10)[0]
    return tot


@pytest.mark.parametrize("k,dp,dq,dr", [(0, 1, 1, 0), (2, 2, 3, 1), (1, 1, 1, 0)])
def test_box_integral_vs_quadpack(orc, k, dp, dq, dr):
    rho = 4 / math.sqrt(3)
    assert abs(orc.box(k, rho, dp, dq, dr) - _box_bf(orc, k, rho, dp, dq, dr)) < 2e-12
