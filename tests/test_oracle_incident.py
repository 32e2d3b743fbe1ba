"""Pins of the oracle's incident-field right-hand side (Eq. 7-8) and of its
row-sampled product (the checker of every full-size GPU test).

The incident pin never differentiates Eq. 7 by hand: it evaluates the field of
Eq. 7 itself at the eight 2x2x2 Gauss-Legendre points of each voxel (numpy's
own nodes, mapped to the voxel), differentiates in t by a Richardson-
extrapolated central difference, and finds the reference corner by brute force
over the eight corners of the grid box.  A dropped 1/(sigma sqrt(2 pi)), a sign
flip of the time derivative, a reference corner taken on the wrong side for a
negative k-hat component, or the field sampled at the voxel centre instead of
averaged each move the result far outside the tolerance.

The row-sampled product is compared with the full matrix-free product for
lag 0 and later lags, with real lag tables and with a random table that has no
d -> -d symmetry, on rows that include every grid corner and edge.
"""
import math

import numpy as np
import pytest

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def _field(t, r, pw, rref):
    """E^i of Eq. 7 (a vector, its polarisation times the scalar pulse), Eq. 8 for tau."""
    E0, sig, t0, f0 = pw["E0"], pw["sigma"], pw["t0"], pw["f0"]
    kh = np.asarray(pw["khat"])
    tau = t - t0 - ((r - rref) @ kh) / C0
    s = E0 / (sig * math.sqrt(2.0 * math.pi)) * np.exp(-tau ** 2 / (2.0 * sig ** 2)) * np.cos(2.0 * math.pi * f0 * tau)
    return s[..., None] * np.asarray(pw["pol"])


def _dfield_dt(t, r, pw, rref, dt):
    """Richardson-extrapolated central difference of the field in t (error O(dt^4))."""
    d1 = (_field(t + dt, r, pw, rref) - _field(t - dt, r, pw, rref)) / (2 * dt)
    d2 = (_field(t + 2 * dt, r, pw, rref) - _field(t - 2 * dt, r, pw, rref)) / (4 * dt)
    return (4.0 * d1 - d2) / 3.0


def _reference_corner(N, h, khat):
    """The corner of the grid box [0, N h] with the smallest khat . r (by brute force)."""
    best = None
    for cx in (0, N[0]):
        for cy in (0, N[1]):
            for cz in (0, N[2]):
                c = np.array([cx, cy, cz], dtype=float) * h
                if best is None or c @ khat < best @ khat - 1e-30:
                    best = c
    return best


def _incident_by_difference(N, h, eps, pw, t):
    Nx, Ny, Nz = N
    xg, wg = np.polynomial.legendre.leggauss(2)
    u = 0.5 * (xg + 1.0)          # nodes on [0, 1]
    w = 0.5 * wg                  # weights summing to 1 per axis
    rref = _reference_corner(N, h, np.asarray(pw["khat"], dtype=float))
    out = np.zeros((3, Nz, Ny, Nx))
    mz, my, mx = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    dt = pw["sigma"] * 1e-3
    for i in range(2):
        for j in range(2):
            for l in range(2):
                r = np.stack([(mx + u[i]) * h, (my + u[j]) * h, (mz + u[l]) * h], axis=-1)
                dE = _dfield_dt(t, r, pw, rref, dt)          # [Nz, Ny, Nx, 3]
                out += w[i] * w[j] * w[l] * np.moveaxis(dE, -1, 0)
    return (eps - 1.0)[None] * EPS0 * out


def _pulse(khat, pol, h):
    # a pulse short enough that the field changes by O(1) across a voxel:
    # the voxel average then differs from the centre value by ~1e-2
    sigma = 1.2 * h / C0
    return {"E0": 1.7, "sigma": sigma, "t0": 4.0 * sigma, "f0": 0.35 / sigma,
            "khat": list(khat), "pol": list(pol)}


_CASES = [
    ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)),
    ((0.0, 0.0, -1.0), (0.0, 1.0, 0.0)),
    # oblique with two negative components: the reference corner is (N_x h, 0, N_z h)
    ((-0.48, 0.64, -0.6), (0.8, 0.6, 0.0)),
]


@pytest.mark.parametrize("khat,pol", _CASES)
def test_incident_matches_difference_of_eq7(orc, khat, pol):
    N = (5, 4, 6)
    h = 10e-9
    rng = np.random.default_rng(7)
    eps = rng.uniform(1.5, 6.0, size=N[::-1])
    pw = _pulse(khat, pol, h)
    assert abs(np.dot(khat, pol)) < 1e-14 and abs(np.linalg.norm(khat) - 1) < 1e-14
    for t in (pw["t0"] - 0.7 * pw["sigma"], pw["t0"] + 2.3 * h / C0, pw["t0"] + 1.9 * pw["sigma"]):
        want = _incident_by_difference(N, h, eps, pw, t)
        got = orc.incident(N, h, eps, pw, t)
        scale = np.abs(want).max()
        assert scale > 0
        assert np.abs(got - want).max() <= 2e-7 * scale


def test_incident_average_differs_from_centre_value(orc):
    """The case above is sensitive to the quadrature: the voxel-centre value is
    far outside the tolerance that the 2x2x2 average meets."""
    N = (5, 4, 6)
    h = 10e-9
    eps = np.full(N[::-1], 3.0)
    pw = _pulse((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), h)
    t = pw["t0"] + 2.3 * h / C0
    rref = _reference_corner(N, h, np.asarray(pw["khat"]))
    mz, my, mx = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    r = np.stack([(mx + 0.5) * h, (my + 0.5) * h, (mz + 0.5) * h], axis=-1)
    centre = 2.0 * EPS0 * np.moveaxis(_dfield_dt(t, r, pw, rref, pw["sigma"] * 1e-3), -1, 0)
    got = orc.incident(N, h, eps, pw, t)
    scale = np.abs(got).max()
    assert np.abs(got - centre).max() > 1e-3 * scale


def test_incident_zero_contrast_and_reference_corner(orc):
    """eps_r = 1 voxels carry no incident term; with khat = -z the pulse enters
    through the top face at t0 (tau = t - t0 there)."""
    N = (3, 3, 4)
    h = 10e-9
    eps = np.ones(N[::-1])
    eps[2, 1, 1] = 4.0
    pw = _pulse((0.0, 0.0, -1.0), (1.0, 0.0, 0.0), h)
    b = orc.incident(N, h, eps, pw, pw["t0"])
    mask = np.ones(N[::-1], dtype=bool)
    mask[2, 1, 1] = False
    assert np.all(b[:, mask] == 0.0)
    assert b[1, 2, 1, 1] == 0.0 and b[2, 2, 1, 1] == 0.0 and b[0, 2, 1, 1] != 0.0


@pytest.mark.parametrize("k", [0, 1, 3])
def test_Zk_rows_equal_full_product(orc, k):
    rng = np.random.default_rng(100 + k)
    N = (7, 5, 6)
    Nx, Ny, Nz = N
    n = Nx * Ny * Nz
    eps = rng.uniform(1.0, 5.0, size=N[::-1])
    rho = orc.rho_of_alpha(4)
    R = orc.table_extent(k, rho, N)
    g = orc.lag_table(k, rho, R)
    x = rng.standard_normal((3,) + N[::-1])
    # every corner and edge midpoint of the grid, plus random interior rows, all three components
    pts = set()
    for cx in (0, Nx // 2, Nx - 1):
        for cy in (0, Ny // 2, Ny - 1):
            for cz in (0, Nz // 2, Nz - 1):
                pts.add((cz * Ny + cy) * Nx + cx)
    pts.update(int(v) for v in rng.integers(0, n, size=20))
    pts = sorted(pts)
    rows_p = np.repeat(np.arange(3), len(pts))
    rows_m = np.tile(np.asarray(pts, dtype=np.int64), 3)
    for table in (g, rng.standard_normal(g.shape)):
        full = orc.Zk_apply(k, N, eps, R, table, x).reshape(3, n)
        got = orc.Zk_rows(k, N, eps, R, table, x, rows_p, rows_m)
        want = full[rows_p, rows_m]
        assert np.abs(got - want).max() <= 1e-13 * (1.0 + np.abs(want).max())
