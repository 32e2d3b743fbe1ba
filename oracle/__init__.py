"""Plain FP64 CPU oracle of the MOT-JVIE solver.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; the
product package never imports it and shares no code with it.

The numerics live in ``oracle.c`` (compiled to ``_oracle.so`` by
``oracle.build()``); this module marshals arrays and writes out the
marching-on-in-time recursion (Eq. 3) with a direct sparse LU solve of the
present-time system in place of TFQMR, so that the oracle's J_n is the exact
solution of Z0 J_n = b_n up to rounding.

Units and notation follow the paper (Sec. II): rho = c0 dt / h = alpha/sqrt(3)
(Eq. 9), ell = ceil(R_max / (c0 dt)) + p with p = 2 (Eq. 4), Z_k = eps_r T(k dt) I
- (eps_r - 1) G_k (Eq. 10 applied at every lag).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

C0 = 299792458.0
EPS0 = 8.8541878128e-12

_here = os.path.dirname(os.path.abspath(__file__))
_so = os.path.join(_here, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc, -O2, OpenMP, no fast-math)."""
    src = os.path.join(_here, "oracle.c")
    if force or not os.path.exists(_so) or os.path.getmtime(_so) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _so, src, "-lm"]
        subprocess.check_call(cmd)
    return _so


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_so)
        d, i, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        L.oracle_init.restype = None
        L.oracle_gauss_legendre.argtypes = [i, P, P]
        L.oracle_bspline2.argtypes = [d]
        L.oracle_bspline2.restype = d
        L.oracle_temporal.argtypes = [i]
        L.oracle_temporal.restype = d
        L.oracle_ang_tent.argtypes = [d, d, d]
        L.oracle_ang_tent.restype = d
        L.oracle_ang_quad.argtypes = [d, d, d]
        L.oracle_ang_quad.restype = d
        L.oracle_face.argtypes = [i, d, d, d, d]
        L.oracle_face.restype = d
        L.oracle_box.argtypes = [i, d, d, d, d]
        L.oracle_box.restype = d
        L.oracle_in_support.argtypes = [i, d, i, i, i]
        L.oracle_in_support.restype = i
        L.oracle_A_raw.argtypes = [i, d, i, i, i, P]
        L.oracle_g_raw.argtypes = [i, d, i, i, i, P]
        L.oracle_lag_table.argtypes = [i, d, i, i, i, P]
        L.oracle_green_apply.argtypes = [i, i, i, i, i, i, P, P, P]
        L.oracle_Zk_apply.argtypes = [i, i, i, i, P, i, i, i, P, P, P]
        L.oracle_incident.argtypes = [i, i, i, d, P, P, d, P]
        L.oracle_Zk_rows.argtypes = [i, i, i, i, P, i, i, i, P, P, i, P, P, P]
        L.oracle_init()
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- basics
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().oracle_gauss_legendre(n, _ptr(x), _ptr(w)) != 0:
        raise ValueError("n out of range")
    return x, w


def bspline2(u: float) -> float:
    """Quadratic B-spline B2 on [0, 3] (the p = 2 temporal basis, Sec. II)."""
    return lib().oracle_bspline2(float(u))


def temporal(k: int) -> float:
    """T(k dt) = B2(k + 1): 1/2, 1/2, 0, ..."""
    return lib().oracle_temporal(int(k))


def rho_of_alpha(alpha: float) -> float:
    """rho = c0 dt / h with dt = alpha dt_CFL, dt_CFL = h/(c0 sqrt 3) (Eq. 9)."""
    return alpha / math.sqrt(3.0)


def dt_cfl(h: float) -> float:
    return h / (C0 * math.sqrt(3.0))


def history_length(N, rho: float, p: int = 2) -> int:
    """ell = ceil(R_max / (c0 dt)) + p, R_max the corner-to-corner diagonal (Eq. 4)."""
    rmax = math.sqrt(sum(float(n) ** 2 for n in N))
    return int(math.ceil(rmax / rho - 1e-12)) + p


def lag_reach(k: int, rho: float) -> int:
    """Largest |d_i| with a nonzero lag-k entry: d - 1 < (k + 1) rho."""
    return int(math.ceil((k + 1) * rho + 1.0 - 1e-12)) - 1


def table_extent(k: int, rho: float, N):
    r = lag_reach(k, rho)
    return tuple(min(r, n - 1) for n in N)


# ---------------------------------------------------------------- quadrature pieces
def ang_tent(t, a, b):
    return lib().oracle_ang_tent(float(t), float(a), float(b))


def ang_quad(t, a, b):
    return lib().oracle_ang_quad(float(t), float(a), float(b))


def face(k, rho, c, a, b):
    return lib().oracle_face(int(k), float(rho), float(c), float(a), float(b))


def box(k, rho, dp, dq, dr):
    return lib().oracle_box(int(k), float(rho), float(dp), float(dq), float(dr))


def in_support(k, rho, d) -> bool:
    return bool(lib().oracle_in_support(int(k), float(rho), int(d[0]), int(d[1]), int(d[2])))


def A_raw(k, rho, d) -> np.ndarray:
    A = np.zeros(9)
    lib().oracle_A_raw(int(k), float(rho), int(d[0]), int(d[1]), int(d[2]), _ptr(A))
    return A.reshape(3, 3)


def g_raw(k, rho, d) -> np.ndarray:
    """(xx, yy, zz, xy, xz, yz) of g_k(d) computed directly at d."""
    g = np.zeros(6)
    lib().oracle_g_raw(int(k), float(rho), int(d[0]), int(d[1]), int(d[2]), _ptr(g))
    return g


def lag_table(k: int, rho: float, R) -> np.ndarray:
    """g_k(d) for |d_i| <= R_i; shape [6][2Rz+1][2Ry+1][2Rx+1] (x fastest)."""
    Rx, Ry, Rz = (int(v) for v in R)
    g = np.zeros((6, 2 * Rz + 1, 2 * Ry + 1, 2 * Rx + 1))
    lib().oracle_lag_table(int(k), float(rho), Rx, Ry, Rz, _ptr(g))
    return g


def lag_tables(N, rho: float, ell: int | None = None):
    if ell is None:
        ell = history_length(N, rho)
    out = []
    for k in range(ell + 1):
        R = table_extent(k, rho, N)
        out.append((R, lag_table(k, rho, R)))
    return out


# ---------------------------------------------------------------- products
def green_apply(N, R, g, x) -> np.ndarray:
    """(G x)_p(m) = sum_q sum_d g(d)_pq x_q(m - d) by direct summation."""
    Nx, Ny, Nz = N
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3, Nz, Ny, Nx)
    y = np.zeros_like(x)
    lib().oracle_green_apply(Nx, Ny, Nz, R[0], R[1], R[2], _ptr(np.ascontiguousarray(g)), _ptr(x), _ptr(y))
    return y


def Zk_apply(k, N, eps, R, g, x) -> np.ndarray:
    """Z_k x = eps_r T(k dt) x - (eps_r - 1) G_k x (Eq. 10, Eq. 12)."""
    Nx, Ny, Nz = N
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3, Nz, Ny, Nx)
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(Nz, Ny, Nx)
    y = np.zeros_like(x)
    lib().oracle_Zk_apply(int(k), Nx, Ny, Nz, _ptr(eps), R[0], R[1], R[2],
                          _ptr(np.ascontiguousarray(g)), _ptr(x), _ptr(y))
    return y


def Zk_rows(k, N, eps, R, g, x, rows_p, rows_m) -> np.ndarray:
    """Selected rows (p_i, m_i) of Z_k x, same definition as Zk_apply."""
    Nx, Ny, Nz = N
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3, Nz, Ny, Nx)
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(Nz, Ny, Nx)
    rp = np.ascontiguousarray(rows_p, dtype=np.int32)
    rm = np.ascontiguousarray(rows_m, dtype=np.int64)
    out = np.zeros(len(rp))
    lib().oracle_Zk_rows(int(k), Nx, Ny, Nz, _ptr(eps), R[0], R[1], R[2], _ptr(np.ascontiguousarray(g)), _ptr(x),
                         len(rp), _ptr(rp), _ptr(rm), _ptr(out))
    return out


def planewave_array(pw) -> np.ndarray:
    """(E0, sigma, t0, f0, khat[3], pol[3]) as 10 doubles."""
    if isinstance(pw, dict):
        v = [pw["E0"], pw["sigma"], pw["t0"], pw["f0"], *pw["khat"], *pw["pol"]]
    else:
        v = list(pw)
    return np.asarray(v, dtype=np.float64)


def incident(N, h, eps, pw, t) -> np.ndarray:
    """(eps_r - 1) eps0 <dE^i/dt>_voxel at time t (Eq. 7-8), 2x2x2 Gauss average."""
    Nx, Ny, Nz = N
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(Nz, Ny, Nx)
    b = np.zeros((3, Nz, Ny, Nx))
    lib().oracle_incident(Nx, Ny, Nz, float(h), _ptr(eps), _ptr(planewave_array(pw)), float(t), _ptr(b))
    return b


# ---------------------------------------------------------------- dense / sparse assembly
def assemble_Zk(k, N, eps, R, g, dense: bool = False):
    """Z_k as an explicit (3n x 3n) matrix; row (p, m), column (q, m')."""
    import scipy.sparse as sp

    Nx, Ny, Nz = N
    n = Nx * Ny * Nz
    eps = np.asarray(eps, dtype=np.float64).reshape(-1)
    Rx, Ry, Rz = R
    mz, my, mx = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    mz, my, mx = mz.ravel(), my.ravel(), mx.ravel()
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    rows, cols, vals = [], [], []
    for dz in range(-Rz, Rz + 1):
        for dy in range(-Ry, Ry + 1):
            for dx in range(-Rx, Rx + 1):
                gd = g[:, dz + Rz, dy + Ry, dx + Rx]
                if not np.any(gd):
                    continue
                sx, sy, sz = mx - dx, my - dy, mz - dz
                ok = (sx >= 0) & (sx < Nx) & (sy >= 0) & (sy < Ny) & (sz >= 0) & (sz < Nz)
                m = np.nonzero(ok)[0]
                s = (sz[ok] * Ny + sy[ok]) * Nx + sx[ok]
                for p in range(3):
                    for q in range(3):
                        v = gd[comp[(p, q)]]
                        if v == 0.0:
                            continue
                        rows.append(p * n + m)
                        cols.append(q * n + s)
                        vals.append(-(eps[m] - 1.0) * v)
    Tk = temporal(k)
    if Tk != 0.0:
        for p in range(3):
            rows.append(p * n + np.arange(n))
            cols.append(p * n + np.arange(n))
            vals.append(eps * Tk)
    if rows:
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    else:
        rows = cols = np.zeros(0, dtype=np.int64)
        vals = np.zeros(0)
    Z = sp.coo_matrix((vals, (rows, cols)), shape=(3 * n, 3 * n)).tocsc()
    return Z.toarray() if dense else Z


# ---------------------------------------------------------------- the march (Eq. 3)
class Problem:
    """Geometry, permittivity, time step and the lag tables of one MOT-JVIE problem.

    delta: the diagonal shift of the delta-regularised MOT (Sec. II, Z^delta_n =
    Z_n + delta_n I), applied to the present-time matrix only (delta_0 = delta,
    delta_n = 0 for n >= 1); the paper uses 0."""

    def __init__(self, N, h, eps, alpha, tables=None, delta=0.0):
        self.N = tuple(int(v) for v in N)
        self.h = float(h)
        self.eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(self.N[2], self.N[1], self.N[0])
        self.alpha = float(alpha)
        self.rho = rho_of_alpha(alpha)
        self.dt = alpha * dt_cfl(h)
        self.ell = history_length(self.N, self.rho)
        self.tables = tables if tables is not None else lag_tables(self.N, self.rho, self.ell)
        self.delta = float(delta)
        self._lu = None

    def apply(self, k, x):
        R, g = self.tables[k]
        y = Zk_apply(k, self.N, self.eps, R, g, x)
        if k == 0 and self.delta != 0.0:
            y = y + self.delta * np.asarray(x, dtype=np.float64).reshape(y.shape)
        return y

    def solve_Z0(self, b):
        """J = Z0^-1 b exactly (up to rounding): dense LU with partial pivoting
        (LAPACK) while 3n <= 12288 unknowns, sparse LU (SuperLU) above that."""
        import scipy.linalg as sla
        import scipy.sparse.linalg as spla

        rhs = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        if self._lu is None:
            R, g = self.tables[0]
            Z = assemble_Zk(0, self.N, self.eps, R, g)
            if self.delta != 0.0:
                import scipy.sparse as sp

                Z = (Z + self.delta * sp.identity(Z.shape[0], format="csc")).tocsc()
            if Z.shape[0] <= 12288:
                self._lu = ("dense", sla.lu_factor(Z.toarray(), check_finite=False))
            else:
                self._lu = ("sparse", spla.splu(Z))
        kind, f = self._lu
        x = sla.lu_solve(f, rhs, check_finite=False) if kind == "dense" else f.solve(rhs)
        return x.reshape(b.shape)

    def rhs(self, n, pw, Jhist):
        """b_n = E^i_n - sum_{k=1..ell} Z_k J_{n-k}  (Eq. 3, J_j = 0 for j < 0)."""
        b = incident(self.N, self.h, self.eps, pw, n * self.dt)
        for k in range(1, self.ell + 1):
            if n - k < 0:
                break
            b -= self.apply(k, Jhist[n - k])
        return b

    def march(self, planewaves, nsteps):
        """J[n][rhs][3][Nz][Ny][Nx] for n = 0..nsteps-1, Z0 J_n = b_n solved exactly."""
        Nx, Ny, Nz = self.N
        out = np.zeros((nsteps, len(planewaves), 3, Nz, Ny, Nx))
        for r, pw in enumerate(planewaves):
            J = out[:, r]
            for n in range(nsteps):
                J[n] = self.solve_Z0(self.rhs(n, pw, J))
        return out
