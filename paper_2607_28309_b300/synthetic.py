"""Seeded synthetic inputs shaped like the paper's workloads (no solver arithmetic).

Stands in for the paper's dielectric cubes (Sec. III-B, Sec. V-A) and its 8x8
nanopillar metasurface (Sec. V-B); no dataset is involved.  Used by the tests,
bench.py and the smoke check for both the CUDA path and the oracle.

Recipe
------
- voxel size h = 10 nm, c0 = 299,792,458 m/s, dt_CFL = h/(c0 sqrt 3);
- random numbers: SplitMix64 seeded per workload, u = (x >> 11) * 2^-53,
  drawn per permittivity block with blocks enumerated x fastest;
- pulse of Eq. 7-8 over a window T = nsteps * alpha * dt_CFL: sigma = T/20,
  t0 = 5 sigma, sigma_f = 1/(2 pi sigma), f0 = 2.5 sigma_f, f_max = f0 + 3 sigma_f;
- nanopillars: cylinders of 24-voxel diameter (voxel centre within 12 voxels of
  the axis) at 32-voxel pitch, axes at 16 + 32 i, occupying z in [8, 72): the
  lower 43 layers eps_r = 3.5, the upper 21 eps_r = 6.0, background 1;
- the paper's bilayer metasurface (Sec. V-B): 240 x 240 x 90 voxels of 10 nm, a
  20-voxel quartz substrate (eps_r 2.1) at the bottom, 8 x 8 pillars of a 40-voxel
  a-Si base (12.0) under a 20-voxel GST cap, 10 voxels of air on top; pillars are
  16 x 10-voxel rectangles rotated by 0, 45, 90, 135 degrees in each 2 x 2
  supercell of 56-voxel period, centred 14 voxels off the supercell centre; caps of
  the 0 / 90 degree pillars amorphous GST (16.0), of the 45 / 135 degree pillars
  crystalline GST (25.0); x-polarised pulse along -z with sigma 11.06 fs,
  t0 68.85 fs, f0 312 THz, dt = 16 dt_CFL.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
H_DEFAULT = 10e-9
_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from SplitMix64 (Steele, Lea, Flood 2014)."""
    out = np.empty(n)
    x = seed & _MASK
    for i in range(n):
        x = (x + 0x9E3779B97F4A7C15) & _MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        z ^= z >> 31
        out[i] = (z >> 11) * 2.0**-53
    return out


def block_eps(N, block: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """eps_r uniform in [lo, hi] per block^3 sub-block; array [Nz][Ny][Nx]."""
    Nx, Ny, Nz = N
    bx, by, bz = (-(-Nx // block), -(-Ny // block), -(-Nz // block))
    u = splitmix64(seed, bx * by * bz).reshape(bz, by, bx)
    vals = lo + (hi - lo) * u
    iz = np.arange(Nz) // block
    iy = np.arange(Ny) // block
    ix = np.arange(Nx) // block
    return np.ascontiguousarray(vals[iz[:, None, None], iy[None, :, None], ix[None, None, :]])


def pillar_eps(nx: int, ny: int, Nz: int = 80, pitch: int = 32, diameter: int = 24, z0: int = 8,
               base: int = 43, cap: int = 21, eps_base: float = 3.5, eps_cap: float = 6.0,
               layer_eps=None) -> np.ndarray:
    """nx x ny pillar array on a (pitch*nx) x (pitch*ny) x Nz grid.
    layer_eps, if given, is a list of (eps_base, eps_cap) per pillar (x fastest)."""
    Nx, Ny = pitch * nx, pitch * ny
    eps = np.ones((Nz, Ny, Nx))
    r = diameter / 2.0
    yy, xx = np.meshgrid(np.arange(pitch) + 0.5, np.arange(pitch) + 0.5, indexing="ij")
    disk = (xx - pitch / 2.0) ** 2 + (yy - pitch / 2.0) ** 2 <= r * r
    for j in range(ny):
        for i in range(nx):
            eb, ec = (eps_base, eps_cap) if layer_eps is None else layer_eps[j * nx + i]
            sl = (slice(j * pitch, (j + 1) * pitch), slice(i * pitch, (i + 1) * pitch))
            for z in range(z0, z0 + base):
                eps[z][sl][disk] = eb
            for z in range(z0 + base, z0 + base + cap):
                eps[z][sl][disk] = ec
    return eps


def metasurface_eps(n_super: int = 4, period: int = 56, margin: int = 8, offset: int = 14, long_edge: int = 16,
                    short_edge: int = 10, z_sub: int = 20, z_base: int = 40, z_cap: int = 20, z_air: int = 10,
                    eps_quartz: float = 2.10, eps_asi: float = 12.0, eps_gst_a: float = 16.0,
                    eps_gst_c: float = 25.0) -> np.ndarray:
    """The bilayer GST/a-Si nanopillar metasurface of Sec. V-B on a voxel grid
    (array [Nz][Ny][Nx]).  In each 2 x 2 supercell the pillar at (-, -) is rotated
    by 0 degrees, (+, -) by 45, (-, +) by 90 and (+, +) by 135 (x fastest); a voxel
    belongs to a pillar when its centre lies in the rotated rectangle."""
    N = 2 * margin + n_super * period
    Nz = z_sub + z_base + z_cap + z_air
    eps = np.ones((Nz, N, N))
    eps[:z_sub] = eps_quartz
    yy, xx = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5, indexing="ij")
    base = np.zeros((N, N), dtype=bool)
    cap = np.ones((N, N))
    angles = ((0, 45), (90, 135))  # [row (y)][column (x)]
    for sj in range(n_super):
        for si in range(n_super):
            cx0 = margin + si * period + period / 2.0
            cy0 = margin + sj * period + period / 2.0
            for j in range(2):
                for i in range(2):
                    th = math.radians(angles[j][i])
                    cx = cx0 + (2 * i - 1) * offset
                    cy = cy0 + (2 * j - 1) * offset
                    dx, dy = xx - cx, yy - cy
                    u = dx * math.cos(th) + dy * math.sin(th)
                    v = -dx * math.sin(th) + dy * math.cos(th)
                    inside = (np.abs(u) <= long_edge / 2.0) & (np.abs(v) <= short_edge / 2.0)
                    base |= inside
                    cap[inside] = eps_gst_a if angles[j][i] in (0, 90) else eps_gst_c
    for z in range(z_sub, z_sub + z_base):
        eps[z][base] = eps_asi
    for z in range(z_sub + z_base, z_sub + z_base + z_cap):
        eps[z][base] = cap[base]
    return eps


def dt_cfl(h: float = H_DEFAULT) -> float:
    return h / (C0 * math.sqrt(3.0))


def pulse(nsteps: int, alpha: float, h: float = H_DEFAULT, khat=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0), E0=1.0):
    """Gaussian-modulated plane wave (Eq. 7-8) fitted to the window nsteps*alpha*dt_CFL."""
    T = nsteps * alpha * dt_cfl(h)
    sigma = T / 20.0
    sf = 1.0 / (2.0 * math.pi * sigma)
    return {"E0": E0, "sigma": sigma, "t0": 5.0 * sigma, "f0": 2.5 * sf, "khat": tuple(khat), "pol": tuple(pol)}


def pulse_fmax(pw) -> float:
    return pw["f0"] + 3.0 / (2.0 * math.pi * pw["sigma"])


def oblique_set(nsteps: int, alpha: float, h: float = H_DEFAULT, angles_deg=(0, 10, 20, 30, 40, 50, 60, 70)):
    """8 incidence angles x 2 polarisations: khat = (sin t, 0, cos t), TE pol = y,
    TM pol = (cos t, 0, -sin t)."""
    out = []
    for a in angles_deg:
        t = math.radians(a)
        k = (math.sin(t), 0.0, math.cos(t))
        out.append(pulse(nsteps, alpha, h, khat=k, pol=(0.0, 1.0, 0.0)))
        out.append(pulse(nsteps, alpha, h, khat=k, pol=(math.cos(t), 0.0, -math.sin(t))))
    return out


# ---------------------------------------------------------------- named workloads
def cube16(seed: int = 1):
    """16^3 cube, eps_r U[2,4] per 4^3 block, x-pol along +z, alpha 4, 100 steps, FP64."""
    N = (16, 16, 16)
    return {"name": "cube16_a4", "N": N, "h": H_DEFAULT, "eps": block_eps(N, 4, 2.0, 4.0, seed), "alpha": 4.0,
            "steps": 100, "exc": [pulse(100, 4.0)]}


def cube64(alpha: float = 8.0, seed: int = 2):
    """64^3 cube, eps_r U[1.5,6] per 8^3 block; window 400 dt_CFL -> 400/alpha steps."""
    N = (64, 64, 64)
    steps = int(round(400 / alpha))
    return {"name": f"cube64_a{int(alpha)}", "N": N, "h": H_DEFAULT, "eps": block_eps(N, 8, 1.5, 6.0, seed),
            "alpha": float(alpha), "steps": steps, "exc": [pulse(steps, alpha)]}


def pillars8x8():
    """8x8 pillars on 256x256x80, normal incidence along -z, x-pol, alpha 8, 200 steps."""
    eps = pillar_eps(8, 8)
    return {"name": "pillars8x8_a8", "N": (256, 256, 80), "h": H_DEFAULT, "eps": eps, "alpha": 8.0, "steps": 200,
            "exc": [pulse(200, 8.0, khat=(0.0, 0.0, -1.0))]}


def pillars2x2():
    """2x2 pillars on 64x64x80 (the pillar array's layers and pitch), normal incidence
    along -z, x-pol, alpha 8, 200 steps: a history grid of 128x128x160 whose ring
    and Lambda_k tables exceed L2 while the whole run holds a few GB."""
    eps = pillar_eps(2, 2)
    return {"name": "pillars2x2_a8", "N": (64, 64, 80), "h": H_DEFAULT, "eps": eps, "alpha": 8.0, "steps": 200,
            "exc": [pulse(200, 8.0, khat=(0.0, 0.0, -1.0))]}


def metasurface8x8(nsteps: int = 1250):
    """The paper's 8 x 8 bilayer metasurface (Sec. V-B): 240 x 240 x 90 voxels,
    dt = 16 dt_CFL, its own pulse (sigma 11.06 fs, t0 68.85 fs, f0 312 THz, -z, x-pol);
    1250 steps span the paper's 385.17 fs window."""
    pw = {"E0": 1.0, "sigma": 11.06e-15, "t0": 68.85e-15, "f0": 312e12, "khat": (0.0, 0.0, -1.0),
          "pol": (1.0, 0.0, 0.0)}
    return {"name": "metasurface8x8_a16", "N": (240, 240, 90), "h": H_DEFAULT, "eps": metasurface_eps(),
            "alpha": 16.0, "steps": int(nsteps), "exc": [pw]}


def cube64_batch16(seed: int = 4):
    """64^3 cube, eps_r U[2,4] per 4^3 block, 16 oblique plane waves, alpha 8, 200 steps."""
    N = (64, 64, 64)
    return {"name": "cube64_b16_a8", "N": N, "h": H_DEFAULT, "eps": block_eps(N, 4, 2.0, 4.0, seed), "alpha": 8.0,
            "steps": 200, "exc": oblique_set(200, 8.0)}


WORKLOADS = {
    "cube16_a4": lambda: cube16(),
    "cube64_a4": lambda: cube64(4.0),
    "cube64_a8": lambda: cube64(8.0),
    "cube64_a16": lambda: cube64(16.0),
    "cube64_b16": lambda: cube64_batch16(),
    "pillars2x2": lambda: pillars2x2(),
    "pillars8x8": lambda: pillars8x8(),
    "metasurface8x8": lambda: metasurface8x8(),
}


def workload(name: str):
    """The named synthetic workload (see WORKLOADS)."""
    if name not in WORKLOADS:
        raise ValueError(f"unknown workload {name}; one of {sorted(WORKLOADS)}")
    return WORKLOADS[name]()
