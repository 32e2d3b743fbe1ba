// direct.cuh -- the present-time product Z0 x by direct summation over the
// lag-0 table's support, on the GPU: the paper's "direct" MVP (Sec. IV: Z0
// applied through its nonzero entries rather than by FFT; Sec. V-A compares
// the two), for the alpha crossover against the FFT product.
//
//   (Z0 x)_p(m) = eps(m) T(0) x_p(m) - (eps(m) - 1) sum_d sum_q g0(d)_pq x_q(m - d)   (Eq. 10, 12)
//
// (+ delta x_p(m) for the regularised Z0 + delta I, Sec. II; delta = 0 in the paper)
//
// with x = 0 outside the grid.  The offsets d with a nonzero entry (the causal
// support of lag 0, |d_i| <= R_i) come as a list with their six table values
// (xx yy zz xy xz yz), signs of the mixed entries already applied.  One CTA per
// output tile of blockDim voxels of one right-hand side: the input tile with a
// halo of R on each side (three components) is staged in shared memory, each
// thread sums its voxel over the offset list (the same offset in every thread
// at a time, so the list is read by broadcast).
#pragma once

#include "common.cuh"

namespace mot {

template <typename T>
__global__ void __launch_bounds__(512) k_z0_direct(const T *__restrict__ x, T *__restrict__ y,
                                                   const T *__restrict__ eps, const int4 *__restrict__ dlist,
                                                   const T *__restrict__ gval, int nd, int Rx, int Ry, int Rz,
                                                   int Nx, int Ny, int Nz, T dl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    const int TX = blockDim.x, TY = blockDim.y, TZ = blockDim.z;
    const int SX = TX + 2 * Rx, SY = TY + 2 * Ry, SZ = TZ + 2 * Rz;
    const long nv = (long)Nx * Ny * Nz;
    const int tilesx = (Nx + TX - 1) / TX, tilesy = (Ny + TY - 1) / TY;
    const int bx = blockIdx.x % tilesx, by = (blockIdx.x / tilesx) % tilesy, bz = blockIdx.x / (tilesx * tilesy);
    const int b = blockIdx.y;  // right-hand side
    const int x0 = bx * TX - Rx, y0 = by * TY - Ry, z0 = bz * TZ - Rz;
    const T *xb = x + (long)b * 3 * nv;
    const int nthr = TX * TY * TZ, tid = (threadIdx.z * TY + threadIdx.y) * TX + threadIdx.x;
    const int sn = SX * SY * SZ;
    for (int i = tid; i < 3 * sn; i += nthr) {
        const int q = i / sn, rem = i - q * sn;
        const int sx = rem % SX, sy = (rem / SX) % SY, sz = rem / (SX * SY);
        const int gx = x0 + sx, gy = y0 + sy, gz = z0 + sz;
        T v = T(0);
        if (gx >= 0 && gx < Nx && gy >= 0 && gy < Ny && gz >= 0 && gz < Nz)
            v = xb[(long)q * nv + ((long)gz * Ny + gy) * Nx + gx];
        tile[i] = v;
    }
    __syncthreads();
    const int ox = bx * TX + threadIdx.x, oy = by * TY + threadIdx.y, oz = bz * TZ + threadIdx.z;
    if (ox >= Nx || oy >= Ny || oz >= Nz) return;
    // the output voxel's place in the tile (d = 0)
    const int c0 = ((threadIdx.z + Rz) * SY + (threadIdx.y + Ry)) * SX + (threadIdx.x + Rx);
    T g0 = T(0), g1 = T(0), g2 = T(0);
    for (int i = 0; i < nd; ++i) {
        const int4 d = dlist[i];  // d.w = tile offset of x(m - d) relative to c0
        const T *gv = gval + 6 * (long)i;
        const int c = c0 - d.w;
        const T u0 = tile[c], u1 = tile[sn + c], u2 = tile[2 * sn + c];
        const T gxx = gv[0], gyy = gv[1], gzz = gv[2], gxy = gv[3], gxz = gv[4], gyz = gv[5];
        g0 += gxx * u0 + gxy * u1 + gxz * u2;
        g1 += gxy * u0 + gyy * u1 + gyz * u2;
        g2 += gxz * u0 + gyz * u1 + gzz * u2;
    }
    const long m = ((long)oz * Ny + oy) * Nx + ox;
    const T e = eps[m];
    T *yb = y + (long)b * 3 * nv;
    const T dg = e * T(0.5) + dl;  // the diagonal D (+ delta of Z0 + delta I)
    yb[m] = dg * tile[c0] - (e - T(1)) * g0;
    yb[nv + m] = dg * tile[sn + c0] - (e - T(1)) * g1;
    yb[2 * nv + m] = dg * tile[2 * sn + c0] - (e - T(1)) * g2;
}

// the same sum without staging, for reaches whose haloed tile does not fit in
// shared memory (large alpha, FP64): neighbours are read from global memory
// (L1 / L2), one thread per voxel of one right-hand side
template <typename T>
__global__ void __launch_bounds__(256) k_z0_direct_g(const T *__restrict__ x, T *__restrict__ y,
                                                     const T *__restrict__ eps, const int4 *__restrict__ dlist,
                                                     const T *__restrict__ gval, int nd, int Nx, int Ny, int Nz,
                                                     T dl) {
    const long nv = (long)Nx * Ny * Nz;
    const int b = blockIdx.y;
    const T *xb = x + (long)b * 3 * nv;
    for (long m = (long)blockIdx.x * blockDim.x + threadIdx.x; m < nv; m += (long)gridDim.x * blockDim.x) {
        const int ox = (int)(m % Nx), oy = (int)((m / Nx) % Ny), oz = (int)(m / ((long)Nx * Ny));
        T g0 = T(0), g1 = T(0), g2 = T(0);
        for (int i = 0; i < nd; ++i) {
            const int4 d = dlist[i];
            const int sx = ox - d.x, sy = oy - d.y, sz = oz - d.z;
            if (sx < 0 || sx >= Nx || sy < 0 || sy >= Ny || sz < 0 || sz >= Nz) continue;
            const long s = ((long)sz * Ny + sy) * Nx + sx;
            const T *gv = gval + 6 * (long)i;
            const T u0 = xb[s], u1 = xb[nv + s], u2 = xb[2 * nv + s];
            g0 += gv[0] * u0 + gv[3] * u1 + gv[4] * u2;
            g1 += gv[3] * u0 + gv[1] * u1 + gv[5] * u2;
            g2 += gv[4] * u0 + gv[5] * u1 + gv[2] * u2;
        }
        const T e = eps[m];
        T *yb = y + (long)b * 3 * nv;
        const T dg = e * T(0.5) + dl;
        yb[m] = dg * xb[m] - (e - T(1)) * g0;
        yb[nv + m] = dg * xb[nv + m] - (e - T(1)) * g1;
        yb[2 * nv + m] = dg * xb[2 * nv + m] - (e - T(1)) * g2;
    }
}

}  // namespace mot
