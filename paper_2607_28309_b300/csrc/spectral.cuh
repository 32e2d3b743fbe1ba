// spectral.cuh -- pencil passes of the zero-padded 3-D FFT products (Eq. 11-12).
//
//   (G J)_p = T{ F^-1 [ sum_q Lambda_pq F{J^ext_q} ] },   Z0 J = D J - X (G J)
//
// Data layout on the device (x fastest everywhere, H = Mx/2 + 1):
//   current vectors        [B][3][Nz][Ny][Nx]           real
//   after the x pass       [B][3][Nz][Ny][H]            complex   ("rows")
//   after the y pass       [B][3][Nz][My][H]            complex   ("planes")
//   full spectra (ring)    [B][3][Mz][My][H]            complex
//   Green spectra          [6][Mz/2+1][My/2+1][H]       real octant, components
//                          (xx, yy, zz, xy, xz, yz); 1/(Mx My Mz) folded in.
// Zero padding is implicit: padded rows are never read, they are created as
// zeros in shared memory; truncation T{.} is implicit: only the Nz (Ny, Nx)
// needed outputs are written.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace mot {

// ---------------------------------------------------------------------------
// x pass, forward: two real rows form one complex sequence z = a + i b,
// FFT of length Mx (a, b zero padded from Nx), then
//   A[k] = (Z[k] + conj Z[M-k]) / 2,  B[k] = -i (Z[k] - conj Z[M-k]) / 2,  k < H.
// grid.x = ceil(nrows / (2 * pairs)); dynamic smem: (2 * pairs + 1) * Mx complex
// ---------------------------------------------------------------------------
template <typename TI, typename T>
__global__ void __launch_bounds__(256) k_x_forward(const TI *__restrict__ x, cplx<T> *__restrict__ out,
                                                   long nrows, int Nx, int H, FftPlan pl,
                                                   const cplx<T> *__restrict__ tw_g, int pairs) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int M = pl.M;
    C *a = tw + M;
    C *b = a + pairs * M;
    load_twiddles(tw, tw_g, M);
    const long row0 = (long)blockIdx.x * 2 * pairs;
    const int nload = 2 * pairs * Nx;
    for (int i = threadIdx.x; i < nload; i += blockDim.x) {
        int rr = i / Nx, e = i - rr * Nx;
        long row = row0 + rr;
        T v = row < nrows ? (T)x[row * Nx + e] : T(0);
        T *slot = reinterpret_cast<T *>(&a[(rr >> 1) * M + e]);
        slot[rr & 1] = v;
    }
    const int npad = M - Nx;
    for (int i = threadIdx.x; i < pairs * npad; i += blockDim.x) {
        int p = i / npad, e = Nx + (i - p * npad);
        a[p * M + e] = cmake<C>(T(0), T(0));
    }
    __syncthreads();
    C *res = block_fft<-1>(a, b, pl, pairs, M, 1, tw, false);
    for (int i = threadIdx.x; i < pairs * H; i += blockDim.x) {
        int p = i / H, k = i - p * H;
        C z = res[p * M + k];
        C zm = cconj(res[p * M + (k == 0 ? 0 : M - k)]);
        C s = cadd(z, zm), d = csub(z, zm);
        long r = row0 + 2 * p;
        if (r < nrows) out[r * H + k] = cmake<C>(T(0.5) * s.x, T(0.5) * s.y);
        if (r + 1 < nrows) out[(r + 1) * H + k] = cmake<C>(T(0.5) * d.y, T(-0.5) * d.x);
    }
}

// ---------------------------------------------------------------------------
// strided-axis pass (y or z), forward or inverse, over a tile of tx columns.
// Input pencil element e (e < Lin) of column c at
//   in + o1*is1 + o2*is2 + e*ias + kx0 + c ;   elements Lin..M-1 are zero.
// Output elements e < Lout at out + o1*os1 + o2*os2 + e*oas + kx0 + c.
// grid = (ceil(H/tx), O1*O2); dynamic smem: (2*M*tx + M) complex
// ---------------------------------------------------------------------------
template <typename T, int S>
__global__ void __launch_bounds__(256) k_axis(const cplx<T> *__restrict__ in, cplx<T> *__restrict__ out,
                                              FftPlan pl, const cplx<T> *__restrict__ tw_g, int H, int tx,
                                              int Lin, int Lout, int O2, long is1, long is2, long ias,
                                              long os1, long os2, long oas) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int M = pl.M;
    C *a = tw + M;
    C *b = a + M * tx;
    load_twiddles(tw, tw_g, M);
    const int o = blockIdx.y, o1 = o / O2, o2 = o - o1 * O2;
    const int kx0 = blockIdx.x * tx;
    const int w = min(tx, H - kx0);
    const C *src = in + o1 * is1 + o2 * is2 + kx0;
    for (int i = threadIdx.x; i < M * tx; i += blockDim.x) {
        int e = i / tx, c = i - e * tx;
        a[i] = (e < Lin && c < w) ? src[e * ias + c] : cmake<C>(T(0), T(0));
    }
    __syncthreads();
    C *res = block_fft<S>(a, b, pl, tx, 1, tx, tw, true);
    C *dst = out + o1 * os1 + o2 * os2 + kx0;
    for (int i = threadIdx.x; i < Lout * tx; i += blockDim.x) {
        int e = i / tx, c = i - e * tx;
        if (c < w) dst[e * oas + c] = res[i];
    }
}

// Green-spectrum lookup: octant value with the parity signs of each component.
// comp: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz (even in every axis for xx..zz,
// odd in both axes of its indices for the mixed ones).
struct Octant {
    int Mz, My, Kz, Ky, H;
    __device__ __forceinline__ void fold(int kz, int ky, int &fz, int &fy, float &sz, float &sy) const {
        if (2 * kz > Mz) { fz = Mz - kz; sz = -1.f; } else { fz = kz; sz = 1.f; }
        if (2 * ky > My) { fy = My - ky; sy = -1.f; } else { fy = ky; sy = 1.f; }
    }
};

template <typename T>
__device__ __forceinline__ void green_mul(const T *__restrict__ L, long cstride, long idx, float sz, float sy,
                                          const cplx<T> u[3], cplx<T> v[3]) {
    using C = cplx<T>;
    T gxx = L[idx], gyy = L[cstride + idx], gzz = L[2 * cstride + idx];
    T gxy = sy * L[3 * cstride + idx], gxz = sz * L[4 * cstride + idx], gyz = (sy * sz) * L[5 * cstride + idx];
    v[0] = cmake<C>(gxx * u[0].x + gxy * u[1].x + gxz * u[2].x, gxx * u[0].y + gxy * u[1].y + gxz * u[2].y);
    v[1] = cmake<C>(gxy * u[0].x + gyy * u[1].x + gyz * u[2].x, gxy * u[0].y + gyy * u[1].y + gyz * u[2].y);
    v[2] = cmake<C>(gxz * u[0].x + gyz * u[1].x + gzz * u[2].x, gxz * u[0].y + gyz * u[1].y + gzz * u[2].y);
}

// ---------------------------------------------------------------------------
// present-time z pass (Eq. 11): for one (b, ky) and a tile of tx kx-columns,
// FFT_z of the three components (Nz rows, zero padded to Mz), 3x3 multiply by
// Lambda0, inverse FFT_z, keep z < Nz.  In place on the [B][3][Nz][My][H] buffer.
// grid = (ceil(H/tx), B*My); dynamic smem: (6*Mz*tx + Mz) complex
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_z_green(cplx<T> *__restrict__ buf, const T *__restrict__ L,
                                                 FftPlan pl, const cplx<T> *__restrict__ tw_g, int Nz,
                                                 int My, int H, int tx, Octant oc) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int M = pl.M;
    C *a = tw + M;
    C *b = a + 3 * M * tx;
    load_twiddles(tw, tw_g, M);
    const int bb = blockIdx.y / My, ky = blockIdx.y - bb * My;
    const int kx0 = blockIdx.x * tx;
    const int w = min(tx, H - kx0);
    const long plane = (long)My * H;   // z stride
    const long comp = (long)Nz * plane;  // component stride
    C *base = buf + (long)bb * 3 * comp + (long)ky * H + kx0;
    const int ntx = 3 * tx;
    // smem layout [e][q][c]: pencil p = q*tx + c, element stride 3*tx
    for (int i = threadIdx.x; i < M * ntx; i += blockDim.x) {
        int e = i / ntx, r = i - e * ntx, q = r / tx, c = r - q * tx;
        a[i] = (e < Nz && c < w) ? base[q * comp + e * plane + c] : cmake<C>(T(0), T(0));
    }
    __syncthreads();
    C *res = block_fft<-1>(a, b, pl, ntx, 1, ntx, tw, true);
    const long cs = (long)oc.Kz * oc.Ky * oc.H;
    for (int i = threadIdx.x; i < M * tx; i += blockDim.x) {
        int kz = i / tx, c = i - kz * tx;
        if (c >= w) continue;
        int fz, fy;
        float sz, sy;
        oc.fold(kz, ky, fz, fy, sz, sy);
        long idx = ((long)fz * oc.Ky + fy) * oc.H + kx0 + c;
        C u[3], v[3];
        for (int q = 0; q < 3; ++q) u[q] = res[kz * ntx + q * tx + c];
        green_mul<T>(L, cs, idx, sz, sy, u, v);
        for (int q = 0; q < 3; ++q) res[kz * ntx + q * tx + c] = v[q];
    }
    __syncthreads();
    C *other = (res == a) ? b : a;
    C *res2 = block_fft<+1>(res, other, pl, ntx, 1, ntx, tw, true);
    for (int i = threadIdx.x; i < Nz * ntx; i += blockDim.x) {
        int e = i / ntx, r = i - e * ntx, q = r / tx, c = r - q * tx;
        if (c < w) base[q * comp + e * plane + c] = res2[i];
    }
}

// ---------------------------------------------------------------------------
// history z pass: S = sum_{k=1..ell} Lambda_k Jhat_{n-k} on the full Mz column
// of one (b, ky, kx tile), then inverse FFT_z and keep z < Nz.
// ring slot s holds Jhat_{j} for j = s (mod ell); lag k pairs with slot
// (n - k) mod ell.  Lambda_k octants are stacked [ell+1][6][Kz][Ky][H].
// out: [B][3][Nz][My][H].  grid = (ceil(H/tx), B*My); smem (6*Mz*tx + Mz) complex
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_z_history(const cplx<T> *__restrict__ ring, const T *__restrict__ Lh,
                                                   cplx<T> *__restrict__ out, FftPlan pl,
                                                   const cplx<T> *__restrict__ tw_g, int Nz, int My, int H,
                                                   int tx, Octant oc, int nrhs, int ell, long n, int kmax) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int M = pl.M;
    C *a = tw + M;
    C *b = a + 3 * M * tx;
    load_twiddles(tw, tw_g, M);
    const int bb = blockIdx.y / My, ky = blockIdx.y - bb * My;
    const int kx0 = blockIdx.x * tx;
    const int w = min(tx, H - kx0);
    const long plane = (long)My * H;
    const long slot_comp = (long)M * plane;              // ring component stride
    const long slot_size = (long)nrhs * 3 * slot_comp;   // one ring slot
    const long cs = (long)oc.Kz * oc.Ky * oc.H;          // octant component stride
    const int ntx = 3 * tx;
    for (int i = threadIdx.x; i < M * tx; i += blockDim.x) {
        int kz = i / tx, c = i - kz * tx;
        C acc[3] = {cmake<C>(T(0), T(0)), cmake<C>(T(0), T(0)), cmake<C>(T(0), T(0))};
        if (c < w) {
            int fz, fy;
            float sz, sy;
            oc.fold(kz, ky, fz, fy, sz, sy);
            long lidx = ((long)fz * oc.Ky + fy) * oc.H + kx0 + c;
            long ridx = (long)bb * 3 * slot_comp + (long)kz * plane + (long)ky * H + kx0 + c;
            for (int k = 1; k <= kmax; ++k) {
                long s = (n - k) % ell;
                if (s < 0) s += ell;
                const C *R = ring + s * slot_size + ridx;
                C u[3] = {R[0], R[slot_comp], R[2 * slot_comp]}, v[3];
                green_mul<T>(Lh + (long)k * 6 * cs, cs, lidx, sz, sy, u, v);
                acc[0] = cadd(acc[0], v[0]);
                acc[1] = cadd(acc[1], v[1]);
                acc[2] = cadd(acc[2], v[2]);
            }
        }
        for (int q = 0; q < 3; ++q) a[kz * ntx + q * tx + c] = acc[q];
    }
    __syncthreads();
    C *res = block_fft<+1>(a, b, pl, ntx, 1, ntx, tw, true);
    const long comp = (long)Nz * plane;
    C *dst = out + (long)bb * 3 * comp + (long)ky * H + kx0;
    for (int i = threadIdx.x; i < Nz * ntx; i += blockDim.x) {
        int e = i / ntx, r = i - e * ntx, q = r / tx, c = r - q * tx;
        if (c < w) dst[q * comp + e * plane + c] = res[i];
    }
}

// ---------------------------------------------------------------------------
// x pass, inverse (C2R) with a fused epilogue.  Rows 2p, 2p+1 of half spectra
// A, B become Z[k] = A[k] + i B[k] (Hermitian extension for k > M/2), inverse
// FFT, and a = Re z, b = Im z for e < Nx.  The epilogue receives the Green
// product G at (row, e).  grid.x = ceil(nrows/(2*pairs));
// dynamic smem: (2*pairs*H + 2*pairs*Mx + Mx) complex
// ---------------------------------------------------------------------------
template <typename T, class Epi>
__global__ void __launch_bounds__(256) k_x_inverse(const cplx<T> *__restrict__ in, long nrows, int Nx, int H,
                                                   FftPlan pl, const cplx<T> *__restrict__ tw_g, int pairs,
                                                   Epi epi) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int M = pl.M;
    C *stage = tw + M;
    C *a = stage + 2 * pairs * H;
    C *b = a + pairs * M;
    load_twiddles(tw, tw_g, M);
    const long row0 = (long)blockIdx.x * 2 * pairs;
    for (int i = threadIdx.x; i < 2 * pairs * H; i += blockDim.x) {
        int rr = i / H, k = i - rr * H;
        long row = row0 + rr;
        C v = row < nrows ? in[row * H + k] : cmake<C>(T(0), T(0));
        // the DC and (even M) Nyquist bins of a real sequence are real
        if (k == 0 || 2 * k == M) v.y = T(0);
        stage[i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pairs * M; i += blockDim.x) {
        int p = i / M, k = i - p * M;
        C A, B;
        if (k < H) { A = stage[(2 * p) * H + k]; B = stage[(2 * p + 1) * H + k]; }
        else { A = cconj(stage[(2 * p) * H + (M - k)]); B = cconj(stage[(2 * p + 1) * H + (M - k)]); }
        a[i] = cmake<C>(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    C *res = block_fft<+1>(a, b, pl, pairs, M, 1, tw, false);
    for (int i = threadIdx.x; i < 2 * pairs * Nx; i += blockDim.x) {
        int rr = i / Nx, e = i - rr * Nx;
        long row = row0 + rr;
        if (row >= nrows) continue;
        C z = res[(rr >> 1) * M + e];
        double g = (rr & 1) ? (double)z.y : (double)z.x;
        epi(row, e, g);
    }
}

// ----- epilogues (row = ((b*3 + p)*Nz + z)*Ny + y, element row*Nx + e) -----

// Z0 product (Eq. 12): y = eps T(0) x - (eps - 1) G
template <typename TX, typename TY>
struct EpiZ0 {
    const TX *x;
    TY *y;
    const double *eps;
    long plane_rows;  // Nz * Ny
    int Nx;
    __device__ __forceinline__ void operator()(long row, int e, double g) const {
        long idx = row * Nx + e;
        long m = (row % plane_rows) * Nx + e;
        double ep = eps[m];
        y[idx] = (TY)(ep * 0.5 * (double)x[idx] - (ep - 1.0) * g);
    }
};

// refinement residual: r = b - (eps T(0) x - (eps - 1) G), all FP64
struct EpiResidual {
    const double *x, *b;
    double *r;
    const double *eps;
    long plane_rows;
    int Nx;
    __device__ __forceinline__ void operator()(long row, int e, double g) const {
        long idx = row * Nx + e;
        long m = (row % plane_rows) * Nx + e;
        double ep = eps[m];
        r[idx] = b[idx] - (ep * 0.5 * x[idx] - (ep - 1.0) * g);
    }
};

// right-hand side (Eq. 3): b_n = E^i_n - eps T(dt) J_{n-1} + (eps - 1) sum_k G_k J_{n-k}
// (T(k dt) = 0 for k >= 2, so only lag 1 carries the constitutive term);
// E^i_n[b][p][m] = inc[b][m] * pol[b][p]
struct EpiHistory {
    const double *inc;    // [B][n]: (eps - 1) eps0 <dE/dt>/|pol| scalar per voxel
    const double *pol;    // [B][3]
    const double *Jprev;  // [B][3][n] (null at n = 0)
    double *out;          // [B][3][n]
    const double *eps;
    long plane_rows;
    int Nx;
    long nvox;
    __device__ __forceinline__ void operator()(long row, int e, double g) const {
        long idx = row * Nx + e;
        long prow = row % plane_rows;
        long m = prow * Nx + e;
        long bp = row / plane_rows;  // b*3 + p
        long bb = bp / 3;
        int p = (int)(bp - 3 * bb);
        double ep = eps[m];
        double v = inc[bb * nvox + m] * pol[bb * 3 + p] + (ep - 1.0) * g;
        if (Jprev) v -= ep * 0.5 * Jprev[idx];
        out[idx] = v;
    }
};

}  // namespace mot
