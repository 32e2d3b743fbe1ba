// tables.cuh -- device generation of the lag tables g_k(d) and of their
// circulant spectra Lambda_k (Sec. IV: "precomputed spectral coefficients of
// the circulant Green-function kernel").
//
// Lag tables are computed once per sorted offset 0 <= a <= b <= c and spread
// to the nonnegative octant with the permutation covariance of the Galerkin
// kernel.  The quadrature runs once per distinct plane integral (one GPU thread
// per face) and once per sorted offset for the box integrals (one thread per
// offset), as knot-interval moments; a third kernel combines them into the
// entries of every lag (one thread per lag/offset item).  Because g_pp is even in every
// coordinate and g_pq (p != q) is odd in d_p and d_q and even in the third, the
// DFT of the circulant embedding is real and is a product of one-dimensional
// cosine / sine sums over the octant:
//   Lambda_pq(k) = sgn * prod_i sum_{d_i = 0..R_i} c_i(k_i, d_i) g_pq(d),
//   c(k, d) = 1 (d = 0) or 2 cos(2 pi k d / M) on even axes, 2 sin(2 pi k d / M)
//   on odd axes, sgn = -1 for the mixed components ((-i)^2), and 1/(Mx My Mz)
//   folded in.  This is the FFT of Eq. 11's kernel written out exactly.
#pragma once

#include "common.cuh"
#include "galerkin.cuh"

namespace mot {

// one item: lag k and sorted offset (a, b, c); t = its TripleRec
struct TableItem {
    int k, a, b, c, t;
};

// one plane integral of the second-difference stencil: plane at distance c,
// in-plane offset (a, b) with 0 <= a <= b; its moments are FM[off .. off + 3 nj)
struct FaceRec {
    int c, a, b, jlo, nj;
    long off;
};

// one sorted offset x <= y <= z: the moments of its three box integrals
// ((x, y; z), (x, z; y), (y, z; x)) are BM[off + 3 nj comp .. + 3 nj), and
// face[3 p + e + 1] is the FaceRec of the plane at d_p + e (e = -1, 0, 1)
struct TripleRec {
    int x, y, z, jlo, nj;
    long off;
    int face[9];
};

__global__ void k_face_moments(const FaceRec *__restrict__ faces, int n, double rho, const double *__restrict__ glx,
                               const double *__restrict__ glw, int gln, double *__restrict__ FM) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const FaceRec f = faces[i];
    if (f.nj <= 0) return;
    double *o = FM + f.off;
    for (int m = 0; m < 3 * f.nj; ++m) o[m] = 0.0;
    gk::Rule q = {glx, glw, gln};
    gk::face_moments(q, rho, (double)f.c, (double)f.a, (double)f.b, f.jlo, f.nj, o);
}

// glx / glw hold the gln-point rule followed by the gl8-point rule of the z-lines
__global__ void k_box_moments(const TripleRec *__restrict__ tri, int n, double rho, const double *__restrict__ glx,
                              const double *__restrict__ glw, int gln, int gl8, double *__restrict__ BM) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TripleRec t = tri[i];
    if (t.nj <= 0) return;
    double *o = BM + t.off;
    for (int m = 0; m < 9 * t.nj; ++m) o[m] = 0.0;
    gk::Rule q = {glx, glw, gln}, q8 = {glx + gln, glw + gln, gl8};
    const double x = t.x, y = t.y, z = t.z;
    gk::box_moments(q, q8, rho, x, y, z, t.jlo, t.nj, o);
    gk::box_moments(q, q8, rho, x, z, y, t.jlo, t.nj, o + 3 * t.nj);
    gk::box_moments(q, q8, rho, y, z, x, t.jlo, t.nj, o + 6 * t.nj);
}

// A_k(d) of one item from its faces' and boxes' moments: A00, A11, A22, A01, A02, A12
__host__ __device__ inline void combine_item(const TableItem &it, const TripleRec *tri, const FaceRec *faces,
                                             const double *FM, const double *BM, double *A6) {
    const TripleRec &t = tri[it.t];
    for (int p = 0; p < 3; ++p) {
        double acc = 0.0;
        for (int e = 0; e < 3; ++e) {
            const FaceRec &f = faces[t.face[3 * p + e]];
            const double v = f.nj > 0 ? gk::lag_from_moments(FM + f.off, f.jlo, f.nj, it.k) : 0.0;
            acc += (e == 1 ? -2.0 : 1.0) * v;
        }
        A6[p] = acc;
    }
    for (int c = 0; c < 3; ++c)
        A6[3 + c] = t.nj > 0 ? gk::lag_from_moments(BM + t.off + 3 * t.nj * c, t.jlo, t.nj, it.k) : 0.0;
}

__global__ void k_combine_items(const TableItem *__restrict__ items, int n, const TripleRec *__restrict__ tri,
                                const FaceRec *__restrict__ faces, const double *__restrict__ FM,
                                const double *__restrict__ BM, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    combine_item(items[i], tri, faces, FM, BM, out + 6 * (long)i);
}

__host__ __device__ inline int a6_index(int p, int q) {
    if (p == q) return p;
    int s = p + q;  // 1 -> (0,1), 2 -> (0,2), 3 -> (1,2)
    return 2 + s;
}

// g on the octant d >= 0 from the sorted-offset values A6 (A00 A11 A22 A01 A02 A12);
// map[(a*(Rm+1) + b)*(Rm+1) + c] = item index (or -1).  out: [6][Rz+1][Ry+1][Rx+1]
__host__ __device__ inline void expand_one(const double *A6, const int *map, int Rm, int dx, int dy, int dz,
                                           double *g6) {
    int d[3] = {dx, dy, dz}, ax[3] = {0, 1, 2};
    for (int i = 1; i < 3; ++i) {
        int j = i;
        while (j > 0 && d[ax[j - 1]] > d[ax[j]]) {
            int t = ax[j];
            ax[j] = ax[j - 1];
            ax[j - 1] = t;
            --j;
        }
    }
    long key = ((long)d[ax[0]] * (Rm + 1) + d[ax[1]]) * (Rm + 1) + d[ax[2]];
    int id = map[key];
    for (int c = 0; c < 6; ++c) g6[c] = 0.0;
    if (id < 0) return;
    int pos[3];
    for (int j = 0; j < 3; ++j) pos[ax[j]] = j;
    const double *A = A6 + 6 * (long)id;
    double tr = A[0] + A[1] + A[2];
    const int pp[6] = {0, 1, 2, 0, 0, 1}, qq[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; ++c) {
        double v = A[a6_index(pos[pp[c]], pos[qq[c]])];
        g6[c] = (c < 3) ? v - tr : v;
    }
}

// the item index of lag k for every sorted offset (dense key), -1 where lag k
// has no item: map = base + (k - klo) for klo <= k < klo + cnt
__global__ void k_lag_map(const int *__restrict__ base, const int *__restrict__ klo, const int *__restrict__ cnt,
                          long n, int k, int *__restrict__ map) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = base[i], lo = klo[i];
        map[i] = (b >= 0 && k >= lo && k < lo + cnt[i]) ? b + (k - lo) : -1;
    }
}

__global__ void k_expand_octant(const double *__restrict__ A6, const int *__restrict__ map, int Rm, int Rx, int Ry,
                                int Rz, double *__restrict__ oct) {
    long n = (long)(Rx + 1) * (Ry + 1) * (Rz + 1);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        int dx = (int)(i % (Rx + 1)), dy = (int)((i / (Rx + 1)) % (Ry + 1)), dz = (int)(i / ((long)(Rx + 1) * (Ry + 1)));
        double g6[6];
        expand_one(A6, map, Rm, dx, dy, dz, g6);
        for (int c = 0; c < 6; ++c) oct[c * n + i] = g6[c];
    }
}

// one separable pass: out[o][k][i] = sum_d coef[k][d] in[o][d][i]
__global__ void k_axis_sum(const double *__restrict__ in, double *__restrict__ out, const double *__restrict__ coef,
                           int nouter, int Rin, int K, int ninner) {
    long n = (long)nouter * K * ninner;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        int i = (int)(t % ninner);
        int k = (int)((t / ninner) % K);
        long o = t / ((long)ninner * K);
        const double *src = in + o * Rin * ninner + i;
        const double *cf = coef + (long)k * Rin;
        double acc = 0.0;
        for (int d = 0; d < Rin; ++d) acc += cf[d] * src[(long)d * ninner];
        out[t] = acc;
    }
}

// batched C = s A B in double-float arithmetic on FP64 data, for the separable
// transforms of the history spectra (each pass a product of a coefficient
// matrix and a stack of table lines).  Element (m, k) of batch z of A is at
// A + z sAz + m sAm + k sAk (B and C alike).  64 x 64 outputs per block of 256
// threads, 4 x 4 per thread, K in chunks of 16 staged in shared memory as
// (hi, lo) pairs; products by the double-word product, sums by the double-word
// sum (absolute error about 2^-47 of the magnitudes summed: K <= 256 terms of
// one sign-mixed sum stay within 2e-12 of their absolute sum, far below what
// the spectra's users resolve).  grid (ceil(N/64), ceil(M/64), batches)
struct GemmView {
    const double *p;
    long sz, sr, sc;  // batch, row, column strides (elements)
};
__global__ void __launch_bounds__(256) k_gemm_df(GemmView A, GemmView B, double *__restrict__ C, long sCz, long sCm,
                                                 long sCn, int M, int N, int K, double s) {
    __shared__ dfl As[16][64 + 1];
    __shared__ dfl Bs[16][64 + 1];
    const int z = blockIdx.z, m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const double *Ab = A.p + z * A.sz, *Bb = B.p + z * B.sz;
    dfl acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = dfl(0.0f, 0.0f);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? to_dfl(Ab[m * A.sr + k * A.sc]) : dfl(0.0f, 0.0f);
            const int n = n0 + mm;
            Bs[kk][mm] = (n < N && k < K) ? to_dfl(Bb[k * B.sr + n * B.sc]) : dfl(0.0f, 0.0f);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            dfl a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = acc[i][j] + a[i] * b[j];
        }
        __syncthreads();
    }
    double *Cb = C + z * sCz;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m < M && n < N) Cb[m * sCm + n * sCn] = s * to_double(acc[i][j]);
        }
}

template <typename T>
__global__ void k_scale_store(const double *__restrict__ src, T *__restrict__ dst, long n, double s) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (T)(src[i] * s);
}

}  // namespace mot
