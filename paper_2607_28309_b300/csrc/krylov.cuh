// krylov.cuh -- batched TFQMR (Freund 1993, the solver of Sec. II) vector
// kernels, FP64 inner products, and the incident right-hand side (Eq. 7-8).
//
// Vectors are [B][L] (L = 3 * Nx * Ny * Nz); every right-hand side b keeps
// its own scalars in TfqmrScal.  Inner products and norms use a deterministic
// two-level reduction: each thread sums its strided elements in the vector
// precision, block sums and the final sum (one warp per right-hand side, fixed
// order) are FP64.
#pragma once

#include <math.h>

#include "common.cuh"

namespace mot {

struct TfqmrScal {
    double rho, alpha, theta, eta, tau, beta;
    double eta_prev;     // eta of the half step whose x update is pending
    double bnorm;        // ||b||
    double tolabs;       // tol * ||b||
    int m;               // half steps done
    int conv;            // 1 once tau sqrt(m+1) <= tolabs (or b == 0)
    int pending;         // 1 if x += eta_prev d is still to be applied
    int pad;
    // the vector-update coefficients rounded to FP32 once per scalar update,
    // so FP32 kernels read them without FP64 arithmetic:
    // alpha, theta^2 eta / alpha, eta_prev, beta
    float f_alpha, f_coef, f_eta_prev, f_beta;
    // stagnation test (inner FP32 solves of the mixed form): tau at half step
    // m_ck; stag = 1 enables it
    double tau_ck;
    int m_ck, stag;
};

// an inner solve whose tau has not halved over kStagHalfSteps half steps has
// met its precision's floor: it stops (conv 2) and the FP64 refinement goes on
// from the true residual
constexpr int kStagHalfSteps = 16;
constexpr double kStagRatio = 0.5;

__host__ __device__ inline void refresh_coefs(TfqmrScal &s) {
    s.f_alpha = (float)s.alpha;
    s.f_coef = s.alpha != 0.0 ? (float)(s.theta * s.theta * s.eta / s.alpha) : 0.f;
    s.f_eta_prev = (float)s.eta_prev;
    s.f_beta = (float)s.beta;
}

// the coefficients of a vector update in the vector precision V
template <typename V> struct Coefs;
template <> struct Coefs<float> {
    __device__ static float al(const TfqmrScal &s) { return s.f_alpha; }
    __device__ static float coef(const TfqmrScal &s) { return s.f_coef; }
    __device__ static float ep(const TfqmrScal &s) { return s.f_eta_prev; }
    __device__ static float be(const TfqmrScal &s) { return s.f_beta; }
};
template <> struct Coefs<double> {
    __device__ static double al(const TfqmrScal &s) { return s.alpha; }
    __device__ static double coef(const TfqmrScal &s) { return s.theta * s.theta * s.eta / s.alpha; }
    __device__ static double ep(const TfqmrScal &s) { return s.eta_prev; }
    __device__ static double be(const TfqmrScal &s) { return s.beta; }
};

constexpr int kRedBlocks = 296;  // 2 x 148 SMs
constexpr int kRedThreads = 256;

// per-thread accumulator of the element sums: the vector precision (a thread
// sums about L / (kRedBlocks * kRedThreads) terms), FP64 from the block sums on
template <typename V> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float; };

// 16-byte packs of vector elements (4 floats, 2 doubles): the fused kernels
// move whole packs when the per-right-hand-side length L is a multiple of the
// pack width (then every right-hand side's slice starts 16-byte aligned) and
// fall back to single elements otherwise
template <typename V> struct PackW { static constexpr int W = 16 / sizeof(V); };

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block, valid in thread 0: the warp sums in the accumulator
// precision A, the sum of the warp sums in FP64
template <typename A> __device__ __forceinline__ double block_sum(A v, double *sh) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// part[b*kRedBlocks + blk] = sum a*c over the block's slice;  grid (kRedBlocks, B)
template <typename TA, typename TC>
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const TA *__restrict__ a, const TC *__restrict__ c,
                                                          long L, double *__restrict__ part) {
    __shared__ double sh[32];
    const int b = blockIdx.y;
    const TA *pa = a + (long)b * L;
    const TC *pc = c + (long)b * L;
    using A = typename AccOf<TA>::type;
    A s = A(0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        s += (A)pa[i] * (A)pc[i];
    const double bs = block_sum(s, sh);
    if (threadIdx.x == 0) part[b * kRedBlocks + blockIdx.x] = bs;
}

__device__ __forceinline__ double reduce_parts(const double *part, int b) {
    // one warp, fixed order
    double s = 0.0;
    for (int i = threadIdx.x; i < kRedBlocks; i += 32) s += part[b * kRedBlocks + i];
    return warp_sum(s);
}

// ---- initialisation: r = b - A x0 already in w; tau = ||w||, rho = tau^2 --
// (conv 3: b = 0, whose solution is 0 whatever x0 is; x still to be zeroed)
__device__ __forceinline__ TfqmrScal init_scalars(double r2, double b2, double tol, int stag) {
    TfqmrScal s;
    s.tau = sqrt(r2);
    s.rho = r2;
    s.theta = 0.0;
    s.eta = 0.0;
    s.alpha = 0.0;
    s.beta = 0.0;
    s.eta_prev = 0.0;
    s.bnorm = sqrt(b2);
    s.tolabs = tol * s.bnorm;
    s.m = 0;
    s.conv = b2 == 0.0 ? 3 : ((s.tau <= s.tolabs || r2 == 0.0) ? 1 : 0);
    s.pending = 0;
    s.pad = 0;
    s.tau_ck = s.tau;
    s.m_ck = 0;
    s.stag = stag;
    refresh_coefs(s);
    return s;
}

// Relative tolerance of an inner (correction) solve of the mixed refinement:
// the correction only has to bring the outer residual r below the outer
// tolerance, so a solve whose residual is already small relative to the outer
// right-hand side b needs less than inner_tol:
//   tol_b = min(max(inner_tol, otol ||b|| / ||r||), 1/2),  otol = a fraction of the outer tol.
// bo2 / ro2: ||b||^2 / ||r||^2 per right-hand side (nullptr: inner_tol as given).
struct InnerTol {
    const double *bo2 = nullptr, *ro2 = nullptr;
    double otol = 0.0;
};
__device__ __forceinline__ double inner_tol_of(double tol, const InnerTol &it, int b) {
    if (!it.bo2 || !it.ro2) return tol;
    const double rr = it.ro2[b];
    if (!(rr > 0.0)) return tol;
    return fmin(fmax(tol, it.otol * sqrt(it.bo2[b] / rr)), 0.5);
}

// grid B, block 32
__global__ void k_tfqmr_init(TfqmrScal *sc, const double *part_r2, const double *part_b2, double tol, int stag,
                             InnerTol itol) {
    const int b = blockIdx.x;
    double r2 = reduce_parts(part_r2, b);
    double b2 = reduce_parts(part_b2, b);
    if (threadIdx.x == 0) sc[b] = init_scalars(r2, b2, inner_tol_of(tol, itol, b), stag);
}

// x = 0 for right-hand sides with b = 0 (conv == 3), then mark them done
template <typename V>
__global__ void k_tfqmr_zero_rhs(V *__restrict__ x, TfqmrScal *__restrict__ sc, long L) {
    const int b = blockIdx.y;
    if (sc[b].conv != 3) return;
    const long o = (long)b * L;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x) x[o + i] = V(0);
}

__global__ void k_tfqmr_zero_done(TfqmrScal *sc, int B) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B && sc[b].conv == 3) sc[b].conv = 1;
}

// sigma = (r*, v): alpha = rho / sigma.  grid B, block 32
__global__ void k_tfqmr_alpha(TfqmrScal *sc, const double *part) {
    const int b = blockIdx.x;
    double sigma = reduce_parts(part, b);
    if (threadIdx.x == 0 && !sc[b].conv) {
        if (sigma == 0.0) sc[b].conv = 2;  // breakdown: keep the current iterate
        else {
            TfqmrScal u = sc[b];
            u.alpha = u.rho / sigma;
            refresh_coefs(u);
            sc[b] = u;
        }
    }
}

// Fused iteration kernels.  Each reduction kernel ends with its scalar update:
// the block that finishes last (counted with an atomic ticket after a memory
// fence) reduces every right-hand side's partials in fixed order, so the
// result does not depend on which block finished last.
// true in every thread of the block that finished last; ctr is left at 0 by
// that block (kernel end), ready for the next launch
__device__ __forceinline__ bool last_block(unsigned *ctr, unsigned total) {
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ctr, 1u) == total - 1u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last != 0;
}

__device__ __forceinline__ double reduce_parts_lane(const double *part, int b, int lane) {
    double s = 0.0;
    for (int i = lane; i < kRedBlocks; i += 32) s += __ldcg(part + b * kRedBlocks + i);
    return warp_sum(s);
}

// theta = ||w||/tau, c = 1/sqrt(1+theta^2), tau = tau theta c, eta = c^2 alpha;
// converged once tau sqrt(m+1) <= tol ||b|| (conv 2: pending update still due)
__device__ __forceinline__ void half_scalars(TfqmrScal &s, double w2) {
    double th = sqrt(w2) / s.tau;
    double c = 1.0 / sqrt(1.0 + th * th);
    s.tau = s.tau * th * c;
    s.theta = th;
    s.eta = c * c * s.alpha;
    s.eta_prev = s.eta;
    s.pending = 1;
    s.m += 1;
    if (s.tau * sqrt((double)s.m + 1.0) <= s.tolabs) s.conv = 2;
    else if (s.stag && s.m - s.m_ck >= kStagHalfSteps) {
        if (s.tau > kStagRatio * s.tau_ck) s.conv = 2;
        s.tau_ck = s.tau;
        s.m_ck = s.m;
    }
    refresh_coefs(s);
}

// first half step of an iteration, on (y1, Ay1):
//   x += eta_prev d (pending); w -= alpha Ay1; d = y1 + (theta^2 eta/alpha) d;
//   y2 = y1 - alpha v;  ||w||^2  ->  theta, tau, eta.   grid (kRedBlocks, B)
template <typename V>
__global__ void __launch_bounds__(kRedThreads) k_tfqmr_half_a(V *__restrict__ x, V *__restrict__ w,
                                                              V *__restrict__ d, V *__restrict__ y2,
                                                              const V *__restrict__ y1, const V *__restrict__ Ay1,
                                                              const V *__restrict__ v, TfqmrScal *__restrict__ sc,
                                                              long L, double *__restrict__ part, unsigned *ctr) {
    using A = typename AccOf<V>::type;
    __shared__ double sh[32];
    const int b = blockIdx.y;
    const TfqmrScal s = sc[b];
    A w2 = A(0);
    if (!s.conv) {
        const V al = Coefs<V>::al(s);
        const V coef = Coefs<V>::coef(s);
        const V ep = Coefs<V>::ep(s);
        const long o = (long)b * L;
        constexpr int W = PackW<V>::W;
        const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
        const long np = L % W == 0 ? L / W : 0;
#pragma unroll 2
        for (long j = t0; j < np; j += ts) {
            const long i = o + j * W;
            V dd[W], yy[W], ww[W], aa[W], vv[W], xx[W];
            ldv<W>(dd, d + i);
            ldv<W>(yy, y1 + i);
            ldv<W>(ww, w + i);
            ldv<W>(aa, Ay1 + i);
            ldv<W>(vv, v + i);
            if (s.pending) ldv<W>(xx, x + i);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (s.pending) xx[k] += ep * dd[k];
                ww[k] -= al * aa[k];
                w2 += ww[k] * ww[k];
                dd[k] = yy[k] + coef * dd[k];
                yy[k] -= al * vv[k];
            }
            if (s.pending) stv<W>(x + i, xx);
            stv<W>(w + i, ww);
            stv<W>(d + i, dd);
            stv<W>(y2 + i, yy);
        }
        for (long i = np * W + t0; i < L; i += ts) {
            const V dold = d[o + i], yv = y1[o + i];
            if (s.pending) x[o + i] += ep * dold;
            const V wn = w[o + i] - al * Ay1[o + i];
            w[o + i] = wn;
            d[o + i] = yv + coef * dold;
            y2[o + i] = yv - al * v[o + i];
            w2 += wn * wn;
        }
    }
    const double bs = block_sum(w2, sh);
    if (threadIdx.x == 0) part[b * kRedBlocks + blockIdx.x] = bs;
    if (!last_block(ctr, gridDim.x * gridDim.y)) return;
    const int lane = threadIdx.x & 31;
    for (int bb = threadIdx.x >> 5; bb < (int)gridDim.y; bb += blockDim.x >> 5) {
        const double t = reduce_parts_lane(part, bb, lane);
        if (lane == 0 && !sc[bb].conv) {
            TfqmrScal u = sc[bb];
            half_scalars(u, t);
            sc[bb] = u;
        }
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// second half step, on (y2, Ay2): as above without y2, plus rho_new = (r*, w)
// -> beta = rho_new / rho (breakdown at rho = 0).   grid (kRedBlocks, B)
template <typename V>
__global__ void __launch_bounds__(kRedThreads) k_tfqmr_half_b(V *__restrict__ x, V *__restrict__ w,
                                                              V *__restrict__ d, const V *__restrict__ y2,
                                                              const V *__restrict__ Ay2, const V *__restrict__ rs,
                                                              TfqmrScal *__restrict__ sc, long L,
                                                              double *__restrict__ part_w2,
                                                              double *__restrict__ part_rw, unsigned *ctr) {
    using A = typename AccOf<V>::type;
    __shared__ double sh[32];
    const int b = blockIdx.y;
    const TfqmrScal s = sc[b];
    A w2 = A(0), rw = A(0);
    if (!s.conv) {
        const V al = Coefs<V>::al(s);
        const V coef = Coefs<V>::coef(s);
        const V ep = Coefs<V>::ep(s);
        const long o = (long)b * L;
        constexpr int W = PackW<V>::W;
        const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
        const long np = L % W == 0 ? L / W : 0;
#pragma unroll 2
        for (long j = t0; j < np; j += ts) {
            const long i = o + j * W;
            V dd[W], yy[W], ww[W], aa[W], rr[W], xx[W];
            ldv<W>(dd, d + i);
            ldv<W>(yy, y2 + i);
            ldv<W>(ww, w + i);
            ldv<W>(aa, Ay2 + i);
            ldv<W>(rr, rs + i);
            if (s.pending) ldv<W>(xx, x + i);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (s.pending) xx[k] += ep * dd[k];
                ww[k] -= al * aa[k];
                w2 += ww[k] * ww[k];
                rw += rr[k] * ww[k];
                dd[k] = yy[k] + coef * dd[k];
            }
            if (s.pending) stv<W>(x + i, xx);
            stv<W>(w + i, ww);
            stv<W>(d + i, dd);
        }
        for (long i = np * W + t0; i < L; i += ts) {
            const V dold = d[o + i];
            if (s.pending) x[o + i] += ep * dold;
            const V wn = w[o + i] - al * Ay2[o + i];
            w[o + i] = wn;
            d[o + i] = y2[o + i] + coef * dold;
            w2 += wn * wn;
            rw += rs[o + i] * wn;
        }
    }
    const double bw = block_sum(w2, sh);
    const double br = block_sum(rw, sh);
    if (threadIdx.x == 0) {
        part_w2[b * kRedBlocks + blockIdx.x] = bw;
        part_rw[b * kRedBlocks + blockIdx.x] = br;
    }
    if (!last_block(ctr, gridDim.x * gridDim.y)) return;
    const int lane = threadIdx.x & 31;
    for (int bb = threadIdx.x >> 5; bb < (int)gridDim.y; bb += blockDim.x >> 5) {
        const double t = reduce_parts_lane(part_w2, bb, lane);
        const double rn = reduce_parts_lane(part_rw, bb, lane);
        if (lane == 0 && !sc[bb].conv) {
            TfqmrScal u = sc[bb];
            half_scalars(u, t);
            if (!u.conv) {
                if (u.rho == 0.0) u.conv = 2;
                else {
                    u.beta = rn / u.rho;
                    u.rho = rn;
                    refresh_coefs(u);
                }
            }
            sc[bb] = u;
        }
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// y1 = w + beta y2 (used where the product cannot form y1 on the fly)
template <typename V>
__global__ void k_tfqmr_y1(V *__restrict__ y1, const V *__restrict__ w, const V *__restrict__ y2,
                           const TfqmrScal *__restrict__ sc, long L) {
    const int b = blockIdx.y;
    if (sc[b].conv) return;
    const V be = Coefs<V>::be(sc[b]);
    const long o = (long)b * L;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        y1[o + i] = w[o + i] + be * y2[o + i];
}

// y1 = w + beta y2 formed while a forward plane kernel stages it, and stored;
// unchanged for right-hand sides that stopped
template <typename V> struct SrcY1 {
    V *y1;
    const V *w, *y2;
    const TfqmrScal *sc;
    long L;  // vector length of one right-hand side (a multiple of the plane size)
    struct Plane {
        V *y1;
        const V *w, *y2;
        V beta;
        int skip;
        __device__ __forceinline__ void stage(V *sm, int n, StageMap m = StageMap{FastDiv{}, 0}) const {
            constexpr int W = PackW<V>::W;
            if (n % W == 0) {
                for (int j = threadIdx.x; j < n / W; j += blockDim.x) {
                    V a[W], c[W];
                    if (skip) ldv<W>(a, y1 + j * W);
                    else {
                        ldv<W>(a, w + j * W);
                        ldv<W>(c, y2 + j * W);
#pragma unroll
                        for (int k = 0; k < W; ++k) a[k] += beta * c[k];
                        stv<W>(y1 + j * W, a);
                    }
                    V *dst = sm + m(j * W);
#pragma unroll
                    for (int k = 0; k < W; ++k) dst[k] = a[k];
                }
            } else {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    V a;
                    if (skip) a = y1[i];
                    else {
                        a = w[i] + beta * y2[i];
                        y1[i] = a;
                    }
                    sm[m(i)] = a;
                }
            }
        }
    };
    __device__ __forceinline__ Plane bind(long plane, long plane_size) const {
        const long off = plane * plane_size;
        const int b = (int)(off / L);
        return Plane{y1 + off, w + off, y2 + off, Coefs<V>::be(sc[b]), sc[b].conv != 0};
    }
    __device__ __forceinline__ void finish(const Plane &, long, long) const {}
};

// ---------------------------------------------------------------------------
// TFQMR vector updates fused into the Z0 product's plane kernels.  The plane
// kernels load (forward) and store (inverse) every element of every
// right-hand side exactly once, one (b, component, z) plane per block, so an
// element-wise update can ride along: SrcHalfA forms y2 (and the first half
// step's w, d, x updates) while the forward pass reads it, EpiHalfB applies
// the second half step to Ay2 as the inverse pass writes it, EpiV the v
// update to Ay1.  Each block leaves its partial sums at part[b*P + j]
// (P = 3 Nz planes per right-hand side, j the block's plane within it) and
// the last block to finish does the scalar update, as the kernels above do.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double reduce_parts_n(const double *part, int b, int lane, int P) {
    double s = 0.0;
    for (int i = lane; i < P; i += 32) s += __ldcg(part + (long)b * P + i);
    return warp_sum(s);
}

// block sums of NV thread values into part[k][slot]; true in the last block
template <int NV, typename A>
__device__ __forceinline__ bool plane_block_done(const A (&v)[NV], double *const (&part)[NV], long slot,
                                                 unsigned *ctr) {
    __shared__ double sh[32];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double t = block_sum(v[k], sh);
        if (threadIdx.x == 0) part[k][slot] = t;
    }
    return last_block(ctr, gridDim.x * gridDim.y);
}

// first half step (see k_tfqmr_half_a) formed while the forward pass loads y2
template <typename V> struct SrcHalfA {
    V *x, *w, *d, *y2;
    const V *y1, *Ay1, *v;
    TfqmrScal *sc;
    long L;          // vector length of one right-hand side
    double *part;    // ||w||^2 partials [B][P]
    int P;           // planes per right-hand side
    unsigned *ctr;
    struct Plane {
        V *x, *w, *d, *y2;
        const V *y1, *Ay1, *v;
        V al, coef, ep;
        int pending, skip;
        typename AccOf<V>::type w2;
        __device__ __forceinline__ void stage(V *sm, int n, StageMap m = StageMap{FastDiv{}, 0}) {
            constexpr int W = PackW<V>::W;
            if (n % W == 0) {
                for (int j = threadIdx.x; j < n / W; j += blockDim.x) {
                    const long o = (long)j * W;
                    V yy[W];
                    if (skip) {
                        ldv<W>(yy, y2 + o);
                    } else {
                        V dd[W], ww[W], aa[W], vv[W], xx[W];
                        ldv<W>(dd, d + o);
                        ldv<W>(yy, y1 + o);
                        ldv<W>(ww, w + o);
                        ldv<W>(aa, Ay1 + o);
                        ldv<W>(vv, v + o);
                        if (pending) ldv<W>(xx, x + o);
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            if (pending) xx[k] += ep * dd[k];
                            ww[k] -= al * aa[k];
                            w2 += ww[k] * ww[k];
                            dd[k] = yy[k] + coef * dd[k];
                            yy[k] -= al * vv[k];
                        }
                        if (pending) stv<W>(x + o, xx);
                        stv<W>(w + o, ww);
                        stv<W>(d + o, dd);
                        stv<W>(y2 + o, yy);
                    }
                    V *dst = sm + m((int)o);
#pragma unroll
                    for (int k = 0; k < W; ++k) dst[k] = yy[k];
                }
            } else {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    if (skip) {
                        sm[m(i)] = y2[i];
                        continue;
                    }
                    const V dold = d[i], yv = y1[i];
                    if (pending) x[i] += ep * dold;
                    const V wn = w[i] - al * Ay1[i];
                    w[i] = wn;
                    w2 += wn * wn;
                    d[i] = yv + coef * dold;
                    const V y = yv - al * v[i];
                    y2[i] = y;
                    sm[m(i)] = y;
                }
            }
        }
    };
    __device__ __forceinline__ Plane bind(long plane, long plane_size) const {
        const long off = plane * plane_size;
        const TfqmrScal s = sc[(int)(off / L)];
        Plane p{x + off, w + off, d + off, y2 + off, y1 + off, Ay1 + off, v + off, V(0), V(0), V(0),
                s.pending, s.conv != 0, 0};
        if (!p.skip) {
            p.al = Coefs<V>::al(s);
            p.coef = Coefs<V>::coef(s);
            p.ep = Coefs<V>::ep(s);
        }
        return p;
    }
    __device__ __forceinline__ void finish(const Plane &pl, long plane, long plane_size) const {
        const int b = (int)(plane * plane_size / L);
        const typename AccOf<V>::type vals[1] = {pl.w2};
        double *const parts[1] = {part};
        if (!plane_block_done<1>(vals, parts, (long)b * P + (plane - (long)b * P), ctr)) return;
        const int lane = threadIdx.x & 31, B = (int)(gridDim.x / P);
        for (int bb = threadIdx.x >> 5; bb < B; bb += blockDim.x >> 5) {
            const double t = reduce_parts_n(part, bb, lane, P);
            if (lane == 0 && !sc[bb].conv) {
                TfqmrScal u = sc[bb];
                half_scalars(u, t);
                sc[bb] = u;
            }
        }
        if (threadIdx.x == 0) *ctr = 0u;
    }
};

// Ay2 = Z0 y2 (Eq. 12) and the second half step (see k_tfqmr_half_b)
template <typename V> struct EpiHalfB {
    static constexpr bool kPlaneOnly = true;
    const V *y2;
    V *Ay2;
    const V *eps;
    V *x, *w, *d;
    const V *rs;
    TfqmrScal *sc;
    double *part_w2, *part_rw;  // [B][P]
    int P;
    unsigned *ctr;
    V dl = V(0);  // delta of Z0 + delta I
    struct Plane {
        const V *y2;
        V *Ay2;
        const V *eps;
        V *x, *w, *d;
        const V *rs;
        V al, coef, ep;
        int pending, skip;
        typename AccOf<V>::type w2, rw;
        V dl = V(0);
        __device__ __forceinline__ void operator()(int i, V g) {
            const V e = eps[i], yv = y2[i];
            const V ay = (e * V(0.5) + dl) * yv - (e - V(1)) * g;
            Ay2[i] = ay;
            if (skip) return;
            const V dold = d[i];
            if (pending) x[i] += ep * dold;
            const V wn = w[i] - al * ay;
            w[i] = wn;
            d[i] = yv + coef * dold;
            w2 += wn * wn;
            rw += rs[i] * wn;
        }
        template <int W> __device__ __forceinline__ void pack(int i, const V (&g)[W]) {
            V e[W], yv[W], ay[W];
            ldv<W>(e, eps + i);
            ldv<W>(yv, y2 + i);
#pragma unroll
            for (int k = 0; k < W; ++k) ay[k] = (e[k] * V(0.5) + dl) * yv[k] - (e[k] - V(1)) * g[k];
            stv<W>(Ay2 + i, ay);
            if (skip) return;
            V dd[W], ww[W], rr[W], xx[W];
            ldv<W>(dd, d + i);
            ldv<W>(ww, w + i);
            ldv<W>(rr, rs + i);
            if (pending) ldv<W>(xx, x + i);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (pending) xx[k] += ep * dd[k];
                ww[k] -= al * ay[k];
                w2 += ww[k] * ww[k];
                rw += rr[k] * ww[k];
                dd[k] = yv[k] + coef * dd[k];
            }
            if (pending) stv<W>(x + i, xx);
            stv<W>(w + i, ww);
            stv<W>(d + i, dd);
        }
    };
    __device__ __forceinline__ Plane bind(long plane, int Nz, int NyNx) const {
        const long off = plane * (long)NyNx, zoff = (plane % Nz) * (long)NyNx;
        const TfqmrScal s = sc[(int)(plane / P)];
        Plane p{y2 + off, Ay2 + off, eps + zoff, x + off, w + off, d + off, rs + off, V(0), V(0), V(0),
                s.pending, s.conv != 0, 0, 0, dl};
        if (!p.skip) {
            p.al = Coefs<V>::al(s);
            p.coef = Coefs<V>::coef(s);
            p.ep = Coefs<V>::ep(s);
        }
        return p;
    }
    __device__ __forceinline__ void finish(const Plane &pl, long plane) const {
        const int b = (int)(plane / P);
        const typename AccOf<V>::type vals[2] = {pl.w2, pl.rw};
        double *const parts[2] = {part_w2, part_rw};
        if (!plane_block_done<2>(vals, parts, plane, ctr)) return;
        const int lane = threadIdx.x & 31, B = (int)(gridDim.x / P);
        (void)b;
        for (int bb = threadIdx.x >> 5; bb < B; bb += blockDim.x >> 5) {
            const double t = reduce_parts_n(part_w2, bb, lane, P);
            const double rn = reduce_parts_n(part_rw, bb, lane, P);
            if (lane == 0 && !sc[bb].conv) {
                TfqmrScal u = sc[bb];
                half_scalars(u, t);
                if (!u.conv) {
                    if (u.rho == 0.0) u.conv = 2;
                    else {
                        u.beta = rn / u.rho;
                        u.rho = rn;
                        refresh_coefs(u);
                    }
                }
                sc[bb] = u;
            }
        }
        if (threadIdx.x == 0) *ctr = 0u;
    }
};

// Ay1 = Z0 y1 (Eq. 12) and v = Ay1 + beta (Ay2 + beta v), then alpha and the
// loop test (see k_tfqmr_v)
template <typename V> struct EpiV {
    static constexpr bool kPlaneOnly = true;
    const V *y1;
    V *Ay1;
    const V *eps;
    V *v;
    const V *Ay2, *rs;
    TfqmrScal *sc;
    double *part;  // [B][P]
    int P;
    unsigned *ctr;
    int *ctl;
    cudaGraphConditionalHandle h;
    int use_h;
    int start;  // the solve's first product: v = Ay1, alpha from (r*, v), no loop test
    V dl = V(0);  // delta of Z0 + delta I
    struct Plane {
        const V *y1;
        V *Ay1;
        const V *eps;
        V *v;
        const V *Ay2, *rs;
        V be;
        int skip;
        typename AccOf<V>::type acc;
        int start;
        V dl = V(0);
        __device__ __forceinline__ void operator()(int i, V g) {
            const V e = eps[i];
            const V ay = (e * V(0.5) + dl) * y1[i] - (e - V(1)) * g;
            Ay1[i] = ay;
            if (skip) return;
            const V vn = start ? ay : ay + be * (Ay2[i] + be * v[i]);
            v[i] = vn;
            acc += rs[i] * vn;
        }
        template <int W> __device__ __forceinline__ void pack(int i, const V (&g)[W]) {
            V e[W], yv[W], ay[W];
            ldv<W>(e, eps + i);
            ldv<W>(yv, y1 + i);
#pragma unroll
            for (int k = 0; k < W; ++k) ay[k] = (e[k] * V(0.5) + dl) * yv[k] - (e[k] - V(1)) * g[k];
            stv<W>(Ay1 + i, ay);
            if (skip) return;
            V vv[W], rr[W];
            ldv<W>(rr, rs + i);
            if (start) {
#pragma unroll
                for (int k = 0; k < W; ++k) vv[k] = ay[k];
            } else {
                V a2[W];
                ldv<W>(a2, Ay2 + i);
                ldv<W>(vv, v + i);
#pragma unroll
                for (int k = 0; k < W; ++k) vv[k] = ay[k] + be * (a2[k] + be * vv[k]);
            }
#pragma unroll
            for (int k = 0; k < W; ++k) acc += rr[k] * vv[k];
            stv<W>(v + i, vv);
        }
    };
    __device__ __forceinline__ Plane bind(long plane, int Nz, int NyNx) const {
        const long off = plane * (long)NyNx, zoff = (plane % Nz) * (long)NyNx;
        const TfqmrScal s = sc[(int)(plane / P)];
        return Plane{y1 + off, Ay1 + off, eps + zoff, v + off, Ay2 + off, rs + off, Coefs<V>::be(s), s.conv != 0, 0, start,
                     dl};
    }
    __device__ __forceinline__ void finish(const Plane &pl, long plane) const {
        __shared__ int active;
        const typename AccOf<V>::type vals[1] = {pl.acc};
        double *const parts[1] = {part};
        if (!plane_block_done<1>(vals, parts, plane, ctr)) return;
        if (threadIdx.x == 0) active = 0;
        __syncthreads();
        const int lane = threadIdx.x & 31, B = (int)(gridDim.x / P);
        for (int bb = threadIdx.x >> 5; bb < B; bb += blockDim.x >> 5) {
            const double sigma = reduce_parts_n(part, bb, lane, P);
            if (lane == 0) {
                TfqmrScal u = sc[bb];
                if (!u.conv) {
                    if (sigma == 0.0) u.conv = 2;
                    else {
                        u.alpha = u.rho / sigma;
                        refresh_coefs(u);
                    }
                    sc[bb] = u;
                }
                if (u.conv == 0) active = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!start) {
                const int it = ctl[0] + 1;
                ctl[0] = it;
                const int cont = (active && it < ctl[1]) ? 1 : 0;
                if (use_h) cudaGraphSetConditional(h, (unsigned)cont);
                else ctl[2] = cont;
            }
            *ctr = 0u;
        }
    }
};

// end of an iteration: v = Ay1 + beta (Ay2 + beta v), sigma = (r*, v) ->
// alpha = rho / sigma for the next iteration (breakdown at sigma = 0), then the
// loop test: count the iteration in ctl[0] and continue while some right-hand
// side is active and ctl[0] < ctl[1] -- through the graph's conditional handle
// (use_h) or into ctl[2] for a host-driven loop.   grid (kRedBlocks, B)
template <typename V>
__global__ void __launch_bounds__(kRedThreads) k_tfqmr_v(V *__restrict__ v, const V *__restrict__ Ay1,
                                                         const V *__restrict__ Ay2, const V *__restrict__ rs,
                                                         TfqmrScal *__restrict__ sc, long L, double *__restrict__ part,
                                                         unsigned *ctr, int *ctl, cudaGraphConditionalHandle h,
                                                         int use_h) {
    using A = typename AccOf<V>::type;
    __shared__ double sh[32];
    __shared__ int active;
    const int b = blockIdx.y;
    A acc = A(0);
    if (!sc[b].conv) {
        const V be = Coefs<V>::be(sc[b]);
        const long o = (long)b * L;
        constexpr int W = PackW<V>::W;
        const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
        const long np = L % W == 0 ? L / W : 0;
#pragma unroll 2
        for (long j = t0; j < np; j += ts) {
            const long i = o + j * W;
            V a1[W], a2[W], vv[W], rr[W];
            ldv<W>(a1, Ay1 + i);
            ldv<W>(a2, Ay2 + i);
            ldv<W>(vv, v + i);
            ldv<W>(rr, rs + i);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                vv[k] = a1[k] + be * (a2[k] + be * vv[k]);
                acc += rr[k] * vv[k];
            }
            stv<W>(v + i, vv);
        }
        for (long i = np * W + t0; i < L; i += ts) {
            const V vn = Ay1[o + i] + be * (Ay2[o + i] + be * v[o + i]);
            v[o + i] = vn;
            acc += rs[o + i] * vn;
        }
    }
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) part[b * kRedBlocks + blockIdx.x] = bs;
    if (!last_block(ctr, gridDim.x * gridDim.y)) return;
    if (threadIdx.x == 0) active = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int bb = threadIdx.x >> 5; bb < (int)gridDim.y; bb += blockDim.x >> 5) {
        const double sigma = reduce_parts_lane(part, bb, lane);
        if (lane == 0) {
            TfqmrScal u = sc[bb];
            if (!u.conv) {
                if (sigma == 0.0) u.conv = 2;
                else {
                    u.alpha = u.rho / sigma;
                    refresh_coefs(u);
                }
                sc[bb] = u;
            }
            if (u.conv == 0) active = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = ctl[0] + 1;
        ctl[0] = it;
        const int cont = (active && it < ctl[1]) ? 1 : 0;
        if (use_h) cudaGraphSetConditional(h, (unsigned)cont);
        else ctl[2] = cont;
        *ctr = 0u;
    }
}

// apply the pending x += eta d of right-hand sides that converged (conv == 2)
// or that stop at the iteration cap (flush = 1)
template <typename V, typename VX>
__global__ void k_tfqmr_flush(VX *__restrict__ x, const V *__restrict__ d, TfqmrScal *__restrict__ sc, long L,
                              int flush_all) {
    const int b = blockIdx.y;
    const TfqmrScal s = sc[b];
    if (!s.pending || !(s.conv == 2 || flush_all)) return;
    const VX ep = (VX)s.eta_prev;
    const long o = (long)b * L;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        x[o + i] += ep * (VX)d[o + i];
}

// mark flushed right-hand sides
__global__ void k_tfqmr_settle(TfqmrScal *sc, int B, int flush_all) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B && sc[b].pending && (sc[b].conv == 2 || flush_all)) {
        sc[b].pending = 0;
        if (sc[b].conv == 2) sc[b].conv = 1;
    }
}

// ||v||^2 per right-hand side into out[b] (after k_dot_part). grid B, block 32
__global__ void k_finish_dot(const double *part, double *out) {
    double s = reduce_parts(part, blockIdx.x);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// ---- scaling of the FP32 correction solve ----
// The residual handed to the FP32 solve is scaled per right-hand side by 2^-e
// with 2^e ~ its 2-norm (exact: a power of two), so the FP32 vectors and their
// squared sums stay near 1 whatever the units of the problem; the correction
// is scaled back by 2^e when it is added to J.  n2 = squared norms ([B]).
__device__ __forceinline__ int pow2_exponent(double n2) {
    if (!(n2 > 0.0) || !isfinite(n2)) return 0;
    return ilogb(n2) / 2;
}

// 2^k as a double, built from its exponent field (|k| <= 1022; pow2_exponent's
// range, |k| <= 537, lies well inside): x * pow2d(k) is ldexp(x, k), rounded
// the same way where the result is subnormal
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// dst = 2^-e src in FP32 (e from ||src||^2 per right-hand side); 16-byte packs
// when L allows (vectors of L elements per right-hand side start 16-byte aligned)
__global__ void k_convert_scaled(float *__restrict__ dst, const double *__restrict__ src,
                                 const double *__restrict__ n2, long L) {
    const int b = blockIdx.y;
    const double sc = pow2d(-pow2_exponent(n2[b]));
    const long o = (long)b * L;
    const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
    if (L % 4 == 0) {
        for (long j = t0; j < L / 4; j += ts) {
            double v[4];
            float f[4];
            ldv<4>(v, src + o + 4 * j);
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] = (float)(v[k] * sc);
            stv<4>(dst + o + 4 * j, f);
        }
    } else {
        for (long i = t0; i < L; i += ts) dst[o + i] = (float)(src[o + i] * sc);
    }
}

// J += 2^e c (the correction of a refinement sweep; the product is exact, so the
// sum rounds once as with ldexp)
__global__ void k_add_scaled(double *__restrict__ J, const float *__restrict__ c, const double *__restrict__ n2,
                             long L) {
    const int b = blockIdx.y;
    const double sc = pow2d(pow2_exponent(n2[b]));
    const long o = (long)b * L;
    const long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x, ts = (long)gridDim.x * blockDim.x;
    if (L % 4 == 0) {
        for (long j = t0; j < L / 4; j += ts) {
            double v[4];
            float f[4];
            ldv<4>(v, J + o + 4 * j);
            ldv<4>(f, c + o + 4 * j);
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += (double)f[k] * sc;
            stv<4>(J + o + 4 * j, v);
        }
    } else {
        for (long i = t0; i < L; i += ts) J[o + i] += (double)c[o + i] * sc;
    }
}

// start of a solve from x0 = 0 in one kernel: w = y1 = r* = rhs, x = d = 0, the
// block partials of ||rhs||^2, and in the last block the scalar
// initialisation (tau = ||rhs||; b = 0 is done at once, x being 0).  rhs =
// src, or with n2 given 2^-e src (the scaled residual of the mixed form's
// correction solve, as k_convert_scaled forms it).  The partials are the
// ones k_dot_part forms (same grid, same order).  grid (kRedBlocks, B)
template <typename V, typename S>
__global__ void __launch_bounds__(kRedThreads) k_tfqmr_start_zero(const S *__restrict__ src,
                                                                  const double *__restrict__ n2, V *__restrict__ x,
                                                                  V *__restrict__ w, V *__restrict__ y1,
                                                                  V *__restrict__ rs, V *__restrict__ d, long L,
                                                                  double *__restrict__ part,
                                                                  TfqmrScal *__restrict__ sc, double tol, int stag,
                                                                  unsigned *ctr, InnerTol itol) {
    __shared__ double sh[32];
    const int b = blockIdx.y;
    const long o = (long)b * L;
    const double scl = n2 ? pow2d(-pow2_exponent(n2[b])) : 1.0;  // 2^-e: the product is k_convert_scaled's
    using A = typename AccOf<V>::type;
    A s = A(0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x) {
        const V v = n2 ? (V)((double)src[o + i] * scl) : (V)src[o + i];
        w[o + i] = v;
        y1[o + i] = v;
        rs[o + i] = v;
        x[o + i] = V(0);
        d[o + i] = V(0);
        s += (A)v * (A)v;
    }
    const double bs = block_sum(s, sh);
    if (threadIdx.x == 0) part[b * kRedBlocks + blockIdx.x] = bs;
    if (!last_block(ctr, gridDim.x * gridDim.y)) return;
    const int lane = threadIdx.x & 31, B = (int)gridDim.y;
    for (int bb = threadIdx.x >> 5; bb < B; bb += blockDim.x >> 5) {
        const double r2 = reduce_parts_lane(part, bb, lane);
        if (lane == 0) {
            TfqmrScal u = init_scalars(r2, r2, inner_tol_of(tol, itol, bb), stag);
            if (u.conv == 3) u.conv = 1;
            sc[bb] = u;
        }
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// ||v||^2 per right-hand side into out[b] in one kernel (the k_dot_part
// partials, then the k_finish_dot reduction in the last block).  grid (kRedBlocks, B)
__global__ void __launch_bounds__(kRedThreads) k_norm2(const double *__restrict__ v, long L,
                                                       double *__restrict__ part, double *__restrict__ out,
                                                       unsigned *ctr) {
    __shared__ double sh[32];
    const int b = blockIdx.y;
    const double *pv = v + (long)b * L;
    double s = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x)
        s += pv[i] * pv[i];
    const double bs = block_sum(s, sh);
    if (threadIdx.x == 0) part[b * kRedBlocks + blockIdx.x] = bs;
    if (!last_block(ctr, gridDim.x * gridDim.y)) return;
    const int lane = threadIdx.x & 31, B = (int)gridDim.y;
    for (int bb = threadIdx.x >> 5; bb < B; bb += blockDim.x >> 5) {
        const double t = reduce_parts_lane(part, bb, lane);
        if (lane == 0) out[bb] = t;
    }
    if (threadIdx.x == 0) *ctr = 0u;
}


// ---------------------------------------------------------------------------
// incident right-hand side (Eq. 7-8):
//   inc[b][m] = (eps_r(m) - 1) eps0 E0 < dg/dt (tau) >_m
//   g(tau) = exp(-tau^2 / (2 sigma^2)) cos(2 pi f0 tau) / (sigma sqrt(2 pi)),
//   tau = t - t0 - khat.(r - r_ref)/c0,
// voxel average by the 2x2x2 Gauss-Legendre rule.  The Cartesian direction
// pol[b] multiplies it in the right-hand-side epilogue.
// ---------------------------------------------------------------------------
struct PlaneWaveDev {
    double E0, sigma, t0, f0;
    double khat[3];
    double pol[3];
    double rref[3];
    // factorisation of the 2x2x2 Gauss average: the point offsets are
    // +-a (a = h/(2 sqrt 3)) per axis, so tau = tau_c - delta(s) with
    // delta(s) = sum_i s_i beta_i, beta_i = khat_i a / c0, and
    //   E(tau_c - delta) = E(tau_c) prod_i exp(s_i beta_i tau_c / sigma^2) C(s),
    //   E(tau) = exp(-tau^2/(2 sigma^2) + i w tau), C(s) = exp(-delta^2/(2 sigma^2) - i w delta).
    double beta[3];
    double Cre[8], Cim[8], delta[8];
    // FP32 copies for the fast path: delta(s)/sigma, C(s), beta_i/sigma, w sigma,
    // and the FP64 scale eps0 (1/(sigma sqrt(2 pi))) E0 (1/8) / sigma
    float delta_over_sigma[8];
    float f_Cre[8], f_Cim[8];
    float f_beta_over_sigma[3];
    float f_w_sigma;
    double fast_scale;
};

// host: fill beta, C(s), delta(s) of a plane wave for voxel size h
inline void planewave_factors(PlaneWaveDev &P, double h) {
    const double c0 = 299792458.0;
    const double a = h / (2.0 * 1.7320508075688772935);
    const double w = 2.0 * 3.141592653589793238462643 * P.f0;
    for (int i = 0; i < 3; ++i) P.beta[i] = P.khat[i] * a / c0;
    for (int q = 0; q < 8; ++q) {
        double d = 0.0;
        for (int i = 0; i < 3; ++i) d += ((q >> i) & 1 ? 1.0 : -1.0) * P.beta[i];
        double mag = exp(-0.5 * d * d / (P.sigma * P.sigma));
        P.Cre[q] = mag * cos(w * d);
        P.Cim[q] = -mag * sin(w * d);
        P.delta[q] = d;
        P.delta_over_sigma[q] = (float)(d / P.sigma);
        P.f_Cre[q] = (float)P.Cre[q];
        P.f_Cim[q] = (float)P.Cim[q];
    }
    for (int i = 0; i < 3; ++i) P.f_beta_over_sigma[i] = (float)(P.beta[i] / P.sigma);
    P.f_w_sigma = (float)(w * P.sigma);
    const double eps0 = 8.8541878128e-12;
    P.fast_scale = eps0 * P.E0 / (P.sigma * 2.5066282746310005024) * 0.125 / P.sigma;
}

// Per-axis tables of the fast incident path, per plane wave b (S = Nx+Ny+Nz
// entries, x then y then z): time offsets s_i(m) = -khat_i ((m + 1/2) h -
// rref_i) / c0 in FP64 and FP32, and phase factors exp(i w s_i(m)) in FP32, so
// that tau_c = (t - t0) + s_x + s_y + s_z and exp(i w tau_c) is a product of
// table entries.  Layout: ts[B][S] doubles, tsf[B][S] floats, ph[B][S] float2.
inline void incident_tables(const PlaneWaveDev &P, const int N[3], double h, double *ts, float *tsf, float2 *ph) {
    const double c0 = 299792458.0, w = 2.0 * 3.141592653589793238462643 * P.f0;
    int o = 0;
    for (int i = 0; i < 3; ++i)
        for (int m = 0; m < N[i]; ++m, ++o) {
            const double sv = -P.khat[i] * ((m + 0.5) * h - P.rref[i]) / c0;
            ts[o] = sv;
            tsf[o] = (float)sv;
            ph[o] = make_float2((float)cos(w * sv), (float)sin(w * sv));
        }
}

// fast incident right-hand side (mixed-precision path): one block row per
// (z, y) line of plane wave blockIdx.y; the FP64 work is the line's time
// (t - t0) + s_y + s_z and exp(i w (t - t0)) once per block; per voxel only
// FP32.  inc as k_incident (FP64 storage).
__global__ void k_incident_rows(double *__restrict__ inc, const float *__restrict__ eps32,
                                const PlaneWaveDev *__restrict__ pw, const double *__restrict__ ts,
                                const float *__restrict__ tsf, const float2 *__restrict__ ph, int Nx, int Ny, int Nz,
                                double t, const long long *__restrict__ nptr, double dt) {
    if (nptr) t = (double)(*nptr) * dt;
    const int b = blockIdx.y, S = Nx + Ny + Nz;
    const PlaneWaveDev &P = pw[b];
    const double *sy = ts + (long)b * S + Nx, *sz = sy + Ny;
    const float *sxf = tsf + (long)b * S;
    const float2 *px = ph + (long)b * S, *py = px + Nx, *pz = py + Ny;
    const double T = t - P.t0;
    __shared__ float2 pt;
    if (threadIdx.x == 0) {
        double sn, cs;
        sincos(2.0 * 3.141592653589793238462643 * P.f0 * T, &sn, &cs);
        pt = make_float2((float)cs, (float)sn);
    }
    __syncthreads();
    const float is = (float)(1.0 / P.sigma), ws = P.f_w_sigma;
    const long nv = (long)Nx * Ny * Nz;
    for (int row = blockIdx.x; row < Ny * Nz; row += gridDim.x) {
        const int z = row / Ny, y = row - z * Ny;
        const float trow = (float)(T + sy[y] + sz[z]);
        const float2 a = py[y], c = pz[z];
        const float2 yz = make_float2(a.x * c.x - a.y * c.y, a.x * c.y + a.y * c.x);
        const float2 pr = make_float2(pt.x * yz.x - pt.y * yz.y, pt.x * yz.y + pt.y * yz.x);
        for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
            const long m = (long)row * Nx + x;
            const float e = eps32[m];
            double out = 0.0;
            if (e != 1.f) {
                const float tcs = (trow + sxf[x]) * is;  // tau_c / sigma
                const float2 q = px[x];
                const float g = expf(-0.5f * tcs * tcs);
                const float Er = g * (pr.x * q.x - pr.y * q.y), Ei = g * (pr.x * q.y + pr.y * q.x);
                const float a0 = P.f_beta_over_sigma[0] * tcs, a1 = P.f_beta_over_sigma[1] * tcs,
                            a2 = P.f_beta_over_sigma[2] * tcs;
                const float u0 = expf(a0), u1 = expf(a1), u2 = expf(a2);
                const float v0 = 1.f / u0, v1 = 1.f / u1, v2 = 1.f / u2;
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float f = ((k & 1) ? u0 : v0) * ((k & 2) ? u1 : v1) * ((k & 4) ? u2 : v2);
                    const float zr = f * (Er * P.f_Cre[k] - Ei * P.f_Cim[k]);
                    const float zi = f * (Er * P.f_Cim[k] + Ei * P.f_Cre[k]);
                    acc += -(tcs - P.delta_over_sigma[k]) * zr - ws * zi;
                }
                out = (double)((e - 1.f) * acc) * P.fast_scale;
            }
            inc[(long)b * nv + m] = out;
        }
    }
}

// inc[b][m] = (eps_r(m) - 1) eps0 E0 (1/8) sum_s g'(tau_c - delta(s)),
// g'(tau) = Re[(-tau/sigma^2 + i w) E(tau)] / (sigma sqrt(2 pi)), all FP64
// (the FP64 path; k_incident_rows is the mixed path's FP32 form).
// nptr (graph mode): t = (*nptr) * dt instead of the argument t
__global__ void k_incident(double *__restrict__ inc, const double *__restrict__ eps,
                           const PlaneWaveDev *__restrict__ pw, int Nx, int Ny, int Nz, double h, double t,
                           int nrhs, const long long *__restrict__ nptr, double dt) {
    if (nptr) t = (double)(*nptr) * dt;
    const long n = (long)Nx * Ny * Nz;
    const double c0 = 299792458.0, eps0 = 8.8541878128e-12;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n * nrhs; i += (long)gridDim.x * blockDim.x) {
        long b = i / n, m = i - b * n;
        double ep = eps[m];
        if (ep == 1.0) { inc[i] = 0.0; continue; }
        int mx = (int)(m % Nx), my = (int)((m / Nx) % Ny), mz = (int)(m / ((long)Nx * Ny));
        const PlaneWaveDev &P = pw[b];
        const double w = 2.0 * 3.141592653589793238462643 * P.f0;
        const double amp = P.E0 / (P.sigma * 2.5066282746310005024);  // sigma sqrt(2 pi)
        const double is2 = 1.0 / (P.sigma * P.sigma);
        double rx = (mx + 0.5) * h - P.rref[0], ry = (my + 0.5) * h - P.rref[1], rz = (mz + 0.5) * h - P.rref[2];
        double tc = t - P.t0 - (P.khat[0] * rx + P.khat[1] * ry + P.khat[2] * rz) / c0;
        double acc;
        {
            double s, c;
            sincos(w * tc, &s, &c);
            double g = exp(-0.5 * tc * tc * is2);
            double u0 = exp(P.beta[0] * tc * is2), u1 = exp(P.beta[1] * tc * is2), u2 = exp(P.beta[2] * tc * is2);
            double v0 = 1.0 / u0, v1 = 1.0 / u1, v2 = 1.0 / u2;
            double Er = g * c, Ei = g * s;
            acc = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                double f = ((q & 1) ? u0 : v0) * ((q & 2) ? u1 : v1) * ((q & 4) ? u2 : v2);
                double zr = f * (Er * P.Cre[q] - Ei * P.Cim[q]);
                double zi = f * (Er * P.Cim[q] + Ei * P.Cre[q]);
                double tau = tc - P.delta[q];
                acc += -tau * is2 * zr - w * zi;  // Re[(-tau/sigma^2 + i w)(zr + i zi)]
            }
        }
        inc[i] = (ep - 1.0) * eps0 * amp * 0.125 * acc;
    }
}

}  // namespace mot
