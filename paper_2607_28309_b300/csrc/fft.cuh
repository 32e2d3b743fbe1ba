// fft.cuh -- shared-memory mixed-radix (2, 3, 4, 5) Stockham FFT for batches of
// pencils, the building block of the zero-padded 3-D transforms of Eq. 11.
//
// A CTA holds `nb` pencils of length M in shared memory at addresses
// base + p*ps + e*es (pencil p, element e) and transforms all of them in place
// by ping-ponging through a second buffer of the same shape.  Each stage of
// radix R does M/R butterflies per pencil: load R strided inputs, apply the
// twiddles W^(r k M/(Ns R)) (W = exp(-+2 pi i / M), k = j mod Ns), an R-point DFT
// in registers, and store at the Stockham positions (j/Ns) Ns R + k + r Ns, so
// the result comes out in natural order.  Twiddles come from a table of the M
// roots exp(-2 pi i m / M) staged in shared memory.
#pragma once

#include "common.cuh"

namespace mot {

constexpr int kMaxStages = 12;

struct FftPlan {
    int M;
    int nstage;
    int radix[kMaxStages];
};

// host: split M into radices 4, 2 (at most one), 3, 5; returns false if M has
// another prime factor
inline bool make_plan(int M, FftPlan *pl) {
    pl->M = M;
    pl->nstage = 0;
    int m = M;
    while (m % 4 == 0) { pl->radix[pl->nstage++] = 4; m /= 4; }
    while (m % 2 == 0) { pl->radix[pl->nstage++] = 2; m /= 2; }
    while (m % 3 == 0) { pl->radix[pl->nstage++] = 3; m /= 3; }
    while (m % 5 == 0) { pl->radix[pl->nstage++] = 5; m /= 5; }
    return m == 1 && pl->nstage <= kMaxStages;
}

// smallest size >= n whose prime factors are 2, 3 and 5
inline int smooth235(int n) {
    for (int m = n > 1 ? n : 1;; ++m) {
        int k = m;
        while (k % 2 == 0) k /= 2;
        while (k % 3 == 0) k /= 3;
        while (k % 5 == 0) k /= 5;
        if (k == 1) return m;
    }
}

// R-point DFTs with exponent sign S (-1 forward, +1 inverse)
template <int S, typename C> __device__ __forceinline__ void dft2(C *v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int S, typename C> __device__ __forceinline__ void dft3(C *v) {
    using T = decltype(C::x);
    const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
    C t1 = cadd(v[1], v[2]);
    C t2 = cscale(cmuli<S>(csub(v[1], v[2])), h);
    C m = csub(v[0], cscale(t1, T(0.5)));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, t2);
    v[2] = csub(m, t2);
}

template <int S, typename C> __device__ __forceinline__ void dft4(C *v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmuli<S>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
}

template <int S, typename C> __device__ __forceinline__ void dft5(C *v) {
    using T = decltype(C::x);
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos 2pi/5, cos 4pi/5
    const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin 2pi/5, sin 4pi/5
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C b1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
    C b2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
    C d1 = cmuli<S>(cadd(cscale(t3, s1), cscale(t4, s2)));
    C d2 = cmuli<S>(csub(cscale(t3, s2), cscale(t4, s1)));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(b1, d1);
    v[4] = csub(b1, d1);
    v[2] = cadd(b2, d2);
    v[3] = csub(b2, d2);
}

// one Stockham stage over nb pencils; src/dst share the (ps, es) layout.
// When batch_fast is set consecutive threads walk consecutive pencils (good
// for column pencils with ps = 1), else consecutive butterflies of a pencil.
template <int S, int R, typename C>
__device__ __forceinline__ void fft_stage(const C *__restrict__ src, C *__restrict__ dst, int M, int Ns,
                                          int nb, int ps, int es, const C *__restrict__ tw, bool batch_fast) {
    const int nbf = M / R;  // butterflies per pencil
    const int total = nb * nbf;
    const int tstep = M / (Ns * R);
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int p, j;
        if (batch_fast) { p = it % nb; j = it / nb; }
        else { j = it % nbf; p = it / nbf; }
        const int k = j % Ns;
        const C *s = src + p * ps;
        C *d = dst + p * ps;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * nbf) * es];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * k * tstep];
                if (S > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 2) dft2<S>(v);
        if (R == 3) dft3<S>(v);
        if (R == 4) dft4<S>(v);
        if (R == 5) dft5<S>(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(base + r * Ns) * es] = v[r];
    }
}

// full transform; data starts in `a`, `b` is scratch of the same shape.
// Returns the buffer holding the result (a or b).
template <int S, typename C>
__device__ C *block_fft(C *a, C *b, const FftPlan &pl, int nb, int ps, int es, const C *tw, bool batch_fast) {
    int Ns = 1;
    for (int s = 0; s < pl.nstage; ++s) {
        const int R = pl.radix[s];
        switch (R) {
            case 2: fft_stage<S, 2>(a, b, pl.M, Ns, nb, ps, es, tw, batch_fast); break;
            case 3: fft_stage<S, 3>(a, b, pl.M, Ns, nb, ps, es, tw, batch_fast); break;
            case 4: fft_stage<S, 4>(a, b, pl.M, Ns, nb, ps, es, tw, batch_fast); break;
            default: fft_stage<S, 5>(a, b, pl.M, Ns, nb, ps, es, tw, batch_fast); break;
        }
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// stage the M-root twiddle table (global -> shared)
template <typename C> __device__ __forceinline__ void load_twiddles(C *dst, const C *src, int M) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) dst[i] = src[i];
}

}  // namespace mot
