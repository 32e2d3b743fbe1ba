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

// division by a runtime constant d for dividends below 2^24:
// q = (x * m) >> s with s = 24 + ceil(log2 d), m = ceil(2^s / d)  (Granlund-Montgomery)
struct FastDiv {
    unsigned int m;
    int s;
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned int d) {
    int l = 0;
    while ((1u << l) < d) ++l;
    FastDiv f;
    f.s = 24 + l;
    f.m = (unsigned int)(((1ull << f.s) + d - 1) / d);
    return f;
}
__host__ __device__ __forceinline__ unsigned int fdiv(unsigned int x, FastDiv f) {
    return (unsigned int)(((unsigned long long)x * f.m) >> f.s);
}

// where a plane staged into shared memory puts element i: row pairs of rp = 2 Nx
// elements, each followed by pad elements (pad 0: contiguous).  The padding
// moves consecutive pencils (row pairs) of the x pass onto different banks.
struct StageMap {
    FastDiv frp;
    int pad;
    __device__ __forceinline__ int operator()(int i) const { return pad ? i + (int)fdiv((unsigned)i, frp) * pad : i; }
};

struct FftPlan {
    int M;
    int nstage;
    int radix[kMaxStages];
    FastDiv ns_div[kMaxStages];   // division by Ns (product of earlier radices)
    FastDiv nbf_div[kMaxStages];  // division by M / radix
};

// host: split M into radices (16 when max_radix allows, then 9, 8, 4, 2, 3,
// 5: fewer, register-resident stages); false if M has another prime factor
inline bool make_plan(int M, FftPlan *pl, int max_radix = 16) {
    pl->M = M;
    pl->nstage = 0;
    int m = M;
    if (max_radix >= 16)
        while (m % 16 == 0) { pl->radix[pl->nstage++] = 16; m /= 16; }
    if (max_radix >= 9)
        while (m % 9 == 0) { pl->radix[pl->nstage++] = 9; m /= 9; }
    if (max_radix >= 8)
        while (m % 8 == 0) { pl->radix[pl->nstage++] = 8; m /= 8; }
    while (m % 4 == 0) { pl->radix[pl->nstage++] = 4; m /= 4; }
    while (m % 2 == 0) { pl->radix[pl->nstage++] = 2; m /= 2; }
    while (m % 3 == 0) { pl->radix[pl->nstage++] = 3; m /= 3; }
    while (m % 5 == 0) { pl->radix[pl->nstage++] = 5; m /= 5; }
    int ns = 1;
    for (int s = 0; s < pl->nstage; ++s) {
        pl->ns_div[s] = make_fastdiv((unsigned)ns);
        pl->nbf_div[s] = make_fastdiv((unsigned)(M / pl->radix[s]));
        ns *= pl->radix[s];
    }
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

// cos / sin of 2 pi j / N for the register-resident composite radices
template <int N> struct Root;
template <> struct Root<8> {
    static constexpr double h = 0.70710678118654752440;  // cos(pi/4)
    __host__ __device__ static constexpr double c(int j) {
        return (j & 7) == 0 ? 1.0 : (j & 7) == 1 ? h : (j & 7) == 2 ? 0.0 : (j & 7) == 3 ? -h
             : (j & 7) == 4 ? -1.0 : (j & 7) == 5 ? -h : (j & 7) == 6 ? 0.0 : h;
    }
    __host__ __device__ static constexpr double s(int j) { return c(j + 6); }  // sin x = cos(x - pi/2)
};
template <> struct Root<16> {
    static constexpr double a = 0.92387953251128675613, b = 0.38268343236508977173, h = 0.70710678118654752440;
    __host__ __device__ static constexpr double c(int j) {
        return (j & 15) == 0 ? 1.0 : (j & 15) == 1 ? a : (j & 15) == 2 ? h : (j & 15) == 3 ? b
             : (j & 15) == 4 ? 0.0 : (j & 15) == 5 ? -b : (j & 15) == 6 ? -h : (j & 15) == 7 ? -a
             : (j & 15) == 8 ? -1.0 : (j & 15) == 9 ? -a : (j & 15) == 10 ? -h : (j & 15) == 11 ? -b
             : (j & 15) == 12 ? 0.0 : (j & 15) == 13 ? b : (j & 15) == 14 ? h : a;
    }
    __host__ __device__ static constexpr double s(int j) { return c(j + 12); }
};
template <> struct Root<9> {
    // cos / sin of 2 pi j / 9, j = 0..8
    static constexpr double c1 = 0.76604444311897803520, s1 = 0.64278760968653932632;
    static constexpr double c2 = 0.17364817766693034885, s2 = 0.98480775301220805936;
    static constexpr double c3 = -0.5, s3 = 0.86602540378443864676;
    static constexpr double c4 = -0.93969262078590838405, s4 = 0.34202014332566873304;
    __host__ __device__ static constexpr double c(int j) {
        return (j % 9) == 0 ? 1.0 : (j % 9) == 1 ? c1 : (j % 9) == 2 ? c2 : (j % 9) == 3 ? c3 : (j % 9) == 4 ? c4
             : (j % 9) == 5 ? c4 : (j % 9) == 6 ? c3 : (j % 9) == 7 ? c2 : c1;
    }
    __host__ __device__ static constexpr double s(int j) {
        return (j % 9) == 0 ? 0.0 : (j % 9) == 1 ? s1 : (j % 9) == 2 ? s2 : (j % 9) == 3 ? s3 : (j % 9) == 4 ? s4
             : (j % 9) == 5 ? -s4 : (j % 9) == 6 ? -s3 : (j % 9) == 7 ? -s2 : -s1;
    }
};

template <> struct Root<10> {
    // cos / sin of 2 pi j / 10 for j = 0..5; the rest by j -> 10 - j symmetry
    __host__ __device__ static constexpr double ch(int k) { return k == 0 ? 1.000000000000000000000 : k == 1 ? 0.8090169943749474241023 : k == 2 ? 0.3090169943749474241023 : k == 3 ? -0.3090169943749474241023 : k == 4 ? -0.8090169943749474241023 : -1.000000000000000000000; }
    __host__ __device__ static constexpr double sh(int k) { return k == 0 ? 0.0 : k == 1 ? 0.5877852522924731291687 : k == 2 ? 0.9510565162951535721164 : k == 3 ? 0.9510565162951535721164 : k == 4 ? 0.5877852522924731291687 : 0.0; }
    __host__ __device__ static constexpr double c(int j) { return ch((j % 10) <= 5 ? j % 10 : 10 - j % 10); }
    __host__ __device__ static constexpr double s(int j) { return (j % 10) <= 5 ? sh(j % 10) : -sh(10 - j % 10); }
};
template <> struct Root<15> {
    // cos / sin of 2 pi j / 15 for j = 0..7; the rest by j -> 15 - j symmetry
    __host__ __device__ static constexpr double ch(int k) { return k == 0 ? 1.000000000000000000000 : k == 1 ? 0.9135454576426008955021 : k == 2 ? 0.6691306063588582138263 : k == 3 ? 0.3090169943749474241023 : k == 4 ? -0.1045284632676534713998 : k == 5 ? -0.5000000000000000000000 : k == 6 ? -0.8090169943749474241023 : -0.9781476007338056379286; }
    __host__ __device__ static constexpr double sh(int k) { return k == 0 ? 0.0 : k == 1 ? 0.4067366430758002077540 : k == 2 ? 0.7431448254773942350147 : k == 3 ? 0.9510565162951535721164 : k == 4 ? 0.9945218953682733369227 : k == 5 ? 0.8660254037844386467637 : k == 6 ? 0.5877852522924731291687 : 0.2079116908177593371017; }
    __host__ __device__ static constexpr double c(int j) { return ch((j % 15) <= 7 ? j % 15 : 15 - j % 15); }
    __host__ __device__ static constexpr double s(int j) { return (j % 15) <= 7 ? sh(j % 15) : -sh(15 - j % 15); }
};
template <> struct Root<18> {
    // cos / sin of 2 pi j / 18 for j = 0..9; the rest by j -> 18 - j symmetry
    __host__ __device__ static constexpr double ch(int k) { return k == 0 ? 1.000000000000000000000 : k == 1 ? 0.9396926207859083840541 : k == 2 ? 0.7660444431189780352024 : k == 3 ? 0.5000000000000000000000 : k == 4 ? 0.1736481776669303488517 : k == 5 ? -0.1736481776669303488517 : k == 6 ? -0.5000000000000000000000 : k == 7 ? -0.7660444431189780352024 : k == 8 ? -0.9396926207859083840541 : -1.000000000000000000000; }
    __host__ __device__ static constexpr double sh(int k) { return k == 0 ? 0.0 : k == 1 ? 0.3420201433256687330441 : k == 2 ? 0.6427876096865393263226 : k == 3 ? 0.8660254037844386467637 : k == 4 ? 0.9848077530122080593667 : k == 5 ? 0.9848077530122080593667 : k == 6 ? 0.8660254037844386467637 : k == 7 ? 0.6427876096865393263226 : k == 8 ? 0.3420201433256687330441 : 0.0; }
    __host__ __device__ static constexpr double c(int j) { return ch((j % 18) <= 9 ? j % 18 : 18 - j % 18); }
    __host__ __device__ static constexpr double s(int j) { return (j % 18) <= 9 ? sh(j % 18) : -sh(18 - j % 18); }
};

template <> struct Root<32> {
    // cos(k pi / 16), k = 0..8; the rest of the circle by symmetry
    __host__ __device__ static constexpr double q(int k) {
        return k == 0 ? 1.0 : k == 1 ? 0.9807852804032304491262 : k == 2 ? 0.9238795325112867561282
             : k == 3 ? 0.8314696123025452370788 : k == 4 ? 0.7071067811865475244008
             : k == 5 ? 0.5555702330196022247428 : k == 6 ? 0.3826834323650897717285
             : k == 7 ? 0.1950903220161282678483 : 0.0;
    }
    __host__ __device__ static constexpr double c(int j) {
        return (j & 31) <= 8 ? q(j & 31) : (j & 31) <= 16 ? -q(16 - (j & 31))
             : (j & 31) <= 24 ? -q((j & 31) - 16) : q(32 - (j & 31));
    }
    __host__ __device__ static constexpr double s(int j) { return c(j + 24); }  // sin x = cos(x - pi/2)
};

template <int N, int S, typename C> __device__ __forceinline__ void dft_small(C *v);

// N1 x N2 Cooley-Tukey in registers: x[t + N2 m] -> DFT_N1 over m, twiddle
// W_N^(t k1), DFT_N2 over t -> X[k1 + N1 k2]; all indices compile-time
template <int N1, int N2, int S, typename C> __device__ __forceinline__ void dft_nested(C *v) {
    using T = decltype(C::x);
    constexpr int N = N1 * N2;
    C a[N];
#pragma unroll
    for (int t = 0; t < N2; ++t) {
        C col[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) col[m] = v[t + N2 * m];
        dft_small<N1, S>(col);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            C x = col[k1];
            if ((t * k1) % N != 0) {
                const T c = T(Root<N>::c((t * k1) % N)), s = T(S * Root<N>::s((t * k1) % N));
                x = cmake<C>(x.x * c - x.y * s, x.x * s + x.y * c);
            }
            a[t + N2 * k1] = x;
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        C row[N2];
#pragma unroll
        for (int t = 0; t < N2; ++t) row[t] = a[t + N2 * k1];
        dft_small<N2, S>(row);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k1 + N1 * k2] = row[k2];
    }
}

template <int N, int S, typename C> __device__ __forceinline__ void dft_small(C *v) {
    if constexpr (N == 1) return;
    else if constexpr (N == 2) dft2<S>(v);
    else if constexpr (N == 3) dft3<S>(v);
    else if constexpr (N == 4) dft4<S>(v);
    else if constexpr (N == 5) dft5<S>(v);
    else if constexpr (N == 8) dft_nested<4, 2, S>(v);
    else if constexpr (N == 9) dft_nested<3, 3, S>(v);
    else if constexpr (N == 10) dft_nested<5, 2, S>(v);
    else if constexpr (N == 15) dft_nested<5, 3, S>(v);
    else if constexpr (N == 16) dft_nested<4, 4, S>(v);
    else if constexpr (N == 18) dft_nested<9, 2, S>(v);
    else if constexpr (N == 32) dft_nested<8, 4, S>(v);
    else static_assert(N == 1, "no register DFT of this length");
}

// one Stockham stage over nb pencils; src/dst share the (ps, es) layout.
// When batch_fast is set consecutive threads walk consecutive pencils (good
// for column pencils with ps = 1), else consecutive butterflies of a pencil.
template <int S, int R, typename C>
__device__ __forceinline__ void fft_stage(const C *__restrict__ src, C *__restrict__ dst, int M, int Ns,
                                          FastDiv fns, FastDiv fnbf, int nb, FastDiv fnb, int ps, int es,
                                          const C *__restrict__ tw, bool batch_fast) {
    const int nbf = M / R;  // butterflies per pencil
    const int total = nb * nbf;
    const int tstep = M / (Ns * R);
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int p, j;
        if (batch_fast) { j = (int)fdiv((unsigned)it, fnb); p = it - j * nb; }
        else { p = (int)fdiv((unsigned)it, fnbf); j = it - p * nbf; }
        const int jh = (int)fdiv((unsigned)j, fns);
        const int k = j - jh * Ns;
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
        dft_small<R, S>(v);
        const int base = jh * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(base + r * Ns) * es] = v[r];
    }
}

// full transform; data starts in `a`, `b` is scratch of the same shape.
// Returns the buffer holding the result (a or b).
template <int S, typename C>
__device__ C *block_fft(C *a, C *b, const FftPlan &pl, int nb, int ps, int es, const C *tw, bool batch_fast) {
    int Ns = 1;
    const FastDiv fnb = make_fastdiv((unsigned)nb);
    for (int s = 0; s < pl.nstage; ++s) {
        const int R = pl.radix[s];
        const FastDiv fns = pl.ns_div[s], fnbf = pl.nbf_div[s];
        switch (R) {
            case 2: fft_stage<S, 2>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            case 3: fft_stage<S, 3>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            case 4: fft_stage<S, 4>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            case 5: fft_stage<S, 5>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            case 8: fft_stage<S, 8>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            case 9: fft_stage<S, 9>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
            default: fft_stage<S, 16>(a, b, pl.M, Ns, fns, fnbf, nb, fnb, ps, es, tw, batch_fast); break;
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

// programmatic dependent launch (the chain kernels of a Z0 product): a block
// lets the next kernel of the stream start launching once its main work is
// done (the next kernel's blocks then take the SMs this kernel's tail leaves
// idle), and waits for the previous kernel's completion (and its memory) before
// touching anything that kernel writes.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void chain_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void chain_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace mot
