// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipe, for
// the FP64-accuracy Z0 product on a GPU whose FP64 rate is a small fraction of
// its FP32 rate.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| at most
// half an ulp of hi: about 48 significant bits.  The building blocks are the
// error-free transformations
//   TwoSum   (Knuth, TAOCP vol. 2, 4.2.2):  s + e = a + b exactly, no ordering condition;
//   Fast2Sum (Dekker 1971):                 the same when |a| >= |b|;
//   TwoProd  (through the FMA):             p + e = a * b exactly;
// and the double-word sum and product built from them as analysed by Joldes,
// Muller and Popescu ("Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44, 2017):
//   add: TwoSum of the high parts, the low parts added to the error term,
//        Fast2Sum to renormalise (their "sloppy" sum: absolute error below
//        about 2^-47 (|a| + |b|), which is the norm-wise bound an FFT needs);
//   mul: TwoProd of the high parts, both cross products folded into the error
//        term by FMA, Fast2Sum (relative error below about 2^-46.6).
// Every step uses the round-to-nearest intrinsics (__fadd_rn, __fmul_rn,
// __fmaf_rn), which the compiler neither contracts nor reorders.
//
// The exponent range is FP32's: values must stay within about 1e-30 .. 1e38 in
// magnitude for the low part to keep its 24 bits (the solver vectors of the MOT
// scale with the incident field, far inside that range).
#pragma once

#include <cuda_runtime.h>

namespace mot {

struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    // exact for values representable in 48 bits; rounds otherwise.  Folded at
    // compile time for constant arguments.
    __host__ __device__ constexpr dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

namespace dfop {
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
}  // namespace dfop

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    float s, e, h, l;
    dfop::two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    dfop::fast_two_sum(s, e, h, l);
    return dfl(h, l);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float h, l;
    dfop::fast_two_sum(p, e, h, l);
    return dfl(h, l);
}
// the accurate double-word sum (their Algorithm 6: both pairs through TwoSum,
// two renormalisations): relative error below about 2^-46 even under
// cancellation, for long accumulations whose terms differ in sign
__device__ __forceinline__ dfl add_accurate(dfl a, dfl b) {
    float sh, sl, th, tl, vh, vl, zh, zl;
    dfop::two_sum(a.hi, b.hi, sh, sl);
    dfop::two_sum(a.lo, b.lo, th, tl);
    dfop::fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
    dfop::fast_two_sum(vh, __fadd_rn(tl, vl), zh, zl);
    return dfl(zh, zl);
}
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl &operator*=(dfl &a, dfl b) { return a = a * b; }

// FP64 <-> double-float on the device (one FP64 subtraction and three
// conversions in, two conversions and one FP64 addition out)
__device__ __forceinline__ dfl to_dfl(double d) {
    const float h = __double2float_rn(d);
    return dfl(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double to_double(dfl a) { return (double)a.hi + (double)a.lo; }

struct __align__(16) dfl2 {  // complex double-float, the layout of double2 (16-byte packs)
    dfl x, y;
};

}  // namespace mot
