// common.cuh -- shared types and helpers of the libmotjvie CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "dfloat.cuh"

#ifndef MOT_HD
#define MOT_HD __host__ __device__
#endif

namespace mot {

// complex helpers on float2 / double2 / dfl2
template <typename T> struct cx;
template <> struct cx<float> { using type = float2; };
template <> struct cx<double> { using type = double2; };
template <> struct cx<dfl> { using type = dfl2; };  // double-float (FP32 pair) complex
template <typename T> using cplx = typename cx<T>::type;

template <typename C> MOT_HD inline C cmake(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> MOT_HD inline C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> MOT_HD inline C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> MOT_HD inline C cmul(C a, C b) { return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> MOT_HD inline C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }
template <typename C> MOT_HD inline C cconj(C a) { return cmake<C>(a.x, -a.y); }
// multiply by i (sign +1) or -i (sign -1)
template <int S, typename C> MOT_HD inline C cmuli(C a) { return S > 0 ? cmake<C>(-a.y, a.x) : cmake<C>(a.y, -a.x); }

// W consecutive elements moved with 16-byte accesses; p must be 16-byte
// aligned and W * sizeof(E) a multiple of 16
template <int W, typename E> __device__ __forceinline__ void ldv(E (&r)[W], const E *p) {
    static_assert((W * sizeof(E)) % 16 == 0, "whole 16-byte accesses");
#pragma unroll
    for (int k = 0; k < (int)(W * sizeof(E) / 16); ++k) {
        const uint4 u = reinterpret_cast<const uint4 *>(p)[k];
        memcpy(reinterpret_cast<char *>(r) + 16 * k, &u, 16);
    }
}
template <int W, typename E> __device__ __forceinline__ void stv(E *p, const E (&r)[W]) {
    static_assert((W * sizeof(E)) % 16 == 0, "whole 16-byte accesses");
#pragma unroll
    for (int k = 0; k < (int)(W * sizeof(E) / 16); ++k) {
        uint4 u;
        memcpy(&u, reinterpret_cast<const char *>(r) + 16 * k, 16);
        reinterpret_cast<uint4 *>(p)[k] = u;
    }
}

// thread-local error message + status helpers (host side)
void set_error(const std::string &msg);
const char *get_error();

}  // namespace mot

#define MOT_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            ::mot::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));           \
            return MOT_ECUDA;                                                               \
        }                                                                                   \
    } while (0)
