// peak.cuh -- FMA throughput microkernel (instrumentation for the roofline of
// the FP64 and FP32 product paths; no counterpart in the paper).
//
// Every thread runs kChains independent FMA chains of `iters` steps each, so
// the FMA pipe is never waiting on a dependency; the chains' sum is stored so
// that nothing is dead code.  The grid is a whole multiple of the SM count with
// several resident blocks per SM.  FLOP/s = 2 * FMAs / elapsed (CUDA events).
#pragma once

#include "common.cuh"

namespace mot {

constexpr int kPeakChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *__restrict__ out, int iters, T a, T b) {
    T c[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) c[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) c[j] = fma(c[j], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += c[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mot
