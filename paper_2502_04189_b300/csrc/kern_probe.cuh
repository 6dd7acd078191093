// Arithmetic-throughput probe (measurement support, not part of the
// projection): the FP64 and FP32 fused multiply-add issue rates of the GPU,
// measured the way the FP64-bound projection kernels use the pipe.
//
// Every thread runs PROBE_CHAINS independent FMA chains x <- x a + b for
// `iters` rounds (a slightly below 1, so the values stay bounded); the chains
// are independent, so the pipe, not the FMA latency, sets the rate.  The
// final values are folded into one number that is stored only if it equals a
// value it can never take, so the compiler must keep every FMA while the
// kernel writes nothing.
#pragma once
#include "kern_common.cuh"

namespace fz {

constexpr int PROBE_CHAINS = 8;

__device__ double g_probe_sink64;
__device__ float g_probe_sink32;
__device__ __forceinline__ void probe_sink(double v) { g_probe_sink64 = v; }
__device__ __forceinline__ void probe_sink(float v) { g_probe_sink32 = v; }

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b) {
    T x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x & 31) * (T)1e-3 + (T)c;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fmaT(x[c], a, b);
        }
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (s == (T)-1234.5) probe_sink(s);  // never true; keeps the chains live
}

}  // namespace fz
