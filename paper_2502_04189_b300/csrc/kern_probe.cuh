// Arithmetic-throughput probe (measurement support, not part of the
// projection): the FP64 and FP32 issue rates of the GPU, measured the way the
// FP64-bound projection kernels use the pipe.
//
// Every thread runs CH independent chains for `iters` rounds of 4 operations
// each: x <- x a + b (OP 0, fused multiply-add), x <- x + b (OP 1), x <- x a
// (OP 2), a multiply-add and an add in turn (OP 3), a multiply-add with an
// independent FP32 multiply-add issued after it (OP 4; FP64 kernels
// interleave such work; only the FP64 instructions are counted), or
// x_c <- x_c x_(c+1) + b (OP 5: the multiplicand a register, not a
// constant).  a is slightly below 1, so the values stay bounded; the chains
// are independent, so the pipe, not the latency, sets the rate.  The final values are folded into one
// number that is stored only if it equals a value it can never take, so the
// compiler must keep every operation while the kernel writes nothing.
#pragma once
#include "kern_common.cuh"

namespace fz {

__device__ double g_probe_sink64;
__device__ float g_probe_sink32;
__device__ __forceinline__ void probe_sink(double v) { g_probe_sink64 = v; }
__device__ __forceinline__ void probe_sink(float v) { g_probe_sink32 = v; }
__device__ __forceinline__ double addT(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float addT(float a, float b) { return __fadd_rn(a, b); }

template <typename T, int OP, int CH>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b) {
    T x[CH];
    float y[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        x[c] = (T)(threadIdx.x & 31) * (T)1e-3 + (T)c * (T)0.01;
        y[c] = (float)c;
    }
    const float af = 0.999f, bf = 1e-3f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (OP == 0 || OP == 4 || (OP == 3 && (r & 1) == 0)) x[c] = fmaT(x[c], a, b);
                else if (OP == 1 || OP == 3) x[c] = addT(x[c], b);
                else if (OP == 5) x[c] = fmaT(x[c], x[(c + 1) % CH], b);
                else x[c] = mulT(x[c], a);
                if (OP == 4) y[c] = __fmaf_rn(y[c], af, bf);
            }
        }
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c] + (T)y[c];
    if (s == (T)-1234.5) probe_sink(s);  // never true; keeps the chains live
}

}  // namespace fz
