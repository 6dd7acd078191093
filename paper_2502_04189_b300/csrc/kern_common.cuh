// Shared device helpers for the projection kernels (sm_103a).
//
// Design note: on this part FP64 instructions (DFMA/DADD/DMUL and the
// F2F conversions between float and double) issue at roughly 1/74 of the FP32
// rate, so every kernel here counts FP64 instructions per grid point.  Bit-level
// conversions below move values between float and double with integer
// instructions only (IEEE 754 field arithmetic) where a conversion would
// otherwise cost an FP64 issue slot.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fz {

template <typename T> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Products that must not be fused into a following add: the rounding of every
// kernel body then does not depend on the context it is compiled in (a body
// gives bit-identical results as a stand-alone kernel and inside the
// persistent batch kernel).
__device__ __forceinline__ double mulT(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mulT(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ double2 mk2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk2(float x, float y) { return make_float2(x, y); }

// double -> float for a positive normal value whose exponent fits a float
// (|x| in about [1.2e-38, 3.4e38]); truncates the mantissa (relative error
// below 2^-23).  Three integer instructions instead of an FP64 conversion.
__device__ __forceinline__ float pos_f64_to_f32_trunc(double x) {
    const int hi = __double2hiint(x);
    const int lo = __double2loint(x);
    // (hi << 3 | lo >> 29) puts the low 9 exponent bits on top of the 23
    // leading mantissa bits; re-biasing the exponent (1023 -> 127) is a
    // subtraction of 896 = 512 + 384 modulo 2^9 on that field.
    const unsigned b = __funnelshift_l((unsigned)lo, (unsigned)hi, 3) - (384u << 23);
    return __uint_as_float(b);
}

// float -> double for a positive normal float (exact).  Integer-only.
__device__ __forceinline__ double pos_f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    return __hiloint2double((int)((b >> 3) + (896u << 20)), (int)(b << 29));
}

// 1/s for s > 0 (positive normal double within float range), relative error
// about 2^-44: an FP32 seed (approximate reciprocal of the truncated
// argument, error below 2^-22) refined by one Newton-Raphson step in FP64,
// r1 = r0 + r0 (1 - s r0), which squares the relative error.  Costs two FP64
// instructions.
__device__ __forceinline__ double rcp_pos_nr1(double s) {
    float sf = pos_f64_to_f32_trunc(s);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(sf));
    const double r0 = pos_f32_to_f64(rf);
    const double e = __fma_rn(-s, r0, 1.0);
    return __fma_rn(r0, e, r0);
}

// |x| as an unsigned 64-bit pattern: for non-negative doubles the integer
// order of the bit patterns is the numeric order, so max-reductions run on the
// integer units (and atomicMax on the pattern is exact and order-independent).
__device__ __forceinline__ unsigned long long absbits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned absbits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__device__ __forceinline__ int block_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int block_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

// Block-wide max of a 64-bit pattern, then one atomicMax per block.
// Every thread of the block must call it (it contains barriers).
__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long *dst) {
    __shared__ unsigned long long red[32];
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = block_tid() & 31, wid = block_tid() >> 5;
    const int nw = (block_nthreads() + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v) atomicMax(dst, v);
    }
}

// Block-wide sum (deterministic order within the block); thread 0 gets the
// result.  Every thread of the block must call it (it contains barriers).
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = block_tid() & 31, wid = block_tid() >> 5;
    const int nw = (block_nthreads() + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// 2^e as a double (e within the normal range)
__device__ __forceinline__ double pow2d(int e) {
    return __hiloint2double((e + 1023) << 20, 0);
}
// binary exponent of a positive double given by its bit pattern (0 -> 0)
__device__ __forceinline__ int exp_of_bits(unsigned long long b) {
    return b ? (int)((b >> 52) & 0x7ff) - 1023 : 0;
}

// double -> float with the binary exponent shifted by -es (x * 2^-es),
// truncating; |result| below 2^-126 flushes to zero.  Integer-only.
__device__ __forceinline__ float f64_to_f32_shift(double x, int es) {
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ff) - es;  // biased double exponent after the shift
    if (e <= 896) return __uint_as_float(hi & 0x80000000u);
    const unsigned b = ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(b | (hi & 0x80000000u));
}
// float -> double times 2^es (flush float denormals to zero).  Integer-only.
__device__ __forceinline__ double f32_to_f64_shift(float f, int es) {
    const unsigned b = __float_as_uint(f);
    const unsigned a = b & 0x7fffffffu;
    if (a < 0x00800000u) return __hiloint2double((int)(b & 0x80000000u), 0);
    const unsigned hi = (((a >> 23) + 896u + (unsigned)es) << 20) | ((a >> 3) & 0xfffffu);
    return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(a << 29));
}

// f 2^-es for a float, as f64_to_f32_shift(f32_to_f64_shift(f, 0), es)
// gives it (integer operations): float denormals and results below 2^-126
// flush to a signed zero.
__device__ __forceinline__ float f32_shift(float f, int es) {
    const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu;
    const int ne = (int)(a >> 23) - es;
    if (a < 0x00800000u || ne <= 0) return __uint_as_float(b & 0x80000000u);
    return __uint_as_float(((unsigned)ne << 23) | (a & 0x7fffffu) | (b & 0x80000000u));
}

// Double-float arithmetic (an unevaluated sum hi + lo of two floats, about
// 48 significant bits): Knuth's two-sum, Dekker's fast two-sum and the
// FMA-based exact product, written with explicit round-to-nearest
// operations so the compiler neither contracts nor reorders them.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
    const float2 s = two_sum(x.x, y.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 c) {
    const float p = __fmul_rn(x.x, c.x);
    float e = __fmaf_rn(x.x, c.x, -p);  // the product's rounding error, exactly
    e = __fmaf_rn(x.x, c.y, e);
    e = __fmaf_rn(x.y, c.x, e);
    return fast_two_sum(p, e);
}
// A double as hi + lo floats with integer operations only: hi is the double
// truncated to 24 bits, lo the remaining 29 mantissa bits rounded to 24, so
// |x - hi - lo| <= 2^-47 |x| for 2^-74 <= |x| < 2^128 (below 2^-74 lo
// flushes to 0 and the error is at most 2^-24 |x|).
__device__ __forceinline__ float2 f64_split(double x) {
    const float hi = f64_to_f32_shift(x, 0);
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    const int sb = (int)((h >> 20) & 0x7ff) - 1075 + 127;  // biased float exponent of 2^(E - 1075)
    float lo = 0.f;
    if (sb > 0) lo = __fmul_rn(__uint2float_rn(l & 0x1fffffffu), __int_as_float(sb << 23));
    return make_float2(hi, (h & 0x80000000u) ? -lo : lo);
}

// A double as the exact sum h + m + l of three floats (integer operations):
// h the top 24 significant bits, m the next 24, l the last 5, for
// 2^-78 <= |x| < 2^128 (below, the parts that fall under the float range
// flush to 0).
struct F3 {
    float h, m, l;
};
__device__ __forceinline__ F3 f64_split3(double x) {
    const unsigned hb = (unsigned)__double2hiint(x), lb = (unsigned)__double2loint(x);
    const int E = (int)((hb >> 20) & 0x7ff);
    const bool neg = (hb & 0x80000000u) != 0;
    F3 r;
    r.h = f64_to_f32_shift(x, 0);
    const int sm = E - 1070 + 127, sl = E - 1075 + 127;  // biased float exponents of 2^(E-1070), 2^(E-1075)
    const float m = sm > 0 ? __fmul_rn(__uint2float_rn((lb >> 5) & 0xffffffu), __int_as_float(sm << 23)) : 0.f;
    const float l = sl > 0 ? __fmul_rn(__uint2float_rn(lb & 0x1fu), __int_as_float(sl << 23)) : 0.f;
    r.m = neg ? -m : m;
    r.l = neg ? -l : l;
    return r;
}

// x 2^-es as hi + lo floats, integer operations only (f64_split with the
// binary exponent shifted by -es): hi is x 2^-es truncated to 24 bits, lo the
// remaining 29 mantissa bits rounded to 24, |x 2^-es - hi - lo| <= 2^-47 |x 2^-es|
// while x 2^-es lies in [2^-74, 2^128).  x = 0 gives 0 only for es >= -896
// (below, the zero exponent field would read as a normal number after the
// shift), so callers shifting by the exponent of a small x pass non-zero x.
__device__ __forceinline__ float2 f64_split_sh(double x, int es) {
    const float hi = f64_to_f32_shift(x, es);
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    const int sb = (int)((h >> 20) & 0x7ff) - es - 1075 + 127;
    float lo = 0.f;
    if (sb > 0) lo = __fmul_rn(__uint2float_rn(l & 0x1fffffffu), __int_as_float(sb << 23));
    return make_float2(hi, (h & 0x80000000u) ? -lo : lo);
}

// a / b in double-float (b.x a positive normal float): the FP32 reciprocal y
// of b.x (rcp.approx, then one Newton step), the quotient q1 = a.x y, its
// remainder a - b q1 (a.x - b.x q1 is exact by Sterbenz, the rounding error
// of b.x q1 comes from an FMA) and the correction q2 = remainder * y:
// relative error about 2^-45.  a = 0 gives exactly 0.
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(b.x));
    y = __fmaf_rn(__fmaf_rn(-b.x, y, 1.f), y, y);
    const float q1 = __fmul_rn(a.x, y);
    const float p = __fmul_rn(b.x, q1);
    float e = __fmaf_rn(b.x, q1, -p);
    e = __fmaf_rn(b.y, q1, e);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), e), a.y);
    return fast_two_sum(q1, __fmul_rn(r, y));
}

// A normalized float pair hi + lo (|lo| <= half an ulp of hi) times 2^-es
// as one double, integer operations only: hi moves to FP64 exactly and lo is
// added as an integer count of that double's last places, k = lo 2^(52 - e)
// for hi = 1.m 2^e (|k| <= 2^28, truncated toward zero: relative error below
// 2^-52).  The one case whose sum leaves hi's binade is hi a power of two and
// lo of the other sign: there the lower binade's places are half as large
// and the count doubles.  hi below the float normal range gives 0, as
// f32_to_f64_shift does.
__device__ __forceinline__ double df_pair_to_f64_shift(float2 d, int es) {
    const double h = f32_to_f64_shift(d.x, es);
    const unsigned bh = __float_as_uint(d.x), bl = __float_as_uint(d.y);
    const unsigned al = bl & 0x7fffffffu;
    if (al < 0x00800000u || (bh & 0x7fffffffu) < 0x00800000u) return h;
    const int s = (int)(al >> 23) - (int)((bh >> 23) & 0xffu) + 29;
    if (s < -24) return h;  // lo below the double's last place
    const unsigned ml = (al & 0x7fffffu) | 0x800000u;
    long long k = (long long)(s >= 0 ? (ml << s) : (ml >> -s));
    const bool opposite = ((bh ^ bl) & 0x80000000u) != 0;
    if (opposite && (bh & 0x7fffffu) == 0u) k <<= 1;  // hi a power of two, sum below it
    const long long hb = __double_as_longlong(h);
    return __longlong_as_double(opposite ? hb - k : hb + k);
}

// Asynchronous global -> shared copies (cp.async, LDGSTS): the copy runs in
// the background and the issuing thread waits for its own groups.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Device-side state of one solve (reset at the start of every solve).
struct DevStats {
    unsigned long long fmax_bits;      // max|f|
    unsigned long long rmax_bits[20];  // max|r| per residual evaluation (mixed)
    unsigned long long divmax_bits;    // max|D u|
    unsigned int done_blocks[20];      // last-block counters of the residual kernels
    int converged;                     // mixed: set once relres <= tol
    int iterations;                    // mixed: sweeps that ran
    int n_resid;                       // residual evaluations that ran
    double relres;                     // last relres
    double usq_partial_dummy;          // (alignment)
};

}  // namespace fz
