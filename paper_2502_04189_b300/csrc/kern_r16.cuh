// Register-resident FP32 transforms of length 32, 48, 64, 96, 128, 192, 256,
// 384 and 512 (mixed mode).
//
// The FP32 transform passes of the mixed-precision solve (the fast direct
// solver's real FFTs, or DCT-II for wall directions, along x and y).  A DFT of
// length NH = P M (P = 12, 16 or 24 values per thread, M = 2, 4, 8 or 16
// threads, M dividing P) is split P x M, the four-step form of the
// Cooley-Tukey factorisation: with n = M n1 + n2 and k = k1 + P k2,
//     X[k1 + P k2] = sum_n2 WM^(n2 k2) [ WNH^(n2 k1) sum_n1 x[M n1 + n2] WP^(n1 k1) ],
// W_L = exp(-2 pi i / L) (the inverse uses the conjugates; neither direction
// is scaled).  A complex line (two real lines as real and imaginary part) is
// held by M threads: thread t owns the samples x[M n1 + t], computes their
// P-point DFT in registers (16 = 4 x 4, 12 = 3 x 4, 24 = 3 x 8) and applies
// the twiddles WNH^(t k1); one pass through shared memory then hands it the
// values of k1 = t + M j (j < P/M), whose M-point DFTs give
// X[t + M j + P k2].  The separation of the two real spectra (forward) pairs
// X[k] with X[N - k], held in register P - 1 - r of thread (M - t) mod M of
// the same line, through warp shuffles; the inverse combination reads both
// values of a pair.  A wall direction keeps Makhoul's packing of the DCT-II
// (even samples forward, odd backward) and applies the post-twiddles
// (cos, sin)(pi m / (2N)) in the separation and combination.
//
// Lengths 384 and 512 first take one radix-2 step of decimation in
// frequency, N = 2 NH,
//     X[2k]     = DFT_NH( x[n] + x[n + NH] )[k],
//     X[2k + 1] = DFT_NH( (x[n] - x[n + NH]) W_N^n )[k],
// over two groups of M threads of a line that swap their halves with one
// shuffle; each group then runs the NH-point transform.
//
// Same arithmetic as the Stockham passes (about 11 FP32 multiply-adds per
// real point at n = 256); what it removes is their per-stage shared-memory
// round trips, index divisions and the select work of the FMA-form twiddles.
#pragma once
#include "kern_passes.cuh"

namespace fz {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * (c + i s)
__device__ __forceinline__ float2 c_mul(float2 a, float c, float s) {
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

// 2-point DFT in place.
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
    const float2 t = a0;
    a0 = c_add(t, a1);
    a1 = c_sub(t, a1);
}

// 3-point DFT in place (forward: W3 = -1/2 - i sqrt(3)/2).
template <bool INV>
__device__ __forceinline__ void dft3(float2 &a0, float2 &a1, float2 &a2) {
    constexpr float H = 0.86602540378443864676f;  // sqrt(3)/2
    const float2 s = c_add(a1, a2), d = c_sub(a1, a2);
    const float2 m = make_float2(fmaf(-0.5f, s.x, a0.x), fmaf(-0.5f, s.y, a0.y));
    a0 = c_add(a0, s);
    if (!INV) {  // X1 = m - i H d, X2 = m + i H d
        a1 = make_float2(fmaf(H, d.y, m.x), fmaf(-H, d.x, m.y));
        a2 = make_float2(fmaf(-H, d.y, m.x), fmaf(H, d.x, m.y));
    } else {
        a1 = make_float2(fmaf(-H, d.y, m.x), fmaf(H, d.x, m.y));
        a2 = make_float2(fmaf(H, d.y, m.x), fmaf(-H, d.x, m.y));
    }
}

// 4-point DFT in place (forward: W4 = -i).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    const float2 t0 = c_add(a0, a2), t1 = c_sub(a0, a2), t2 = c_add(a1, a3), t3 = c_sub(a1, a3);
    a0 = c_add(t0, t2);
    a2 = c_sub(t0, t2);
    if (!INV) {  // X1 = t1 - i t3, X3 = t1 + i t3
        a1 = make_float2(t1.x + t3.y, t1.y - t3.x);
        a3 = make_float2(t1.x - t3.y, t1.y + t3.x);
    } else {
        a1 = make_float2(t1.x - t3.y, t1.y + t3.x);
        a3 = make_float2(t1.x + t3.y, t1.y - t3.x);
    }
}

// v times W24^e (forward) or its conjugate (INV), 0 <= e < 24; e is a
// compile-time value once the callers' loops are unrolled.  cos and sin of
// pi e / 12 from the exact values of 15-degree multiples:
// cos 15 = (sqrt 6 + sqrt 2)/4, sin 15 = (sqrt 6 - sqrt 2)/4.
__device__ __forceinline__ float cos_pi12(int e) {
    constexpr float C15 = 0.96592582628906828675f, S15 = 0.25881904510252076235f;
    constexpr float H3 = 0.86602540378443864676f, H2 = 0.70710678118654752440f;
    e = e % 24;
    if (e > 12) e = 24 - e;  // cos is even about pi
    switch (e) {
    case 0: return 1.f;
    case 1: return C15;
    case 2: return H3;
    case 3: return H2;
    case 4: return 0.5f;
    case 5: return S15;
    case 6: return 0.f;
    case 7: return -S15;
    case 8: return -0.5f;
    case 9: return -H2;
    case 10: return -H3;
    case 11: return -C15;
    default: return -1.f;
    }
}
__device__ __forceinline__ float sin_pi12(int e) { return cos_pi12(e + 18); }  // sin x = cos(x - pi/2)

template <bool INV>
__device__ __forceinline__ float2 w24(float2 v, int e) {
    e %= 24;
    if (e == 0) return v;
    if (e == 12) return make_float2(-v.x, -v.y);
    if (e == 6) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);  // -+ i
    if (e == 18) return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);  // +- i
    const float s = sin_pi12(e);
    return c_mul(v, cos_pi12(e), INV ? s : -s);
}

// v times W16^e (forward) or its conjugate (INV), e in {1, 2, 3, 4, 6, 9}.
template <bool INV, int E>
__device__ __forceinline__ float2 w16(float2 v) {
    constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
    constexpr float R = 0.70710678118654752440f;   // cos(pi/4)
    constexpr float sg = INV ? 1.f : -1.f;         // sign of the sine part
    if constexpr (E == 4) {  // -i (forward), +i (inverse)
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (E == 2) {  // R (1 -+ i)
        return INV ? make_float2(R * (v.x - v.y), R * (v.y + v.x))
                   : make_float2(R * (v.x + v.y), R * (v.y - v.x));
    } else if constexpr (E == 6) {  // R (-1 -+ i)
        return INV ? make_float2(-R * (v.x + v.y), R * (v.x - v.y))
                   : make_float2(R * (v.y - v.x), -R * (v.x + v.y));
    } else if constexpr (E == 1) {
        return c_mul(v, C1, sg * S1);
    } else if constexpr (E == 3) {
        return c_mul(v, S1, sg * C1);
    } else {  // E == 9: -W16^1
        return c_mul(v, -C1, -sg * S1);
    }
}

// 16-point DFT of v[0..15] in place, natural order in and out (4 x 4 split).
template <bool INV, int S>
__device__ __forceinline__ void dft16(float2 (&v)[S]) {
    static_assert(S == 16, "dft16 works on 16 values");
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<INV>(v[b], v[4 + b], v[8 + b], v[12 + b]);
    // v[4 k1 + b] now holds the k1-th output of column b: twiddle W16^(b k1)
    v[5] = w16<INV, 1>(v[5]);
    v[6] = w16<INV, 2>(v[6]);
    v[7] = w16<INV, 3>(v[7]);
    v[9] = w16<INV, 2>(v[9]);
    v[10] = w16<INV, 4>(v[10]);
    v[11] = w16<INV, 6>(v[11]);
    v[13] = w16<INV, 3>(v[13]);
    v[14] = w16<INV, 6>(v[14]);
    v[15] = w16<INV, 9>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // X[k1 + 4 k2] sits in v[4 k1 + k2]: transpose the 4 x 4 index
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = o[k];
}

// 8-point DFT of v[O..O+7] in place, natural order in and out: 4-point DFTs
// of the even and the odd samples joined by W8^k (= W16^(2k)).
template <bool INV, int O, int S>
__device__ __forceinline__ void dft8(float2 (&v)[S]) {
    float2 e0 = v[O], e1 = v[O + 2], e2 = v[O + 4], e3 = v[O + 6];
    float2 o0 = v[O + 1], o1 = v[O + 3], o2 = v[O + 5], o3 = v[O + 7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = w16<INV, 2>(o1);
    o2 = w16<INV, 4>(o2);
    o3 = w16<INV, 6>(o3);
    v[O] = c_add(e0, o0);
    v[O + 4] = c_sub(e0, o0);
    v[O + 1] = c_add(e1, o1);
    v[O + 5] = c_sub(e1, o1);
    v[O + 2] = c_add(e2, o2);
    v[O + 6] = c_sub(e2, o2);
    v[O + 3] = c_add(e3, o3);
    v[O + 7] = c_sub(e3, o3);
}

// 12- and 24-point DFTs in place, natural order in and out: L = 3 Q with
// n = Q n1 + n2, k = k1 + 3 k2: 3-point DFTs over n1, the twiddles
// W_L^(n2 k1), then Q-point DFTs over n2 (Q = 4, 8).
template <bool INV, int Q>
__device__ __forceinline__ void dft3q(float2 (&v)[3 * Q]) {
    float2 y[3 * Q];  // y[Q k1 + n2]
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        float2 a = v[n2], b = v[Q + n2], c = v[2 * Q + n2];
        dft3<INV>(a, b, c);
        y[n2] = a;
        y[Q + n2] = w24<INV>(b, (24 / (3 * Q)) * n2);
        y[2 * Q + n2] = w24<INV>(c, (24 / (3 * Q)) * 2 * n2);
    }
    if constexpr (Q == 4) {
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) dft4<INV>(y[4 * k1], y[4 * k1 + 1], y[4 * k1 + 2], y[4 * k1 + 3]);
    } else {
        dft8<INV, 0>(y);
        dft8<INV, 8>(y);
        dft8<INV, 16>(y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + 3 * k2] = y[Q * k1 + k2];
}

// The P-point DFT of a thread's values.
template <bool INV, int P>
__device__ __forceinline__ void dft_p(float2 (&v)[P]) {
    if constexpr (P == 16) dft16<INV>(v);
    else if constexpr (P == 12) dft3q<INV, 4>(v);
    else dft3q<INV, 8>(v);
}

constexpr bool r_supported(int n) {
    return n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 || n == 384 ||
           n == 512;
}

// Launch shape of a length.  G: 2 for the radix-2 step (384, 512), else 1;
// NH = N / G = P M; TPL = G M threads hold a complex line; THREADS per CTA
// (fewer for the short and the 24-value lengths, so that small grids still
// spread over the SMs and the 24-value threads keep their registers);
// LINES complex lines per CTA and LPW per warp, the line stride in shared
// memory (padded), the y-pass tile width TX in real columns, and the
// resident CTAs per SM the kernels are compiled for.
template <int N> struct RShape {
    static_assert(r_supported(N), "register-resident lengths");
    static constexpr int G = (N == 384 || N == 512) ? 2 : 1;
    static constexpr int NH = N / G;
    static constexpr int P = (NH % 3 != 0) ? 16 : (NH == 48 ? 12 : 24);
    static constexpr int M = NH / P;
    static constexpr int TPL = G * M;
    static constexpr int THREADS = N == 32 ? 64 : (N == 128 || N == 256 || N == 512) ? 256 : 128;
    static constexpr int LINES = THREADS / TPL;
    static constexpr int LPW = 32 / TPL;
    static constexpr int LS = N + 1;
    static constexpr int TX = 2 * LINES;
    static constexpr int MINB = P == 24 ? 5 : P == 12 ? 6 : 65536 / (THREADS * 64);
    static constexpr int YCH = P == 12 ? 12 : 16;  // y-pass loads of a thread in flight
    static_assert(P % M == 0 && TPL <= 32 && TPL % 2 == 0, "shape");
};
constexpr int r_threads(int n) {
    return n == 32 ? RShape<32>::THREADS : n == 48 ? RShape<48>::THREADS : n == 64 ? RShape<64>::THREADS
         : n == 96 ? RShape<96>::THREADS : n == 128 ? RShape<128>::THREADS : n == 192 ? RShape<192>::THREADS
         : n == 256 ? RShape<256>::THREADS : n == 384 ? RShape<384>::THREADS : RShape<512>::THREADS;
}
constexpr int r_tile_cols(int n) {
    return n == 32 ? RShape<32>::TX : n == 48 ? RShape<48>::TX : n == 64 ? RShape<64>::TX
         : n == 96 ? RShape<96>::TX : n == 128 ? RShape<128>::TX : n == 192 ? RShape<192>::TX
         : n == 256 ? RShape<256>::TX : n == 384 ? RShape<384>::TX : RShape<512>::TX;
}
constexpr int r_tile_lines(int n) { return r_tile_cols(n); }  // x-passes: real lines per CTA

// Shared memory of one CTA: its lines, reused for the P x M exchanges; the
// twiddles W_NH^(t k1) at [k1][t] and, for the radix-2 lengths, W_N^n
// (n < NH), conjugated for the inverse; for a DCT direction the
// post-twiddles (cos, sin)(pi m / (2N)), m < N/2.
template <int N> struct RSmem {
    float2 x[RShape<N>::LINES * RShape<N>::LS];
    float2 tw[RShape<N>::NH];
    float2 tw2[RShape<N>::G == 2 ? RShape<N>::NH : 1];
    float2 cs[N / 2];
};

// (SM: any shared-memory struct with the tw, tw2 and cs tables of RSmem)
template <bool INV, int N, int KIND, typename SM>
__device__ __forceinline__ void r16_tables(SM &sm) {
    constexpr int M = RShape<N>::M, NH = RShape<N>::NH;
    float s, c;
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        const int k1 = i / M, t = i % M;
        sincospif(-(float)(2 * t * k1) / (float)NH, &s, &c);
        sm.tw[i] = make_float2(c, INV ? -s : s);
    }
    if constexpr (RShape<N>::G == 2) {
        for (int i = threadIdx.x; i < NH; i += blockDim.x) {
            sincospif(-(float)(2 * i) / (float)N, &s, &c);
            sm.tw2[i] = make_float2(c, INV ? -s : s);
        }
    }
    if constexpr (KIND == KIND_DCT) {
        for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
            sincospif((float)i / (float)(2 * N), &s, &c);
            sm.cs[i] = make_float2(c, s);
        }
    }
}

// The sample held at position p of a packed line: p itself (periodic), or,
// for the DCT, the even samples forward then the odd ones backward
// (2p for p < n/2, 2(n - 1 - p) + 1 above), the reordering of Makhoul's
// DCT-II through one complex FFT.
template <int N, int KIND>
__device__ __forceinline__ int r_src(int p) {
    if (KIND == KIND_PERIODIC) return p;
    return p < N / 2 ? 2 * p : 2 * (N - 1 - p) + 1;
}
constexpr float R_SQRT2 = 1.41421356237309504880f;  // the n/2 term of the DCT (2 cos(pi/4))

// The P x M four-step DFT on the P M values at X: thread t holds
// v[n1] = x[M n1 + t] and ends with v[j M + k2] = X[t + M j + P k2]
// (j < P/M, k2 < M): a P-point DFT, the twiddles W_(PM)^(t k1), one
// swizzled exchange through X (a permutation of M slots both ways), then
// P/M M-point DFTs.  X is overwritten; its threads (all in one warp) must
// have finished reading X before the call (warp barriers inside, the last
// one after the exchange reads).
template <bool INV, int P, int M, typename SM>
__device__ __forceinline__ void r_core(const SM &sm, float2 *X, int t, float2 (&v)[P]) {
    dft_p<INV, P>(v);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) {
        const float2 w = sm.tw[k1 * M + t];
        v[k1] = c_mul(v[k1], w.x, w.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) X[k1 * M + (t ^ (k1 & (M - 1)))] = v[k1];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < P / M; ++j)
#pragma unroll
        for (int n2 = 0; n2 < M; ++n2) v[j * M + n2] = X[(t + M * j) * M + (n2 ^ t)];
    __syncwarp();
    if constexpr (M == 16) {
        dft16<INV>(v);
    } else if constexpr (M == 8) {
        dft8<INV, 0>(v);
        dft8<INV, 8>(v);
        if constexpr (P == 24) dft8<INV, 16>(v);
    } else if constexpr (M == 4) {
#pragma unroll
        for (int j = 0; j < P / 4; ++j) dft4<INV>(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < P / 2; ++j) dft2(v[2 * j], v[2 * j + 1]);
    }
}

// Position of a thread: complex line ln of the CTA, group h (the half of a
// radix-2 line), index t in its P x M transform.  Its inputs are the
// samples in_index(n1), its outputs the indices out_index(r).
template <int N> struct RPos {
    static constexpr int M = RShape<N>::M, P = RShape<N>::P, NH = RShape<N>::NH;
    int ln, h, t;
    __device__ __forceinline__ RPos() {
        t = threadIdx.x & (M - 1);
        ln = threadIdx.x / RShape<N>::TPL;
        h = RShape<N>::G == 2 ? (threadIdx.x / M) & 1 : 0;
    }
    __device__ __forceinline__ int in_index(int n1) const { return M * n1 + t + NH * h; }
    __device__ __forceinline__ int out_index(int r) const {
        const int k = t + M * (r / M) + P * (r % M);
        return RShape<N>::G == 2 ? 2 * k + h : k;
    }
};

// The register holding the partner X[NH - k] of register r when the thread
// is its own partner (t = 0, group 0): r = j M + k2 maps to
// (M - k2) mod M for j = 0, else (P/M - j) M + M - 1 - k2.
template <int P, int M> constexpr int self_reg(int r) {
    return r / M == 0 ? (M - r % M) % M : (P / M - r / M) * M + (M - 1 - r % M);
}

// The transform of one line: v[n1] = the input at in_index(n1) on entry,
// v[r] = the output at out_index(r) on return.  X: the line's region
// (N values); warp barriers only (a line never spans warps).
template <bool INV, int N, typename SM>
__device__ __forceinline__ void r_fft(const SM &sm, float2 *X, const RPos<N> &q,
                                      float2 (&v)[RShape<N>::P]) {
    constexpr int P = RShape<N>::P, M = RShape<N>::M;
    if constexpr (RShape<N>::G == 2) {  // radix-2 step: group 0 gets lo + hi, group 1 (lo - hi) W_N^n
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) {
            const float2 own = v[n1];
            const float2 oth = make_float2(__shfl_xor_sync(0xffffffffu, own.x, M),
                                           __shfl_xor_sync(0xffffffffu, own.y, M));
            const float2 lo = q.h ? oth : own, hi = q.h ? own : oth;
            if (q.h == 0) {
                v[n1] = c_add(lo, hi);
            } else {
                const float2 w = sm.tw2[M * n1 + q.t];
                v[n1] = c_mul(c_sub(lo, hi), w.x, w.y);
            }
        }
        r_core<INV, P, M>(sm, X + RShape<N>::NH * q.h, q.t, v);
    } else {
        r_core<INV, P, M>(sm, X, q.t, v);
    }
}

// Separation of the forward transform of a packed line (two real lines as
// real and imaginary part): the spectra of both, scaled by 2 (the
// conventions of the Stockham passes: half-complex for a periodic direction,
// DCT-II coefficients through the post-twiddle (c, s)_m for a wall), through
// fn(k, a_k, b_k).  X[K] pairs with X[N - K], held in register P - 1 - r of
// thread (M - t) mod M of the line, or (t = 0) in this thread's register
// self_reg(r); for the radix-2 lengths the odd outputs pair within group 1
// with thread M - 1 - t, register P - 1 - r.
template <int N, int KIND, typename SM, typename F>
__device__ __forceinline__ void r_separate(const float2 (&v)[RShape<N>::P], const RPos<N> &q,
                                           const SM &sm, F &&fn) {
    constexpr int M = RShape<N>::M, P = RShape<N>::P;
    const int lane = threadIdx.x & 31, base = lane & ~(M - 1);
    const int src = q.h == 0 ? (base | ((M - q.t) & (M - 1))) : (base | (M - 1 - q.t));
    const bool self = q.h == 0 && q.t == 0;
#pragma unroll
    for (int r = 0; r < P; ++r) {
        const float qx = __shfl_sync(0xffffffffu, v[P - 1 - r].x, src);
        const float qy = __shfl_sync(0xffffffffu, v[P - 1 - r].y, src);
        const float2 z = v[r];
        const float2 y = self ? v[self_reg<P, M>(r)] : make_float2(qx, qy);
        const int k = q.out_index(r);
        if (KIND == KIND_PERIODIC) {
            // k <= n/2: (Re A_k, Re B_k) x 2; k > n/2: (Im A_m, Im B_m) x 2, m = n - k
            if (k <= N / 2) fn(k, z.x + y.x, z.y + y.y);
            else fn(k, y.y - z.y, z.x - y.x);
        } else if (k == 0) {
            fn(k, z.x + y.x, z.y + y.y);
        } else if (k == N / 2) {
            fn(k, R_SQRT2 * z.x, R_SQRT2 * z.y);
        } else if (k < N / 2) {  // 2 V_k = (var + i vai, vbr + i vbi); X_k = Re(w V_k)
            const float2 w = sm.cs[k];
            const float var = z.x + y.x, vai = z.y - y.y, vbr = z.y + y.y, vbi = y.x - z.x;
            fn(k, fmaf(w.x, var, w.y * vai), fmaf(w.x, vbr, w.y * vbi));
        } else {  // X_(n-m) = -Im(w V_m), m = n - k (Z_m is the partner's value)
            const float2 w = sm.cs[N - k];
            const float var = y.x + z.x, vai = y.y - z.y, vbr = y.y + z.y, vbi = z.x - y.x;
            fn(k, fmaf(w.y, var, -w.x * vai), fmaf(w.y, vbr, -w.x * vbi));
        }
    }
}

// Combination ahead of the inverse transform: v[n1] = Z[in_index(n1)] from
// the spectra of the two real lines read through get(k) = (a_k, b_k)
// (half-complex, or DCT-II coefficients pre-twiddled by (c, s)_m).
template <int N, int KIND, typename SM, typename G>
__device__ __forceinline__ void r_combine(float2 (&v)[RShape<N>::P], const RPos<N> &q, const SM &sm,
                                          G &&get) {
#pragma unroll
    for (int n1 = 0; n1 < RShape<N>::P; ++n1) {
        const int k = q.in_index(n1);
        const float2 o = get(k), p = get(k == 0 ? 0 : N - k);  // indices k and n - k
        if (KIND == KIND_PERIODIC) {
            if (k == 0 || k == N / 2) v[n1] = o;
            else if (k < N / 2) v[n1] = make_float2(o.x - p.y, p.x + o.y);
            else v[n1] = make_float2(p.x + o.y, p.y - o.x);
        } else if (k == 0) {
            v[n1] = o;
        } else if (k == N / 2) {
            v[n1] = make_float2(R_SQRT2 * o.x, R_SQRT2 * o.y);
        } else {
            // m = min(k, n - k); V_m = (c + i s)(X_m - i X_(n-m)) for each line
            const bool lo = k < N / 2;
            const float2 w = sm.cs[lo ? k : N - k];
            const float2 xm = lo ? o : p, xn = lo ? p : o;  // (a, b) at m and at n - m
            const float ar = fmaf(w.x, xm.x, w.y * xn.x), ai = fmaf(w.y, xm.x, -w.x * xn.x);
            const float br = fmaf(w.x, xm.y, w.y * xn.y), bi = fmaf(w.y, xm.y, -w.x * xn.y);
            v[n1] = lo ? make_float2(ar - bi, ai + br) : make_float2(ar + bi, br - ai);
        }
    }
}

// ---- y-passes: the columns of an (nz, N, nx) FP32 array, flattened over the
// planes (column cc = k nx + i), in tiles of TX consecutive columns, each
// transformed along y in place.  Thread e of the CTA owns column e mod TX of
// the tile and rows e / TX + (THREADS / TX) i, i < 2P (THREADS / TX = TPL/2
// rows apart): one address per thread, each warp access 32 consecutive
// columns (TX >= 32) or two rows of 16 (YCH of a thread's loads in flight).
// Column 2l + c of the tile is
// component c of complex line l.  Forward: real columns -> spectra scaled by
// 2 (half-complex, or DCT-II for a wall direction); inverse: the reverse,
// unscaled.
template <bool INV, int N, int KIND>
__device__ __forceinline__ void ypass_r_tile(int nx, int ncol, float *data, int tile, RSmem<N> &sm) {
    typedef RShape<N> S;
    constexpr int TX = S::TX, LS = S::LS, P = S::P, RSTEP = S::THREADS / TX;
    static_assert(S::THREADS % TX == 0 && N * TX == 2 * P * S::THREADS, "tile shape");
    const RPos<N> q;
    const int col = threadIdx.x % TX, row0 = threadIdx.x / TX;
    const int cc = tile * TX + col;
    const bool ok = cc < ncol;
    const int kp = ok ? cc / nx : 0;
    // the thread's column (32-bit row offsets within its plane)
    float *gcol = data + (size_t)kp * N * nx + (ok ? cc - kp * nx : 0);
    float *scol = (float *)sm.x + (col >> 1) * (2 * LS) + (col & 1);
    float2 *X = sm.x + q.ln * LS;
    // 1. stage the tile: every element of the thread's column as an
    // asynchronous 4-byte global -> shared copy (all 2P in flight, no
    // registers held), zeros past the last column
    if (ok) {
#pragma unroll
        for (int i = 0; i < 2 * P; ++i) {
            const int row = row0 + RSTEP * i;
            cp_async<4>(scol + 2 * row, gcol + (size_t)row * nx);
        }
        cp_async_commit();
        cp_async_wait<0>();
    } else {
#pragma unroll
        for (int i = 0; i < 2 * P; ++i) scol[2 * (row0 + RSTEP * i)] = 0.f;
    }
    __syncthreads();
    float2 v[P];
    if (!INV) {
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
    } else {
        r_combine<N, KIND>(v, q, sm, [&](int k) { return X[k]; });
    }
    __syncwarp();  // the line's region is the exchange buffer next
    r_fft<INV, N>(sm, X, q, v);
    if (!INV) {
        r_separate<N, KIND>(v, q, sm, [&](int k, float a, float b) { X[k] = make_float2(a, b); });
    } else {
#pragma unroll
        for (int r = 0; r < P; ++r) X[r_src<N, KIND>(q.out_index(r))] = v[r];
    }
    __syncthreads();
    // 2. write the tile back
#pragma unroll
    for (int i = 0; i < 2 * P; ++i) {
        const int row = row0 + RSTEP * i;
        if (ok) gcol[(size_t)row * nx] = scol[2 * row];
    }
    __syncthreads();  // the buffer is free for the next tile
}

// y-pass with the signature of k_ypass, so the plan can launch either: the
// launch covers ntiles = ygx nz per-plane tiles of the Stockham pass
// (ygx = ceil(nx / TX)), the kernel the ceil(nx nz / TX) flattened tiles
// (never more).  conv: return at once when the refinement has converged.
template <bool INV, int N, int KIND>
__global__ void __launch_bounds__(RShape<N>::THREADS, RShape<N>::MINB)
    k_ypass_r(int nx, int ny, FFTDesc D, int TX, float *data, const int *conv, int ygx, int ntiles) {
    (void)ny;
    (void)D;
    (void)TX;
    __shared__ RSmem<N> sm;
    if (conv && *(volatile const int *)conv) return;
    r16_tables<INV, N, KIND>(sm);
    __syncthreads();
    const int nz = ntiles / ygx, ncol = nx * nz;
    const int nflat = (ncol + RShape<N>::TX - 1) / RShape<N>::TX;
    for (int tile = blockIdx.x; tile < nflat; tile += gridDim.x)
        ypass_r_tile<INV, N, KIND>(nx, ncol, data, tile, sm);
}

// ---- x-passes: 2 LINES real lines of the [nz][ny] line set per CTA.  A
// warp owns LPW complex lines (2 LPW real rows, rows 2l and 2l + 1 packed as
// line l), 2 LPW N = 64 P consecutive floats of the array; it stages them
// through their shared-memory regions (element e = lane + 32 s of the warp's
// span: 128-byte accesses), transforms them and writes them back the same
// way, with warp barriers only.

// The warp's first line (of the CTA).
template <int N> __device__ __forceinline__ int r_warp_line() {
    return (threadIdx.x >> 5) * RShape<N>::LPW;
}

// Slot s (s < 2P) of a lane: element e = lane + 32 s of the warp's rows,
// row e / N of the warp, x = e mod N.
template <int N> __device__ __forceinline__ int r_slot_row(int s) { return ((threadIdx.x & 31) + 32 * s) / N; }
template <int N> __device__ __forceinline__ int r_slot_x(int s) { return ((threadIdx.x & 31) + 32 * s) % N; }
// The shared-memory float of (row r of the warp, x): line l0 + r/2, component r & 1.
template <int N> __device__ __forceinline__ int r_slot_f(int r, int x) {
    return (r_warp_line<N>() + (r >> 1)) * (2 * RShape<N>::LS) + 2 * x + (r & 1);
}

// Rows of the warp from an FP32 array [nlines][N] into the line regions
// (zeros past the last line), CH loads of a lane in flight (all 2P, or
// 16 at a time for the 24-value lengths, whose registers are the tighter).
template <int N>
__device__ __forceinline__ void r_rows_in(const float *src, int row0, int nlines, RSmem<N> &sm) {
    constexpr int P = RShape<N>::P, CH = P == 24 ? 16 : 2 * P;
    float *sf = (float *)sm.x;
    const float *base = src + (size_t)row0 * N + (threadIdx.x & 31);
#pragma unroll 1
    for (int s0 = 0; s0 < 2 * P; s0 += CH) {
        float x[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u)
            x[u] = row0 + r_slot_row<N>(s0 + u) < nlines ? base[32 * (s0 + u)] : 0.f;
#pragma unroll
        for (int u = 0; u < CH; ++u) sf[r_slot_f<N>(r_slot_row<N>(s0 + u), r_slot_x<N>(s0 + u))] = x[u];
    }
    __syncwarp();
}

// Rows of the warp from the line regions back to an FP32 array.
template <int N>
__device__ __forceinline__ void r_rows_out(float *dst, int row0, int nlines, const RSmem<N> &sm) {
    const float *sf = (const float *)sm.x;
    float *base = dst + (size_t)row0 * N + (threadIdx.x & 31);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2 * RShape<N>::P; ++s)
        if (row0 + r_slot_row<N>(s) < nlines) base[32 * s] = sf[r_slot_f<N>(r_slot_row<N>(s), r_slot_x<N>(s))];
    __syncwarp();
}

// Forward transform of the staged lines: inputs from the line region X,
// the spectra back into it.
template <int N, int KIND>
__device__ __forceinline__ void r_forward_line(const RSmem<N> &sm, float2 *X, const RPos<N> &q) {
    float2 v[RShape<N>::P];
#pragma unroll
    for (int n1 = 0; n1 < RShape<N>::P; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
    __syncwarp();  // the line's region is the exchange buffer next
    r_fft<false, N>(sm, X, q, v);
    r_separate<N, KIND>(v, q, sm, [&](int k, float a, float b) { X[k] = make_float2(a, b); });
}

// Lengths whose M = 16 threads of a line read and write their two rows in
// 64-byte runs: the x-passes access global memory directly.
template <int N> constexpr bool r_direct() { return N == 256 || N == 512; }

// The transform of the stored FP32 residual (refinement sweeps), in place:
// the mode XF_MIX_LOAD of k_xfwd.
template <int N, int KIND>
__global__ void __launch_bounds__(RShape<N>::THREADS, RShape<N>::MINB)
    k_xfwd_r_load(GridDev g, FFTDesc D, int L, XArgs a, int ntiles) {
    (void)D;
    (void)L;
    __shared__ RSmem<N> sm;
    if (*(volatile const int *)&a.st->converged) return;
    r16_tables<false, N, KIND>(sm);
    __syncthreads();
    const RPos<N> q;
    const int nlines = g.ny * g.nz;
    float *data = (float *)a.out;
    float2 *X = sm.x + q.ln * RShape<N>::LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * r_tile_lines(N) + 2 * r_warp_line<N>();
        if constexpr (r_direct<N>()) {
            const int ra = tile * r_tile_lines(N) + 2 * q.ln;
            const bool oka = ra < nlines, okb = ra + 1 < nlines;
            float *la = data + (size_t)ra * N, *lb = la + N;
            float2 v[RShape<N>::P];
#pragma unroll
            for (int n1 = 0; n1 < RShape<N>::P; ++n1) {
                const int i = r_src<N, KIND>(q.in_index(n1));
                v[n1] = make_float2(oka ? la[i] : 0.f, okb ? lb[i] : 0.f);
            }
            r_fft<false, N>(sm, X, q, v);
            r_separate<N, KIND>(v, q, sm, [&](int k, float va, float vb) {
                if (oka) la[k] = va;
                if (okb) lb[k] = vb;
            });
            __syncwarp();  // every lane has read its line before the next tile
        } else {
            r_rows_in<N>(data, row0, nlines, sm);
            r_forward_line<N, KIND>(sm, X, q);
            r_rows_out<N>(data, row0, nlines, sm);
        }
    }
}

// The first x-pass of the mixed solve (the mode XF_MIX_DIVQ of k_xfwd):
// f = rho0 D(q') in double-float (div_q_eval_df; stored in FP64, and max|f|
// recorded), then the forward transform of its FP32 image sigma f.  f is
// formed into the line regions
// row by row for rows of N >= 256 cells (lane = x mod 32, the row's
// constants once), else slot by slot (coalesced either way).
template <int N, int KIND>
__global__ void __launch_bounds__(RShape<N>::THREADS, RShape<N>::MINB)
    k_xfwd_r_divq(GridDev g, FFTDesc D, int L, XArgs a, int ntiles) {
    (void)D;
    (void)L;
    __shared__ RSmem<N> sm;
    r16_tables<false, N, KIND>(sm);
    __syncthreads();
    constexpr int P = RShape<N>::P;
    const RPos<N> q;
    const int nlines = g.ny * g.nz, l0 = r_warp_line<N>();
    constexpr int LS = RShape<N>::LS;
    const float scale32 = (float)g.sigma;
    const float2 cx = f64_split(g.dvx), cy = f64_split(g.dvy);
    float *out = (float *)a.out;
    float *sf = (float *)sm.x;
    float2 *X = sm.x + q.ln * LS;
    unsigned long long mx = 0ull;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * r_tile_lines(N) + 2 * l0;
        if constexpr (N >= 256) {  // rows of N/32 >= 8 cells per lane: per-row constants once
            const int lane = threadIdx.x & 31;
#pragma unroll 1
            for (int r = 0; r < 2 * RShape<N>::LPW; ++r) {
                const int row = row0 + r;
                float *dr = sf + r_slot_f<N>(r, 0);
                if (row < nlines) {
                    const int k = fdiv(row, g.ny, g.rny), j = row - k * g.ny;
                    const float2 cz = f64_split(g.dvz[k]);
                    // the face loads of two cells ahead of their arithmetic
                    // and stores (a store to f could alias a later load)
                    constexpr int U = 2;
#pragma unroll 1
                    for (int i0 = 0; i0 < N / 32; i0 += U) {
                        QFaces qf[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) qf[u] = div_q_ld<false>(g, lane + 32 * (i0 + u), j, k, a.qx, a.qy, a.qz);
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int x = lane + 32 * (i0 + u);
                            const double f = div_q_eval_df(qf[u], cx, cy, cz);
                            a.f_out[(size_t)row * N + x] = f;
                            mx = umax64(mx, absbits(f));
                            dr[2 * x] = f64_to_f32_shift(f, 0) * scale32;
                        }
                    }
                } else {
                    for (int i = 0; i < N / 32; ++i) dr[2 * (lane + 32 * i)] = 0.f;
                }
            }
        } else {  // short rows: the warp's 2P slots per lane
#pragma unroll 4
            for (int s = 0; s < 2 * P; ++s) {
                const int r = r_slot_row<N>(s), x = r_slot_x<N>(s), row = row0 + r;
                float val = 0.f;
                if (row < nlines) {
                    const int k = fdiv(row, g.ny, g.rny), j = row - k * g.ny;
                    const double f = div_q_eval_df(div_q_ld<false>(g, x, j, k, a.qx, a.qy, a.qz), cx, cy,
                                                   f64_split(g.dvz[k]));
                    a.f_out[(size_t)row * N + x] = f;
                    mx = umax64(mx, absbits(f));
                    val = f64_to_f32_shift(f, 0) * scale32;
                }
                sf[r_slot_f<N>(r, x)] = val;
            }
        }
        __syncwarp();
        if constexpr (r_direct<N>()) {  // the spectra straight to global memory
            float2 v[P];
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
            __syncwarp();  // the line's region is the exchange buffer next
            r_fft<false, N>(sm, X, q, v);
            const int ra = tile * r_tile_lines(N) + 2 * q.ln;
            const bool oka = ra < nlines, okb = ra + 1 < nlines;
            float *la = out + (size_t)ra * N, *lb = la + N;
            r_separate<N, KIND>(v, q, sm, [&](int kk, float va, float vb) {
                if (oka) la[kk] = va;
                if (okb) lb[kk] = vb;
            });
            __syncwarp();  // the region is rewritten by the next tile
        } else {
            r_forward_line<N, KIND>(sm, X, q);
            r_rows_out<N>(out, row0, nlines, sm);
        }
    }
    block_max_atomic(mx, &a.st->fmax_bits);
}

// Inverse x-pass to p (FP64): XI_STORE p = the FP32 solution, XI_ACCUM
// p += delta 2^e (e: exponent of max|f|); the modes of k_xinv.
template <int MODE, int N, int KIND>
__global__ void __launch_bounds__(RShape<N>::THREADS, RShape<N>::MINB)
    k_xinv_r(GridDev g, FFTDesc D, int L, const float *in, double *p, const DevStats *st, int ntiles) {
    (void)D;
    (void)L;
    __shared__ RSmem<N> sm;
    if (MODE == XI_ACCUM && *(volatile const int *)&st->converged) return;
    r16_tables<true, N, KIND>(sm);
    __syncthreads();
    constexpr int P = RShape<N>::P;
    const int ef = MODE == XI_ACCUM ? exp_of_bits(*(volatile const unsigned long long *)&st->fmax_bits) : 0;
    const RPos<N> q;
    const int nlines = g.ny * g.nz, l0 = r_warp_line<N>();
    float2 *X = sm.x + q.ln * RShape<N>::LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * r_tile_lines(N) + 2 * l0;
        r_rows_in<N>(in, row0, nlines, sm);
        float2 v[P];
        r_combine<N, KIND>(v, q, sm, [&](int k) { return X[k]; });
        __syncwarp();  // the line's region is the exchange buffer next
        r_fft<true, N>(sm, X, q, v);
#pragma unroll
        for (int r = 0; r < P; ++r) X[r_src<N, KIND>(q.out_index(r))] = v[r];
        __syncwarp();
        // p (or p += delta) by slots (lane = x mod 32), eight values of p in
        // flight per lane
        const float *sf = (const float *)sm.x;
        double *pb = p + (size_t)row0 * N + (threadIdx.x & 31);
#pragma unroll(P == 24 ? 1 : 2 * P / 8)
        for (int s0 = 0; s0 < 2 * P; s0 += 8) {
            double qv[8];
            if (MODE == XI_ACCUM) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    qv[u] = row0 + r_slot_row<N>(s0 + u) < nlines ? pb[32 * (s0 + u)] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r_slot_row<N>(s0 + u), x = r_slot_x<N>(s0 + u);
                const double d = f32_to_f64_shift(sf[r_slot_f<N>(r, x)], ef);
                if (row0 + r < nlines) pb[32 * (s0 + u)] = MODE == XI_ACCUM ? qv[u] + d : d;
            }
        }
        __syncwarp();  // the line regions are rewritten by the next tile
    }
}

}  // namespace fz
