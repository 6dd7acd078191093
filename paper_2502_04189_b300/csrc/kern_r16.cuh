// Register-resident FP32 transforms of length 128, 256 and 512 (mixed mode).
//
// The FP32 transform passes of the mixed-precision solve (the fast direct
// solver's real FFTs, or DCT-II for wall directions, along x and y).  A DFT of length
// N = 16 M (M = 8, 16; 4 builds too) is split 16 x M, the four-step form of
// the Cooley-Tukey factorisation: with n = M n1 + n2 and k = k1 + 16 k2,
//     X[k1 + 16 k2] = sum_n2 WM^(n2 k2) [ WN^(n2 k1) sum_n1 x[M n1 + n2] W16^(n1 k1) ],
// W_N = exp(-2 pi i / N) (the inverse uses the conjugates; neither direction
// is scaled).  A complex line (two real lines as real and imaginary part) is
// held by M threads: thread t owns the samples x[M n1 + t], computes their
// 16-point DFT in registers and applies the twiddles WN^(t k1); one pass
// through shared memory then hands it the values of k1 = t + M j, whose
// M-point DFTs give X[t + M j + 16 k2].  The separation of the two real
// spectra (forward) pairs X[k] with X[N - k], held in register 15 - r of
// thread (M - t) mod M of the same line, through warp shuffles; the inverse
// combination reads both values of a pair.  A wall direction keeps
// Makhoul's packing of the DCT-II (even samples forward, odd backward) and
// applies the post-twiddles (cos, sin)(pi m / (2N)) in the separation and
// combination.
//
// Length 512 first takes one radix-2 step of decimation in frequency,
//     X[2k]     = DFT256( x[n] + x[n + 256] )[k],
//     X[2k + 1] = DFT256( (x[n] - x[n + 256]) W512^n )[k],
// over two groups of 16 threads (a warp per line) that swap their halves
// with one shuffle; each group then runs the 256-point transform.
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
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
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
template <bool INV, int O>
__device__ __forceinline__ void dft8(float2 (&v)[16]) {
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

// Launch shape of a length.  N = 16 M (M = 4, 8, 16): M threads hold a
// line, 16 values each; N = 512: a warp per line, two 16-thread groups.
// Complex lines per CTA of 256 threads and per warp, the line stride in
// shared memory (padded), and the y-pass tile width in real columns.
template <int N> struct RShape {
    static_assert(N == 64 || N == 128 || N == 256 || N == 512, "register-resident lengths");
    static constexpr int M = N == 512 ? 16 : N / 16;  // threads of one 16 x M transform
    static constexpr int TPL = N == 512 ? 32 : M;     // threads per line
    static constexpr int LINES = 256 / TPL;
    static constexpr int LPW = 32 / TPL;
    static constexpr int LS = N + 1;
    static constexpr int TX = 2 * LINES;
};
constexpr int r_tile_cols(int n) {
    return n == 64 ? RShape<64>::TX : n == 128 ? RShape<128>::TX : n == 256 ? RShape<256>::TX : RShape<512>::TX;
}
constexpr int r_tile_lines(int n) { return r_tile_cols(n); }  // x-passes: real lines per CTA

// Shared memory of one CTA: its lines (64 x 65 complex values covers every
// length's LINES x LS), reused for the 16 x M exchanges; the twiddles
// W_(16M)^(t k1) at [k1][t] and W512^n (n < 256), conjugated for the
// inverse; for a DCT direction the post-twiddles (cos, sin)(pi m / (2n)),
// m < n/2.
struct R16Smem {
    float2 x[64 * 65];
    float2 tw[256];
    float2 tw2[256];
    float2 cs[256];
};

// (SM: any shared-memory struct with the tw, tw2 and cs tables of R16Smem)
template <bool INV, int N, int KIND, typename SM>
__device__ __forceinline__ void r16_tables(SM &sm) {
    constexpr int M = RShape<N>::M;
    float s, c;
    if (threadIdx.x < 16 * M) {
        const int k1 = threadIdx.x / M, t = threadIdx.x % M;
        sincospif(-(float)(t * k1) / (float)(8 * M), &s, &c);
        sm.tw[threadIdx.x] = make_float2(c, INV ? -s : s);
    }
    if (N == 512 && threadIdx.x < 256) {  // (blocks may have more than 256 threads)
        sincospif(-(float)threadIdx.x / 256.f, &s, &c);
        sm.tw2[threadIdx.x] = make_float2(c, INV ? -s : s);
    }
    if (KIND == KIND_DCT && threadIdx.x < N / 2) {
        sincospif((float)threadIdx.x / (float)(2 * N), &s, &c);
        sm.cs[threadIdx.x] = make_float2(c, s);
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

// The 16 x M four-step DFT on the 16 M values at X: thread t holds
// v[n1] = x[M n1 + t] and ends with v[j M + k2] = X[t + M j + 16 k2]
// (j < 16/M, k2 < M): a 16-point DFT, the twiddles W_(16M)^(t k1), one
// swizzled exchange through X (a permutation of M slots both ways), then
// 16/M M-point DFTs.  X is overwritten; its threads (all in one warp) must
// have finished reading X before the call (warp barriers inside, the last
// one after the exchange reads).
template <bool INV, int M, typename SM>
__device__ __forceinline__ void r_core(const SM &sm, float2 *X, int t, float2 (&v)[16]) {
    dft16<INV>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        const float2 w = sm.tw[k1 * M + t];
        v[k1] = c_mul(v[k1], w.x, w.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) X[k1 * M + (t ^ (k1 & (M - 1)))] = v[k1];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16 / M; ++j)
#pragma unroll
        for (int n2 = 0; n2 < M; ++n2) v[j * M + n2] = X[(t + M * j) * M + (n2 ^ t)];
    __syncwarp();
    if constexpr (M == 16) {
        dft16<INV>(v);
    } else if constexpr (M == 8) {
        dft8<INV, 0>(v);
        dft8<INV, 8>(v);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) dft4<INV>(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
}

// Position of a thread: complex line ln of the CTA, group h (the half of a
// 512-line), index t in its 16 x M transform.  Its inputs are the samples
// in_index(n1), its outputs the indices out_index(r).
template <int N> struct RPos {
    static constexpr int M = RShape<N>::M;
    int ln, h, t;
    __device__ __forceinline__ RPos() {
        t = threadIdx.x & (M - 1);
        ln = threadIdx.x / RShape<N>::TPL;
        h = N == 512 ? (threadIdx.x >> 4) & 1 : 0;
    }
    __device__ __forceinline__ int in_index(int n1) const {
        return N == 512 ? 16 * n1 + t + 256 * h : M * n1 + t;
    }
    __device__ __forceinline__ int out_index(int r) const {
        return N == 512 ? 2 * (t + 16 * r) + h : t + M * (r / M) + 16 * (r % M);
    }
};

// The register holding the partner X[N - k] of register r when the thread
// is its own partner (t = 0, group 0): r = j M + k2 maps to
// (M - k2) mod M for j = 0, else (16/M - j) M + M - 1 - k2.
template <int M> constexpr int self_reg(int r) {
    return r / M == 0 ? (M - r % M) % M : (16 / M - r / M) * M + (M - 1 - r % M);
}

// The transform of one line: v[n1] = the input at in_index(n1) on entry,
// v[r] = the output at out_index(r) on return.  X: the line's region
// (N values); warp barriers only (a line never spans warps).
template <bool INV, int N, typename SM>
__device__ __forceinline__ void r_fft(const SM &sm, float2 *X, const RPos<N> &q, float2 (&v)[16]) {
    if constexpr (N == 512) {  // radix-2 step: group 0 gets lo + hi, group 1 (lo - hi) W512^n
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const float2 own = v[n1];
            const float2 oth = make_float2(__shfl_xor_sync(0xffffffffu, own.x, 16),
                                           __shfl_xor_sync(0xffffffffu, own.y, 16));
            const float2 lo = q.h ? oth : own, hi = q.h ? own : oth;
            if (q.h == 0) {
                v[n1] = c_add(lo, hi);
            } else {
                const float2 w = sm.tw2[16 * n1 + q.t];
                v[n1] = c_mul(c_sub(lo, hi), w.x, w.y);
            }
        }
        r_core<INV, 16>(sm, X + 256 * q.h, q.t, v);
    } else {
        r_core<INV, RShape<N>::M>(sm, X, q.t, v);
    }
}

// Separation of the forward transform of a packed line (two real lines as
// real and imaginary part): the spectra of both, scaled by 2 (the
// conventions of the Stockham passes: half-complex for a periodic direction,
// DCT-II coefficients through the post-twiddle (c, s)_m for a wall), through
// fn(k, a_k, b_k).  X[K] pairs with X[N - K], held in register 15 - r of
// thread (M - t) mod M of the line, or (t = 0) in this thread's register
// self_reg(r); at 512 the odd outputs pair within group 1 with thread
// 15 - t, register 15 - r.
template <int N, int KIND, typename SM, typename F>
__device__ __forceinline__ void r_separate(const float2 (&v)[16], const RPos<N> &q, const SM &sm,
                                           F &&fn) {
    constexpr int M = RShape<N>::M;
    const int lane = threadIdx.x & 31;
    const int src = (N != 512 || q.h == 0) ? ((lane & ~(M - 1)) | ((M - q.t) & (M - 1)))
                                           : (16 | (15 - q.t));
    const bool self = q.h == 0 && q.t == 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const float qx = __shfl_sync(0xffffffffu, v[15 - r].x, src);
        const float qy = __shfl_sync(0xffffffffu, v[15 - r].y, src);
        const float2 z = v[r];
        const float2 y = self ? v[self_reg<M>(r)] : make_float2(qx, qy);
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
__device__ __forceinline__ void r_combine(float2 (&v)[16], const RPos<N> &q, const SM &sm, G &&get) {
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        const int k = q.in_index(n1);
        const float2 o = get(k), p = get((N - k) & (N - 1));  // indices k and n - k
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

// ---- y-passes: one tile = TX real columns (bx) of one z-plane of an
// (nz, N, nx) FP32 array, transformed along y in place.  The N x TX tile
// (8192 values at every length) moves between global and shared memory as
// elements e = lane + 32 (warp + 8 i): each warp access is 32 consecutive
// columns (TX >= 32) or two rows of 16 (TX = 16).  Column 2l + c of the tile
// is component c of complex line l.  Forward: real columns -> spectra
// scaled by 2 (half-complex, or DCT-II for a wall direction); inverse: the
// reverse, unscaled.
template <bool INV, int N, int KIND>
__device__ __forceinline__ void ypass_r_tile(int nx, float *data, int bx, int kplane, R16Smem &sm) {
    constexpr int TX = RShape<N>::TX, LS = RShape<N>::LS;
    static_assert(N * TX == 32 * 256, "one tile is 32 values per thread");
    const RPos<N> q;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = bx * TX;
    float *plane = data + (size_t)kplane * N * nx + c0;
    float *sf = (float *)sm.x;
    float2 *X = sm.x + q.ln * LS;
    // element i of this thread: (row, col) of e = lane + 32 (warp + 8 i); for
    // TX <= 32 the column is the thread's own (one pointer per thread)
    auto rc = [&](int i, int &row, int &col) {
        const int e = lane + 32 * (warp + 8 * i);
        row = e / TX;
        col = e % TX;
    };
    // one column per thread (TX <= 32): its pointers and the rows linear in i
    constexpr int RPW = TX <= 32 ? 32 / TX : 1;
    const int tcol = lane % TX, rsub = lane / TX;
    const bool tcol_ok = c0 + tcol < nx;
    float *gcol = plane + tcol;
    float *scol = sf + (tcol >> 1) * (2 * LS) + (tcol & 1);
    auto row_of = [&](int i) { return i * (8 * RPW) + warp * RPW + rsub; };
    // 1. stage the tile (sixteen loads in flight)
#pragma unroll 1
    for (int i0 = 0; i0 < 32; i0 += 16) {
        float r[16];
        if constexpr (TX <= 32) {
#pragma unroll
            for (int u = 0; u < 16; ++u) r[u] = tcol_ok ? gcol[(size_t)row_of(i0 + u) * nx] : 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) scol[2 * row_of(i0 + u)] = r[u];
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                int row, col;
                rc(i0 + u, row, col);
                r[u] = c0 + col < nx ? plane[(size_t)row * nx + col] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                int row, col;
                rc(i0 + u, row, col);
                sf[(col >> 1) * (2 * LS) + 2 * row + (col & 1)] = r[u];
            }
        }
    }
    __syncthreads();
    float2 v[16];
    if (!INV) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
    } else {
        r_combine<N, KIND>(v, q, sm, [&](int k) { return X[k]; });
    }
    __syncwarp();  // the line's region is the exchange buffer next
    r_fft<INV, N>(sm, X, q, v);
    if (!INV) {
        r_separate<N, KIND>(v, q, sm, [&](int k, float a, float b) { X[k] = make_float2(a, b); });
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) X[r_src<N, KIND>(q.out_index(r))] = v[r];
    }
    __syncthreads();
    // 2. write the tile back
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if constexpr (TX <= 32) {
            const int row = row_of(i);
            if (tcol_ok) gcol[(size_t)row * nx] = scol[2 * row];
        } else {
            int row, col;
            rc(i, row, col);
            if (c0 + col < nx) plane[(size_t)row * nx + col] = sf[(col >> 1) * (2 * LS) + 2 * row + (col & 1)];
        }
    }
    __syncthreads();  // the buffer is free for the next tile
}

// y-pass over ntiles = ygx x nz tiles (ygx = ceil(nx / TX)); the signature of
// k_ypass, so the plan can launch either.  conv: return at once when the
// refinement has converged.
template <bool INV, int N, int KIND>
__global__ void __launch_bounds__(256, 4) k_ypass_r(int nx, int ny, FFTDesc D, int TX, float *data,
                                                    const int *conv, int ygx, int ntiles) {
    (void)ny;
    (void)D;
    (void)TX;
    __shared__ R16Smem sm;
    if (conv && *(volatile const int *)conv) return;
    r16_tables<INV, N, KIND>(sm);
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int kplane = tile / ygx;
        ypass_r_tile<INV, N, KIND>(nx, data, tile - kplane * ygx, kplane, sm);
    }
}

// ---- x-passes: 2 LINES real lines of the [nz][ny] line set per CTA.  A
// warp owns LPW complex lines (2 LPW real rows, rows 2l and 2l + 1 packed as
// line l); it stages them row by row through their shared-memory regions
// (lane = x mod 32: 128-byte accesses), transforms them and writes them back
// the same way, with warp barriers only.

// The warp's first line (of the CTA).
template <int N> __device__ __forceinline__ int r_warp_line() {
    return (threadIdx.x >> 5) * RShape<N>::LPW;
}

// A warp's rows hold 2 LPW x N = 32 x 32 values at every length: slot s
// (s < 32) of a lane is row s / (N/32), x = lane + 32 (s mod N/32).
template <int N> __device__ __forceinline__ int r_slot_row(int s) { return s / (N / 32); }
template <int N> __device__ __forceinline__ int r_slot_x(int s) {
    return (threadIdx.x & 31) + 32 * (s % (N / 32));
}
// The shared-memory float of (row r of the warp, x): line l0 + r/2, component r & 1.
template <int N> __device__ __forceinline__ int r_slot_f(int r, int x) {
    return (r_warp_line<N>() + (r >> 1)) * (2 * RShape<N>::LS) + 2 * x + (r & 1);
}

// Rows of the warp from an FP32 array [nlines][N] into the line regions
// (zeros past the last line), all 32 loads of a lane in flight.
template <int N>
__device__ __forceinline__ void r_rows_in(const float *src, int row0, int nlines, R16Smem &sm) {
    float *sf = (float *)sm.x;
    float x[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        const int row = row0 + r_slot_row<N>(s);
        x[s] = row < nlines ? src[(size_t)row * N + r_slot_x<N>(s)] : 0.f;
    }
#pragma unroll
    for (int s = 0; s < 32; ++s) sf[r_slot_f<N>(r_slot_row<N>(s), r_slot_x<N>(s))] = x[s];
    __syncwarp();
}

// Rows of the warp from the line regions back to an FP32 array.
template <int N>
__device__ __forceinline__ void r_rows_out(float *dst, int row0, int nlines, const R16Smem &sm) {
    const float *sf = (const float *)sm.x;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        const int row = row0 + r_slot_row<N>(s);
        if (row < nlines) dst[(size_t)row * N + r_slot_x<N>(s)] = sf[r_slot_f<N>(r_slot_row<N>(s), r_slot_x<N>(s))];
    }
    __syncwarp();
}

// Forward transform of the staged lines: inputs from the line region X,
// the spectra back into it.
template <int N, int KIND>
__device__ __forceinline__ void r_forward_line(const R16Smem &sm, float2 *X, const RPos<N> &q) {
    float2 v[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
    __syncwarp();  // the line's region is the exchange buffer next
    r_fft<false, N>(sm, X, q, v);
    r_separate<N, KIND>(v, q, sm, [&](int k, float a, float b) { X[k] = make_float2(a, b); });
}

// The transform of the stored FP32 residual (refinement sweeps), in place:
// the mode XF_MIX_LOAD of k_xfwd.
template <int N, int KIND>
__global__ void __launch_bounds__(256, 4) k_xfwd_r_load(GridDev g, FFTDesc D, int L, XArgs a,
                                                        int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    if (*(volatile const int *)&a.st->converged) return;
    r16_tables<false, N, KIND>(sm);
    __syncthreads();
    const RPos<N> q;
    const int nlines = g.ny * g.nz;
    float *data = (float *)a.out;
    float2 *X = sm.x + q.ln * RShape<N>::LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * r_tile_lines(N) + 2 * r_warp_line<N>();
        if constexpr (N >= 256) {
            // a 16-thread group reads and writes 64 consecutive bytes of each
            // of its line's two rows at a time: direct global access
            const int ra = tile * r_tile_lines(N) + 2 * q.ln;
            const bool oka = ra < nlines, okb = ra + 1 < nlines;
            float *la = data + (size_t)ra * N, *lb = la + N;
            float2 v[16];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
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
// f = rho0 D(q') in FP64 (stored, and max|f| recorded), then the forward
// transform of its FP32 image sigma f.  f is formed row by row (lane = x mod
// 32, coalesced) into the line regions.
template <int N, int KIND>
__global__ void __launch_bounds__(256, 4) k_xfwd_r_divq(GridDev g, FFTDesc D, int L, XArgs a,
                                                        int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    r16_tables<false, N, KIND>(sm);
    __syncthreads();
    const RPos<N> q;
    const int nlines = g.ny * g.nz, l0 = r_warp_line<N>();
    constexpr int LS = RShape<N>::LS;
    const float scale32 = (float)g.sigma;
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
                    const double cz = g.dvz[k];
#pragma unroll 4
                    for (int i = 0; i < N / 32; ++i) {
                        const int x = lane + 32 * i;
                        const double f = div_q<false>(g, x, j, k, g.dvx, g.dvy, cz, a.qx, a.qy, a.qz);
                        a.f_out[(size_t)row * N + x] = f;
                        mx = umax64(mx, absbits(f));
                        dr[2 * x] = f64_to_f32_shift(f, 0) * scale32;
                    }
                } else {
                    for (int i = 0; i < N / 32; ++i) dr[2 * (lane + 32 * i)] = 0.f;
                }
            }
        } else {  // short rows: the warp's 32 slots per lane
#pragma unroll 4
            for (int s = 0; s < 32; ++s) {
                const int r = r_slot_row<N>(s), x = r_slot_x<N>(s), row = row0 + r;
                float val = 0.f;
                if (row < nlines) {
                    const int k = fdiv(row, g.ny, g.rny), j = row - k * g.ny;
                    const double f = div_q<false>(g, x, j, k, g.dvx, g.dvy, g.dvz[k], a.qx, a.qy, a.qz);
                    a.f_out[(size_t)row * N + x] = f;
                    mx = umax64(mx, absbits(f));
                    val = f64_to_f32_shift(f, 0) * scale32;
                }
                sf[r_slot_f<N>(r, x)] = val;
            }
        }
        __syncwarp();
        if constexpr (N >= 256) {  // the spectra straight to global memory
            float2 v[16];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) v[n1] = X[r_src<N, KIND>(q.in_index(n1))];
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
__global__ void __launch_bounds__(256, 4) k_xinv_r(GridDev g, FFTDesc D, int L, const float *in,
                                                   double *p, const DevStats *st, int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    if (MODE == XI_ACCUM && *(volatile const int *)&st->converged) return;
    r16_tables<true, N, KIND>(sm);
    __syncthreads();
    const int ef = MODE == XI_ACCUM ? exp_of_bits(*(volatile const unsigned long long *)&st->fmax_bits) : 0;
    const RPos<N> q;
    const int nlines = g.ny * g.nz, l0 = r_warp_line<N>();
    float2 *X = sm.x + q.ln * RShape<N>::LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * r_tile_lines(N) + 2 * l0;
        r_rows_in<N>(in, row0, nlines, sm);
        float2 v[16];
        r_combine<N, KIND>(v, q, sm, [&](int k) { return X[k]; });
        __syncwarp();  // the line's region is the exchange buffer next
        r_fft<true, N>(sm, X, q, v);
#pragma unroll
        for (int r = 0; r < 16; ++r) X[r_src<N, KIND>(q.out_index(r))] = v[r];
        __syncwarp();
        // p (or p += delta) by slots (lane = x mod 32), eight values of p in
        // flight per lane
        const float *sf = (const float *)sm.x;
#pragma unroll
        for (int s0 = 0; s0 < 32; s0 += 8) {
            double qv[8];
            if (MODE == XI_ACCUM) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int row = row0 + r_slot_row<N>(s0 + u);
                    qv[u] = row < nlines ? p[(size_t)row * N + r_slot_x<N>(s0 + u)] : 0.0;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r_slot_row<N>(s0 + u), x = r_slot_x<N>(s0 + u), row = row0 + r;
                const double d = f32_to_f64_shift(sf[r_slot_f<N>(r, x)], ef);
                if (row < nlines) p[(size_t)row * N + x] = MODE == XI_ACCUM ? qv[u] + d : d;
            }
        }
        __syncwarp();  // the line regions are rewritten by the next tile
    }
}

}  // namespace fz
