// Register-resident FP32 transforms of periodic length 256 and 512 (mixed mode).
//
// The FP32 transform passes of the mixed-precision solve (Sec. 3.2: real
// FFTs along the periodic directions) for n = 256 and 512.  The DFT of length
// 256 is split as 16 x 16 (the four-step form of the Cooley-Tukey
// factorisation): with n = 16 n1 + n2 and k = k1 + 16 k2,
//     X[k1 + 16 k2] = sum_n2 W16^(n2 k2) [ W256^(n2 k1) sum_n1 x[16 n1 + n2] W16^(n1 k1) ],
// W_N = exp(-2 pi i / N) (the inverse uses the conjugates; neither direction
// is scaled).  A complex line (two real columns, real and imaginary part) is
// held by 16 threads: thread t first owns the samples x[16 n1 + t],
// computes their 16-point DFT in registers and applies the twiddles
// W256^(t k1); one pass through shared
// memory then hands thread t the values of k1 = t, whose 16-point DFT gives
// X[t + 16 k2].  The separation of the two real spectra (forward) pairs X[k]
// with X[256 - k], held by thread (16 - t) mod 16 of the same line, through
// warp shuffles; the inverse combination reads both rows of a pair.  The
// tile is staged through shared memory with one 128-byte row segment per
// warp access (a load straight into the per-thread order would touch 16 rows
// per warp instruction).
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

// Launch shape of a length: complex lines per CTA of 256 threads (16
// threads per line at 256, a warp per line at 512), the line stride in
// shared memory (padded) and the y-pass tile width in real columns.
template <int N> struct RShape {
    static_assert(N == 256 || N == 512, "register-resident lengths");
    static constexpr int LINES = N == 256 ? 16 : 8;
    static constexpr int LS = N + 1;
    static constexpr int TX = 2 * LINES;
};
constexpr int r_tile_cols(int n) { return n == 256 ? RShape<256>::TX : RShape<512>::TX; }
constexpr int r_tile_lines(int n) { return n == 256 ? 2 * RShape<256>::LINES : 2 * RShape<512>::LINES; }

// Shared memory of one CTA: its lines (16 x 257 >= 8 x 513 complex values),
// reused for the 16 x 16 exchanges; the twiddles W256^(n2 k1) at [k1][n2]
// and W512^n (n < 256), conjugated for the inverse; for a DCT direction the
// post-twiddles (cos, sin)(pi m / (2n)), m < n/2.
struct R16Smem {
    float2 x[16 * 257];
    float2 tw[256];
    float2 tw2[256];
    float2 cs[256];
};

template <bool INV, int N, int KIND>
__device__ __forceinline__ void r16_tables(R16Smem &sm) {
    const int n2 = threadIdx.x & 15, k1 = threadIdx.x >> 4;
    float s, c;
    sincospif(-(float)(n2 * k1) / 128.f, &s, &c);
    sm.tw[threadIdx.x] = make_float2(c, INV ? -s : s);
    sincospif(-(float)threadIdx.x / 256.f, &s, &c);
    sm.tw2[threadIdx.x] = make_float2(c, INV ? -s : s);
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

// Steps 1-3 of the four-step DFT on the 256 values at X: thread t holds
// v[n1] = x[16 n1 + t] and ends with v[k2] = X[t + 16 k2].  X is overwritten;
// its threads (all in one warp) must have finished reading X before the call
// (warp barriers inside, the last one after the exchange reads).
template <bool INV>
__device__ __forceinline__ void r16_fft(const R16Smem &sm, float2 *X, int t, float2 (&v)[16]) {
    dft16<INV>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        const float2 w = sm.tw[k1 * 16 + t];
        v[k1] = c_mul(v[k1], w.x, w.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) X[k1 * 16 + (t ^ k1)] = v[k1];  // conflict-free both ways
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = X[t * 16 + (n2 ^ t)];
    __syncwarp();
    dft16<INV>(v);
}

// Position of a thread: complex line ln of the CTA, group h (the half of a
// 512-line), index t in the group.  Its inputs are the samples
// 16 n1 + t + 256 h, its outputs the indices out_index(k2).
template <int N> struct RPos {
    int ln, h, t;
    __device__ __forceinline__ RPos() {
        t = threadIdx.x & 15;
        ln = N == 256 ? threadIdx.x >> 4 : threadIdx.x >> 5;
        h = N == 256 ? 0 : (threadIdx.x >> 4) & 1;
    }
    __device__ __forceinline__ int in_index(int n1) const { return 16 * n1 + t + 256 * h; }
    __device__ __forceinline__ int out_index(int k2) const {
        return N == 256 ? t + 16 * k2 : 2 * (t + 16 * k2) + h;
    }
};

// The transform of one line: v[n1] = the input at in_index(n1) on entry,
// v[k2] = the output at out_index(k2) on return.  X: the line's region
// (N values); warp barriers only (a line never spans warps).
template <bool INV, int N>
__device__ __forceinline__ void r_fft(const R16Smem &sm, float2 *X, const RPos<N> &q, float2 (&v)[16]) {
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
    }
    r16_fft<INV>(sm, X + 256 * q.h, q.t, v);
}

// Separation of the forward transform of a packed line (two real lines as
// real and imaginary part): the spectra of both, scaled by 2 (the
// conventions of the Stockham passes: half-complex for a periodic direction,
// DCT-II coefficients through the post-twiddle (c, s)_m for a wall), through
// fn(k, a_k, b_k).  X[K] pairs with X[N - K]: at 256 the partner's register
// 15 - k2 of thread (16 - t) mod 16, or this thread's register (16 - k2)
// mod 16 (t = 0); at 512 the odd outputs pair within group 1 with thread
// 15 - t, register 15 - k2.
template <int N, int KIND, typename F>
__device__ __forceinline__ void r_separate(const float2 (&v)[16], const RPos<N> &q,
                                           const R16Smem &sm, F &&fn) {
    const int lane = threadIdx.x & 31;
    const int src = (N == 256 || q.h == 0) ? ((lane & 16) | ((16 - q.t) & 15)) : (16 | (15 - q.t));
    const bool self = q.h == 0 && q.t == 0;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const float qx = __shfl_sync(0xffffffffu, v[15 - k2].x, src);
        const float qy = __shfl_sync(0xffffffffu, v[15 - k2].y, src);
        const float2 z = v[k2];
        const float2 y = self ? v[(16 - k2) & 15] : make_float2(qx, qy);
        const int k = q.out_index(k2);
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
template <int N, int KIND, typename G>
__device__ __forceinline__ void r_combine(float2 (&v)[16], const RPos<N> &q, const R16Smem &sm,
                                          G &&get) {
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
// (nz, N, nx) FP32 array, transformed along y in place.  Rows move between
// global and shared memory a warp at a time (32 columns of one row at 256,
// 16 columns of two rows at 512); column 2l + e of the tile is component e
// of complex line l.  Forward: real columns -> spectra scaled by 2
// (half-complex, or DCT-II for a wall direction); inverse: the reverse,
// unscaled.
template <bool INV, int N, int KIND>
__device__ __forceinline__ void ypass_r_tile(int nx, float *data, int bx, int kplane, R16Smem &sm) {
    constexpr int TX = RShape<N>::TX, LS = RShape<N>::LS;
    constexpr int RPW = 32 / TX;  // rows per warp access
    const RPos<N> q;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = lane % TX, rsub = lane / TX;
    const bool col_ok = bx * TX + col < nx;
    float *gcol = data + (size_t)kplane * N * nx + bx * TX + col;
    float *scol = (float *)sm.x + (col >> 1) * (2 * LS) + (col & 1);
    float2 *X = sm.x + q.ln * LS;
    auto row_of = [&](int i) { return i * (8 * RPW) + warp * RPW + rsub; };  // i < 32
    // 1. stage the tile (sixteen loads in flight)
#pragma unroll 1
    for (int i0 = 0; i0 < 32; i0 += 16) {
        float r[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) r[u] = col_ok ? gcol[(size_t)row_of(i0 + u) * nx] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) scol[2 * row_of(i0 + u)] = r[u];
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
        for (int k2 = 0; k2 < 16; ++k2) X[r_src<N, KIND>(q.out_index(k2))] = v[k2];
    }
    __syncthreads();
    // 2. write the tile back
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int row = row_of(i);
        if (col_ok) gcol[(size_t)row * nx] = scol[2 * row];
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

// ---- x-passes: 2 LINES real lines of the [nz][ny] line set per CTA; a
// line's threads load, transform and store it alone (warp barriers only).
// At each register index the 16 threads of a group touch 64 consecutive
// bytes of each of the two rows of their line.

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
    }
}

// The first x-pass of the mixed solve (the mode XF_MIX_DIVQ of k_xfwd):
// f = rho0 D(q') in FP64 (stored, and max|f| recorded), then the forward
// transform of its FP32 image sigma f.  f is formed row by row (lane = x mod
// 32, coalesced) into the line's region of shared memory, from which the
// threads of the line take their inputs.
template <int N, int KIND>
__global__ void __launch_bounds__(256, 4) k_xfwd_r_divq(GridDev g, FFTDesc D, int L, XArgs a,
                                                        int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    r16_tables<false, N, KIND>(sm);
    __syncthreads();
    const RPos<N> q;
    const int nlines = g.ny * g.nz, lane = threadIdx.x & 31;
    constexpr int LS = RShape<N>::LS;
    const int l0 = N == 256 ? (q.ln & ~1) : q.ln;  // the warp's first line
    constexpr int WROWS = N == 256 ? 4 : 2;         // real rows of the warp
    const float scale32 = (float)g.sigma;
    float *out = (float *)a.out;
    float2 *X = sm.x + q.ln * LS;
    unsigned long long mx = 0ull;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll 1
        for (int r = 0; r < WROWS; ++r) {
            const int row = tile * r_tile_lines(N) + 2 * l0 + r;
            float *dr = (float *)(sm.x + (l0 + (r >> 1)) * LS) + (r & 1);
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
        __syncwarp();
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
    const int nlines = g.ny * g.nz;
    constexpr int LS = RShape<N>::LS;
    float2 *X = sm.x + q.ln * LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ra = tile * r_tile_lines(N) + 2 * q.ln;
        const bool oka = ra < nlines, okb = ra + 1 < nlines;
        const float *ia = in + (size_t)ra * N, *ib = ia + N;
        float2 v[16];
        r_combine<N, KIND>(v, q, sm, [&](int k) { return make_float2(oka ? ia[k] : 0.f, okb ? ib[k] : 0.f); });
        r_fft<true, N>(sm, X, q, v);
        if (MODE == XI_STORE) {
            double *pa = p + (size_t)ra * N, *pb = pa + N;
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int x = r_src<N, KIND>(q.out_index(k2));
                if (oka) pa[x] = f32_to_f64_shift(v[k2].x, 0);
                if (okb) pb[x] = f32_to_f64_shift(v[k2].y, 0);
            }
        } else {
            // delta through the line's region, then p += delta row by row:
            // lane = x mod 32, eight loads of p in flight per lane
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) X[r_src<N, KIND>(q.out_index(k2))] = v[k2];
            __syncwarp();
            const int lane = threadIdx.x & 31;
            const int l0 = N == 256 ? (q.ln & ~1) : q.ln;  // the warp's first line
            constexpr int WROWS = N == 256 ? 4 : 2;         // real rows of the warp
#pragma unroll 1
            for (int r = 0; r < WROWS; ++r) {
                const int row = tile * r_tile_lines(N) + 2 * l0 + r;
                if (row < nlines) {
                    double *pr = p + (size_t)row * N + lane;
                    const float *dr = (const float *)(sm.x + (l0 + (r >> 1)) * LS) + (r & 1) + 2 * lane;
#pragma unroll
                    for (int i0 = 0; i0 < N / 32; i0 += 8) {
                        double qv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) qv[i] = pr[32 * (i0 + i)];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            pr[32 * (i0 + i)] = qv[i] + f32_to_f64_shift(dr[64 * (i0 + i)], ef);
                    }
                }
            }
        }
        __syncwarp();  // the line's region is rewritten by the next tile
    }
}

}  // namespace fz
