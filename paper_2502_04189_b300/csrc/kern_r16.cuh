// Register-resident FP32 transforms of periodic length 256 (mixed mode).
//
// The y-passes of the FP32 solve (Sec. 3.2: real FFTs along the periodic
// directions) for ny = 256.  The DFT of length 256 is split as 16 x 16 (the
// four-step form of the Cooley-Tukey factorisation): with n = 16 n1 + n2 and
// k = k1 + 16 k2,
//     X[k1 + 16 k2] = sum_n2 W16^(n2 k2) [ W256^(n2 k1) sum_n1 x[16 n1 + n2] W16^(n1 k1) ],
// W_N = exp(-2 pi i / N) (the inverse uses the conjugates; neither direction
// is scaled).  A complex line (two real columns, real and imaginary part) is
// held by 16 threads: thread t first owns the samples x[16 n1 + t],
// computes their 16-point DFT in
// registers and applies the twiddles W256^(t k1); one pass through shared
// memory then hands thread t the values of k1 = t, whose 16-point DFT gives
// X[t + 16 k2].  The separation of the two real spectra (forward) pairs X[k]
// with X[256 - k], held by thread (16 - t) mod 16 of the same line, through
// warp shuffles; the inverse combination reads both rows of a pair.  The
// tile is staged through shared memory with one 128-byte row segment per
// warp access (a load straight into the per-thread order would touch 16 rows
// per warp instruction).
//
// Same arithmetic as the Stockham passes (about 11 FP32 multiply-adds per
// real point); what it removes is their per-stage shared-memory round trips,
// index divisions and the select work of the FMA-form twiddles.
#pragma once
#include "kern_passes.cuh"

namespace fz {

constexpr int R16_N = 256;
constexpr int R16_TX = 32;  // real columns of one CTA (16 complex lines x 16 threads)

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

// Shared memory of one CTA: its 16 complex lines (line stride R16_LS, so
// that both the row-wise staging and the per-line accesses are free of bank
// conflicts), reused for the 16 x 16 exchange, and the twiddles W256^(n2 k1)
// at [k1][n2] (conjugated for the inverse).
constexpr int R16_LS = R16_N + 1;
struct R16Smem {
    float2 x[16 * R16_LS];
    float2 tw[R16_N];
};

template <bool INV>
__device__ __forceinline__ void r16_tables(R16Smem &sm) {
    const int n2 = threadIdx.x & 15, k1 = threadIdx.x >> 4;
    float s, c;
    sincospif(-(float)(n2 * k1) / 128.f, &s, &c);
    sm.tw[threadIdx.x] = make_float2(c, INV ? -s : s);
}

// Steps 1-3 of the four-step DFT on line X: thread t holds v[n1] =
// x[16 n1 + t] and ends with v[k2] = X[t + 16 k2].  X is overwritten; all
// threads must have finished reading X before the call (barriers inside,
// the last one after the exchange reads).  WARP: every line lives in one
// warp (the x-passes), so warp barriers suffice.
template <bool WARP>
__device__ __forceinline__ void r16_sync() {
    if (WARP) __syncwarp();
    else __syncthreads();
}
template <bool INV, bool WARP = false>
__device__ __forceinline__ void r16_fft(const R16Smem &sm, float2 *X, int t, float2 (&v)[16]) {
    dft16<INV>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        const float2 w = sm.tw[k1 * 16 + t];
        v[k1] = c_mul(v[k1], w.x, w.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) X[k1 * 16 + (t ^ k1)] = v[k1];  // conflict-free both ways
    r16_sync<WARP>();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = X[t * 16 + (n2 ^ t)];
    r16_sync<WARP>();
    dft16<INV>(v);
}

// One tile: 32 real columns (bx) of one z-plane of an (nz, 256, nx) FP32
// array, transformed along y in place.  Forward: real columns -> half-complex
// spectra scaled by 2 (the convention of the Stockham passes); inverse: the
// reverse, unscaled.  Rows move between global and shared memory one warp
// per row (32 columns, one 128-byte segment); column 2l + e of the tile is
// component e of complex line l.
template <bool INV>
__device__ __forceinline__ void ypass_r16_tile(int nx, float *data, int bx, int kplane, R16Smem &sm) {
    const int ln = threadIdx.x >> 4, t = threadIdx.x & 15;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool col_ok = bx * R16_TX + lane < nx;
    float *gcol = data + (size_t)kplane * R16_N * nx + bx * R16_TX + lane;
    float *scol = (float *)sm.x + (lane >> 1) * (2 * R16_LS) + (lane & 1);
    float2 *X = sm.x + ln * R16_LS;
    // 1. stage the tile: warp w moves rows w, w + 8, ... (eight loads in flight)
#pragma unroll 1
    for (int i0 = 0; i0 < R16_N / 8; i0 += 16) {
        float r[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) r[u] = col_ok ? gcol[(size_t)(warp + 8 * (i0 + u)) * nx] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) scol[2 * (warp + 8 * (i0 + u))] = r[u];
    }
    __syncthreads();
    float2 v[16];
    if (!INV) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) v[n1] = X[16 * n1 + t];
    } else {
        // combine the half-complex spectra of the two real lines into Z[k]
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int k = t + 16 * n1;
            const float2 o = X[k], p = X[(R16_N - k) & (R16_N - 1)];  // rows k and n - k
            if (k == 0 || k == R16_N / 2) v[n1] = o;
            else if (k < R16_N / 2) v[n1] = make_float2(o.x - p.y, p.x + o.y);
            else v[n1] = make_float2(p.x + o.y, p.y - o.x);
        }
    }
    __syncthreads();
    r16_fft<INV>(sm, X, t, v);
    if (!INV) {
        // separation: X[k] pairs with X[256 - k] = the partner's register
        // 15 - k2 (t != 0) or this thread's register (16 - k2) mod 16 (t = 0)
        const int src = (threadIdx.x & 16) | ((16 - t) & 15);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const float qx = __shfl_sync(0xffffffffu, v[15 - k2].x, src);
            const float qy = __shfl_sync(0xffffffffu, v[15 - k2].y, src);
            const float2 z = v[k2];
            const float2 y = (t == 0) ? v[(16 - k2) & 15] : make_float2(qx, qy);
            const int k = t + 16 * k2;
            // k <= n/2: (Re A_k, Re B_k) x 2; k > n/2: (Im A_m, Im B_m) x 2, m = n - k
            X[k] = k <= R16_N / 2 ? make_float2(z.x + y.x, z.y + y.y) : make_float2(y.y - z.y, z.x - y.x);
        }
    } else {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) X[t + 16 * k2] = v[k2];
    }
    __syncthreads();
    // 2. write the tile back, one row per warp
#pragma unroll
    for (int i = 0; i < R16_N / 8; ++i) {
        const int row = warp + 8 * i;
        if (col_ok) gcol[(size_t)row * nx] = scol[2 * row];
    }
    __syncthreads();  // the buffer is free for the next tile
}

// y-pass over ntiles = ygx x nz tiles (ygx = ceil(nx / 32)); the signature of
// k_ypass, so the plan can launch either.  conv: return at once when the
// refinement has converged.
template <bool INV>
__global__ void __launch_bounds__(256, 4) k_ypass_r16(int nx, int ny, FFTDesc D, int TX, float *data,
                                                   const int *conv, int ygx, int ntiles) {
    (void)ny;
    (void)D;
    (void)TX;
    __shared__ R16Smem sm;
    if (conv && *(volatile const int *)conv) return;
    r16_tables<INV>(sm);
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int kplane = tile / ygx;
        ypass_r16_tile<INV>(nx, data, tile - kplane * ygx, kplane, sm);
    }
}

// ---- x-passes (nx = 256): 32 real lines of the [nz][ny] line set per CTA;
// the warp of complex line l (real lines 2l, 2l + 1 of the tile) loads, transforms
// and stores it alone, so only warp barriers are needed.  At each register
// index the 16 threads of a line touch 64 consecutive bytes of each of its
// two rows.

// Separation of the forward transform (see the y-pass) through fn(k, a, b).
template <typename F>
__device__ __forceinline__ void r16_separate(const float2 (&v)[16], int t, F &&fn) {
    const int src = (threadIdx.x & 16) | ((16 - t) & 15);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const float qx = __shfl_sync(0xffffffffu, v[15 - k2].x, src);
        const float qy = __shfl_sync(0xffffffffu, v[15 - k2].y, src);
        const float2 z = v[k2];
        const float2 y = (t == 0) ? v[(16 - k2) & 15] : make_float2(qx, qy);
        const int k = t + 16 * k2;
        if (k <= R16_N / 2) fn(k, z.x + y.x, z.y + y.y);
        else fn(k, y.y - z.y, z.x - y.x);
    }
}

// Combination of the inverse transform: v[n1] = Z[t + 16 n1] from the
// half-complex spectra read through get(k) = (a[k], b[k]).
template <typename G>
__device__ __forceinline__ void r16_combine(float2 (&v)[16], int t, G &&get) {
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        const int k = t + 16 * n1;
        const float2 o = get(k), p = get((R16_N - k) & (R16_N - 1));
        if (k == 0 || k == R16_N / 2) v[n1] = o;
        else if (k < R16_N / 2) v[n1] = make_float2(o.x - p.y, p.x + o.y);
        else v[n1] = make_float2(p.x + o.y, p.y - o.x);
    }
}

// The transform of the stored FP32 residual (refinement sweeps), in place:
// the mode XF_MIX_LOAD of k_xfwd.
__global__ void __launch_bounds__(256, 4) k_xfwd_r16_load(GridDev g, FFTDesc D, int L, XArgs a,
                                                          int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    if (*(volatile const int *)&a.st->converged) return;
    r16_tables<false>(sm);
    __syncthreads();
    const int nlines = g.ny * g.nz, ln = threadIdx.x >> 4, t = threadIdx.x & 15;
    float *data = (float *)a.out;
    float2 *X = sm.x + ln * R16_LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ra = tile * 32 + 2 * ln;
        const bool oka = ra < nlines, okb = ra + 1 < nlines;
        float *la = data + (size_t)ra * R16_N, *lb = la + R16_N;
        float2 v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1)
            v[n1] = make_float2(oka ? la[16 * n1 + t] : 0.f, okb ? lb[16 * n1 + t] : 0.f);
        r16_fft<false, true>(sm, X, t, v);
        r16_separate(v, t, [&](int k, float va, float vb) {
            if (oka) la[k] = va;
            if (okb) lb[k] = vb;
        });
    }
}

// Inverse x-pass to p (FP64): XI_STORE p = the FP32 solution, XI_ACCUM
// p += delta 2^e (e: exponent of max|f|); the modes of k_xinv.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_xinv_r16(GridDev g, FFTDesc D, int L, const float *in,
                                                     double *p, const DevStats *st, int ntiles) {
    (void)D;
    (void)L;
    __shared__ R16Smem sm;
    if (MODE == XI_ACCUM && *(volatile const int *)&st->converged) return;
    r16_tables<true>(sm);
    __syncthreads();
    const int ef = MODE == XI_ACCUM ? exp_of_bits(*(volatile const unsigned long long *)&st->fmax_bits) : 0;
    const int nlines = g.ny * g.nz, ln = threadIdx.x >> 4, t = threadIdx.x & 15;
    float2 *X = sm.x + ln * R16_LS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ra = tile * 32 + 2 * ln;
        const bool oka = ra < nlines, okb = ra + 1 < nlines;
        const float *ia = in + (size_t)ra * R16_N, *ib = ia + R16_N;
        float2 v[16];
        r16_combine(v, t, [&](int k) { return make_float2(oka ? ia[k] : 0.f, okb ? ib[k] : 0.f); });
        r16_fft<true, true>(sm, X, t, v);
        double *pa = p + (size_t)ra * R16_N, *pb = pa + R16_N;
        if (MODE == XI_STORE) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int x = t + 16 * k2;
                if (oka) pa[x] = f32_to_f64_shift(v[k2].x, 0);
                if (okb) pb[x] = f32_to_f64_shift(v[k2].y, 0);
            }
        } else {
            // delta through the line's exchange buffer, then p += delta row by
            // row: lane = x mod 32, eight loads of p in flight per lane
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) X[t + 16 * k2] = v[k2];
            __syncwarp();
            const int lane = threadIdx.x & 31, l0 = ln & ~1;
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {  // rows a, b of the warp's two lines
                const int row = tile * 32 + 2 * l0 + r;
                if (row < nlines) {
                    double *pr = p + (size_t)row * R16_N + lane;
                    const float *dr = (const float *)(sm.x + (l0 + (r >> 1)) * R16_LS) + (r & 1) + 2 * lane;
                    double q[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) q[i] = pr[32 * i];
#pragma unroll
                    for (int i = 0; i < 8; ++i) pr[32 * i] = q[i] + f32_to_f64_shift(dr[64 * i], ef);
                }
            }
            __syncwarp();  // the buffer is rewritten by the next tile
        }
    }
}

}  // namespace fz
