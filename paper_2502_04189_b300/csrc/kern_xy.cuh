// Fused two-dimensional x-y transform passes of the FP32 solve (mixed mode,
// nx = ny = N with N = 256 or 512, periodic or wall x and y) on a
// thread-block cluster: one z-plane per cluster of XY_CL CTAs, exchanged
// through distributed shared memory instead of a round trip through HBM.
//
// Forward (k_xy_fwd): CTA c of the cluster owns rows [cR, cR + R) of the
// plane (R = N / XY_CL).  It transforms them along x with the
// register-resident 16 x M four-step FFT of kern_r16.cuh (two rows packed as
// one complex line), leaving the row spectra in its shared memory, row by
// row.  After a cluster barrier it owns the columns [cR, cR + R) instead:
// each thread reads its 16 values of a column pair (one complex y-line) from
// the shared memory of the CTAs holding those rows, a second barrier frees
// the buffers, the y-transform runs in registers with the CTA's own buffer
// as the exchange, and the column stripe of the spectrum is staged and
// written to global memory row by row.  The plane's data crosses HBM once in
// and once out, where separate x and y passes move it twice each way.  Modes:
// XY_DIVQ (the first solve: f = rho0 D(q') in FP64 per row, stored, its FP32
// image sigma f transformed) and XY_LOAD (the refinement sweeps: the stored
// FP32 residual, transformed in place).
//
// Inverse (k_xy_inv): the mirror image.  CTA c reads its column stripe of
// the spectrum, inverts it along y into its shared memory (row j of the
// stripe at row j), and after a cluster barrier inverts its rows along x,
// reading each row's spectrum from the CTAs holding its columns; after a
// second barrier it writes p (XI_STORE) or p += delta 2^e (XI_ACCUM) in FP64
// with coalesced rows.
//
// The transforms are the very code of the separate register-resident passes
// on the same values, so the fused passes give the same bits.  A launch
// returns at once (every CTA alike: the flag was set before the launch) once
// the refinement has converged.
#pragma once
#include "kern_r16.cuh"
#include <cooperative_groups.h>

namespace fz {

constexpr int XY_CL = 8;  // CTAs per cluster

enum { XY_DIVQ = 0, XY_LOAD = 1 };

template <int N> struct XYShape {
    static_assert(N == 256 || N == 512, "fused x-y passes: N = 256 or 512");
    static constexpr int R = N / XY_CL;                    // rows, then columns, per CTA
    static constexpr int LINES = R / 2;                    // complex lines per CTA
    static constexpr int THREADS = LINES * RShape<N>::TPL;
    static constexpr int RS = N + 2;                       // floats per row (even: 8-byte column pairs)
    static constexpr int SS = R + 1;                       // floats per staged stripe row
    static constexpr int BUF = (2 * LINES * RS > N * SS) ? 2 * LINES * RS : N * SS;  // floats
};

struct XYTab {  // the tables r16_tables fills
    float2 tw[256];
    float2 tw2[256];
    float2 cs[256];
};

template <int N> constexpr size_t xy_smem_bytes() {
    return sizeof(XYTab) + sizeof(float) * (size_t)XYShape<N>::BUF;
}

template <int N, int KX, int KY, int MODE>
__global__ void __cluster_dims__(XY_CL, 1, 1) __launch_bounds__(XYShape<N>::THREADS, 1)
    k_xy_fwd(GridDev g, XArgs a) {
    namespace cg = cooperative_groups;
    typedef XYShape<N> S;
    extern __shared__ __align__(16) unsigned char xy_smem[];
    XYTab &tab = *(XYTab *)xy_smem;
    float *buf = (float *)(xy_smem + sizeof(XYTab));
    if (MODE == XY_LOAD && *(volatile const int *)&a.st->converged) return;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int z = blockIdx.x / XY_CL;
    r16_tables<false, N, (KX == KIND_DCT || KY == KIND_DCT) ? KIND_DCT : KIND_PERIODIC>(tab);
    __syncthreads();
    const RPos<N> q;
    const int lane = threadIdx.x & 31;
    const size_t plane = (size_t)N * N;
    float *out = (float *)a.out + (size_t)z * plane;
    float2 *X = (float2 *)(buf + 2 * q.ln * S::RS);  // line ln: rows 2 ln, 2 ln + 1
    unsigned long long mx = 0ull;
    // ---- 1. rows [rank R, rank R + R) along x
    {
        const int ya = rank * S::R + 2 * q.ln;  // the line's rows ya, ya + 1 (global y)
        float2 v[16];
        if constexpr (MODE == XY_LOAD) {
            const float *la = out + (size_t)ya * N, *lb = la + N;
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const int i = r_src<N, KX>(q.in_index(n1));
                v[n1] = make_float2(la[i], lb[i]);
            }
        } else {
            // f row by row into the line's region (x = lane + 32 i, component = row)
            const float scale32 = (float)g.sigma;
            const float2 cx = f64_split(g.dvx), cy = f64_split(g.dvy), cz = f64_split(g.dvz[z]);
            // the warp's rows: lines ln0 .. ln0 + LPW - 1, as interleaved
            // (row 2l, row 2l + 1) pairs in their line regions
            constexpr int LPW = RShape<N>::LPW;
            const int ln0 = (threadIdx.x >> 5) * LPW;
#pragma unroll 1
            for (int r = 0; r < 2 * LPW; ++r) {
                const int lr = 2 * ln0 + r;                  // row of the CTA
                const int y = rank * S::R + lr;
                float *dr = buf + (lr >> 1) * 2 * S::RS + (lr & 1);
#pragma unroll 4
                for (int i = 0; i < N / 32; ++i) {
                    const int x = lane + 32 * i;
                    const double f = div_q_eval_df(div_q_ld<false>(g, x, y, z, a.qx, a.qy, a.qz), cx, cy, cz);
                    a.f_out[((size_t)z * N + y) * N + x] = f;
                    mx = umax64(mx, absbits(f));
                    dr[2 * x] = f64_to_f32_shift(f, 0) * scale32;
                }
            }
            __syncwarp();
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) v[n1] = X[r_src<N, KX>(q.in_index(n1))];
            __syncwarp();  // the line's region is the exchange buffer next
        }
        r_fft<false, N>(tab, X, q, v);
        // row spectra into the line's region, row-major (row 2 ln, then 2 ln + 1)
        float *ra = buf + 2 * q.ln * S::RS, *rb = ra + S::RS;
        r_separate<N, KX>(v, q, tab, [&](int k, float va, float vb) {
            ra[k] = va;
            rb[k] = vb;
        });
    }
    if constexpr (MODE == XY_DIVQ) block_max_atomic(mx, &a.st->fmax_bits);
    cl.sync();
    // ---- 2. columns [rank R, rank R + R) along y: the column pair of line ln
    {
        const int x0 = rank * S::R + 2 * q.ln;
        float2 v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int j = r_src<N, KY>(q.in_index(n1));
            const float *src = buf + (size_t)(j % S::R) * S::RS + x0;
            v[n1] = *cl.map_shared_rank((const float2 *)src, (unsigned)(j / S::R));
        }
        cl.sync();  // every CTA has read the row spectra: the buffers are free
        r_fft<false, N>(tab, X, q, v);
        __syncthreads();  // every exchange is done before the stripe is staged
        r_separate<N, KY>(v, q, tab, [&](int k, float va, float vb) {
            buf[k * S::SS + 2 * q.ln] = va;
            buf[k * S::SS + 2 * q.ln + 1] = vb;
        });
        __syncthreads();
        // the stripe's rows to global memory: a warp writes R floats of a row
        const int warp = threadIdx.x >> 5, nw = S::THREADS / 32;
        float *o = out + (size_t)rank * S::R;
        for (int k = warp; k < N; k += nw)
#pragma unroll
            for (int c = lane; c < S::R; c += 32) o[(size_t)k * N + c] = buf[k * S::SS + c];
    }
}

template <int N, int KX, int KY, int MODE>
__global__ void __cluster_dims__(XY_CL, 1, 1) __launch_bounds__(XYShape<N>::THREADS, 1)
    k_xy_inv(GridDev g, const float *in, double *p, const DevStats *st) {
    namespace cg = cooperative_groups;
    typedef XYShape<N> S;
    extern __shared__ __align__(16) unsigned char xy_smem[];
    XYTab &tab = *(XYTab *)xy_smem;
    float *buf = (float *)(xy_smem + sizeof(XYTab));
    if (MODE == XI_ACCUM && *(volatile const int *)&st->converged) return;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int z = blockIdx.x / XY_CL;
    r16_tables<true, N, (KX == KIND_DCT || KY == KIND_DCT) ? KIND_DCT : KIND_PERIODIC>(tab);
    const RPos<N> q;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = S::THREADS / 32;
    const size_t plane = (size_t)N * N;
    const float *sp = in + (size_t)z * plane + (size_t)rank * S::R;
    float2 *X = (float2 *)(buf + 2 * q.ln * S::RS);
    // ---- 1. the column stripe [rank R, rank R + R) of the spectrum, staged
    for (int k = warp; k < N; k += nw)
#pragma unroll
        for (int c = lane; c < S::R; c += 32) buf[k * S::SS + c] = sp[(size_t)k * N + c];
    __syncthreads();
    {
        float2 v[16];
        r_combine<N, KY>(v, q, tab, [&](int k) {
            return make_float2(buf[k * S::SS + 2 * q.ln], buf[k * S::SS + 2 * q.ln + 1]);
        });
        __syncthreads();  // the stripe is read before the regions become exchange buffers
        r_fft<true, N>(tab, X, q, v);
        __syncthreads();  // every exchange is done before the stripe is rewritten
        // the column pair's samples back as stripe rows (row j of the plane)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int j = r_src<N, KY>(q.out_index(r));
            buf[j * S::SS + 2 * q.ln] = v[r].x;
            buf[j * S::SS + 2 * q.ln + 1] = v[r].y;
        }
    }
    cl.sync();
    // ---- 2. rows [rank R, rank R + R) along x, each row's spectrum read from
    // the CTAs holding its columns
    {
        const int ya = rank * S::R + 2 * q.ln;
        float2 v[16];
        r_combine<N, KX>(v, q, tab, [&](int k) {
            const unsigned owner = (unsigned)(k / S::R);
            const int kk = k % S::R;
            const float *pa = cl.map_shared_rank(buf + ya * S::SS + kk, owner);
            return make_float2(pa[0], pa[S::SS]);  // rows ya and ya + 1
        });
        cl.sync();  // every CTA has read its rows: the buffers are free
        r_fft<true, N>(tab, X, q, v);
#pragma unroll
        for (int r = 0; r < 16; ++r) X[r_src<N, KX>(q.out_index(r))] = v[r];
        __syncwarp();
        // p (or p += delta 2^e) row by row, lane = x mod 32, coalesced
        const int ef = MODE == XI_ACCUM ? exp_of_bits(*(volatile const unsigned long long *)&st->fmax_bits) : 0;
        constexpr int LPW = RShape<N>::LPW;
        const int ln0 = warp * LPW;
#pragma unroll 1
        for (int r = 0; r < 2 * LPW; ++r) {
            const int lr = 2 * ln0 + r;
            const float *row = buf + (lr >> 1) * 2 * S::RS + (lr & 1);
            double *pr = p + ((size_t)z * N + rank * S::R + lr) * N;
#pragma unroll 4
            for (int i = 0; i < N / 32; ++i) {
                const int x = lane + 32 * i;
                const double d = f32_to_f64_shift(row[2 * x], ef);
                pr[x] = MODE == XI_ACCUM ? pr[x] + d : d;
            }
        }
    }
}

}  // namespace fz
