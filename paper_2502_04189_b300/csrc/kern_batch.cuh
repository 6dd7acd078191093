// Persistent batch kernel: many independent projections of uneven sizes in
// one launch (sm_103a).
//
// The host lists every tile of every pass of every instance as a work item
// (instance, pass, tile).  Each CTA of the persistent grid repeatedly claims
// the next item from an atomic queue head, waits until all tiles of the same
// instance's previous pass are done (a bounded spin on that pass's completion
// counter), runs the pass body on that tile, and then bumps its own pass
// counter.  Items are claimed in list order and a dependency always points to
// an item earlier in the list, i.e. one already claimed by a running CTA, so
// the schedule cannot deadlock whatever the grid size.  Data written by other
// CTAs during the launch is read with ld.global.cg (L2), and every completion
// is published with a fence before its counter increment.
//
// A spin that exceeds its limit records FIZZY_ERR_TIMEOUT in the status word,
// skips its item (still counting it done so nothing else waits on it) and
// carries on; the host reports the status.
#pragma once
#include "kern_passes.cuh"

namespace fz {

constexpr int BATCH_THREADS = 256;
constexpr int BATCH_MAXP = 64;  // passes per instance (mixed: 9 + 6 * max_refine <= 64)

enum BatchKind : int {
    BK_FLUX = 0,
    BK_SUM,
    BK_XFWD64,
    BK_YF64,
    BK_TH64,
    BK_YI64,
    BK_XI64,
    BK_XFWD_MIX,
    BK_YF32,
    BK_TH32,
    BK_YI32,
    BK_XI32,
    BK_RES0,    // residual of the FP32 solution (slot 0)
    BK_XLOAD,   // transform of the stored residual (sweep s)
    BK_YF32C,
    BK_TH32C,
    BK_YI32C,
    BK_XACC,
    BK_RCORR,   // residual fused with the correction (slot s)
    BK_CORRIF,  // the correction, unless a fused residual pass has run
    BK_CORRECT,
    // grouped form only: the flux pass split by its compile-time density
    // branch (rho0 = rho_l, rho0 = rho_g), so each launch holds one body
    BK_FLUX_L,
    BK_FLUX_G
};

// One instance as the persistent kernel sees it (device memory, read-only
// during the launch).
struct BatchInst {
    GridDev g;
    FFTDesc fx64, fy64, fx32, fy32;
    int rho0_is_g;
    int kc;              // flux planes per tile
    int Lx, TXy;         // x-pass lines per tile (pairs), y-pass columns per tile
    int Ux, Uy;
    double tol;
    // caller arrays
    const double *phi, *pn, *pnm1;
    double *u, *v, *w, *p;
    // plan workspace and tables
    double *qx, *qy, *qz;
    double *fhat64;
    float *fhat32;
    double *f;
    const double *mtab64, *ibtab64, *cup64;
    const double *wtab64, *qtab64;  // periodic z (else null)
    const float *mtab32, *ibtab32, *cup32;
    const float *wtab32, *qtab32;
    DevStats *st;
    double *usq_part, *usq_sum;
    int n_usq_part;
    // pass chain
    int npass;
    int kind[BATCH_MAXP];
    int tiles[BATCH_MAXP];
    int slot[BATCH_MAXP];
    // tile decode helpers
    int fgx, fgy;        // flux grid x, y
    int ygx;             // y-pass tiles along x
    int cgx, cgy;        // correction grid x, y
};

// A work item: tiles tile0 .. tile0 + ntile - 1 of one pass of one instance
// (consecutive tiles are grouped so each item carries enough work to hide the
// claim / wait / publish overhead).
struct BatchItem {
    int inst, pass, tile0, ntile;
};

struct BatchArgs {
    const BatchInst *insts;
    const BatchItem *items;
    int n_items;
    int *head;       // next item to claim
    int *done;       // [n_inst][BATCH_MAXP] completed tiles
    int *status;     // 0 or FIZZY-style negative code
    long long spin_limit;
    int stall_inst;  // test support: this instance's first dependency never completes (-1: none)
};

// One tile of a pass of kind KIND (compile-time) of instance I.  CG: data
// written by other CTAs of the same launch is read through L2 (the persistent
// form); the grouped form reads it after a launch boundary and passes false.
// The same body, with the same arithmetic, runs in either form and in the
// stand-alone kernels.
template <int KIND, bool CG>
__device__ __forceinline__ void run_kind(const BatchInst &I, int pass, int tile, unsigned char *smem) {
    const GridDev &g = I.g;
    if constexpr (KIND == BK_FLUX || KIND == BK_FLUX_L || KIND == BK_FLUX_G) {
        const VB vb{tile % I.fgx, (tile / I.fgx) % I.fgy, tile / (I.fgx * I.fgy)};
        double *slot = I.usq_part ? I.usq_part + tile : nullptr;
        if (KIND == BK_FLUX_G || (KIND == BK_FLUX && I.rho0_is_g))
            flux_any<true>(g, I.kc, vb, I.phi, I.pn, I.pnm1, I.u, I.v, I.w, I.qx, I.qy, I.qz, slot);
        else
            flux_any<false>(g, I.kc, vb, I.phi, I.pn, I.pnm1, I.u, I.v, I.w, I.qx, I.qy, I.qz, slot);
    } else if constexpr (KIND == BK_SUM) {
        sum_partials_body<CG>(I.usq_part, I.n_usq_part, I.usq_sum);
    } else if constexpr (KIND == BK_XFWD64 || KIND == BK_XFWD_MIX || KIND == BK_XLOAD) {
        XArgs a;
        memset(&a, 0, sizeof(a));
        a.qx = I.qx;
        a.qy = I.qy;
        a.qz = I.qz;
        a.f_out = I.f;
        a.st = I.st;
        if constexpr (KIND == BK_XFWD64) {
            a.out = I.fhat64;
            xfwd_body<double, XF_F64_DIVQ, CG>(g, I.fx64, I.Lx, a, tile, I.tiles[pass], smem);
        } else if constexpr (KIND == BK_XFWD_MIX) {
            a.out = I.fhat32;
            xfwd_body<float, XF_MIX_DIVQ, CG>(g, I.fx32, I.Lx, a, tile, I.tiles[pass], smem);
        } else {
            a.out = I.fhat32;
            xfwd_body<float, XF_MIX_LOAD, CG>(g, I.fx32, I.Lx, a, tile, I.tiles[pass], smem);
        }
    } else if constexpr (KIND == BK_RES0 || KIND == BK_RCORR) {
        RArgs a;
        a.p = I.p;
        a.f = I.f;
        a.qx = I.qx;
        a.qy = I.qy;
        a.qz = I.qz;
        a.u = I.u;
        a.v = I.v;
        a.w = I.w;
        a.r32 = I.fhat32;
        a.st = I.st;
        a.slot = I.slot[pass];
        a.tol = I.tol;
        const int txy = I.cgx * I.cgy, z = tile / txy, r = tile - z * txy, y = r / I.cgx;
        const VB vb{r - y * I.cgx, y, z};
        resid_body<CG, KIND == BK_RCORR>(g, RESID_KC, a, vb, I.tiles[pass], (double *)smem);
    } else if constexpr (KIND == BK_YF64 || KIND == BK_YI64) {
        ypass_body<double, KIND == BK_YI64, CG>(g.nx, g.ny, I.fy64, I.TXy, I.fhat64, nullptr,
                                                tile % I.ygx, tile / I.ygx, smem);
    } else if constexpr (KIND == BK_YF32 || KIND == BK_YF32C || KIND == BK_YI32 || KIND == BK_YI32C) {
        ypass_body<float, KIND == BK_YI32 || KIND == BK_YI32C, CG>(
            g.nx, g.ny, I.fy32, I.TXy, I.fhat32,
            (KIND == BK_YF32C || KIND == BK_YI32C) ? &I.st->converged : nullptr, tile % I.ygx,
            tile / I.ygx, smem);
    } else if constexpr (KIND == BK_TH64) {
        thomas_body<double, false, CG>(g, I.Ux, I.Uy, I.mtab64, I.ibtab64, I.cup64, I.fhat64, nullptr,
                                       tile * BATCH_THREADS, nullptr, I.wtab64, I.qtab64);
    } else if constexpr (KIND == BK_TH32 || KIND == BK_TH32C) {
        thomas_body<float, false, CG>(g, I.Ux, I.Uy, I.mtab32, I.ibtab32, I.cup32, I.fhat32,
                                      KIND == BK_TH32C ? &I.st->converged : nullptr,
                                      tile * BATCH_THREADS, nullptr, I.wtab32, I.qtab32);
    } else if constexpr (KIND == BK_XI64) {
        xinv_body<double, XI_STORE, CG>(g, I.fx64, I.Lx, I.fhat64, I.p, I.st, tile, smem);
    } else if constexpr (KIND == BK_XI32) {
        xinv_body<float, XI_STORE, CG>(g, I.fx32, I.Lx, I.fhat32, I.p, I.st, tile, smem);
    } else if constexpr (KIND == BK_XACC) {
        xinv_body<float, XI_ACCUM, CG>(g, I.fx32, I.Lx, I.fhat32, I.p, I.st, tile, smem);
    } else if constexpr (KIND == BK_CORRIF || KIND == BK_CORRECT) {
        if (KIND == BK_CORRIF && ldp<CG>(&I.st->n_resid) != 1) return;  // a fused residual pass wrote u
        const VB vb{tile % I.cgx, (tile / I.cgx) % I.cgy, tile / (I.cgx * I.cgy)};
        correct_body<CG>(g, I.p, I.qx, I.qy, I.qz, I.u, I.v, I.w, vb);
    }
}

// Refinement-sweep passes: empty once the instance has converged.
__host__ __device__ constexpr bool refine_kind(int kind) {
    return kind == BK_XLOAD || kind == BK_YF32C || kind == BK_TH32C || kind == BK_YI32C ||
           kind == BK_XACC || kind == BK_RCORR;
}

__device__ __forceinline__ void batch_run_tile(const BatchInst &I, const BatchItem &w, int tile,
                                               unsigned char *smem) {
#define FZ_RUN(K)                                    \
    case K:                                          \
        run_kind<K, true>(I, w.pass, tile, smem);    \
        break;
    switch (I.kind[w.pass]) {
        FZ_RUN(BK_FLUX)
        FZ_RUN(BK_SUM)
        FZ_RUN(BK_XFWD64)
        FZ_RUN(BK_YF64)
        FZ_RUN(BK_TH64)
        FZ_RUN(BK_YI64)
        FZ_RUN(BK_XI64)
        FZ_RUN(BK_XFWD_MIX)
        FZ_RUN(BK_YF32)
        FZ_RUN(BK_TH32)
        FZ_RUN(BK_YI32)
        FZ_RUN(BK_XI32)
        FZ_RUN(BK_RES0)
        FZ_RUN(BK_XLOAD)
        FZ_RUN(BK_YF32C)
        FZ_RUN(BK_TH32C)
        FZ_RUN(BK_YI32C)
        FZ_RUN(BK_XACC)
        FZ_RUN(BK_RCORR)
        FZ_RUN(BK_CORRIF)
        FZ_RUN(BK_CORRECT)
    default:
        break;
    }
#undef FZ_RUN
}

// Five resident CTAs per SM (48 registers; about 400 bytes of spills, served
// by L1): the
// FP64-bound pass bodies need the warps more than the registers (measured on
// the 64-instance batch: 3 CTAs 5.29, 4: 5.76, 5: 5.92, 6: 5.94 Gpt/s mixed;
// FP64 5.28, 5.67, 5.54, 5.46).
__global__ void __launch_bounds__(BATCH_THREADS, 5) k_batch(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const BatchItem w = A.items[it];
        const BatchInst &I = A.insts[w.inst];
        if (threadIdx.x == 0) {
            int ok = 1;
            const int kind = I.kind[w.pass];
            const bool refine = refine_kind(kind);
            // refinement work of an instance that has already converged is
            // empty: publish it without waiting (the flag is set once, by the
            // last tile of a residual pass, and never cleared in the launch)
            if (refine && *(const volatile int *)&I.st->converged) ok = 0;
            else if (w.pass > 0) {
                const int need = (w.inst == A.stall_inst && w.pass == 1) ? INT_MAX : I.tiles[w.pass - 1];
                const volatile int *cnt = A.done + (size_t)w.inst * BATCH_MAXP + (w.pass - 1);
                long long spins = 0;
                while (*cnt < need) {
                    if (++spins > A.spin_limit) {
                        ok = 0;
                        atomicCAS(A.status, 0, -6);  // FIZZY_ERR_TIMEOUT
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok)
            for (int t = 0; t < w.ntile; ++t) {
                batch_run_tile(I, w, w.tile0 + t, smem_raw);
                __syncthreads();  // shared memory is reused by the next tile
            }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(A.done + (size_t)w.inst * BATCH_MAXP + w.pass, w.ntile);
    }
}

// ---- Grouped form: pass s of many instances as one ordinary launch.
//
// The host captures one launch per (chain, pass index, pass kind): the tiles
// of every instance of the chain whose pass s has that kind, numbered one
// after another (segment i covers global tiles seg[i].tile0 onward).  Launch
// order carries the dependencies, so no tile waits for another; each kernel
// has its own registers and occupancy (the persistent kernel must fit the
// largest body in one register budget).  Refinement tiles of an instance that
// has converged return at once.  The z-solve uses the shared-memory cp.async
// ring of the stand-alone kernel (32-line tiles) on wall-bounded z.
struct GroupSeg {
    int inst, tile0;
};

struct GroupArgs {
    const BatchInst *insts;
    const GroupSeg *seg;  // n_seg segments, ascending tile0, seg[0].tile0 = 0
    int n_seg, pass, total;
};

__device__ __forceinline__ int group_seg(const GroupArgs &A, int t) {
    int lo = 0, hi = A.n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.seg[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A segment whose tiles are all empty: a refinement pass of an instance that
// has converged, or the conditional correction after a fused residual pass.
template <int KIND>
__device__ __forceinline__ bool seg_empty(const BatchInst &I) {
    if constexpr (refine_kind(KIND)) return *(volatile const int *)&I.st->converged != 0;
    if constexpr (KIND == BK_CORRIF) return *(volatile const int *)&I.st->n_resid != 1;
    return false;
}

// The next tile of this block's stride past the end of segment s.
__device__ __forceinline__ int skip_seg(const GroupArgs &A, int s, int t) {
    const int end = s + 1 < A.n_seg ? A.seg[s + 1].tile0 : A.total;
    return t + ((end - t + (int)gridDim.x - 1) / (int)gridDim.x) * (int)gridDim.x;
}

// Resident CTAs per SM the FP64-bound grouped kernels are compiled for: the
// instance's constants and pointers live in registers here (kernel
// parameters in the stand-alone kernels), which would otherwise cost them
// occupancy.
constexpr int group_min_blocks(int kind) {
    return (kind == BK_FLUX_L || kind == BK_FLUX_G || kind == BK_RES0 || kind == BK_RCORR) ? 5 : 1;
}

template <int KIND>
__global__ void __launch_bounds__(BATCH_THREADS, group_min_blocks(KIND)) k_bgroup(GroupArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int t = blockIdx.x; t < A.total;) {
        const int s = group_seg(A, t);
        const GroupSeg sg = A.seg[s];
        const BatchInst &I = A.insts[sg.inst];
        if (seg_empty<KIND>(I)) {
            t = skip_seg(A, s, t);
            continue;
        }
        run_kind<KIND, false>(I, A.pass, t - sg.tile0, smem_raw);
        __syncthreads();  // shared memory is reused by the next tile
        t += gridDim.x;
    }
}

// z-solve of the grouped form: THOMAS_BLOCK lines per tile, the cp.async ring
// on wall-bounded z, the register-prefetch cyclic solve on periodic z.
template <typename T, bool C>
__global__ void __launch_bounds__(THOMAS_BLOCK) k_bgroup_th(GroupArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int t = blockIdx.x; t < A.total; t += gridDim.x) {
        const int s = group_seg(A, t);
        const GroupSeg sg = A.seg[s];
        const BatchInst &I = A.insts[sg.inst];
        const int *conv = C ? &I.st->converged : nullptr;
        if (C && *(volatile const int *)conv) {
            t = skip_seg(A, s, t) - (int)gridDim.x;
            continue;
        }
        const int lb = (t - sg.tile0) * THOMAS_BLOCK;
        if constexpr (sizeof(T) == 8) {
            if (I.g.perz)
                thomas_body<double, false, false>(I.g, I.Ux, I.Uy, I.mtab64, I.ibtab64, I.cup64, I.fhat64,
                                                  nullptr, lb, nullptr, I.wtab64, I.qtab64);
            else
                thomas_body<double, true, false>(I.g, I.Ux, I.Uy, I.mtab64, I.ibtab64, I.cup64, I.fhat64,
                                                 nullptr, lb, (double *)smem_raw);
        } else {
            if (I.g.perz)
                thomas_body<float, false, false>(I.g, I.Ux, I.Uy, I.mtab32, I.ibtab32, I.cup32, I.fhat32,
                                                 conv, lb, nullptr, I.wtab32, I.qtab32);
            else
                thomas_body<float, true, false>(I.g, I.Ux, I.Uy, I.mtab32, I.ibtab32, I.cup32, I.fhat32,
                                                conv, lb, (float *)smem_raw);
        }
    }
}

// Zero every instance's stats (block i: instance i) before a grouped solve.
__global__ void k_bgroup_reset(const BatchInst *insts, int n) {
    if ((int)blockIdx.x >= n) return;
    unsigned *s = (unsigned *)insts[blockIdx.x].st;
    for (int i = threadIdx.x; i < (int)(sizeof(DevStats) / sizeof(unsigned)); i += blockDim.x) s[i] = 0u;
}

}  // namespace fz
