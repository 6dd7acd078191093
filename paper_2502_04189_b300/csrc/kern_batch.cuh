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
    BK_CORRECT
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

__device__ __forceinline__ void batch_run_tile(const BatchInst &I, const BatchItem &w, int tile,
                                               unsigned char *smem) {
    const int kind = I.kind[w.pass];
    const GridDev &g = I.g;
    switch (kind) {
    case BK_FLUX: {
        const VB vb{tile % I.fgx, (tile / I.fgx) % I.fgy, tile / (I.fgx * I.fgy)};
        double *slot = I.usq_part ? I.usq_part + tile : nullptr;
        if (I.rho0_is_g)
            flux_body<true>(g, I.kc, vb, I.phi, I.pn, I.pnm1, I.u, I.v, I.w, I.qx, I.qy, I.qz, slot);
        else
            flux_body<false>(g, I.kc, vb, I.phi, I.pn, I.pnm1, I.u, I.v, I.w, I.qx, I.qy, I.qz, slot);
        break;
    }
    case BK_SUM:
        sum_partials_body<true>(I.usq_part, I.n_usq_part, I.usq_sum);
        break;
    case BK_XFWD64:
    case BK_XFWD_MIX:
    case BK_XLOAD: {
        XArgs a;
        memset(&a, 0, sizeof(a));
        a.qx = I.qx;
        a.qy = I.qy;
        a.qz = I.qz;
        a.f_out = I.f;
        a.st = I.st;
        if (kind == BK_XFWD64) {
            a.out = I.fhat64;
            xfwd_body<double, XF_F64_DIVQ, true>(g, I.fx64, I.Lx, a, tile, I.tiles[w.pass], smem);
        } else if (kind == BK_XFWD_MIX) {
            a.out = I.fhat32;
            xfwd_body<float, XF_MIX_DIVQ, true>(g, I.fx32, I.Lx, a, tile, I.tiles[w.pass], smem);
        } else {
            a.out = I.fhat32;
            xfwd_body<float, XF_MIX_LOAD, true>(g, I.fx32, I.Lx, a, tile, I.tiles[w.pass], smem);
        }
        break;
    }
    case BK_RES0:
    case BK_RCORR: {
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
        a.slot = I.slot[w.pass];
        a.tol = I.tol;
        const int txy = I.cgx * I.cgy, z = tile / txy, r = tile - z * txy, y = r / I.cgx;
        const VB vb{r - y * I.cgx, y, z};
        if (kind == BK_RES0) resid_body<true, false>(g, RESID_KC, a, vb, I.tiles[w.pass], (double *)smem);
        else resid_body<true, true>(g, RESID_KC, a, vb, I.tiles[w.pass], (double *)smem);
        break;
    }
    case BK_YF64:
        ypass_body<double, false, true>(g.nx, g.ny, I.fy64, I.TXy, I.fhat64, nullptr, tile % I.ygx,
                                        tile / I.ygx, smem);
        break;
    case BK_YI64:
        ypass_body<double, true, true>(g.nx, g.ny, I.fy64, I.TXy, I.fhat64, nullptr, tile % I.ygx,
                                       tile / I.ygx, smem);
        break;
    case BK_YF32:
    case BK_YF32C:
        ypass_body<float, false, true>(g.nx, g.ny, I.fy32, I.TXy, I.fhat32,
                                       kind == BK_YF32C ? &I.st->converged : nullptr, tile % I.ygx,
                                       tile / I.ygx, smem);
        break;
    case BK_YI32:
    case BK_YI32C:
        ypass_body<float, true, true>(g.nx, g.ny, I.fy32, I.TXy, I.fhat32,
                                      kind == BK_YI32C ? &I.st->converged : nullptr, tile % I.ygx,
                                      tile / I.ygx, smem);
        break;
    case BK_TH64:
        thomas_body<double, false, true>(g, I.Ux, I.Uy, I.mtab64, I.ibtab64, I.cup64, I.fhat64,
                                         nullptr, tile * BATCH_THREADS, nullptr, I.wtab64, I.qtab64);
        break;
    case BK_TH32:
    case BK_TH32C:
        thomas_body<float, false, true>(g, I.Ux, I.Uy, I.mtab32, I.ibtab32, I.cup32, I.fhat32,
                                        kind == BK_TH32C ? &I.st->converged : nullptr,
                                        tile * BATCH_THREADS, nullptr, I.wtab32, I.qtab32);
        break;
    case BK_XI64:
        xinv_body<double, XI_STORE, true>(g, I.fx64, I.Lx, I.fhat64, I.p, I.st, tile, smem);
        break;
    case BK_XI32:
        xinv_body<float, XI_STORE, true>(g, I.fx32, I.Lx, I.fhat32, I.p, I.st, tile, smem);
        break;
    case BK_XACC:
        xinv_body<float, XI_ACCUM, true>(g, I.fx32, I.Lx, I.fhat32, I.p, I.st, tile, smem);
        break;
    case BK_CORRIF:
        if (__ldcg(&I.st->n_resid) != 1) break;  // a fused residual pass wrote u
        [[fallthrough]];
    case BK_CORRECT: {
        const VB vb{tile % I.cgx, (tile / I.cgx) % I.cgy, tile / (I.cgx * I.cgy)};
        correct_body<true>(g, I.p, I.qx, I.qy, I.qz, I.u, I.v, I.w, vb);
        break;
    }
    default:
        break;
    }
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
            const bool refine = kind == BK_XLOAD || kind == BK_YF32C || kind == BK_TH32C ||
                                kind == BK_YI32C || kind == BK_XACC || kind == BK_RCORR;
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

}  // namespace fz
