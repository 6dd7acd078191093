// Kernels of the stand-alone Poisson solve (fizzy_poisson_solve): the fast
// direct solver of the projection applied to a given right-hand side, with
// the boundary kinds of the CaNS solver in x and y (periodic; Neumann,
// Dirichlet or mixed at the two faces).
//
//   k_poisson_load  : the transform input from f: sigma f (FP64), or
//                     FP32(f) sigma (mixed), and max|f|
//   k_poisson_resid : r = f - L_h p in FP64 with the ghost rules of the
//                     boundary kinds, max|r|, and (mixed) the FP32 right-hand
//                     side sigma 2^-e r of the next refinement sweep; the last
//                     block decides convergence
#pragma once
#include "kern_passes.cuh"

namespace fz {

// Boundary kinds of an x or y direction (the values of fizzy_proj_desc.bc_x):
// 0 periodic, 1 Neumann at both faces, 2 Dirichlet at both faces, 3 Neumann
// near and Dirichlet far, 4 Dirichlet near and Neumann far.  Beyond a Neumann
// face the ghost value is the cell value, beyond a Dirichlet face its
// negative.
__device__ __forceinline__ double ghost_val(int bc, int far_side, double pc) {
    const bool dir = bc == 2 || (bc == 3 && far_side) || (bc == 4 && !far_side);
    return dir ? -pc : pc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_poisson_load(GridDev g, const double *__restrict__ f,
                                                      T *__restrict__ out, DevStats *st) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    unsigned long long mx = 0ull;
    const float s32 = (float)g.sigma;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const double v = f[c];
        mx = umax64(mx, absbits(v));
        if (sizeof(T) == 8) out[c] = (T)(v * g.sigma);
        else out[c] = (T)(f64_to_f32_shift(v, 0) * s32);
    }
    block_max_atomic(mx, &st->fmax_bits);
}

// One cell's L_h p in flux form (each face difference formed first).
__device__ __forceinline__ double lap_bc_cell(const GridDev &g, const double *p, int i, int j, int k) {
    const size_t c = cidx(g, i, j, k), pl = (size_t)g.nx * g.ny;
    const double pc = p[c];
    const double pe = i < g.nx - 1 ? p[c + 1] : (g.bcx == BC_PERIODIC ? p[c - i] : ghost_val(g.bcx, 1, pc));
    const double pw = i > 0 ? p[c - 1] : (g.bcx == BC_PERIODIC ? p[c + g.nx - 1] : ghost_val(g.bcx, 0, pc));
    const double pn = j < g.ny - 1 ? p[c + g.nx]
                                   : (g.bcy == BC_PERIODIC ? p[c - (size_t)j * g.nx] : ghost_val(g.bcy, 1, pc));
    const double ps = j > 0 ? p[c - g.nx]
                            : (g.bcy == BC_PERIODIC ? p[c + (size_t)(g.ny - 1) * g.nx] : ghost_val(g.bcy, 0, pc));
    const double pt = k < g.nz - 1 ? p[c + pl] : (g.perz ? p[c - (size_t)k * pl] : pc);
    const double pb = k > 0 ? p[c - pl] : (g.perz ? p[c + (size_t)(g.nz - 1) * pl] : pc);
    double acc = mulT((pe - pc) - (pc - pw), g.idx2);
    acc = fmaT((pn - pc) - (pc - ps), g.idy2, acc);
    acc = fmaT(g.lzc[k], pt - pc, acc);
    return fmaT(-g.lza[k], pc - pb, acc);
}

// r = f - L_h p over the grid (grid-stride); slot indexes the residual
// evaluation (0: after the first solve, s: after sweep s).  With r32 the
// FP32 right-hand side sigma 2^-e r is stored (e the exponent of max|f|).
// The last block to finish sets relres and the sweep count, and sets the
// stop flag: 1 when relres <= tol (converged), 2 when a sweep no longer
// halved max|r| above tol (stagnation).  check_only: relres alone (FP64
// solves).
__global__ void __launch_bounds__(256) k_poisson_resid(GridDev g, const double *__restrict__ f,
                                                       const double *__restrict__ p,
                                                       float *__restrict__ r32, DevStats *st, int slot,
                                                       double tol, int check_only) {
    if (*(volatile const int *)&st->converged) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    const int ef = exp_of_bits(*(volatile const unsigned long long *)&st->fmax_bits);
    const float s32 = (float)g.sigma;
    unsigned long long mx = 0ull;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / pl);
        const size_t rem = c - (size_t)k * pl;
        const int j = (int)(rem / g.nx), i = (int)(rem - (size_t)j * g.nx);
        const double res = f[c] - lap_bc_cell(g, p, i, j, k);
        mx = umax64(mx, absbits(res));
        if (r32) r32[c] = f64_to_f32_shift(res, ef) * s32;
    }
    block_max_atomic(mx, &st->rmax_bits[slot]);
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(&st->done_blocks[slot], 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double rmax = __longlong_as_double((long long)atomicMax(&st->rmax_bits[slot], 0ull));
        const double fmax = __longlong_as_double((long long)atomicMax(&st->fmax_bits, 0ull));
        const double rel = fmax > 0.0 ? rmax / fmax : rmax;
        st->relres = rel;
        if (check_only) return;
        st->n_resid = slot + 1;
        st->iterations = slot;
        int done = rel <= tol ? 1 : 0;
        if (!done && slot > 0) {
            const double prev = __longlong_as_double((long long)atomicMax(&st->rmax_bits[slot - 1], 0ull));
            if (rmax > 0.5 * prev) done = 2;  // stagnated above tol: stop, not converged
        }
        __threadfence();
        if (done) st->converged = done;
    }
}

}  // namespace fz
