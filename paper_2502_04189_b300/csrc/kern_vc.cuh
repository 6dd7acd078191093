// Variable-coefficient projection without splitting (sm_103a):
//     D(beta_f G p) = D(u*)/dt,   u = u* - dt beta_f G p,
// beta_f = 1/rho_f (face mean of rho = rho_g + phi (rho_l - rho_g)).  This is
// the pressure equation that the constant-coefficient splitting replaces (the
// paper's Hypre path solves it directly).  Here it is solved by conjugate
// gradients preconditioned with M^-1 = L^-1 D(rho_f G) L^-1, two
// constant-coefficient FFT/tridiagonal solves L^-1 of the projection's own
// passes around the density-weighted operator (exact for a constant density,
// where A = L / rho; with the plain L^-1 instead, the iterations grow with
// the density ratio: 383 against 41 at ratio 1000 in a 32^3 model).
// A = D beta G, L = D G and D rho G are symmetric in the cell-volume
// (dzf-weighted) inner product and negative semi-definite with the constants
// as null space, so CG on (-A) x = -b with the preconditioner -M^-1 runs with
// the same formulas as on A x = b:
//     r = b - A x,  z = L^-1 r,  rho = <r, z>,  d = z + (rho / rho_old) d,
//     alpha = rho / <d, A d>,  x += alpha d,  r -= alpha A d,
// stopped when max|r| / max|b| <= tol.  On a mixed plan the preconditioner
// is the FP32 solve (the register-resident passes where the lengths allow),
// applied to r 2^-e (e the exponent of max|b|, a fixed scale), and the
// direction update is the flexible (Polak-Ribiere) form
// beta = (<z, r> - <z, r_prev>) / rho_old, which tolerates the FP32 rounding
// of the preconditioner; residuals, the operator and x stay FP64.
// Every dot product is a fixed-order
// reduction (grid-stride partial per block, then one block), so a solve is
// bitwise repeatable.  The iteration's scalars live in device memory
// (VcState); the kernels of an iteration return at once after convergence.
#pragma once
#include "kern_passes.cuh"

namespace fz {

struct VcState {
    double rho;       // <r, z> of the current residual
    double alpha, beta;
    double usq;       // sum of u*^2 over all face values
    double rz_prev;   // flexible form: <z, r_prev>
    unsigned long long bmax_bits;  // max|b|
    unsigned long long rmax_bits;  // max|r| of the current iteration
    unsigned int done;             // last-block ticket of the update kernel
    int iters;                     // CG iterations run
};

constexpr int VC_THREADS = 256;
constexpr int VC_MAX_BLOCKS = 2048;  // partial-sum slots

// rho at a cell centre
__device__ __forceinline__ double vc_rho(double rho_l, double rho_g, double phi) {
    return fmaT(phi, rho_l - rho_g, rho_g);
}

// Face coefficients on the +x, +y, +z faces of every cell, stored pre-scaled
// for the flux form of the operators: beta_f/dx^2, beta_f/dy^2 and the z
// conductance beta_f/dzc (the divergence then multiplies by 1/dzf), and the
// same for rho_f (0 on walls;
// beta_f = 2/(rho_a + rho_b) by the FP32-seeded Newton reciprocal, relative
// error about 2^-44: the operator and the correction use the same stored
// beta_f, so u stays divergence-free to round-off; rho_a + rho_b lies within
// [2e-30, 2e30] for the densities a plan accepts),
// b = D(u*)/dt, r = b, x = d = 0, the preconditioner's input sigma r in the
// spectral workspace, max|b| and the partial sums of u*^2.
__global__ void __launch_bounds__(VC_THREADS) k_vc_init(GridDev g, double rho_l, double rho_g, double dt,
                                                       const double *__restrict__ phi,
                                                       const double *__restrict__ u,
                                                       const double *__restrict__ v,
                                                       const double *__restrict__ w,
                                                       double *__restrict__ bx, double *__restrict__ by,
                                                       double *__restrict__ bz,
                                                       double *__restrict__ rx, double *__restrict__ ry,
                                                       double *__restrict__ rzf, double *__restrict__ r,
                                                       double *__restrict__ x, double *__restrict__ d,
                                                       double *__restrict__ spec,
                                                       double *__restrict__ part, VcState *vs) {
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    const double idt = 1.0 / dt, cx = g.idx1 * idt, cy = g.idy1 * idt;
    unsigned long long mx = 0ull;
    double usq = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / pl);
        const size_t rem = c - (size_t)k * pl;
        const int j = (int)(rem / g.nx), i = (int)(rem - (size_t)j * g.nx);
        const double rc = vc_rho(rho_l, rho_g, phi[c]);
        double b = 0.0, s = 0.0;
        if (!(g.bcx == BC_NEUMANN && i == g.nx - 1)) {
            s = rc + vc_rho(rho_l, rho_g, phi[i < g.nx - 1 ? c + 1 : c - i]);
            b = 2.0 * rcp_pos_nr1(s);
        }
        bx[c] = mulT(b, g.idx2);
        rx[c] = mulT(0.5 * s, g.idx2);
        b = s = 0.0;
        if (!(g.bcy == BC_NEUMANN && j == g.ny - 1)) {
            s = rc + vc_rho(rho_l, rho_g, phi[j < g.ny - 1 ? c + g.nx : c - (size_t)j * g.nx]);
            b = 2.0 * rcp_pos_nr1(s);
        }
        by[c] = mulT(b, g.idy2);
        ry[c] = mulT(0.5 * s, g.idy2);
        b = s = 0.0;
        if (k < g.nz - 1 || g.perz) {
            s = rc + vc_rho(rho_l, rho_g, phi[k < g.nz - 1 ? c + pl : c - (size_t)k * pl]);
            b = 2.0 * rcp_pos_nr1(s);
        }
        const double idzc = mulT(g.lzc[k], g.dzf[k]);  // 1/dzc_(k+1/2) (0 on the top wall)
        bz[c] = mulT(b, idzc);
        rzf[c] = mulT(0.5 * s, idzc);
        const double f = div_q<false>(g, i, j, k, cx, cy, mulT(g.izf[k], idt), u, v, w);
        r[c] = f;
        x[c] = 0.0;
        d[c] = 0.0;
        if (spec) spec[c] = mulT(f, g.sigma);
        mx = umax64(mx, absbits(f));
        usq = fmaT(u[c], u[c], fmaT(v[c], v[c], fmaT(w[c], w[c], usq)));
    }
    block_max_atomic(mx, &vs->bmax_bits);
    const double s = block_sum(usq);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// u*^2 total (one block, fixed order); resets the iteration state.
__global__ void __launch_bounds__(1024) k_vc_init_sum(const double *__restrict__ part, int nparts,
                                                      VcState *vs) {
    double s = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += part[t];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        vs->usq = s;
        vs->rho = 0.0;
        vs->iters = 0;
    }
}

// Partial sums of <a, b> = sum dzf_k a b (one per block); FLEX also
// <a, b2> into part2.
template <bool FLEX>
__global__ void __launch_bounds__(VC_THREADS) k_vc_dot(GridDev g, const double *__restrict__ a,
                                                      const double *__restrict__ b,
                                                      const double *__restrict__ b2,
                                                      double *__restrict__ part, double *__restrict__ part2,
                                                      const DevStats *st) {
    if (*(volatile const int *)&st->converged) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    double s = 0.0, s2 = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const double wa = mulT(g.dzf[c / pl], a[c]);
        s = fmaT(wa, b[c], s);
        if (FLEX) s2 = fmaT(wa, b2[c], s2);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (FLEX) {
        s2 = block_sum(s2);
        if (threadIdx.x == 0) part2[blockIdx.x] = s2;
    }
}

// rho = <r, z>; beta = rho / rho_old, or (rho - <z, r_prev>) / rho_old in the
// flexible form (0 on the first iteration).
template <bool FLEX>
__global__ void __launch_bounds__(1024) k_vc_beta(const double *__restrict__ part,
                                                  const double *__restrict__ part2, int nparts,
                                                  VcState *vs, const DevStats *st) {
    if (*(volatile const int *)&st->converged) return;
    double s = 0.0, s2 = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) {
        s += part[t];
        if (FLEX) s2 += part2[t];
    }
    s = block_sum(s);
    if (FLEX) s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        const double num = FLEX ? s - s2 : s;
        vs->beta = vs->iters == 0 ? 0.0 : num / vs->rho;
        vs->rho = s;
    }
}

// Mixed plans: the first preconditioner input, r 2^-e sigma in FP32.
__global__ void __launch_bounds__(VC_THREADS) k_vc_spec32(GridDev g, const double *__restrict__ r,
                                                         float *__restrict__ spec, const VcState *vs) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const int eb = exp_of_bits(vs->bmax_bits);
    const float sc = (float)g.sigma;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        spec[c] = f64_to_f32_shift(r[c], eb) * sc;
}

// d = z + beta d
__global__ void __launch_bounds__(VC_THREADS) k_vc_dir(GridDev g, const double *__restrict__ z,
                                                      double *__restrict__ d, const VcState *vs,
                                                      const DevStats *st) {
    if (*(volatile const int *)&st->converged) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double beta = vs->beta;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        d[c] = fmaT(beta, d[c], z[c]);
}

// q = D(c_f G d) in flux form (each face flux c (d_nbr - d_c)/h formed once
// per face and cell side) for face coefficients c_f: beta_f (the operator A,
// OUT = VC_OUT_Q: q and the partial sums of <d, q>) or rho_f (the middle of
// the preconditioner, OUT = VC_OUT_SPEC64 / VC_OUT_SPEC32: q written as the
// next FFT solve's input, sigma q in FP64 or FP32).
enum { VC_OUT_Q = 0, VC_OUT_SPEC64 = 1, VC_OUT_SPEC32 = 2 };
template <int OUT>
__global__ void __launch_bounds__(VC_THREADS) k_vc_apply(GridDev g, const double *__restrict__ d,
                                                        const double *__restrict__ bx,
                                                        const double *__restrict__ by,
                                                        const double *__restrict__ bz,
                                                        void *__restrict__ q, double *__restrict__ part,
                                                        const DevStats *st) {
    if (*(volatile const int *)&st->converged) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    double s = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / pl);
        const size_t rem = c - (size_t)k * pl;
        const int j = (int)(rem / g.nx), i = (int)(rem - (size_t)j * g.nx);
        const double dc = d[c];
        // sum over the six faces of c_f (d_nbr - d_c), coefficients 0 on walls
        const size_t e = i < g.nx - 1 ? c + 1 : c - i;
        const size_t wst = i > 0 ? c - 1 : c + g.nx - 1;
        const double cw = (i > 0 || g.bcx == BC_PERIODIC) ? bx[wst] : 0.0;
        double acc = mulT(bx[c], d[e] - dc);
        acc = fmaT(cw, d[wst] - dc, acc);
        const size_t nn = j < g.ny - 1 ? c + g.nx : c - (size_t)j * g.nx;
        const size_t ss = j > 0 ? c - g.nx : c + (size_t)(g.ny - 1) * g.nx;
        const double cs = (j > 0 || g.bcy == BC_PERIODIC) ? by[ss] : 0.0;
        acc = fmaT(by[c], d[nn] - dc, acc);
        acc = fmaT(cs, d[ss] - dc, acc);
        const size_t t = k < g.nz - 1 ? c + pl : c - (size_t)k * pl;
        const size_t b = k > 0 ? c - pl : c + (size_t)(g.nz - 1) * pl;
        const double cb = (k > 0 || g.perz) ? bz[b] : 0.0;
        double az = mulT(bz[c], d[t] - dc);  // 0 on the top wall
        az = fmaT(cb, d[b] - dc, az);
        acc = fmaT(g.izf[k], az, acc);
        if (OUT == VC_OUT_Q) {
            ((double *)q)[c] = acc;
            s = fmaT(mulT(g.dzf[k], dc), acc, s);
        } else if (OUT == VC_OUT_SPEC64) {
            ((double *)q)[c] = mulT(acc, g.sigma);
        } else {
            ((float *)q)[c] = f64_to_f32_shift(acc, 0) * (float)g.sigma;
        }
    }
    if (OUT == VC_OUT_Q) {
        s = block_sum(s);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// alpha = rho / <d, A d>; resets the update kernel's max and ticket.
__global__ void __launch_bounds__(1024) k_vc_alpha(const double *__restrict__ part, int nparts, VcState *vs,
                                                   const DevStats *st) {
    if (*(volatile const int *)&st->converged) return;
    double s = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += part[t];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        vs->alpha = vs->rho / s;
        vs->rmax_bits = 0ull;
        vs->done = 0u;
    }
}

// x += alpha d, r -= alpha q, the next preconditioner input in the spectral
// workspace (sigma r in FP64; mixed: r 2^-e sigma in FP32, and r_prev = the
// old r for the flexible update), max|r|; the last block decides convergence.
template <bool MIX>
__global__ void __launch_bounds__(VC_THREADS) k_vc_update(GridDev g, double *__restrict__ x,
                                                         double *__restrict__ r,
                                                         const double *__restrict__ d,
                                                         const double *__restrict__ q,
                                                         void *__restrict__ spec, double *__restrict__ r_prev,
                                                         VcState *vs, DevStats *st, double tol) {
    if (*(volatile const int *)&st->converged) return;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const double alpha = vs->alpha;
    const int eb = MIX ? exp_of_bits(vs->bmax_bits) : 0;
    const float sc = (float)g.sigma;
    unsigned long long mx = 0ull;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        x[c] = fmaT(alpha, d[c], x[c]);
        const double ro = r[c];
        const double rv = fmaT(-alpha, q[c], ro);
        r[c] = rv;
        if (MIX) {
            r_prev[c] = ro;
            ((float *)spec)[c] = f64_to_f32_shift(rv, eb) * sc;
        } else {
            ((double *)spec)[c] = mulT(rv, g.sigma);
        }
        mx = umax64(mx, absbits(rv));
    }
    block_max_atomic(mx, &vs->rmax_bits);
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&vs->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double rm = __longlong_as_double((long long)atomicMax(&vs->rmax_bits, 0ull));
        const double bm = __longlong_as_double((long long)vs->bmax_bits);
        const double rel = bm > 0.0 ? rm / bm : rm;
        vs->iters += 1;
        st->iterations = vs->iters;
        st->relres = rel;
        if (rel <= tol) st->converged = 1;
    }
}

// u = u* - dt beta_f G x on every non-wall face (in place); dtx = dt dx,
// dty = dt dy.
__global__ void __launch_bounds__(VC_THREADS) k_vc_correct(GridDev g, double dt, double dtx, double dty,
                                                          const double *__restrict__ x,
                                                          const double *__restrict__ bx,
                                                          const double *__restrict__ by,
                                                          const double *__restrict__ bz,
                                                          double *__restrict__ u, double *__restrict__ v,
                                                          double *__restrict__ w) {
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(c / pl);
        const size_t rem = c - (size_t)k * pl;
        const int j = (int)(rem / g.nx), i = (int)(rem - (size_t)j * g.nx);
        const double xc = x[c];
        // beta/h = (beta/h^2) h in x and y; the z coefficient is beta/dzc already
        if (!(g.bcx == BC_NEUMANN && i == g.nx - 1))
            u[c] = fmaT(-mulT(dtx, bx[c]), x[i < g.nx - 1 ? c + 1 : c - i] - xc, u[c]);
        if (!(g.bcy == BC_NEUMANN && j == g.ny - 1))
            v[c] = fmaT(-mulT(dty, by[c]), x[j < g.ny - 1 ? c + g.nx : c - (size_t)j * g.nx] - xc, v[c]);
        if (k < g.nz - 1 || g.perz)
            w[c] = fmaT(-mulT(dt, bz[c]), x[k < g.nz - 1 ? c + pl : c - (size_t)k * pl] - xc, w[c]);
    }
}

}  // namespace fz
