// Pass kernels of the projection (sm_103a).
//
//   k_flux      : q' = dt q = u* - dt (beta_f - 1/rho0) G phat on every face (FP64)
//                 (beta_f - 1/rho0 formed without cancellation, see face_flux)
//   k_xfwd      : f = rho0 D(q) (or a stored FP32 residual), then the forward
//                 x-transform
//   k_ypass     : forward / inverse y-transform on strided column tiles
//   k_thomas    : one tridiagonal solve per (kx, ky) z-line (factorised tables)
//   k_xinv      : inverse x-transform, p = value or p += value
//   k_resid     : mixed: r = f - L_h p (FP64), stored in FP32 for the next
//                 sweep, and the convergence decision; fused with the
//                 correction in the refinement sweeps
//   k_correct   : u = q' - (dt/rho0) G p^(n+1)                               (FP64)
//   k_divmax    : max |D u| (diagnostics)
//   k_residmax  : max |f - L_h p| without a transform (FP64-mode check)
//
// The provisional face flux q = u*/dt - (beta_f - 1/rho0) G phat carries the
// split: the right-hand side of the constant-coefficient equation is rho0 D(q)
// (= (rho0/dt) D(u*) + D[(1 - rho0 beta_f) G phat] since
// rho0 (beta_f - 1/rho0) = -(1 - rho0 beta_f)), and the correction
// u = u* - dt[G p/rho0 + (beta_f - 1/rho0) G phat] is dt q - (dt/rho0) G p.
// It is stored as q' = dt q, so f = (rho0/dt) D(q') and u = q' - (dt/rho0) G p
// (two FP64 instructions per face); the right-hand side and the correction
// use the very same face coefficients, so D(u) equals (dt/rho0)(f - L_h p) to
// round-off.
#pragma once
#include "kern_common.cuh"
#include "kern_fft.cuh"

namespace fz {

enum { BC_PERIODIC = 0, BC_NEUMANN = 1 };

// Grid and physical constants (kernel argument, by value).
struct GridDev {
    int nx, ny, nz;
    int bcx, bcy;
    int perz;          // 1: periodic z (plane nz-1 joins plane 0 through the seam face nz-1/2)
    int sing;          // 1: no Dirichlet face in x or y, so the (0,0) z-line is singular
                       // (mean removed, pressure gauge); 0: every z-line is regular
    unsigned rny;      // multiply-high reciprocal of ny (fdiv)
    // face-flux constants.  The split-term flux of a face with spacing h is
    // q' = u* + dt |drho|/(rho0 h) * t/(|drho| t + 2 rho0) * (p^_b - p^_a),
    // kept here with dt |drho|/(rho0 h) folded into the denominator:
    // q' = u* + t/(a' t + r') (p^_b - p^_a), a' = rho0 h/dt,
    // r' = 2 rho0^2 h/(dt |drho|).
    double idt;        // 1/dt
    int var_rho;       // 0: rho_l == rho_g, the split term vanishes (q' = u*)
    int fsh;           // seed-shift offset floor(log2(1 + |drho|/rho0) / 2)
    double fax, frx;   // a', r' of x faces
    double fay, fry;   // a', r' of y faces
    // divergence constants, unscaled (rho0/h) and scaled by sigma = 1/(4 nx ny)
    double dvx, dvy, dvx_s, dvy_s;
    // correction constants
    double dt, cgx, cgy;  // dt, dt/(rho0 dx), dt/(rho0 dy)
    // Laplacian / divergence constants
    double idx2, idy2;    // 1/dx^2, 1/dy^2
    double idx1, idy1;    // 1/dx, 1/dy
    // per-k tables (device, FP64, length nz).  "0 at k = nz-1" holds for z
    // walls; with periodic z that entry belongs to the seam face, whose centre
    // distance is dzc_(nz-1/2) = (dzf_0 + dzf_(nz-1))/2, and a_0 couples plane
    // 0 to plane nz-1 through it.
    const double *faz;    // a' of the z face above k: rho0 dzc_(k+1/2)/dt  (0 at k = nz-1)
    const double *frz;    // r' of that face: 2 rho0^2 dzc_(k+1/2)/(dt |drho|)  (0 at k = nz-1)
    const double *dvz;    // rho0/dzf_k
    const double *dvz_s;  // sigma rho0/dzf_k
    const double *cgz;    // dt/(rho0 dzc_(k+1/2))    (0 at k = nz-1)
    const double *lza;    // a_k = 1/(dzf_k dzc_(k-1/2)), 0 at k = 0
    const double *lzc;    // c_k = 1/(dzf_k dzc_(k+1/2)), 0 at k = nz-1
    const double *izf;    // 1/dzf_k
    const double *dzf;    // dzf_k
    const double *dzc;    // dzc_(k+1/2), 0 at k = nz-1
    double inv_lz;        // 1 / sum_k dzf_k
    double sigma;         // 1/(4 nx ny)
    // mixed-mode stopping rule
    double div_scale;     // (dt/rho0) dx: max|D u| dx = div_scale max|f - L p|
    double inv_3n;        // 1/(3 nx ny nz)
    double div_tol;       // < 0: divergence criterion off
    const double *usq;    // sum of u*^2 over all faces (device scalar)
    int flux_df;          // 1: the face flux's split term in double-float (mixed plans)
};

// Mixed-mode stopping rule, evaluated by one thread once max|r| is known:
// relres <= tol and, unless disabled, the divergence the correction will
// leave, max|D u| dx / U = (dt/rho0) max|r| dx / U, <= div_tol.  The
// divergence rule is a bound through the FP64 residual, whose own rounding
// (about eps max|p| / h^2 of the stencil terms) can exceed div_tol U when U
// is small against the pressure correction; once a sweep no longer halves
// max|r| (rmax_prev >= 0: the previous evaluation) the residual is at that
// floor and further sweeps cannot lower it, so the solve stops there (the
// divergence it reached is measured after the correction, div_metric).
template <bool CG>
__device__ __forceinline__ bool refine_done(const GridDev &g, double rmax, double fmax, double tol,
                                            double rmax_prev, double *rel_out) {
    const double rel = fmax > 0.0 ? rmax / fmax : rmax;
    *rel_out = rel;
    if (!(rel <= tol)) return false;
    if (g.div_tol < 0.0) return true;
    const double U = sqrt((CG ? __ldcg(g.usq) : *g.usq) * g.inv_3n);
    if (U > 0.0 ? rmax * g.div_scale / U <= g.div_tol : rmax == 0.0) return true;
    return rmax_prev >= 0.0 && rmax > 0.5 * rmax_prev;  // stagnated at the evaluation floor
}

__device__ __forceinline__ size_t cidx(const GridDev &g, int i, int j, int k) {
    return ((size_t)k * g.ny + j) * (size_t)g.nx + i;
}

// Every kernel body below works on a "virtual block" VB (the CTA-level
// coordinates it would get from blockIdx) so that the same code runs as a
// stand-alone kernel and as a work item of the persistent batch kernel.
// CG selects how data written earlier in the same launch is read: the
// persistent kernel reads such data with ld.global.cg (L2 only), because a
// line another SM has rewritten may still sit in this SM's L1.
struct VB {
    int x, y, z;
};
__device__ __forceinline__ VB vb_of_grid() { return VB{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z}; }

template <bool CG, typename T> __device__ __forceinline__ T ldp(const T *p) {
    if (CG) return __ldcg(p);
    return *p;
}

// ---------------------------------------------------------------------------
// Provisional face flux, stored scaled by dt:  q' = dt q  (3 face families).
//
// The split coefficient gamma_f = beta_f - 1/rho0 is formed without the
// cancellation of that difference: with rho_f - rho0 = |drho| psi_f, where
// psi = phi when rho0 = rho_g and psi = 1 - phi when rho0 = rho_l,
//     gamma_f = -(|drho| / rho0) psi_f beta_f,
// so gamma_f keeps the relative accuracy of the division (and is exactly 0
// in the pure rho0 phase).  With t = psi_a + psi_b and s = rho_a + rho_b =
// 2 rho0 + |drho| t (so beta_f = 2/s) and kappa = t/s,
//     q' = dt q = u* - dt gamma_f (phat_b - phat_a)/h = u* + (dt |drho|/(rho0 h)) kappa dphat.
// dt |drho|/(rho0 h) is folded into the denominator: with s' = a' t + r'
// (a' = rho0 h/dt, r' = 2 rho0^2 h/(dt |drho|)),  q' = u* + (t/s') dphat.
// t/s' comes from an FP32 quotient refined by one Newton step in FP64,
// kappa' = k0 + r0 (t - s' k0) (r0 the FP32 reciprocal of s'), which squares
// the FP32 error (relative error about 2^-43).  The FP32 seed is taken of
// s' 2^-sh, sh = exponent(r') + fsh, which puts it inside [2^-102, 2^102]
// for any density ratio the plan accepts; all FP64 <-> FP32 moves are integer
// operations.  psi = 1 - phi (rho0 = rho_l) is formed once per cell.
// 6 FP64 instructions per face.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int seed_shift(double r, int fsh) {
    return ((__double2hiint(r) >> 20) & 0x7ff) - 1023 + fsh;
}

__device__ __forceinline__ double face_flux(double psi_a, double psi_b, double ph_a, double ph_b,
                                            double ustar, double ap, double rp, int fsh) {
    const int sh = seed_shift(rp, fsh);
    const double t = psi_a + psi_b;
    const double s = fmaT(ap, t, rp);
    const float tf = f64_to_f32_shift(t, 0);
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f64_to_f32_shift(s, sh)));
    const double k0 = f32_to_f64_shift(tf * rf, -sh);
    const double r0 = f32_to_f64_shift(rf, -sh);
    const double kappa = fmaT(r0, fmaT(-s, k0, t), k0);
    return fmaT(kappa, ph_b - ph_a, ustar);
}

// |x| 2^-64 as FP32 (truncated; 0 below 2^-190, FLT_MAX from 2^192 up), by
// integer operations: the squares of the U statistic of the stopping rule
// are summed in FP32 (U only scales a threshold).
__device__ __forceinline__ float abs_scaled_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
    const unsigned lo = (unsigned)__double2loint(x);
    const int e = (int)(hi >> 20) - 64;
    if (e <= 896) return 0.f;
    if (e >= 896 + 255) return 3.40282347e38f;
    return __uint_as_float(((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

constexpr int FLUX_BX = 32, FLUX_BY = 8;

// One CTA covers a 32 x 8 (i, j) tile and marches up kc planes; phat and phi
// of each plane sit in shared memory with a one-cell halo in +x and +y, and
// the +z neighbour read in one plane is carried as the centre of the next,
// so phat (and psi) is evaluated about once per cell.  The optional sum of
// u*^2 (for U of the stopping rule) is accumulated in FP32 on |u*| 2^-64.
template <bool RHO0_IS_G>
__device__ __forceinline__ void flux_body(const GridDev &g, int kc, VB vb, const double *phi,
                                          const double *pn, const double *pnm1, const double *u,
                                          const double *v, const double *w, double *qx, double *qy,
                                          double *qz, double *usq_slot) {
    __shared__ double s_ph[FLUX_BY + 1][FLUX_BX + 1];
    __shared__ double s_phi[FLUX_BY + 1][FLUX_BX + 1];
    const int tid = block_tid();
    const int tx = tid & (FLUX_BX - 1), ty = tid / FLUX_BX;
    const int i0 = vb.x * FLUX_BX, j0 = vb.y * FLUX_BY;
    const int i = i0 + tx, j = j0 + ty;
    const int k0 = vb.z * kc;
    const int k1 = min(k0 + kc, g.nz);
    const bool in = (i < g.nx && j < g.ny);
    const size_t plane = (size_t)g.nx * g.ny;
    // source cell of every tile slot: wrap (periodic) or clamp (wall; the
    // value of a clamped slot is never used)
    auto src_i = [&](int ii) { return ii < g.nx ? ii : (g.bcx == BC_PERIODIC ? ii % g.nx : g.nx - 1); };
    auto src_j = [&](int jj) { return jj < g.ny ? jj : (g.bcy == BC_PERIODIC ? jj % g.ny : g.ny - 1); };
    const size_t own = (size_t)src_j(j) * g.nx + src_i(i);
    // halo slot handled by this thread: tid < 32 -> row FLUX_BY, 32..39 -> column FLUX_BX
    int hy = -1, hx = -1;
    size_t hoff = 0;
    if (tid < FLUX_BX) {
        hy = FLUX_BY;
        hx = tid;
    } else if (tid < FLUX_BX + FLUX_BY) {
        hy = tid - FLUX_BX;
        hx = FLUX_BX;
    }
    if (hy >= 0) hoff = (size_t)src_j(j0 + hy) * g.nx + src_i(i0 + hx);
    // psi of one cell: phi (rho0 = rho_g) or 1 - phi (rho0 = rho_l)
    auto psi = [&](size_t at) { return RHO0_IS_G ? phi[at] : 1.0 - phi[at]; };
    const bool var = g.var_rho != 0;
    double ph_c = 0.0, psi_c = 0.0;
    float usq = 0.f;
    for (int k = k0; k < k1; ++k) {
        const size_t base = (size_t)k * plane;
        if (k == k0) {
            psi_c = psi(base + own);
            ph_c = fmaT(2.0, pn[base + own], -pnm1[base + own]);
        }
        s_ph[ty][tx] = ph_c;
        s_phi[ty][tx] = psi_c;
        if (hy >= 0) {
            s_phi[hy][hx] = psi(base + hoff);
            s_ph[hy][hx] = fmaT(2.0, pn[base + hoff], -pnm1[base + hoff]);
        }
        __syncthreads();
        double ph_t = 0.0, psi_t = 0.0;
        const bool top_face = k + 1 < g.nz || g.perz;  // periodic z: the seam joins plane 0
        if (top_face) {
            const size_t nxt = (k + 1 < g.nz) ? base + plane : 0;
            psi_t = psi(nxt + own);
            ph_t = fmaT(2.0, pn[nxt + own], -pnm1[nxt + own]);
        }
        if (in) {
            const size_t c = base + (size_t)j * g.nx + i;
            const double uc = u[c], vc = v[c], wc = w[c];
            if (usq_slot) {
                const float a = abs_scaled_f32(uc), b = abs_scaled_f32(vc), d = abs_scaled_f32(wc);
                usq = fmaf(a, a, fmaf(b, b, fmaf(d, d, usq)));
            }
            double q = 0.0;
            if (!(g.bcx == BC_NEUMANN && i == g.nx - 1))
                q = var ? face_flux(psi_c, s_phi[ty][tx + 1], ph_c, s_ph[ty][tx + 1], uc, g.fax, g.frx, g.fsh) : uc;
            qx[c] = q;
            q = 0.0;
            if (!(g.bcy == BC_NEUMANN && j == g.ny - 1))
                q = var ? face_flux(psi_c, s_phi[ty + 1][tx], ph_c, s_ph[ty + 1][tx], vc, g.fay, g.fry, g.fsh) : vc;
            qy[c] = q;
            q = 0.0;
            if (top_face) q = var ? face_flux(psi_c, psi_t, ph_c, ph_t, wc, g.faz[k], g.frz[k], g.fsh) : wc;
            qz[c] = q;
        }
        ph_c = ph_t;
        psi_c = psi_t;
        __syncthreads();
    }
    if (usq_slot) {
        // back to FP64 and to the unscaled square (x 2^128), integer-only
        const double sm = block_sum(f32_to_f64_shift(usq, 128));
        if (tid == 0) *usq_slot = sm;
    }
}

// Mixed plans: the same face flux with its density factor in double-float on
// the FP32 pipe.  FP64 issues at 2 instructions per clock per SM against 128
// for FP32, and the FP64 body above spends 19 FP64 instructions per cell;
// here phat = 2 p^n - p^(n-1) keeps its one FP64 FMA per cell (the same value
// the FP64 body forms) and each face spends two FP64 instructions,
// q' = u* + kappa (phat_b - phat_a): the difference and the multiply-add, as
// the FP64 body ends:
//   * psi (= phi, or 1 - phi when rho0 = rho_l) as a float pair, 2^-47 |phi|;
//   * t = psi_a + psi_b, s' = a' t + r' and kappa = t / s' in double-float,
//     with a' and r' scaled by 2^-sh (the seed shift of the FP64 body), which
//     keeps s' near [2^-fsh, 2^(2+fsh)] and kappa within float range for
//     every density ratio the plan accepts; kappa is scaled back by 2^sh when
//     its two floats are merged into one double (integer operations,
//     df_pair_to_f64_shift);
//   * relative error of kappa about 2^-44, of the difference 2^-53; the pure
//     rho0 phase (psi = 0 on both sides) gives kappa = 0 and q' = u* exactly,
//     as in the FP64 body.
// The divergence identity D(u) = (dt/rho0)(f - L_h p) does not depend on
// this precision: the right-hand side and the correction read the same
// stored q'.
__device__ __forceinline__ double face_flux_df(float2 psi_a, float2 psi_b, double ph_a, double ph_b,
                                               double ustar, float2 A, float2 R, int sh) {
    const float2 t = df_add(psi_a, psi_b);
    const float2 kap = df_div(t, df_add(df_mul(t, A), R));
    const double kd = df_pair_to_f64_shift(kap, -sh);
    return fmaT(kd, __dsub_rn(ph_b, ph_a), ustar);
}

// The double-float flux tile: the tile, halo and face order of flux_body;
// phat (FP64) and psi (as a float pair) of each plane sit in shared memory, and one thread splits the z-face constants a', r' of the
// plane for the others.  The march is software-pipelined one plane ahead:
// while plane k is evaluated, the loads of plane k+1's face values u*, v*, w*
// and halo cell and of the own cell above plane k+1 are in flight, so
// neither the barrier nor the faces wait on a fresh load.
template <bool RHO0_IS_G>
__device__ __forceinline__ void flux_body_df(const GridDev &g, int kc, VB vb, const double *phi,
                                             const double *pn, const double *pnm1, const double *u,
                                             const double *v, const double *w, double *qx, double *qy,
                                             double *qz, double *usq_slot) {
    __shared__ double s_ph[FLUX_BY + 1][FLUX_BX + 1];
    __shared__ float2 s_psi[FLUX_BY + 1][FLUX_BX + 1];
    __shared__ float2 s_zc[2];
    __shared__ int s_zsh;
    const int tid = block_tid();
    const int tx = tid & (FLUX_BX - 1), ty = tid / FLUX_BX;
    const int i0 = vb.x * FLUX_BX, j0 = vb.y * FLUX_BY;
    const int i = i0 + tx, j = j0 + ty;
    const int k0 = vb.z * kc;
    const int k1 = min(k0 + kc, g.nz);
    const bool in = (i < g.nx && j < g.ny);
    const size_t plane = (size_t)g.nx * g.ny;
    auto src_i = [&](int ii) { return ii < g.nx ? ii : (g.bcx == BC_PERIODIC ? ii % g.nx : g.nx - 1); };
    auto src_j = [&](int jj) { return jj < g.ny ? jj : (g.bcy == BC_PERIODIC ? jj % g.ny : g.ny - 1); };
    const size_t own = (size_t)src_j(j) * g.nx + src_i(i);
    const size_t cell = (size_t)(in ? j : 0) * g.nx + (in ? i : 0);
    int hy = -1, hx = -1;
    size_t hoff = 0;
    if (tid < FLUX_BX) {
        hy = FLUX_BY;
        hx = tid;
    } else if (tid < FLUX_BX + FLUX_BY) {
        hy = tid - FLUX_BX;
        hx = FLUX_BX;
    }
    if (hy >= 0) hoff = (size_t)src_j(j0 + hy) * g.nx + src_i(i0 + hx);
    // raw FP64 values of one cell (phi, p^n, p^(n-1)) and their split forms
    struct Raw {
        double phi, pn, pm;
    };
    auto load = [&](size_t at) { return Raw{phi[at], pn[at], pnm1[at]}; };
    auto psi = [&](const Raw &r) {
        const float2 f = f64_split(r.phi);
        return RHO0_IS_G ? f : df_add(make_float2(1.f, 0.f), df_neg(f));
    };
    auto phat = [&](const Raw &r) { return fmaT(2.0, r.pn, -r.pm); };
    // the plane above plane kk (periodic z: the seam joins plane 0); -1: none
    auto above = [&](int kk) { return kk + 1 < g.nz ? kk + 1 : (g.perz ? 0 : -1); };
    const bool var = g.var_rho != 0;
    const int shx = var ? seed_shift(g.frx, g.fsh) : 0, shy = var ? seed_shift(g.fry, g.fsh) : 0;
    const float2 Ax = var ? f64_split_sh(g.fax, shx) : make_float2(0.f, 0.f);
    const float2 Rx = var ? f64_split_sh(g.frx, shx) : make_float2(0.f, 0.f);
    const float2 Ay = var ? f64_split_sh(g.fay, shy) : make_float2(0.f, 0.f);
    const float2 Ry = var ? f64_split_sh(g.fry, shy) : make_float2(0.f, 0.f);
    float usq = 0.f;
    // the pipeline's first stage: plane k0's own cell (split), halo cell and
    // face values, and the own cell above it; every virtual block holds at
    // least one plane (k0 < k1 <= nz)
    const Raw c0 = load((size_t)k0 * plane + own);
    float2 psi_c = psi(c0);
    double ph_c = phat(c0);
    Raw hr{0.0, 0.0, 0.0}, tr{0.0, 0.0, 0.0};
    double uc = 0.0, vc = 0.0, wc = 0.0;
    if (hy >= 0) hr = load((size_t)k0 * plane + hoff);
    if (above(k0) >= 0) tr = load((size_t)above(k0) * plane + own);
    if (in) {
        const size_t c = (size_t)k0 * plane + cell;
        uc = u[c];
        vc = v[c];
        wc = w[c];
    }
    for (int k = k0; k < k1; ++k) {
        const size_t base = (size_t)k * plane;
        const int kt = above(k);
        const bool more = k + 1 < k1;
        // the next stage's loads
        Raw hr_n{0.0, 0.0, 0.0}, tr_n{0.0, 0.0, 0.0};
        double un = 0.0, vn = 0.0, wn = 0.0;
        if (more) {
            if (hy >= 0) hr_n = load(base + plane + hoff);
            if (above(k + 1) >= 0) tr_n = load((size_t)above(k + 1) * plane + own);
            if (in) {
                const size_t c = base + plane + cell;
                un = u[c];
                vn = v[c];
                wn = w[c];
            }
        }
        s_ph[ty][tx] = ph_c;
        s_psi[ty][tx] = psi_c;
        if (hy >= 0) {
            s_psi[hy][hx] = psi(hr);
            s_ph[hy][hx] = phat(hr);
        }
        if (tid == FLUX_BX * FLUX_BY - 1 && var && kt >= 0) {
            // r' > 0 on every face that exists; the top wall's zero entry is never split
            const double rz = g.frz[k];
            const int sh = seed_shift(rz, g.fsh);
            s_zc[0] = f64_split_sh(g.faz[k], sh);
            s_zc[1] = f64_split_sh(rz, sh);
            s_zsh = sh;
        }
        float2 psi_t = make_float2(0.f, 0.f);
        double ph_t = 0.0;
        if (kt >= 0) {
            psi_t = psi(tr);
            ph_t = phat(tr);
        }
        __syncthreads();
        if (in) {
            const size_t c = base + cell;
            if (usq_slot) {
                const float a = abs_scaled_f32(uc), b = abs_scaled_f32(vc), d = abs_scaled_f32(wc);
                usq = fmaf(a, a, fmaf(b, b, fmaf(d, d, usq)));
            }
            double q = 0.0;
            if (!(g.bcx == BC_NEUMANN && i == g.nx - 1)) {
                q = var ? face_flux_df(psi_c, s_psi[ty][tx + 1], ph_c, s_ph[ty][tx + 1], uc, Ax, Rx, shx) : uc;
            }
            qx[c] = q;
            q = 0.0;
            if (!(g.bcy == BC_NEUMANN && j == g.ny - 1)) {
                q = var ? face_flux_df(psi_c, s_psi[ty + 1][tx], ph_c, s_ph[ty + 1][tx], vc, Ay, Ry, shy) : vc;
            }
            qy[c] = q;
            q = 0.0;
            if (kt >= 0) q = var ? face_flux_df(psi_c, psi_t, ph_c, ph_t, wc, s_zc[0], s_zc[1], s_zsh) : wc;
            qz[c] = q;
        }
        ph_c = ph_t;
        psi_c = psi_t;
        hr = hr_n;
        tr = tr_n;
        uc = un;
        vc = vn;
        wc = wn;
        __syncthreads();
    }
    if (usq_slot) {
        const double sm = block_sum(f32_to_f64_shift(usq, 128));
        if (tid == 0) *usq_slot = sm;
    }
}

// The flux tile of a plan: double-float split term on mixed plans
// (g.flux_df), FP64 otherwise.
template <bool RHO0_IS_G>
__device__ __forceinline__ void flux_any(const GridDev &g, int kc, VB vb, const double *phi, const double *pn,
                                         const double *pnm1, const double *u, const double *v,
                                         const double *w, double *qx, double *qy, double *qz,
                                         double *usq_slot) {
    if (g.flux_df)
        flux_body_df<RHO0_IS_G>(g, kc, vb, phi, pn, pnm1, u, v, w, qx, qy, qz, usq_slot);
    else
        flux_body<RHO0_IS_G>(g, kc, vb, phi, pn, pnm1, u, v, w, qx, qy, qz, usq_slot);
}

template <bool RHO0_IS_G>
__global__ void __launch_bounds__(256) k_flux(GridDev g, int kc, const double *__restrict__ phi,
                                              const double *__restrict__ pn,
                                              const double *__restrict__ pnm1,
                                              const double *__restrict__ u,
                                              const double *__restrict__ v,
                                              const double *__restrict__ w,
                                              double *__restrict__ qx, double *__restrict__ qy,
                                              double *__restrict__ qz,
                                              double *__restrict__ usq_part) {
    double *slot = usq_part ? usq_part + ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x
                            : nullptr;
    flux_body<RHO0_IS_G>(g, kc, vb_of_grid(), phi, pn, pnm1, u, v, w, qx, qy, qz, slot);
}

// The double-float body (mixed plans, g.flux_df = 1) as a kernel of its own,
// held to four CTAs per SM (64 registers for its one-plane-ahead loads).
template <bool RHO0_IS_G>
__global__ void __launch_bounds__(256, 4) k_flux_df(GridDev g, int kc, const double *__restrict__ phi,
                                                    const double *__restrict__ pn,
                                                    const double *__restrict__ pnm1,
                                                    const double *__restrict__ u,
                                                    const double *__restrict__ v,
                                                    const double *__restrict__ w,
                                                    double *__restrict__ qx, double *__restrict__ qy,
                                                    double *__restrict__ qz,
                                                    double *__restrict__ usq_part) {
    double *slot = usq_part ? usq_part + ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x
                            : nullptr;
    flux_body_df<RHO0_IS_G>(g, kc, vb_of_grid(), phi, pn, pnm1, u, v, w, qx, qy, qz, slot);
}

// Deterministic final sum of per-block partials (one block).
template <bool CG>
__device__ __forceinline__ void sum_partials_body(const double *part, int n, double *out) {
    double s = 0.0;
    for (int t = block_tid(); t < n; t += block_nthreads()) s += ldp<CG>(part + t);
    s = block_sum(s);
    if (block_tid() == 0) *out = s;
}
__global__ void k_sum_partials(const double *__restrict__ part, int n, double *__restrict__ out) {
    sum_partials_body<false>(part, n, out);
}

// rho0-weighted divergence of q' at one cell; cx, cy, cz are rho0/(dt h) (maybe scaled).
// (split into its loads and its arithmetic, so that a pass can issue the
// loads of several cells before their arithmetic)
struct QFaces {
    double qe, qw, qn, qs, qt, qb;
};
template <bool CG>
__device__ __forceinline__ QFaces div_q_ld(const GridDev &g, int i, int j, int k, const double *qx,
                                           const double *qy, const double *qz) {
    const size_t c = cidx(g, i, j, k);
    QFaces q;
    q.qe = ldp<CG>(qx + c);
    q.qw = (i > 0) ? ldp<CG>(qx + c - 1) : (g.bcx == BC_PERIODIC ? ldp<CG>(qx + c + g.nx - 1) : 0.0);
    q.qn = ldp<CG>(qy + c);
    q.qs = (j > 0) ? ldp<CG>(qy + c - g.nx)
                   : (g.bcy == BC_PERIODIC ? ldp<CG>(qy + c + (size_t)(g.ny - 1) * g.nx) : 0.0);
    q.qt = ldp<CG>(qz + c);
    q.qb = (k > 0) ? ldp<CG>(qz + c - (size_t)g.nx * g.ny)
                   : (g.perz ? ldp<CG>(qz + c + (size_t)(g.nz - 1) * g.nx * g.ny) : 0.0);
    return q;
}
__device__ __forceinline__ double div_q_eval(const QFaces &q, double cx, double cy, double cz) {
    return fmaT(cx, q.qe - q.qw, fmaT(cy, q.qn - q.qs, mulT(cz, q.qt - q.qb)));
}
template <bool CG>
__device__ __forceinline__ double div_q(const GridDev &g, int i, int j, int k, double cx, double cy,
                                        double cz, const double *qx, const double *qy,
                                        const double *qz) {
    return div_q_eval(div_q_ld<CG>(g, i, j, k, qx, qy, qz), cx, cy, cz);
}
// The same divergence in double-float (the mixed plans' first x-pass): each
// face value as a float pair (f64_split, 2^-47 relative), the differences,
// their products with the split constants and the sum in double-float on the
// FP32 pipe, f moved to FP64 with one addition.  Error about 2^-46 max|q'| c,
// the size of the double-float flux's own rounding of q'; the divergence the
// correction leaves sees it as (dt/rho0)|df| dx/U, about 2^-46 max|q'|/U.
// q' = 0 on all six faces gives f = 0 exactly.
__device__ __forceinline__ double div_q_eval_df(const QFaces &q, float2 cx, float2 cy, float2 cz) {
    const float2 ex = df_add(f64_split(q.qe), df_neg(f64_split(q.qw)));
    const float2 ey = df_add(f64_split(q.qn), df_neg(f64_split(q.qs)));
    const float2 ez = df_add(f64_split(q.qt), df_neg(f64_split(q.qb)));
    const float2 f = df_add(df_add(df_mul(ex, cx), df_mul(ey, cy)), df_mul(ez, cz));
    return __dadd_rn(f32_to_f64_shift(f.x, 0), f32_to_f64_shift(f.y, 0));
}

// L_h p at one cell in flux (difference) form: each face difference is
// formed first, so a smooth p loses no accuracy to cancellation.  Wall faces
// carry zero flux (ghost value = centre value).
template <bool CG>
__device__ __forceinline__ double lap(const GridDev &g, int i, int j, int k, const double *p) {
    const size_t c = cidx(g, i, j, k);
    const double pc = ldp<CG>(p + c);
    double pe, pw, pn_, ps;
    if (i < g.nx - 1) pe = ldp<CG>(p + c + 1);
    else pe = (g.bcx == BC_PERIODIC) ? ldp<CG>(p + c - i) : pc;
    if (i > 0) pw = ldp<CG>(p + c - 1);
    else pw = (g.bcx == BC_PERIODIC) ? ldp<CG>(p + c + g.nx - 1) : pc;
    if (j < g.ny - 1) pn_ = ldp<CG>(p + c + g.nx);
    else pn_ = (g.bcy == BC_PERIODIC) ? ldp<CG>(p + c - (size_t)j * g.nx) : pc;
    if (j > 0) ps = ldp<CG>(p + c - g.nx);
    else ps = (g.bcy == BC_PERIODIC) ? ldp<CG>(p + c + (size_t)(g.ny - 1) * g.nx) : pc;
    const size_t pl = (size_t)g.nx * g.ny;
    const double pt = (k < g.nz - 1) ? ldp<CG>(p + c + pl) : (g.perz ? ldp<CG>(p + c - k * pl) : pc);
    const double pb = (k > 0) ? ldp<CG>(p + c - pl) : (g.perz ? ldp<CG>(p + c + (g.nz - 1) * pl) : pc);
    double acc = mulT((pe - pc) - (pc - pw), g.idx2);
    acc = fmaT((pn_ - pc) - (pc - ps), g.idy2, acc);
    acc = fmaT(g.lzc[k], pt - pc, acc);
    return fmaT(-g.lza[k], pc - pb, acc);
}

enum {
    XF_F64_DIVQ = 0,   // FP64 mode: sigma rho0 D(q), FP64 transform
    XF_MIX_DIVQ = 1,   // mixed: f = rho0 D(q) (double-float) stored in FP64, FP32 transform of sigma f
    XF_MIX_LOAD = 2    // transform, in place, of a stored right-hand side: mixed mode's FP32
                       // sigma 2^-e r; with T = double the preconditioner of the
                       // variable-coefficient solve (sigma r)
};

struct XArgs {
    const double *qx, *qy, *qz;  // divergence sources
    const double *p;             // FP64-mode check: the pressure
    double *f_out;               // MIX_DIVQ: f stored here
    void *out;                   // transformed output (T), [nz][ny][nx]; MIX_LOAD: also the input
    DevStats *st;
    int track_fmax;              // F64_DIVQ: record max|sigma f|
};

// Shapes of the transform passes (host and device): x-pass line pairs per
// CTA (about 1024 complex values per tile) and y-pass columns per tile
// (rows of 8 doubles or 16 floats, 64 B, at n = 256; about 1024 (FP64) or
// 2048 (FP32) complex values per tile).
constexpr int x_lines_per_cta(int n) {
    const int L = 1024 / n;
    return L < 1 ? 1 : (L > 16 ? 16 : L);
}
constexpr int y_tile_cols(int n, bool fp32 = false) {
    const int cap = fp32 ? 16 : 8;
    const int L = (fp32 ? 2048 : 1024) / n;
    return 2 * (L < 2 ? 2 : (L > cap ? cap : L));
}

constexpr int PASS_U = 4;   // global loads per thread issued together in the pass load loops
constexpr int XDIV_U = 2;   // cells per thread whose six face loads the divergence issues together
constexpr int PASS_UC = 2;  // spectral pairs per thread loaded together before the inverse combine

// The transform of a pass: length-specialised when NF != 0 (NF = the length
// of a periodic direction), else driven by the runtime descriptor.
template <typename T, bool INV, int NF>
__device__ __forceinline__ const typename C2<T>::t *fft_any(typename C2<T>::t *a, typename C2<T>::t *b,
                                                            int L, int ls, const FFTDesc &D,
                                                            const typename C2<T>::t *tw) {
    if constexpr (NF != 0) return fft_fixed<T, INV, NF>(a, b, L, ls, tw);
    else return fft_lines<T, INV>(a, b, L, ls, D, tw);
}

// DCT-IV (times 2) of the R real lines of a tile, in shared memory, by one
// complex FFT of half the length per line (n = 2M):
//     z_t = (x_(2t) + i x_(n-1-2t)) exp(-i pi (4t+1)/(4n)),   t < M,
//     Z = FFT_M(z),   Y_k = 2 Z_k exp(-i pi k/n),
//     X_(2k) = Re Y_k,   X_(n-1-2k) = -Im Y_k.
// The DCT-IV is its own inverse up to n/2, so the forward and the inverse
// passes run the same steps (the round trip then scales by 2n, as the other
// kinds do).  ld(r, i) returns sample i of line r, st(r, k, v) stores value k;
// LFAST orders the load and store loops with the line index fastest (the
// y-pass, whose lines are columns), else the sample index fastest.  tw_s holds
// the M twiddles of the length-M FFT then the M pre-twiddles, cs_s the M
// post-twiddles; A and B hold R lines of M complex values each.
template <typename T, bool LFAST, typename LD, typename ST>
__device__ __forceinline__ void dct4_tile(const FFTDesc &D, int R, typename C2<T>::t *A,
                                          typename C2<T>::t *B, const typename C2<T>::t *tw_s,
                                          const typename C2<T>::t *cs_s, LD &&ld, ST &&st) {
    typedef typename C2<T>::t T2;
    const int n = D.n, M = n >> 1;
    const unsigned rR = fdiv_recip(R);
    const T2 *pre = tw_s + M;
    // 1. pack the two halves of each line into M complex values
    const int total = R * n;
    for (int base = threadIdx.x; base < total; base += PASS_U * blockDim.x) {
        T v[PASS_U];
#pragma unroll
        for (int u = 0; u < PASS_U; ++u) {
            const int idx = base + u * blockDim.x;
            int r, i;
            if (LFAST) { i = fdiv(idx, R, rR); r = idx - i * R; }
            else { r = fdiv(idx, n, D.rn); i = idx - r * n; }
            v[u] = idx < total ? ld(r, i) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < PASS_U; ++u) {
            const int idx = base + u * blockDim.x;
            int r, i;
            if (LFAST) { i = fdiv(idx, R, rR); r = idx - i * R; }
            else { r = fdiv(idx, n, D.rn); i = idx - r * n; }
            const int t = (i & 1) ? (n - 1 - i) >> 1 : i >> 1;
            if (idx < total) ((T *)(A + r * M))[2 * t + (i & 1)] = v[u];
        }
    }
    __syncthreads();
    // 2. pre-twiddle
    for (int t = threadIdx.x; t < R * M; t += blockDim.x) {
        const int r = fdiv(t, M, D.rK), q = t - r * M;
        const T2 a = A[r * M + q], w = pre[q];
        A[r * M + q] = mk2(fmaT(a.x, w.x, -mulT(a.y, w.y)), fmaT(a.x, w.y, mulT(a.y, w.x)));
    }
    __syncthreads();
    // 3. complex FFT of length M (the descriptor's stages)
    const T2 *Z = fft_lines<T, false>(A, B, R, M, D, tw_s);
    // 4. post-twiddle (carrying the factor 2) and store
    for (int t = threadIdx.x; t < R * M; t += blockDim.x) {
        int r, k;
        if (LFAST) { k = fdiv(t, R, rR); r = t - k * R; }
        else { r = fdiv(t, M, D.rK); k = t - r * M; }
        const T2 z = Z[r * M + k], w = cs_s[k];
        st(r, 2 * k, fmaT(z.x, w.x, -mulT(z.y, w.y)));
        st(r, n - 1 - 2 * k, -fmaT(z.x, w.y, mulT(z.y, w.x)));
    }
}

// Forward x-pass: per CTA 2L real x-lines (flattened line index (k, j)).
template <typename T, int MODE, bool CG, int NF = 0>
__device__ __forceinline__ void xfwd_body(const GridDev &g, const FFTDesc &D, int L, const XArgs &a,
                                          int bx, int ntiles, unsigned char *smem_raw) {
    typedef typename C2<T>::t T2;
    constexpr bool FX = NF != 0;  // compile-time length (periodic)
    const int n = FX ? NF : D.n, ls = n + 1;
    const int kind = FX ? (int)KIND_PERIODIC : D.kind;
    T2 *tw_s = (T2 *)smem_raw;
    T2 *cs_s = tw_s + n;
    T2 *A = cs_s + (n / 2 + 2);
    T2 *B = A + L * ls;
    if (MODE == XF_MIX_LOAD && ldp<CG>(&a.st->converged)) return;
    load_tables<T>(D, tw_s, cs_s);
    const int nlines = g.ny * g.nz;
    const int line0 = bx * 2 * L;
    (void)ntiles;
    if constexpr (!FX && MODE == XF_MIX_LOAD) {
        if (kind == KIND_DCT4) {  // in place on the stored right-hand side
            T *data = (T *)a.out;
            dct4_tile<T, false>(
                D, 2 * L, A, B, tw_s, cs_s,
                [&](int r, int i) -> T {
                    const int line = line0 + r;
                    return line < nlines ? flip_odd(ldp<CG>(data + (size_t)line * n + i), D.flip, i) : (T)0;
                },
                [&](int r, int k, T v) {
                    const int line = line0 + r;
                    if (line < nlines) data[(size_t)line * n + k] = v;
                });
            return;
        }
    }
    unsigned long long mx = 0ull;
    const float scale32 = (float)g.sigma;
    // 1. source values into the packed complex lines
    if (MODE == XF_MIX_LOAD) {  // PASS_U loads per thread in flight
        const int total = 2 * L * n;
        for (int base = threadIdx.x; base < total; base += PASS_U * blockDim.x) {
            T v[PASS_U];
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                v[u] = (idx < total && line0 + r < nlines)
                           ? ldp<CG>((const T *)a.out + (size_t)(line0 + r) * n + i) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                if (idx < total)
                    ((T *)(A + (r >> 1) * ls))[2 * line_pos(i, n, kind) + (r & 1)] =
                        FX ? v[u] : flip_odd(v[u], D.flip, i);
            }
        }
    } else {  // the divergence: the face loads of UD cells per thread issued together
        // (one in the persistent batch kernel, whose 48 registers it would spill)
        constexpr int UD = CG ? 1 : XDIV_U;
        const int total = 2 * L * n;
        for (int base = threadIdx.x; base < total; base += UD * blockDim.x) {
            QFaces qf[UD];
#pragma unroll
            for (int u = 0; u < UD; ++u) {
                const int idx = base + u * blockDim.x;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                const int line = line0 + r;
                if (idx < total && line < nlines) {
                    const int k = fdiv(line, g.ny, g.rny), j = line - k * g.ny;
                    qf[u] = div_q_ld<CG>(g, i, j, k, a.qx, a.qy, a.qz);
                }
            }
#pragma unroll
            for (int u = 0; u < UD; ++u) {
                const int idx = base + u * blockDim.x;
                if (idx >= total) break;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                const int line = line0 + r;
                T val = (T)0;
                if (line < nlines) {
                    const int k = fdiv(line, g.ny, g.rny);
                    if (MODE == XF_F64_DIVQ) {
                        const double f = div_q_eval(qf[u], g.dvx_s, g.dvy_s, g.dvz_s[k]);
                        if (a.track_fmax) mx = umax64(mx, absbits(f));
                        val = (T)f;
                    } else {
                        const double f = div_q_eval_df(qf[u], f64_split(g.dvx), f64_split(g.dvy),
                                                       f64_split(g.dvz[k]));
                        a.f_out[(size_t)line * n + i] = f;
                        mx = umax64(mx, absbits(f));
                        val = (T)(f64_to_f32_shift(f, 0) * scale32);
                    }
                }
                ((T *)(A + (r >> 1) * ls))[2 * line_pos(i, n, kind) + (r & 1)] = val;
            }
        }
    }
    if (MODE == XF_MIX_DIVQ) block_max_atomic(mx, &a.st->fmax_bits);
    if (MODE == XF_F64_DIVQ && a.track_fmax) block_max_atomic(mx, &a.st->fmax_bits);
    __syncthreads();
    // 2. complex FFT
    const T2 *Z = fft_any<T, false, NF>(A, B, L, ls, D, tw_s);
    // 3. separate and store
    T *out = (T *)a.out;
    const int M = n / 2 + 1;
    for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
        const int l = (FX ? t / (NF / 2 + 1) : fdiv(t, M, D.rM)), m = t - l * M;
        const int la = line0 + 2 * l;
        fwd_separate<T>(Z + l * ls, n, m, kind, cs_s, [&](int ab, int ix, T v) {
            const int line = la + ab;
            if (line < nlines) out[(size_t)line * n + ix] = v;
        });
    }
}

// Stand-alone launches of the pass bodies: the grid strides over the pass's
// tiles.  Launched with one block per tile on the main path; a refinement
// pass that is likely to find the solve converged is launched with the
// resident grid (CTAs per SM x SMs) and reads the flag once per block, so
// returning at once costs a few hundred block starts, not one per tile.
// (The flag is set only by the last tile of a residual pass, so no tile of
// the same launch is pending once it is set.)
template <typename T, int MODE, int NF = 0>
__global__ void __launch_bounds__(256) k_xfwd(GridDev g, FFTDesc D, int L, XArgs a, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (MODE == XF_MIX_LOAD && *(volatile const int *)&a.st->converged) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        xfwd_body<T, MODE, false, NF>(g, D, L, a, t, ntiles, smem_raw);
        __syncthreads();  // shared memory is reused by the next tile
    }
}

// FP64-mode check (FIZZY_FLAG_CHECK): relres = max|f - L_h p| / max|f| with
// f = rho0 D(q') recomputed; the last block writes relres.
// Virtual block: x = tile of 256 cells along x, y = j, z = k.
template <bool CG>
__device__ __forceinline__ void residmax_body(const GridDev &g, const XArgs &a, VB vb, int ntiles) {
    const int i = vb.x * blockDim.x + threadIdx.x;
    const int j = vb.y, k = vb.z;
    unsigned long long mx = 0ull, fm = 0ull;
    if (i < g.nx) {
        const double f = div_q<CG>(g, i, j, k, g.dvx, g.dvy, g.dvz[k], a.qx, a.qy, a.qz);
        fm = absbits(f);
        mx = absbits(f - lap<CG>(g, i, j, k, a.p));
    }
    block_max_atomic(mx, &a.st->rmax_bits[0]);
    block_max_atomic(fm, &a.st->fmax_bits);
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(&a.st->done_blocks[0], 1u);
        last = (ticket == (unsigned)ntiles - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double rmax = __longlong_as_double((long long)atomicMax(&a.st->rmax_bits[0], 0ull));
        const double fmax = __longlong_as_double((long long)atomicMax(&a.st->fmax_bits, 0ull));
        a.st->relres = fmax > 0.0 ? rmax / fmax : rmax;
    }
}

// tiles: rgx x-segments of 256 cells per (j, k) row
__global__ void __launch_bounds__(256) k_residmax(GridDev g, XArgs a, int rgx, int ntiles) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int row = t / rgx;
        residmax_body<false>(g, a, VB{t - row * rgx, row % g.ny, row / g.ny}, ntiles);
        __syncthreads();
    }
}

// Forward / inverse y-pass on a tile of TX columns (tile bx) of plane k (in place).
template <typename T, bool INV, bool CG, int NF = 0>
__device__ __forceinline__ void ypass_body(int nx, int ny, const FFTDesc &D, int TX, T *data,
                                           const int *conv, int bx, int kplane,
                                           unsigned char *smem_raw) {
    typedef typename C2<T>::t T2;
    if (conv && ldp<CG>(conv)) return;
    constexpr bool FX = NF != 0;  // compile-time length (periodic)
    const int n = FX ? NF : D.n, ls = n + 1;
    const int kind = FX ? (int)KIND_PERIODIC : D.kind;
    const int L = TX / 2;
    T2 *tw_s = (T2 *)smem_raw;
    T2 *cs_s = tw_s + n;
    T2 *A = cs_s + (n / 2 + 2);
    T2 *B = A + L * ls;
    load_tables<T>(D, tw_s, cs_s);
    const int i0 = bx * TX;
    const int ncols = min(TX, nx - i0);
    T *plane = data + (size_t)kplane * ny * nx + i0;
    if constexpr (!FX) {
        if (kind == KIND_DCT4) {  // the same steps forward and inverse (columns = lines)
            dct4_tile<T, true>(
                D, TX, A, B, tw_s, cs_s,
                [&](int c, int j) -> T {
                    if (c >= ncols) return (T)0;
                    const T v = ldp<CG>(plane + (size_t)j * nx + c);
                    return INV ? v : flip_odd(v, D.flip, j);
                },
                [&](int c, int k, T v) {
                    if (c < ncols) plane[(size_t)k * nx + c] = INV ? flip_odd(v, D.flip, k) : v;
                });
            return;
        }
    }
    const int M = n / 2 + 1;
    const unsigned rTX = fdiv_recip(TX), rL = fdiv_recip(L);
    if (!INV) {
        // PASS_U loads per thread in flight before their shared-memory stores
        const int total = n * TX;
        for (int base = threadIdx.x; base < total; base += PASS_U * blockDim.x) {
            T v[PASS_U];
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int j = fdiv(idx, TX, rTX), c = idx - j * TX;
                v[u] = (idx < total && c < ncols) ? ldp<CG>(plane + (size_t)j * nx + c) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int j = fdiv(idx, TX, rTX), c = idx - j * TX;
                if (idx < total)
                    ((T *)(A + (c >> 1) * ls))[2 * line_pos(j, n, kind) + (c & 1)] =
                        FX ? v[u] : flip_odd(v[u], D.flip, j);
            }
        }
        __syncthreads();
        const T2 *Z = fft_any<T, false, NF>(A, B, L, ls, D, tw_s);
        for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
            const int m = fdiv(t, L, rL), l = t - m * L;
            fwd_separate<T>(Z + l * ls, n, m, kind, cs_s, [&](int ab, int ix, T v) {
                const int c = 2 * l + ab;
                if (c < ncols) plane[(size_t)ix * nx + c] = v;
            });
        }
    } else {
        __syncthreads();
        // the spectral values of PASS_UC pairs (m, n-m) of both lines are
        // loaded before they are combined
        const int total = L * M;
        for (int base = threadIdx.x; base < total; base += PASS_UC * blockDim.x) {
            T v[PASS_UC][4];
#pragma unroll
            for (int u = 0; u < PASS_UC; ++u) {
                const int t = base + u * blockDim.x;
                const int m = fdiv(t, L, rL), l = t - m * L;
                const bool two = m > 0 && 2 * m != n;  // Z[m] and Z[n-m] both read
#pragma unroll
                for (int ab = 0; ab < 2; ++ab) {
                    const int c = 2 * l + ab;
                    const bool ok = t < total && c < ncols;
                    v[u][2 * ab] = ok ? ldp<CG>(plane + (size_t)m * nx + c) : (T)0;
                    v[u][2 * ab + 1] = (ok && two) ? ldp<CG>(plane + (size_t)(n - m) * nx + c) : (T)0;
                }
            }
#pragma unroll
            for (int u = 0; u < PASS_UC; ++u) {
                const int t = base + u * blockDim.x;
                const int m = fdiv(t, L, rL), l = t - m * L;
                if (t < total)
                    inv_combine<T>(A + l * ls, n, m, kind, cs_s,
                                   [&](int ab, int ix) -> T {
                                       return ab == 0 ? (ix == m ? v[u][0] : v[u][1])
                                                      : (ix == m ? v[u][2] : v[u][3]);
                                   });
            }
        }
        __syncthreads();
        const T2 *Z = fft_any<T, true, NF>(A, B, L, ls, D, tw_s);
        for (int idx = threadIdx.x; idx < n * TX; idx += blockDim.x) {
            const int j = fdiv(idx, TX, rTX), c = idx - j * TX;
            if (c < ncols) {
                const T v = ((const T *)(Z + (c >> 1) * ls))[2 * line_pos(j, n, kind) + (c & 1)];
                plane[(size_t)j * nx + c] = FX ? v : flip_odd(v, D.flip, j);
            }
        }
    }
}

// tiles: ygx column tiles per plane, nz planes
template <typename T, bool INV, int NF = 0>
__global__ void __launch_bounds__(256) k_ypass(int nx, int ny, FFTDesc D, int TX, T *data,
                                               const int *conv, int ygx, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (conv && *(volatile const int *)conv) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int k = t / ygx;
        ypass_body<T, INV, false, NF>(nx, ny, D, TX, data, conv, t - k * ygx, k, smem_raw);
        __syncthreads();
    }
}

enum { XI_STORE = 0, XI_ACCUM = 1 };

// Inverse x-pass: per CTA 2L real x-lines; writes p (FP64).
template <typename T, int MODE, bool CG, int NF = 0>
__device__ __forceinline__ void xinv_body(const GridDev &g, const FFTDesc &D, int L, const T *in,
                                          double *p, const DevStats *st, int bx,
                                          unsigned char *smem_raw) {
    typedef typename C2<T>::t T2;
    if (MODE == XI_ACCUM && ldp<CG>(&st->converged)) return;
    constexpr bool FX = NF != 0;  // compile-time length (periodic)
    const int n = FX ? NF : D.n, ls = n + 1;
    const int kind = FX ? (int)KIND_PERIODIC : D.kind;
    T2 *tw_s = (T2 *)smem_raw;
    T2 *cs_s = tw_s + n;
    T2 *A = cs_s + (n / 2 + 2);
    T2 *B = A + L * ls;
    load_tables<T>(D, tw_s, cs_s);
    const int nlines = g.ny * g.nz;
    const int line0 = bx * 2 * L;
    if constexpr (!FX) {
        if (kind == KIND_DCT4) {
            const int es = (MODE == XI_ACCUM) ? exp_of_bits(ldp<CG>(&st->fmax_bits)) : 0;
            dct4_tile<T, false>(
                D, 2 * L, A, B, tw_s, cs_s,
                [&](int r, int k) -> T {
                    const int line = line0 + r;
                    return line < nlines ? ldp<CG>(in + (size_t)line * n + k) : (T)0;
                },
                [&](int r, int i, T v) {
                    const int line = line0 + r;
                    if (line >= nlines) return;
                    v = flip_odd(v, D.flip, i);
                    double *dst = p + (size_t)line * n + i;
                    const double dv = sizeof(T) == 8 ? (double)v : f32_to_f64_shift((float)v, es);
                    if (MODE == XI_STORE) *dst = dv;
                    else *dst = ldp<CG>(dst) + dv;
                });
            return;
        }
    }
    const int M = n / 2 + 1;
    __syncthreads();
    const int total = L * M;
    for (int base = threadIdx.x; base < total; base += PASS_UC * blockDim.x) {
        T v[PASS_UC][4];
#pragma unroll
        for (int u = 0; u < PASS_UC; ++u) {
            const int t = base + u * blockDim.x;
            const int l = (FX ? t / (NF / 2 + 1) : fdiv(t, M, D.rM)), m = t - l * M;
            const bool two = m > 0 && 2 * m != n;  // Z[m] and Z[n-m] both read
#pragma unroll
            for (int ab = 0; ab < 2; ++ab) {
                const int line = line0 + 2 * l + ab;
                const bool ok = t < total && line < nlines;
                v[u][2 * ab] = ok ? ldp<CG>(in + (size_t)line * n + m) : (T)0;
                v[u][2 * ab + 1] = (ok && two) ? ldp<CG>(in + (size_t)line * n + (n - m)) : (T)0;
            }
        }
#pragma unroll
        for (int u = 0; u < PASS_UC; ++u) {
            const int t = base + u * blockDim.x;
            const int l = (FX ? t / (NF / 2 + 1) : fdiv(t, M, D.rM)), m = t - l * M;
            if (t < total)
                inv_combine<T>(A + l * ls, n, m, kind, cs_s,
                               [&](int ab, int ix) -> T {
                                       return ab == 0 ? (ix == m ? v[u][0] : v[u][1])
                                                      : (ix == m ? v[u][2] : v[u][3]);
                                   });
        }
    }
    __syncthreads();
    const T2 *Z = fft_any<T, true, NF>(A, B, L, ls, D, tw_s);
    int ef = 0;
    if (MODE == XI_ACCUM) ef = exp_of_bits(ldp<CG>(&st->fmax_bits));
    if (MODE == XI_STORE) {
        for (int idx = threadIdx.x; idx < 2 * L * n; idx += blockDim.x) {
            const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
            const int line = line0 + r;
            if (line < nlines) {
                T v = ((const T *)(Z + (r >> 1) * ls))[2 * line_pos(i, n, kind) + (r & 1)];
                if (!FX) v = flip_odd(v, D.flip, i);
                double *dst = p + (size_t)line * n + i;
                if (sizeof(T) == 8) *dst = (double)v;
                else *dst = f32_to_f64_shift((float)v, 0);
            }
        }
    } else {  // p += delta: PASS_U loads of p per thread in flight
        const int total = 2 * L * n;
        for (int base = threadIdx.x; base < total; base += PASS_U * blockDim.x) {
            double pv[PASS_U];
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                pv[u] = (idx < total && line0 + r < nlines) ? ldp<CG>(p + (size_t)(line0 + r) * n + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < PASS_U; ++u) {
                const int idx = base + u * blockDim.x;
                const int r = (FX ? idx / NF : fdiv(idx, n, D.rn)), i = idx - r * n;
                if (idx < total && line0 + r < nlines) {
                    T v = ((const T *)(Z + (r >> 1) * ls))[2 * line_pos(i, n, kind) + (r & 1)];
                    if (!FX) v = flip_odd(v, D.flip, i);
                    p[(size_t)(line0 + r) * n + i] = pv[u] + f32_to_f64_shift((float)v, ef);
                }
            }
        }
    }
}

template <typename T, int MODE, int NF = 0>
__global__ void __launch_bounds__(256) k_xinv(GridDev g, FFTDesc D, int L, const T *in, double *p,
                                              const DevStats *st, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (MODE == XI_ACCUM && *(volatile const int *)&st->converged) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        xinv_body<T, MODE, false, NF>(g, D, L, in, p, st, t, smem_raw);
        __syncthreads();
    }
}

// Tridiagonal z-solves, one per (kx, ky) line, with factorisation tables
// m_k and 1/beta_k that depend only on the eigenvalue pair and are stored once
// per distinct pair at index ((k*Uy + uy)*Ux + ux).  In a periodic
// direction the half-complex indices i and nx-i share their eigenvalue and
// so their table.  The forward sweep keeps its modified right-hand side in
// place and the backward sweep overwrites it with the solution.
// The (0,0) line is singular: its right-hand side mean is removed, the fluxes
// are integrated from the bottom wall and the result is given zero
// dzf-weighted mean (the pressure gauge).
constexpr int THOMAS_S = 16;      // ring stages: planes in flight per line
constexpr int THOMAS_U = 4;       // planes per block of the recurrence
constexpr int THOMAS_BLOCK = 32;

// One z-line per thread (forward elimination y_k = f_k - m_k y_(k-1), back
// substitution p_k = (y_k - c_k p_(k+1)) / beta_k, the factors m_k and
// 1/beta_k read from the per-eigenvalue tables).  The line's data and table
// values stream through a cp.async ring in shared memory, THOMAS_S planes
// ahead; the ring is consumed in blocks of THOMAS_U planes (one wait per
// block, all ring loads issued before the recurrence, the refill issued
// before the stores), so the dependent chain of a block is THOMAS_U
// back-to-back FMAs.  Each thread reads only its own ring slots.
template <typename T>
__device__ __forceinline__ void thomas_line_ring(int nz, size_t plane, T *d, size_t ts, size_t tb,
                                                 const T *__restrict__ mtab,
                                                 const T *__restrict__ ibtab,
                                                 const T *__restrict__ cup, T *ring) {
    constexpr int U = THOMAS_U, G = THOMAS_S / THOMAS_U;
    static_assert(THOMAS_S % THOMAS_U == 0, "ring holds whole blocks");
    const int tid = threadIdx.x;
    // slot (stage, item): item 0 = line value, 1 = table value
    auto slot = [&](int stage, int item) -> T * {
        return ring + ((size_t)(stage * 2 + item) * THOMAS_BLOCK + tid);
    };
    const int nb = (nz - 1 + U - 1) / U;  // blocks per sweep (nz - 1 planes each)
    // ---- forward: block b holds planes 1 + bU + q in stages (b % G) U + q
    auto issue_f = [&](int b) {
        const int s0 = (b % G) * U;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = 1 + b * U + q;
            if (k < nz) {
                cp_async<sizeof(T)>(slot(s0 + q, 1), mtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 0), d + (size_t)k * plane);
            }
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int b = 0; b < G; ++b) issue_f(b);
    T prev = d[0];
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        cp_async_wait<G - 1>();
        const int s0 = (b % G) * U, k0 = 1 + b * U;
        T mv[U], fv[U], out[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            mv[q] = *slot(s0 + q, 1);
            fv[q] = *slot(s0 + q, 0);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (k0 + q < nz) prev = fmaT(-mv[q], prev, fv[q]);
            out[q] = prev;
        }
        issue_f(b + G);
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 + q < nz) d[(size_t)(k0 + q) * plane] = out[q];
    }
    cp_async_wait<0>();
    // ---- backward: p_(nz-1) = y_(nz-1)/beta; block b holds planes nz-2-bU-q
    prev = mulT(prev, ibtab[(size_t)(nz - 1) * ts + tb]);
    d[(size_t)(nz - 1) * plane] = prev;
    auto issue_b = [&](int b) {
        const int s0 = (b % G) * U;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = nz - 2 - b * U - q;
            if (k >= 0) {
                cp_async<sizeof(T)>(slot(s0 + q, 1), ibtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 0), d + (size_t)k * plane);
            }
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int b = 0; b < G; ++b) issue_b(b);
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        cp_async_wait<G - 1>();
        const int s0 = (b % G) * U, k0 = nz - 2 - b * U;
        T iv[U], dv[U], cv[U], out[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            iv[q] = *slot(s0 + q, 1);
            dv[q] = *slot(s0 + q, 0);
            cv[q] = (k0 - q >= 0) ? cup[k0 - q] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (k0 - q >= 0) prev = mulT(fmaT(-cv[q], prev, dv[q]), iv[q]);
            out[q] = prev;
        }
        issue_b(b + G);
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 - q >= 0) d[(size_t)(k0 - q) * plane] = out[q];
    }
    cp_async_wait<0>();
}

// Periodic z: each (kx, ky) line is a cyclic tridiagonal system A p = f (the
// seam couples row 0 to p_(nz-1) by a_0 and row nz-1 to p_0 by c_(nz-1)).
// It is solved with the Sherman-Morrison formula: A = B + u v^T with
// u = (gamma, 0, ..., 0, c_(nz-1)), v = (1, 0, ..., 0, a_0/gamma),
// gamma = -b_0, B tridiagonal with its first and last diagonal entries
// changed; then p = y - (v^T y) q with B y = f and q = B^(-1) u / (1 + v^T B^(-1) u).
// The tables hold B's factorisation (m_k, 1/beta_k), q_k, and the weights w_k
// for which v^T y = sum_k w_k g_k, g the forward-eliminated right-hand side
// (back substitution makes y_0 a fixed combination of the g_k), so v^T y is
// accumulated during the forward sweep and the back substitution writes
// p_k = y_k - (v^T y) q_k directly: 5 instructions per point instead of 3,
// one ring item more per stage, and no extra sweep.
template <typename T>
__device__ __forceinline__ void thomas_line_ring_cyc(int nz, size_t plane, T *d, size_t ts, size_t tb,
                                                     const T *__restrict__ mtab,
                                                     const T *__restrict__ ibtab,
                                                     const T *__restrict__ cup,
                                                     const T *__restrict__ wtab,
                                                     const T *__restrict__ qtab, T *ring) {
    constexpr int U = THOMAS_U, G = THOMAS_S / THOMAS_U;
    const int tid = threadIdx.x;
    // slot (stage, item): item 0 = line value, 1 = m_k or 1/beta_k, 2 = w_k or q_k
    auto slot = [&](int stage, int item) -> T * {
        return ring + ((size_t)(stage * 3 + item) * THOMAS_BLOCK + tid);
    };
    const int nb = (nz - 1 + U - 1) / U;
    auto issue_f = [&](int b) {
        const int s0 = (b % G) * U;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = 1 + b * U + q;
            if (k < nz) {
                cp_async<sizeof(T)>(slot(s0 + q, 1), mtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 2), wtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 0), d + (size_t)k * plane);
            }
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int b = 0; b < G; ++b) issue_f(b);
    T prev = d[0];
    T acc = mulT(wtab[tb], prev);  // v^T y, accumulated over k
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        cp_async_wait<G - 1>();
        const int s0 = (b % G) * U, k0 = 1 + b * U;
        T mv[U], wv[U], fv[U], out[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            mv[q] = *slot(s0 + q, 1);
            wv[q] = *slot(s0 + q, 2);
            fv[q] = *slot(s0 + q, 0);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (k0 + q < nz) {
                prev = fmaT(-mv[q], prev, fv[q]);
                acc = fmaT(wv[q], prev, acc);
            }
            out[q] = prev;
        }
        issue_f(b + G);
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 + q < nz) d[(size_t)(k0 + q) * plane] = out[q];
    }
    cp_async_wait<0>();
    const T sv = acc;
    // ---- backward: y carried, p_k = y_k - (v^T y) q_k stored
    prev = mulT(prev, ibtab[(size_t)(nz - 1) * ts + tb]);
    d[(size_t)(nz - 1) * plane] = fmaT(-sv, qtab[(size_t)(nz - 1) * ts + tb], prev);
    auto issue_b = [&](int b) {
        const int s0 = (b % G) * U;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = nz - 2 - b * U - q;
            if (k >= 0) {
                cp_async<sizeof(T)>(slot(s0 + q, 1), ibtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 2), qtab + (size_t)k * ts + tb);
                cp_async<sizeof(T)>(slot(s0 + q, 0), d + (size_t)k * plane);
            }
        }
        cp_async_commit();
    };
#pragma unroll 1
    for (int b = 0; b < G; ++b) issue_b(b);
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        cp_async_wait<G - 1>();
        const int s0 = (b % G) * U, k0 = nz - 2 - b * U;
        T iv[U], qv[U], dv[U], cv[U], out[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            iv[q] = *slot(s0 + q, 1);
            qv[q] = *slot(s0 + q, 2);
            dv[q] = *slot(s0 + q, 0);
            cv[q] = (k0 - q >= 0) ? cup[k0 - q] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (k0 - q >= 0) {
                prev = mulT(fmaT(-cv[q], prev, dv[q]), iv[q]);
                out[q] = fmaT(-sv, qv[q], prev);
            } else {
                out[q] = prev;
            }
        }
        issue_b(b + G);
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (k0 - q >= 0) d[(size_t)(k0 - q) * plane] = out[q];
    }
    cp_async_wait<0>();
}

// The singular (0,0) line, solved by one warp.  With a_k = dzf_k (f_k - fbar)
// (fbar the dzf-weighted mean, removed so the line is compatible), the flux
// through face k+1/2 is the inclusive prefix sum F_(k+1/2) = sum_(k'<=k) a_k'
// (zero flux through the bottom wall) and the pressure is the exclusive prefix
// sum p_k = sum_(k'<k) dzc_(k'+1/2) F_(k'+1/2) (p_0 = 0); both sums run as warp
// scans over chunks of 32 planes.  Finally the dzf-weighted mean of p is
// removed (the pressure gauge).  With periodic z the flux through the seam is
// not zero but a constant C added to every face flux, F_(k+1/2) = C + S_k;
// going once around the periodic line must return to the same pressure,
// sum_k dzc_(k+1/2) F_(k+1/2) = 0, so C = -sum_k dzc_(k+1/2) S_k / sum_k dzc_(k+1/2),
// found by a first scan over the line.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_inclusive_scan(double v, int lane) {
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <typename T, bool CG>
__device__ void singular_line_warp(const GridDev &g, T *d, size_t plane) {
    const int lane = threadIdx.x & 31;
    const int nz = g.nz;
    double s = 0.0;
    for (int k = lane; k < nz; k += 32) s = fmaT(g.dzf[k], (double)ldp<CG>(d + (size_t)k * plane), s);
    const double fbar = mulT(warp_sum(s), g.inv_lz);
    double Fc = 0.0, pc = 0.0, ps = 0.0;
    if (g.perz) {
        double Sc = 0.0, num = 0.0, den = 0.0;
        for (int k0 = 0; k0 < nz; k0 += 32) {
            const int k = k0 + lane;
            double a = 0.0, h = 0.0;
            if (k < nz) {
                a = mulT(g.dzf[k], (double)ldp<CG>(d + (size_t)k * plane) - fbar);
                h = g.dzc[k];  // the seam at k = nz-1
            }
            const double S = warp_inclusive_scan(a, lane) + Sc;
            num = fmaT(h, S, num);
            den += h;
            Sc = __shfl_sync(0xffffffffu, S, 31);
        }
        Fc = -warp_sum(num) / warp_sum(den);
    }
    for (int k0 = 0; k0 < nz; k0 += 32) {
        const int k = k0 + lane;
        double a = 0.0, h = 0.0;
        if (k < nz) {
            a = mulT(g.dzf[k], (double)ldp<CG>(d + (size_t)k * plane) - fbar);
            h = g.dzc[k];  // 0 at the top wall
        }
        const double F = warp_inclusive_scan(a, lane) + Fc;  // F_(k+1/2)
        const double inc = mulT(h, F);                        // p_(k+1) - p_k
        const double sc = warp_inclusive_scan(inc, lane);
        const double pk = pc + (sc - inc);                    // exclusive: p_k
        if (k < nz) {
            d[(size_t)k * plane] = (T)pk;
            ps = fmaT(g.dzf[k], pk, ps);
        }
        Fc = __shfl_sync(0xffffffffu, F, 31);
        pc += __shfl_sync(0xffffffffu, sc, 31);
    }
    const double pbar = mulT(warp_sum(ps), g.inv_lz);
    for (int k = lane; k < nz; k += 32)
        d[(size_t)k * plane] = (T)((double)ldp<CG>(d + (size_t)k * plane) - pbar);
}

// Register-prefetch variant for the persistent batch kernel (no shared-memory
// ring): THOMAS_U planes of loads (L2-only when CG) are issued ahead of each
// block of the recurrence.
template <typename T, bool CG>
__device__ __forceinline__ void thomas_line_reg(int nz, size_t plane, T *d, size_t ts, size_t tb,
                                                const T *__restrict__ mtab,
                                                const T *__restrict__ ibtab,
                                                const T *__restrict__ cup) {
    constexpr int U = THOMAS_U;
    T prev = ldp<CG>(d);
    int k = 1;
    for (; k + U <= nz; k += U) {
        T fv[U], mv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            mv[q] = mtab[(size_t)(k + q) * ts + tb];
            fv[q] = ldp<CG>(d + (size_t)(k + q) * plane);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            prev = fmaT(-mv[q], prev, fv[q]);
            d[(size_t)(k + q) * plane] = prev;
        }
    }
    for (; k < nz; ++k) {
        prev = fmaT(-mtab[(size_t)k * ts + tb], prev, ldp<CG>(d + (size_t)k * plane));
        d[(size_t)k * plane] = prev;
    }
    prev = mulT(prev, ibtab[(size_t)(nz - 1) * ts + tb]);
    d[(size_t)(nz - 1) * plane] = prev;
    k = nz - 2;
    for (; k - U + 1 >= 0; k -= U) {
        T dv[U], iv[U], cv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            iv[q] = ibtab[(size_t)(k - q) * ts + tb];
            cv[q] = cup[k - q];
            dv[q] = ldp<CG>(d + (size_t)(k - q) * plane);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            prev = mulT(fmaT(-cv[q], prev, dv[q]), iv[q]);
            d[(size_t)(k - q) * plane] = prev;
        }
    }
    for (; k >= 0; --k) {
        prev = mulT(fmaT(-cup[k], prev, ldp<CG>(d + (size_t)k * plane)), ibtab[(size_t)k * ts + tb]);
        d[(size_t)k * plane] = prev;
    }
}

// Periodic-z form of thomas_line_reg (the cyclic solve of
// thomas_line_ring_cyc with register prefetch), for the persistent batch kernel.
template <typename T, bool CG>
__device__ __forceinline__ void thomas_line_reg_cyc(int nz, size_t plane, T *d, size_t ts, size_t tb,
                                                    const T *__restrict__ mtab,
                                                    const T *__restrict__ ibtab,
                                                    const T *__restrict__ cup,
                                                    const T *__restrict__ wtab,
                                                    const T *__restrict__ qtab) {
    constexpr int U = THOMAS_U;
    T prev = ldp<CG>(d);
    T acc = mulT(wtab[tb], prev);
    int k = 1;
    for (; k + U <= nz; k += U) {
        T fv[U], mv[U], wv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            mv[q] = mtab[(size_t)(k + q) * ts + tb];
            wv[q] = wtab[(size_t)(k + q) * ts + tb];
            fv[q] = ldp<CG>(d + (size_t)(k + q) * plane);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            prev = fmaT(-mv[q], prev, fv[q]);
            acc = fmaT(wv[q], prev, acc);
            d[(size_t)(k + q) * plane] = prev;
        }
    }
    for (; k < nz; ++k) {
        prev = fmaT(-mtab[(size_t)k * ts + tb], prev, ldp<CG>(d + (size_t)k * plane));
        acc = fmaT(wtab[(size_t)k * ts + tb], prev, acc);
        d[(size_t)k * plane] = prev;
    }
    const T sv = acc;
    prev = mulT(prev, ibtab[(size_t)(nz - 1) * ts + tb]);
    d[(size_t)(nz - 1) * plane] = fmaT(-sv, qtab[(size_t)(nz - 1) * ts + tb], prev);
    k = nz - 2;
    for (; k - U + 1 >= 0; k -= U) {
        T dv[U], iv[U], cv[U], qv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            iv[q] = ibtab[(size_t)(k - q) * ts + tb];
            qv[q] = qtab[(size_t)(k - q) * ts + tb];
            cv[q] = cup[k - q];
            dv[q] = ldp<CG>(d + (size_t)(k - q) * plane);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            prev = mulT(fmaT(-cv[q], prev, dv[q]), iv[q]);
            d[(size_t)(k - q) * plane] = fmaT(-sv, qv[q], prev);
        }
    }
    for (; k >= 0; --k) {
        prev = mulT(fmaT(-cup[k], prev, ldp<CG>(d + (size_t)k * plane)), ibtab[(size_t)k * ts + tb]);
        d[(size_t)k * plane] = fmaT(-sv, qtab[(size_t)k * ts + tb], prev);
    }
}

// Lines are numbered line = i + nx*j (one thread each); one virtual block
// covers lines line_base .. line_base + blockDim - 1.  Warp 0 of the block
// holding line 0 first solves the singular (0,0) line.  Both half-complex
// slots i and nx-i of a periodic direction use the table of wavenumber
// min(i, nx-i).  ASYNC: shared-memory ring (THOMAS_S*2*blockDim values;
// walls in z only, periodic z has k_thomas_cyc); otherwise register prefetch,
// with the cyclic solve when g.perz (tables wtab, qtab).
template <typename T, bool ASYNC, bool CG>
__device__ __forceinline__ void thomas_body(const GridDev &g, int Ux, int Uy, const T *mtab,
                                            const T *ibtab, const T *cup, T *data, const int *conv,
                                            int line_base, T *ring, const T *wtab = nullptr,
                                            const T *qtab = nullptr) {
    if (conv && ldp<CG>(conv)) return;
    const size_t plane = (size_t)g.nx * g.ny;
    if (g.sing && line_base == 0 && threadIdx.x < 32) {
        singular_line_warp<T, CG>(g, data, plane);  // line (0,0)
        if (threadIdx.x == 0) return;
    }
    const int line = line_base + threadIdx.x;
    if (line >= g.nx * g.ny) return;
    const int j = line / g.nx, i = line - j * g.nx;
    const int ux = (g.bcx == BC_PERIODIC) ? min(i, g.nx - i) : i;
    const int uy = (g.bcy == BC_PERIODIC) ? min(j, g.ny - j) : j;
    const size_t tb = (size_t)uy * Ux + ux;
    const size_t ts = (size_t)Ux * Uy;
    T *d = data + line;
    if (ASYNC) thomas_line_ring<T>(g.nz, plane, d, ts, tb, mtab, ibtab, cup, ring);
    else if (g.perz) thomas_line_reg_cyc<T, CG>(g.nz, plane, d, ts, tb, mtab, ibtab, cup, wtab, qtab);
    else thomas_line_reg<T, CG>(g.nz, plane, d, ts, tb, mtab, ibtab, cup);
}

template <typename T>
__global__ void __launch_bounds__(THOMAS_BLOCK) k_thomas(GridDev g, int Ux, int Uy,
                                                         const T *__restrict__ mtab,
                                                         const T *__restrict__ ibtab,
                                                         const T *__restrict__ cup, T *data,
                                                         const int *conv, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (conv && *(volatile const int *)conv) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
        thomas_body<T, true, false>(g, Ux, Uy, mtab, ibtab, cup, data, conv, t * THOMAS_BLOCK,
                                    (T *)smem_raw);
}

template <typename T> constexpr size_t thomas_smem() {
    return (size_t)THOMAS_S * 2 * THOMAS_BLOCK * sizeof(T);
}
template <typename T> constexpr size_t thomas_cyc_smem() {
    return (size_t)THOMAS_S * 3 * THOMAS_BLOCK * sizeof(T);
}

// u = q' - (dt/rho0) G p on non-wall faces (q' = dt q); wall faces 0.
// 2 FP64 instructions per face.  Virtual block: 32 x 8 cells of plane z.
template <bool CG>
__device__ __forceinline__ void correct_body(const GridDev &g, const double *p, const double *qx,
                                             const double *qy, const double *qz, double *u, double *v,
                                             double *w, VB vb) {
    const int tid = block_tid();
    const int i = vb.x * FLUX_BX + (tid & (FLUX_BX - 1));
    const int j = vb.y * FLUX_BY + tid / FLUX_BX;
    const int k = vb.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c = cidx(g, i, j, k);
    const double pc = ldp<CG>(p + c);
    double r = 0.0;
    if (!(g.bcx == BC_NEUMANN && i == g.nx - 1)) {
        const size_t e = (i == g.nx - 1) ? c - i : c + 1;
        r = fmaT(-g.cgx, ldp<CG>(p + e) - pc, ldp<CG>(qx + c));
    }
    u[c] = r;
    r = 0.0;
    if (!(g.bcy == BC_NEUMANN && j == g.ny - 1)) {
        const size_t nn = (j == g.ny - 1) ? c - (size_t)j * g.nx : c + g.nx;
        r = fmaT(-g.cgy, ldp<CG>(p + nn) - pc, ldp<CG>(qy + c));
    }
    v[c] = r;
    r = 0.0;
    if (k < g.nz - 1 || g.perz) {
        const size_t pl = (size_t)g.nx * g.ny;
        const size_t t = (k < g.nz - 1) ? c + pl : c - (size_t)k * pl;  // periodic z: the seam
        r = fmaT(-g.cgz[k], ldp<CG>(p + t) - pc, ldp<CG>(qz + c));
    }
    w[c] = r;
}

__global__ void __launch_bounds__(256) k_correct(GridDev g, const double *__restrict__ p,
                                                 const double *__restrict__ qx,
                                                 const double *__restrict__ qy,
                                                 const double *__restrict__ qz,
                                                 double *__restrict__ u, double *__restrict__ v,
                                                 double *__restrict__ w) {
    correct_body<false>(g, p, qx, qy, qz, u, v, w, vb_of_grid());
}

// Mixed-mode residual r = f - L_h p in FP64, stored as sigma 2^-e r in FP32
// (the right-hand side of the next FP32 solve, e the exponent of max|f|),
// with max|r| reduced and the last tile deciding convergence (relres and the
// divergence rule, refine_done).  CORR fuses the correction
// u = q' - (dt/rho0) G p, which forms the same face differences; a residual
// pass that converges has then also written the final u.  Every face
// difference is formed once: dE, dN, dT from the loads, dW from the lane to
// the left, dS from the row below through shared memory (double-buffered per
// plane), dB carried from the plane below.  Wall faces carry zero flux.
// Virtual block: 32 x 8 cells marching kc planes; sdn: 2 x 8 x 32 doubles.
constexpr int RESID_KC = 32;  // planes marched by one residual tile

struct RArgs {
    const double *p, *f, *qx, *qy, *qz;
    double *u, *v, *w;
    float *r32;
    DevStats *st;
    int slot;
    double tol;
};

// The residual marches in double-float.  The first residual's p is the FP32
// solution, every value exactly a float; later p (the solution plus
// corrections, FP64) is held as the exact sum of three floats (f64_split3).
// Either way each face difference p_b - p_a is formed from exact float
// differences (two-sum), so it carries no cancellation error; the rest of
// r = f - L_h p (the second differences, the metric factors, f split from
// FP64) runs in double-float arithmetic on the FP32 pipe, relative error
// about 2^-44 per operation: |r - r_exact| stays near 1e-13 max|f|, far below
// the 1e-10 the refinement aims at.  CORR also writes the correction
// u = q' - (dt/rho0) G p from the same face values, with the FP64 difference
// of the FP64 p and one FP64 multiply-add per face (as the FP64 correction
// forms it; the p values are loaded once for both).  Same tile, order of faces and
// neighbour exchange as before; sdn holds the float pairs of dN.
template <bool CORR> struct PVal {
    float h;
    __device__ __forceinline__ static PVal load(double x) { return PVal{f64_to_f32_shift(x, 0)}; }  // exact
    __device__ __forceinline__ static PVal zero() { return PVal{0.f}; }
    __device__ __forceinline__ float2 minus(const PVal &a) const { return two_sum(h, -a.h); }
};
template <> struct PVal<true> {
    F3 v;
    __device__ __forceinline__ static PVal load(double x) { return PVal{f64_split3(x)}; }
    __device__ __forceinline__ static PVal zero() { return PVal{F3{0.f, 0.f, 0.f}}; }
    __device__ __forceinline__ float2 minus(const PVal &a) const {
        const float2 d = df_add(two_sum(v.h, -a.v.h), two_sum(v.m, -a.v.m));
        return df_add(d, make_float2(__fsub_rn(v.l, a.v.l), 0.f));
    }
};
__device__ __forceinline__ double df_to_f64(float2 d) {
    return f32_to_f64_shift(d.x, 0) + f32_to_f64_shift(d.y, 0);
}

template <bool CG, bool CORR>
__device__ __forceinline__ unsigned long long resid_df_march(
    const GridDev &g, const RArgs &a, int k0, int k1, size_t c, bool on, int i, int j, int tx, int ty,
    bool hasE, bool hasW, bool hasN, bool hasS, long long oE, long long oW, long long oN, long long oS,
    int ef, float scale32, double *sdn) {
    typedef PVal<CORR> PV;
    const size_t pl = (size_t)g.nx * g.ny;
    float2 *sd = (float2 *)sdn;
    auto pv = [&](size_t at) { return PV::load(ldp<CG>(a.p + at)); };
    const float2 cx = f64_split(-g.idx2), cy = f64_split(-g.idy2);
    // the tile's per-plane factors -c_k and a_k as float pairs, split once
    __shared__ float2 s_cz[2][RESID_KC];
    {
        const int t = threadIdx.x + threadIdx.y * blockDim.x;
        if (t < k1 - k0) {
            s_cz[0][t] = f64_split(-g.lzc[k0 + t]);
            s_cz[1][t] = f64_split(g.lza[k0 + t]);
        }
    }
    // pcr: the raw FP64 p of the current cell (the correction's differences)
    double pcr = on ? ldp<CG>(a.p + c) : 0.0;
    PV pc = PV::load(pcr);
    float2 db = make_float2(0.f, 0.f);
    if (on && k0 > 0) db = pc.minus(pv(c - pl));
    else if (on && g.perz) db = pc.minus(pv(c + (size_t)(g.nz - 1) * pl));  // seam
    // f and the east, north and top p of a plane (and the west / south p on
    // the tile's first column / row), loaded one plane ahead of the
    // arithmetic (raw FP64 values, split when used)
    struct Ahead {
        double f, pe, pn, pt, pw, ps;
    };
    auto load_ahead = [&](size_t cc, int kk) {
        Ahead r{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        r.f = ldp<CG>(a.f + cc);
        if (hasE) r.pe = ldp<CG>(a.p + cc + oE);
        if (hasN) r.pn = ldp<CG>(a.p + cc + oN);
        if (tx == 0 && hasW) r.pw = ldp<CG>(a.p + cc + oW);
        if (ty == 0 && hasS) r.ps = ldp<CG>(a.p + cc + oS);
        if (kk < g.nz - 1) r.pt = ldp<CG>(a.p + cc + pl);
        else if (g.perz) r.pt = ldp<CG>(a.p + cc - (size_t)kk * pl);  // seam to plane 0
        return r;
    };
    Ahead cur{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (on) cur = load_ahead(c, k0);
    unsigned mxf = 0u;  // max |r| as float bits (monotone in |r|)
    int buf = 0;
    for (int k = k0; k < k1; ++k) {
        Ahead nxt{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (on && k + 1 < k1) nxt = load_ahead(c + pl, k + 1);
        float2 de = make_float2(0.f, 0.f), dn = de, dt = de;
        PV pt = PV::zero();
        double qxc = 0.0, qyc = 0.0, qzc = 0.0;
        if (on) {
            if (CORR) {
                qxc = ldp<CG>(a.qx + c);
                qyc = ldp<CG>(a.qy + c);
                qzc = ldp<CG>(a.qz + c);
            }
            if (hasE) de = PV::load(cur.pe).minus(pc);
            if (hasN) dn = PV::load(cur.pn).minus(pc);
            if (k < g.nz - 1) {
                pt = PV::load(cur.pt);
                dt = pt.minus(pc);
            } else if (g.perz) {
                dt = PV::load(cur.pt).minus(pc);
            }
            sd[(buf * FLUX_BY + ty) * FLUX_BX + tx] = dn;
        }
        float2 dw = make_float2(__shfl_up_sync(0xffffffffu, de.x, 1), __shfl_up_sync(0xffffffffu, de.y, 1));
        __syncthreads();
        if (on) {
            // the correction's stores come after every load of this plane
            // and the next (they could alias the q' loads)
            if (CORR) {
                // FP64 differences of the FP64 p, as the FP64 correction forms them
                a.u[c] = (g.bcx == BC_NEUMANN && i == g.nx - 1) ? 0.0 : fmaT(-g.cgx, __dsub_rn(cur.pe, pcr), qxc);
                a.v[c] = (g.bcy == BC_NEUMANN && j == g.ny - 1) ? 0.0 : fmaT(-g.cgy, __dsub_rn(cur.pn, pcr), qyc);
                a.w[c] = (k < g.nz - 1 || g.perz) ? fmaT(-g.cgz[k], __dsub_rn(cur.pt, pcr), qzc) : 0.0;
            }
            if (tx == 0) dw = hasW ? pc.minus(PV::load(cur.pw)) : make_float2(0.f, 0.f);
            const float2 ds = (ty > 0) ? sd[(buf * FLUX_BY + ty - 1) * FLUX_BX + tx]
                                       : (hasS ? pc.minus(PV::load(cur.ps)) : make_float2(0.f, 0.f));
            float2 res = f64_split(cur.f);
            res = df_add(res, df_mul(df_add(de, df_neg(dw)), cx));
            res = df_add(res, df_mul(df_add(dn, df_neg(ds)), cy));
            res = df_add(res, df_mul(dt, s_cz[0][k - k0]));
            res = df_add(res, df_mul(db, s_cz[1][k - k0]));
            const float r = __fadd_rn(res.x, res.y);
            mxf = max(mxf, absbits(r));
            a.r32[c] = f32_shift(r, ef) * scale32;
        }
        db = dt;
        pc = pt;
        pcr = cur.pt;
        cur = nxt;
        c += pl;
        buf ^= 1;
    }
    return absbits(f32_to_f64_shift(__uint_as_float(mxf), 0));
}

template <bool CG, bool CORR>
__device__ __forceinline__ void resid_body(const GridDev &g, int kc, const RArgs &a, VB vb,
                                           int ntiles, double *sdn) {
    if (ldp<CG>(&a.st->converged)) return;
    const int tid = block_tid();
    const int tx = tid & (FLUX_BX - 1), ty = tid / FLUX_BX;
    const int i = vb.x * FLUX_BX + tx, j = vb.y * FLUX_BY + ty;
    const int k0 = vb.z * kc, k1 = min(g.nz, k0 + kc);
    const bool on = i < g.nx && j < g.ny;
    const int ef = exp_of_bits(ldp<CG>(&a.st->fmax_bits));
    const float scale32 = (float)g.sigma;
    const bool per_x = g.bcx == BC_PERIODIC, per_y = g.bcy == BC_PERIODIC;
    const bool hasE = i < g.nx - 1 || per_x, hasW = i > 0 || per_x;
    const bool hasN = j < g.ny - 1 || per_y, hasS = j > 0 || per_y;
    const long long oE = (i < g.nx - 1) ? 1 : -(long long)i;
    const long long oW = (i > 0) ? -1 : (long long)(g.nx - 1);
    const long long oN = (j < g.ny - 1) ? (long long)g.nx : -(long long)j * g.nx;
    const long long oS = (j > 0) ? -(long long)g.nx : (long long)(g.ny - 1) * g.nx;
    const size_t c = on ? cidx(g, i, j, k0) : 0;
    const unsigned long long mx = resid_df_march<CG, CORR>(g, a, k0, k1, c, on, i, j, tx, ty, hasE, hasW, hasN,
                                                           hasS, oE, oW, oN, oS, ef, scale32, sdn);
    block_max_atomic(mx, &a.st->rmax_bits[a.slot]);
    __shared__ int last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(&a.st->done_blocks[a.slot], 1u);
        last = (ticket == (unsigned)ntiles - 1);
    }
    __syncthreads();
    if (last && tid == 0) {
        __threadfence();
        const unsigned long long rb = atomicMax(&a.st->rmax_bits[a.slot], 0ull);
        const unsigned long long fb = atomicMax(&a.st->fmax_bits, 0ull);
        double rel;
        const double prev = a.slot > 0
                                ? __longlong_as_double((long long)atomicMax(&a.st->rmax_bits[a.slot - 1], 0ull))
                                : -1.0;
        const bool done = refine_done<CG>(g, __longlong_as_double((long long)rb),
                                          __longlong_as_double((long long)fb), a.tol, prev, &rel);
        a.st->relres = rel;
        a.st->n_resid = a.slot + 1;
        a.st->iterations = a.slot;
        __threadfence();  // the stats are visible before the flag
        if (done) a.st->converged = 1;
    }
}

// One block per tile; tiles of kc planes.  The fused residual-correction
// (CORR) is held to four CTAs per SM (64 registers): its march's loads run
// one plane ahead, which costs registers.
template <bool CORR>
__device__ __forceinline__ void resid_tiles(const GridDev &g, int kc, const RArgs &a, int tgx, int tgy,
                                            int ntiles, double *sdn) {
    if (*(volatile const int *)&a.st->converged) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int txy = tgx * tgy, z = t / txy, r = t - z * txy, y = r / tgx;
        resid_body<false, CORR>(g, kc, a, VB{r - y * tgx, y, z}, ntiles, sdn);
        __syncthreads();
    }
}
template <bool CORR>
__global__ void __launch_bounds__(256) k_resid(GridDev g, int kc, RArgs a, int tgx, int tgy,
                                               int ntiles) {
    __shared__ double sdn[2 * FLUX_BY * FLUX_BX];
    resid_tiles<CORR>(g, kc, a, tgx, tgy, ntiles, sdn);
}
template <bool CORR>
__global__ void __launch_bounds__(256, 4) k_resid_corr(GridDev g, int kc, RArgs a, int tgx, int tgy,
                                                       int ntiles) {
    __shared__ double sdn[2 * FLUX_BY * FLUX_BX];
    resid_tiles<CORR>(g, kc, a, tgx, tgy, ntiles, sdn);
}

// The correction when no fused residual pass has run (the solve converged
// at the first residual, or no refinement sweep is allowed): runs only when
// n_resid == 1; otherwise the fused pass has written u.  Tiles: 32 x 8 cells
// of one plane.
__global__ void __launch_bounds__(256) k_correct_if(GridDev g, const double *__restrict__ p,
                                                    const double *__restrict__ qx,
                                                    const double *__restrict__ qy,
                                                    const double *__restrict__ qz,
                                                    double *__restrict__ u, double *__restrict__ v,
                                                    double *__restrict__ w, const DevStats *st,
                                                    int tgx, int tgy, int ntiles) {
    if (*(volatile const int *)&st->n_resid != 1) return;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int txy = tgx * tgy, z = t / txy, r = t - z * txy, y = r / tgx;
        correct_body<false>(g, p, qx, qy, qz, u, v, w, VB{r - y * tgx, y, z});
    }
}

// Periodic z: the cyclic z-solves (thomas_line_ring_cyc), lines as in
// k_thomas; the singular (0,0) line takes its periodic branch.
template <typename T>
__global__ void __launch_bounds__(THOMAS_BLOCK) k_thomas_cyc(GridDev g, int Ux, int Uy,
                                                             const T *__restrict__ mtab,
                                                             const T *__restrict__ ibtab,
                                                             const T *__restrict__ cup,
                                                             const T *__restrict__ wtab,
                                                             const T *__restrict__ qtab, T *data,
                                                             const int *conv, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (conv && *(volatile const int *)conv) return;
    const size_t plane = (size_t)g.nx * g.ny;
    const size_t ts = (size_t)Ux * Uy;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int line_base = t * THOMAS_BLOCK;
        if (g.sing && line_base == 0 && threadIdx.x < 32) {
            singular_line_warp<T, false>(g, data, plane);  // line (0,0)
            if (threadIdx.x == 0) continue;
        }
        const int line = line_base + threadIdx.x;
        if (line >= g.nx * g.ny) continue;
        const int j = line / g.nx, i = line - j * g.nx;
        const int ux = (g.bcx == BC_PERIODIC) ? min(i, g.nx - i) : i;
        const int uy = (g.bcy == BC_PERIODIC) ? min(j, g.ny - j) : j;
        thomas_line_ring_cyc<T>(g.nz, plane, data + line, ts, (size_t)uy * Ux + ux, mtab, ibtab, cup,
                                wtab, qtab, (T *)smem_raw);
    }
}

// max |D u| (diagnostics).
__global__ void __launch_bounds__(256) k_divmax(GridDev g, const double *__restrict__ u,
                                                const double *__restrict__ v,
                                                const double *__restrict__ w, DevStats *st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    unsigned long long mx = 0ull;
    if (i < g.nx) {
        const size_t c = cidx(g, i, j, k);
        const double ue = (g.bcx == BC_NEUMANN && i == g.nx - 1) ? 0.0 : u[c];
        const double uw = (i > 0) ? u[c - 1] : (g.bcx == BC_PERIODIC ? u[c + g.nx - 1] : 0.0);
        const double vn = (g.bcy == BC_NEUMANN && j == g.ny - 1) ? 0.0 : v[c];
        const double vs = (j > 0) ? v[c - g.nx] : (g.bcy == BC_PERIODIC ? v[c + (size_t)(g.ny - 1) * g.nx] : 0.0);
        const double wt = (k == g.nz - 1 && !g.perz) ? 0.0 : w[c];
        const double wb = (k > 0) ? w[c - (size_t)g.nx * g.ny]
                                  : (g.perz ? w[c + (size_t)(g.nz - 1) * g.nx * g.ny] : 0.0);
        const double d = fmaT(ue - uw, g.idx1, fmaT(vn - vs, g.idy1, (wt - wb) * g.izf[k]));
        mx = absbits(d);
    }
    block_max_atomic(mx, &st->divmax_bits);
}

// z-factorisation tables of a plan, one thread per distinct eigenvalue pair
// (ux, uy): beta_0 = b_0 + lambda, m_k = a_k / beta_(k-1),
// beta_k = (b_k + lambda) - m_k c_(k-1), stored as m_k and 1/beta_k (FP64, and
// rounded to FP32 when t32 is given).  Every operation is an explicit IEEE
// round-to-nearest operation in the order of that recurrence.  The singular
// pair (0,0) gets zeros when sing != 0 (no Dirichlet face in x or y).
__global__ void k_ztables(int Ux, int Uy, int nz, const double *__restrict__ lamx,
                          const double *__restrict__ lamy, const double *__restrict__ A,
                          const double *__restrict__ C, double *mt, double *ib, float *mt32,
                          float *ib32, int sing) {
    const size_t ts = (size_t)Ux * Uy;
    for (size_t uu = (size_t)blockIdx.x * blockDim.x + threadIdx.x; uu < ts;
         uu += (size_t)gridDim.x * blockDim.x) {
        const int ux = (int)(uu % Ux), uy = (int)(uu / Ux);
        if (sing && ux == 0 && uy == 0) {
            for (int k = 0; k < nz; ++k) {
                mt[(size_t)k * ts + uu] = 0.0;
                ib[(size_t)k * ts + uu] = 0.0;
                if (mt32) {
                    mt32[(size_t)k * ts + uu] = 0.f;
                    ib32[(size_t)k * ts + uu] = 0.f;
                }
            }
            continue;
        }
        const double lam = __dadd_rn(lamx[ux], lamy[uy]);
        double beta = __dadd_rn(-__dadd_rn(A[0], C[0]), lam);
        double r = __ddiv_rn(1.0, beta);
        mt[uu] = 0.0;
        ib[uu] = r;
        if (mt32) {
            mt32[uu] = 0.f;
            ib32[uu] = __double2float_rn(r);
        }
        for (int k = 1; k < nz; ++k) {
            const double m = __ddiv_rn(A[k], beta);
            beta = __dsub_rn(__dadd_rn(-__dadd_rn(A[k], C[k]), lam), __dmul_rn(m, C[k - 1]));
            r = __ddiv_rn(1.0, beta);
            mt[(size_t)k * ts + uu] = m;
            ib[(size_t)k * ts + uu] = r;
            if (mt32) {
                mt32[(size_t)k * ts + uu] = __double2float_rn(m);
                ib32[(size_t)k * ts + uu] = __double2float_rn(r);
            }
        }
    }
}

// Periodic-z tables (Sherman-Morrison form of the cyclic z-solve, see
// thomas_line_ring_cyc), one thread per eigenvalue pair.  With b_k the
// diagonal -(a_k + c_k) + lambda, gamma = -b_0, alpha = a_0 (row 0's seam
// coupling) and beta_c = c_(nz-1) (row nz-1's): B has diagonal b_0 - gamma,
// b_1, ..., b_(nz-2), b_(nz-1) - alpha beta_c / gamma; m_k and 1/beta_k factor
// B as in k_ztables; w_k = (1/beta_k) prod_(j<k) (-c_j / beta_j), plus
// (alpha/gamma)/beta_(nz-1) at k = nz-1; q = B^(-1) (gamma, 0, ..., 0, beta_c),
// divided by 1 + q_0 + (alpha/gamma) q_(nz-1).  Explicit round-to-nearest
// operations; FP32 copies rounded from the FP64 values.  The singular pair
// (0,0) (sing != 0) gets zeros.
__global__ void k_ztables_cyc(int Ux, int Uy, int nz, const double *__restrict__ lamx,
                              const double *__restrict__ lamy, const double *__restrict__ A,
                              const double *__restrict__ C, double *mt, double *ib, double *wt,
                              double *qt, float *mt32, float *ib32, float *wt32, float *qt32,
                              int sing) {
    const size_t ts = (size_t)Ux * Uy;
    for (size_t uu = (size_t)blockIdx.x * blockDim.x + threadIdx.x; uu < ts;
         uu += (size_t)gridDim.x * blockDim.x) {
        const int ux = (int)(uu % Ux), uy = (int)(uu / Ux);
        auto at = [&](int k) { return (size_t)k * ts + uu; };
        if (sing && ux == 0 && uy == 0) {
            for (int k = 0; k < nz; ++k) {
                mt[at(k)] = ib[at(k)] = wt[at(k)] = qt[at(k)] = 0.0;
                if (mt32) mt32[at(k)] = ib32[at(k)] = wt32[at(k)] = qt32[at(k)] = 0.f;
            }
            continue;
        }
        const double lam = __dadd_rn(lamx[ux], lamy[uy]);
        const double b0 = __dadd_rn(-__dadd_rn(A[0], C[0]), lam);
        const double gam = -b0;
        const double ag = __ddiv_rn(A[0], gam);                 // alpha / gamma
        const double corner = __dmul_rn(ag, C[nz - 1]);          // alpha beta_c / gamma
        // factorisation of B
        double beta = __dsub_rn(b0, gam);
        mt[at(0)] = 0.0;
        ib[at(0)] = __ddiv_rn(1.0, beta);
        for (int k = 1; k < nz; ++k) {
            const double m = __ddiv_rn(A[k], beta);
            double bk = __dadd_rn(-__dadd_rn(A[k], C[k]), lam);
            if (k == nz - 1) bk = __dsub_rn(bk, corner);
            beta = __dsub_rn(bk, __dmul_rn(m, C[k - 1]));
            mt[at(k)] = m;
            ib[at(k)] = __ddiv_rn(1.0, beta);
        }
        // weights of y_0 in the forward-eliminated right-hand side
        double P = 1.0;
        for (int k = 0; k < nz; ++k) {
            if (k > 0) P = __dmul_rn(P, __dmul_rn(-C[k - 1], ib[at(k - 1)]));
            wt[at(k)] = __dmul_rn(ib[at(k)], P);
        }
        wt[at(nz - 1)] = __dadd_rn(wt[at(nz - 1)], __dmul_rn(ag, ib[at(nz - 1)]));
        // q = B^(-1) u: forward elimination into qt, then back substitution in place
        double g = gam;
        qt[at(0)] = g;
        for (int k = 1; k < nz; ++k) {
            const double uk = (k == nz - 1) ? C[nz - 1] : 0.0;
            g = __dsub_rn(uk, __dmul_rn(mt[at(k)], g));
            qt[at(k)] = g;
        }
        double y = __dmul_rn(qt[at(nz - 1)], ib[at(nz - 1)]);
        qt[at(nz - 1)] = y;
        for (int k = nz - 2; k >= 0; --k) {
            y = __dmul_rn(__dsub_rn(qt[at(k)], __dmul_rn(C[k], y)), ib[at(k)]);
            qt[at(k)] = y;
        }
        const double iden = __ddiv_rn(1.0, __dadd_rn(1.0, __dadd_rn(qt[at(0)], __dmul_rn(ag, qt[at(nz - 1)]))));
        for (int k = 0; k < nz; ++k) {
            qt[at(k)] = __dmul_rn(qt[at(k)], iden);
            if (mt32) {
                mt32[at(k)] = __double2float_rn(mt[at(k)]);
                ib32[at(k)] = __double2float_rn(ib[at(k)]);
                wt32[at(k)] = __double2float_rn(wt[at(k)]);
                qt32[at(k)] = __double2float_rn(qt[at(k)]);
            }
        }
    }
}

}  // namespace fz
