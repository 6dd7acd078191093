// ACDI phase-field transport (sm_103a): the step that produces phi ahead of
// the projection.  The accurate conservative diffuse-interface model of Jain
// (2022), which the paper uses for the phase field:
//   d phi/dt + div(u phi) = div{ Gamma [ eps grad phi
//                                        - 1/4 (1 - tanh^2(psi/(2 eps))) n ] },
//   psi = eps ln((phi + delta)/(1 - phi + delta)),   n = grad psi / |grad psi|,
// in conservative face-flux form on the staggered grid (FP64):
//   k_acdi_psi    : r = max(phi + delta, delta)/max(1 - phi + delta, delta),
//                   psi = eps ln r and q = sqrt(r) at the centres (one log
//                   per cell; the bounds keep r > 0 for any phi, so a phi
//                   slightly outside [0, 1] saturates psi near +-230 eps
//                   instead of giving NaN; inside [0, 1] r is unchanged);
//   k_acdi_normal : n at the centres from central differences of psi (a wall
//                   mirrors psi; the centre distances are the sums of the two
//                   half spacings, so stretched and periodic z need nothing
//                   else); |grad psi| = 0 gives n = 0;
//   k_acdi_flux   : on the +x, +y, +z face of every cell
//                   F = u_f (phi_a + phi_b)/2 - Gamma [ eps (phi_b - phi_a)/h
//                       - 1/4 (1 - tanh^2((psi_a + psi_b)/(4 eps))) (n_a + n_b)/2 ],
//                   0 on walls;
//   k_acdi_update : rhs = -D F, phi_out = phi + dt rhs.
// The face coefficient 1 - tanh^2(x), x = (psi_a + psi_b)/(4 eps), is formed
// without the tanh: psi/eps = ln r gives e^(2x) = sqrt(r_a r_b) = q_a q_b = S,
// so tanh x = (S - 1)/(S + 1) and 1 - tanh^2 x = 4 S/(1 + S)^2 exactly (one
// multiply and one division per face instead of an FP64 tanh, and no
// cancellation where tanh x is near +-1; S stays within [1e-100, 1e100]).
// Mass is conserved to round-off: every face flux enters two cells with
// opposite signs (walls carry none).
#pragma once
#include "kern_passes.cuh"

namespace fz {

constexpr double ACDI_DELTA = 1e-100;  // keeps the logarithm finite at phi = 0 and 1

__device__ __forceinline__ void acdi_ijk(const GridDev &g, size_t c, int &i, int &j, int &k) {
    const size_t pl = (size_t)g.nx * g.ny;
    k = (int)(c / pl);
    const size_t rem = c - (size_t)k * pl;
    j = (int)(rem / g.nx);
    i = (int)(rem - (size_t)j * g.nx);
}

__global__ void __launch_bounds__(256) k_acdi_psi(GridDev g, double eps, const double *__restrict__ phi,
                                                  double *__restrict__ psi, double *__restrict__ rr) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const double f = phi[c];
        // both sides bounded below by delta: a phi that advection has pushed
        // slightly outside [0, 1] still gives a finite psi (saturated at
        // about +-230 eps) instead of the logarithm of a negative number
        const double r = fmax(f + ACDI_DELTA, ACDI_DELTA) / fmax(1.0 - f + ACDI_DELTA, ACDI_DELTA);
        rr[c] = sqrt(r);
        psi[c] = eps * log(r);
    }
}

__global__ void __launch_bounds__(256) k_acdi_normal(GridDev g, const double *__restrict__ psi,
                                                     double *__restrict__ nxo, double *__restrict__ nyo,
                                                     double *__restrict__ nzo) {
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    const double hx = 0.5 * g.idx1, hy = 0.5 * g.idy1;  // 1/(2 dx), 1/(2 dy)
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        acdi_ijk(g, c, i, j, k);
        const double pc = psi[c];
        // x, y: wrap (periodic) or mirror (wall)
        const double pe = i < g.nx - 1 ? psi[c + 1] : (g.bcx == BC_PERIODIC ? psi[c - i] : pc);
        const double pw = i > 0 ? psi[c - 1] : (g.bcx == BC_PERIODIC ? psi[c + g.nx - 1] : pc);
        const double pn = j < g.ny - 1 ? psi[c + g.nx] : (g.bcy == BC_PERIODIC ? psi[c - (size_t)j * g.nx] : pc);
        const double ps = j > 0 ? psi[c - g.nx] : (g.bcy == BC_PERIODIC ? psi[c + (size_t)(g.ny - 1) * g.nx] : pc);
        // z: neighbour values and the centre distances to them (a wall's
        // mirrored ghost centre lies dzf_k away)
        double pt, pb, up, dn;
        if (k < g.nz - 1) {
            pt = psi[c + pl];
            up = g.dzc[k];
        } else if (g.perz) {
            pt = psi[c - (size_t)k * pl];
            up = g.dzc[k];  // the seam
        } else {
            pt = pc;
            up = g.dzf[k];
        }
        if (k > 0) {
            pb = psi[c - pl];
            dn = g.dzc[k - 1];
        } else if (g.perz) {
            pb = psi[c + (size_t)(g.nz - 1) * pl];
            dn = g.dzc[g.nz - 1];
        } else {
            pb = pc;
            dn = g.dzf[0];
        }
        const double gx = (pe - pw) * hx, gy = (pn - ps) * hy, gz = (pt - pb) / (up + dn);
        const double m2 = fmaT(gx, gx, fmaT(gy, gy, mulT(gz, gz)));
        const double inv = m2 > 0.0 ? rsqrt(m2) : 0.0;
        nxo[c] = gx * inv;
        nyo[c] = gy * inv;
        nzo[c] = gz * inv;
    }
}

// One face: advective plus diffusive-sharpening flux between cells a and b;
// 1/4 (1 - tanh^2) = S/(1 + S)^2 with S = q_a q_b.
__device__ __forceinline__ double acdi_face(double ua, double fa, double fb, double qa, double qb, double na,
                                            double nb, double ih, double eps, double gam) {
    const double S = qa * qb, S1 = 1.0 + S;
    const double sharp = S / (S1 * S1) * (0.5 * (na + nb));
    return fmaT(ua, 0.5 * (fa + fb), -gam * (eps * (fb - fa) * ih - sharp));
}

__global__ void __launch_bounds__(256) k_acdi_flux(GridDev g, double eps, double gam,
                                                   const double *__restrict__ phi,
                                                   const double *__restrict__ rr,
                                                   const double *__restrict__ nxv,
                                                   const double *__restrict__ nyv,
                                                   const double *__restrict__ nzv,
                                                   const double *__restrict__ u,
                                                   const double *__restrict__ v,
                                                   const double *__restrict__ w, double *__restrict__ fx,
                                                   double *__restrict__ fy, double *__restrict__ fz) {
    const size_t n = (size_t)g.nx * g.ny * g.nz, pl = (size_t)g.nx * g.ny;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        acdi_ijk(g, c, i, j, k);
        const double fc = phi[c], sc = rr[c];
        double q = 0.0;
        if (i < g.nx - 1 || g.bcx == BC_PERIODIC) {
            const size_t b = i < g.nx - 1 ? c + 1 : c - i;
            q = acdi_face(u[c], fc, phi[b], sc, rr[b], nxv[c], nxv[b], g.idx1, eps, gam);
        }
        fx[c] = q;
        q = 0.0;
        if (j < g.ny - 1 || g.bcy == BC_PERIODIC) {
            const size_t b = j < g.ny - 1 ? c + g.nx : c - (size_t)j * g.nx;
            q = acdi_face(v[c], fc, phi[b], sc, rr[b], nyv[c], nyv[b], g.idy1, eps, gam);
        }
        fy[c] = q;
        q = 0.0;
        if (k < g.nz - 1 || g.perz) {
            const size_t b = k < g.nz - 1 ? c + pl : c - (size_t)k * pl;
            q = acdi_face(w[c], fc, phi[b], sc, rr[b], nzv[c], nzv[b], 1.0 / g.dzc[k], eps, gam);
        }
        fz[c] = q;
    }
}

// rhs = -D F (wall faces read as 0), phi_out = phi + dt rhs; either output
// may be null.
// (phi and phi_out may be the same array: each element is read, then written,
// by one thread, and nothing else in the kernel reads phi.)
__global__ void __launch_bounds__(256) k_acdi_update(GridDev g, double dt, const double *phi,
                                                     const double *__restrict__ fx,
                                                     const double *__restrict__ fy,
                                                     const double *__restrict__ fz,
                                                     double *__restrict__ rhs_out, double *phi_out) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        acdi_ijk(g, c, i, j, k);
        const double r = -div_q<false>(g, i, j, k, g.idx1, g.idy1, g.izf[k], fx, fy, fz);
        if (rhs_out) rhs_out[c] = r;
        if (phi_out) phi_out[c] = fmaT(dt, r, phi[c]);
    }
}

}  // namespace fz
