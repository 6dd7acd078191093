/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the variable-density
 * pressure-correction projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this file.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (paper, "Methods and Implementation strategy": second-order
 * finite differences on a staggered Cartesian grid; pressure correction whose
 * variable-coefficient Poisson equation is turned into a constant-coefficient
 * one by the Dong & Shen (2012) / Dodd & Ferrante (2014) splitting of
 * Frantzis & Grigoriadis (2019); fast direct FFT solver of CaNS, Costa 2018;
 * "Mathematical model": properties mapped linearly over the phase field):
 *
 *   rho   = rho_g + phi (rho_l - rho_g)                 cell centres
 *   rho_f = mean of the two adjacent centre values      faces, beta_f = 1/rho_f
 *   rho0  = min(rho_l, rho_g)
 *   phat  = 2 p^n - p^(n-1)
 *   f     = (rho0/dt) D(u*) + D[(1 - rho0 beta_f) G phat],  minus its dzf-weighted mean
 *   D G p = f,  p with zero dzf-weighted mean
 *   u     = u* - dt [G p / rho0 + (beta_f - 1/rho0) G phat]   on every non-wall face
 *
 * G: centre-to-face gradient, D: face-to-centre divergence; wall faces are 0.
 * A periodic z direction (the triperiodic domains of the paper's
 * "Numerical experiments", e.g. the emulsion in homogeneous isotropic
 * turbulence) couples plane nz-1 to plane 0 through the face nz-1/2, whose
 * centre distance is (dzf_0 + dzf_(nz-1))/2.
 *
 * The Poisson solve is deliberately a *different* algorithm from the GPU's:
 *   - full complex DFTs in x and y by a plain recursive mixed-radix
 *     Cooley-Tukey FFT (naive DFT at prime lengths);
 *   - a Neumann (wall) direction is handled by even extension to a periodic
 *     problem of twice the length, solved the same way and restricted back;
 *   - each (kx, ky) z-line is solved by Gaussian elimination with partial
 *     pivoting on the tridiagonal band (walls in z), or by dense Gaussian
 *     elimination of the assembled cyclic matrix (periodic z); the singular
 *     (0,0) line by dense Gaussian elimination with the gauge row
 *     sum_k dzf_k p_k = 0;
 *   - small grids also have a dense LU path on the assembled operator.
 *
 * Layout: double arrays [nz][ny][nx], x fastest.  u[k][j][i] is the x-face
 * i+1/2, v the y-face j+1/2, w the z-face k+1/2.  bc = 0 periodic, 1 Neumann
 * (walls), in x, y and z alike.  In a wall direction the last face is the far
 * wall and the near wall face is implicit; both are treated as 0.
 *
 * The Poisson solve alone (ora_apply_L, ora_poisson_fft, ora_poisson_dense)
 * also takes the boundary kinds of the CaNS fast solver in x and y:
 * bc = 2 Dirichlet (p = 0 on both boundary faces), 3 Neumann at the near end
 * and Dirichlet at the far end, 4 Dirichlet near and Neumann far.  The ghost
 * value beyond a Neumann face mirrors the cell (zero flux), beyond a
 * Dirichlet face it mirrors it with the opposite sign (zero face value).
 * The FFT path extends such a direction to a periodic problem by reflection:
 * odd about both faces (length 2n), or even about the Neumann face and odd
 * about the Dirichlet face (the quarter-wave extension, length 4n).  With a
 * Dirichlet face in x or y the problem is not singular: no gauge, p unique.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int nx, ny, nz;
    double dx, dy;
    const double *zf; /* nz+1 face coordinates */
    int bcx, bcy, bcz;
} grid_t;

#define IDX(g, i, j, k) (((size_t)(k) * (g)->ny + (size_t)(j)) * (g)->nx + (size_t)(i))

static grid_t mkgrid(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx,
                     int bcy, int bcz) {
    grid_t g = {nx, ny, nz, dx, dy, zf, bcx, bcy, bcz};
    return g;
}

static double dzf(const grid_t *g, int k) { return g->zf[k + 1] - g->zf[k]; }
static double zc(const grid_t *g, int k) { return 0.5 * (g->zf[k] + g->zf[k + 1]); }
/* distance between centres k and k+1 (the spacing at z-face k+1/2); for
 * k = nz-1 in a periodic z direction, the distance from centre nz-1 across the
 * periodic boundary to centre 0 */
static double dzc(const grid_t *g, int k) {
    if (k == g->nz - 1) return 0.5 * (dzf(g, 0) + dzf(g, g->nz - 1));
    return zc(g, k + 1) - zc(g, k);
}

/* ------------------------------------------------------------------ */
/* Staggered operators                                                  */
/* ------------------------------------------------------------------ */

/* G q on the three face families; wall faces are 0. */
static void grad(const grid_t *g, const double *q, double *gx, double *gy, double *gz) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(g, i, j, k);
                /* x-face i+1/2 */
                if (i < nx - 1)
                    gx[c] = (q[IDX(g, i + 1, j, k)] - q[c]) / g->dx;
                else
                    gx[c] = g->bcx == 0 ? (q[IDX(g, 0, j, k)] - q[c]) / g->dx : 0.0;
                /* y-face j+1/2 */
                if (j < ny - 1)
                    gy[c] = (q[IDX(g, i, j + 1, k)] - q[c]) / g->dy;
                else
                    gy[c] = g->bcy == 0 ? (q[IDX(g, i, 0, k)] - q[c]) / g->dy : 0.0;
                /* z-face k+1/2 */
                if (k < nz - 1)
                    gz[c] = (q[IDX(g, i, j, k + 1)] - q[c]) / dzc(g, k);
                else
                    gz[c] = g->bcz == 0 ? (q[IDX(g, i, j, 0)] - q[c]) / dzc(g, k) : 0.0;
            }
}

/* D of a face field; wall faces are read as 0 whatever is stored there. */
static void divergence(const grid_t *g, const double *u, const double *v, const double *w,
                       double *out) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(g, i, j, k);
                double ue = (g->bcx == 1 && i == nx - 1) ? 0.0 : u[c];
                double uw = (i > 0) ? u[IDX(g, i - 1, j, k)]
                                    : (g->bcx == 0 ? u[IDX(g, nx - 1, j, k)] : 0.0);
                double vn = (g->bcy == 1 && j == ny - 1) ? 0.0 : v[c];
                double vs = (j > 0) ? v[IDX(g, i, j - 1, k)]
                                    : (g->bcy == 0 ? v[IDX(g, i, ny - 1, k)] : 0.0);
                double wt = (g->bcz == 1 && k == nz - 1) ? 0.0 : w[c];
                double wb = (k > 0) ? w[IDX(g, i, j, k - 1)]
                                    : (g->bcz == 0 ? w[IDX(g, i, j, nz - 1)] : 0.0);
                out[c] = (ue - uw) / g->dx + (vn - vs) / g->dy + (wt - wb) / dzf(g, k);
            }
}

/* beta_f = 1/rho_f on the three face families (wall faces: value unused, set 0). */
static void face_beta(const grid_t *g, double rho_l, double rho_g, const double *phi, double *bx,
                      double *by, double *bz) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(g, i, j, k);
                double rc = rho_g + phi[c] * (rho_l - rho_g);
                int ie = (i < nx - 1) ? i + 1 : (g->bcx == 0 ? 0 : -1);
                int jn = (j < ny - 1) ? j + 1 : (g->bcy == 0 ? 0 : -1);
                if (ie >= 0) {
                    double re = rho_g + phi[IDX(g, ie, j, k)] * (rho_l - rho_g);
                    bx[c] = 1.0 / (0.5 * (rc + re));
                } else
                    bx[c] = 0.0;
                if (jn >= 0) {
                    double rn = rho_g + phi[IDX(g, i, jn, k)] * (rho_l - rho_g);
                    by[c] = 1.0 / (0.5 * (rc + rn));
                } else
                    by[c] = 0.0;
                int kt = (k < nz - 1) ? k + 1 : (g->bcz == 0 ? 0 : -1);
                if (kt >= 0) {
                    double rt = rho_g + phi[IDX(g, i, j, kt)] * (rho_l - rho_g);
                    bz[c] = 1.0 / (0.5 * (rc + rt));
                } else
                    bz[c] = 0.0;
            }
}

static double weighted_mean(const grid_t *g, const double *a) {
    double num = 0.0, den = 0.0;
    for (int k = 0; k < g->nz; ++k) {
        double s = 0.0;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) s += a[IDX(g, i, j, k)];
        num += dzf(g, k) * s;
        den += dzf(g, k) * (double)g->nx * (double)g->ny;
    }
    return num / den;
}

static void remove_weighted_mean(const grid_t *g, double *a) {
    double m = weighted_mean(g, a);
    size_t n = (size_t)g->nx * g->ny * g->nz;
    for (size_t c = 0; c < n; ++c) a[c] -= m;
}

/* ------------------------------------------------------------------ */
/* Public operator entry points                                          */
/* ------------------------------------------------------------------ */

void ora_grad(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
              int bcz, const double *q, double *gx, double *gy, double *gz) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    grad(&g, q, gx, gy, gz);
}

void ora_div(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
             int bcz, const double *u, const double *v, const double *w, double *out) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    divergence(&g, u, v, w, out);
}

/* Ghost rule of an x or y direction of kind bc (>= 1) at its near (side 0)
 * or far (side 1) boundary face: +1 mirrors the cell (Neumann), -1 mirrors
 * it with the opposite sign (Dirichlet). */
static double ghost_sign(int bc, int side) {
    int dir = (bc == 2) || (bc == 3 && side == 1) || (bc == 4 && side == 0);
    return dir ? -1.0 : 1.0;
}

/* L_h p with the boundary kinds 0..4 in x and y: every face gradient
 * (neighbour - centre)/h, the neighbour beyond a boundary face being the
 * ghost value; z as in grad(). */
static void lap_bc(const grid_t *g, const double *q, double *out) {
    int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(g, i, j, k);
                double qc = q[c], qe, qw, qn, qs;
                if (i < nx - 1) qe = q[IDX(g, i + 1, j, k)];
                else qe = g->bcx == 0 ? q[IDX(g, 0, j, k)] : ghost_sign(g->bcx, 1) * qc;
                if (i > 0) qw = q[IDX(g, i - 1, j, k)];
                else qw = g->bcx == 0 ? q[IDX(g, nx - 1, j, k)] : ghost_sign(g->bcx, 0) * qc;
                if (j < ny - 1) qn = q[IDX(g, i, j + 1, k)];
                else qn = g->bcy == 0 ? q[IDX(g, i, 0, k)] : ghost_sign(g->bcy, 1) * qc;
                if (j > 0) qs = q[IDX(g, i, j - 1, k)];
                else qs = g->bcy == 0 ? q[IDX(g, i, ny - 1, k)] : ghost_sign(g->bcy, 0) * qc;
                double ue = (qe - qc) / g->dx, uw = (qc - qw) / g->dx;
                double vn = (qn - qc) / g->dy, vs = (qc - qs) / g->dy;
                double wt, wb;
                if (k < nz - 1) wt = (q[IDX(g, i, j, k + 1)] - qc) / dzc(g, k);
                else wt = g->bcz == 0 ? (q[IDX(g, i, j, 0)] - qc) / dzc(g, k) : 0.0;
                if (k > 0) wb = (qc - q[IDX(g, i, j, k - 1)]) / dzc(g, k - 1);
                else wb = g->bcz == 0 ? (qc - q[IDX(g, i, j, nz - 1)]) / dzc(g, nz - 1) : 0.0;
                out[c] = (ue - uw) / g->dx + (vn - vs) / g->dy + (wt - wb) / dzf(g, k);
            }
}

/* The Poisson problem is singular (constants in its null space) unless a
 * Dirichlet face bounds x or y. */
static int singular(const grid_t *g) { return g->bcx <= 1 && g->bcy <= 1; }

/* L_h p = D(G p) */
void ora_apply_L(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
                 int bcz, const double *p, double *out) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    if (bcx > 1 || bcy > 1) {
        lap_bc(&g, p, out);
        return;
    }
    size_t n = (size_t)nx * ny * nz;
    double *gx = malloc(n * sizeof(double)), *gy = malloc(n * sizeof(double)),
           *gz = malloc(n * sizeof(double));
    grad(&g, p, gx, gy, gz);
    divergence(&g, gx, gy, gz, out);
    free(gx);
    free(gy);
    free(gz);
}

double ora_weighted_mean(int nx, int ny, int nz, const double *zf, const double *a) {
    grid_t g = mkgrid(nx, ny, nz, 1.0, 1.0, zf, 0, 0, 1);
    return weighted_mean(&g, a);
}

/* Split right-hand side: f = (rho0/dt) D(u*) + D[(1 - rho0 beta_f) G phat], then the
 * dzf-weighted mean is removed. */
void ora_rhs(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
             int bcz, double rho_l, double rho_g, double dt, const double *phi, const double *pn,
             const double *pnm1, const double *u, const double *v, const double *w, double *f) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    double rho0 = rho_l < rho_g ? rho_l : rho_g;
    double *ph = malloc(n * sizeof(double));
    double *gx = malloc(n * sizeof(double)), *gy = malloc(n * sizeof(double)),
           *gz = malloc(n * sizeof(double));
    double *bx = malloc(n * sizeof(double)), *by = malloc(n * sizeof(double)),
           *bz = malloc(n * sizeof(double));
    double *d2 = malloc(n * sizeof(double));
    for (size_t c = 0; c < n; ++c) ph[c] = 2.0 * pn[c] - pnm1[c];
    grad(&g, ph, gx, gy, gz);
    face_beta(&g, rho_l, rho_g, phi, bx, by, bz);
    for (size_t c = 0; c < n; ++c) {
        gx[c] *= (1.0 - rho0 * bx[c]);
        gy[c] *= (1.0 - rho0 * by[c]);
        gz[c] *= (1.0 - rho0 * bz[c]);
    }
    divergence(&g, gx, gy, gz, d2);
    divergence(&g, u, v, w, f);
    for (size_t c = 0; c < n; ++c) f[c] = (rho0 / dt) * f[c] + d2[c];
    remove_weighted_mean(&g, f);
    free(ph);
    free(gx);
    free(gy);
    free(gz);
    free(bx);
    free(by);
    free(bz);
    free(d2);
}

/* u = u* - dt [G p / rho0 + (beta_f - 1/rho0) G phat] on non-wall faces (in place). */
void ora_correct(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
                 int bcz, double rho_l, double rho_g, double dt, const double *phi, const double *pn,
                 const double *pnm1, const double *p, double *u, double *v, double *w) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    double rho0 = rho_l < rho_g ? rho_l : rho_g;
    double *ph = malloc(n * sizeof(double));
    double *px = malloc(n * sizeof(double)), *py = malloc(n * sizeof(double)),
           *pz = malloc(n * sizeof(double));
    double *hx = malloc(n * sizeof(double)), *hy = malloc(n * sizeof(double)),
           *hz = malloc(n * sizeof(double));
    double *bx = malloc(n * sizeof(double)), *by = malloc(n * sizeof(double)),
           *bz = malloc(n * sizeof(double));
    for (size_t c = 0; c < n; ++c) ph[c] = 2.0 * pn[c] - pnm1[c];
    grad(&g, p, px, py, pz);
    grad(&g, ph, hx, hy, hz);
    face_beta(&g, rho_l, rho_g, phi, bx, by, bz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(&g, i, j, k);
                if (!(bcx == 1 && i == nx - 1))
                    u[c] -= dt * (px[c] / rho0 + (bx[c] - 1.0 / rho0) * hx[c]);
                if (!(bcy == 1 && j == ny - 1))
                    v[c] -= dt * (py[c] / rho0 + (by[c] - 1.0 / rho0) * hy[c]);
                if (!(g.bcz == 1 && k == nz - 1))
                    w[c] -= dt * (pz[c] / rho0 + (bz[c] - 1.0 / rho0) * hz[c]);
            }
    free(ph);
    free(px);
    free(py);
    free(pz);
    free(hx);
    free(hy);
    free(hz);
    free(bx);
    free(by);
    free(bz);
}

/* ------------------------------------------------------------------ */
/* Fourier transforms                                                    */
/* ------------------------------------------------------------------ */

/* Table of the n-th roots of unity: w[t] = exp(sign * 2 pi i t / n), t = 0..n-1. */
static cplx *roots_table(int n, int sign) {
    cplx *w = malloc(sizeof(cplx) * (size_t)n);
    for (int t = 0; t < n; ++t) {
        double a = 2.0 * M_PI * (double)t / (double)n;
        w[t] = cos(a) + sign * I * sin(a);
    }
    return w;
}

/* Recursive decimation-in-time Cooley-Tukey FFT of any length n that divides
 * the table length ntab (w = roots_table(ntab, sign)).
 * n = r * m with r the smallest prime factor; the r interleaved sub-sequences
 * in[q + r s] are transformed recursively, then combined with
 *   out[k + m t] = sum_q W_n^(q (k + m t)) sub_q[k],   W_n = exp(sign 2 pi i / n);
 * a prime n is done as a plain DFT sum.  scratch must hold 2n values. */
static void fft_rec(int n, const cplx *in, int stride, cplx *out, const cplx *w, int ntab,
                    cplx *scratch) {
    int step = ntab / n; /* W_n^e = w[(e mod n) * step] */
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int r = 0;
    for (int d = 2; d * d <= n; ++d)
        if (n % d == 0) {
            r = d;
            break;
        }
    if (r == 0) { /* prime length: direct sum */
        for (int m = 0; m < n; ++m) {
            cplx s = 0;
            for (int t = 0; t < n; ++t)
                s += in[(size_t)t * stride] * w[(size_t)(((long)m * t) % n) * step];
            out[m] = s;
        }
        return;
    }
    int m = n / r;
    cplx *sub = scratch;        /* r blocks of m */
    cplx *deeper = scratch + n; /* scratch for the recursion */
    for (int q = 0; q < r; ++q)
        fft_rec(m, in + (size_t)q * stride, stride * r, sub + (size_t)q * m, w, ntab, deeper);
    for (int t = 0; t < r; ++t)
        for (int k = 0; k < m; ++k) {
            cplx s = 0;
            for (int q = 0; q < r; ++q)
                s += w[(size_t)(((long)q * (k + m * t)) % n) * step] * sub[(size_t)q * m + k];
            out[k + m * t] = s;
        }
}

/* In-place FFT of a strided complex sequence of length n (no scaling). */
static void fft_strided(int n, cplx *a, size_t stride, const cplx *w, cplx *tmp_in, cplx *tmp_out,
                        cplx *scratch) {
    for (int t = 0; t < n; ++t) tmp_in[t] = a[(size_t)t * stride];
    fft_rec(n, tmp_in, 1, tmp_out, w, n, scratch);
    for (int t = 0; t < n; ++t) a[(size_t)t * stride] = tmp_out[t];
}

/* out = sum_t in[t] exp(sign 2 pi i m t / n) by the recursive FFT. */
void ora_fft(int n, const double *re, const double *im, double *out_re, double *out_im, int sign) {
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n),
         *s = malloc(sizeof(cplx) * (2 * (size_t)n + 2));
    cplx *w = roots_table(n, sign);
    for (int t = 0; t < n; ++t) a[t] = re[t] + I * im[t];
    fft_rec(n, a, 1, b, w, n, s);
    for (int t = 0; t < n; ++t) {
        out_re[t] = creal(b[t]);
        out_im[t] = cimag(b[t]);
    }
    free(a);
    free(b);
    free(s);
    free(w);
}

/* Same sum evaluated directly, O(n^2), with the angle computed per term. */
void ora_dft(int n, const double *re, const double *im, double *out_re, double *out_im, int sign) {
    for (int m = 0; m < n; ++m) {
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < n; ++t) {
            double a = 2.0 * M_PI * (double)(((long)m * t) % n) / (double)n;
            double c = cos(a), s = sign * sin(a);
            sr += re[t] * c - im[t] * s;
            si += re[t] * s + im[t] * c;
        }
        out_re[m] = sr;
        out_im[m] = si;
    }
}

/* ------------------------------------------------------------------ */
/* Linear solvers                                                        */
/* ------------------------------------------------------------------ */

/* Gaussian elimination with partial pivoting on a real tridiagonal matrix with a
 * complex right-hand side.  dl[k] = A[k][k-1] (k >= 1), d[k] = A[k][k],
 * du[k] = A[k][k+1] (k <= n-2).  Row interchanges create a second
 * superdiagonal du2.  Arrays are overwritten; x = solution (in b).
 * Returns 0, or -1 if a zero pivot is met. */
static int tri_gepp(int n, double *dl, double *d, double *du, double *du2, cplx *b) {
    for (int k = 0; k < n; ++k) du2[k] = 0.0;
    for (int k = 0; k < n - 1; ++k) {
        double sub = dl[k + 1];
        if (fabs(d[k]) >= fabs(sub)) {
            if (d[k] == 0.0) return -1;
            double l = sub / d[k];
            d[k + 1] -= l * du[k];
            b[k + 1] -= l * b[k];
        } else {
            /* Interchange rows k and k+1, then eliminate.  Before: row k = [d_k, du_k]
             * at columns k, k+1; row k+1 = [sub, d_k1, du_k1] at columns k, k+1, k+2. */
            double d_k = d[k], du_k = du[k], d_k1 = d[k + 1];
            double du_k1 = (k + 1 < n - 1) ? du[k + 1] : 0.0;
            double l = d_k / sub;
            d[k] = sub; /* new row k = old row k+1 */
            du[k] = d_k1;
            du2[k] = du_k1;
            d[k + 1] = du_k - l * d_k1; /* new row k+1 = old row k - l * old row k+1 */
            if (k + 1 < n - 1) du[k + 1] = -l * du_k1;
            cplx bk = b[k];
            b[k] = b[k + 1];
            b[k + 1] = bk - l * b[k];
        }
    }
    if (d[n - 1] == 0.0) return -1;
    b[n - 1] /= d[n - 1];
    if (n > 1) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / d[n - 2];
    for (int k = n - 3; k >= 0; --k) b[k] = (b[k] - du[k] * b[k + 1] - du2[k] * b[k + 2]) / d[k];
    return 0;
}

/* Dense Gaussian elimination with partial pivoting, A (n x n, row major) x = b,
 * complex right-hand side.  A and b are overwritten; the solution is left in b. */
static int dense_gepp(int n, double *A, cplx *b) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + k]) > best) {
                best = fabs(A[(size_t)r * n + k]);
                piv = r;
            }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[(size_t)k * n + c];
                A[(size_t)k * n + c] = A[(size_t)piv * n + c];
                A[(size_t)piv * n + c] = t;
            }
            cplx t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double l = A[(size_t)r * n + k] / A[(size_t)k * n + k];
            if (l == 0.0) continue;
            for (int c = k; c < n; ++c) A[(size_t)r * n + c] -= l * A[(size_t)k * n + c];
            b[r] -= l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        cplx s = b[k];
        for (int c = k + 1; c < n; ++c) s -= A[(size_t)k * n + c] * b[c];
        b[k] = s / A[(size_t)k * n + k];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Poisson solve D G p = f                                               */
/* ------------------------------------------------------------------ */

/* Assemble A_z + lam I (nz x nz, row major) from the coupling coefficients:
 * row k has -(lo_k + up_k) + lam on the diagonal, lo_k in column k-1 and up_k
 * in column k+1, both taken cyclically (lo_0 and up_(nz-1) are 0 with walls,
 * so the wrapped entries only appear for periodic z; for nz = 2 the two
 * couplings of a row land in the same column and add). */
static void z_matrix(int nz, const double *lo, const double *up, double lam, double *A) {
    memset(A, 0, sizeof(double) * (size_t)nz * nz);
    for (int k = 0; k < nz; ++k) {
        A[(size_t)k * nz + k] += -(lo[k] + up[k]) + lam;
        A[(size_t)k * nz + (k + nz - 1) % nz] += lo[k];
        A[(size_t)k * nz + (k + 1) % nz] += up[k];
    }
}

/* Source index of extended position e in a direction of n cells:
 * periodic -> e; Neumann (extended to 2n by even reflection) -> mirror. */
static int ext_src(int e, int n, int bc) { return (bc == 0 || e < n) ? e : 2 * n - 1 - e; }

/* Length of the periodic problem a direction of kind bc extends to. */
static int ext_len(int n, int bc) { return bc == 0 ? n : (bc <= 2 ? 2 * n : 4 * n); }

/* Source cell and sign of extended position e (0 <= e < ext_len).  Neumann:
 * even about the far face (period 2n).  Dirichlet: odd about the far face
 * (period 2n, hence odd about the near face too).  Neumann near, Dirichlet
 * far: the first 2n positions odd about face n-1/2, the next 2n their even
 * mirror about face -1/2 (period 4n).  Dirichlet near, Neumann far: the first
 * 2n even about face n-1/2, the next 2n their odd mirror about face -1/2. */
static int ext_map(int e, int n, int bc, double *sign) {
    *sign = 1.0;
    if (bc == 0 || e < n) return e;
    if (bc == 1) return 2 * n - 1 - e;
    if (bc == 2) {
        *sign = -1.0;
        return 2 * n - 1 - e;
    }
    double s2 = 1.0;
    int e2 = e;
    if (e >= 2 * n) {          /* mirror about face -1/2 of the first 2n positions */
        e2 = 4 * n - 1 - e;
        s2 = bc == 3 ? 1.0 : -1.0;
    }
    if (e2 < n) {
        *sign = s2;
        return e2;
    }
    *sign = s2 * (bc == 3 ? -1.0 : 1.0);  /* reflection about face n-1/2 */
    return 2 * n - 1 - e2;
}

int ora_poisson_fft(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx,
                    int bcy, int bcz, const double *f, double *p) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    int mx = ext_len(nx, bcx); /* extent of the periodic problem */
    int my = ext_len(ny, bcy);
    const int sing = singular(&g);
    size_t plane = (size_t)mx * my;
    cplx *F = malloc(sizeof(cplx) * plane * nz);
    if (!F) return -3;
    int status = 0;

    /* even extension in wall directions (odd or quarter-wave with Dirichlet faces) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) {
                double sa, sb;
                int ia = (bcx <= 1) ? ext_src(a, nx, bcx) : ext_map(a, nx, bcx, &sa);
                int ib = (bcy <= 1) ? ext_src(b, ny, bcy) : ext_map(b, ny, bcy, &sb);
                double v = f[IDX(&g, ia, ib, k)];
                if (bcx > 1) v *= sa;
                if (bcy > 1) v *= sb;
                F[(size_t)k * plane + (size_t)b * mx + a] = v;
            }

    /* forward complex FFTs along x then y */
    cplx *wxf = roots_table(mx, -1), *wyf = roots_table(my, -1);
    cplx *wxb = roots_table(mx, +1), *wyb = roots_table(my, +1);
#pragma omp parallel
    {
        int nmax = mx > my ? mx : my;
        cplx *ti = malloc(sizeof(cplx) * nmax), *to = malloc(sizeof(cplx) * nmax),
             *sc = malloc(sizeof(cplx) * (2 * (size_t)nmax + 2));
#pragma omp for schedule(static) collapse(2)
        for (int k = 0; k < nz; ++k)
            for (int b = 0; b < my; ++b)
                fft_strided(mx, F + (size_t)k * plane + (size_t)b * mx, 1, wxf, ti, to, sc);
#pragma omp for schedule(static) collapse(2)
        for (int k = 0; k < nz; ++k)
            for (int a = 0; a < mx; ++a)
                fft_strided(my, F + (size_t)k * plane + a, (size_t)mx, wyf, ti, to, sc);
        free(ti);
        free(to);
        free(sc);
    }

    /* per-wavenumber z solve: A_z p + (lx + ly) p = F, where
       (A_z p)_k = [ (p_{k+1}-p_k)/dzc_{k+1/2} - (p_k-p_{k-1})/dzc_{k-1/2} ] / dzf_k
       and lx(m) = -(4/dx^2) sin^2(pi m / mx) is the eigenvalue of the periodic
       second difference of length mx on exp(2 pi i m x / mx). */
    double *lam_x = malloc(sizeof(double) * mx), *lam_y = malloc(sizeof(double) * my);
    for (int a = 0; a < mx; ++a) {
        double s = sin(M_PI * (double)a / (double)mx);
        lam_x[a] = -4.0 / (dx * dx) * s * s;
    }
    for (int b = 0; b < my; ++b) {
        double s = sin(M_PI * (double)b / (double)my);
        lam_y[b] = -4.0 / (dy * dy) * s * s;
    }
    /* z coefficients: lo[k] couples p_k to p_(k-1), up[k] to p_(k+1); with
       periodic z, lo[0] couples plane 0 to plane nz-1 and up[nz-1] plane nz-1
       to plane 0 (both through the face nz-1/2), with walls both are 0 */
    double *lo = malloc(sizeof(double) * nz), *up = malloc(sizeof(double) * nz);
    for (int k = 0; k < nz; ++k) {
        int per = g.bcz == 0;
        lo[k] = (k > 0) ? 1.0 / (dzf(&g, k) * dzc(&g, k - 1))
                        : (per ? 1.0 / (dzf(&g, 0) * dzc(&g, nz - 1)) : 0.0);
        up[k] = (k < nz - 1 || per) ? 1.0 / (dzf(&g, k) * dzc(&g, k)) : 0.0;
    }

#pragma omp parallel
    {
        double *dl = malloc(sizeof(double) * nz), *d = malloc(sizeof(double) * nz),
               *du = malloc(sizeof(double) * nz), *du2 = malloc(sizeof(double) * nz);
        double *A = g.bcz == 0 ? malloc(sizeof(double) * (size_t)nz * nz) : NULL;
        cplx *rhs = malloc(sizeof(cplx) * nz);
#pragma omp for schedule(static) collapse(2)
        for (int b = 0; b < my; ++b)
            for (int a = 0; a < mx; ++a) {
                if (a == 0 && b == 0) continue;
                double lam = lam_x[a] + lam_y[b];
                for (int k = 0; k < nz; ++k) rhs[k] = F[(size_t)k * plane + (size_t)b * mx + a];
                int bad;
                if (A) {
                    z_matrix(nz, lo, up, lam, A);
                    bad = dense_gepp(nz, A, rhs);
                } else {
                    for (int k = 0; k < nz; ++k) {
                        dl[k] = lo[k];
                        du[k] = up[k];
                        d[k] = -(lo[k] + up[k]) + lam;
                    }
                    bad = tri_gepp(nz, dl, d, du, du2, rhs);
                }
                if (bad != 0) {
#pragma omp atomic write
                    status = -1;
                }
                for (int k = 0; k < nz; ++k) F[(size_t)k * plane + (size_t)b * mx + a] = rhs[k];
            }
        free(dl);
        free(d);
        free(du);
        free(du2);
        free(A);
        free(rhs);
    }
    /* (0,0): singular; rows 0..nz-2 of A_z plus the gauge row sum_k dzf_k p_k = 0.
       With a Dirichlet face in x or y the extension has no mean: that mode
       is exactly zero. */
    if (!sing) {
        for (int k = 0; k < nz; ++k) F[(size_t)k * plane] = 0.0;
    } else {
        double *A = malloc(sizeof(double) * (size_t)nz * nz);
        cplx *rhs = malloc(sizeof(cplx) * nz);
        z_matrix(nz, lo, up, 0.0, A);
        for (int k = 0; k < nz - 1; ++k) rhs[k] = F[(size_t)k * plane];
        for (int k = 0; k < nz; ++k) A[(size_t)(nz - 1) * nz + k] = dzf(&g, k);
        rhs[nz - 1] = 0.0;
        if (nz == 1) A[0] = 1.0;
        if (dense_gepp(nz, A, rhs) != 0) status = -1;
        for (int k = 0; k < nz; ++k) F[(size_t)k * plane] = rhs[k];
        free(A);
        free(rhs);
    }

    /* backward FFTs along y then x, scale, restrict */
#pragma omp parallel
    {
        int nmax = mx > my ? mx : my;
        cplx *ti = malloc(sizeof(cplx) * nmax), *to = malloc(sizeof(cplx) * nmax),
             *sc = malloc(sizeof(cplx) * (2 * (size_t)nmax + 2));
#pragma omp for schedule(static) collapse(2)
        for (int k = 0; k < nz; ++k)
            for (int a = 0; a < mx; ++a)
                fft_strided(my, F + (size_t)k * plane + a, (size_t)mx, wyb, ti, to, sc);
#pragma omp for schedule(static) collapse(2)
        for (int k = 0; k < nz; ++k)
            for (int b = 0; b < my; ++b)
                fft_strided(mx, F + (size_t)k * plane + (size_t)b * mx, 1, wxb, ti, to, sc);
        free(ti);
        free(to);
        free(sc);
    }
    double scale = 1.0 / ((double)mx * (double)my);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                p[IDX(&g, i, j, k)] = creal(F[(size_t)k * plane + (size_t)j * mx + i]) * scale;
    if (sing) remove_weighted_mean(&g, p);
    free(wxf);
    free(wyf);
    free(wxb);
    free(wyb);
    free(lam_x);
    free(lam_y);
    free(lo);
    free(up);
    free(F);
    return status;
}

/* Dense path for small grids: assemble L_h column by column from ora_apply_L,
 * replace the last row by the gauge row (weights dzf_k) when the problem is
 * singular, solve by dense GEPP. */
int ora_poisson_dense(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx,
                      int bcy, int bcz, const double *f, double *p) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    if (n > 4096) return -2;
    double *A = calloc(n * n, sizeof(double));
    double *e = calloc(n, sizeof(double)), *col = malloc(n * sizeof(double));
    cplx *b = malloc(n * sizeof(cplx));
    for (size_t c = 0; c < n; ++c) {
        e[c] = 1.0;
        ora_apply_L(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, e, col);
        for (size_t r = 0; r < n; ++r) A[r * n + c] = col[r];
        e[c] = 0.0;
    }
    const int sing = singular(&g);
    if (sing)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) A[(n - 1) * n + IDX(&g, i, j, k)] = dzf(&g, k);
    for (size_t r = 0; r < n; ++r) b[r] = f[r];
    if (sing) b[n - 1] = 0.0;
    int st = dense_gepp((int)n, A, b);
    for (size_t r = 0; r < n; ++r) p[r] = creal(b[r]);
    if (sing) remove_weighted_mean(&g, p);
    free(A);
    free(e);
    free(col);
    free(b);
    return st;
}

/* ------------------------------------------------------------------ */
/* Whole projection                                                      */
/* ------------------------------------------------------------------ */

static double maxabs(const double *a, size_t n) {
    double m = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double v = fabs(a[c]);
        if (v > m) m = v;
    }
    return m;
}

/* Right-hand side, Poisson solve, correction.  u, v, w hold u* on entry and u on
 * exit; p receives p^(n+1) (zero dzf-weighted mean).  f (optional, may be NULL)
 * receives the right-hand side.  diag (optional, 3 doubles) receives
 * [relres = max|f - L p| / max|f|, max|D u|, max|f|].  Returns 0 on success. */
int ora_project(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
                int bcz, double rho_l, double rho_g, double dt, const double *phi, const double *pn,
                const double *pnm1, double *u, double *v, double *w, double *p, double *f_out,
                double *diag, int dense) {
    size_t n = (size_t)nx * ny * nz;
    double *f = malloc(n * sizeof(double)), *t = malloc(n * sizeof(double));
    ora_rhs(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, rho_l, rho_g, dt, phi, pn, pnm1, u, v, w, f);
    int st = dense ? ora_poisson_dense(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, f, p)
                   : ora_poisson_fft(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, f, p);
    ora_correct(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, rho_l, rho_g, dt, phi, pn, pnm1, p, u, v, w);
    if (diag) {
        ora_apply_L(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, p, t);
        for (size_t c = 0; c < n; ++c) t[c] = f[c] - t[c];
        double fm = maxabs(f, n);
        diag[0] = fm > 0 ? maxabs(t, n) / fm : maxabs(t, n);
        ora_div(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, u, v, w, t);
        diag[1] = maxabs(t, n);
        diag[2] = fm;
    }
    if (f_out) memcpy(f_out, f, n * sizeof(double));
    free(f);
    free(t);
    return st;
}

/* ------------------------------------------------------------------ */
/* Variable-coefficient projection (no splitting)                       */
/* ------------------------------------------------------------------ */
/* The pressure equation before the constant-coefficient splitting (the
 * paper's "Methods and Implementation strategy": the variable-coefficient
 * Poisson equation that the splitting replaces; the Hypre path of the code
 * solves it directly):
 *     D(beta_f G p) = D(u*)/dt,   u = u* - dt beta_f G p,
 * with beta_f = 1/rho_f as in face_beta (wall faces 0).  p has zero
 * dzf-weighted mean. */

/* out = D(beta_f G p) */
void ora_apply_vc(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
                  int bcz, double rho_l, double rho_g, const double *phi, const double *p,
                  double *out) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    double *gx = malloc(n * sizeof(double)), *gy = malloc(n * sizeof(double)),
           *gz = malloc(n * sizeof(double));
    double *bx = malloc(n * sizeof(double)), *by = malloc(n * sizeof(double)),
           *bz = malloc(n * sizeof(double));
    grad(&g, p, gx, gy, gz);
    face_beta(&g, rho_l, rho_g, phi, bx, by, bz);
    for (size_t c = 0; c < n; ++c) {
        gx[c] *= bx[c];
        gy[c] *= by[c];
        gz[c] *= bz[c];
    }
    divergence(&g, gx, gy, gz, out);
    free(gx);
    free(gy);
    free(gz);
    free(bx);
    free(by);
    free(bz);
}

/* Whole variable-coefficient projection on a small grid (n <= 4096 cells):
 * the operator is assembled column by column from ora_apply_vc, its last row
 * replaced by the gauge row (weights dzf_k), and solved by dense Gaussian
 * elimination with partial pivoting.  u, v, w hold u* on entry and u on
 * exit.  diag (optional, 2 doubles): [max|b - A p| / max|b|, max|D u|].
 * Returns 0, -2 if the grid is too large, -1 on a zero pivot. */
int ora_project_vc(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx,
                   int bcy, int bcz, double rho_l, double rho_g, double dt, const double *phi,
                   double *u, double *v, double *w, double *p, double *diag) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    if (n > 4096) return -2;
    double *A = calloc(n * n, sizeof(double));
    double *e = calloc(n, sizeof(double)), *col = malloc(n * sizeof(double));
    double *rhs = malloc(n * sizeof(double));
    cplx *b = malloc(n * sizeof(cplx));
    for (size_t c = 0; c < n; ++c) {
        e[c] = 1.0;
        ora_apply_vc(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, rho_l, rho_g, phi, e, col);
        for (size_t r = 0; r < n; ++r) A[r * n + c] = col[r];
        e[c] = 0.0;
    }
    divergence(&g, u, v, w, rhs);
    for (size_t c = 0; c < n; ++c) rhs[c] /= dt;
    remove_weighted_mean(&g, rhs);
    for (size_t r = 0; r < n; ++r) b[r] = rhs[r];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) A[(n - 1) * n + IDX(&g, i, j, k)] = dzf(&g, k);
    b[n - 1] = 0.0;
    int st = dense_gepp((int)n, A, b);
    for (size_t r = 0; r < n; ++r) p[r] = creal(b[r]);
    remove_weighted_mean(&g, p);
    /* u = u* - dt beta_f G p on non-wall faces */
    double *gx = malloc(n * sizeof(double)), *gy = malloc(n * sizeof(double)),
           *gz = malloc(n * sizeof(double));
    double *bx = malloc(n * sizeof(double)), *by = malloc(n * sizeof(double)),
           *bz = malloc(n * sizeof(double));
    grad(&g, p, gx, gy, gz);
    face_beta(&g, rho_l, rho_g, phi, bx, by, bz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(&g, i, j, k);
                if (!(bcx == 1 && i == nx - 1)) u[c] -= dt * bx[c] * gx[c];
                if (!(bcy == 1 && j == ny - 1)) v[c] -= dt * by[c] * gy[c];
                if (!(bcz == 1 && k == nz - 1)) w[c] -= dt * bz[c] * gz[c];
            }
    if (diag) {
        ora_apply_vc(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz, rho_l, rho_g, phi, p, col);
        double rm = 0.0, bm = 0.0;
        for (size_t c = 0; c < n; ++c) {
            double d = fabs(rhs[c] - col[c]);
            if (d > rm) rm = d;
            if (fabs(rhs[c]) > bm) bm = fabs(rhs[c]);
        }
        diag[0] = bm > 0 ? rm / bm : rm;
        divergence(&g, u, v, w, col);
        diag[1] = maxabs(col, n);
    }
    free(A);
    free(e);
    free(col);
    free(rhs);
    free(b);
    free(gx);
    free(gy);
    free(gz);
    free(bx);
    free(by);
    free(bz);
    return st;
}

/* ------------------------------------------------------------------ */
/* ACDI phase-field transport (the step that produces phi)              */
/* ------------------------------------------------------------------ */
/* The paper advances the phase field with the accurate conservative
 * diffuse-interface (ACDI) model of Jain (2022):
 *   d phi/dt + div(u phi) = div{ Gamma [ eps grad phi
 *                                        - 1/4 (1 - tanh^2(psi/(2 eps))) n ] },
 *   psi = eps ln((phi + delta)/(1 - phi + delta)),   n = grad psi / |grad psi|
 *   (each side of the quotient bounded below by delta, see acdi_psi).
 * Discretised in conservative (face-flux) form on the staggered grid:
 *   psi and n at cell centres (n from central differences of psi, a wall
 *   mirrors psi, |grad psi| = 0 gives n = 0);
 *   on a face between cells a and b: F = u_f (phi_a + phi_b)/2
 *       - Gamma [ eps (phi_b - phi_a)/h_ab
 *                 - 1/4 (1 - tanh^2((psi_a + psi_b)/(4 eps))) (n_a + n_b)/2 ],
 *   h_ab the centre distance, n the face-normal component; wall faces carry
 *   no flux;
 *   rhs = -D F;  one forward-Euler stage phi + dt rhs (stages of any explicit
 *   scheme are made of these). */

/* Jain's psi is defined for phi inside (0, 1).  A discrete phi can leave
 * [0, 1] by a small undershoot or overshoot (central advection does when the
 * velocity scale Gamma is below max|u|), and the plain quotient would then be
 * negative and its logarithm NaN.  Reading taken here: each side of the
 * quotient is bounded below by delta, so psi saturates (near -230 eps below
 * phi = 0, +230 eps above phi = 1) and stays finite; inside [0, 1] nothing
 * changes. */
static double acdi_psi(double phi, double eps, double delta) {
    const double a = phi + delta, b = 1.0 - phi + delta;
    return eps * log((a > delta ? a : delta) / (b > delta ? b : delta));
}

/* rhs = -D F for the ACDI face fluxes F (see above). */
void ora_acdi_rhs(int nx, int ny, int nz, double dx, double dy, const double *zf, int bcx, int bcy,
                  int bcz, double eps, double gam, double delta, const double *phi, const double *u,
                  const double *v, const double *w, double *rhs) {
    grid_t g = mkgrid(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz);
    size_t n = (size_t)nx * ny * nz;
    double *psi = malloc(n * sizeof(double));
    double *nxv = malloc(n * sizeof(double)), *nyv = malloc(n * sizeof(double)),
           *nzv = malloc(n * sizeof(double));
    double *fx = malloc(n * sizeof(double)), *fy = malloc(n * sizeof(double)),
           *fz = malloc(n * sizeof(double));
    for (size_t c = 0; c < n; ++c) psi[c] = acdi_psi(phi[c], eps, delta);
    /* unit normals at centres: central differences; at a wall the missing
     * neighbour mirrors the cell (psi_ghost = psi_cell, ghost centre mirrored
     * across the wall face) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(&g, i, j, k);
                int ip = i + 1, im = i - 1, jp = j + 1, jm = j - 1;
                double pxp, pxm, pyp, pym, pzp, pzm;
                if (ip == nx) ip = bcx == 0 ? 0 : -1;
                if (im < 0) im = bcx == 0 ? nx - 1 : -1;
                if (jp == ny) jp = bcy == 0 ? 0 : -1;
                if (jm < 0) jm = bcy == 0 ? ny - 1 : -1;
                pxp = ip >= 0 ? psi[IDX(&g, ip, j, k)] : psi[c];
                pxm = im >= 0 ? psi[IDX(&g, im, j, k)] : psi[c];
                pyp = jp >= 0 ? psi[IDX(&g, i, jp, k)] : psi[c];
                pym = jm >= 0 ? psi[IDX(&g, i, jm, k)] : psi[c];
                double gx = (pxp - pxm) / (2.0 * dx), gy = (pyp - pym) / (2.0 * dy);
                /* z: centre distance between the two neighbours used */
                double zlo, zhi;
                if (k + 1 < nz) {
                    pzp = psi[IDX(&g, i, j, k + 1)];
                    zhi = zc(&g, k + 1);
                } else if (bcz == 0) {
                    pzp = psi[IDX(&g, i, j, 0)];
                    zhi = zc(&g, 0) + (zf[nz] - zf[0]);
                } else {
                    pzp = psi[c];
                    zhi = 2.0 * zf[nz] - zc(&g, k);
                }
                if (k > 0) {
                    pzm = psi[IDX(&g, i, j, k - 1)];
                    zlo = zc(&g, k - 1);
                } else if (bcz == 0) {
                    pzm = psi[IDX(&g, i, j, nz - 1)];
                    zlo = zc(&g, nz - 1) - (zf[nz] - zf[0]);
                } else {
                    pzm = psi[c];
                    zlo = 2.0 * zf[0] - zc(&g, 0);
                }
                double gz = (pzp - pzm) / (zhi - zlo);
                double mag = sqrt(gx * gx + gy * gy + gz * gz);
                nxv[c] = mag > 0 ? gx / mag : 0.0;
                nyv[c] = mag > 0 ? gy / mag : 0.0;
                nzv[c] = mag > 0 ? gz / mag : 0.0;
            }
    /* face fluxes on the +x, +y, +z face of every cell (0 on walls) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(&g, i, j, k);
                int ie = (i < nx - 1) ? i + 1 : (bcx == 0 ? 0 : -1);
                int jn = (j < ny - 1) ? j + 1 : (bcy == 0 ? 0 : -1);
                int kt = (k < nz - 1) ? k + 1 : (bcz == 0 ? 0 : -1);
                fx[c] = fy[c] = fz[c] = 0.0;
                if (ie >= 0) {
                    size_t b = IDX(&g, ie, j, k);
                    double t = tanh((psi[c] + psi[b]) / (4.0 * eps));
                    fx[c] = u[c] * 0.5 * (phi[c] + phi[b]) -
                            gam * (eps * (phi[b] - phi[c]) / dx -
                                   0.25 * (1.0 - t * t) * 0.5 * (nxv[c] + nxv[b]));
                }
                if (jn >= 0) {
                    size_t b = IDX(&g, i, jn, k);
                    double t = tanh((psi[c] + psi[b]) / (4.0 * eps));
                    fy[c] = v[c] * 0.5 * (phi[c] + phi[b]) -
                            gam * (eps * (phi[b] - phi[c]) / dy -
                                   0.25 * (1.0 - t * t) * 0.5 * (nyv[c] + nyv[b]));
                }
                if (kt >= 0) {
                    size_t b = IDX(&g, i, j, kt);
                    double t = tanh((psi[c] + psi[b]) / (4.0 * eps));
                    fz[c] = w[c] * 0.5 * (phi[c] + phi[b]) -
                            gam * (eps * (phi[b] - phi[c]) / dzc(&g, k) -
                                   0.25 * (1.0 - t * t) * 0.5 * (nzv[c] + nzv[b]));
                }
            }
    divergence(&g, fx, fy, fz, rhs);
    for (size_t c = 0; c < n; ++c) rhs[c] = -rhs[c];
    free(psi);
    free(nxv);
    free(nyv);
    free(nzv);
    free(fx);
    free(fy);
    free(fz);
}

int ora_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
