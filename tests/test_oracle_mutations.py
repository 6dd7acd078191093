"""Planted mistakes in a copy of the oracle must make the pins fail.

Each case edits one plausible slip into a temporary copy of oracle/oracle.c
(a sign, a dropped term, a wrong index or spacing, a transposed operand),
compiles it, and runs the pin tests against that copy in a subprocess; the
pins must catch every one.  (Dropping the explicit mean removal of f is not
listed: the dzf-weighted sum of a discrete divergence with zero wall fluxes
telescopes to zero, so that edit changes only round-off.)  Nothing here touches a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

PINS = ("exact_rational or eigenmodes or apply_then_solve or divergence_free or "
        "constant_density or dense_solves or stretched_z or correction_identity or "
        "triperiodic or rotation_commutes or vc_ or acdi_ or poisson_bc")

MUTATIONS = [
    ("grad_sign", "gx[c] = (q[IDX(g, i + 1, j, k)] - q[c]) / g->dx;",
     "gx[c] = (q[c] - q[IDX(g, i + 1, j, k)]) / g->dx;"),
    ("grad_z_spacing", "(q[IDX(g, i, j, k + 1)] - q[c]) / dzc(g, k)",
     "(q[IDX(g, i, j, k + 1)] - q[c]) / dzf(g, k)"),
    ("div_z_spacing", "(wt - wb) / dzf(g, k)", "(wt - wb) / dzc(g, k > 0 ? k - 1 : 0)"),
    ("div_periodic_wrap", "(g->bcx == 0 ? u[IDX(g, nx - 1, j, k)] : 0.0)",
     "(g->bcx == 0 ? u[IDX(g, 0, j, k)] : 0.0)"),
    ("rhs_drop_rho0_over_dt", "f[c] = (rho0 / dt) * f[c] + d2[c];", "f[c] = f[c] + d2[c];"),
    ("rhs_split_sign", "gx[c] *= (1.0 - rho0 * bx[c]);", "gx[c] *= (rho0 * bx[c] - 1.0);"),
    ("face_density_sum", "bx[c] = 1.0 / (0.5 * (rc + re));", "bx[c] = 1.0 / (rc + re);"),
    ("rho0_max", "double rho0 = rho_l < rho_g ? rho_l : rho_g;\n    double *ph = malloc(n * sizeof(double));\n    double *gx",
     "double rho0 = rho_l > rho_g ? rho_l : rho_g;\n    double *ph = malloc(n * sizeof(double));\n    double *gx"),
    ("rhs_no_extrapolation", "for (size_t c = 0; c < n; ++c) ph[c] = 2.0 * pn[c] - pnm1[c];\n    grad(&g, ph, gx, gy, gz);",
     "for (size_t c = 0; c < n; ++c) ph[c] = pn[c];\n    grad(&g, ph, gx, gy, gz);"),
    ("correct_sign", "u[c] -= dt * (px[c] / rho0 + (bx[c] - 1.0 / rho0) * hx[c]);",
     "u[c] -= dt * (px[c] / rho0 + (1.0 / rho0 - bx[c]) * hx[c]);"),
    ("correct_transposed", "w[c] -= dt * (pz[c] / rho0 + (bz[c] - 1.0 / rho0) * hz[c]);",
     "w[c] -= dt * (hz[c] / rho0 + (bz[c] - 1.0 / rho0) * pz[c]);"),
    ("eigen_angle", "double s = sin(M_PI * (double)a / (double)mx);",
     "double s = sin(2.0 * M_PI * (double)a / (double)mx);"),
    ("z_coeff_index", "lo[k] = (k > 0) ? 1.0 / (dzf(&g, k) * dzc(&g, k - 1))",
     "lo[k] = (k > 0) ? 1.0 / (dzf(&g, k) * dzc(&g, k > 1 ? k - 2 : 0))"),
    ("inverse_scale", "double scale = 1.0 / ((double)mx * (double)my);", "double scale = 1.0 / (double)mx;"),
    ("correct_no_extrapolation",
     "for (size_t c = 0; c < n; ++c) ph[c] = 2.0 * pn[c] - pnm1[c];\n    grad(&g, p, px, py, pz);",
     "for (size_t c = 0; c < n; ++c) ph[c] = pn[c];\n    grad(&g, p, px, py, pz);"),
    ("z_coeff_upper", "up[k] = (k < nz - 1 || per) ? 1.0 / (dzf(&g, k) * dzc(&g, k)) : 0.0;",
     "up[k] = (k < nz - 1 || per) ? 1.0 / (dzc(&g, k) * dzc(&g, k)) : 0.0;"),
    # periodic z
    ("z_seam_spacing", "if (k == g->nz - 1) return 0.5 * (dzf(g, 0) + dzf(g, g->nz - 1));",
     "if (k == g->nz - 1) return dzf(g, g->nz - 1);"),
    ("grad_z_seam_sign", "gz[c] = g->bcz == 0 ? (q[IDX(g, i, j, 0)] - q[c]) / dzc(g, k) : 0.0;",
     "gz[c] = g->bcz == 0 ? (q[c] - q[IDX(g, i, j, 0)]) / dzc(g, k) : 0.0;"),
    ("div_z_seam_index", "(g->bcz == 0 ? w[IDX(g, i, j, nz - 1)] : 0.0)",
     "(g->bcz == 0 ? w[IDX(g, i, j, 0)] : 0.0)"),
    ("face_density_z_seam", "int kt = (k < nz - 1) ? k + 1 : (g->bcz == 0 ? 0 : -1);",
     "int kt = (k < nz - 1) ? k + 1 : (g->bcz == 0 ? k : -1);"),
    ("correct_skips_z_seam", "if (!(g.bcz == 1 && k == nz - 1))\n                    w[c]",
     "if (k < nz - 1)\n                    w[c]"),
    ("z_solve_seam_coupling", "(per ? 1.0 / (dzf(&g, 0) * dzc(&g, nz - 1)) : 0.0)",
     "(per ? 1.0 / (dzf(&g, nz - 1) * dzc(&g, nz - 1)) : 0.0)"),
    # variable-coefficient projection
    ("vc_beta_dropped_x", "        gx[c] *= bx[c];\n        gy[c] *= by[c];",
     "        gx[c] *= 1.0;\n        gy[c] *= by[c];"),
    ("vc_correct_sign", "if (!(bcx == 1 && i == nx - 1)) u[c] -= dt * bx[c] * gx[c];",
     "if (!(bcx == 1 && i == nx - 1)) u[c] += dt * bx[c] * gx[c];"),
    ("vc_rhs_dt", "for (size_t c = 0; c < n; ++c) rhs[c] /= dt;",
     "for (size_t c = 0; c < n; ++c) rhs[c] *= dt;"),
    # ACDI transport
    ("acdi_quarter", "0.25 * (1.0 - t * t) * 0.5 * (nxv[c] + nxv[b])",
     "0.5 * (1.0 - t * t) * 0.5 * (nxv[c] + nxv[b])"),
    ("acdi_tanh_width", "double t = tanh((psi[c] + psi[b]) / (4.0 * eps));",
     "double t = tanh((psi[c] + psi[b]) / (2.0 * eps));"),
    ("acdi_normal_one_sided", "0.5 * (nxv[c] + nxv[b])", "nxv[c]"),
    ("acdi_advect_upwind", "fx[c] = u[c] * 0.5 * (phi[c] + phi[b])", "fx[c] = u[c] * phi[c]"),
    ("acdi_psi_sign", "return eps * log((a > delta ? a : delta) / (b > delta ? b : delta));",
     "return eps * log((b > delta ? b : delta) / (a > delta ? a : delta));"),
    ("acdi_psi_unbounded", "return eps * log((a > delta ? a : delta) / (b > delta ? b : delta));",
     "return eps * log(a / b);"),
    ("acdi_z_wall_ghost", "zhi = 2.0 * zf[nz] - zc(&g, k);", "zhi = zf[nz];"),
    ("acdi_z_seam_distance", "zlo = zc(&g, nz - 1) - (zf[nz] - zf[0]);", "zlo = zc(&g, nz - 1);"),
    # Dirichlet and mixed x/y boundary kinds of the Poisson solve
    ("bc_ghost_sign", "    return dir ? -1.0 : 1.0;", "    return dir ? 1.0 : -1.0;"),
    ("bc_mixed_side", "int dir = (bc == 2) || (bc == 3 && side == 1) || (bc == 4 && side == 0);",
     "int dir = (bc == 2) || (bc == 3 && side == 0) || (bc == 4 && side == 1);"),
    ("bc_quarter_wave_length", "static int ext_len(int n, int bc) { return bc == 0 ? n : (bc <= 2 ? 2 * n : 4 * n); }",
     "static int ext_len(int n, int bc) { return bc == 0 ? n : 2 * n; }"),
    ("bc_odd_extension_sign", "    if (bc == 2) {\n        *sign = -1.0;", "    if (bc == 2) {\n        *sign = 1.0;"),
    ("bc_quarter_wave_mirror_sign", "        s2 = bc == 3 ? 1.0 : -1.0;", "        s2 = bc == 3 ? -1.0 : 1.0;"),
    ("bc_gauge_when_regular", "    if (sing) remove_weighted_mean(&g, p);\n    free(wxf);",
     "    remove_weighted_mean(&g, p);\n    free(wxf);"),
    ("z_matrix_wrap_column", "A[(size_t)k * nz + (k + nz - 1) % nz] += lo[k];",
     "A[(size_t)k * nz + (k + nz - 2) % nz] += lo[k];"),
    ("neumann_extension", "return (bc == 0 || e < n) ? e : 2 * n - 1 - e;",
     "return (bc == 0 || e < n) ? e : 2 * n - e - (e == 2 * n - 1 ? 1 : 0) - 0;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, "mutation anchor not found: " + name
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "oracle_mut.c"
    so_path = tmp_path / "oracle_mut.so"
    c_path.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o",
                           str(so_path), str(c_path), "-lm"])
    env = dict(os.environ, FIZZY_ORACLE_SO=str(so_path), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", PINS],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake %s was not caught:\n%s" % (name, r.stdout[-2000:])
