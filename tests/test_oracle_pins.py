"""Pins of the FP64 CPU oracle against facts other than itself.

Each test checks the oracle against mathematics: exact rational evaluation
(tests/golden), closed-form eigenfunctions of the discrete operator, exact
discrete identities, an independent library FFT, an independently assembled
dense matrix, and symmetries.  No test here needs a GPU.
"""
import glob
import json
import os
from fractions import Fraction as Q

import numpy as np
import pytest

import oracle as O
from paper_2502_04189_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    m = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (m if m > 0 else 1.0)


def uniform_zf(nz, lz=1.0):
    return np.arange(nz + 1) * (lz / nz)


# --------------------------------------------------------------------------
# FFT building block vs the plain DFT sum and vs numpy's FFT (independent)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 27, 32, 48, 96, 97, 128, 192, 256, 384])
def test_fft_matches_numpy_and_direct_sum(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    scale = np.sqrt(n) * 4
    assert np.max(np.abs(O.fft(x, -1) - ref)) < 1e-15 * scale * max(1, np.log2(n)) * 4
    assert np.max(np.abs(O.dft(x, -1) - ref)) < 1e-14 * scale * max(1, np.log2(n))
    assert np.max(np.abs(O.fft(x, +1) - np.fft.ifft(x) * n)) < 1e-14 * scale * max(1, np.log2(n))


# --------------------------------------------------------------------------
# Exact rational fixtures (the whole projection)
# --------------------------------------------------------------------------
def _golden_cases():
    return sorted(glob.glob(os.path.join(GOLDEN, "exact_*.json")))


@pytest.mark.parametrize("path", _golden_cases(), ids=lambda p: os.path.basename(p))
@pytest.mark.parametrize("dense", [False, True])
def test_projection_matches_exact_rational(path, dense):
    d = json.load(open(path))
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    shape = (nz, ny, nx)
    zf = np.array([float(Q(z)) for z in d["zf"]])
    g = O.Grid(nx, ny, nz, float(Q(d["dx"])), float(Q(d["dy"])), zf, d["bcx"], d["bcy"],
               d.get("bcz", I.NEUMANN))
    inp = {k: np.array(v).reshape(shape) for k, v in d["inputs"].items()}
    exp = {k: np.array(v).reshape(shape) for k, v in d["expected"].items()}
    r = O.project(g, float(Q(d["rho_l"])), float(Q(d["rho_g"])), float(Q(d["dt"])), inp["phi"],
                  inp["pn"], inp["pnm1"], inp["u"], inp["v"], inp["w"], dense=dense)
    assert relerr(r["f"], exp["f"]) < 1e-14
    assert relerr(r["p"], exp["p"]) < 1e-13
    uu = np.concatenate([r["u"].ravel(), r["v"].ravel(), r["w"].ravel()])
    ue = np.concatenate([exp["u"].ravel(), exp["v"].ravel(), exp["w"].ravel()])
    assert relerr(uu, ue) < 1e-13


# --------------------------------------------------------------------------
# T1: Fourier eigenmodes of the discrete Laplacian (closed form)
# --------------------------------------------------------------------------
def _mode_1d(n, h, m, bc, phase):
    """(values at cell centres, eigenvalue of the second difference)."""
    i = np.arange(n)
    if bc == I.PERIODIC:
        return np.cos(2 * np.pi * m * i / n + phase), -4.0 / h ** 2 * np.sin(np.pi * m / n) ** 2
    return np.cos(np.pi * m * (i + 0.5) / n), -4.0 / h ** 2 * np.sin(np.pi * m / (2 * n)) ** 2


@pytest.mark.parametrize("nx,ny,nz,bcx,bcy", [
    (16, 12, 10, 0, 0), (12, 16, 9, 1, 0), (8, 18, 8, 0, 1), (9, 8, 12, 1, 1), (27, 6, 7, 0, 0)])
def test_eigenmodes_closed_form(nx, ny, nz, bcx, bcy):
    dx, dy, dz = 1.0 / nx, 0.7 / ny, 1.3 / nz
    g = O.Grid(nx, ny, nz, dx, dy, uniform_zf(nz, 1.3), bcx, bcy)
    rng = np.random.default_rng(nx * 100 + ny)
    modes = [(0, 0, 1), (1, 0, 0), (0, 1, 0), (nx // 2, ny // 2, nz - 1), (1, 2, 3),
             (nx - 1, 1, 2), (2, ny - 1, nz // 2)]
    for a, b, c in modes:
        X, lx = _mode_1d(nx, dx, a, bcx, rng.random() * 6.28)
        Y, ly = _mode_1d(ny, dy, b, bcy, rng.random() * 6.28)
        Z, lz = _mode_1d(nz, dz, c, I.NEUMANN, 0.0)
        q = Z[:, None, None] * Y[None, :, None] * X[None, None, :]
        lam = lx + ly + lz
        Lq = O.apply_L(g, q)
        assert np.max(np.abs(Lq - lam * q)) < 1e-12 * max(1.0, abs(lam))
        if abs(lam) > 0 and np.max(np.abs(q)) > 1e-12:
            p = O.poisson(g, lam * q)
            q0 = q - O.weighted_mean(g, q)
            assert relerr(p, q0) < 1e-12


@pytest.mark.parametrize("nx,ny,nz,bcx,bcy", [
    (16, 12, 10, 0, 0), (12, 16, 9, 1, 0), (9, 8, 12, 1, 1), (8, 6, 2, 0, 1), (6, 8, 3, 1, 0)])
def test_eigenmodes_closed_form_periodic_z(nx, ny, nz, bcx, bcy):
    """Periodic z (triperiodic boxes of the paper's emulsion case): the z
    factor is a Fourier mode of the periodic second difference."""
    dx, dy, dz = 1.0 / nx, 0.7 / ny, 1.3 / nz
    g = O.Grid(nx, ny, nz, dx, dy, uniform_zf(nz, 1.3), bcx, bcy, I.PERIODIC)
    rng = np.random.default_rng(nx * 100 + ny + 7)
    modes = [(0, 0, 1), (1, 0, 0), (0, 1, 1), (nx // 2, ny // 2, nz // 2), (1, 2, 1),
             (nx - 1, 1, nz - 1), (2, ny - 1, 0)]
    for a, b, c in modes:
        X, lx = _mode_1d(nx, dx, a, bcx, rng.random() * 6.28)
        Y, ly = _mode_1d(ny, dy, b, bcy, rng.random() * 6.28)
        Z, lz = _mode_1d(nz, dz, c, I.PERIODIC, rng.random() * 6.28)
        q = Z[:, None, None] * Y[None, :, None] * X[None, None, :]
        lam = lx + ly + lz
        Lq = O.apply_L(g, q)
        assert np.max(np.abs(Lq - lam * q)) < 1e-12 * max(1.0, abs(lam))
        if abs(lam) > 0 and np.max(np.abs(q)) > 1e-12:
            p = O.poisson(g, lam * q)
            q0 = q - O.weighted_mean(g, q)
            assert relerr(p, q0) < 1e-12


def test_triperiodic_poisson_matches_numpy_fft():
    """Uniform triperiodic grid: D G is diagonal in the 3-D discrete Fourier
    basis, so numpy's FFT with the closed-form eigenvalues solves it exactly
    (an independent library routine against the oracle's z-line solves)."""
    nx, ny, nz = 12, 10, 16
    dx, dy, dz = 1.0 / nx, 0.8 / ny, 1.2 / nz
    g = O.Grid(nx, ny, nz, dx, dy, uniform_zf(nz, 1.2), I.PERIODIC, I.PERIODIC, I.PERIODIC)
    f = np.random.default_rng(4).standard_normal(g.shape)
    f -= f.mean()
    lam = (-4 / dz ** 2 * np.sin(np.pi * np.arange(nz) / nz) ** 2)[:, None, None] + \
          (-4 / dy ** 2 * np.sin(np.pi * np.arange(ny) / ny) ** 2)[None, :, None] + \
          (-4 / dx ** 2 * np.sin(np.pi * np.arange(nx) / nx) ** 2)[None, None, :]
    F = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    F /= lam
    F[0, 0, 0] = 0.0
    p_np = np.real(np.fft.ifftn(F))
    assert relerr(O.poisson(g, f), p_np) < 1e-12
    assert relerr(O.apply_L(g, p_np), f) < 1e-12


def test_periodic_z_rotation_commutes_stretched():
    """A periodic z direction has no distinguished plane: rotating the cell
    spacings and every field by s planes (so the periodic seam moves inside
    the domain, where the centre distance is formed from the neighbouring
    centres) must rotate the projection's results."""
    spec = I.CaseSpec(nx=10, ny=8, nz=12, beta=1.8, n_bubbles=2, radius_cells=2.0, config=12,
                      bcz=I.PERIODIC)
    c = I.make_case(spec)
    g0 = O.Grid.of_case(c)
    r0 = O.project_case(c)
    for sh in (1, 5):
        dzf = np.roll(np.diff(c.zf), sh)
        zf1 = np.concatenate([[0.0], np.cumsum(dzf)])
        g1 = O.Grid(spec.nx, spec.ny, spec.nz, c.dx, c.dy, zf1, spec.bcx, spec.bcy, I.PERIODIC)
        rl = lambda a: np.roll(a, sh, axis=0)
        r1 = O.project(g1, spec.rho_l, spec.rho_g, spec.dt, rl(c.phi), rl(c.pn), rl(c.pnm1),
                       rl(c.u), rl(c.v), rl(c.w))
        for key in ("p", "u", "v", "w"):
            assert relerr(r1[key], rl(r0[key])) < 1e-11, (sh, key)
    assert abs(O.weighted_mean(g0, r0["p"])) < 1e-12 * np.max(np.abs(r0["p"]))


# --------------------------------------------------------------------------
# Stretched z: closed-form action on linear and quadratic profiles
# --------------------------------------------------------------------------
@pytest.mark.parametrize("beta", [0.0, 1.5, 2.5])
def test_stretched_z_operator_closed_form(beta):
    nx, ny, nz = 4, 3, 11
    zf = I.z_faces(nz, 1.0, beta)
    zc = 0.5 * (zf[:-1] + zf[1:])
    dzf = np.diff(zf)
    g = O.Grid(nx, ny, nz, 0.25, 0.3, zf, 0, 1)
    ones = np.ones((nz, ny, nx))
    # q = z: interior fluxes are exactly 1, wall fluxes 0
    L1 = O.apply_L(g, zc[:, None, None] * ones)
    e1 = np.zeros(nz)
    e1[0] = 1.0 / dzf[0]
    e1[-1] = -1.0 / dzf[-1]
    assert np.max(np.abs(L1 - e1[:, None, None] * ones)) < 1e-10 * np.max(np.abs(e1))
    # q = z^2: flux at k+1/2 is zc[k+1] + zc[k]
    L2 = O.apply_L(g, (zc ** 2)[:, None, None] * ones)
    F = np.concatenate([[0.0], zc[1:] + zc[:-1], [0.0]])
    e2 = (F[1:] - F[:-1]) / dzf
    assert np.max(np.abs(L2 - e2[:, None, None] * ones)) < 1e-10 * np.max(np.abs(e2))


# --------------------------------------------------------------------------
# T3: apply-then-solve on random fields (uniform and stretched, all BCs)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,nz,bcx,bcy,beta,bcz", [
    (16, 16, 16, 0, 0, 0.0, 1), (12, 18, 10, 1, 0, 1.5, 1), (18, 8, 13, 0, 1, 2.0, 1),
    (6, 9, 24, 1, 1, 1.0, 1), (32, 24, 20, 0, 0, 1.5, 1),
    (16, 12, 16, 0, 0, 0.0, 0), (12, 8, 11, 1, 0, 1.5, 0), (8, 6, 3, 0, 1, 0.0, 0)])
def test_apply_then_solve(nx, ny, nz, bcx, bcy, beta, bcz):
    g = O.Grid(nx, ny, nz, 1.0 / nx, 1.1 / ny, I.z_faces(nz, 0.9, beta), bcx, bcy, bcz)
    q = np.random.default_rng(7).standard_normal(g.shape)
    p = O.poisson(g, O.apply_L(g, q))
    q0 = q - O.weighted_mean(g, q)
    assert relerr(p, q0) < 1e-11
    assert abs(O.weighted_mean(g, p)) < 1e-14


# --------------------------------------------------------------------------
# T2: dense solves (oracle's own dense path and an independent numpy matrix)
# --------------------------------------------------------------------------
def _numpy_laplacian(nx, ny, nz, dx, dy, zf, bcx, bcy, bcz=I.NEUMANN):
    """7-point operator assembled independently from the stencil weights; with
    periodic z the seam face joins centre nz-1 to centre 0 + lz."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    dzf = np.diff(zf)
    zc = 0.5 * (zf[:-1] + zf[1:])
    dzc = np.diff(np.concatenate([zc, [zc[0] + (zf[-1] - zf[0])]]))  # dzc[nz-1]: the seam

    def ix(i, j, k):
        return (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = ix(i, j, k)
                # x neighbours
                for s in (-1, 1):
                    ii = i + s
                    if 0 <= ii < nx or bcx == I.PERIODIC:
                        A[r, ix(ii % nx, j, k)] += 1 / dx ** 2
                        A[r, r] -= 1 / dx ** 2
                for s in (-1, 1):
                    jj = j + s
                    if 0 <= jj < ny or bcy == I.PERIODIC:
                        A[r, ix(i, jj % ny, k)] += 1 / dy ** 2
                        A[r, r] -= 1 / dy ** 2
                if k + 1 < nz or bcz == I.PERIODIC:
                    A[r, ix(i, j, (k + 1) % nz)] += 1 / (dzf[k] * dzc[k])
                    A[r, r] -= 1 / (dzf[k] * dzc[k])
                if k - 1 >= 0 or bcz == I.PERIODIC:
                    A[r, ix(i, j, (k - 1) % nz)] += 1 / (dzf[k] * dzc[k - 1])
                    A[r, r] -= 1 / (dzf[k] * dzc[k - 1])
    return A


@pytest.mark.parametrize("nx,ny,nz,bcx,bcy,beta,bcz", [
    (8, 8, 8, 0, 0, 0.0, 1), (8, 6, 10, 1, 0, 1.5, 1), (6, 8, 7, 0, 1, 1.0, 1), (4, 6, 8, 1, 1, 2.0, 1),
    (8, 6, 8, 0, 0, 0.0, 0), (6, 8, 9, 1, 0, 1.5, 0), (4, 6, 2, 0, 1, 0.0, 0), (6, 4, 7, 1, 1, 2.0, 0)])
def test_dense_solves(nx, ny, nz, bcx, bcy, beta, bcz):
    zf = I.z_faces(nz, 1.0, beta)
    g = O.Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, zf, bcx, bcy, bcz)
    A = _numpy_laplacian(nx, ny, nz, g.dx, g.dy, zf, bcx, bcy, bcz)
    q = np.random.default_rng(3).standard_normal(g.shape)
    # the oracle's operator is the independently assembled matrix
    assert np.max(np.abs(O.apply_L(g, q).ravel() - A @ q.ravel())) < 1e-9 * np.max(np.abs(A))
    f = O.apply_L(g, q)
    f -= O.weighted_mean(g, f)
    p_fft = O.poisson(g, f)
    p_dense = O.poisson(g, f, dense=True)
    # numpy least-squares on the singular system, gauge fixed afterwards
    p_np = np.linalg.lstsq(A, f.ravel(), rcond=None)[0].reshape(g.shape)
    p_np -= O.weighted_mean(g, p_np)
    assert relerr(p_fft, p_dense) < 1e-11
    assert relerr(p_fft, p_np) < 1e-10


# --------------------------------------------------------------------------
# T4: the corrected velocity is discretely divergence-free
# --------------------------------------------------------------------------
@pytest.mark.parametrize("spec", [I.drop32_spec(),
                                  I.bubbles_spec(24, 3, 3.0, 1.5, config=1),
                                  I.CaseSpec(nx=16, ny=24, nz=20, bcx=1, bcy=0, n_bubbles=2,
                                             radius_cells=3, beta=1.0, config=3),
                                  I.CaseSpec(nx=20, ny=16, nz=18, n_bubbles=3, radius_cells=3,
                                             config=13, bcz=I.PERIODIC),
                                  I.CaseSpec(nx=12, ny=16, nz=14, bcx=1, n_bubbles=2,
                                             radius_cells=2.5, beta=1.5, config=14,
                                             bcz=I.PERIODIC)],
                         ids=["drop32", "bubbles24_stretched", "neumann_x", "triperiodic",
                              "periodic_z_stretched"])
def test_divergence_free(spec):
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    r = O.project_case(c)
    U = np.sqrt((np.sum(c.u ** 2) + np.sum(c.v ** 2) + np.sum(c.w ** 2)) / (3 * c.u.size))
    assert r["relres"] < 1e-12
    assert r["divmax"] * c.dx / U < 1e-10
    assert abs(O.weighted_mean(g, r["p"])) < 1e-12 * np.max(np.abs(r["p"]))
    assert abs(O.weighted_mean(g, r["f"])) < 1e-12 * np.max(np.abs(r["f"]))
    # wall faces untouched (zero)
    if spec.bcx == I.NEUMANN:
        assert np.all(r["u"][:, :, -1] == 0)
    if spec.bcz == I.NEUMANN:
        assert np.all(r["w"][-1] == 0)


# --------------------------------------------------------------------------
# T5: equal densities -> constant-density projection in closed form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bcx,bcy,beta", [(0, 0, 0.0), (1, 0, 1.5), (1, 1, 1.0)])
def test_constant_density_closed_form(bcx, bcy, beta):
    spec = I.CaseSpec(nx=16, ny=12, nz=14, bcx=bcx, bcy=bcy, beta=beta, n_bubbles=2,
                      radius_cells=2.5, rho_l=0.5, rho_g=0.5, dt=1e-3, noise=0.0, config=9)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    s = (c.u, c.v, c.w)                        # discrete curl: solenoidal
    assert np.max(np.abs(O.div(g, *s))) < 1e-10 * np.max(np.abs(c.u)) / c.dx
    q = np.random.default_rng(5).standard_normal(g.shape)
    gq = O.grad(g, q)
    ustar = [s[a] + gq[a] for a in range(3)]
    r = O.project(g, 0.5, 0.5, 1e-3, c.phi, c.pn, c.pnm1, *ustar)
    p_exact = (0.5 / 1e-3) * (q - O.weighted_mean(g, q))
    assert relerr(r["p"], p_exact) < 1e-11
    for a, key in enumerate("uvw"):
        assert np.max(np.abs(r[key] - s[a])) < 1e-11 * np.max(np.abs(ustar[a]))


# --------------------------------------------------------------------------
# Helmholtz decomposition identity at every non-wall face
# --------------------------------------------------------------------------
def test_correction_identity():
    c = I.make_case(I.CaseSpec(nx=12, ny=10, nz=9, bcx=1, bcy=0, beta=1.2, n_bubbles=1,
                               radius_cells=2.5, rho_l=1.0, rho_g=0.01, dt=1e-3, config=8))
    g = O.Grid.of_case(c)
    s = c.spec
    r = O.project_case(c)
    rho0 = min(s.rho_l, s.rho_g)
    gp = O.grad(g, r["p"])
    gh = O.grad(g, 2 * c.pn - c.pnm1)
    rho = s.rho_g + c.phi * (s.rho_l - s.rho_g)
    # face densities by neighbour averaging (independent numpy restatement)
    rf = [0.5 * (rho + np.roll(rho, -1, axis=2)), 0.5 * (rho + np.roll(rho, -1, axis=1)),
          0.5 * (rho + np.concatenate([rho[1:], rho[-1:]], axis=0))]
    for a, (ust, un) in enumerate(((c.u, r["u"]), (c.v, r["v"]), (c.w, r["w"]))):
        lhs = (rho0 / s.dt) * (ust - un) - rho0 * (1.0 / rf[a] - 1.0 / rho0) * gh[a]
        mask = np.ones(g.shape, bool)
        if a == 0 and s.bcx == I.NEUMANN:
            mask[:, :, -1] = False
        if a == 2:
            mask[-1] = False
        scale = np.max(np.abs(gp[a][mask])) + np.max(np.abs(rho0 * (1.0 / rf[a] - 1.0 / rho0) * gh[a]))
        assert np.max(np.abs(lhs[mask] - gp[a][mask])) < 1e-10 * scale


# --------------------------------------------------------------------------
# T8: symmetries
# --------------------------------------------------------------------------
def test_periodic_shift_commutes():
    c = I.make_case(I.CaseSpec(nx=16, ny=12, nz=10, beta=1.5, n_bubbles=2, radius_cells=2.5,
                               config=7))
    g = O.Grid.of_case(c)
    s = c.spec
    r0 = O.project_case(c)
    sh = 5
    rl = lambda a: np.roll(a, sh, axis=2)
    r1 = O.project(g, s.rho_l, s.rho_g, s.dt, rl(c.phi), rl(c.pn), rl(c.pnm1), rl(c.u), rl(c.v),
                   rl(c.w))
    for key in ("p", "u", "v", "w"):
        assert relerr(r1[key], rl(r0[key])) < 1e-12


def test_z_mirror_symmetry():
    c = I.make_case(I.CaseSpec(nx=10, ny=8, nz=12, beta=1.5, n_bubbles=2, radius_cells=2.0,
                               config=6))
    g = O.Grid.of_case(c)
    s = c.spec
    r0 = O.project_case(c)
    fz = lambda a: a[::-1].copy()

    def fw(w):  # face k+1/2 -> face (nz-2-k)+1/2, sign flipped; top wall stays 0
        out = np.zeros_like(w)
        out[:-1] = -w[:-1][::-1]
        return out
    r1 = O.project(g, s.rho_l, s.rho_g, s.dt, fz(c.phi), fz(c.pn), fz(c.pnm1), fz(c.u), fz(c.v),
                   fw(c.w))
    assert relerr(r1["p"], fz(r0["p"])) < 1e-12
    assert relerr(r1["u"], fz(r0["u"])) < 1e-12
    assert relerr(r1["w"], fw(r0["w"])) < 1e-12


def test_linearity_in_velocity_and_pressure():
    c = I.make_case(I.CaseSpec(nx=12, ny=12, nz=8, bcy=1, n_bubbles=1, radius_cells=3, config=5))
    g = O.Grid.of_case(c)
    s = c.spec
    rng = np.random.default_rng(2)
    a, b = 0.7, -1.3
    u2, v2, w2 = (rng.standard_normal(g.shape) for _ in range(3))
    v2[:, -1, :] = 0
    w2[-1] = 0
    pn2, pm2 = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    r1 = O.project(g, s.rho_l, s.rho_g, s.dt, c.phi, c.pn, c.pnm1, c.u, c.v, c.w)
    r2 = O.project(g, s.rho_l, s.rho_g, s.dt, c.phi, pn2, pm2, u2, v2, w2)
    r3 = O.project(g, s.rho_l, s.rho_g, s.dt, c.phi, a * c.pn + b * pn2, a * c.pnm1 + b * pm2,
                   a * c.u + b * u2, a * c.v + b * v2, a * c.w + b * w2)
    for key in ("p", "u", "v", "w"):
        assert relerr(r3[key], a * r1[key] + b * r2[key]) < 1e-11


def test_phase_swap_is_the_same_problem():
    """(phi, rho_l, rho_g) and (1 - phi, rho_g, rho_l) describe the same density
    field, so the projections agree to round-off; the swapped run has
    rho0 = rho_l, the split coefficient then being formed from 1 - phi."""
    c = I.make_case(I.CaseSpec(nx=12, ny=10, nz=9, bcx=1, beta=1.2, n_bubbles=2, radius_cells=2.5,
                               rho_l=1.0, rho_g=1e-3, config=4))
    g = O.Grid.of_case(c)
    s = c.spec
    r0 = O.project(g, s.rho_l, s.rho_g, s.dt, c.phi, c.pn, c.pnm1, c.u, c.v, c.w)
    r1 = O.project(g, s.rho_g, s.rho_l, s.dt, 1.0 - c.phi, c.pn, c.pnm1, c.u, c.v, c.w)
    for key in ("p", "u", "v", "w"):
        assert relerr(r1[key], r0[key]) < 1e-12, key



# --------------------------------------------------------------------------
# Variable-coefficient projection without splitting (D beta G p = D u*/dt)
# --------------------------------------------------------------------------
def _numpy_vc_operator(g, rho_l, rho_g, phi):
    """D(beta_f G .) assembled independently from face densities (walls 0;
    periodic neighbours wrap; the periodic-z seam spacing joins the last
    centre to the first + lz)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    zf = g.zf
    dzf = np.diff(zf)
    zc = 0.5 * (zf[:-1] + zf[1:])
    dzc = np.diff(np.concatenate([zc, [zc[0] + (zf[-1] - zf[0])]]))
    rho = rho_g + phi * (rho_l - rho_g)
    n = nx * ny * nz
    A = np.zeros((n, n))

    def ix(i, j, k):
        return (k * ny + j) * nx + i

    def couple(r, c, coef):
        A[r, c] += coef
        A[r, r] -= coef
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = ix(i, j, k)
                for s in (-1, 1):
                    ii = i + s
                    if 0 <= ii < nx or g.bcx == I.PERIODIC:
                        b = 2.0 / (rho[k, j, i] + rho[k, j, ii % nx])
                        couple(r, ix(ii % nx, j, k), b / g.dx ** 2)
                    jj = j + s
                    if 0 <= jj < ny or g.bcy == I.PERIODIC:
                        b = 2.0 / (rho[k, j, i] + rho[k, jj % ny, i])
                        couple(r, ix(i, jj % ny, k), b / g.dy ** 2)
                    kk = k + s
                    if 0 <= kk < nz or g.bcz == I.PERIODIC:
                        b = 2.0 / (rho[k, j, i] + rho[kk % nz, j, i])
                        h = dzc[k] if s == 1 else dzc[k - 1]
                        couple(r, ix(i, j, kk % nz), b / (dzf[k] * h))
    return A


@pytest.mark.parametrize("bcx,bcy,bcz,beta", [(0, 0, 1, 0.0), (1, 0, 1, 1.5), (0, 1, 0, 1.2),
                                              (1, 1, 0, 0.0)])
def test_vc_operator_matches_numpy_assembly(bcx, bcy, bcz, beta):
    nx, ny, nz = 6, 5, 7
    spec = I.CaseSpec(nx=nx, ny=ny, nz=nz, bcx=bcx, bcy=bcy, bcz=bcz, beta=beta, n_bubbles=1,
                      radius_cells=1.5, rho_l=1.0, rho_g=0.02, config=80)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    A = _numpy_vc_operator(g, spec.rho_l, spec.rho_g, c.phi)
    q = np.random.default_rng(8).standard_normal(g.shape)
    Aq = O.apply_vc(g, spec.rho_l, spec.rho_g, c.phi, q)
    assert np.max(np.abs(Aq.ravel() - A @ q.ravel())) < 1e-12 * np.max(np.abs(A)) * np.max(np.abs(q)) * 10
    # symmetric in the cell-volume (dzf-weighted) inner product
    W = np.repeat(np.diff(c.zf), nx * ny)
    WA = W[:, None] * A
    assert np.max(np.abs(WA - WA.T)) < 1e-12 * np.max(np.abs(WA))


@pytest.mark.parametrize("bcz", [1, 0])
def test_vc_constant_density_reduces_to_poisson(bcz):
    """rho_l = rho_g = rho: D(G p)/rho = D(u*)/dt, so p = rho L^-1 (D u*/dt),
    and the projected velocity equals the split projection's (the splitting
    is exact for a constant density)."""
    spec = I.CaseSpec(nx=12, ny=10, nz=8, bcx=1, beta=1.3, n_bubbles=1, radius_cells=2,
                      rho_l=0.7, rho_g=0.7, dt=1e-3, velocity="iid", config=81, bcz=bcz)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    r = O.project_vc(g, 0.7, 0.7, 1e-3, c.phi, c.u, c.v, c.w)
    b = O.div(g, c.u, c.v, c.w) / 1e-3
    b -= O.weighted_mean(g, b)
    assert relerr(r["p"], 0.7 * O.poisson(g, b)) < 1e-11
    s = O.project(g, 0.7, 0.7, 1e-3, c.phi, c.pn, c.pnm1, c.u, c.v, c.w)
    for k in "uvw":
        assert relerr(r[k], s[k]) < 1e-11, k
    assert r["relres"] < 1e-12


@pytest.mark.parametrize("bcz", [1, 0])
def test_vc_divergence_free_and_helmholtz(bcz):
    """Ratio 1000: D u = 0, and u* - u = dt beta_f G p on every non-wall face
    (beta_f, G restated in numpy)."""
    spec = I.CaseSpec(nx=12, ny=10, nz=9, bcy=1, beta=1.5, n_bubbles=2, radius_cells=2.0,
                      rho_l=1.0, rho_g=1e-3, dt=1e-3, config=82, bcz=bcz)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    r = O.project_vc(g, spec.rho_l, spec.rho_g, spec.dt, c.phi, c.u, c.v, c.w)
    U = np.sqrt((np.sum(c.u ** 2) + np.sum(c.v ** 2) + np.sum(c.w ** 2)) / (3 * c.u.size))
    assert r["relres"] < 1e-11
    assert r["divmax"] * c.dx / U < 1e-10
    assert np.max(np.abs(O.div(g, r["u"], r["v"], r["w"]))) * c.dx / U < 1e-10
    rho = spec.rho_g + c.phi * (spec.rho_l - spec.rho_g)
    gp = O.grad(g, r["p"])
    nbr = [np.roll(rho, -1, axis=2), np.roll(rho, -1, axis=1), np.roll(rho, -1, axis=0)]
    for a, (key, ust) in enumerate((("u", c.u), ("v", c.v), ("w", c.w))):
        bf = 2.0 / (rho + nbr[a])
        lhs = ust - r[key]
        mask = np.ones(g.shape, bool)
        if a == 1:
            mask[:, -1, :] = False
        if a == 2 and bcz == 1:
            mask[-1] = False
        rhs = spec.dt * bf * gp[a]
        assert np.max(np.abs(lhs[mask] - rhs[mask])) < 1e-10 * np.max(np.abs(rhs[mask])), key


def test_vc_layered_closed_form():
    """Density and u* depending on z only, walls in z: the face fluxes of the
    exact projection vanish, so u = 0 and p_(k+1) - p_k =
    dzc_(k+1/2) w*_(k+1/2) / (dt beta_(k+1/2))."""
    nx, ny, nz = 4, 3, 10
    zf = I.z_faces(nz, 1.0, 1.4)
    zc = 0.5 * (zf[:-1] + zf[1:])
    g = O.Grid(nx, ny, nz, 0.25, 1 / 3, zf, 0, 0, 1)
    phi = np.broadcast_to((0.5 * (1 + np.tanh((0.3 - np.abs(zc - 0.5)) / 0.05)))[:, None, None],
                          g.shape).copy()
    ws = np.broadcast_to(np.sin(2 * np.pi * zf[1:])[:, None, None], g.shape).copy()
    ws[-1] = 0.0
    z0 = np.zeros(g.shape)
    rho_l, rho_g, dt = 1.0, 1e-2, 1e-3
    r = O.project_vc(g, rho_l, rho_g, dt, phi, z0, z0, ws)
    for k in "uvw":  # zero up to the round-off of the dense solve
        assert np.max(np.abs(r[k])) < 1e-12 * np.max(np.abs(ws)), k
    rho = rho_g + phi[:, 0, 0] * (rho_l - rho_g)
    beta = 2.0 / (rho[:-1] + rho[1:])
    dp = np.diff(zc) * ws[:-1, 0, 0] / (dt * beta)
    p = np.concatenate([[0.0], np.cumsum(dp)])
    p -= np.sum(np.diff(zf) * p) / np.sum(np.diff(zf))
    assert relerr(r["p"][:, 1, 2], p) < 1e-12


@pytest.mark.parametrize("bcz", [1, 0])
def test_vc_is_the_split_fixed_point(bcz):
    """The split projection with phat = p equals the unsplit one: if p solves
    D(beta_f G p) = D(u*)/dt, then with p^n = p^(n-1) = p (so phat = p) the
    split right-hand side (rho0/dt) D u* + D[(1 - rho0 beta_f) G p] equals
    D G p (multiply the unsplit equation by rho0 and add D G p to both sides),
    so the split solve returns p and the same u.  This ties the two oracle
    paths to each other at density ratio 1000."""
    spec = I.CaseSpec(nx=12, ny=10, nz=9, bcx=1, beta=1.4, n_bubbles=2, radius_cells=2.0,
                      rho_l=1.0, rho_g=1e-3, dt=1e-3, config=83, bcz=bcz)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    r = O.project_vc(g, spec.rho_l, spec.rho_g, spec.dt, c.phi, c.u, c.v, c.w)
    s = O.project(g, spec.rho_l, spec.rho_g, spec.dt, c.phi, r["p"], r["p"], c.u, c.v, c.w)
    assert relerr(s["p"], r["p"]) < 1e-10
    for k in "uvw":
        assert relerr(s[k], r[k]) < 1e-10, k


# --------------------------------------------------------------------------
# ACDI phase-field transport (Jain 2022), conservative face-flux form
# --------------------------------------------------------------------------
def _acdi_case(bcx, bcy, bcz, beta, config, noise=0.0):
    spec = I.CaseSpec(nx=14, ny=12, nz=10, bcx=bcx, bcy=bcy, bcz=bcz, beta=beta, n_bubbles=2,
                      radius_cells=3.0, noise=noise, config=config)
    return spec, I.make_case(spec)


@pytest.mark.parametrize("bcx,bcy,bcz,beta", [(0, 0, 1, 0.0), (1, 0, 1, 1.5), (0, 1, 0, 1.2),
                                              (1, 1, 0, 0.0)])
def test_acdi_conserves_mass(bcx, bcy, bcz, beta):
    """The face-flux form telescopes: sum_c dV_c rhs_c = 0 (walls carry no
    flux, periodic faces appear twice with opposite signs)."""
    spec, c = _acdi_case(bcx, bcy, bcz, beta, 84, noise=0.1)
    g = O.Grid.of_case(c)
    r = O.acdi_rhs(g, c.dx, 1.3, c.phi, c.u, c.v, c.w)
    dv = np.diff(c.zf)[:, None, None] * c.dx * c.dy
    assert abs(np.sum(dv * r)) <= 1e-13 * np.sum(np.abs(dv * r))
    assert np.max(np.abs(r)) > 0


@pytest.mark.parametrize("bcz", [1, 0])
def test_acdi_central_advection_conserves_phi_squared(bcz):
    """Gamma = 0 and a discretely divergence-free u (the staggered curl of
    the input recipe): sum_c dV phi rhs = -1/2 sum_c dV phi^2 D u = 0."""
    spec, c = _acdi_case(0, 1, bcz, 1.3, 85)
    g = O.Grid.of_case(c)
    assert np.max(np.abs(O.div(g, c.u, c.v, c.w))) < 1e-10 * np.max(np.abs(c.u)) / c.dx
    phi = np.random.default_rng(3).uniform(0.05, 0.95, g.shape)
    r = O.acdi_rhs(g, c.dx, 0.0, phi, c.u, c.v, c.w)
    dv = np.diff(c.zf)[:, None, None]
    assert abs(np.sum(dv * phi * r)) <= 1e-12 * np.sum(np.abs(dv * phi * r))
    # and a constant phi does not move
    r0 = O.acdi_rhs(g, c.dx, 0.0, np.full(g.shape, 0.3), c.u, c.v, c.w)
    assert np.max(np.abs(r0)) <= 1e-10 * np.max(np.abs(c.u)) / c.dx


def test_acdi_equilibrium_profile_second_order():
    """u = 0 and the kernel profile phi = 1/2 (1 + tanh((x - x0)/(2 eps))):
    psi is then the signed distance x - x0, |n| = 1 and the diffusive and
    sharpening fluxes cancel in the continuum, so the discrete rhs is pure
    truncation error.  Halving dx at fixed eps divides it by about 4."""
    eps, x0 = 0.04, 0.5 + 1e-3
    errs = []
    for nx in (64, 128, 256):
        dx = 1.0 / nx
        g = O.Grid(nx, 2, 2, dx, dx, np.array([0.0, dx, 2 * dx]), I.NEUMANN, I.PERIODIC, I.PERIODIC)
        xc = (np.arange(nx) + 0.5) * dx
        phi = np.broadcast_to(0.5 * (1 + np.tanh((xc - x0) / (2 * eps))), g.shape).copy()
        z = np.zeros(g.shape)
        r = O.acdi_rhs(g, eps, 1.0, phi, z, z, z)
        errs.append(np.max(np.abs(r)))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs
    # a profile of the wrong width is not in equilibrium
    g = O.Grid(128, 2, 2, 1 / 128, 1 / 128, np.array([0.0, 1 / 128, 2 / 128]), I.NEUMANN, 0, 0)
    xc = (np.arange(128) + 0.5) / 128
    phi = np.broadcast_to(0.5 * (1 + np.tanh((xc - x0) / (4 * eps))), g.shape).copy()
    z = np.zeros(g.shape)
    assert np.max(np.abs(O.acdi_rhs(g, eps, 1.0, phi, z, z, z))) > 30 * errs[1]


def test_acdi_axis_swap_symmetry():
    """On a square x-y grid, swapping x and y (and u with v) swaps the rhs."""
    spec = I.CaseSpec(nx=12, ny=12, nz=8, bcx=1, bcy=1, beta=1.2, n_bubbles=2, radius_cells=2.5,
                      config=86, noise=0.05)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    r = O.acdi_rhs(g, c.dx, 0.8, c.phi, c.u, c.v, c.w)
    sw = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 2))
    r2 = O.acdi_rhs(g, c.dx, 0.8, sw(c.phi), sw(c.v), sw(c.u), sw(c.w))
    assert relerr(r2, sw(r)) < 1e-13


@pytest.mark.parametrize("bc", [I.NEUMANN, I.PERIODIC])
def test_acdi_x_z_swap_symmetry(bc):
    """On a uniform cubic grid with the same boundary in x and z, swapping
    the x and z axes (and u with w) swaps the rhs: the z code (wall mirror
    with its ghost centre, the periodic seam, centre distances from the
    z tables) is pinned to the x code."""
    n = 10
    spec = I.CaseSpec(nx=n, ny=8, nz=n, bcx=bc, bcy=I.PERIODIC, bcz=bc, n_bubbles=2,
                      radius_cells=2.5, config=87, noise=0.05)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    assert np.allclose(np.diff(c.zf), c.dx, rtol=0, atol=1e-15)
    r = O.acdi_rhs(g, c.dx, 0.9, c.phi, c.u, c.v, c.w)
    sw = lambda a: np.ascontiguousarray(np.swapaxes(a, 0, 2))
    g2 = O.Grid(n, 8, n, c.dx, c.dy, c.zf, bc, I.PERIODIC, bc)
    r2 = O.acdi_rhs(g2, c.dx, 0.9, sw(c.phi), sw(c.w), sw(c.v), sw(c.u))
    assert relerr(r2, sw(r)) < 1e-12


# An independent numpy restatement of the ACDI right-hand side (Jain 2022's
# model in the conservative face-flux form read by the oracle), written with
# whole-array shifts instead of the oracle's loops.  form = "tanh" evaluates
# 1 - tanh^2((psi_a + psi_b)/(4 eps)) directly; form = "S" uses the identity
# 1 - tanh^2 x = 4 S/(1 + S)^2 with S = sqrt(r_a) sqrt(r_b) = e^(2x), the form
# the GPU kernels evaluate.
def _acdi_rhs_numpy(c, eps, gam, phi, u, v, w, form="tanh", delta=1e-100):
    s = c.spec
    nz, ny, nx = phi.shape
    a = np.maximum(phi + delta, delta)
    b = np.maximum(1.0 - phi + delta, delta)
    r = a / b
    psi = eps * np.log(r)
    q = np.sqrt(r)
    zf = np.asarray(c.zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzf = np.diff(zf)
    lz = zf[-1] - zf[0]

    def nb(arr, axis, step, periodic):
        """Neighbour along axis (step +1 or -1); a wall mirrors the cell."""
        out = np.roll(arr, -step, axis=axis)
        if not periodic:
            idx = [slice(None)] * 3
            idx[axis] = -1 if step > 0 else 0
            out[tuple(idx)] = arr[tuple(idx)]
        return out

    px, py, pz = s.bcx == I.PERIODIC, s.bcy == I.PERIODIC, s.bcz == I.PERIODIC
    gx = (nb(psi, 2, 1, px) - nb(psi, 2, -1, px)) / (2 * c.dx)
    gy = (nb(psi, 1, 1, py) - nb(psi, 1, -1, py)) / (2 * c.dy)
    zhi = np.append(zc[1:], zc[0] + lz if pz else 2 * zf[-1] - zc[-1])
    zlo = np.insert(zc[:-1], 0, zc[-1] - lz if pz else 2 * zf[0] - zc[0])
    gz = (nb(psi, 0, 1, pz) - nb(psi, 0, -1, pz)) / (zhi - zlo)[:, None, None]
    mag = np.sqrt(gx * gx + gy * gy + gz * gz)
    safe = np.where(mag > 0, mag, 1.0)
    n = [np.where(mag > 0, gg / safe, 0.0) for gg in (gx, gy, gz)]
    # centre distance across each +z face (the seam for periodic z)
    hz = np.append(np.diff(zc), zc[0] + lz - zc[-1])

    def face(axis, vel, h, periodic, nn):
        pb, sb, qb, nbv = (np.roll(t, -1, axis=axis) for t in (phi, psi, q, nn))
        if form == "tanh":
            t = np.tanh((psi + sb) / (4 * eps))
            k = 1.0 - t * t
        else:
            S = q * qb
            k = 4 * S / ((1 + S) * (1 + S))
        F = vel * 0.5 * (phi + pb) - gam * (eps * (pb - phi) / h - 0.25 * k * 0.5 * (nn + nbv))
        if not periodic:
            idx = [slice(None)] * 3
            idx[axis] = -1
            F[tuple(idx)] = 0.0
        return F

    Fx = face(2, u, c.dx, px, n[0])
    Fy = face(1, v, c.dy, py, n[1])
    Fz = face(0, w, hz[:, None, None], pz, n[2])
    west = np.roll(Fx, 1, axis=2)
    south = np.roll(Fy, 1, axis=1)
    below = np.roll(Fz, 1, axis=0)
    if not px:
        west[:, :, 0] = 0.0
    if not py:
        south[:, 0, :] = 0.0
    if not pz:
        below[0] = 0.0
    return -((Fx - west) / c.dx + (Fy - south) / c.dy + (Fz - below) / dzf[:, None, None])


ACDI_FLOOR_CASES = [(0, 0, 1, 0.0, 88), (1, 0, 1, 1.5, 89), (0, 1, 0, 1.2, 90), (1, 1, 0, 0.0, 91)]


@pytest.mark.parametrize("bcx,bcy,bcz,beta,config", ACDI_FLOOR_CASES)
def test_acdi_matches_numpy_restatement(bcx, bcy, bcz, beta, config):
    """The oracle's loops against the whole-array numpy restatement (same
    tanh form): independent code for the normals, the wall mirrors, the
    seam and the face fluxes agrees to a few ulps of max|rhs|."""
    spec, c = _acdi_case(bcx, bcy, bcz, beta, config, noise=0.1)
    g = O.Grid.of_case(c)
    r = O.acdi_rhs(g, c.dx, 1.3, c.phi, c.u, c.v, c.w)
    ref = _acdi_rhs_numpy(c, c.dx, 1.3, c.phi, c.u, c.v, c.w, form="tanh")
    assert relerr(r, ref) < 2e-14


def acdi_form_floor(c, eps, gam, phi, u, v, w):
    """Spread, relative to max|rhs|, between two FP64 evaluations of the same
    discrete rhs that differ only in how 1 - tanh^2 is formed (the tanh of
    the oracle, the S form of the GPU): the rounding floor any FP64
    implementation of the S form sits at against the oracle."""
    a = _acdi_rhs_numpy(c, eps, gam, phi, u, v, w, form="tanh")
    b = _acdi_rhs_numpy(c, eps, gam, phi, u, v, w, form="S")
    return relerr(b, a)


def test_acdi_form_floor_is_measured():
    """The floor of the S form against the tanh form on the GPU parity
    recipes: both are FP64-exact readings of the same formula, yet they
    differ by the rounding of tanh near +-1, amplified by the division by
    h (the sharpening flux is O(1) while rhs = -D F is O(1/h)).  The floor
    must stay well below the GPU parity bar of 1e-12 (measured: under
    8e-16 on these recipes)."""
    worst = 0.0
    for spec in (I.CaseSpec(nx=32, ny=32, nz=32, n_bubbles=3, radius_cells=5, config=100),
                 I.CaseSpec(nx=48, ny=36, nz=20, bcx=1, beta=1.5, n_bubbles=3, radius_cells=4,
                            config=101)):
        c = I.make_case(spec)
        worst = max(worst, acdi_form_floor(c, c.dx, 1.5, c.phi, c.u, c.v, c.w))
    assert worst < 5e-15, worst


def test_acdi_phi_outside_unit_interval_stays_finite():
    """A phi pushed slightly outside [0, 1] (central advection undershoots
    where Gamma < max|u|) and a few points far outside: the bounded quotient
    keeps psi, the normals and the fluxes finite, and the face-flux form
    still conserves mass.  Inside [0, 1] the bounds change nothing: the
    rhs equals the unbounded numpy form there."""
    spec, c = _acdi_case(1, 0, 1, 1.3, 92, noise=0.1)
    g = O.Grid.of_case(c)
    inside = O.acdi_rhs(g, c.dx, 0.7, c.phi, c.u, c.v, c.w)
    assert np.all(np.isfinite(inside))
    rng = np.random.default_rng(7)
    phi = c.phi + rng.uniform(-2e-3, 2e-3, g.shape)
    flat = phi.reshape(-1)
    flat[rng.choice(flat.size, 6, replace=False)] = [-0.4, -1e-12, 1.0 + 1e-12, 1.5, -3.0, 4.0]
    r = O.acdi_rhs(g, c.dx, 0.7, phi, c.u, c.v, c.w)
    assert np.all(np.isfinite(r))
    dv = np.diff(c.zf)[:, None, None] * c.dx * c.dy
    assert abs(np.sum(dv * r)) <= 1e-13 * np.sum(np.abs(dv * r))
    assert relerr(r, _acdi_rhs_numpy(c, c.dx, 0.7, phi, c.u, c.v, c.w)) < 2e-14
    # the unbounded quotient would give NaN here
    with np.errstate(invalid="ignore"):
        assert np.isnan(np.log((phi + 1e-100) / (1 - phi + 1e-100))).any()


# --------------------------------------------------------------------------
# The Poisson solve with Dirichlet and mixed x/y boundary kinds (bc 2: p = 0
# on both boundary faces; 3: Neumann near, Dirichlet far; 4: Dirichlet near,
# Neumann far), the boundary kinds of the CaNS fast solver
# --------------------------------------------------------------------------
def _poisson_golden():
    return sorted(glob.glob(os.path.join(GOLDEN, "poisson_*.json")))


@pytest.mark.parametrize("path", _poisson_golden(), ids=lambda p: os.path.basename(p))
@pytest.mark.parametrize("dense", [False, True])
def test_poisson_bc_matches_exact_rational(path, dense):
    d = json.load(open(path))
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    shape = (nz, ny, nx)
    zf = np.array([float(Q(z)) for z in d["zf"]])
    g = O.Grid(nx, ny, nz, float(Q(d["dx"])), float(Q(d["dy"])), zf, d["bcx"], d["bcy"], d["bcz"])
    f = np.array(d["inputs"]["f"]).reshape(shape)
    p = O.poisson(g, f, dense=dense)
    assert relerr(p, np.array(d["expected"]["p"]).reshape(shape)) < 1e-13


def _mode_bc(n, h, m, bc):
    """Closed-form eigenvector of the second difference of kind bc at the
    cell centres, and its eigenvalue."""
    x = np.arange(n) + 0.5
    if bc == 2:    # p = 0 on both faces: sin(pi (m+1) x / n)
        return np.sin(np.pi * (m + 1) * x / n), -4 / h ** 2 * np.sin(np.pi * (m + 1) / (2 * n)) ** 2
    if bc == 3:    # zero flux near, p = 0 far: cos(pi (m + 1/2) x / n)
        return np.cos(np.pi * (m + 0.5) * x / n), -4 / h ** 2 * np.sin(np.pi * (m + 0.5) / (2 * n)) ** 2
    if bc == 4:    # p = 0 near, zero flux far: sin(pi (m + 1/2) x / n)
        return np.sin(np.pi * (m + 0.5) * x / n), -4 / h ** 2 * np.sin(np.pi * (m + 0.5) / (2 * n)) ** 2
    if bc == 1:
        return np.cos(np.pi * m * x / n), -4 / h ** 2 * np.sin(np.pi * m / (2 * n)) ** 2
    i = np.arange(n)
    return np.cos(2 * np.pi * m * i / n), -4 / h ** 2 * np.sin(np.pi * m / n) ** 2


@pytest.mark.parametrize("bcx,bcy,bcz", [(2, 0, 1), (3, 2, 1), (4, 1, 1), (2, 3, 0), (1, 4, 0),
                                         (3, 3, 1), (4, 4, 0), (2, 2, 1)])
def test_poisson_bc_eigenmodes_closed_form(bcx, bcy, bcz):
    """Products of closed-form eigenvectors are solved exactly (to round-off)
    by both oracle paths, and L_h maps them to lambda times themselves."""
    nx, ny, nz = 12, 9, 8
    dx, dy, lz = 1.0 / nx, 0.7 / ny, 1.3
    g = O.Grid(nx, ny, nz, dx, dy, uniform_zf(nz, lz), bcx, bcy, bcz)
    for mx, my, mz in ((0, 0, 0), (0, 1, 0), (3, 2, 1), (nx - 1, ny - 1, nz - 1), (5, 4, 2)):
        qx, lx = _mode_bc(nx, dx, mx, bcx)
        qy, ly = _mode_bc(ny, dy, my, bcy)
        if bcz == 1:
            qz, lzv = _mode_bc(nz, lz / nz, mz, 1)
        else:
            qz, lzv = _mode_bc(nz, lz / nz, mz, 0)
        q = qz[:, None, None] * qy[None, :, None] * qx[None, None, :]
        lam = lx + ly + lzv
        if lam == 0:
            continue
        f = lam * q
        assert relerr(O.apply_L(g, q), f) < 1e-13
        for dense in (False, True):
            assert relerr(O.poisson(g, f, dense=dense), q) < 1e-12, (mx, my, mz, dense)


def _lap1d_bc(n, h, bc):
    """Dense second-difference matrix of one direction from its ghost rules
    (numpy; independent of the oracle's loops)."""
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] -= 2
        for s in (-1, 1):
            j = i + s
            if 0 <= j < n:
                A[i, j] += 1
            elif bc == 0:
                A[i, j % n] += 1
            else:
                side = 0 if j < 0 else 1
                dirichlet = bc == 2 or (bc == 3 and side == 1) or (bc == 4 and side == 0)
                A[i, i] += -1 if dirichlet else 1
    return A / h ** 2


@pytest.mark.parametrize("bcx,bcy", [(2, 0), (3, 1), (4, 2), (2, 4), (3, 3)])
def test_poisson_bc_operator_and_solve_match_numpy_assembly(bcx, bcy):
    """The operator against a Kronecker-sum assembly of 1-D matrices built
    from the ghost rules, and both oracle solves against numpy's dense solve
    of that matrix (a non-singular system: no gauge)."""
    nx, ny, nz = 6, 5, 4
    dx, dy, dz = 0.3, 0.25, 0.2
    g = O.Grid(nx, ny, nz, dx, dy, uniform_zf(nz, nz * dz), bcx, bcy, I.NEUMANN)
    Ax, Ay, Az = _lap1d_bc(nx, dx, bcx), _lap1d_bc(ny, dy, bcy), _lap1d_bc(nz, dz, 1)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    L = np.kron(Iz, np.kron(Iy, Ax)) + np.kron(Iz, np.kron(Ay, Ix)) + np.kron(Az, np.kron(Iy, Ix))
    rng = np.random.default_rng(bcx * 10 + bcy)
    q = rng.standard_normal((nz, ny, nx))
    assert relerr(O.apply_L(g, q), (L @ q.ravel()).reshape(q.shape)) < 1e-14
    f = rng.standard_normal((nz, ny, nx))
    ref = np.linalg.solve(L, f.ravel()).reshape(f.shape)
    for dense in (False, True):
        assert relerr(O.poisson(g, f, dense=dense), ref) < 1e-12


@pytest.mark.parametrize("bcx,bcy,bcz,beta", [(2, 0, 1, 1.4), (3, 4, 0, 0.0), (4, 2, 1, 1.2),
                                              (1, 3, 0, 1.1)])
def test_poisson_bc_apply_then_solve(bcx, bcy, bcz, beta):
    """f := L_h q for a random q on stretched and periodic z: the solve
    returns q itself (p is unique with a Dirichlet face, no gauge)."""
    nx, ny, nz = 12, 8, 10
    zf = I.z_faces(nz, 1.0, beta)
    g = O.Grid(nx, ny, nz, 1.0 / nx, 0.8 / ny, zf, bcx, bcy, bcz)
    q = np.random.default_rng(5 + bcx).standard_normal(g.shape)
    f = O.apply_L(g, q)
    assert relerr(O.poisson(g, f), q) < 1e-12
    assert relerr(O.poisson(g, f, dense=True), q) < 1e-12


def test_poisson_bc_one_dimensional_against_scipy_transforms():
    """A right-hand side constant in y and in z (periodic y, walls in z)
    reduces the solve to one x-line: p = T^-1 [T(f) / lambda] with T scipy's
    DST-II (p = 0 on both faces), DCT-IV (zero flux near, p = 0 far) or
    DST-IV (p = 0 near, zero flux far), an independent library routine."""
    import scipy.fft as sf
    nx, ny, nz, dx = 16, 4, 3, 1.0 / 16
    f1 = np.random.default_rng(9).standard_normal(nx)
    f = np.broadcast_to(f1, (nz, ny, nx)).copy()
    m = np.arange(nx)
    for bc, kind, fwd, inv, lam in (
            (2, "dst", 2, 3, -4 / dx ** 2 * np.sin(np.pi * (m + 1) / (2 * nx)) ** 2),
            (3, "dct", 4, 4, -4 / dx ** 2 * np.sin(np.pi * (m + 0.5) / (2 * nx)) ** 2),
            (4, "dst", 4, 4, -4 / dx ** 2 * np.sin(np.pi * (m + 0.5) / (2 * nx)) ** 2)):
        T = getattr(sf, kind)
        ref = T(T(f1, type=fwd, norm="ortho") / lam, type=inv, norm="ortho")
        g = O.Grid(nx, ny, nz, dx, 0.25, uniform_zf(nz), bc, I.PERIODIC, I.NEUMANN)
        p = O.poisson(g, f)
        assert relerr(p[1, 2], ref) < 1e-13, bc
        assert relerr(p, np.broadcast_to(ref, p.shape)) < 1e-13
