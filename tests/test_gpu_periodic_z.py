"""Periodic z on the GPU against the FP64 CPU oracle (needs a B300).

Triperiodic boxes are the setting of the paper's emulsion in homogeneous
isotropic turbulence ("Numerical experiments"; its weak-scaling test).  With
periodic z every (kx, ky) z-line is a cyclic tridiagonal system, solved by
the Sherman-Morrison form of the z-sweep (k_thomas_cyc), and the seam face
nz-1/2 joins plane nz-1 to plane 0 in the flux, divergence, residual and
correction kernels.  Same bars as the wall-bounded cases: max relative error
<= 1e-12 (FP64) and <= 1e-9 (mixed, relres <= 1e-10), max|D u| dx / U <= 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import compare, gpu_project, relerr, run_alone, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-9
P = I.PERIODIC


def cases():
    return {
        # uniform triperiodic box, several drops
        "t32_ppp": I.CaseSpec(nx=32, ny=32, nz=32, n_bubbles=4, radius_cells=4, config=60, bcz=P),
        # walls in x, stretched periodic z (the seam between the finest cells)
        "t48x36x20_npp_stretch": I.CaseSpec(nx=48, ny=36, nz=20, bcx=1, bcy=0, beta=1.5,
                                            n_bubbles=3, radius_cells=4, config=61, bcz=P),
        # odd nx, walls in y, odd nz (a ragged last block of the z-ring)
        "t27x18x13_pnp": I.CaseSpec(nx=27, ny=18, nz=13, bcx=0, bcy=1, n_bubbles=1,
                                    radius_cells=3, config=62, bcz=P),
        # the smallest periodic z: two planes, both couplings of a row in one column
        "t16x12x2": I.CaseSpec(nx=16, ny=12, nz=2, n_bubbles=1, radius_cells=2, config=63,
                               velocity="iid", bcz=P),
        "t8x6x3_nn": I.CaseSpec(nx=8, ny=6, nz=3, bcx=1, bcy=1, n_bubbles=1, radius_cells=1.5,
                                config=64, bcz=P),
        # register-resident FP32 passes along x (128) and y (256) in mixed mode
        "t128x24x18": I.CaseSpec(nx=128, ny=24, nz=18, n_bubbles=2, radius_cells=3, config=65,
                                 bcz=P),
        "t24x256x17_wx": I.CaseSpec(nx=24, ny=256, nz=17, bcx=1, bcy=0, beta=1.2, n_bubbles=2,
                                    radius_cells=3, config=66, bcz=P),
        "t256x8x33_wy": I.CaseSpec(nx=256, ny=8, nz=33, bcx=0, bcy=1, n_bubbles=1,
                                   radius_cells=2, config=67, bcz=P),
        # light drops in a heavy phase (rho0 = rho_l)
        "t48x32x24_swapped": I.CaseSpec(nx=48, ny=32, nz=24, n_bubbles=3, radius_cells=4,
                                        rho_l=1e-3, rho_g=1.0, config=68, bcz=P),
    }


CASES = cases()


@pytest.mark.parametrize("name", list(CASES))
def test_periodic_z_fp64_matches_oracle(cuda_ok, name):
    c = I.make_case(CASES[name])
    ref = O.project_case(c)
    got = gpu_project(c, F.FP64)
    ep, eu = compare(c, got, ref)
    assert ep <= TOL64, ep
    assert eu <= TOL64, eu
    st = got["stats"]
    assert st["relres"] < 1e-11
    assert st["div_metric"] < 1e-10
    assert abs(O.weighted_mean(O.Grid.of_case(c), got["p"])) <= 1e-12 * np.max(np.abs(got["p"]))


@pytest.mark.parametrize("name", list(CASES))
def test_periodic_z_mixed_matches_oracle(cuda_ok, name):
    c = I.make_case(CASES[name])
    ref = O.project_case(c)
    got = gpu_project(c, F.MIXED)
    st = got["stats"]
    assert st["converged"] == 1 and st["relres"] <= 1e-10 and 1 <= st["iterations"] <= 4, st
    ep, eu = compare(c, got, ref)
    assert ep <= TOLMIX, ep
    assert eu <= TOLMIX, eu
    assert st["div_metric"] < 1e-10


def test_periodic_z_equal_density_closed_form(cuda_ok):
    """rho_l = rho_g and u* = s + G q with s a discrete curl: p = (rho0/dt) q
    and u = s exactly, on a stretched triperiodic grid."""
    spec = I.CaseSpec(nx=32, ny=24, nz=20, beta=1.5, n_bubbles=2, radius_cells=3, rho_l=0.5,
                      rho_g=0.5, dt=1e-3, noise=0.0, config=69, bcz=P)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    s = (c.u.copy(), c.v.copy(), c.w.copy())
    assert np.max(np.abs(O.div(g, *s))) < 1e-10 * np.max(np.abs(s[0])) / c.dx
    q = np.random.default_rng(6).standard_normal(g.shape)
    gq = O.grad(g, q)
    c.u, c.v, c.w = (s[a] + gq[a] for a in range(3))
    for prec, tol in ((F.FP64, 1e-11), (F.MIXED, 1e-9)):
        got = gpu_project(c, prec)
        p_exact = (0.5 / 1e-3) * (q - O.weighted_mean(g, q))
        assert relerr(got["p"] - O.weighted_mean(g, got["p"]), p_exact) < tol
        for a, key in enumerate("uvw"):
            assert np.max(np.abs(got[key] - s[a])) < tol * np.max(np.abs(gq[a]) + np.abs(s[a]))


def test_periodic_z_seam_rotation(cuda_ok):
    """Rotating the z spacings and every field by s planes rotates the GPU
    result (the seam is not a special plane), within the FP64 bar."""
    spec = CASES["t48x36x20_npp_stretch"]
    c = I.make_case(spec)
    a = gpu_project(c, F.FP64)
    sh = 7
    dzf = np.roll(np.diff(c.zf), sh)
    c.zf = np.concatenate([[0.0], np.cumsum(dzf)])
    for k in ("phi", "pn", "pnm1", "u", "v", "w"):
        setattr(c, k, np.roll(getattr(c, k), sh, axis=0))
    b = gpu_project(c, F.FP64)
    for k in ("u", "v", "w"):
        assert relerr(b[k], np.roll(a[k], sh, axis=0)) < TOL64, k
    g = O.Grid.of_case(c)
    pa = np.roll(a["p"], sh, axis=0)
    assert relerr(b["p"] - O.weighted_mean(g, b["p"]), pa - O.weighted_mean(g, pa)) < TOL64


@pytest.mark.parametrize("precision", [F.FP64, F.MIXED])
def test_periodic_z_in_the_batch(cuda_ok, precision):
    """Periodic-z instances in one persistent batch launch, next to a
    wall-bounded one: each equals the instance solved alone with the same
    passes (bit for bit) and the oracle within the bar."""
    specs = [CASES["t48x36x20_npp_stretch"], CASES["t27x18x13_pnp"], CASES["t16x12x2"],
             I.CaseSpec(nx=36, ny=24, nz=20, bcx=1, beta=1.2, n_bubbles=2, radius_cells=3,
                        config=70)]
    cs = [I.make_case(sp) for sp in specs]
    plans = [F.Plan.for_case(c, precision=precision) for c in cs]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch_empty(c.shape)) for c in cs]
    batch = F.Batch(plans, arrays)
    batch.solve()
    assert batch.status() == 0
    bar = TOL64 if precision == F.FP64 else TOLMIX
    for c, a, pl in zip(cs, arrays, plans):
        got = dict(p=a[6].cpu().numpy(), u=a[3].cpu().numpy(), v=a[4].cpu().numpy(),
                   w=a[5].cpu().numpy())
        alone = run_alone(c, precision)
        for k in ("p", "u", "v", "w"):
            assert np.array_equal(got[k], alone[k]), k
        ep, eu = compare(c, got, O.project_case(c))
        assert ep <= bar and eu <= bar, (ep, eu)
        if precision == F.MIXED:
            assert pl.stats()["converged"] == 1
    batch.close()
    for pl in plans:
        pl.close()


def torch_empty(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, device="cuda")


def test_emulsion_full_size_properties(cuda_ok):
    """The 256^3 triperiodic emulsion workload, in the configuration bench.py
    times (FP64 and mixed): checked through the oracle's O(N) operators, since
    its dense cyclic z-solves are too slow at this size.  The oracle's own
    right-hand side and Laplacian give relres = max|f - L p| / max|f| of the
    GPU's p; its divergence gives max|D u| of the GPU's u; its correction of
    the GPU's p gives u.  The discrete Poisson problem has one solution up to
    the gauge, so these pin the result."""
    c = I.make_case(I.emulsion256_spec())
    g = O.Grid.of_case(c)
    s = c.spec
    f = O.rhs(g, s.rho_l, s.rho_g, s.dt, c.phi, c.pn, c.pnm1, c.u, c.v, c.w)
    U = np.sqrt((np.sum(c.u ** 2) + np.sum(c.v ** 2) + np.sum(c.w ** 2)) / (3 * c.u.size))
    for prec, bar, ubar in ((F.FP64, 1e-11, TOL64), (F.MIXED, 1e-10, TOLMIX)):
        got = gpu_project(c, prec)
        r = f - O.apply_L(g, got["p"])
        assert np.max(np.abs(r)) / np.max(np.abs(f)) <= bar
        assert np.max(np.abs(O.div(g, got["u"], got["v"], got["w"]))) * c.dx / U <= 1e-10
        uo, vo, wo = O.correct(g, s.rho_l, s.rho_g, s.dt, c.phi, c.pn, c.pnm1, got["p"], c.u, c.v,
                               c.w)
        ug = np.concatenate([got[k].ravel() for k in "uvw"])
        assert relerr(ug, np.concatenate([uo.ravel(), vo.ravel(), wo.ravel()])) <= ubar
