"""Variable-coefficient projection without splitting on the GPU
(fizzy_proj_solve_vc) against the FP64 CPU oracle (needs a B300).

D(beta_f G p) = D(u*)/dt is the pressure equation that the constant-
coefficient splitting replaces; the library solves it by conjugate gradients
preconditioned with its own FFT/tridiagonal solve.  Stopped at
max|r| / max|b| <= 1e-12, the solution carries an error of about the
condition number times that residual; the bar is 1e-9 relative for p and u
(the mixed mode's bar) and max|D u| dx / U <= 1e-10, against the oracle's
dense solve of the same system (grids of at most 4096 cells).
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import gpu_project, relerr, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-9
P = I.PERIODIC


def cases():
    return {
        "v16x16x12_ratio1000": I.CaseSpec(nx=16, ny=16, nz=12, n_bubbles=2, radius_cells=2.5,
                                          config=90, velocity="iid"),
        "v24x12x14_nx_stretch_ratio10": I.CaseSpec(nx=24, ny=12, nz=14, bcx=1, beta=1.5, n_bubbles=2,
                                                   radius_cells=2.5, rho_l=1.0, rho_g=0.1, config=91),
        "v12x18x16_ny_periodic_z": I.CaseSpec(nx=12, ny=18, nz=16, bcy=1, n_bubbles=2, radius_cells=2.5,
                                              config=92, bcz=P),
        "v18x12x16_swapped_stretch_pz": I.CaseSpec(nx=18, ny=12, nz=16, beta=1.2, n_bubbles=2,
                                                   radius_cells=2.5, rho_l=1e-3, rho_g=1.0, config=93,
                                                   bcz=P),
        "v27x9x16_nn": I.CaseSpec(nx=27, ny=9, nz=16, bcx=1, bcy=1, n_bubbles=1, radius_cells=2.5,
                                  rho_l=1.0, rho_g=0.02, config=94),
    }


CASES = cases()


def gpu_vc(case, max_iter=2000, tol=1e-12, precision=F.FP64):
    import torch
    plan = F.Plan.for_case(case, precision=precision)
    u, v, w = to_dev(case.u), to_dev(case.v), to_dev(case.w)
    p = torch.empty_like(u)
    st = plan.solve_vc(to_dev(case.phi), u, v, w, p, max_iter=max_iter, tol=tol)
    torch.cuda.synchronize()
    plan.close()
    return dict(p=p.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy(), stats=st)


@pytest.mark.parametrize("precision", [F.FP64, F.MIXED], ids=["fp64_precond", "fp32_precond"])
@pytest.mark.parametrize("name", list(CASES))
def test_vc_matches_dense_oracle(cuda_ok, name, precision):
    """FP64 plans precondition with the FP64 solve, mixed plans with the FP32
    solve (flexible CG); both reach the same FP64 residual bar."""
    c = I.make_case(CASES[name])
    s = c.spec
    g = O.Grid.of_case(c)
    ref = O.project_vc(g, s.rho_l, s.rho_g, s.dt, c.phi, c.u, c.v, c.w)
    got = gpu_vc(c, precision=precision)
    st = got["stats"]
    assert st["converged"] == 1 and st["relres"] <= 1e-12, st
    pg = got["p"] - O.weighted_mean(g, got["p"])
    assert relerr(pg, ref["p"]) <= TOL
    ug = np.concatenate([got[k].ravel() for k in "uvw"])
    ur = np.concatenate([ref[k].ravel() for k in "uvw"])
    assert relerr(ug, ur) <= TOL
    assert st["div_metric"] <= 1e-10, st


def test_vc_constant_density_is_the_split_projection(cuda_ok):
    """rho_l = rho_g: the splitting is exact, the preconditioner is the exact
    inverse up to the factor rho, and one CG step solves the system."""
    spec = I.CaseSpec(nx=48, ny=36, nz=20, bcx=1, beta=1.5, n_bubbles=3, radius_cells=4, rho_l=0.5,
                      rho_g=0.5, dt=1e-3, config=95)
    c = I.make_case(spec)
    a = gpu_vc(c)
    b = gpu_project(c, F.FP64)
    assert a["stats"]["iterations"] == 1
    g = O.Grid.of_case(c)
    pa = a["p"] - O.weighted_mean(g, a["p"])
    pb = b["p"] - O.weighted_mean(g, b["p"])
    assert relerr(pa, pb) < 1e-11
    for k in "uvw":
        assert relerr(a[k], b[k]) < 1e-11, k


@pytest.mark.parametrize("precision", [F.FP64, F.MIXED], ids=["fp64_precond", "fp32_precond"])
@pytest.mark.parametrize("bcz", [I.NEUMANN, P])
def test_vc_properties_at_64(cuda_ok, bcz, precision):
    """64^3, density ratio 1000: through the oracle's O(N) operators, the
    GPU's p solves D(beta_f G p) = D(u*)/dt to the reported relres, u is
    divergence-free and u = u* - dt beta_f G p face by face."""
    spec = I.CaseSpec(nx=64, ny=64, nz=64, n_bubbles=6, radius_cells=5, config=96, bcz=bcz)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    got = gpu_vc(c, max_iter=3000, tol=1e-11, precision=precision)
    st = got["stats"]
    assert st["converged"] == 1
    b = O.div(g, c.u, c.v, c.w) / spec.dt
    r = b - O.apply_vc(g, spec.rho_l, spec.rho_g, c.phi, got["p"])
    assert np.max(np.abs(r)) / np.max(np.abs(b)) <= 2e-11
    U = np.sqrt((np.sum(c.u ** 2) + np.sum(c.v ** 2) + np.sum(c.w ** 2)) / (3 * c.u.size))
    assert np.max(np.abs(O.div(g, got["u"], got["v"], got["w"]))) * c.dx / U <= 1e-10
    rho = spec.rho_g + c.phi * (spec.rho_l - spec.rho_g)
    gp = O.grad(g, got["p"])
    nbr = [np.roll(rho, -1, axis=2), np.roll(rho, -1, axis=1), np.roll(rho, -1, axis=0)]
    for a, (key, ust) in enumerate((("u", c.u), ("v", c.v), ("w", c.w))):
        mask = np.ones(g.shape, bool)
        if a == 2 and bcz == I.NEUMANN:
            mask[-1] = False
        rhs = spec.dt * (2.0 / (rho + nbr[a])) * gp[a]
        assert np.max(np.abs((ust - got[key])[mask] - rhs[mask])) <= 1e-11 * np.max(np.abs(rhs)), key


def test_vc_not_converged_is_reported(cuda_ok):
    import torch
    c = I.make_case(CASES["v16x16x12_ratio1000"])
    plan = F.Plan.for_case(c, precision=F.FP64)
    u, v, w = to_dev(c.u), to_dev(c.v), to_dev(c.w)
    p = torch.empty_like(u)
    with pytest.raises(F.FizzyError) as e:
        plan.solve_vc(to_dev(c.phi), u, v, w, p, max_iter=3, tol=1e-14)
    assert e.value.code == -5
    plan.close()


@pytest.mark.parametrize("bcz", [I.NEUMANN, P])
def test_vc_is_the_split_fixed_point_on_the_gpu(cuda_ok, bcz):
    """Density ratio 1000, 96 x 64 x 48: the GPU's split projection, given
    p^n = p^(n-1) = the GPU's unsplit p (so phat = p), returns that p and the
    same u (the split right-hand side is then exactly D G p).  The unsplit
    solve stops at relres 1e-12, so both agree to about the condition number
    times that: bar 1e-8."""
    import torch
    spec = I.CaseSpec(nx=96, ny=64, nz=48, beta=1.3, n_bubbles=5, radius_cells=4, config=97, bcz=bcz)
    c = I.make_case(spec)
    a = gpu_vc(c, max_iter=3000, tol=1e-12)
    c2 = I.make_case(spec)
    c2.pn = a["p"].copy()
    c2.pnm1 = a["p"].copy()
    b = gpu_project(c2, F.FP64)
    g = O.Grid.of_case(c)
    pa = a["p"] - O.weighted_mean(g, a["p"])
    pb = b["p"] - O.weighted_mean(g, b["p"])
    assert relerr(pb, pa) < 1e-8
    ua = np.concatenate([a[k].ravel() for k in "uvw"])
    ub = np.concatenate([b[k].ravel() for k in "uvw"])
    assert relerr(ub, ua) < 1e-8
