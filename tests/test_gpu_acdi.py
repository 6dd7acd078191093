"""ACDI phase-field step on the GPU (fizzy_acdi_step) against the FP64 CPU
oracle (needs a B300).

Element by element, rhs within 1e-12 of max|rhs|, phi + dt rhs likewise;
mass conserved to round-off on the GPU too.  The two sides form the
sharpening coefficient differently (the oracle's tanh, the kernels'
4S/(1+S)^2 with rsqrt normals); an FP64 numpy restatement measures the
spread of those two forms at under 8e-16 of max|rhs| on these recipes
(tests/test_oracle_pins.py, test_acdi_form_floor_is_measured), so 1e-12
leaves three orders of magnitude for the kernels' own rounding.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import relerr, to_dev

pytestmark = pytest.mark.gpu

P = I.PERIODIC
TOL = 1e-12


def cases():
    return {
        "a32_ppw": I.CaseSpec(nx=32, ny=32, nz=32, n_bubbles=3, radius_cells=5, config=100),
        "a48x36x20_wx_stretch": I.CaseSpec(nx=48, ny=36, nz=20, bcx=1, beta=1.5, n_bubbles=3,
                                           radius_cells=4, config=101),
        "a27x18x13_wy_pz": I.CaseSpec(nx=27, ny=18, nz=13, bcy=1, n_bubbles=2, radius_cells=3,
                                      config=102, bcz=P),
        "a48x24x16_ww_pz_stretch": I.CaseSpec(nx=48, ny=24, nz=16, bcx=1, bcy=1, beta=1.2,
                                              n_bubbles=2, radius_cells=3, config=103, bcz=P),
        "a6x4x2_iid": I.CaseSpec(nx=6, ny=4, nz=2, n_bubbles=1, radius_cells=1.5, config=104,
                                 velocity="iid"),
    }


CASES = cases()


def gpu_acdi(c, eps, gam, dt, precision=F.FP64):
    import torch
    plan = F.Plan.for_case(c, precision=precision)
    phi = to_dev(c.phi)
    rhs = torch.empty_like(phi)
    out = torch.empty_like(phi)
    plan.acdi_step(phi, to_dev(c.u), to_dev(c.v), to_dev(c.w), eps, gam, dt, rhs_out=rhs, phi_out=out)
    # in place: phi_out = phi
    plan.acdi_step(phi, to_dev(c.u), to_dev(c.v), to_dev(c.w), eps, gam, dt, phi_out=phi)
    torch.cuda.synchronize()
    plan.close()
    return rhs.cpu().numpy(), out.cpu().numpy(), phi.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_acdi_matches_oracle(cuda_ok, name):
    c = I.make_case(CASES[name])
    g = O.Grid.of_case(c)
    eps, gam, dt = c.dx, 1.5, 1e-3
    ref = O.acdi_rhs(g, eps, gam, c.phi, c.u, c.v, c.w)
    rhs, out, inplace = gpu_acdi(c, eps, gam, dt)
    assert relerr(rhs, ref) <= TOL
    step = c.phi + dt * ref
    assert np.max(np.abs(out - step)) <= TOL * dt * np.max(np.abs(ref)) + 1e-15
    assert np.array_equal(inplace, out)
    dv = np.diff(c.zf)[:, None, None]
    assert abs(np.sum(dv * rhs)) <= 1e-13 * np.sum(np.abs(dv * rhs))


def test_acdi_mixed_plan_is_fp64(cuda_ok):
    """The step is FP64 in either precision mode: a mixed plan gives the same bits."""
    c = I.make_case(CASES["a48x36x20_wx_stretch"])
    a = gpu_acdi(c, c.dx, 1.0, 1e-3, F.FP64)
    b = gpu_acdi(c, c.dx, 1.0, 1e-3, F.MIXED)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_acdi_rejects_bad_arguments(cuda_ok):
    import torch
    c = I.make_case(CASES["a6x4x2_iid"])
    plan = F.Plan.for_case(c)
    phi, u = to_dev(c.phi), to_dev(c.u)
    for kw in (dict(eps=0.0, gamma=1.0), dict(eps=1.0, gamma=-1.0)):
        with pytest.raises(F.FizzyError):
            plan.acdi_step(phi, u, u, u, kw["eps"], kw["gamma"], 0.1, phi_out=torch.empty_like(phi))
    with pytest.raises(F.FizzyError):  # no output requested
        plan.acdi_step(phi, u, u, u, 1.0, 1.0, 0.1)
    plan.close()


def test_acdi_phi_outside_unit_interval(cuda_ok):
    """phi pushed slightly outside [0, 1] (and a few points far outside):
    the bounded logarithm keeps every output finite, and the GPU still
    matches the oracle element by element."""
    c = I.make_case(CASES["a48x36x20_wx_stretch"])
    g = O.Grid.of_case(c)
    rng = np.random.default_rng(11)
    phi = c.phi + rng.uniform(-2e-3, 2e-3, g.shape)
    flat = phi.reshape(-1)
    flat[rng.choice(flat.size, 6, replace=False)] = [-0.4, -1e-12, 1.0 + 1e-12, 1.5, -3.0, 4.0]
    c.phi = phi
    eps, gam, dt = c.dx, 0.7, 1e-3
    ref = O.acdi_rhs(g, eps, gam, phi, c.u, c.v, c.w)
    rhs, out, _ = gpu_acdi(c, eps, gam, dt)
    assert np.all(np.isfinite(rhs)) and np.all(np.isfinite(out))
    assert relerr(rhs, ref) <= TOL
