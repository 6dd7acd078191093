"""The stand-alone Poisson solve (fizzy_poisson_solve) with every x/y
boundary kind of the CaNS solver, against the FP64 CPU oracle (needs a B300).

f := L_h q for a seeded random q, applied by the oracle.  The GPU p is
compared element by element with the oracle's solve of the same f (1e-12 in
FP64, 1e-9 after mixed refinement to relres <= 1e-10) and with q itself
(the discrete solution, up to the gauge when no Dirichlet face bounds x or
y).  Grids span several transform tiles and ragged tails, odd extents
(Dirichlet via the DST-II), the DCT-IV at n = 2 and at 512, periodic and
stretched z.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import relerr, to_dev

pytestmark = pytest.mark.gpu

D, ND, DN, N, P = F.DIRICHLET, F.NEUMANN_DIRICHLET, F.DIRICHLET_NEUMANN, F.NEUMANN, F.PERIODIC

CASES = {  # nx, ny, nz, bcx, bcy, z (walls or periodic), beta
    "dd_p_48x36x20_stretched": (48, 36, 20, D, P, N, 1.3),
    "nd_dn_64x48x17": (64, 48, 17, ND, DN, N, 0.0),
    "dn_n_48x24x16_periodic_z": (48, 24, 16, DN, N, P, 0.0),
    "d_d_36x54x12_periodic_z_stretched": (36, 54, 12, D, D, P, 1.1),
    "n_nd_96x64x10": (96, 64, 10, N, ND, N, 1.2),
    "d_p_256x64x8": (256, 64, 8, D, P, N, 0.0),
    "p_p_128x128x6_singular": (128, 128, 6, P, P, N, 1.4),
    "n_p_96x128x7_singular_periodic_z": (96, 128, 7, N, P, P, 0.0),
    "nd_p_512x8x4": (512, 8, 4, ND, P, N, 0.0),
    "d_n_27x18x13_odd": (27, 18, 13, D, N, N, 1.5),
    "nd_d_2x6x3": (2, 6, 3, ND, D, N, 0.0),
    "dn_dn_6x4x5": (6, 4, 5, DN, DN, N, 0.0),
}


def make(name):
    nx, ny, nz, bcx, bcy, bcz, beta = CASES[name]
    zf = I.z_faces(nz, 1.0, beta)
    g = O.Grid(nx, ny, nz, 1.0 / nx, 0.9 / ny, zf, bcx, bcy, bcz)
    q = np.random.default_rng(sum(map(ord, name))).standard_normal(g.shape)
    f = O.apply_L(g, q)
    return g, q, f


def singular(g):
    return g.bcx <= 1 and g.bcy <= 1


def gauge(g, a):
    return a - O.weighted_mean(g, a) if singular(g) else a


def gpu_poisson(g, f, precision):
    import torch
    plan = F.Plan(g.nx, g.ny, g.nz, g.dx, g.dy, zf=g.zf, bcx=g.bcx, bcy=g.bcy, precision=precision,
                  periodic_z=g.bcz == P)
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    st = plan.poisson(to_dev(f), p, stats=True)
    torch.cuda.synchronize()
    plan.close()
    return p.cpu().numpy(), st


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [F.FP64, F.MIXED], ids=["fp64", "mixed"])
def test_poisson_matches_oracle(cuda_ok, name, precision):
    g, q, f = make(name)
    ref = O.poisson(g, f)
    p, st = gpu_poisson(g, f, precision)
    tol = 1e-12 if precision == F.FP64 else 1e-9
    e_ref = relerr(gauge(g, p), gauge(g, ref))
    e_q = relerr(gauge(g, p), gauge(g, q))
    assert e_ref <= tol and e_q <= 10 * tol, (e_ref, e_q, st)
    assert st["relres"] <= (1e-10 if precision == F.MIXED else 1e-12), st
    if precision == F.MIXED:
        assert st["converged"] == 1 and st["iterations"] >= 1, st


def test_poisson_fp64_random_rhs_regular(cuda_ok):
    """A plain random right-hand side (no compatibility needed with a
    Dirichlet face): the GPU solve equals the oracle's."""
    g = O.Grid(72, 48, 9, 1 / 72, 1 / 48, I.z_faces(9, 1.0, 1.2), D, ND, N)
    f = np.random.default_rng(3).standard_normal(g.shape)
    p, st = gpu_poisson(g, f, F.FP64)
    assert relerr(p, O.poisson(g, f)) <= 1e-12


def test_projection_rejects_dirichlet_plans(cuda_ok):
    import torch
    plan = F.Plan(16, 16, 8, 1 / 16, 1 / 16, dz=1 / 8, bcx=D, bcy=P)
    a = torch.zeros((8, 16, 16), dtype=torch.float64, device="cuda")
    arrs = [a.clone() for _ in range(7)]
    with pytest.raises(F.FizzyError) as e:
        plan.solve(*arrs)
    assert e.value.code == -2
    plan.close()
