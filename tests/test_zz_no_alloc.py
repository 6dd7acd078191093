"""The allocation-free entry point fizzy_proj_solve_noalloc.

It serves callers that may not allocate device memory (host codes that own
all device memory through their own pool, or that must not stall their
stream-ordered work on an allocation); it runs the FP64 projection in a static
scratch array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I
from paper_2502_04189_b300 import _abi

TOL64 = 1e-12  # the FP64 tolerance of the parity tests


def desc_of(case):
    s = case.spec
    return dict(nx=s.nx, ny=s.ny, nz=s.nz, dx=case.dx, dy=case.dy, zf=case.zf, bcx=s.bcx,
                bcy=s.bcy, rho_l=s.rho_l, rho_g=s.rho_g, dt=s.dt, precision=F.FP64)


def relerr(a, b):
    m = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (m if m > 0 else 1.0))


def test_rejects_grids_beyond_the_scratch():
    import ctypes
    d, keep = F.make_desc(nx=512, ny=512, nz=2, dx=1.0, dy=1.0, dz=1.0)
    buf = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    rc = _abi.lib().fizzy_proj_solve_noalloc(ctypes.byref(d), *([buf] * 7), None)
    assert rc == -2
    d, keep = F.make_desc(nx=64, ny=64, nz=64, dx=1.0, dy=1.0, dz=1.0, precision=F.MIXED)
    assert _abi.lib().fizzy_proj_solve_noalloc(ctypes.byref(d), *([buf] * 7), None) == -1


@pytest.mark.gpu
def test_noalloc_matches_plan_solve_twice_in_a_row(cuda_ok):
    import torch
    cases = [I.make_case(I.CaseSpec(nx=48, ny=32, nz=24, bcx=1, bcy=0, beta=1.5, n_bubbles=2,
                                    radius_cells=4, config=31)),
             I.make_case(I.CaseSpec(nx=36, ny=64, nz=20, bcx=0, bcy=1, n_bubbles=3,
                                    radius_cells=3, config=32))]

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    for case in cases:  # two calls in a row, the second on another grid
        # the existing entry point (plan-based)
        plan = F.Plan.for_case(case, precision=F.FP64)
        u1, v1, w1 = dev(case.u), dev(case.v), dev(case.w)
        p1 = torch.empty_like(u1)
        plan.solve(dev(case.phi), dev(case.pn), dev(case.pnm1), u1, v1, w1, p1)
        torch.cuda.synchronize()
        plan.close()
        # the allocation-free entry point
        u2, v2, w2 = dev(case.u), dev(case.v), dev(case.w)
        p2 = torch.empty_like(u2)
        F.solve_noalloc(dev(case.phi), dev(case.pn), dev(case.pnm1), u2, v2, w2, p2,
                        **desc_of(case))
        torch.cuda.synchronize()
        for a, b in ((p2, p1), (u2, u1), (v2, v1), (w2, w1)):
            assert relerr(a.cpu().numpy(), b.cpu().numpy()) <= TOL64


@pytest.mark.gpu
def test_noalloc_at_capacity_matches_oracle(cuda_ok):
    """Grids at the scratch limit (nx * ny * nz = FIZZY_NOALLOC_MAX_CELLS) with
    a 512-length x direction, where the generic transform path stands in for
    the plan's length-specialised one: periodic x, then walls in x (the
    DCT-II path), two calls in a row.  Each call is compared element by
    element with the FP64 oracle (p with its gauge removed, u, v, w) and with
    the plan-based solve."""
    import torch
    import oracle as O
    from gpu_util import compare

    assert 512 * 32 * 16 == _abi.NOALLOC_MAX_CELLS

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    for bcx, bcy, cfg in ((I.PERIODIC, I.NEUMANN, 33), (I.NEUMANN, I.PERIODIC, 34)):
        spec = I.CaseSpec(nx=512, ny=32, nz=16, bcx=bcx, bcy=bcy, lx=1.0, ly=32 / 512,
                          lz=16 / 512, beta=1.2, n_bubbles=3, radius_cells=4, config=cfg)
        case = I.make_case(spec)
        ref = O.project_case(case)
        u, v, w = dev(case.u), dev(case.v), dev(case.w)
        p = torch.empty_like(u)
        F.solve_noalloc(dev(case.phi), dev(case.pn), dev(case.pnm1), u, v, w, p, **desc_of(case))
        torch.cuda.synchronize()
        got = dict(p=p.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy())
        ep, eu = compare(case, got, ref)
        assert ep <= TOL64 and eu <= TOL64, (bcx, ep, eu)
        plan = F.Plan.for_case(case, precision=F.FP64)
        u1, v1, w1 = dev(case.u), dev(case.v), dev(case.w)
        p1 = torch.empty_like(u1)
        plan.solve(dev(case.phi), dev(case.pn), dev(case.pnm1), u1, v1, w1, p1)
        torch.cuda.synchronize()
        plan.close()
        for a, b in ((p, p1), (u, u1), (v, v1), (w, w1)):
            assert relerr(a.cpu().numpy(), b.cpu().numpy()) <= TOL64
