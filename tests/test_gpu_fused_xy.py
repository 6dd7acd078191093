"""Cluster-fused x-y FP32 passes (FIZZY_FLAG_FUSED_XY: mixed plans with
nx = ny = 256 or 512, periodic or wall x/y) against the separate
register-resident x and y passes they replace, and against the FP64 oracle
(needs a B300).

The fused kernels run the same transforms on the same values; only the data
movement differs (distributed shared memory in place of an HBM round trip),
so the two forms must agree bit for bit in p, u, v, w and the solve's stats.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import compare, to_dev

pytestmark = pytest.mark.gpu

P, N = I.PERIODIC, I.NEUMANN
CASES = {
    "256x256x12_pp": I.CaseSpec(nx=256, ny=256, nz=12, lz=12 / 256, n_bubbles=3, radius_cells=6,
                                config=120),
    "256x256x10_np_stretched": I.CaseSpec(nx=256, ny=256, nz=10, lz=10 / 256, bcx=N, beta=1.3,
                                          n_bubbles=2, radius_cells=5, config=121),
    "512x512x6_pn": I.CaseSpec(nx=512, ny=512, nz=6, lz=6 / 512, bcy=N, n_bubbles=2, radius_cells=4,
                               config=122),
    "512x512x5_nn": I.CaseSpec(nx=512, ny=512, nz=5, lz=5 / 512, bcx=N, bcy=N, n_bubbles=2,
                               radius_cells=4, config=123),
}


def run(case, fused):
    import torch
    plan = F.Plan.for_case(case, precision=F.MIXED, fused_xy=fused)
    u, v, w = to_dev(case.u), to_dev(case.v), to_dev(case.w)
    p = torch.empty_like(u)
    plan.solve(to_dev(case.phi), to_dev(case.pn), to_dev(case.pnm1), u, v, w, p)
    torch.cuda.synchronize()
    st = plan.stats()
    launches = plan.launches_per_solve()
    plan.close()
    return dict(p=p.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy()), st, launches


@pytest.mark.parametrize("name", list(CASES))
def test_fused_equals_separate_bit_for_bit(cuda_ok, name):
    case = I.make_case(CASES[name])
    a, sa, la = run(case, fused=True)
    b, sb, lb = run(case, fused=False)
    assert la < lb  # the fused plan launches fewer kernels per solve
    for k in "puvw":
        assert np.array_equal(a[k], b[k]), k
    assert sa == sb
    ref = O.project_case(case)
    ep, eu = compare(case, a, ref)
    assert ep <= 1e-9 and eu <= 1e-9, (ep, eu, sa)
    assert sa["converged"] == 1 and sa["relres"] <= 1e-10
