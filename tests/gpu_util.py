"""Helpers shared by the GPU tests."""
import numpy as np

import oracle as O
import paper_2502_04189_b300 as F


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def gpu_project(case, precision=F.FP64, check=True, plan=None, **kw):
    """Run one projection on the GPU; returns numpy p, u, v, w and stats."""
    import torch
    own = plan is None
    if own:
        plan = F.Plan.for_case(case, precision=precision, check=check, **kw)
    phi, pn, pnm1 = to_dev(case.phi), to_dev(case.pn), to_dev(case.pnm1)
    u, v, w = to_dev(case.u), to_dev(case.v), to_dev(case.w)
    p = torch.empty_like(phi)
    st = plan.solve(phi, pn, pnm1, u, v, w, p, stats=True)
    torch.cuda.synchronize()
    out = dict(p=p.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy(), stats=st)
    if own:
        plan.close()
    return out


def relerr(a, b):
    m = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (m if m > 0 else 1.0))


def compare(case, got, ref):
    """Relative errors (spec definition) of p (gauge removed) and u."""
    g = O.Grid.of_case(case)
    pg = got["p"] - O.weighted_mean(g, got["p"])
    pr = ref["p"] - O.weighted_mean(g, ref["p"])
    ug = np.concatenate([got[k].ravel() for k in "uvw"])
    ur = np.concatenate([ref[k].ravel() for k in "uvw"])
    return relerr(pg, pr), relerr(ug, ur)


# ---- one instance solved alone, as the batched executor solves it

# register-resident FP32 passes in plain mixed solves (periodic or Neumann)
R_LENGTHS = (32, 48, 64, 96, 128, 192, 256, 384, 512)


def plain_differs(case, precision):
    s = case.spec
    return precision == F.MIXED and (s.nx in R_LENGTHS or s.ny in R_LENGTHS)


def run_plain(case, precision, **kw):
    import torch
    plan = F.Plan.for_case(case, precision=precision, **kw)
    u, v, w = to_dev(case.u), to_dev(case.v), to_dev(case.w)
    p = torch.empty_like(u)
    plan.solve(to_dev(case.phi), to_dev(case.pn), to_dev(case.pnm1), u, v, w, p)
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    return dict(p=p.cpu().numpy(), u=u.cpu().numpy(), v=v.cpu().numpy(), w=w.cpu().numpy(), stats=st)


def run_batched_alone(case, precision, **kw):
    import torch
    plan = F.Plan.for_case(case, precision=precision, **kw)
    arr = (to_dev(case.phi), to_dev(case.pn), to_dev(case.pnm1), to_dev(case.u), to_dev(case.v),
           to_dev(case.w), torch.empty(case.shape, dtype=torch.float64, device="cuda"))
    batch = F.Batch([plan], [arr])
    batch.solve()
    assert batch.status() == 0
    out = dict(p=arr[6].cpu().numpy(), u=arr[3].cpu().numpy(), v=arr[4].cpu().numpy(),
               w=arr[5].cpu().numpy(), stats=plan.stats())
    batch.close()
    plan.close()
    return out


def run_alone(case, precision, **kw):
    """The instance solved by itself with the passes the batch runs."""
    if plain_differs(case, precision):
        return run_batched_alone(case, precision, **kw)
    return run_plain(case, precision, **kw)
