"""Serving runtime on a B300: requests admitted while others run overlap on
the device, and every served result equals the same request solved alone."""
import numpy as np
import pytest

import paper_2502_04189_b300 as F
import paper_2502_04189_b300.serve as S
from paper_2502_04189_b300 import inputs as I

from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def crop(case, desc, off):
    """The host-side equivalent of TemplateFields.fill."""
    nz, ny, nx = desc["nz"], desc["ny"], desc["nx"]
    Tz, Ty, Tx = case.phi.shape
    iz = (np.arange(nz) + off[0]) % Tz
    iy = (np.arange(ny) + off[1]) % Ty
    ix = (np.arange(nx) + off[2]) % Tx
    out = [np.ascontiguousarray(a[np.ix_(iz, iy, ix)]) for a in
           (case.phi, case.pn, case.pnm1, case.u, case.v, case.w)]
    if desc["bcx"] == 1:
        out[3][:, :, -1] = 0.0
    if desc["bcy"] == 1:
        out[4][:, -1, :] = 0.0
    out[5][-1] = 0.0
    return out


@pytest.mark.parametrize("shape,off,bcx,bcy", [
    ((40, 48, 48), (0, 0, 0), 0, 0),        # the whole template
    ((23, 17, 31), (39, 5, 47), 1, 0),      # ragged crop wrapping in every direction
    ((90, 100, 70), (7, 47, 13), 0, 1),     # larger than the template: wraps more than once
    ((1, 1, 1), (3, 4, 5), 1, 1),           # a single point: every wall face at once
])
def test_crop_fill_equals_host_crop(cuda_ok, shape, off, bcx, bcy):
    """fizzy_crop_fill is a copy: bit-identical to the host crop."""
    import torch
    tmpl = I.make_case(I.CaseSpec(nx=48, ny=48, nz=40, n_bubbles=4, radius_cells=5, config=41))
    src = [to_dev(a) for a in (tmpl.phi, tmpl.pn, tmpl.pnm1, tmpl.u, tmpl.v, tmpl.w)]
    dst = [torch.full(shape, np.nan, dtype=torch.float64, device="cuda") for _ in range(6)]
    F.crop_fill(src, dst, off, bcx, bcy)
    torch.cuda.synchronize()
    nz, ny, nx = shape
    want = crop(tmpl, dict(nz=nz, ny=ny, nx=nx, bcx=bcx, bcy=bcy), off)
    for f in range(6):
        assert np.array_equal(dst[f].cpu().numpy(), want[f]), f


@pytest.mark.parametrize("budget", [4 << 30, 12 << 20], ids=["roomy", "evicting"])
def test_served_equals_alone_and_overlaps(cuda_ok, budget):
    import torch
    tmpl = I.make_case(I.CaseSpec(nx=48, ny=48, nz=40, n_bubbles=4, radius_cells=5, config=41))
    fields = S.TemplateFields(tmpl)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(16):
        nx, ny = int(rng.choice([32, 48])), int(rng.choice([32, 48]))
        nz = int(rng.integers(16, 41))
        if i % 4 == 3:  # repeat a geometry: the plan cache must serve it
            nx, ny, nz = 32, 32, 24
        beta = float(rng.uniform(1, 2)) if i % 3 == 0 else 0.0
        bcx, bcy = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        desc = dict(nx=nx, ny=ny, nz=nz, dx=1.0 / nx, dy=1.0 / nx, zf=I.z_faces(nz, nz / nx, beta),
                    bcx=bcx, bcy=bcy, rho_l=1.0, rho_g=1.0 / float(rng.uniform(10, 1000)), dt=1e-4,
                    precision=F.MIXED)
        off = tuple(int(rng.integers(0, m)) for m in tmpl.phi.shape)
        # one burst: the server admits while earlier requests run whatever the
        # speed of a single small solve, so overlap does not depend on timing
        reqs.append(S.Request(i, 0.0, desc, off))
    server = F.Server(budget, slots=4)
    served = {}

    def fill(r, views, stream):
        fields.fill(views, r.desc, r.offset, stream)

    def on_done(r, views):
        served[r.index] = [views[k].cpu().numpy() for k in (6, 3, 4, 5)]  # p, u, v, w

    out, summ = S.run(server, reqs, fill, deadline=30.0, on_done=on_done)
    info = server.info()
    server.close()
    assert summ["admitted"] == 16 and summ["all_converged"]
    assert summ["max_inflight"] >= 2
    if budget > (1 << 30):
        assert info["plans_built"] < 16  # the repeated geometry is served from the cache
    else:
        assert info["plans_cached"] < info["plans_built"]  # plans were evicted
    for r in reqs:
        inp = crop(tmpl, r.desc, r.offset)
        d = dict(r.desc)
        plan = F.Plan(d["nx"], d["ny"], d["nz"], d["dx"], d["dy"], zf=d["zf"], bcx=d["bcx"],
                      bcy=d["bcy"], rho_l=d["rho_l"], rho_g=d["rho_g"], dt=d["dt"], precision=F.MIXED)
        phi, pn, pm, u, v, w = (to_dev(a) for a in inp)
        p = torch.empty_like(phi)
        plan.solve(phi, pn, pm, u, v, w, p)
        torch.cuda.synchronize()
        plan.close()
        for got, ref in zip(served[r.index], (p, u, v, w)):
            assert np.array_equal(got, ref.cpu().numpy()), r.index


def test_served_periodic_z_requests(cuda_ok):
    """Periodic-z requests through the serving runtime, next to a
    wall-bounded request of the same grid (the plan cache keys on the z
    boundary): each result equals the same request solved alone, bit for bit,
    and the periodic ones match the oracle within the mixed bar."""
    import torch
    import oracle as O
    from gpu_util import compare
    specs = [I.CaseSpec(nx=32, ny=24, nz=20, n_bubbles=2, radius_cells=3, config=110, bcz=I.PERIODIC),
             I.CaseSpec(nx=32, ny=24, nz=20, n_bubbles=2, radius_cells=3, config=111),
             I.CaseSpec(nx=48, ny=32, nz=18, bcx=1, beta=1.3, n_bubbles=2, radius_cells=3, config=112,
                        bcz=I.PERIODIC)]
    cases = [I.make_case(s) for s in specs]
    reqs = []
    for i, c in enumerate(cases):
        s = c.spec
        desc = dict(nx=s.nx, ny=s.ny, nz=s.nz, dx=c.dx, dy=c.dy, zf=c.zf, bcx=s.bcx, bcy=s.bcy,
                    rho_l=s.rho_l, rho_g=s.rho_g, dt=s.dt, precision=F.MIXED,
                    periodic_z=s.bcz == I.PERIODIC)
        reqs.append(S.Request(i, 0.0, desc, (0, 0, 0)))
    server = F.Server(4 << 30, slots=4)
    served = {}

    def fill(r, views, stream):
        c = cases[r.index]
        with torch.cuda.stream(stream):
            for k, a in enumerate((c.phi, c.pn, c.pnm1, c.u, c.v, c.w)):
                views[k].copy_(torch.from_numpy(np.ascontiguousarray(a)), non_blocking=False)

    def on_done(r, views):
        served[r.index] = [views[k].cpu().numpy() for k in (6, 3, 4, 5)]

    out, summ = S.run(server, reqs, fill, deadline=30.0, on_done=on_done)
    info = server.info()
    server.close()
    assert summ["admitted"] == 3 and summ["all_converged"]
    assert info["plans_built"] == 3  # same grid, different z boundary: two plans
    for i, c in enumerate(cases):
        plan = F.Plan.for_case(c, precision=F.MIXED)
        phi, pn, pm, u, v, w = (to_dev(a) for a in (c.phi, c.pn, c.pnm1, c.u, c.v, c.w))
        p = torch.empty_like(phi)
        plan.solve(phi, pn, pm, u, v, w, p)
        torch.cuda.synchronize()
        plan.close()
        for got, ref in zip(served[i], (p, u, v, w)):
            assert np.array_equal(got, ref.cpu().numpy()), i
        if c.spec.bcz == I.PERIODIC:
            got = dict(p=served[i][0], u=served[i][1], v=served[i][2], w=served[i][3])
            ep, eu = compare(c, got, O.project_case(c))
            assert ep <= 1e-9 and eu <= 1e-9, (i, ep, eu)


def test_served_sweeps_beyond_the_first_two(cuda_ok):
    """A served mixed solve is queued with two refinement sweeps; one that
    has not converged by then (here: tol = 1e-30, divergence rule off, so it
    stops only at the residual floor) gets its remaining sweeps queued when
    it is polled.  Results and stats equal the plain solve's bit for bit."""
    import ctypes
    import torch
    from paper_2502_04189_b300 import _abi
    tmpl = I.make_case(I.CaseSpec(nx=48, ny=48, nz=40, n_bubbles=4, radius_cells=5, config=41))
    fields = S.TemplateFields(tmpl)
    reqs = []
    for i, (nx, ny, nz, beta) in enumerate([(32, 48, 24, 0.0), (48, 32, 30, 1.5), (32, 32, 16, 1.2)]):
        desc = dict(nx=nx, ny=ny, nz=nz, dx=1.0 / nx, dy=1.0 / nx, zf=I.z_faces(nz, nz / nx, beta),
                    bcx=i % 2, bcy=0, rho_l=1.0, rho_g=1e-3, dt=1e-4, precision=F.MIXED,
                    tol=1e-30, div_tol=-1.0, max_refine=6)
        reqs.append(S.Request(i, 0.0, desc, (3 * i, 5, 7)))
    server = F.Server(4 << 30, slots=4)
    served, stats = {}, {}

    def fill(r, views, stream):
        fields.fill(views, r.desc, r.offset, stream)

    def on_done(r, views):
        served[r.index] = [views[k].cpu().numpy() for k in (6, 3, 4, 5)]

    out, summ = S.run(server, reqs, fill, deadline=30.0, on_done=on_done)
    server.close()
    assert summ["admitted"] == 3
    for o in out:
        stats[o.index] = o.stats
    for r in reqs:
        d = dict(r.desc)
        plan = F.Plan(d["nx"], d["ny"], d["nz"], d["dx"], d["dy"], zf=d["zf"], bcx=d["bcx"],
                      bcy=d["bcy"], rho_l=d["rho_l"], rho_g=d["rho_g"], dt=d["dt"], precision=F.MIXED,
                      tol=d["tol"], div_tol=d["div_tol"], max_refine=d["max_refine"])
        phi, pn, pm, u, v, w = (to_dev(a) for a in crop(tmpl, d, r.offset))
        p = torch.empty_like(phi)
        plan.solve(phi, pn, pm, u, v, w, p)
        torch.cuda.synchronize()
        raw = _abi.Stats()  # read directly: a solve at the floor may report not converged
        _abi.lib().fizzy_proj_get_stats(plan._h, ctypes.byref(raw), None)
        st = raw.as_dict()
        plan.close()
        assert st["iterations"] >= 3, st  # the continuation ran
        assert stats[r.index]["iterations"] == st["iterations"]
        assert stats[r.index]["relres"] == st["relres"]
        assert stats[r.index]["converged"] == st["converged"]
        for got, ref in zip(served[r.index], (p, u, v, w)):
            assert np.array_equal(got, ref.cpu().numpy()), r.index
