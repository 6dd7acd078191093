"""Batched projections in one persistent launch (needs a B300).

Each instance solved inside the batch must equal the same plan solved alone,
bit for bit (the same kernel bodies run per tile), and match the FP64 oracle
within the mixed-mode tolerance.  "Alone" is the plain solve, except for
mixed instances with an x or y length of 128, 256 or 512: plain mixed
solves run register-resident FP32 transform passes there while the batch
keeps the Stockham bodies, so such an instance is compared with the same
instance batched alone, and with the plain solve within the mixed tolerance.
The instances are drawn with the uneven-batch recipe (sizes 32-192, periodic
or wall x/y, 1-20 drops, density ratio 10-1000).
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import R_LENGTHS, compare, plain_differs, run_alone, run_plain, to_dev

pytestmark = pytest.mark.gpu


def small_batch_specs(k=6):
    specs = I.batch_specs(64)
    specs.sort(key=lambda s: s.nx * s.ny * s.nz)
    return specs[:k - 1] + [specs[20]]  # the smallest ones plus one mid-size


@pytest.mark.parametrize("precision", [F.MIXED, F.FP64], ids=["mixed", "fp64"])
def test_batch_equals_alone(cuda_ok, precision):
    import torch
    cases = [I.make_case(s) for s in small_batch_specs()]
    alone = [run_alone(c, precision) for c in cases]
    plans, arrays = [], []
    for c in cases:
        plans.append(F.Plan.for_case(c, precision=precision))
        arrays.append((to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v),
                       to_dev(c.w), torch.empty(c.shape, dtype=torch.float64, device="cuda")))
    batch = F.Batch(plans, arrays)
    info = batch.info()
    assert info["items"] > len(cases) and info["grid"] >= 1
    for rep in range(2):  # replay the graph twice: same answer
        for c, arr in zip(cases, arrays):
            arr[3].copy_(to_dev(c.u))
            arr[4].copy_(to_dev(c.v))
            arr[5].copy_(to_dev(c.w))
        batch.solve()
        assert batch.status() == 0
        for c, arr, a, plan in zip(cases, arrays, alone, plans):
            got = dict(p=arr[6].cpu().numpy(), u=arr[3].cpu().numpy(), v=arr[4].cpu().numpy(),
                       w=arr[5].cpu().numpy())
            for k in ("p", "u", "v", "w"):
                assert np.array_equal(got[k], a[k]), (c.spec, k)
            st = plan.stats()
            assert st["converged"] == 1
            assert st["iterations"] == a["stats"]["iterations"]
    # the largest instance against the oracle
    c = cases[-1]
    ref = O.project_case(c)
    got = dict(p=arrays[-1][6].cpu().numpy(), u=arrays[-1][3].cpu().numpy(),
               v=arrays[-1][4].cpu().numpy(), w=arrays[-1][5].cpu().numpy())
    ep, eu = compare(c, got, ref)
    tol = 1e-9 if precision == F.MIXED else 1e-12
    assert ep <= tol and eu <= tol, (ep, eu)
    batch.close()
    for p in plans:
        p.close()


def test_batch_first_residual_convergence_equals_alone(cuda_ok):
    """Mixed instances with a loose tolerance stop at the residual of the FP32
    solution, so the batch takes its conditional-correction pass; results
    stay bitwise equal to each instance solved alone."""
    import torch
    cases = [I.make_case(s) for s in small_batch_specs(4)]
    kw = dict(tol=1e-3, div_tol=1.0)
    alone = [run_alone(c, F.MIXED, **kw) for c in cases]
    assert all(a["stats"]["iterations"] == 0 for a in alone)
    plans = [F.Plan.for_case(c, precision=F.MIXED, **kw) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays)
    batch.solve()
    assert batch.status() == 0
    for c, arr, a, plan in zip(cases, arrays, alone, plans):
        for key, t in (("p", arr[6]), ("u", arr[3]), ("v", arr[4]), ("w", arr[5])):
            assert np.array_equal(t.cpu().numpy(), a[key]), (c.spec, key)
        st = plan.stats()
        assert st["converged"] == 1 and st["iterations"] == 0
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", [F.MIXED, F.FP64], ids=["mixed", "fp64"])
def test_batch_swapped_density_equals_alone(cuda_ok, precision):
    """An instance whose lighter phase is the drop phase (rho0 = rho_l, the
    split term formed from 1 - phi) batched with an ordinary one."""
    import dataclasses
    import torch
    base = small_batch_specs(3)
    specs = [base[0], dataclasses.replace(base[1], rho_l=base[1].rho_g, rho_g=base[1].rho_l)]
    assert specs[1].rho_l < specs[1].rho_g
    cases = [I.make_case(sp) for sp in specs]
    alone = [run_alone(c, precision) for c in cases]
    plans = [F.Plan.for_case(c, precision=precision) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays)
    batch.solve()
    assert batch.status() == 0
    for c, arr, a in zip(cases, arrays, alone):
        for key, t in (("p", arr[6]), ("u", arr[3]), ("v", arr[4]), ("w", arr[5])):
            assert np.array_equal(t.cpu().numpy(), a[key]), (c.spec, key)
    ref = O.project_case(cases[1])
    got = dict(p=arrays[1][6].cpu().numpy(), u=arrays[1][3].cpu().numpy(),
               v=arrays[1][4].cpu().numpy(), w=arrays[1][5].cpu().numpy())
    ep, eu = compare(cases[1], got, ref)
    tol = 1e-9 if precision == F.MIXED else 1e-12
    assert ep <= tol and eu <= tol, (ep, eu)
    batch.close()
    for p in plans:
        p.close()


def test_batch_autotune_keeps_results(cuda_ok):
    import torch
    cases = [I.make_case(s) for s in small_batch_specs(4)]
    plans, arrays = [], []
    for c in cases:
        plans.append(F.Plan.for_case(c, precision=F.MIXED))
        arrays.append((to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v),
                       to_dev(c.w), torch.empty(c.shape, dtype=torch.float64, device="cuda")))
    batch = F.Batch(plans, arrays)
    tuning, ms = batch.autotune(reps=2)
    assert ms > 0 and tuning["form"] in (0, 1, 2)
    assert tuning["form"] == 2 or tuning["flux_planes"] in (32, 64)  # solo chains keep the plan's tiles
    for c, arr in zip(cases, arrays):
        arr[3].copy_(to_dev(c.u))
        arr[4].copy_(to_dev(c.v))
        arr[5].copy_(to_dev(c.w))
    batch.solve()
    assert batch.status() == 0
    for c, arr in zip(cases, arrays):
        # the solo-chain form runs each plan's own passes
        a = run_plain(c, F.MIXED) if tuning["form"] == 2 else run_alone(c, F.MIXED)
        assert np.array_equal(arr[6].cpu().numpy(), a["p"])
        assert np.array_equal(arr[3].cpu().numpy(), a["u"])
    batch.close()
    for p in plans:
        p.close()


def test_batch_mixed_matches_plain_within_tolerance(cuda_ok):
    """Mixed instances whose plain solves run the register-resident FP32
    passes: the batched result (Stockham FP32 passes) and the plain one both
    converge to relres <= 1e-10 and agree within the mixed tolerance."""
    import torch
    specs = sorted((s for s in I.batch_specs(64) if s.nx in R_LENGTHS or s.ny in R_LENGTHS),
                   key=lambda s: s.nx * s.ny * s.nz)[:3]
    assert specs
    cases = [I.make_case(s) for s in specs]
    assert all(plain_differs(c, F.MIXED) for c in cases)
    plans = [F.Plan.for_case(c, precision=F.MIXED) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays)
    batch.solve()
    assert batch.status() == 0
    for c, arr, plan in zip(cases, arrays, plans):
        assert plan.stats()["converged"] == 1
        a = run_plain(c, F.MIXED)
        assert a["stats"]["converged"] == 1 and a["stats"]["relres"] <= 1e-10
        got = dict(p=arr[6].cpu().numpy(), u=arr[3].cpu().numpy(), v=arr[4].cpu().numpy(),
                   w=arr[5].cpu().numpy())
        ep, eu = compare(c, got, a)
        assert ep <= 1e-9 and eu <= 1e-9, (c.spec, ep, eu)
    batch.close()
    for p in plans:
        p.close()


def test_batch_wait_timeout_is_reported_and_recoverable(cuda_ok):
    """A dependency wait that can never be met gives up after its poll limit:
    the launch ends, the status is FIZZY_ERR_TIMEOUT, and after restoring the
    defaults the same batch solves correctly (no GPU fault, context usable)."""
    import torch
    cases = [I.make_case(s) for s in small_batch_specs(3)]
    alone = [run_alone(c, F.FP64) for c in cases]
    plans = [F.Plan.for_case(c, precision=F.FP64) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays)
    batch.inject_stall(inst=1, spin_limit=1 << 12)
    batch.solve()
    assert batch.status() == -6  # FIZZY_ERR_TIMEOUT
    batch.inject_stall()
    for c, arr in zip(cases, arrays):
        arr[3].copy_(to_dev(c.u))
        arr[4].copy_(to_dev(c.v))
        arr[5].copy_(to_dev(c.w))
    batch.solve()
    assert batch.status() == 0
    for c, arr, a in zip(cases, arrays, alone):
        for key, t in (("p", arr[6]), ("u", arr[3]), ("v", arr[4]), ("w", arr[5])):
            assert np.array_equal(t.cpu().numpy(), a[key]), (c.spec, key)
    batch.close()
    for p in plans:
        p.close()


FORMS = [dict(form=1, chains=1), dict(form=1, chains=2), dict(form=1, chains=8, flux_planes=32),
         dict(order=2)]
FORM_IDS = ["grouped1", "grouped2", "grouped8", "staggered"]


@pytest.mark.parametrize("precision", [F.MIXED, F.FP64], ids=["mixed", "fp64"])
@pytest.mark.parametrize("tuning", FORMS, ids=FORM_IDS)
def test_batch_forms_equal_alone(cuda_ok, precision, tuning):
    """The grouped launches (one ordinary launch per pass over every instance
    of a chain, 1, 2 or 8 concurrent chains) and the staggered work list run
    the same bodies: each instance equals its solve alone bit for bit, here
    with a swapped-density instance among them."""
    import dataclasses
    import torch
    specs = small_batch_specs(5)
    specs.append(dataclasses.replace(specs[1], rho_l=specs[1].rho_g, rho_g=specs[1].rho_l))
    cases = [I.make_case(s) for s in specs]
    alone = [run_alone(c, precision) for c in cases]
    plans = [F.Plan.for_case(c, precision=precision) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays, tuning=tuning)
    info = batch.info()
    assert info["items"] >= 7 and info["grid"] >= 1
    for rep in range(2):
        for c, arr in zip(cases, arrays):
            arr[3].copy_(to_dev(c.u))
            arr[4].copy_(to_dev(c.v))
            arr[5].copy_(to_dev(c.w))
        batch.solve()
        assert batch.status() == 0
        for c, arr, a, plan in zip(cases, arrays, alone, plans):
            for key, t in (("p", arr[6]), ("u", arr[3]), ("v", arr[4]), ("w", arr[5])):
                assert np.array_equal(t.cpu().numpy(), a[key]), (c.spec, key, rep)
            st = plan.stats()
            assert st["converged"] == 1
            assert st["iterations"] == a["stats"]["iterations"]
    if tuning.get("form") == 1:
        with pytest.raises(F.FizzyError):
            batch.inject_stall(inst=0, spin_limit=16)  # no waits in the grouped form
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", [F.MIXED, F.FP64], ids=["mixed", "fp64"])
def test_batch_grouped_equals_persistent_on_uneven_batch(cuda_ok, precision):
    """All 64 instances of the uneven-batch recipe (sizes 32-192, every
    boundary mix, lengths of the register-resident passes included): the
    grouped form with two chains gives the persistent launch's bits."""
    import torch
    cases = [I.make_case(s) for s in I.batch_specs(64)]
    plans = [F.Plan.for_case(c, precision=precision) for c in cases]
    outs = {}
    for name, tun in (("persistent", None), ("grouped", dict(form=1, chains=2))):
        arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v),
                   to_dev(c.w), torch.empty(c.shape, dtype=torch.float64, device="cuda"))
                  for c in cases]
        batch = F.Batch(plans, arrays, tuning=tun)
        batch.solve()
        assert batch.status() == 0
        outs[name] = [[a[k].cpu().numpy() for k in (6, 3, 4, 5)] for a in arrays]
        outs[name + "_iters"] = [p.stats()["iterations"] for p in plans]
        batch.close()
        del arrays
    for c, a, b in zip(cases, outs["persistent"], outs["grouped"]):
        for x, y, key in zip(a, b, "puvw"):
            assert np.array_equal(x, y), (c.spec, key)
    assert outs["persistent_iters"] == outs["grouped_iters"]
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", [F.MIXED, F.FP64], ids=["mixed", "fp64"])
@pytest.mark.parametrize("chains", [1, 3, 16])
def test_batch_solo_chains_equal_plain(cuda_ok, precision, chains):
    """The solo-chain form replays each instance's own stand-alone launch
    sequence on concurrent chains: every instance equals its plain solve bit
    for bit (register-resident FP32 passes included), over two replays, and
    the largest matches the oracle."""
    import dataclasses
    import torch
    specs = small_batch_specs(5)
    specs.append(dataclasses.replace(specs[1], rho_l=specs[1].rho_g, rho_g=specs[1].rho_l))
    specs += sorted((s for s in I.batch_specs(64) if s.nx in R_LENGTHS or s.ny in R_LENGTHS),
                    key=lambda s: s.nx * s.ny * s.nz)[:2]
    cases = [I.make_case(s) for s in specs]
    plain = [run_plain(c, precision) for c in cases]
    plans = [F.Plan.for_case(c, precision=precision) for c in cases]
    arrays = [(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), to_dev(c.u), to_dev(c.v), to_dev(c.w),
               torch.empty(c.shape, dtype=torch.float64, device="cuda")) for c in cases]
    batch = F.Batch(plans, arrays, tuning=dict(form=2, chains=chains))
    assert batch.info()["items"] == len(cases)
    for rep in range(2):
        for c, arr in zip(cases, arrays):
            arr[3].copy_(to_dev(c.u))
            arr[4].copy_(to_dev(c.v))
            arr[5].copy_(to_dev(c.w))
        batch.solve()
        assert batch.status() == 0
        for c, arr, a, plan in zip(cases, arrays, plain, plans):
            for key, t in (("p", arr[6]), ("u", arr[3]), ("v", arr[4]), ("w", arr[5])):
                assert np.array_equal(t.cpu().numpy(), a[key]), (c.spec, key, rep)
            st = plan.stats()
            assert st["converged"] == 1 and st["iterations"] == a["stats"]["iterations"]
    with pytest.raises(F.FizzyError):
        batch.inject_stall(inst=0, spin_limit=16)  # no waits in the solo-chain form
    k = max(range(len(cases)), key=lambda i: cases[i].npts)
    ref = O.project_case(cases[k])
    got = dict(p=arrays[k][6].cpu().numpy(), u=arrays[k][3].cpu().numpy(),
               v=arrays[k][4].cpu().numpy(), w=arrays[k][5].cpu().numpy())
    ep, eu = compare(cases[k], got, ref)
    tol = 1e-9 if precision == F.MIXED else 1e-12
    assert ep <= tol and eu <= tol, (ep, eu)
    batch.close()
    for p in plans:
        p.close()
