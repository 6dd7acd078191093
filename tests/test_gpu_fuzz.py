"""Seeded random configurations against the FP64 oracle (needs a B300).

Sizes are products of 2 and 3 (including the register-resident lengths 32, 48, 64,
96, 128, 192, 256, 384 and 512 and odd lengths such as 3, 9, 27), boundaries, stretching, density ratio,
drop count, velocity recipe and the phase that is light all drawn at random;
every case must meet the same bars as the named parity cases: FP64 <= 1e-12,
mixed <= 1e-9 after refinement, divergence <= 1e-10.

Some draws are pressure-dominated: the correction (dt/rho0) G p is up to
1e3 times max|u| (a 2-cell direction with a weak velocity field).  A p that
agrees with the oracle to round-off then moves u by (dt/rho0) 2 eps max|p| /
h_min through the gradient, which can exceed 1e-12 of max|u| for any FP64
solver; the velocity bar is the larger of 1e-12 and ten times that floor,
computed from the oracle's fields (the floor is reported beside the error).
test_fuzz_floor_report, the last test of this file, lists every draw whose
velocity error exceeded the plain bar and passed on that floor, with the
largest floor seen."""
import warnings

import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import compare, gpu_project, run_alone, to_dev

pytestmark = pytest.mark.gpu

LENGTHS = (2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 32, 36, 48, 54, 64, 72, 96, 128, 192, 256, 384, 512)


def fuzz_specs(n=32, seed=2024, bcz_mix=False):
    """n random specs; with bcz_mix each draw also picks walls or periodic z
    (the draws of the wall-only lists stay as they were)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        nx, ny = int(rng.choice(LENGTHS)), int(rng.choice(LENGTHS))
        nz = int(rng.integers(2, 41))
        if nx * ny * nz > 160_000:  # keep the oracle to a fraction of a second
            continue
        light_drops = bool(rng.random() < 0.7)
        ratio = float(10 ** rng.uniform(0, 3))
        rho_g, rho_l = (1.0 / ratio, 1.0) if light_drops else (1.0, 1.0 / ratio)
        bcz = int(rng.integers(0, 2)) if bcz_mix else I.NEUMANN
        out.append(I.CaseSpec(
            nx=nx, ny=ny, nz=nz, bcx=int(rng.integers(0, 2)), bcy=int(rng.integers(0, 2)),
            beta=float(rng.uniform(0.5, 2.0)) if rng.random() < 0.5 else 0.0,
            n_bubbles=int(rng.integers(1, 4)), radius_cells=float(rng.uniform(0.5, 4.0)),
            rho_l=rho_l, rho_g=rho_g, dt=float(10 ** rng.uniform(-4, -2)),
            velocity="iid" if rng.random() < 0.3 else "solenoidal",
            config=60, instance=len(out), bcz=bcz))
    return out


SPECS = fuzz_specs()
# walls or periodic z drawn per case (triperiodic boxes among them)
PZ_SPECS = fuzz_specs(24, seed=2025, bcz_mix=True)


def velocity_floor(case, ref):
    """Relative velocity change caused by a one-ulp change of p."""
    s = case.spec
    g = O.Grid.of_case(case)
    rho0 = min(s.rho_l, s.rho_g)
    pmax = np.max(np.abs(ref["p"] - O.weighted_mean(g, ref["p"])))
    hmin = min(case.dx, case.dy, float(np.diff(case.zf).min()))
    umax = max(np.max(np.abs(ref[k])) for k in "uvw")
    return s.dt / rho0 * 2 * np.finfo(np.float64).eps * pmax / hmin / umax


# (draw, precision, velocity error, floor) of every draw that needed the floor,
# and the largest floor over all draws
FLOOR_LOG = []
FLOOR_MAX = [0.0, None]


def check_against_oracle(spec, label):
    c = I.make_case(spec)
    ref = O.project_case(c)
    floor = velocity_floor(c, ref)
    if floor > FLOOR_MAX[0]:
        FLOOR_MAX[:] = [floor, label]
    got = gpu_project(c, F.FP64)
    ep, eu = compare(c, got, ref)
    assert ep <= 1e-12 and eu <= max(1e-12, 10 * floor), (spec, ep, eu, floor)
    if eu > 1e-12:
        FLOOR_LOG.append((label, "fp64", eu, floor))
    assert got["stats"]["div_metric"] <= 1e-10, spec
    got = gpu_project(c, F.MIXED)
    st = got["stats"]
    assert st["converged"] == 1 and st["relres"] <= 1e-10, (spec, st)
    ep, eu = compare(c, got, ref)
    assert ep <= 1e-9 and eu <= max(1e-9, 10 * floor), (spec, ep, eu, floor)
    if eu > 1e-9:
        FLOOR_LOG.append((label, "mixed", eu, floor))
    assert st["div_metric"] <= 1e-10, spec


@pytest.mark.parametrize("i", range(len(SPECS)))
def test_fuzz_matches_oracle(cuda_ok, i):
    check_against_oracle(SPECS[i], "walls-z draw %d" % i)


@pytest.mark.parametrize("i", range(len(PZ_SPECS)))
def test_fuzz_periodic_z_matches_oracle(cuda_ok, i):
    check_against_oracle(PZ_SPECS[i], "mixed-z draw %d" % i)


@pytest.mark.parametrize("precision", [F.FP64, F.MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("seed,bcz_mix", [(7, False), (8, False), (9, True)])
def test_fuzz_batch_equals_alone(cuda_ok, precision, seed, bcz_mix):
    """Random mixes of eight of these instances in one persistent launch
    (the last mix with periodic z drawn per instance): each equals the same
    instance solved alone, bit for bit."""
    import torch
    specs = fuzz_specs(8, seed=seed, bcz_mix=bcz_mix)
    cases = [I.make_case(s) for s in specs]
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
    batch.close()
    for p in plans:
        p.close()


def test_fuzz_floor_report(cuda_ok):
    """The draws that passed only on the velocity floor (error above the
    plain bar, below ten times the floor) and the largest floor seen,
    reported as a warning (pytest prints it in its summary)."""
    lines = ["%s (%s): velocity error %.2e, floor %.2e" % d for d in FLOOR_LOG]
    warnings.warn("fuzz draws passing on the R14 floor: %d%s; largest floor %.2e (%s)" % (
        len(FLOOR_LOG), "".join("\n  " + x for x in lines), FLOOR_MAX[0], FLOOR_MAX[1]))
    for _, prec, eu, floor in FLOOR_LOG:
        assert eu <= 10 * floor, (prec, eu, floor)
