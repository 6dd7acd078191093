"""GPU projection vs the FP64 CPU oracle, element by element (needs a B300).

Tolerances: max relative error (max|x_gpu - x_oracle| / max|x_oracle|, p after
removing its dzf-weighted mean, u over all three face families) <= 1e-12 in
FP64 mode and <= 1e-9 in mixed mode after refinement to relres <= 1e-10;
max|D u| dx / U <= 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import paper_2502_04189_b300 as F
from paper_2502_04189_b300 import inputs as I

from gpu_util import compare, gpu_project, relerr, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-9


def small_cases():
    return {
        "drop32": I.drop32_spec(),
        "b48x36x20_nx_stretch": I.CaseSpec(nx=48, ny=36, nz=20, bcx=1, bcy=0, beta=1.5,
                                           n_bubbles=3, radius_cells=4, config=11),
        "b96x64x33": I.CaseSpec(nx=96, ny=64, nz=33, n_bubbles=4, radius_cells=5, config=12),
        "b27x18x12_ny": I.CaseSpec(nx=27, ny=18, nz=12, bcx=0, bcy=1, n_bubbles=1,
                                   radius_cells=3, config=13),
        "b384x6x5": I.CaseSpec(nx=384, ny=6, nz=5, bcx=1, bcy=1, n_bubbles=1, radius_cells=2,
                               config=14),
        "b6x512x4": I.CaseSpec(nx=6, ny=512, nz=4, bcx=0, bcy=0, n_bubbles=1, radius_cells=1,
                               config=15),
        "b1024x4x3": I.CaseSpec(nx=1024, ny=4, nz=3, bcx=0, bcy=1, n_bubbles=1,
                                radius_cells=1, config=16),
        "b2x2x2": I.CaseSpec(nx=2, ny=2, nz=2, bcx=0, bcy=1, n_bubbles=1, radius_cells=0.5,
                             config=17, velocity="iid"),
        "b81x3x7_nn": I.CaseSpec(nx=81, ny=3, nz=7, bcx=1, bcy=1, beta=2.0, n_bubbles=1,
                                 radius_cells=2, config=18),
        # periodic x of length 512: the length-specialised x-pass instances
        "b512x8x5": I.CaseSpec(nx=512, ny=8, nz=5, bcx=0, bcy=1, n_bubbles=1, radius_cells=2,
                               config=20),
        # periodic y of length 256: the register-resident FP32 y-passes of the
        # mixed mode, with ragged 32-column tiles (even nx: paired loads; odd
        # nx: single loads and a last line without imaginary part)
        "b48x256x12": I.CaseSpec(nx=48, ny=256, nz=12, bcx=0, bcy=0, beta=1.5, n_bubbles=2,
                                 radius_cells=3, config=22),
        "b27x256x6_wx": I.CaseSpec(nx=27, ny=256, nz=6, bcx=1, bcy=0, n_bubbles=1, radius_cells=3,
                                   config=23),
        # periodic x of length 256: the register-resident FP32 x-passes (the
        # second has an odd number of x-lines, 9 x 5: a last line without
        # partner)
        "b256x12x10": I.CaseSpec(nx=256, ny=12, nz=10, bcx=0, bcy=1, beta=1.2, n_bubbles=2,
                                 radius_cells=3, config=24),
        "b256x9x5_wy": I.CaseSpec(nx=256, ny=9, nz=5, bcx=0, bcy=1, n_bubbles=1, radius_cells=2,
                                  config=25),
        # length 512 (radix-2 split ahead of the 16 x 16 transform): periodic
        # y with ragged 16-column tiles (even and odd nx), periodic x with an
        # odd number of x-lines
        "b24x512x8": I.CaseSpec(nx=24, ny=512, nz=8, bcx=1, bcy=0, beta=1.5, n_bubbles=2,
                                radius_cells=3, config=26),
        "b9x512x3": I.CaseSpec(nx=9, ny=512, nz=3, bcx=0, bcy=0, n_bubbles=1, radius_cells=2,
                               config=27),
        "b512x3x3_wy": I.CaseSpec(nx=512, ny=3, nz=3, bcx=0, bcy=1, n_bubbles=1, radius_cells=1,
                                  config=28),
        # walls (DCT-II) along a direction of length 256 or 512: the
        # register-resident passes with the reordered packing and post-twiddles
        "b48x256x12_wy": I.CaseSpec(nx=48, ny=256, nz=12, bcx=0, bcy=1, beta=1.2, n_bubbles=2,
                                    radius_cells=3, config=30),
        "b256x12x10_wx": I.CaseSpec(nx=256, ny=12, nz=10, bcx=1, bcy=0, n_bubbles=2, radius_cells=3,
                                    config=31),
        "b24x512x8_wxy": I.CaseSpec(nx=24, ny=512, nz=8, bcx=1, bcy=1, beta=1.5, n_bubbles=2,
                                    radius_cells=3, config=32),
        "b512x3x3_wxy": I.CaseSpec(nx=512, ny=3, nz=3, bcx=1, bcy=1, n_bubbles=1, radius_cells=1,
                                   config=33),
        # length 128 (the 16 x 8 transform, 4 lines per warp) and 64 (16 x 4):
        # walls and periodic, odd nx, ragged y tiles, odd line counts
        "b27x64x9_wy": I.CaseSpec(nx=27, ny=64, nz=9, bcx=0, bcy=1, beta=1.3, n_bubbles=1,
                                  radius_cells=3, config=34),
        "b36x128x10": I.CaseSpec(nx=36, ny=128, nz=10, bcx=1, bcy=0, n_bubbles=2, radius_cells=3,
                                 config=35),
        "b64x9x7": I.CaseSpec(nx=64, ny=9, nz=7, bcx=0, bcy=1, n_bubbles=1, radius_cells=2, config=36),
        "b128x6x5_wx": I.CaseSpec(nx=128, ny=6, nz=5, bcx=1, bcy=0, beta=1.5, n_bubbles=1,
                                  radius_cells=2, config=37),
        "b64x128x16_w": I.CaseSpec(nx=64, ny=128, nz=16, bcx=1, bcy=1, n_bubbles=2, radius_cells=4,
                                   config=38),
        "b128x3x3_odd": I.CaseSpec(nx=128, ny=3, nz=3, bcx=0, bcy=1, n_bubbles=1, radius_cells=1,
                                   config=39),
        "b27x128x5_wy": I.CaseSpec(nx=27, ny=128, nz=5, bcx=1, bcy=1, beta=1.8, n_bubbles=1,
                                   radius_cells=2, config=42),
        # the register-resident lengths 32 (16 x 2), 48 (12 x 4), 96 (24 x 4),
        # 192 (24 x 8) and 384 (radix-2 split ahead of 24 x 8): periodic and
        # walls, odd line counts, y tiles flattened over ragged planes
        "b32x24x9_wx": I.CaseSpec(nx=32, ny=24, nz=9, bcx=1, bcy=0, beta=1.4, n_bubbles=1,
                                  radius_cells=3, config=43),
        "b9x32x7": I.CaseSpec(nx=9, ny=32, nz=7, bcx=0, bcy=0, n_bubbles=1, radius_cells=3,
                               config=44),
        "b48x6x7_wx": I.CaseSpec(nx=48, ny=6, nz=7, bcx=1, bcy=1, n_bubbles=1, radius_cells=2,
                                 config=45),
        "b27x48x6": I.CaseSpec(nx=27, ny=48, nz=6, bcx=0, bcy=0, beta=1.2, n_bubbles=1,
                               radius_cells=3, config=46),
        "b96x9x5": I.CaseSpec(nx=96, ny=9, nz=5, bcx=0, bcy=1, n_bubbles=1, radius_cells=2,
                              config=47),
        "b27x96x6_wy": I.CaseSpec(nx=27, ny=96, nz=6, bcx=0, bcy=1, beta=1.5, n_bubbles=2,
                                  radius_cells=3, config=48),
        "b192x6x3_wx": I.CaseSpec(nx=192, ny=6, nz=3, bcx=1, bcy=0, n_bubbles=1, radius_cells=2,
                                  config=49),
        "b18x192x4": I.CaseSpec(nx=18, ny=192, nz=4, bcx=1, bcy=0, n_bubbles=1, radius_cells=3,
                                config=50),
        "b9x384x3": I.CaseSpec(nx=9, ny=384, nz=3, bcx=0, bcy=0, n_bubbles=1, radius_cells=3,
                                config=51),
        "b384x9x3": I.CaseSpec(nx=384, ny=9, nz=3, bcx=0, bcy=1, beta=1.3, n_bubbles=1,
                               radius_cells=2, config=52),
        "b18x384x2_wy": I.CaseSpec(nx=18, ny=384, nz=2, bcx=1, bcy=1, n_bubbles=1, radius_cells=3,
                                   config=53),
        # light drops in a heavy phase: rho0 = rho_l, split term from 1 - phi
        "b48x32x24_swapped": I.CaseSpec(nx=48, ny=32, nz=24, bcx=0, bcy=1, beta=1.5, n_bubbles=3,
                                        radius_cells=4, rho_l=1e-3, rho_g=1.0, config=19),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_matches_oracle(cuda_ok, name):
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


@pytest.mark.parametrize("name", ["drop32", "b48x36x20_nx_stretch", "b96x64x33", "b27x18x12_ny",
                                  "b384x6x5", "b81x3x7_nn", "b48x32x24_swapped", "b512x8x5",
                                  "b48x256x12", "b27x256x6_wx", "b256x12x10", "b256x9x5_wy",
                                  "b6x512x4", "b24x512x8", "b9x512x3", "b512x3x3_wy",
                                  "b48x256x12_wy", "b256x12x10_wx", "b24x512x8_wxy", "b512x3x3_wxy",
                                  "b27x64x9_wy", "b36x128x10", "b64x9x7", "b128x6x5_wx",
                                  "b64x128x16_w", "b128x3x3_odd", "b27x128x5_wy",
                                  "b32x24x9_wx", "b9x32x7", "b48x6x7_wx", "b27x48x6", "b96x9x5",
                                  "b27x96x6_wy", "b192x6x3_wx", "b18x192x4", "b9x384x3",
                                  "b384x9x3", "b18x384x2_wy"])
def test_mixed_matches_oracle(cuda_ok, name):
    c = I.make_case(CASES[name])
    ref = O.project_case(c)
    got = gpu_project(c, F.MIXED)
    st = got["stats"]
    assert st["converged"] == 1
    assert st["relres"] <= 1e-10
    assert 1 <= st["iterations"] <= 4
    ep, eu = compare(c, got, ref)
    assert ep <= TOLMIX, ep
    assert eu <= TOLMIX, eu
    assert st["div_metric"] < 1e-10


@pytest.mark.parametrize("name", ["b48x256x12", "b27x256x6_wx", "b256x12x10", "b256x9x5_wy",
                                  "b24x512x8", "b512x8x5", "b48x256x12_wy", "b256x12x10_wx",
                                  "b24x512x8_wxy", "b27x64x9_wy", "b128x6x5_wx", "b64x128x16_w",
                                  "b96x64x33", "b32x24x9_wx", "b27x48x6", "b27x96x6_wy",
                                  "b18x192x4", "b9x384x3", "b384x9x3"])
def test_fp32_solve_accuracy(cuda_ok, name):
    """The FP32 solve alone (stopped at its first residual) is accurate to
    FP32 level, whichever transform kernels it runs: the Stockham and the
    register-resident passes leave the same relres, 1e-6 to 6e-5 at n = 256
    and up to 1.8e-4 at n = 512 with stretched z (24 x 512 x 8), and at most
    two refinement sweeps then reach 1e-10."""
    c = I.make_case(CASES[name])
    got = gpu_project(c, F.MIXED, tol=1e-3, div_tol=1.0)
    st = got["stats"]
    assert st["iterations"] == 0 and 0 < st["relres"] <= 3e-4, st
    st = gpu_project(c, F.MIXED)["stats"]
    assert st["converged"] == 1 and 1 <= st["iterations"] <= 2, st


def test_equal_density_closed_form(cuda_ok):
    """rho_l = rho_g and u* = s + G q (s a discrete curl): p = (rho0/dt) q, u = s."""
    spec = I.CaseSpec(nx=48, ny=32, nz=24, bcx=1, bcy=0, beta=1.5, n_bubbles=2,
                      radius_cells=3, rho_l=0.5, rho_g=0.5, dt=1e-3, noise=0.0, config=21)
    c = I.make_case(spec)
    g = O.Grid.of_case(c)
    s = (c.u.copy(), c.v.copy(), c.w.copy())
    q = np.random.default_rng(4).standard_normal(g.shape)
    gq = O.grad(g, q)
    c.u, c.v, c.w = (s[a] + gq[a] for a in range(3))
    for prec, tol in ((F.FP64, 1e-11), (F.MIXED, 1e-9)):
        got = gpu_project(c, prec)
        p_exact = (0.5 / 1e-3) * (q - O.weighted_mean(g, q))
        assert relerr(got["p"] - O.weighted_mean(g, got["p"]), p_exact) < tol
        for a, key in enumerate("uvw"):
            assert np.max(np.abs(got[key] - s[a])) < tol * np.max(np.abs(gq[a]) + np.abs(s[a]))


def test_repeat_is_bitwise_deterministic(cuda_ok):
    c = I.make_case(CASES["b96x64x33"])
    for prec in (F.FP64, F.MIXED):
        plan = F.Plan.for_case(c, precision=prec, check=True)
        a = gpu_project(c, plan=plan)
        b = gpu_project(c, plan=plan)
        plan.close()
        for k in ("p", "u", "v", "w"):
            assert np.array_equal(a[k], b[k]), k


def test_not_converged_is_reported(cuda_ok):
    c = I.make_case(CASES["b48x36x20_nx_stretch"])
    plan = F.Plan.for_case(c, precision=F.MIXED, check=True, tol=1e-30, max_refine=1)
    got = gpu_project(c, plan=plan)
    plan.close()
    st = got["stats"]
    assert st["converged"] == 0
    assert st["iterations"] == 1
    assert st["relres"] > 0
    ref = O.project_case(c)
    ep, eu = compare(c, got, ref)
    assert ep < 1e-6  # one sweep still lands close


def test_mixed_converged_at_first_residual(cuda_ok):
    """A loose tolerance stops at the residual of the FP32 solution (no
    refinement sweep): the final correction then runs on its own and u must
    be the corrected field, within the accuracy of the FP32 solve."""
    c = I.make_case(CASES["b96x64x33"])
    got = gpu_project(c, F.MIXED, tol=1e-3, div_tol=1.0)
    st = got["stats"]
    assert st["converged"] == 1 and st["iterations"] == 0, st
    assert 0 < st["relres"] <= 1e-3
    ref = O.project_case(c)
    ep, eu = compare(c, got, ref)
    assert ep < 1e-4 and eu < 1e-4, (ep, eu)
    # u is not the provisional velocity
    moved = max(np.max(np.abs(got[k] - getattr(c, k))) for k in "uvw")
    assert moved > 1e3 * eu * max(np.max(np.abs(ref[k])) for k in "uvw")


def test_solve_host_matches_device(cuda_ok):
    c = I.make_case(CASES["b96x64x33"])
    plan = F.Plan.for_case(c, precision=F.FP64)
    d = gpu_project(c, plan=plan)
    u, v, w = c.u.copy(), c.v.copy(), c.w.copy()
    p = np.empty_like(c.phi)
    plan.solve_host(c.phi, c.pn, c.pnm1, u, v, w, p)
    plan.close()
    for key, arr in (("p", p), ("u", u), ("v", v), ("w", w)):
        assert np.array_equal(arr, d[key]), key


def test_solve_host_async_pipeline(cuda_ok):
    """Three pipelined host-array solves queued back to back (different inputs,
    distinct pinned outputs) equal the device-array solves bit for bit."""
    import torch
    c = I.make_case(CASES["b96x64x33"])
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    scales = (1.0, -0.5, 2.0)
    for prec in (F.FP64, F.MIXED):
        plan = F.Plan.for_case(c, precision=prec)
        expect = []
        for sc in scales:
            u, v, w = to_dev(sc * c.u), to_dev(sc * c.v), to_dev(sc * c.w)
            p = torch.empty_like(u)
            plan.solve(to_dev(c.phi), to_dev(c.pn), to_dev(c.pnm1), u, v, w, p)
            torch.cuda.synchronize()
            expect.append([t.cpu().numpy() for t in (u, v, w, p)])
        ins = [[pin(c.phi), pin(c.pn), pin(c.pnm1), pin(sc * c.u), pin(sc * c.v), pin(sc * c.w)]
               for sc in scales]
        outs = [[torch.empty(c.shape, dtype=torch.float64).pin_memory() for _ in range(4)]
                for _ in scales]
        for hin, hout in zip(ins, outs):
            plan.solve_host_async(*hin, *hout)
        plan.host_wait()
        for hout, ref in zip(outs, expect):
            for t, r in zip(hout, ref):
                assert np.array_equal(t.numpy(), r)
        plan.close()


def test_native_library_is_loaded(cuda_ok):
    c = I.make_case(CASES["drop32"])
    gpu_project(c)
    maps = open("/proc/self/maps").read()
    assert "libfizzyproj.so" in maps


# ---------------------------------------------------------------------------
# Full-size workloads, in the launch configuration bench.py times
# ---------------------------------------------------------------------------
def test_bubbles256_fp64_full_size(cuda_ok):
    c = I.make_case(I.bubbles256_spec())
    ref = O.project_case(c)
    got = gpu_project(c, F.FP64)
    ep, eu = compare(c, got, ref)
    assert ep <= TOL64, ep
    assert eu <= TOL64, eu
    assert got["stats"]["div_metric"] <= 1e-10
    got_m = gpu_project(c, F.MIXED)
    ep, eu = compare(c, got_m, ref)
    assert got_m["stats"]["relres"] <= 1e-10
    assert ep <= TOLMIX and eu <= TOLMIX, (ep, eu)


def test_bubbles512_stretched_mixed_full_size(cuda_ok):
    """512^3, tanh-stretched z (beta 1.5), 400 drops of radius 6, ratio 1000,
    mixed precision refined to relres <= 1e-10: the whole field against the
    FP64 oracle, plus the divergence identity."""
    c = I.make_case(I.bubbles512_stretched_spec())
    got = gpu_project(c, F.MIXED)
    st = got["stats"]
    assert st["converged"] == 1 and st["relres"] <= 1e-10 and st["div_metric"] <= 1e-10
    ref = O.project_case(c)
    ep, eu = compare(c, got, ref)
    assert ep <= TOLMIX and eu <= TOLMIX, (ep, eu)
