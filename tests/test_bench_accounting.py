"""bench.py's roofline bookkeeping (CPU): the FP64 instruction counts follow
the radix plan of the transforms, and the whole-projection roofline sums the
per-pass bytes of exactly the passes a solve runs."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_transform_instruction_counts():
    # n = 256 = 4^4: a twiddle-free radix-4 stage (4 per complex point), three
    # more (6 each): 22 per complex point, 11 per real point, +1 separation
    assert bench.fft_fp64_instr_per_point(256, dct=False) == 12
    assert bench.fft_fp64_instr_per_point(256, dct=True) == 14  # +2 post-twiddle
    # n = 512 = 4^4 * 2: + one radix-2 stage with twiddles (3 per complex point)
    assert bench.fft_fp64_instr_per_point(512, dct=False) == 13.5
    # n = 96 = 4^2 * 2 * 3: 4 + 6 + 3 + 20/3 per complex point
    assert bench.fft_fp64_instr_per_point(96, dct=False) == pytest.approx((4 + 6 + 3 + 20 / 3) / 2 + 1)


def test_fp64_mode_path_totals():
    per = bench.algorithmic_per_point(256, 256, mixed=False)
    ins = bench.fp64_instr_per_point(256, 256, 0, 0, mixed=False)
    assert sum(v[0] for v in per.values()) == 224
    assert sum(ins.values()) == 82  # 19 + (6 + 12) + 12 + 3 + 12 + 12 + 6
    r = bench.path_roofline(1e9, 256, 256, 0, 0, False, 0, 6504.1, 0.625e12)
    assert r["bytes_per_pt"] == 224 and r["fp64_instr_per_pt"] == 82
    assert r["hbm_gbs"] == pytest.approx(224.0)
    assert r["fp64_issue_frac"] == pytest.approx(82e9 / 0.625e12)


def test_mixed_path_counts_each_sweep():
    one = bench.path_roofline(1e9, 256, 256, 0, 0, True, 1, 6504.1, 0.6e12)
    two = bench.path_roofline(1e9, 256, 256, 0, 0, True, 2, 6504.1, 0.6e12)
    none = bench.path_roofline(1e9, 256, 256, 0, 0, True, 0, 6504.1, 0.6e12)
    per = bench.algorithmic_per_point(256, 256, mixed=True)
    sweep = sum(per[k][0] for k in ("fwd_x_refine", "fwd_y_refine", "thomas_refine",
                                    "inv_y_refine", "inv_x_update", "resid_correct"))
    assert two["bytes_per_pt"] - one["bytes_per_pt"] == sweep
    # with no sweep the stand-alone correction runs instead of the fused one
    assert one["bytes_per_pt"] - none["bytes_per_pt"] == sweep - per["correct"][0]
    # mixed: double-float flux (7), divergence (1) and first residual (0)
    assert one["fp64_instr_per_pt"] == 7 + 1 + 0 + 1 + 6
    assert none["fp64_instr_per_pt"] == 7 + 1 + 0 + 6
    assert one["io_floor_bytes_per_pt"] == 80


def test_dominant_roofline_against_measured_dfma_rate():
    """The dominant kernel's roofline divides by the DFMA issue rate measured
    in the run: an FP64-mode flux launch is "alu", its flop fraction is the
    algorithmic flops over twice that rate, and its issue fraction the
    counted FP64 instructions over the rate itself."""
    from paper_2502_04189_b300 import inputs as I
    spec = I.bubbles256_spec()
    n = spec.nx * spec.ny * spec.nz
    dfma = 0.6e12
    t_ms = 0.6  # per launch
    st = {"iterations": 1}
    r = bench.dominant_roofline("flux", (t_ms * 20, 20), st, 20, False, 4, spec, n, 6504.1, "m", dfma,
                                "no-such-workload")
    assert r["bound"] == "alu" and r["kernel"] == "flux"
    assert r["achieved"] == pytest.approx(32 * n / (t_ms * 1e-3) / 1e12)
    assert r["peak"] == pytest.approx(2 * dfma / 1e12)
    assert r["fp64_issue"]["frac"] == pytest.approx(19 * n / (t_ms * 1e-3) / dfma)
    assert r["hbm_gbs"] == pytest.approx(72 * n / (t_ms * 1e-3) / 1e9)
    assert r["traffic"] is None
    # the mixed plans' double-float flux reports against HBM, its 7 FP64
    # instructions per point beside it
    r = bench.dominant_roofline("flux", (t_ms * 20, 20), st, 20, True, 4, spec, n, 6504.1, "m", dfma,
                                "no-such-workload")
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(72 * n / (t_ms * 1e-3) / 1e9 / 6504.1)
    assert r["fp64_issue"]["frac"] == pytest.approx(7 * n / (t_ms * 1e-3) / dfma)
    # a refinement kernel counts only the launches of sweeps that ran
    r2 = bench.dominant_roofline("thomas_refine", (1.0, 80), st, 20, True, 4, spec, n, 6504.1, "m",
                                 dfma, "no-such-workload")
    assert r2["bound"] == "hbm" and r2["launches_timed"] == 20
