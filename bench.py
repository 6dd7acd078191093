#!/usr/bin/env python3
"""Benchmark of the variable-density pressure-correction projection on B300.

Metric: grid points per second of one projection (right-hand side, FFT/DCT +
z-tridiagonal Poisson solve, variable-density correction), mixed FP32/FP64
refinement against the plain FP64 form on the same inputs, both refined or
solved to a relative residual of 1e-10.  Default workload: 512^3 cells,
periodic x/y, walls in z with tanh-stretched spacing (beta = 1.5), 400 drops
of radius 6 cells, density ratio 1000, k^-5/3 solenoidal u* (rms 1) plus 1 %
noise, two 8-mode pressure fields, dt = 1e-4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fizzy|reference]
                  [--workload NAME] [--precision mixed|fp64]

Every timed solve starts from the workload's u* (restored from a pristine
device copy before each solve, outside the solve's CUDA events).  The line
states the error of both results against the FP64 CPU oracle on the same
inputs, the roofline of the dominant kernel against peaks measured in the
same run, the oracle's own throughput on the host cores, an end-to-end
number through the host-buffer entry point, and short runs of the 64-instance
uneven batch and of the serving loop.

One JSON line is printed by rank 0.  Under torchrun every rank runs an
independent replica on its own GPU (the projection does not shard in this
build), so scaling is weak and value = points of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_04189_b300 import inputs as I  # noqa: E402

METRIC = "grid pts/s per projection, mixed vs FP64 at 1e-10 residual; HBM %; p50/p99 ms"
HBM_PEAK_FALLBACK = 6400.0        # GB/s, recipe fallback
FP64_PEAK_NOMINAL = 1.25          # TFLOP/s, nominal B300 FP64 (recipe table), context only
# FP64 instructions one SM's FP64 pipe completes per clock when it is always
# busy: the nominal 1.25 TFLOP/s over 148 SMs at about 2.1 GHz.  ncu agrees
# on this part: the in-run probe's 0.506 T instr/s at 2032 MHz is 84.2 % FP64
# pipe activity and k_flux's 0.524 T/s is 89.4 %, both 0.601 T/s = 2 x 148 x
# 2.032 GHz at 100 % (profiles/fp64_pipe_probe_and_flux.md).
FP64_PER_CLK_PER_SM = 2

WORKLOADS = {
    "bubbles512_stretched": I.bubbles512_stretched_spec,
    "bubbles384_stretched": I.bubbles384_stretched_spec,
    "bubbles256": I.bubbles256_spec,
    "drop32": I.drop32_spec,
    "emulsion256": I.emulsion256_spec,
}
DEFAULT_WORKLOAD = "bubbles512_stretched"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def measured_traffic(workload, precision, kernel):
    """DRAM bytes per grid point of one launch of a kernel, from the committed
    ncu summaries: lines 'traffic_per_point <workload> <precision> <kernel>
    <bytes per point> <captured grid>' in profiles/*.md.  Returns (bytes per
    point, source) or (None, None)."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.split()
            if (len(parts) >= 5 and parts[0] == "traffic_per_point" and parts[1] == workload
                    and parts[2] == precision and parts[3] == kernel):
                src = "%s (ncu capture%s)" % (os.path.basename(path),
                                              ", " + parts[5] if len(parts) > 5 else "")
                return float(parts[4]), src
    return None, None


def algorithmic_per_point(nx, ny, mixed):
    """Algorithmic HBM bytes and flops (FMA = 2) per grid point of each
    kernel of one projection (the stencil's flops for the mixed residuals,
    which evaluate it in double-float on the FP32 pipe).  Transform passes use the conventional real-FFT
    count 2.5 log2(n) flops per point (FP64 passes only).  The split-term flux
    counts 32: per face t, s', the Newton quotient (2 FMA), dphat and the
    final FMA (10 flops), times 3, plus phat = 2p^n - p^(n-1)."""
    lx, ly = 2.5 * math.log2(nx), 2.5 * math.log2(ny)
    if not mixed:
        return {
            "flux": (72, 32), "div_fwdx": (32, 8 + lx), "fwd_y": (16, ly), "thomas": (16, 5),
            "inv_y": (16, ly), "inv_x": (16, lx), "correct": (56, 12)}
    return {
        "flux": (72, 32), "div_fwdx": (36, 8), "fwd_y": (8, 0), "thomas": (8, 0), "inv_y": (8, 0),
        "inv_x": (12, 0), "resid": (20, 14), "fwd_x_refine": (8, 0), "fwd_y_refine": (8, 0),
        "thomas_refine": (8, 0), "inv_y_refine": (8, 0), "inv_x_update": (20, 1),
        "resid_correct": (68, 20), "correct": (56, 12)}


def fft_fp64_instr_per_point(n, dct):
    """FP64 instructions per real point of one paired real transform of length
    n, counted from the Stockham stages (radix-4 then 2 then 3; a stage of span
    1 has no twiddles): radix-4 16 adds or 24 FMAs per butterfly, radix-2 4 or
    6, radix-3 12 or 20; two real lines share each complex point.  The
    separation adds 1 per real point, the DCT post-twiddle 2 more."""
    rad = []
    m = n
    for r in (4, 2, 3):
        while m % r == 0:
            rad.append(r)
            m //= r
    first = {4: 16 / 4, 2: 4 / 2, 3: 12 / 3}
    later = {4: 24 / 4, 2: 6 / 2, 3: 20 / 3}
    per_complex = sum(first[r] if i == 0 else later[r] for i, r in enumerate(rad))
    return per_complex / 2 + 1 + (2 if dct else 0)


def fp64_instr_per_point(nx, ny, bcx, bcy, mixed, bcz=1):
    """FP64 instructions per grid point of each kernel, counted from the code
    (flux 6 per face + phat; divergence 6; z-solve 3, or 5 with periodic z
    (the Sherman-Morrison dot product and correction); correction 6).  Mixed
    plans run the flux's density factor, the first x-pass's divergence and
    the residuals in double-float on the FP32 pipe: the flux keeps phat (1
    per cell) and 2 per face (the phat difference and the multiply-add;
    kappa is merged into a double with integer operations), the divergence
    1 (f moved to FP64), the first residual none, and the one fused with the
    correction 2 per face (the FP64 difference of p, the multiply-add)."""
    fx = fft_fp64_instr_per_point(nx, bcx == 1)
    fy = fft_fp64_instr_per_point(ny, bcy == 1)
    if not mixed:
        return {"flux": 19, "div_fwdx": 6 + fx, "fwd_y": fy, "thomas": 5 if bcz == 0 else 3, "inv_y": fy,
                "inv_x": fx, "correct": 6}
    return {"flux": 7, "div_fwdx": 1, "resid": 0, "resid_correct": 6, "inv_x_update": 1,
            "correct": 6}


def path_roofline(value, nx, ny, bcx, bcy, mixed, sweeps, hbm_peak, fp64_issue_peak, bcz=1,
                  fused_xy=False):
    """The whole projection against its bounds: the algorithmic bytes of the
    pass sequence (the kernels' per-point bytes summed over the passes that
    ran; mixed: the refinement passes once per sweep, the stand-alone
    correction only when no sweep ran), the I/O floor (6 FP64 fields read,
    4 written: 80 B/pt), and the FP64 instructions per point against the
    FP64 issue peak.  fused_xy: the mixed solve's x and y passes run fused on
    clusters, so the separate y-passes' bytes are not moved."""
    per = algorithmic_per_point(nx, ny, mixed)
    if mixed and fused_xy:
        for k in ("fwd_y", "inv_y", "fwd_y_refine", "inv_y_refine"):
            per[k] = (0, 0)
    ins = fp64_instr_per_point(nx, ny, bcx, bcy, mixed, bcz)
    if not mixed:
        b = sum(v[0] for v in per.values())
        n_ins = sum(ins.values())
    else:
        once = ("flux", "div_fwdx", "fwd_y", "thomas", "inv_y", "inv_x", "resid")
        sweep = ("fwd_x_refine", "fwd_y_refine", "thomas_refine", "inv_y_refine", "inv_x_update",
                 "resid_correct")
        b = sum(per[k][0] for k in once) + sweeps * sum(per[k][0] for k in sweep)
        n_ins = ins["flux"] + ins["div_fwdx"] + ins["resid"] + sweeps * (ins["inv_x_update"] +
                                                                       ins["resid_correct"])
        if sweeps == 0:
            b += per["correct"][0]
            n_ins += ins["correct"]
    return {"bytes_per_pt": b, "io_floor_bytes_per_pt": 80, "hbm_gbs": value * b / 1e9,
            "hbm_frac": value * b / 1e9 / hbm_peak, "io_floor_frac": value * 80 / 1e9 / hbm_peak,
            "fp64_instr_per_pt": n_ins, "fp64_issue_peak_instr_s": fp64_issue_peak,
            "fp64_issue_bound_pts_s": fp64_issue_peak / n_ins,
            "fp64_issue_frac": value * n_ins / fp64_issue_peak, "sweeps": sweeps}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((int(parts[0]), float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        # the busiest GPU is ours
        by_gpu = {}
        for r in rows:
            by_gpu.setdefault(r[0], []).append(r)
        gid = max(by_gpu, key=lambda g: np.mean([r[3] for r in by_gpu[g]]))
        rs = by_gpu[gid]
        loaded = [r for r in rs if r[3] > 200.0] or rs
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in loaded:
            for nm, val in zip(names[1:], r[4][1:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median([r[1] for r in loaded])),
                "sm_max_mhz": float(max(r[2] for r in rs)),
                "power_w_max": float(max(r[3] for r in rs)),
                "samples": len(loaded), "reasons": sorted(reasons)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def slowest_rank(seconds, dist, device="cuda"):
    """The job time of N replicas: the maximum over ranks of each rank's time
    (every rank projects its own batch; no data-path collective)."""
    if not dist:
        return seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank_step, steps, world, seconds):
    """Whole-job points per second: all ranks' points over the slowest time."""
    return points_per_rank_step * steps * world / seconds


def slab_spec(spec, nz=32):
    """A bounded sample of a workload: the same recipe on a slab of nz planes
    (same x/y transform lengths and spacing, z length and drop count scaled;
    a stretched z keeps its tanh law over the slab)."""
    k = min(spec.nz, nz)
    return I.CaseSpec(**{**spec.__dict__, "nz": k, "lz": spec.lz * k / spec.nz,
                         "n_bubbles": max(1, spec.n_bubbles * k // spec.nz)})


def oracle_time(case, reps=1):
    """Wall time of the CPU oracle's projection on case (rank 0 host cores);
    returns (best seconds, threads, the last result)."""
    import oracle as O
    best, res = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        res = O.project_case(case)
        best.append(time.perf_counter() - t0)
    return min(best), O.num_threads(), res


def errors_vs_oracle(case, got, ref):
    """spec error definitions: max|x - x_oracle| / max|x_oracle| for p
    (the dzf-weighted mean removed on both sides) and for u, v, w together
    (one shared max); plus the divergence metric max|D u| dx / U of the
    result, U the rms of u* over all faces, evaluated by the oracle's D."""
    import oracle as O
    g = O.Grid.of_case(case)
    pg = got["p"] - O.weighted_mean(g, got["p"])
    pr = ref["p"] - O.weighted_mean(g, ref["p"])
    ep = float(np.max(np.abs(pg - pr)) / np.max(np.abs(pr)))
    num = max(float(np.max(np.abs(got[k] - ref[k]))) for k in "uvw")
    den = max(float(np.max(np.abs(ref[k]))) for k in "uvw")
    U = math.sqrt(sum(float(np.sum(getattr(case, k) ** 2)) for k in "uvw") / (3 * case.npts))
    dmax = float(np.max(np.abs(O.div(g, got["u"], got["v"], got["w"]))))
    return {"p": ep, "u": num / den, "div_metric": dmax * case.dx / U}


PROBE_VARIANTS = (  # name, precision (0 FP64, 1 FP32), op (see fizzy_probe_fma_rate), chains
    ("dfma_8", 0, 0, 8), ("dfma_16", 0, 0, 16), ("dadd_8", 0, 1, 8), ("dmul_8", 0, 2, 8),
    ("dfma_dadd_8", 0, 3, 8), ("dfma_with_ffma_8", 0, 4, 8), ("dfma_reg_8", 0, 5, 8),
    ("ffma_8", 1, 0, 8))


def probe_peaks(F, stream, target_ms=120.0):
    """In-run issue-rate probes (fizzy_probe_fma_rate): FP64 chains of
    multiply-adds, adds, multiplies, both in turn, multiply-adds interleaved
    with FP32 work and with register multiplicands, and FP32 multiply-add
    chains; a resident grid, each launch calibrated to about target_ms, best
    of two, with the SM clock sampled during the probes.  The FP64 issue peak
    is the highest FP64 variant."""
    out = {}
    clocks = ClockSampler()
    clocks.start()
    for name, prec, op, ch in PROBE_VARIANTS:
        it0 = 500 if prec == 0 else 20000
        _, ms = F.probe_fma_rate(prec, it0, op=op, chains=ch, stream=stream)
        it = max(1, int(it0 * target_ms / max(ms, 1e-3)))
        rate, ms = max(F.probe_fma_rate(prec, it, op=op, chains=ch, stream=stream) for _ in range(2))
        out[name] = {"instr_per_s": rate, "ms": ms, "iters": it}
    out["clocks"] = clocks.stop()
    best = max((k for k in out if k.startswith("d")), key=lambda k: out[k]["instr_per_s"])
    out["fp64_issue_peak"] = {"instr_per_s": out[best]["instr_per_s"], "variant": best}
    return out


def run_reference(args):
    """The oracle on the host cores: each step = one projection of a 32-plane
    slab drawn with the workload's recipe (same x/y transform lengths and
    spacing)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    spec = WORKLOADS[args.workload]()
    sample_spec = slab_spec(spec)
    case = I.make_case(sample_spec)
    for _ in range(args.warmup):
        O.project_case(case)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.project_case(case)
    dt = time.perf_counter() - t0
    pts = case.npts * args.steps
    value = pts / dt
    sample = "%dx%dx%d slab of the %s recipe per step" % (sample_spec.nx, sample_spec.ny, sample_spec.nz,
                                                          args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "grid": [spec.nx, spec.ny, spec.nz],
                                             "precision": args.precision,
                                             "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def dominant_roofline(dom, live, st, steps, mixed, max_refine, spec, npts, hbm_peak, hbm_src,
                      dfma, workload):
    """Roofline object of the dominant kernel from its live CUDA-event time in
    the timed region.  FP64-bound kernels report "alu": algorithmic FP64 flops
    (FMA = 2) per launch over the launch time, against twice the DFMA issue
    rate measured in the same run; the FP64 instruction rate against that
    issue rate and the HBM rate against the measured copy bandwidth sit
    beside it.  The mixed plans' double-float kernels (flux, first x-pass,
    residuals) do most of their arithmetic on the FP32 pipe, so they report
    against HBM, with their remaining FP64 instructions beside it."""
    tot_ms, cnt = live
    # refinement kernels return at once after convergence: count only the
    # launches that did the pass (from the solve's sweep count)
    it = st["iterations"]
    per_solve = {"fwd_x_refine": it, "fwd_y_refine": it, "thomas_refine": it,
                 "inv_y_refine": it, "inv_x_update": it, "resid_correct": it}.get(dom)
    if mixed and dom == "correct":  # runs only when no fused pass ran
        per_solve = 1 if it == 0 else 0
    if per_solve is not None:
        cnt = max(1, per_solve * steps)
    avg_s = tot_ms / cnt / 1e3
    per_pt = algorithmic_per_point(spec.nx, spec.ny, mixed)
    b_pt, fl_pt = per_pt.get(dom, (0, 0))
    ipt = fp64_instr_per_point(spec.nx, spec.ny, spec.bcx, spec.bcy, mixed, spec.bcz).get(dom, 0)
    gbs = b_pt * npts / avg_s / 1e9
    tpt, tsrc = measured_traffic(workload, "mixed" if mixed else "fp64", dom)
    traffic = tpt * npts if tpt is not None else None
    issue = ipt * npts / avg_s
    df_kernel = mixed and dom in ("flux", "div_fwdx", "resid", "resid_correct")
    if ipt and not df_kernel and ipt / dfma > b_pt / (hbm_peak * 1e9):
        peak = 2.0 * dfma / 1e12
        tfl = fl_pt * npts / avg_s / 1e12
        roof = {"bound": "alu", "achieved": tfl, "peak": peak, "unit": "TFLOP/s", "frac": tfl / peak,
                "peak_source": "FP64 pipe at full rate: 2 FP64 instructions per clock per SM x SMs x "
                               "the median SM clock of the timed region, FMA = 2 flops (the in-run "
                               "probes and ncu's FP64-pipe activity corroborate it: peaks_measured)",
                "nominal_peak": FP64_PEAK_NOMINAL}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "peak_source": hbm_src}
    roof.update({"traffic": traffic, "traffic_source": tsrc, "kernel": dom,
                 "algorithmic_bytes": b_pt * npts, "algorithmic_fp64_flops": fl_pt * npts,
                 "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "hbm_peak_source": hbm_src,
                 "launches_timed": cnt, "duration_ms": tot_ms / cnt})
    if ipt:
        roof["fp64_issue"] = {"instr_per_pt": ipt, "achieved": issue / 1e12, "peak": dfma / 1e12,
                              "unit": "T instr/s", "frac": issue / dfma,
                              "peak_source": "FP64 pipe at full rate (2 / clock / SM at the sampled clock)"}
    return roof


def run_batch_forms(args, F, torch, steps, warmup, reps=3):
    """The 64-instance uneven batch: the mixed batched form (one persistent
    launch replayed from a CUDA graph, autotuned), the FP64 batched form and
    the plain FP64 form (one fizzy_proj_solve per instance).  Each instance's
    outputs are checked against its own plain FP64 solve (max relative p error
    with the gauge removed, and u error)."""
    specs = I.batch_specs(64)
    cases = [I.make_case(s) for s in specs]
    npts = sum(c.npts for c in cases)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    inputs = [(dev(c.phi), dev(c.pn), dev(c.pnm1)) for c in cases]
    ustar = [(dev(c.u), dev(c.v), dev(c.w)) for c in cases]
    work = [tuple(torch.empty_like(t) for t in us) for us in ustar]
    outs = [torch.empty(c.shape, dtype=torch.float64, device="cuda") for c in cases]
    stream = torch.cuda.current_stream()

    def restore():
        for wk, us in zip(work, ustar):
            for a, b in zip(wk, us):
                a.copy_(b)

    def results():
        return [(o.clone(), *[t.clone() for t in wk]) for o, wk in zip(outs, work)]

    forms = {}
    finals = {}
    for prec, name in ((F.MIXED, "mixed_batched"), (F.FP64, "fp64_batched")):
        plans = [F.Plan.for_case(c, precision=prec) for c in cases]
        arrays = [inp + wk + (o,) for inp, wk, o in zip(inputs, work, outs)]
        batch = F.Batch(plans, arrays)
        restore()
        tuning, tuned_ms = batch.autotune(reps=reps)
        for _ in range(warmup):
            restore()
            batch.solve()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / steps
        status = batch.status()
        st = [p.stats() for p in plans]
        finals[name] = results()
        forms[name] = {"value": npts / (ms / 1e3), "ms_per_batch": ms, "tuning": tuning,
                       "status": status, "items": batch.info()["items"],
                       "max_relres": max(x["relres"] for x in st),
                       "sweeps_max": max(x["iterations"] for x in st) if prec == F.MIXED else 0,
                       "all_converged": all(x["converged"] for x in st)}
        batch.close()
        for p in plans:
            p.close()
    # plain FP64 form: one stand-alone solve per instance
    plans = [F.Plan.for_case(c, precision=F.FP64) for c in cases]

    def plain():
        for pl, inp, wk, o in zip(plans, inputs, work, outs):
            pl.solve(*inp, *wk, o)
    for _ in range(warmup):
        restore()
        plain()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / steps
    ref = results()
    forms["fp64_plain_loop"] = {"value": npts / (ms / 1e3), "ms_per_batch": ms}
    for p in plans:
        p.close()
    # accuracy of the batched forms against the plain FP64 solves
    for name in ("mixed_batched", "fp64_batched"):
        ep = eu = 0.0
        for (pb, ub, vb, wb), (pr, ur, vr, wr) in zip(finals[name], ref):
            pb = pb - pb.mean()
            pr = pr - pr.mean()  # uniform cells here: the plain mean is the gauge difference
            ep = max(ep, float((pb - pr).abs().max() / pr.abs().max()))
            m = max(float(t.abs().max()) for t in (ur, vr, wr))
            eu = max(eu, max(float((a - b).abs().max()) for a, b in ((ub, ur), (vb, vr), (wb, wr))) / m)
        forms[name]["err_vs_plain_fp64"] = {"p": ep, "u": eu}
    return {"instances": len(cases), "points": npts, "forms": forms,
            "mixed_over_plain_fp64": forms["mixed_batched"]["value"] / forms["fp64_plain_loop"]["value"]}


def run_serve_loop(args, F, torch, n_requests, slots):
    """Serving: Poisson arrivals (seeded, mean 2000 req/s) of requests with
    nx, ny in {64,...,384}, nz in [64, 384], 30 % tanh-stretched z, periodic
    or wall x/y, density ratio 10-1000, mixed precision refined to 1e-10;
    admission by a 120 GB HBM budget with plans cached on the device, 100 ms
    admission deadline.  Inputs are periodic crops of a device-resident
    256^3 bubble template."""
    import paper_2502_04189_b300.serve as S
    arrivals, specs = I.serve_specs(n_requests)
    tmpl = I.make_case(I.bubbles256_spec())
    fields = S.TemplateFields(tmpl)
    reqs = S.requests_from_specs(arrivals, specs, F.MIXED)
    server = F.Server(120 * (1 << 30), slots=slots)

    def fill(r, views, stream):
        fields.fill(views, r.desc, r.offset, stream)

    # warm-up on a few requests (plan-building code paths, pool growth)
    S.run(server, [S.Request(i, 0.0, r.desc, r.offset) for i, r in enumerate(reqs[:4])], fill,
          deadline=60.0)
    torch.cuda.synchronize()
    out, summ = S.run(server, reqs, fill, deadline=0.1)
    info = server.info()
    server.close()
    del fields
    return summ, info


SMALL_PTS = 128 ** 3  # serving size classes: small <= 128^3 points < large


def run_serve_classes(args, F, torch, slots, n_small=1500, n_large=300):
    """Service capacity by request size: the request recipe's small
    (<= 128^3 points) and large requests served as two separate backlogs
    (every request queued at t = 0, no deadline), so the server stays busy
    and points / wall time is the class's throughput.  Each backlog is served
    once untimed first, so the timed pass finds every plan of the class in
    the server's device-resident cache (the steady state of a server whose
    request grids recur; the Poisson run above builds plans as grids first
    arrive).  The ratio small/large says how well small requests use the
    GPU."""
    import paper_2502_04189_b300.serve as S
    arrivals, specs = I.serve_specs(8 * (n_small + n_large))
    small = [s for s in specs if s.nx * s.ny * s.nz <= SMALL_PTS][:n_small]
    large = [s for s in specs if s.nx * s.ny * s.nz > SMALL_PTS][:n_large]
    tmpl = I.make_case(I.bubbles256_spec())
    fields = S.TemplateFields(tmpl)
    server = F.Server(120 * (1 << 30), slots=slots)

    def fill(r, views, stream):
        fields.fill(views, r.desc, r.offset, stream)

    out = {"split_pts": SMALL_PTS, "slots": slots}
    for name, cls in (("small", small), ("large", large)):
        reqs = S.requests_from_specs([0.0] * len(cls), cls, F.MIXED)
        S.run(server, reqs, fill, deadline=60.0)  # every plan of the class cached, pool warm
        torch.cuda.synchronize()
        _, summ = S.run(server, reqs, fill, deadline=60.0)
        out[name] = {"requests": summ["requests"], "mean_pts": summ["points_done"] / max(1, summ["admitted"]),
                     "throughput_pts_s": summ["throughput_pts_s"], "wall_s": summ["wall_s"],
                     "all_converged": summ["all_converged"]}
    out["small_over_large"] = out["small"]["throughput_pts_s"] / out["large"]["throughput_pts_s"]
    server.close()
    del fields
    return out


def run_fizzy(args):
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec = WORKLOADS[args.workload]()
    if args.nz:
        spec = slab_spec(spec, args.nz)
    case = I.make_case(spec)
    npts = case.npts
    prec = F.MIXED if args.precision == "mixed" else F.FP64
    other = F.FP64 if prec == F.MIXED else F.MIXED
    mixed = prec == F.MIXED

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    phi, pn, pnm1 = dev(case.phi), dev(case.pn), dev(case.pnm1)
    u0, v0, w0 = dev(case.u), dev(case.v), dev(case.w)  # the workload's u*, kept pristine
    u, v, w = torch.empty_like(u0), torch.empty_like(v0), torch.empty_like(w0)
    p = torch.empty_like(phi)
    stream = torch.cuda.current_stream()

    def restore():
        u.copy_(u0)
        v.copy_(v0)
        w.copy_(w0)

    # peaks of this GPU, measured before the timed region
    peaks = probe_peaks(F, stream) if not args.no_probe else None
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count

    def timed_run(precision, steps, warmup, per_kernel):
        """W warm-up solves; with per_kernel, a short breakdown run with every
        kernel bracketed by events picks the dominant kernel; then the timed
        region of `steps` solves, each from the restored u* and bracketed by
        its own CUDA events, in which only the dominant kernel's launches also
        carry events (its live average duration feeds the roofline)."""
        plan = F.Plan.for_case(case, precision=precision, fused_xy=args.fused_xy)
        for _ in range(warmup):
            restore()
            plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
        torch.cuda.synchronize()
        breakdown, dom = {}, None
        if per_kernel:
            plan.set_timing(True)
            for _ in range(3):
                restore()
                plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
            breakdown = plan.timing()
            dom = max(breakdown, key=lambda k: breakdown[k][0])
            plan.set_timing(True, only=dom)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for e0, e1 in evs:
            restore()
            e0.record(stream)
            plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        per = [e0.elapsed_time(e1) for e0, e1 in evs]
        live = plan.timing().get(dom) if dom else None
        st = plan.stats(stream)
        launches = plan.launches_per_solve() * steps
        mr = plan.max_refine
        plan.close()
        # the last solve started from the workload's u*: its outputs
        out = {"p": p.cpu().numpy(), "u": u.cpu().numpy(), "v": v.cpu().numpy(), "w": w.cpu().numpy()}
        return {"ms": sum(per), "ms_each": per, "wall_s": wall, "breakdown": breakdown, "dom": dom,
                "live": live, "stats": st, "launches": launches, "max_refine": mr, "out": out}

    clocks = ClockSampler()
    clocks.start()
    R = timed_run(prec, args.steps, args.warmup, True)
    clk = clocks.stop()
    # the FP64 pipe's full rate at the SM clock of the timed region
    sm_hz = (clk["sm_mhz"] if clk else 2032.0) * 1e6
    dfma = FP64_PER_CLK_PER_SM * n_sm * sm_hz
    ms = slowest_rank(R["ms"], dist)
    value = job_throughput(npts, args.steps, world, ms / 1e3)
    st = R["stats"]

    # the other precision on the same inputs (the "mixed vs FP64" comparison)
    k_o = max(3, args.steps // 4)
    Ro = timed_run(other, k_o, args.warmup, False)
    value_o = npts * k_o / (Ro["ms"] / 1e3)

    hbm_peak, hbm_src = measured_peaks()
    roof = None
    if R["dom"] and R["live"]:
        roof = dominant_roofline(R["dom"], R["live"], st, args.steps, mixed, R["max_refine"], spec, npts,
                                 hbm_peak, hbm_src, dfma, args.workload if not args.nz else None)
    kern = R["breakdown"]
    kernels = {k: {"ms_avg": v[0] / v[1], "launches": v[1],
                   "share": v[0] / max(1e-9, sum(x[0] for x in kern.values()))} for k, v in kern.items()}

    # end-to-end through the public host-buffer entry point: pipelined solves
    # (fizzy_proj_solve_host_async) from pinned host inputs to pinned host
    # outputs; every step copies its six inputs in and its four results out
    e2e = None
    if args.e2e_steps > 0:
        plan = F.Plan.for_case(case, precision=prec)
        hin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
               (case.phi, case.pn, case.pnm1, case.u, case.v, case.w)]
        hout = [torch.empty(case.shape, dtype=torch.float64).pin_memory() for _ in range(4)]
        for _ in range(2):
            plan.solve_host_async(*hin, *hout, stream=stream)
        plan.host_wait()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.solve_host_async(*hin, *hout, stream=stream)
        plan.host_wait()
        el = slowest_rank(time.perf_counter() - t0, dist)
        plan.close()
        # the host link's bound for the same bytes: the step's six input copies
        # and four output copies alone, on two streams, with no solve
        devs = [torch.empty(case.shape, dtype=torch.float64, device="cuda") for _ in range(10)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def copies():
            with torch.cuda.stream(s_in):
                for h, d in zip(hin, devs[:6]):
                    d.copy_(h, non_blocking=True)
            with torch.cuda.stream(s_out):
                for h, d in zip(hout, devs[6:]):
                    h.copy_(d, non_blocking=True)
        copies()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            copies()
        torch.cuda.synchronize()
        el_copy = slowest_rank(time.perf_counter() - t0, dist)
        del devs, hin, hout
        e2e = {"value": job_throughput(npts, args.e2e_steps, world, el), "unit": "pts/s",
               "h2d_bytes_per_step": 6 * 8 * npts, "d2h_bytes_per_step": 4 * 8 * npts,
               "ms_per_step": el / args.e2e_steps * 1e3,
               "copies_only_ms_per_step": el_copy / args.e2e_steps * 1e3,
               "link_frac": el_copy / el,
               "api": "fizzy_proj_solve_host_async (pipelined, pinned host arrays)"}
    del phi, pn, pnm1, u0, v0, w0, u, v, w, p
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # the FP64 CPU oracle on the same inputs: its time is the CPU baseline,
    # its result the reference both GPU results are measured against
    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # periodic z: the oracle's dense cyclic z-line solves grow as nz^3, so
        # it runs on a 32-plane slab of the same recipe (errors then unmeasured)
        full = spec.bcz == I.NEUMANN
        ocase = case if full else I.make_case(slab_spec(spec))
        t_or, cores, ref = oracle_time(ocase, reps=1)
        os_ = ocase.spec
        cpu = {"value": ocase.npts / t_or, "unit": "pts/s", "cores": cores, "kind": "oracle",
               "sample": "one full %dx%dx%d projection of the same inputs%s" % (
                   os_.nx, os_.ny, os_.nz, "" if full else " (a 32-plane slab of the workload)"),
               "seconds": t_or}
        if full:
            name_m = "mixed" if mixed else "fp64"
            name_o = "fp64" if mixed else "mixed"
            err = {name_m: errors_vs_oracle(case, R["out"], ref),
                   name_o: errors_vs_oracle(case, Ro["out"], ref),
                   "definition": "max|x - x_oracle| / max|x_oracle|; p with the dzf-weighted mean "
                                 "removed on both sides; u, v, w with one shared max; div_metric = "
                                 "max|D u| dx / rms(u*)",
                   "bars": {"fp64": 1e-12, "mixed": 1e-9, "div_metric": 1e-10}}
        del ref
    R["out"] = Ro["out"] = None

    batch = serve = None
    if rank == 0 and not args.no_sub:
        batch = run_batch_forms(args, F, torch, steps=5, warmup=2, reps=2)
        torch.cuda.empty_cache()
        summ, info = run_serve_loop(args, F, torch, args.sub_serve_requests, args.serve_slots)
        serve = {"requests": summ["requests"], "arrival_rate_per_s": 2000, "budget_gb": 120,
                 "slots": args.serve_slots, "deadline_ms": 100, "throughput_pts_s": summ["throughput_pts_s"],
                 "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"],
                 "rejected_fraction": summ["rejected_fraction"], "requests_per_s": summ["requests_per_s"],
                 "all_converged": summ["all_converged"], "max_relres": summ["max_relres"],
                 "plans_built": info.get("plans_built")}
        torch.cuda.empty_cache()
        serve["by_size"] = run_serve_classes(args, F, torch, args.serve_slots)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if mixed else "f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "grid": [spec.nx, spec.ny, spec.nz],
                           "precision": args.precision, "tol": 1e-10,
                           "z_stretch_beta": spec.beta,
                           "bc": "%s x, %s y, %s z" % tuple(
                               "periodic" if b == I.PERIODIC else "walls" for b in (spec.bcx, spec.bcy, spec.bcz)),
                           "l2": "inputs (6 x %d MiB) larger than L2" % (npts * 8 >> 20),
                           "timing": "each solve from the workload's u*, restored from a pristine device "
                                     "copy before it, outside its own CUDA events; value = points / sum "
                                     "of the solves' event times",
                           "fused_xy_passes": bool(args.fused_xy),
                           "parallelism": "replicas" if world > 1 else "single"},
                "gpu_launches": R["launches"], "roofline": roof,
                "path_roofline": path_roofline(value, spec.nx, spec.ny, spec.bcx, spec.bcy, mixed,
                                               int(st["iterations"]), hbm_peak, dfma, spec.bcz,
                                               fused_xy=mixed and "fwd_y" not in R["breakdown"]),
                "fused_xy": mixed and "fwd_y" not in R["breakdown"],
                "peaks_measured": dict(peaks or {}, fp64_pipe_full_rate_instr_s=dfma, n_sm=n_sm,
                                       probe_over_pipe=(peaks["fp64_issue_peak"]["instr_per_s"] / dfma)
                                       if peaks else None),
                "err_vs_oracle": err,
                "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "kernels": kernels,
                "stats": {k: st[k] for k in ("iterations", "converged", "relres")},
                "timed_wall_s_incl_restores": R["wall_s"],
                ("fp64" if mixed else "mixed"): {
                    "value": value_o, "unit": "pts/s", "ms_per_step": Ro["ms"] / k_o, "steps": k_o,
                    "iterations": Ro["stats"]["iterations"], "relres": Ro["stats"]["relres"]},
                "mixed_over_fp64": (value / value_o) if mixed else (value_o / value),
                "batch64": batch, "serve": serve}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Uneven batch alone: 64 projections (nx, ny in {32..192}, nz in
    [32, 192], periodic or wall x/y, 1-20 drops, density ratio 10-1000),
    mixed precision, one persistent launch replayed from a CUDA graph with
    autotuned tiles; compared with the plain FP64 form (one fizzy_proj_solve
    per instance)."""
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    res = run_batch_forms(args, F, torch, steps=args.steps, warmup=args.warmup, reps=3)
    if rank == 0:
        r = res["forms"]["mixed_batched"]
        line = {"metric": METRIC, "value": r["value"], "unit": "pts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "batch64", "instances": res["instances"], "points": res["points"],
                           "precision": "mixed", "tol": 1e-10},
                "forms": res["forms"], "mixed_over_plain_fp64": res["mixed_over_plain_fp64"]}
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving alone (see run_serve_loop) with nvidia-smi clock sampling."""
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    clocks = ClockSampler()
    clocks.start()
    summ, info = run_serve_loop(args, F, torch, args.serve_requests, args.serve_slots)
    by_size = run_serve_classes(args, F, torch, args.serve_slots)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": METRIC, "value": summ["throughput_pts_s"], "unit": "pts/s",
                "n_gpus": world, "steps": summ["requests"], "warmup": 4, "ms_per_step": summ["mean_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "serve", "arrival_rate_per_s": 2000,
                           "requests": summ["requests"], "budget_gb": 120, "slots": args.serve_slots,
                           "deadline_ms": 100, "precision": "mixed", "tol": 1e-10},
                "serving": summ, "server": info, "by_size": by_size, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def run_vc(args):
    """The variable-coefficient projection without splitting
    (fizzy_proj_solve_vc, conjugate gradients preconditioned with the
    constant-coefficient solve) on a workload, next to the split projection:
    time per projection, CG iterations, and the splitting's effect on u
    (max|u_vc - u_split| / max|u_split|)."""
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    spec = WORKLOADS[args.workload]()
    case = I.make_case(spec)
    npts = case.npts

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    phi = dev(case.phi)
    prec = F.MIXED if args.precision == "mixed" else F.FP64  # mixed: FP32 preconditioner
    plan = F.Plan.for_case(case, precision=prec)
    p = torch.empty_like(phi)
    stream = torch.cuda.current_stream()
    times, st = [], None
    clocks = ClockSampler()
    clocks.start()
    for i in range(args.warmup + args.steps):
        u, v, w = dev(case.u), dev(case.v), dev(case.w)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = plan.solve_vc(phi, u, v, w, p, max_iter=5000, tol=args.vc_tol)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    uvc = torch.cat([u.flatten(), v.flatten(), w.flatten()])
    us, vs_, ws = dev(case.u), dev(case.v), dev(case.w)
    plan.solve(phi, dev(case.pn), dev(case.pnm1), us, vs_, ws, torch.empty_like(phi))
    usp = torch.cat([us.flatten(), vs_.flatten(), ws.flatten()])
    split_diff = float((uvc - usp).abs().max() / usp.abs().max())
    # the split scheme with phat = the unsplit p returns that p (fixed point)
    us, vs_, ws = dev(case.u), dev(case.v), dev(case.w)
    pf = torch.empty_like(phi)
    plan.solve(phi, p, p, us, vs_, ws, pf)
    ufp = torch.cat([us.flatten(), vs_.flatten(), ws.flatten()])
    fixed_point_diff = float((uvc - ufp).abs().max() / uvc.abs().max())
    plan.close()
    ms = float(np.median(times))
    if rank == 0:
        line = {"metric": METRIC, "value": npts / (ms / 1e3), "unit": "pts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == F.MIXED else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "grid": [spec.nx, spec.ny, spec.nz],
                           "form": "variable-coefficient projection, preconditioned CG",
                           "preconditioner": "FP32 solve, flexible CG" if prec == F.MIXED else "FP64 solve",
                           "tol": args.vc_tol, "density_ratio": max(spec.rho_l, spec.rho_g) / min(spec.rho_l, spec.rho_g)},
                "stats": {k: st[k] for k in ("iterations", "converged", "relres", "div_metric")},
                "ms_per_iteration": ms / max(1, st["iterations"]),
                "splitting_effect_on_u": split_diff,
                "splitting_effect_note": "with the workload's synthetic p^n, p^(n-1), unrelated to the solution",
                "split_fixed_point_diff_u": fixed_point_diff, "clocks": clk,
                "note": "median over steps; each step is one whole solve (host checks every 4 iterations)"}
        print(json.dumps(line), flush=True)
    return 0


def run_acdi(args):
    """One explicit stage of the ACDI phase-field transport (fizzy_acdi_step)
    on a workload: time per stage with inputs resident in HBM, against the
    algorithmic bytes of its four passes (psi and r: 24 B/pt; normals: 32;
    face fluxes: phi, r, 3 normals, u, v, w in, 3 fluxes out = 88; update:
    phi, 3 fluxes in, phi out = 40; 184 B/pt)."""
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    spec = WORKLOADS[args.workload]()
    case = I.make_case(spec)
    npts = case.npts

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    phi, u, v, w = dev(case.phi), dev(case.u), dev(case.v), dev(case.w)
    out = torch.empty_like(phi)
    plan = F.Plan.for_case(case, precision=F.FP64)
    eps, gam, dt = case.dx, 1.0, 1e-4
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.acdi_step(phi, u, v, w, eps, gam, dt, phi_out=out)
    clocks = ClockSampler()
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.acdi_step(phi, u, v, w, eps, gam, dt, phi_out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    plan.close()
    hbm_peak, hbm_src = measured_peaks()
    gbs = 184 * npts / (ms / 1e3) / 1e9
    if rank == 0:
        line = {"metric": "grid pts/s per ACDI stage", "value": npts / (ms / 1e3), "unit": "pts/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "grid": [spec.nx, spec.ny, spec.nz],
                           "form": "ACDI phase-field stage (4 kernels)", "eps": "dx", "gamma": gam},
                "hbm": {"algorithmic_bytes_per_pt": 184, "achieved_gbs": gbs, "peak": hbm_peak,
                        "frac": gbs / hbm_peak, "peak_source": hbm_src},
                "gpu_launches": 4 * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fizzy", choices=["fizzy", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS) + ["batch64", "serve"])
    ap.add_argument("--nz", type=int, default=0,
                    help="run a slab of the workload with this many z planes (profiling captures)")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--sub-serve-requests", type=int, default=1000,
                    help="requests of the serving run embedded in the default line")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the embedded batch and serving runs")
    ap.add_argument("--no-probe", action="store_true", help="skip the FMA-rate probes")
    ap.add_argument("--fused-xy", action="store_true",
                    help="run the cluster-fused x-y FP32 passes (FIZZY_FLAG_FUSED_XY)")
    ap.add_argument("--vc", action="store_true",
                    help="time the variable-coefficient projection without splitting instead")
    ap.add_argument("--vc-tol", type=float, default=1e-10)
    ap.add_argument("--acdi", action="store_true", help="time the ACDI phase-field stage instead")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.vc:
        return run_vc(args)
    if args.acdi:
        return run_acdi(args)
    return run_fizzy(args)


if __name__ == "__main__":
    sys.exit(main())
