#!/usr/bin/env python3
"""Benchmark of the variable-density pressure-correction projection on B300.

Metric: grid points per second of one projection (right-hand side, FFT/DCT +
z-tridiagonal Poisson solve, variable-density correction) on the 256^3
bubble-laden workload: periodic x/y, walls in z, uniform grid, 40 drops of
radius 8 cells, density ratio 1000, k^-5/3 solenoidal u* (rms 1) plus 1 %
noise, two 8-mode pressure fields, dt = 1e-4; FP64 mode (the mixed
FP32/FP64-refinement mode is reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fizzy|reference]

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
FP64_PEAK_NOMINAL = 1.25          # TFLOP/s, nominal B300 FP64 (recipe table)

WORKLOADS = {
    "bubbles256": I.bubbles256_spec,
    "drop32": I.drop32_spec,
    "bubbles512_stretched": I.bubbles512_stretched_spec,
    "emulsion256": I.emulsion256_spec,
}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def measured_traffic(kernel, mixed):
    """DRAM bytes per launch of a kernel from the committed ncu summaries
    (lines 'traffic_per_launch_bytes <kernel> <bytes>' in profiles/*.md)."""
    import glob
    name = {"flux": "k_flux", "resid": "k_resid", "resid_correct": "k_resid_corr",
            "div_fwdx": "k_xfwd_mix" if mixed else "k_xfwd_f64"}.get(kernel, kernel)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.split()
            if len(parts) == 3 and parts[0] == "traffic_per_launch_bytes" and parts[1] == name:
                return int(parts[2])
    return None


def algorithmic_per_point(nx, ny, mixed):
    """Algorithmic HBM bytes and FP64 flops (FMA = 2) per grid point of each
    kernel of one projection.  Transform passes use the conventional real-FFT
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


def path_roofline(value, nx, ny, bcx, bcy, mixed, sweeps, hbm_peak, bcz=1):
    """The whole projection against its bounds: the algorithmic bytes of the
    pass sequence (the kernels' per-point bytes summed over the passes that
    ran; mixed: the refinement passes once per sweep, the stand-alone
    correction only when no sweep ran), the I/O floor (6 FP64 fields read,
    4 written: 80 B/pt), and the FP64 instructions per point against the
    nominal 0.625 T FP64 instructions/s."""
    per = algorithmic_per_point(nx, ny, mixed)
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
    issue_peak = FP64_PEAK_NOMINAL / 2 * 1e12
    return {"bytes_per_pt": b, "io_floor_bytes_per_pt": 80, "hbm_gbs": value * b / 1e9,
            "hbm_frac": value * b / 1e9 / hbm_peak, "io_floor_frac": value * 80 / 1e9 / hbm_peak,
            "fp64_instr_per_pt": n_ins, "fp64_issue_bound_pts_s": issue_peak / n_ins,
            "fp64_issue_frac": value * n_ins / issue_peak, "sweeps": sweeps}


def fp64_instr_per_point(nx, ny, bcx, bcy, mixed, bcz=1):
    """FP64 instructions per grid point of each kernel, counted from the code
    (flux 6 per face + phat; divergence 6; z-solve 3, or 5 with periodic z
    (the Sherman-Morrison dot product and correction); correction 6; mixed
    residual 10, fused with the correction 13)."""
    fx = fft_fp64_instr_per_point(nx, bcx == 1)
    fy = fft_fp64_instr_per_point(ny, bcy == 1)
    if not mixed:
        return {"flux": 19, "div_fwdx": 6 + fx, "fwd_y": fy, "thomas": 5 if bcz == 0 else 3, "inv_y": fy,
                "inv_x": fx, "correct": 6}
    return {"flux": 19, "div_fwdx": 6, "resid": 10, "resid_correct": 13, "inv_x_update": 1,
            "correct": 6}


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
    """A bounded sample of a workload for the CPU oracle: the same recipe on a
    slab of nz planes (same x/y transform lengths and spacing, z length and
    drop count scaled)."""
    k = min(spec.nz, nz)
    return I.CaseSpec(**{**spec.__dict__, "nz": k, "lz": spec.lz * k / spec.nz,
                         "n_bubbles": max(1, spec.n_bubbles * k // spec.nz)})


def oracle_time(case, reps=1):
    """Wall time of the CPU oracle's projection on case (rank 0 host cores)."""
    import oracle as O
    best = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.project_case(case)
        best.append(time.perf_counter() - t0)
    return min(best), O.num_threads()


def run_reference(args):
    """The oracle on the host cores: each step = one projection of a 256 x 256 x 32
    slab drawn with the same recipe (same x/y transform lengths and spacing)."""
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
                                             "precision": "fp64", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    case = I.make_case(spec)
    npts = case.npts
    prec = F.MIXED if args.precision == "mixed" else F.FP64

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    phi, pn, pnm1 = dev(case.phi), dev(case.pn), dev(case.pnm1)
    u, v, w = dev(case.u), dev(case.v), dev(case.w)
    p = torch.empty_like(phi)
    stream = torch.cuda.current_stream()

    def timed_run(precision, steps, warmup, per_kernel):
        """W warm-up solves; with per_kernel, a short breakdown run with every
        kernel bracketed by events picks the dominant kernel; then the timed
        region of `steps` solves, in which only the dominant kernel's launches
        carry events (its live average duration feeds the roofline)."""
        plan = F.Plan.for_case(case, precision=precision)
        for _ in range(warmup):
            plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
        torch.cuda.synchronize()
        breakdown, dom = {}, None
        if per_kernel:
            plan.set_timing(True)
            for _ in range(max(3, steps // 5)):
                plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
            breakdown = plan.timing()
            dom = max(breakdown, key=lambda k: breakdown[k][0])
            plan.set_timing(True, only=dom)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.solve(phi, pn, pnm1, u, v, w, p, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        live = plan.timing().get(dom) if dom else None
        st = plan.stats(stream)
        launches = plan.launches_per_solve() * steps
        plan.close()
        return ms, (breakdown, dom, live, plan.max_refine), st, launches

    clocks = ClockSampler()
    clocks.start()
    ms, (kern, dom, live, max_refine), st, launches = timed_run(prec, args.steps, args.warmup, True)
    clk = clocks.stop()
    ms = slowest_rank(ms, dist)
    value = job_throughput(npts, args.steps, world, ms / 1e3)

    # the other precision on the same inputs (context for "mixed vs FP64")
    other = F.FP64 if prec == F.MIXED else F.MIXED
    ms_o, _, st_o, _ = timed_run(other, max(3, args.steps // 4), args.warmup, False)
    value_o = npts * max(3, args.steps // 4) / (ms_o / 1e3)

    # roofline of the dominant kernel
    hbm_peak, hbm_src = measured_peaks()
    per_pt = algorithmic_per_point(spec.nx, spec.ny, prec == F.MIXED)
    roof = None
    if dom and live:
        tot_ms, cnt = live  # the dominant kernel inside the timed region
        # refinement kernels return at once after convergence: count only the
        # launches that did the pass (from the solve's sweep count)
        it, mr = st["iterations"], max_refine
        per_solve = {"fwd_x_refine": it, "fwd_y_refine": it, "thomas_refine": it,
                     "inv_y_refine": it, "inv_x_update": it, "resid_correct": it}.get(dom)
        if prec == F.MIXED and dom == "correct":  # runs only when no fused pass ran
            per_solve = 1 if it == 0 else 0
        del mr
        if per_solve is not None:
            cnt = max(1, per_solve * args.steps)
        avg_s = tot_ms / cnt / 1e3
        b_pt, fl_pt = per_pt.get(dom, (0, 0))
        gbs = b_pt * npts / avg_s / 1e9
        tfl = fl_pt * npts / avg_s / 1e12
        t_hbm = b_pt / (hbm_peak * 1e9)
        t_alu = fl_pt / (FP64_PEAK_NOMINAL * 1e12)
        traffic = (measured_traffic(dom, prec == F.MIXED)
                   if args.workload == "bubbles256" else None)
        if t_alu > t_hbm:
            roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_NOMINAL, "unit": "TFLOP/s",
                    "frac": tfl / FP64_PEAK_NOMINAL, "traffic": traffic, "kernel": dom,
                    "peak_source": "nominal FP64 (recipe table)",
                    "algorithmic_bytes": b_pt * npts, "hbm_gbs": gbs,
                    "hbm_frac": gbs / hbm_peak, "hbm_peak_source": hbm_src}
        else:
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "traffic": traffic, "kernel": dom,
                    "algorithmic_bytes": b_pt * npts, "peak_source": hbm_src}
    if roof:
        roof["launches_timed"] = cnt
        roof["duration_ms"] = tot_ms / cnt
        # the FP64 issue rate the ALU bound really is: FP64 instructions per
        # point against the nominal 0.625 T FP64 instructions/s (1.25 TFLOP/s
        # counts an FMA as two)
        ipt = fp64_instr_per_point(spec.nx, spec.ny, spec.bcx, spec.bcy, prec == F.MIXED,
                                   spec.bcz).get(dom)
        if ipt:
            ach = ipt * npts / avg_s / 1e12
            roof["fp64_issue"] = {"instr_per_pt": ipt, "achieved": ach, "peak": FP64_PEAK_NOMINAL / 2,
                                  "unit": "T instr/s", "frac": ach / (FP64_PEAK_NOMINAL / 2)}
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
        dev = [torch.empty(case.shape, dtype=torch.float64, device="cuda") for _ in range(10)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def copies():
            with torch.cuda.stream(s_in):
                for h, d in zip(hin, dev[:6]):
                    d.copy_(h, non_blocking=True)
            with torch.cuda.stream(s_out):
                for h, d in zip(hout, dev[6:]):
                    h.copy_(d, non_blocking=True)
        copies()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            copies()
        torch.cuda.synchronize()
        el_copy = slowest_rank(time.perf_counter() - t0, dist)
        del dev
        e2e = {"value": job_throughput(npts, args.e2e_steps, world, el), "unit": "pts/s",
               "h2d_bytes_per_step": 6 * 8 * npts, "d2h_bytes_per_step": 4 * 8 * npts,
               "ms_per_step": el / args.e2e_steps * 1e3,
               "copies_only_ms_per_step": el_copy / args.e2e_steps * 1e3,
               "link_frac": el_copy / el,
               "api": "fizzy_proj_solve_host_async (pipelined, pinned host arrays)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # periodic z: the oracle's dense cyclic z-line solves grow as nz^3, so
        # it is timed on a 32-plane slab of the same recipe
        ocase = case if spec.bcz == I.NEUMANN else I.make_case(slab_spec(spec))
        t_or, cores = oracle_time(ocase, reps=2)
        os_ = ocase.spec
        cpu = {"value": ocase.npts / t_or, "unit": "pts/s", "cores": cores, "kind": "oracle",
               "sample": "one full %dx%dx%d projection (best of 2)%s" % (
                   os_.nx, os_.ny, os_.nz, "" if ocase is case else ", a slab of the workload")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == F.FP64 else "f32+f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "grid": [spec.nx, spec.ny, spec.nz],
                           "precision": args.precision, "bc": "%s x, %s y, %s z" % tuple(
                               "periodic" if b == I.PERIODIC else "walls" for b in (spec.bcx, spec.bcy, spec.bcz)),
                           "l2": "inputs (6 x %d MiB) larger than L2" % (npts * 8 >> 20),
                           "parallelism": "replicas" if world > 1 else "single"},
                "gpu_launches": launches, "roofline": roof,
                "path_roofline": path_roofline(value, spec.nx, spec.ny, spec.bcx, spec.bcy,
                                               prec == F.MIXED, int(st["iterations"]), hbm_peak,
                                               spec.bcz),
                "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "kernels": kernels,
                "stats": {k: st[k] for k in ("iterations", "converged", "relres")},
                ("mixed" if other == F.MIXED else "fp64"): {
                    "value": value_o, "unit": "pts/s", "ms_per_step": ms_o / max(3, args.steps // 4),
                    "iterations": st_o["iterations"], "relres": st_o["relres"]}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Uneven batch: 64 projections (nx, ny in {32..192}, nz in [32, 192],
    periodic or wall x/y, 1-20 drops, density ratio 10-1000), mixed precision,
    one persistent launch replayed from a CUDA graph with autotuned tiles;
    compared with the plain FP64 form (one fizzy_proj_solve per instance)."""
    import torch
    import paper_2502_04189_b300 as F
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    specs = I.batch_specs(64)
    cases = [I.make_case(s) for s in specs]
    npts = sum(c.npts for c in cases)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    inputs = [(dev(c.phi), dev(c.pn), dev(c.pnm1), dev(c.u), dev(c.v), dev(c.w)) for c in cases]
    outs = [torch.empty(c.shape, dtype=torch.float64, device="cuda") for c in cases]
    stream = torch.cuda.current_stream()
    results = {}
    for prec, name in ((F.MIXED, "mixed_batched"), (F.FP64, "fp64_batched")):
        plans = [F.Plan.for_case(c, precision=prec) for c in cases]
        arrays = [inp + (o,) for inp, o in zip(inputs, outs)]
        batch = F.Batch(plans, arrays)
        tuning, tuned_ms = batch.autotune(reps=3)
        for _ in range(args.warmup):
            batch.solve()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            batch.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        status = batch.status()
        st = [p.stats() for p in plans]
        results[name] = {"value": npts / (ms / 1e3), "ms_per_batch": ms, "tuning": tuning,
                         "status": status, "items": batch.info()["items"],
                         "max_relres": max(x["relres"] for x in st),
                         "sweeps": [x["iterations"] for x in st] if prec == F.MIXED else None,
                         "all_converged": all(x["converged"] for x in st)}
        batch.close()
        for p in plans:
            p.close()
    # plain FP64 form: one stand-alone solve per instance
    plans = [F.Plan.for_case(c, precision=F.FP64) for c in cases]
    for _ in range(args.warmup):
        for pl, inp, o in zip(plans, inputs, outs):
            pl.solve(*inp, o)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for pl, inp, o in zip(plans, inputs, outs):
            pl.solve(*inp, o)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    results["fp64_plain_loop"] = {"value": npts / (ms / 1e3), "ms_per_batch": ms}
    for p in plans:
        p.close()
    if rank == 0:
        r = results["mixed_batched"]
        line = {"metric": METRIC, "value": r["value"], "unit": "pts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "batch64", "instances": len(cases), "points": npts,
                           "precision": "mixed", "tol": 1e-10},
                "forms": results}
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving: Poisson arrivals (seeded, mean 2000 req/s) of requests with
    nx, ny in {64,...,384}, nz in [64, 384], 30 % tanh-stretched z, periodic
    or wall x/y, density ratio 10-1000, mixed precision refined to 1e-10;
    admission by a 120 GB HBM budget with plans cached on the device, 100 ms
    admission deadline.  Inputs are periodic crops of a device-resident
    256^3 bubble template."""
    import torch
    import paper_2502_04189_b300 as F
    import paper_2502_04189_b300.serve as S
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    n = args.serve_requests
    arrivals, specs = I.serve_specs(n)
    tmpl = I.make_case(I.bubbles256_spec())
    fields = S.TemplateFields(tmpl)
    reqs = S.requests_from_specs(arrivals, specs, F.MIXED)
    server = F.Server(120 * (1 << 30), slots=args.serve_slots)

    def fill(r, views, stream):
        fields.fill(views, r.desc, r.offset, stream)

    # warm-up on a few requests (plan-building code paths, pool growth)
    S.run(server, [S.Request(i, 0.0, r.desc, r.offset) for i, r in enumerate(reqs[:4])], fill,
          deadline=60.0)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    out, summ = S.run(server, reqs, fill, deadline=0.1)
    clk = clocks.stop()
    info = server.info()
    server.close()
    if rank == 0:
        line = {"metric": METRIC, "value": summ["throughput_pts_s"], "unit": "pts/s",
                "n_gpus": world, "steps": n, "warmup": 4, "ms_per_step": summ["mean_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "serve", "arrival_rate_per_s": 2000, "requests": n,
                           "budget_gb": 120, "slots": args.serve_slots, "deadline_ms": 100,
                           "precision": "mixed", "tol": 1e-10},
                "serving": summ, "server": info, "clocks": clk}
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
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fizzy", choices=["fizzy", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="bubbles256", choices=list(WORKLOADS) + ["batch64", "serve"])
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
