"""Continuous-batching driver over the serving runtime (fizzy_serve_*).

Replays a stream of projection requests with their arrival times in real
time: a request joins a FIFO queue on arrival, is admitted as soon as a slot
and HBM budget are free (the runtime's decision), has its inputs written on
its slot's stream, and runs concurrently with everything else in flight.  A
request that cannot be admitted within `deadline` seconds of its arrival is
rejected.  Latency = completion (seen by polling) minus arrival.

Request inputs come from device-resident template fields: each request takes
a seeded periodic crop of the templates at its own shape (wall faces zeroed),
so inputs of any size are produced on the GPU without host traffic.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Optional

import numpy as np

from . import Server, crop_fill, crop_fill_ptrs, device_view


@dataclasses.dataclass
class Request:
    index: int
    arrival: float           # seconds after the start
    desc: dict               # make_desc keyword arguments
    offset: tuple = (0, 0, 0)


@dataclasses.dataclass
class Outcome:
    index: int
    admitted: bool
    latency: Optional[float] = None
    stats: Optional[dict] = None


class TemplateFields:
    """Device copies of one input case used as periodic crop sources."""

    def __init__(self, case):
        import torch

        def dev(a):
            return torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.fields = [dev(a) for a in (case.phi, case.pn, case.pnm1, case.u, case.v, case.w)]
        self.shape = case.phi.shape

    def fill(self, views, desc, offset, stream):
        """Write crops of shape (nz, ny, nx) starting at offset into views[0..5]
        (one fizzy_crop_fill kernel: 96 bytes of device traffic per point);
        views may be tensors or RequestViews (raw pointers, no tensors made)."""
        if isinstance(views, RequestViews):
            if not hasattr(self, "_src_ptrs"):
                self._src_ptrs = [t.data_ptr() for t in self.fields]
            crop_fill_ptrs(self._src_ptrs, self.shape, views.ptrs, views.shape, offset,
                           desc.get("bcx", 0), desc.get("bcy", 0), stream)
        else:
            crop_fill(self.fields, views[:6], offset, desc.get("bcx", 0), desc.get("bcy", 0), stream)


class RequestViews:
    """A request's seven device arrays: raw pointers, with the tensor view of
    array k made by view_fn on first access (views[k])."""

    def __init__(self, ptrs, shape, view_fn):
        self.ptrs, self.shape, self._fn, self._t = ptrs, shape, view_fn, {}

    def __getitem__(self, k):
        if isinstance(k, slice):
            return [self[i] for i in range(*k.indices(len(self.ptrs)))]
        if k not in self._t:
            self._t[k] = self._fn(self.ptrs[k], self.shape)
        return self._t[k]

    def __len__(self):
        return len(self.ptrs)


def run(server: Server, requests, fill: Callable, deadline: float = 0.1,
        on_done: Optional[Callable] = None, spin_sleep: float = 0.0,
        view_fn: Callable = device_view, clock: Callable = time.perf_counter):
    """Serve `requests` (sorted by arrival).  fill(req, views, stream) writes a
    request's inputs; on_done(req, views) may read its outputs before release.
    Returns (outcomes, summary)."""
    pending = collections.deque()
    inflight = {}
    outcomes = {}
    nxt = 0
    max_inflight = 0
    t0 = clock()
    n = len(requests)
    blocked = None  # the head request that could not be admitted, until a slot frees
    while len(outcomes) < n:
        now = clock() - t0
        while nxt < n and requests[nxt].arrival <= now:
            pending.append(requests[nxt])
            nxt += 1
        # reject requests that waited too long for admission
        while pending and now - pending[0].arrival > deadline:
            r = pending.popleft()
            outcomes[r.index] = Outcome(r.index, False)
        # admit in arrival order while slots and budget allow (a refused head
        # is retried only once a slot has been released or the head changed)
        while pending and pending[0] is not blocked:
            r = pending[0]
            rc, slot, ptrs = server.admit(**r.desc)
            if rc != 0:
                blocked = r
                break
            pending.popleft()
            shape = (r.desc["nz"], r.desc["ny"], r.desc["nx"])
            views = RequestViews(ptrs, shape, view_fn)
            fill(r, views, server.stream(slot))
            server.launch(slot)
            inflight[slot] = (r, views)
            max_inflight = max(max_inflight, len(inflight))
        # completions
        for slot in server.poll():
            r, views = inflight.pop(slot)
            done = clock() - t0
            st = server.stats(slot)
            if on_done is not None:
                on_done(r, views)
            server.release(slot)
            blocked = None
            outcomes[r.index] = Outcome(r.index, True, done - r.arrival, st)
        if spin_sleep:
            time.sleep(spin_sleep)
    wall = clock() - t0
    done = [o for o in outcomes.values() if o.admitted]
    lat = np.array([o.latency for o in done]) if done else np.array([np.nan])
    pts = sum(requests[o.index].desc["nx"] * requests[o.index].desc["ny"] * requests[o.index].desc["nz"]
              for o in done)
    summary = {
        "requests": n, "admitted": len(done), "rejected": n - len(done),
        "rejected_fraction": (n - len(done)) / n,
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(np.mean(lat) * 1e3), "wall_s": wall, "points_done": pts,
        "throughput_pts_s": pts / wall, "requests_per_s": len(done) / wall,
        "max_inflight": max_inflight,
        "all_converged": all(o.stats["converged"] for o in done),
        "max_relres": max((o.stats["relres"] for o in done), default=0.0),
    }
    return [outcomes[i] for i in range(n)], summary


def requests_from_specs(arrivals, specs, precision, seed=0, template_shape=(256, 256, 256)):
    """Request list from inputs.serve_specs(): geometry, BCs, densities and a
    seeded crop offset per request."""
    rng = np.random.default_rng([4, 0, 99, seed])
    from .inputs import z_faces
    out = []
    for i, (t, s) in enumerate(zip(arrivals, specs)):
        desc = dict(nx=s.nx, ny=s.ny, nz=s.nz, dx=s.lx / s.nx, dy=s.ly / s.ny,
                    zf=z_faces(s.nz, s.lz, s.beta), bcx=s.bcx, bcy=s.bcy, rho_l=s.rho_l,
                    rho_g=s.rho_g, dt=s.dt, precision=precision)
        off = tuple(int(rng.integers(0, m)) for m in template_shape)
        out.append(Request(i, float(t), desc, off))
    return out
