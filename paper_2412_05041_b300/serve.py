"""Streaming reconstruction with continuous batching.

Requests (batches of events in host memory) arrive over time.  A request is
admitted as soon as a stream slot is free and its device memory (inputs,
outputs, workspace: ``footprint``) fits in what the budget has left; it then
runs on its own CUDA stream -- copy in, reconstruct, copy the result out --
overlapping with every other admitted request, and returns its memory when
its result is on the host.  Requests wait in arrival order; a request that
does not fit waits for earlier ones to finish (no request overtakes another
that fits the budget on its own).

The paper's first stage processes events as they stream out of the detector
(Sec. "Data flow overview"); this loop is that serving form on one GPU,
measured by events/s and by the latency from a request's arrival to its
result being on the host (p50 / p99).
"""
from __future__ import annotations

import gc
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import STATE_STRIDE, query_sizes
from .api import Reconstructor


@dataclass
class Request:
    rid: int
    offsets: np.ndarray          # uint64 [E + 1]
    pixels: np.ndarray           # uint32 [P]
    arrival: float = 0.0         # seconds after the start of the run
    admitted: float = -1.0
    done: float = -1.0
    result: dict = field(default_factory=dict)

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1


def footprint(n_events: int, n_pixels: int) -> int:
    """Device bytes one request holds while it runs (inputs, outputs, workspace)."""
    s = query_sizes(n_events, n_pixels)
    out = (4 * n_events + 16 * (n_events + 1) + 12 * s.cap_clusters + 8 * (s.cap_tracks + 1) + 4 * s.cap_track_hits
           + 4 * STATE_STRIDE * s.cap_tracks + 32)
    return int(s.workspace_bytes + out + 8 * (n_events + 1) + 4 * n_pixels + 4096)


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.req: Request | None = None
        self.done_evt = None
        self.keep = None
        self.bytes = 0
        self.phase = 0


class Server:
    """Continuous-batching server on one device."""

    def __init__(self, geometry, params=None, memory_budget: int = 40 << 30, n_slots: int = 8, device="cuda",
                 tuning=None):
        self.geometry, self.params, self.tuning = geometry, params, tuning
        self.budget = int(memory_budget)
        self.device = torch.device(device)
        self.slots = [_Slot(self.device) for _ in range(n_slots)]
        self.in_use = 0
        self.peak = 0
        self.max_in_flight = 0

    def _start(self, slot: _Slot, req: Request, now: float) -> None:
        E, P = req.n_events, len(req.pixels)
        with torch.cuda.stream(slot.stream):
            off_h = torch.from_numpy(req.offsets.view(np.int64)).pin_memory()
            pix_h = torch.from_numpy(req.pixels.view(np.int32)).pin_memory()
            off = off_h.to(self.device, non_blocking=True)
            pix = pix_h.to(self.device, non_blocking=True)
            R = Reconstructor(self.geometry, self.params, E, P, device=self.device, tuning=self.tuning)
            R.run(off, pix, slot.stream)
            # copy the whole result back (sizes are known only on the device: copy the capacities'
            # prefixes that the totals will select on the host)
            host = {k: torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for k, t in
                    (("status", R.status), ("cluster_offsets", R.cluster_offsets), ("track_offsets", R.track_offsets),
                     ("totals", R.totals))}
            for k in host:
                host[k].copy_(getattr(R, k), non_blocking=True)
            evt = torch.cuda.Event()
            evt.record(slot.stream)
        slot.req, slot.done_evt = req, evt
        slot.keep = (off_h, pix_h, off, pix, R, host)
        req.admitted = now
        slot.phase = 1

    def _finish_copy(self, slot: _Slot) -> None:
        """Second phase: the totals are on the host; copy the used parts of the outputs."""
        off_h, pix_h, off, pix, R, host = slot.keep
        nc, nt, nh, nf = (int(v) for v in host["totals"][:4])
        E = slot.req.n_events
        with torch.cuda.stream(slot.stream):
            parts = {"cluster_x": R.cluster_x[:nc], "cluster_y": R.cluster_y[:nc], "cluster_z": R.cluster_z[:nc],
                     "track_hit_offsets": R.track_hit_offsets[:nt + 1], "track_hits": R.track_hits[:nh],
                     "track_states": R.track_states[:nt]}
            out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in parts.items()}
            for k in out:
                out[k].copy_(parts[k], non_blocking=True)
            evt = torch.cuda.Event()
            evt.record(slot.stream)
        out.update({"status": host["status"][:E], "cluster_offsets": host["cluster_offsets"][:E + 1],
                    "track_offsets": host["track_offsets"][:E + 1], "n_failed": nf})
        slot.keep = (off_h, pix_h, off, pix, R, out)
        slot.done_evt = evt
        slot.phase = 2

    def run(self, requests: list, poll_sleep: float = 0.0, freeze_gc: bool = True) -> dict:
        """Serve `requests` (arrival times in seconds from now).  Returns statistics;
        every request's result dict (host tensors) is left in request.result.

        With `freeze_gc` the objects that exist when serving starts are moved out
        of the interpreter's cyclic collector (gc.freeze) until it ends: a full
        collection over a large heap stalls the loop for tens of milliseconds,
        which lands on the latency of every request in flight.  The freeze is
        process-wide, so it is taken only when nothing is frozen yet (not when
        an enclosing caller or another Server froze objects), and undone only
        by the call that took it.  Taking it runs one full collection first,
        before the serving clock starts."""
        own_freeze = freeze_gc and gc.get_freeze_count() == 0
        if own_freeze:
            gc.collect()
            gc.freeze()
        try:
            return self._serve(requests, poll_sleep)
        finally:
            if own_freeze:
                gc.unfreeze()

    def _serve(self, requests: list, poll_sleep: float) -> dict:
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        t0 = time.perf_counter()
        waiting = deque()
        finished = []
        while pending or waiting or any(s.req is not None for s in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # progress of running requests
            for s in self.slots:
                if s.req is None or not s.done_evt.query():
                    continue
                if s.phase == 1:
                    self._finish_copy(s)
                    continue
                req = s.req
                req.done = time.perf_counter() - t0
                req.result = {k: v for k, v in s.keep[5].items()}
                finished.append(req)
                self.in_use -= s.bytes
                s.req, s.keep, s.done_evt, s.bytes = None, None, None, 0
            # admission: oldest first, while a slot and the memory budget allow
            while waiting:
                free = [s for s in self.slots if s.req is None]
                if not free:
                    break
                req = waiting[0]
                need = footprint(req.n_events, len(req.pixels))
                if need > self.budget:
                    raise ValueError(f"request {req.rid} needs {need} bytes, more than the budget {self.budget}")
                if self.in_use + need > self.budget:
                    break
                waiting.popleft()
                free[0].bytes = need
                self.in_use += need
                self.peak = max(self.peak, self.in_use)
                self._start(free[0], req, time.perf_counter() - t0)
                self.max_in_flight = max(self.max_in_flight, sum(s.req is not None for s in self.slots))
            if poll_sleep:
                time.sleep(poll_sleep)
        wall = time.perf_counter() - t0
        lat = np.array([r.done - r.arrival for r in finished])
        n_ev = sum(r.n_events for r in finished)
        return dict(requests=len(finished), events=n_ev, wall_s=wall, events_per_s=n_ev / wall,
                    p50_latency_ms=float(np.percentile(lat, 50) * 1e3), p99_latency_ms=float(np.percentile(lat, 99) * 1e3),
                    max_in_flight=self.max_in_flight, peak_memory_bytes=self.peak, budget_bytes=self.budget)


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
