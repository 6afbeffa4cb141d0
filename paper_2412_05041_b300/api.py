"""Torch-facing wrappers of the C ABI: device tensors in, device tensors out.

PyTorch only provides memory and streams here; all reconstruction work is
done by ``libvelo.so``.
"""
from __future__ import annotations

import ctypes

import torch

from . import (N_FEATURES, Events, Output, STATE_STRIDE, VeloError, check, default_params, geometry_struct, lib,
               query_sizes)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


class Reconstructor:
    """Device buffers (outputs + workspace) for batches of up to ``max_events``
    events and ``max_pixels`` pixel words, reused across calls."""

    def __init__(self, geometry, params=None, max_events: int = 1, max_pixels: int = 1, device="cuda",
                 pixel_labels: bool = False, features: bool = False, tuning=None, cap_tracks: int | None = None,
                 cap_clusters: int | None = None):
        """cap_tracks / cap_clusters: output capacities below the always-sufficient
        bounds (a batch that does not fit writes no output; see ``fits()``)."""
        self.geo = geometry_struct(geometry)
        self.params = params if params is not None else default_params()
        self.tuning = tuning
        self.max_events, self.max_pixels = int(max_events), int(max_pixels)
        s = query_sizes(self.max_events, self.max_pixels)
        if cap_clusters is not None:
            s.cap_clusters = min(s.cap_clusters, int(cap_clusters))
            s.cap_track_hits = min(s.cap_track_hits, int(cap_clusters))
        if cap_tracks is not None:
            s.cap_tracks = min(s.cap_tracks, int(cap_tracks))
        dev = torch.device(device)
        E = self.max_events
        self.sizes = s
        # every buffer gets >= 1 element: a zero-size tensor has a NULL data pointer
        self.status = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
        self.cluster_offsets = torch.empty(E + 1, dtype=torch.int64, device=dev)
        self.cluster_x = torch.empty(max(s.cap_clusters, 1), dtype=torch.float32, device=dev)
        self.cluster_y = torch.empty_like(self.cluster_x)
        self.cluster_z = torch.empty_like(self.cluster_x)
        self.pixel_cluster = torch.empty(max(self.max_pixels, 1), dtype=torch.int32, device=dev) if pixel_labels else None
        self.track_offsets = torch.empty(E + 1, dtype=torch.int64, device=dev)
        self.track_hit_offsets = torch.empty(s.cap_tracks + 1, dtype=torch.int64, device=dev)
        self.track_hits = torch.empty(max(s.cap_track_hits, 1), dtype=torch.int32, device=dev)
        self.track_states = torch.empty((max(s.cap_tracks, 1), STATE_STRIDE), dtype=torch.float32, device=dev)
        self.totals = torch.empty(4, dtype=torch.int64, device=dev)
        self.track_features = (torch.empty((max(s.cap_tracks, 1), N_FEATURES), dtype=torch.float32, device=dev)
                               if features else None)
        self.workspace = torch.empty(s.workspace_bytes, dtype=torch.uint8, device=dev)
        self._out = Output(_ptr(self.status), _ptr(self.cluster_offsets), _ptr(self.cluster_x), _ptr(self.cluster_y),
                           _ptr(self.cluster_z), _ptr(self.pixel_cluster), _ptr(self.track_offsets),
                           _ptr(self.track_hit_offsets), _ptr(self.track_hits), _ptr(self.track_states),
                           _ptr(self.totals), _ptr(self.track_features), max(s.cap_clusters, 1),
                           max(s.cap_tracks, 1), max(s.cap_track_hits, 1))
        self.n_events = 0

    def run(self, offsets: torch.Tensor, pixels: torch.Tensor, stream=None, marks=None) -> None:
        """Enqueue the reconstruction of one batch on ``stream`` (default: current stream).

        marks: optional 5 torch.cuda.Event(enable_timing=True) recorded between the kernel stages."""
        if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
            raise VeloError("offsets must be a contiguous CUDA int64 tensor")
        if pixels.dtype != torch.int32 or not pixels.is_cuda or not pixels.is_contiguous():
            raise VeloError("pixels must be a contiguous CUDA int32 tensor (uint32 words)")
        E, P = offsets.numel() - 1, pixels.numel()
        if E < 0 or E > self.max_events or P > self.max_pixels:
            raise VeloError(f"batch ({E} events, {P} pixels) exceeds ({self.max_events}, {self.max_pixels})")
        ev = Events(E, P, _ptr(offsets), _ptr(pixels) if P else None)
        mk = None
        if marks is not None:
            if len(marks) != 5:
                raise VeloError("marks: 5 events")
            for m in marks:
                if not m.cuda_event:  # torch creates the handle lazily at the first record
                    m.record(stream if stream is not None else torch.cuda.current_stream())
            mk = (ctypes.c_void_p * 5)(*[m.cuda_event for m in marks])
        rc = lib().velo_reconstruct_into_tuned(ctypes.byref(ev), ctypes.byref(self.geo.s), ctypes.byref(self.params),
                                               ctypes.byref(self._out), _ptr(self.workspace), self.workspace.numel(),
                                               _stream_handle(stream), mk,
                                               None if self.tuning is None else ctypes.byref(self.tuning))
        check(rc, "velo_reconstruct_into_tuned")
        self.n_events = E
        self.n_pixels = P

    def fits(self, totals) -> bool:
        nc, nt, nh = (int(v) for v in totals[:3])
        return nc <= self.sizes.cap_clusters and nt <= self.sizes.cap_tracks and nh <= self.sizes.cap_track_hits

    def result(self, stream=None) -> dict:
        """Views of the last batch's outputs, trimmed to their sizes (waits for the stream)."""
        s = stream if stream is not None else torch.cuda.current_stream()
        s.synchronize()
        tot = self.totals.cpu()
        if not self.fits(tot):
            raise VeloError(f"batch output {tot[:3].tolist()} exceeds the capacities "
                            f"({self.sizes.cap_clusters}, {self.sizes.cap_tracks}, {self.sizes.cap_track_hits})")
        nc, nt, nh, nf = (int(v) for v in tot)
        E = self.n_events
        r = dict(status=self.status[:E], cluster_offsets=self.cluster_offsets[:E + 1], cluster_x=self.cluster_x[:nc],
                 cluster_y=self.cluster_y[:nc], cluster_z=self.cluster_z[:nc], track_offsets=self.track_offsets[:E + 1],
                 track_hit_offsets=self.track_hit_offsets[:nt + 1], track_hits=self.track_hits[:nh],
                 track_states=self.track_states[:nt], n_failed=nf)
        if self.pixel_cluster is not None:
            r["pixel_cluster"] = self.pixel_cluster[:self.n_pixels]
        if self.track_features is not None:
            r["track_features"] = self.track_features[:nt]
        return r


def reconstruct(offsets: torch.Tensor, pixels: torch.Tensor, geometry, params=None, pixel_labels: bool = False,
                stream=None, features: bool = False, tuning=None) -> dict:
    """One-shot: allocate, run, wait, return trimmed device tensors."""
    R = Reconstructor(geometry, params, max(offsets.numel() - 1, 0), pixels.numel(), device=pixels.device,
                      pixel_labels=pixel_labels, features=features, tuning=tuning)
    R.run(offsets, pixels, stream)
    return R.result(stream)


class GraphReconstructor(Reconstructor):
    """A Reconstructor whose launch sequence (validation, persistent clustering,
    persistent tracking, offsets scan, persistent output) is captured once into
    a CUDA graph for a fixed batch shape and replayed as one graph launch.
    ``load`` copies a new batch of the same shape into the captured inputs."""

    def __init__(self, offsets: torch.Tensor, pixels: torch.Tensor, geometry, params=None, **kw):
        super().__init__(geometry, params, offsets.numel() - 1, pixels.numel(), device=pixels.device, **kw)
        self.off_in = offsets.clone()
        self.pix_in = pixels.clone()
        s = torch.cuda.Stream(device=pixels.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(self.off_in, self.pix_in, s)  # first call outside capture: one-time set-up
        s.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s):
            self.run(self.off_in, self.pix_in, s)
        torch.cuda.current_stream().wait_stream(s)

    def load(self, offsets: torch.Tensor, pixels: torch.Tensor) -> None:
        if offsets.shape != self.off_in.shape or pixels.shape != self.pix_in.shape:
            raise VeloError("a graph replays one batch shape")
        self.off_in.copy_(offsets)
        self.pix_in.copy_(pixels)

    def replay(self) -> None:
        self.graph.replay()


class HostReconstructor:
    """Host-memory form (``velo_reconstruct_host``): a library context owns the
    device buffers; inputs and outputs are pinned host tensors.  A batch is cut
    into up to `chunks` chunks of whole events (0 = the library's choice, 1 =
    no overlap) whose copies overlap with the kernels of the others.  With
    ``clusters=False`` the cluster coordinates are not copied back (tracks,
    their hit ids and the cluster offsets still are)."""

    def __init__(self, geometry, params=None, max_events: int = 1, max_pixels: int = 1, pixel_labels: bool = False,
                 chunks: int = 0, clusters: bool = True):
        self.geo = geometry_struct(geometry)
        self.params = params if params is not None else default_params()
        self.ctx = ctypes.c_void_p()
        check(lib().velo_context_create(max_events, max_pixels, ctypes.byref(self.ctx)), "velo_context_create")
        self.set_chunks(chunks)
        s = query_sizes(max_events, max_pixels)
        E = max_events

        def pin(n, dt):
            return torch.empty(max(n, 1), dtype=dt, pin_memory=True)

        self.status = pin(E, torch.int32)
        self.cluster_offsets = pin(E + 1, torch.int64)
        self.clusters = bool(clusters)
        self.cluster_x, self.cluster_y, self.cluster_z = (
            (pin(s.cap_clusters, torch.float32) if self.clusters else None) for _ in range(3))
        self.pixel_cluster = pin(max_pixels, torch.int32) if pixel_labels else None
        self.track_offsets = pin(E + 1, torch.int64)
        self.track_hit_offsets = pin(s.cap_tracks + 1, torch.int64)
        self.track_hits = pin(s.cap_track_hits, torch.int32)
        self.track_states = pin(max(s.cap_tracks, 1) * STATE_STRIDE, torch.float32).view(-1, STATE_STRIDE)
        self.totals = pin(4, torch.int64)
        self._out = Output(_ptr(self.status), _ptr(self.cluster_offsets), _ptr(self.cluster_x), _ptr(self.cluster_y),
                           _ptr(self.cluster_z), _ptr(self.pixel_cluster), _ptr(self.track_offsets),
                           _ptr(self.track_hit_offsets), _ptr(self.track_hits), _ptr(self.track_states),
                           _ptr(self.totals), None, 0, 0, 0)

    def set_chunks(self, chunks: int) -> None:
        check(lib().velo_context_set_pipeline(self.ctx, int(chunks)), "velo_context_set_pipeline")

    def __del__(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            lib().velo_context_destroy(self.ctx)
            self.ctx = None

    def bytes_out(self) -> int:
        """Host bytes the last call copied back (status, offsets, clusters, tracks)."""
        nc, nt, nh, _ = (int(v) for v in self.totals[:4])
        E = self.n_events
        return (32 + 4 * E + 16 * (E + 1) + (12 * nc if self.clusters else 0) + 8 * (nt + 1) + 4 * nh +
                4 * STATE_STRIDE * nt + (4 * self.n_pixels if self.pixel_cluster is not None else 0))

    def run(self, offsets: torch.Tensor, pixels: torch.Tensor, stream=None) -> dict:
        """offsets (int64) and pixels (int32) in host memory, pinned for full copy speed."""
        E, P = offsets.numel() - 1, pixels.numel()
        ev = Events(E, P, _ptr(offsets), _ptr(pixels) if P else None)
        check(lib().velo_reconstruct_host(self.ctx, ctypes.byref(ev), ctypes.byref(self.geo.s),
                                          ctypes.byref(self.params), ctypes.byref(self._out), _stream_handle(stream)),
              "velo_reconstruct_host")
        self.n_events, self.n_pixels = E, P
        nc, nt, nh, nf = (int(v) for v in self.totals[:4])
        r = dict(status=self.status[:E], cluster_offsets=self.cluster_offsets[:E + 1],
                 track_offsets=self.track_offsets[:E + 1], track_hit_offsets=self.track_hit_offsets[:nt + 1],
                 track_hits=self.track_hits[:nh], track_states=self.track_states[:nt], n_failed=nf)
        if self.clusters:
            r.update(cluster_x=self.cluster_x[:nc], cluster_y=self.cluster_y[:nc], cluster_z=self.cluster_z[:nc])
        if self.pixel_cluster is not None:
            r["pixel_cluster"] = self.pixel_cluster[:P]
        return r
