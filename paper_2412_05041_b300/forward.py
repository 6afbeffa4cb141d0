"""Forward tracking behind the C ABI (``velo_forward``): pixel-tracker tracks
traced through a single magnet kick to the downstream layers (Sec. "HLT1
details and results").  Device tensors in, device tensors out; the work is
done by ``libvelo.so``.
"""
from __future__ import annotations

import ctypes

import torch

from . import (FWD_LAYERS, FWD_STATE, DownstreamHits, ForwardOutput, VeloError, check, default_forward_params,
               downstream_struct, lib)
from .api import _ptr, _stream_handle


class ForwardTracker:
    """Output buffers and scratch for the forward tracking of up to
    ``max_events`` events, ``max_hits`` downstream hits and the tracks of a
    ``Reconstructor`` (its track capacity), reused across calls."""

    def __init__(self, downstream, params=None, max_events: int = 1, max_hits: int = 1, cap_tracks: int = 1,
                 device="cuda"):
        self.geo = downstream_struct(downstream)
        self.params = params if params is not None else default_forward_params()
        self.max_events, self.max_hits, self.cap_tracks = int(max_events), int(max_hits), max(int(cap_tracks), 1)
        dev = torch.device(device)
        ws = ctypes.c_uint64()
        check(lib().velo_forward_workspace_size(self.max_events, self.max_hits, ctypes.byref(ws)),
              "velo_forward_workspace_size")
        self.workspace = torch.empty(int(ws.value), dtype=torch.uint8, device=dev)
        self.n_found = torch.empty(self.cap_tracks, dtype=torch.int32, device=dev)
        self.hits = torch.empty((self.cap_tracks, FWD_LAYERS), dtype=torch.int32, device=dev)
        self.state = torch.empty((self.cap_tracks, FWD_STATE), dtype=torch.float32, device=dev)
        self._out = ForwardOutput(_ptr(self.n_found), _ptr(self.hits), _ptr(self.state), self.cap_tracks)
        self._rec = None

    def run(self, reconstructor, offsets: torch.Tensor, layer: torch.Tensor, x: torch.Tensor, y: torch.Tensor,
            stream=None) -> None:
        """Enqueue the forward tracking of the batch ``reconstructor`` last ran,
        with its downstream hits (offsets int64 [E+1]; layer int32, x, y
        float32 [H]), on ``stream`` (default: current stream)."""
        for name, t, dt in (("offsets", offsets, torch.int64), ("layer", layer, torch.int32),
                            ("x", x, torch.float32), ("y", y, torch.float32)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise VeloError(f"{name} must be a contiguous CUDA {dt} tensor")
        E, H = offsets.numel() - 1, x.numel()
        if layer.numel() != H or y.numel() != H:
            raise VeloError("layer, x and y must have the same length")
        if E != reconstructor.n_events:
            raise VeloError(f"{E} events of downstream hits for a reconstruction of {reconstructor.n_events}")
        if E > self.max_events or H > self.max_hits:
            raise VeloError(f"batch ({E} events, {H} hits) exceeds ({self.max_events}, {self.max_hits})")
        h = DownstreamHits(E, H, _ptr(offsets), _ptr(layer) if H else None, _ptr(x) if H else None,
                           _ptr(y) if H else None)
        rc = lib().velo_forward(ctypes.byref(h), ctypes.byref(reconstructor._out), ctypes.byref(self.geo),
                                ctypes.byref(self.params), ctypes.byref(self._out), _ptr(self.workspace),
                                self.workspace.numel(), _stream_handle(stream))
        check(rc, "velo_forward")
        self._rec = reconstructor

    def result(self, stream=None) -> dict:
        """n_found [T], hits [T, 12] (event-local ids, -1 = none), state [T, 6]
        for the T tracks of the last batch (waits for the stream)."""
        if self._rec is None:
            raise VeloError("no batch has run")
        s = stream if stream is not None else torch.cuda.current_stream()
        s.synchronize()
        T = min(int(self._rec.totals[1].item()), self.cap_tracks)
        return dict(n_found=self.n_found[:T], hits=self.hits[:T], state=self.state[:T])
