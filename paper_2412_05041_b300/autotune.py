"""Autotuner of the persistent kernels' block shapes (velo_tuning_t).

Times every candidate shape on a sample of the target workload (CUDA events,
best of a few repetitions after warm-up), checks that each one reproduces the
default shape's output bit for bit, and returns the fastest.  Results are
cached per (device, workload signature) in a JSON file.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np
import torch

from . import default_tuning, Tuning
from .api import Reconstructor

CTAS_PER_EVENT = 0xFFFFFFFF  # one CTA per event (VELO_CTAS_PER_EVENT)
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "velo_b300", "tuning.json")


# shared-memory tiers of the clustering kernel: 0 = the most that fits (about
# 25k words at 1024 threads, one CTA per SM; about 12k at 512 threads, two),
# or a smaller one (valid for both) that sends larger events to the
# global-memory path and leaves more of the SM's memory to L1
TIERS = (0, 8192)


def candidates():
    """Block shapes searched: clustering threads (one 1024-thread or two
    512-thread CTAs per SM), its shared-memory tier, tracking threads per
    event, the persistent grid (every resident CTA, at most two per SM, or
    one CTA per event scheduled by the hardware), and the fit fused with the
    offsets and the output."""
    out = []
    for ct, tier, tt, cps in itertools.product((1024, 512), TIERS, (128, 256), (0, 2, CTAS_PER_EVENT)):
        out.append(default_tuning(cluster_threads=ct, cluster_smem_pixels=tier, track_threads=tt, ctas_per_sm=cps))
    # the fit with the offsets and the output in one kernel (fewer launches)
    out.append(default_tuning(fused_output=1))
    out.append(default_tuning(track_threads=128, fused_output=1))
    return out


def _signature(offsets: torch.Tensor, pixels: torch.Tensor) -> str:
    n = np.diff(offsets.cpu().numpy())
    return f"{torch.cuda.get_device_name()}|E{len(n)}|P{int(n.sum())}|p99={int(np.percentile(n, 99))}"


def _outputs(R: Reconstructor) -> dict:
    r = R.result()
    return {k: v.cpu().numpy() for k, v in r.items() if hasattr(v, "cpu")}


def tune(offsets: torch.Tensor, pixels: torch.Tensor, geometry, params=None, reps: int = 3, use_cache: bool = True,
         verbose: bool = False):
    """Returns (best Tuning, table of (tuning dict, ms)) for this batch."""
    sig = _signature(offsets, pixels)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
        if sig in cache:
            return default_tuning(**cache[sig]["best"]), cache[sig]["table"]
    E, P = offsets.numel() - 1, pixels.numel()
    ref = None
    table = []
    stream = torch.cuda.current_stream()
    for t in candidates():
        R = Reconstructor(geometry, params, E, P, device=pixels.device, tuning=t)
        R.run(offsets, pixels, stream)
        out = _outputs(R)
        if ref is None:
            ref = out
        else:
            for k in ref:
                if not np.array_equal(ref[k], out[k]):
                    raise RuntimeError(f"tuning {t.as_dict()} changed {k}")
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            R.run(offsets, pixels, stream)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        table.append((t.as_dict(), best))
        if verbose:
            print(t.as_dict(), f"{best:.3f} ms")
        del R
    best_t = min(table, key=lambda x: x[1])[0]
    if use_cache:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        cache[sig] = {"best": best_t, "table": table}
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return default_tuning(**best_t), table
