"""Benchmark: events/s of VELO-like pixel tracking on B300.

Workload: 10,000 synthetic pile-up-5.5 events (n_PV ~ Poisson(5.5), tracks
per PV ~ Poisson(40), 0.5 mrad scattering per module, 99 % hit efficiency,
1e-4 noise per cell per module) -- the stand-in for the paper's pp
collisions at mu ~ 5 (Sec. "Introduction").  One step reconstructs the whole
batch (clustering, seeding + extension, fit + cut, output compaction) with
the inputs resident in HBM; the 0.5 GB of pixel words per step exceed the
126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank with its own 10k
events (weak scaling, no collective on the data path: the events are
independent; the barrier and the max over ranks are timing only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s (1 B300) for VELO-like tracking at pileup 5.5; p99 batch latency"
UNIT = "events/s"
WORKLOAD = "C2: 10k events, pileup 5.5 (n_PV~Poisson(5.5), 40 tracks/PV), 26 modules, MS 0.5 mrad, eff 0.99, noise 1e-4"
# the intervals between the library's five stage marks: clustering, pattern
# recognition (k_track and k_track_wide), the fit (k_fit_out: in the fused
# form it also writes the offsets and the compact output), and the separate
# scan and output kernels (empty in the fused form)
STAGES = ("k_cluster", "k_track", "k_fit_out", "k_scan_output")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=10_000, help="events per GPU per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default block shapes instead of autotuned ones")
    ap.add_argument("--no-batched", action="store_true", help="skip the 100k-event uneven graph-launch measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the streaming (continuous batching) measurement")
    ap.add_argument("--no-forward", action="store_true", help="skip the forward-tracking measurement")
    ap.add_argument("--forward-only", action="store_true",
                    help="only the forward-tracking measurement (one JSON line of its own; for profiling)")
    ap.add_argument("--no-heavy", action="store_true", help="skip the heavy-ion-like event measurement")
    ap.add_argument("--heavy-only", action="store_true",
                    help="only the heavy-ion-like event measurement (one JSON line of its own; for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(rank: int, world: int, events_per_rank: int) -> tuple[int, int]:
    """Events of one rank: a contiguous, disjoint range of the generator's event
    stream (every event regenerates alone from its index), the same size on every
    rank (weak scaling).  No collective is needed: events are independent."""
    if not (0 <= rank < world):
        raise ValueError("rank outside the world")
    return rank * events_per_rank, events_per_rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (the step ends when every rank has finished)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def params_values(ms_theta):
    return dict(win_seed=0.04, win_fwd=0.04, max_slope=0.3, max_scatter_seed=0.01, max_scatter_fwd=0.02,
                max_skipped=1, sigma_meas=0.0159, ms_theta=ms_theta, chi2ndf_max=10.0, chi2ndf_max_3hit=2.0)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of the GPU this process runs on, while running."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str):
        self.bus = bus_id.lower()
        self.p = None
        self.lines = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        rows = []
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            bus = f[1].lower()
            if self.bus and not (bus.endswith(self.bus[-12:]) or self.bus.endswith(bus[-12:])):
                continue
            try:
                rows.append((float(f[2]), float(f[3]), float(f[4]) if f[4] not in ("[N/A]", "N/A") else 0.0, f[5:]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        maxsm = max(r[1] for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[3][1:]) if v.strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": maxsm, "samples": len(rows),
                "power_w_max": max(r[2] for r in rows), "reasons": reasons}


def bus_id_of(dev):
    import torch
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    except AttributeError:
        return ""


# ------------------------------------------------------------------ roofline inputs
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# host-only sources (the host-buffer pipeline, the static-scratch entry point)
# change no kernel and no launch, so they do not invalidate a profile
HOST_ONLY_SOURCES = ("velo_host.cu", "velo_static.cu", "velo_peak.cu")


# the forward-tracking kernel's own source and the device headers it includes;
# the pixel-tracker kernels' summaries cover every other kernel source
FORWARD_SOURCES = ("velo_forward.cu", "velo_device.cuh", "velo_fit.cuh", "velo_internal.cuh")


def kernel_source_hash(kernel: str = ""):
    """First 16 hex digits of the SHA-256 over the sources a kernel's ncu
    summary depends on (a summary of other sources is stale)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2412_05041_b300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in HOST_ONLY_SOURCES:
            continue
        if kernel == "k_forward":
            if name not in FORWARD_SOURCES:
                continue
        elif name == "velo_forward.cu":
            continue
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per event of `kernel` from the committed ncu summary, if it was
    taken from the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_c2.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_event:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_b or m_src.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_b.group(1))


def profiled_metric(kernel: str, name: str):
    """A metric of the committed ncu summary of `kernel` (current sources only)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_c2.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_src = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    m = re.search(r"\|\s*" + re.escape(name) + r"\s*\|\s*([0-9.eE+,-]+)\s*\|", txt)
    if not m_src or not m or m_src.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1).replace(",", ""))


def fp32_peak_tflops():
    """The FP32 FMA rate of this GPU, measured by the library's microbenchmark."""
    import ctypes

    import paper_2412_05041_b300 as velo
    v = ctypes.c_double(0.0)
    velo.check(velo.lib().velo_measure_fp32_peak(ctypes.byref(v), None), "velo_measure_fp32_peak")
    return v.value / 1e12


# ------------------------------------------------------------------ arms
def link_rates(dev, nbytes: int = 256 << 20, reps: int = 5) -> dict:
    """Pinned host <-> device copy rates (GB/s): each direction alone, and
    each direction while the other runs (both at once)."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_b = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def h2d():
        with torch.cuda.stream(s_in):
            d_a.copy_(h_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s_out):
            h_out.copy_(d_b, non_blocking=True)

    def both():
        h2d()
        d2h()

    def rate(fn):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        return nbytes * reps / (time.perf_counter() - t0) / 1e9

    return {"h2d_gbs": rate(h2d), "d2h_gbs": rate(d2h), "duplex_gbs_each": rate(both)}


def link_bound_ms(bytes_in: int, bytes_out: int, link: dict) -> float:
    """Shortest time the host link needs for a step's copies: both directions
    at once while both have bytes left (each at the duplex rate), then the
    rest alone -- or one direction after the other, if that is shorter."""
    dup, r_in, r_out = link["duplex_gbs_each"], link["h2d_gbs"], link["d2h_gbs"]
    both = min(bytes_in, bytes_out) / dup
    rest = (bytes_out - bytes_in) / r_out if bytes_out > bytes_in else (bytes_in - bytes_out) / r_in
    serial = bytes_in / r_in + bytes_out / r_out
    return min(both + rest, serial) / 1e6


def run_reference(args):
    """The CPU oracle as the reference arm: every step is a bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import velogen
    cfg = velogen.C2
    cores = os.cpu_count() or 1
    n = max(32, min(2000, 24 * cores))
    batches = [velogen.generate(cfg, n_events=n, first_event=(i * n) % cfg.n_events)
               for i in range(max(args.steps, 1) + args.warmup)]
    op = oracle.Params(**params_values(cfg.ms_theta))
    for i in range(args.warmup):
        b = batches[i]
        oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    t = []
    for i in range(args.steps):
        b = batches[args.warmup + i]
        t0 = time.perf_counter()
        oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
        t.append(time.perf_counter() - t0)
    sec = float(np.sum(t))
    value = args.steps * n / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_events_per_step": n, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                             "sample": f"{n} events of the C2 workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo), or 'unknown'."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(cfg):
    import oracle
    import velogen
    cores = os.cpu_count() or 1
    op = oracle.Params(**params_values(cfg.ms_theta))
    n_done, t_total, first = 0, 0.0, 0
    per = max(32, 8 * cores)
    while t_total < 4.0 and n_done < cfg.n_events:
        b = velogen.generate(cfg, n_events=per, first_event=first)
        t0 = time.perf_counter()
        oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
        t_total += time.perf_counter() - t0
        n_done += per
        first += per
    # the same on one host thread
    b1 = velogen.generate(cfg, n_events=48)
    t0 = time.perf_counter()
    oracle.reconstruct(b1.offsets, b1.pixels, b1.geometry, op, n_threads=1)
    t1 = time.perf_counter() - t0
    return {"value": n_done / t_total, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
            "sample": f"first {n_done} of the 10k C2 events, all {cores} host threads, {t_total:.1f} s wall",
            "one_thread": {"value": 48 / t1, "unit": UNIT, "sample": f"first 48 C2 events, 1 thread, {t1:.1f} s"}}


def run_batched(args, dev, vp):
    """100k events of uneven occupancy (10 % at pile-up 15, at random positions)
    in one CUDA-graph launch of the persistent kernels, block shapes autotuned
    on a 5k-event sample of the same batch."""
    import torch

    import paper_2412_05041_b300 as velo
    import velogen
    from paper_2412_05041_b300 import autotune
    cfg = velogen.C3
    t0 = time.time()
    b = velogen.generate(cfg)
    gen_s = time.time() - t0
    off = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    pix = torch.from_numpy(b.pixels.view(np.int32)).to(dev)
    E, P = b.n_events, pix.numel()
    sizes = np.diff(b.offsets.astype(np.int64))
    ns = 5000
    best, table = autotune.tune(off[: ns + 1], pix[: int(b.offsets[ns])], b.geometry, vp, reps=2, use_cache=False)
    G = velo.GraphReconstructor(off, pix, b.geometry, vp, tuning=best, cap_clusters=int(0.7 * P),
                                cap_tracks=int(0.03 * P))
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        G.replay()
    torch.cuda.synchronize(dev)
    K = max(3, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        G.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / K
    res = G.result()
    out = {"workload": "C3: 100k events, n_PV ~ Poisson(5.5) (90 %) / Poisson(15) (10 %), one CUDA-graph launch",
           "value": E / (ms / 1000.0), "unit": UNIT, "ms_per_launch": ms, "replays": K, "events": E, "pixels": P,
           "event_words_p50_p99_max": [int(np.percentile(sizes, 50)), int(np.percentile(sizes, 99)), int(sizes.max())],
           "tracks": int(res["track_offsets"][-1]), "failed_events": int(res["n_failed"]), "tuning": best.as_dict(),
           "tuning_table_ms": table, "generation_s": gen_s}
    del G
    torch.cuda.empty_cache()
    return out


def run_serving(args, dev, vp, tuning):
    """Streaming requests of 64 events (pile-up 5.5 with 5 % heavy-ion-like events
    of 2000-10000 tracks), 40 GB device-memory budget, 8 stream slots: after a
    warm-up pass, first all 96 requests at once (throughput), then Poisson
    arrivals at 70 % of that rate (latency from arrival to the result on the
    host)."""
    import velogen
    from paper_2412_05041_b300 import serve
    n_req, per = 96, 64
    b = velogen.generate(velogen.C5, n_events=n_req * per)
    reqs = []
    for i in range(n_req):
        e0, e1 = i * per, (i + 1) * per
        reqs.append(serve.Request(i, (b.offsets[e0:e1 + 1] - b.offsets[e0]).astype(np.uint64),
                                  b.pixels[int(b.offsets[e0]):int(b.offsets[e1])].copy()))
    # warm-up: the whole request set once (allocator pools, launch caches)
    serve.Server(b.geometry, vp, memory_budget=40 << 30, n_slots=8, device=dev, tuning=tuning).run(reqs)
    sat = serve.Server(b.geometry, vp, memory_budget=40 << 30, n_slots=8, device=dev, tuning=tuning).run(reqs)
    rate = 0.7 * sat["events_per_s"] / per
    for r, t in zip(reqs, serve.poisson_arrivals(n_req, rate, seed=6)):
        r.arrival, r.admitted, r.done = float(t), -1.0, -1.0
    poi = serve.Server(b.geometry, vp, memory_budget=40 << 30, n_slots=8, device=dev, tuning=tuning).run(reqs)
    heavy = int(sum(np.diff(b.offsets.astype(np.int64)) > 60000))
    return {"workload": f"C5: {n_req} requests x {per} events, 5 % heavy-ion-like (2000-10000 tracks), "
                        "40 GB budget, 8 streams", "heavy_events": heavy,
            "saturated": sat, "poisson_at_70pct": poi, "value": poi["events_per_s"], "unit": UNIT,
            "p50_latency_ms": poi["p50_latency_ms"], "p99_latency_ms": poi["p99_latency_ms"]}


def run_heavy(args, dev, vp):
    """Heavy-ion-like events (1 PV, 10000 tracks, ~350k pixel words each), four
    per batch: the stage times of one batch (the four events run side by side,
    so a stage's time is about one event's latency), K timed batches."""
    import torch

    import paper_2412_05041_b300 as velo
    import velogen
    from dataclasses import replace
    b = velogen.generate(replace(velogen.C2, seed=9, n_events=4, fixed_pvs=1, fixed_tracks=10000))
    off = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    pix = torch.from_numpy(b.pixels.view(np.int32)).to(dev)
    R = velo.Reconstructor(b.geometry, vp, max_events=b.n_events, max_pixels=pix.numel(), device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        R.run(off, pix, stream)
    K = max(3, args.steps)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    for k in range(K):
        R.run(off, pix, stream, marks=marks[k])
    torch.cuda.synchronize(dev)
    stage = {s_: float(np.median([marks[k][i].elapsed_time(marks[k][i + 1]) for k in range(K)]))
             for i, s_ in enumerate(STAGES)}
    total = float(np.median([marks[k][0].elapsed_time(marks[k][4]) for k in range(K)]))
    return {"workload": "4 heavy-ion-like events (1 PV, 10000 tracks each), one batch",
            "words_per_event": [int(x) for x in np.diff(b.offsets.astype(np.int64))],
            "clusters": int(R.totals[0]), "tracks": int(R.totals[1]), "batch_ms": total, "stage_ms": stage,
            "batches": K}


def run_forward(args, dev, vp, n_ev):
    """Forward tracking of the pixel-tracker tracks of n_ev pile-up-5.5 events
    to twelve downstream layers (invented geometry, 20 noise hits per layer):
    the pixel-tracker path runs once, then K timed launches of velo_forward
    alone and K of both stages back to back (inputs resident in HBM)."""
    import torch

    import paper_2412_05041_b300 as velo
    import velogen
    from velogen import scifi
    b = velogen.generate(velogen.C2, n_events=n_ev, truth=True)
    s = scifi.generate(b)
    stream = torch.cuda.current_stream(dev)
    off = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    pix = torch.from_numpy(b.pixels.view(np.int32)).to(dev)
    R = velo.Reconstructor(b.geometry, vp, max_events=n_ev, max_pixels=pix.numel(), device=dev)
    F = velo.ForwardTracker(s.geometry, max_events=n_ev, max_hits=len(s.x), cap_tracks=R.sizes.cap_tracks, device=dev)
    so = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    la = torch.from_numpy(s.layer.view(np.int32)).to(dev)
    x = torch.from_numpy(s.x).to(dev)
    y = torch.from_numpy(s.y).to(dev)
    R.run(off, pix, stream)
    for _ in range(max(args.warmup, 3)):
        F.run(R, so, la, x, y, stream)
    torch.cuda.synchronize(dev)
    K = max(3, args.steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    for _ in range(K):
        F.run(R, so, la, x, y, stream)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(K):
        R.run(off, pix, stream)
        F.run(R, so, la, x, y, stream)
    ev[3].record(stream)
    torch.cuda.synchronize(dev)
    ms_f = ev[0].elapsed_time(ev[1]) / K
    ms_both = ev[2].elapsed_time(ev[3]) / K
    r = F.result(stream)
    n = r["n_found"].cpu().numpy()
    T, H = len(n), len(s.x)
    # algorithmic bytes of one launch: the hits (layer, x, y) and offsets, per
    # track its last two clusters (x, y, z), two hit ids, its offsets, and
    # the outputs (count, 12 hit ids, 6-float state)
    alg = 12 * H + 8 * (n_ev + 1) + T * (24 + 8 + 16 + 4 + 48 + 24) + 8 * (n_ev + 1)
    peaks, peak_kind = measured_peaks()
    achieved = alg / (ms_f / 1000.0) / 1e9
    traffic = profiled_traffic("k_forward")
    return {"workload": f"C2 ({n_ev} events) pixel-tracker tracks + 12 downstream layers (20 noise hits/layer)",
            "value": n_ev / (ms_f / 1000.0), "unit": UNIT, "ms_per_launch": ms_f, "launches": K,
            "with_pixel_tracking": {"value": n_ev / (ms_both / 1000.0), "unit": UNIT, "ms_per_step": ms_both},
            "downstream_hits": H, "tracks_in": T, "found_fraction": float((n > 0).mean()) if T else 0.0,
            "roofline": {"kernel": "k_forward", "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "algorithmic_bytes": alg,
                         "traffic": None if traffic is None else traffic * n_ev,
                         "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "gpu_launches_per_call": 2 + (H > 4096) + (H > 16384)}  # validate, large events, huge events, the rest


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2412_05041_b300 as velo
    import velogen

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    velo.build()
    cfg = velogen.C2
    n_ev = args.events
    first, n_ev = shard(rank, world, n_ev)
    if args.forward_only or args.heavy_only:
        vp0 = velo.default_params(**params_values(cfg.ms_theta))
        out = run_forward(args, dev, vp0, n_ev) if args.forward_only else run_heavy(args, dev, vp0)
        if rank == 0:
            print(json.dumps({"forward" if args.forward_only else "heavy_events": out}))
        if world > 1:
            dist.destroy_process_group()
        return
    b = velogen.generate(cfg, n_events=n_ev, first_event=first)
    vp = velo.default_params(**params_values(cfg.ms_theta))
    off_h = torch.from_numpy(b.offsets.view(np.int64)).pin_memory()
    pix_h = torch.from_numpy(b.pixels.view(np.int32)).pin_memory()
    off = off_h.to(dev)
    pix = pix_h.to(dev)
    P = pix.numel()
    stream = torch.cuda.current_stream(dev)
    tuning, tuning_table = None, None
    if not args.no_autotune:
        from paper_2412_05041_b300 import autotune
        ns = min(3000, n_ev)
        tuning, tuning_table = autotune.tune(off[: ns + 1], pix[: int(b.offsets[ns])], b.geometry, vp, reps=2,
                                             use_cache=False)
    R = velo.Reconstructor(b.geometry, vp, max_events=n_ev, max_pixels=P, device=dev, tuning=tuning)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        R.run(off, pix, stream)
    torch.cuda.synchronize(dev)
    res = R.result()
    tot = [int(res["cluster_offsets"][-1]), int(res["track_offsets"][-1]), len(res["track_hits"]), int(res["n_failed"])]

    K = args.steps
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    for mk in marks:  # create the handles before the timed region
        for m in mk:
            m.record(stream)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with ClockSampler(bus_id_of(dev)) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        t0.record(stream)
        for k in range(K):
            R.run(off, pix, stream, marks=marks[k])
        t1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = t0.elapsed_time(t1) / K
    stage_ms = {s: float(np.mean([marks[k][i].elapsed_time(marks[k][i + 1]) for k in range(K)]))
                for i, s in enumerate(STAGES)}
    ms = max_over_ranks(ms, world, dev)
    value = world * n_ev / (ms / 1000.0)

    # learned form: the same batch with the ghost-rejection network on tensor cores
    learned, RL = None, None
    model = os.path.join(ROOT, "paper_2412_05041_b300", "models", "ghost_mlp.bin")
    if os.path.exists(model) and not args.no_learned:
        from paper_2412_05041_b300 import mlp as vmlp
        blob, thr = vmlp.load(model)
        blob_dev = torch.from_numpy(blob).to(dev)
        lp = velo.default_params(**params_values(cfg.ms_theta))
        lp.use_mlp, lp.mlp_logit_min, lp.mlp = 1, thr, blob_dev.data_ptr()
        RL = velo.Reconstructor(b.geometry, lp, max_events=n_ev, max_pixels=P, device=dev, tuning=tuning)
        for _ in range(max(args.warmup, 0)):
            RL.run(off, pix, stream)
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        l0.record(stream)
        for _ in range(K):
            RL.run(off, pix, stream)
        l1.record(stream)
        torch.cuda.synchronize(dev)
        lms = l0.elapsed_time(l1) / K
        learned = {"value": n_ev / (lms / 1000.0), "unit": UNIT, "ms_per_step": lms, "logit_min": thr,
                   "tracks": int(RL.result()["track_offsets"][-1])}
        if rank == 0:
            # quality of the tracks each form actually returns: the first 1000 events of
            # this workload (the same words, regenerated with their generator truth; the
            # network was trained on other seeds), reconstructed by the plain and the
            # learned in-kernel forms and matched by the library's truth code
            from paper_2412_05041_b300 import truth as vtruth
            nq = min(1000, n_ev)
            hold = velogen.generate(cfg, n_events=nq, first_event=first, truth=True)
            assert np.array_equal(hold.pixels, b.pixels[: len(hold.pixels)])
            qo = torch.from_numpy(hold.offsets.view(np.int64)).to(dev)
            qp = torch.from_numpy(hold.pixels.view(np.int32)).to(dev)
            qm = {}
            for form, prm in (("plain", vp), ("learned", lp)):
                res = velo.reconstruct(qo, qp, hold.geometry, prm, pixel_labels=True, tuning=tuning)
                qm[form] = vtruth.metrics(hold, {k: (v.cpu().numpy() if hasattr(v, "cpu") else v)
                                                 for k, v in res.items()})
            learned.update({"efficiency_plain": qm["plain"]["efficiency"],
                            "ghost_rate_plain": qm["plain"]["ghost_rate"],
                            "efficiency_learned": qm["learned"]["efficiency"],
                            "ghost_rate_learned": qm["learned"]["ghost_rate"],
                            "tracks_plain_sample": qm["plain"]["tracks"],
                            "tracks_learned_sample": qm["learned"]["tracks"],
                            "quality_sample": f"the first {nq} events of the timed workload, tracks returned by the "
                                              "plain and learned reconstructions, matched by generator truth"})

    # batch latency percentiles: 1k-event batches, one at a time
    lat = []
    nb = min(1000, n_ev)
    off_b = torch.from_numpy(b.offsets[: nb + 1].view(np.int64)).to(dev)
    Rb = velo.Reconstructor(b.geometry, vp, max_events=nb, max_pixels=int(b.offsets[nb]), device=dev, tuning=tuning)
    for _ in range(3):
        Rb.run(off_b, pix[: int(b.offsets[nb])], stream)
    for _ in range(30):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Rb.run(off_b, pix[: int(b.offsets[nb])], stream)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))

    # end to end through the host-buffer entry point (H2D + kernels + D2H inside the timed region)
    e2e = None
    if not args.no_e2e:
        H = velo.HostReconstructor(b.geometry, vp, max_events=n_ev, max_pixels=P)
        ke = max(3, min(K, 10))

        def host_time(chunks):
            H.set_chunks(chunks)
            for _ in range(2):
                H.run(off_h, pix_h, stream)
            barrier()
            tt = time.perf_counter()
            for _ in range(ke):
                H.run(off_h, pix_h, stream)
            return max_over_ranks((time.perf_counter() - tt) / ke, world, dev)

        el_serial = host_time(1)  # copy in, compute, copy out one after another
        el = host_time(0)         # chunked: copies overlap with the kernels
        b_in, b_out = int(8 * (n_ev + 1) + 4 * P), int(H.bytes_out())
        link = link_rates(dev)
        lb = link_bound_ms(b_in, b_out, link)
        e2e = {"value": world * n_ev / el, "unit": UNIT, "h2d_bytes_per_step": b_in,
               "d2h_bytes_per_step": b_out, "ms_per_step": 1000 * el, "pipeline": "auto chunks",
               "serial_value": world * n_ev / el_serial,
               "link": {k: round(v, 2) for k, v in link.items()}, "link_bound_ms": lb, "link_frac": lb / (1000 * el)}
        # the same with tracks-only results (no cluster coordinates copied back)
        del H
        H = velo.HostReconstructor(b.geometry, vp, max_events=n_ev, max_pixels=P, clusters=False)
        el_t = host_time(0)
        lb_t = link_bound_ms(b_in, int(H.bytes_out()), link)
        e2e["tracks_only"] = {"value": world * n_ev / el_t, "d2h_bytes_per_step": int(H.bytes_out()),
                              "ms_per_step": 1000 * el_t, "link_bound_ms": lb_t, "link_frac": lb_t / (1000 * el_t)}
        del H

    serving = None
    if world == 1 and not args.no_serving:
        try:
            serving = run_serving(args, dev, vp, tuning)
        except Exception as exc:
            serving = {"error": repr(exc)[:300]}

    heavy = None
    if world == 1 and not args.no_heavy:
        try:
            heavy = run_heavy(args, dev, vp)
        except Exception as exc:
            heavy = {"error": repr(exc)[:300]}

    forward = None
    if world == 1 and not args.no_forward:
        try:
            forward = run_forward(args, dev, vp, n_ev)
        except Exception as exc:
            forward = {"error": repr(exc)[:300]}
        torch.cuda.empty_cache()

    batched = None
    if world == 1 and not args.no_batched:
        R = RL = Rb = None
        torch.cuda.empty_cache()
        try:
            batched = run_batched(args, dev, vp)
        except Exception as exc:  # report, do not lose the main line
            batched = {"error": repr(exc)[:300]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_kind = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    n_cl, n_tr, n_hits = tot[0], tot[1], tot[2]
    # algorithmic bytes of the whole path per step: read the words, write clusters
    # (x, y, z) and tracks (hit ids, 20-float state, offsets), charged to the kernel
    # that moves them
    alg = {
        "k_cluster": 4 * P + 8 * (n_ev + 1) + 12 * n_cl + 4 * n_cl,
        "k_track": 16 * n_cl,
        "k_fit_out": 8 * n_hits + 8 * n_cl + 12 * n_cl + n_tr * (4 * 20 + 8) + 4 * n_hits + 24 * n_ev,
        "k_scan_output": 0,
    }
    achieved = alg[dom] / (stage_ms[dom] / 1000.0) / 1e9
    traffic = profiled_traffic(dom)
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None if traffic is None else traffic * n_ev,
            "peak_source": f"{peak_kind} hbm_gbs (copy)", "stage_ms": stage_ms}
    # DRAM bytes per second measured by ncu (bytes per event of the committed
    # summaries, current sources only) over the live times: of the dominant
    # stage and of the whole step
    # the kernels of each stage (the default, separate form)
    stage_of = {"k_cluster": ("k_cluster",), "k_track": ("k_track",), "k_fit_out": ("k_fit",),
                "k_scan_output": ("k_output",)}
    dram = {k: profiled_traffic(k) for k in ("k_cluster", "k_track", "k_fit", "k_output")}
    stage_kernels = stage_of.get(dom, (dom,))
    if all(dram.get(k) is not None for k in stage_kernels):
        roof["dram_gbs"] = sum(dram[k] for k in stage_kernels) * n_ev / (stage_ms[dom] / 1000.0) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / peaks["hbm_gbs"]
    if all(v is not None for v in dram.values()):
        roof["step_dram_gbs"] = sum(dram.values()) * n_ev / (ms / 1000.0) / 1e9
    # second ceiling: the plain FP32 pipe (measured on this GPU), with the busy
    # fractions of the dominant kernel's FMA and ALU pipes from its ncu summary
    fma = profiled_metric(dom, "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active")
    alu = profiled_metric(dom, "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active")
    issue = profiled_metric(dom, "smsp__issue_active.avg.pct_of_peak_sustained_active")
    roof["alu_ceiling"] = {"fp32_peak_tflops": fp32_peak_tflops(), "peak_source": "measured (velo_measure_fp32_peak)",
                           "fma_pipe_frac": None if fma is None else fma / 100.0,
                           "alu_pipe_frac": None if alu is None else alu / 100.0,
                           "issue_active_frac": None if issue is None else issue / 100.0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_gpu": n_ev, "pixels_per_gpu": P, "clusters": n_cl,
                   "tracks": n_tr, "failed_events": tot[3], "l2": "inputs larger than L2 (0.5 GB words)",
                   "parallelism": f"replicas x{world} (event sharding)"},
        "p50_batch_latency_ms": float(np.percentile(lat, 50)), "p99_batch_latency_ms": float(np.percentile(lat, 99)),
        "latency_batch_events": nb,
        "gpu_launches": 5 * K,  # validate, cluster, track, track (heavy events), fit + offsets + output per step
        "roofline": roof,
        "clocks": clk.summary(),
        "e2e": e2e,
        "learned": learned,
        "tuning": None if tuning is None else tuning.as_dict(),
        "tuning_table_ms": tuning_table,
        "batched": batched,
        "serving": serving,
        "forward": forward,
        "heavy_events": heavy,
    }
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.warmup < 3 and args.impl == "ours":
        print("note: --warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
