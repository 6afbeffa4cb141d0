"""The allocation-free entry point (velo_reconstruct_static) against the
allocating one (velo_reconstruct_into).

velo_reconstruct_static is for callers that cannot allocate device memory
while they reconstruct (a fixed start-up memory budget, or code inside another
framework's callbacks); its scratch is a fixed array inside the library.  This
file is collected last, so a run that stops at its first failure has run every
other test before it; it passes alone in a fresh process and after the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2412_05041_b300 as velo
import velogen
from _compare import assert_same, to_numpy

pytestmark = pytest.mark.gpu


def _static_run(L, b, params):
    """Caller-owned device outputs; scratch from the library's static array."""
    dev = torch.device("cuda")
    E, P = b.n_events, len(b.pixels)
    s = velo.query_sizes(E, P)
    off = torch.from_numpy(b.offsets.view(np.int64)).to(dev)
    pix = torch.from_numpy(b.pixels.view(np.int32)).to(dev)
    bufs = dict(status=torch.empty(max(E, 1), dtype=torch.int32, device=dev),
                cluster_offsets=torch.empty(E + 1, dtype=torch.int64, device=dev),
                cluster_x=torch.empty(s.cap_clusters, dtype=torch.float32, device=dev),
                cluster_y=torch.empty(s.cap_clusters, dtype=torch.float32, device=dev),
                cluster_z=torch.empty(s.cap_clusters, dtype=torch.float32, device=dev),
                pixel_cluster=torch.empty(P, dtype=torch.int32, device=dev),
                track_offsets=torch.empty(E + 1, dtype=torch.int64, device=dev),
                track_hit_offsets=torch.empty(s.cap_tracks + 1, dtype=torch.int64, device=dev),
                track_hits=torch.empty(s.cap_track_hits, dtype=torch.int32, device=dev),
                track_states=torch.empty((s.cap_tracks, velo.STATE_STRIDE), dtype=torch.float32, device=dev),
                totals=torch.empty(4, dtype=torch.int64, device=dev))
    out = velo.Output(*[bufs[k].data_ptr() for k in ("status", "cluster_offsets", "cluster_x", "cluster_y",
                                                      "cluster_z", "pixel_cluster", "track_offsets",
                                                      "track_hit_offsets", "track_hits", "track_states",
                                                      "totals")])
    ev = velo.Events(E, P, off.data_ptr(), pix.data_ptr())
    geo = velo.geometry_struct(b.geometry)
    stream = torch.cuda.current_stream()
    velo.check(L.velo_reconstruct_static(ctypes.byref(ev), ctypes.byref(geo.s), ctypes.byref(params),
                                         ctypes.byref(out), stream.cuda_stream), "velo_reconstruct_static")
    stream.synchronize()
    nc, nt, nh, _ = (int(v) for v in bufs["totals"].cpu())
    return dict(status=bufs["status"][:E], cluster_offsets=bufs["cluster_offsets"], cluster_x=bufs["cluster_x"][:nc],
                cluster_y=bufs["cluster_y"][:nc], cluster_z=bufs["cluster_z"][:nc],
                track_offsets=bufs["track_offsets"], track_hit_offsets=bufs["track_hit_offsets"][:nt + 1],
                track_hits=bufs["track_hits"][:nh], track_states=bufs["track_states"][:nt],
                pixel_cluster=bufs["pixel_cluster"])


def test_static_scratch_matches_allocating_entry_point_twice():
    velo.build()
    L = velo.lib()
    params = velo.default_params()
    # two calls in a row: a larger batch, then a smaller one over what the first left behind
    batches = [velogen.generate(velogen.C2, n_events=40, first_event=3100),
               velogen.generate(velogen.C2, n_events=17, first_event=777)]
    for b in batches:
        assert velo.query_sizes(b.n_events, len(b.pixels)).workspace_bytes <= velo.STATIC_SCRATCH_BYTES
        got = _static_run(L, b, params)
        off = torch.from_numpy(b.offsets.view(np.int64)).cuda()
        pix = torch.from_numpy(b.pixels.view(np.int32)).cuda()
        ref = to_numpy(velo.reconstruct(off, pix, b.geometry, params, pixel_labels=True))
        assert_same(got, ref)  # the tolerance every parity test uses
        np.testing.assert_array_equal(got["pixel_cluster"].cpu().numpy(), ref["pixel_cluster"])
        assert int(ref["track_offsets"][-1]) > 0


def test_static_scratch_rejects_oversize_batch():
    velo.build()
    L = velo.lib()
    n_pix = 2_000_000  # needs more scratch than the static array holds
    assert velo.query_sizes(100, n_pix).workspace_bytes > velo.STATIC_SCRATCH_BYTES
    off = torch.zeros(101, dtype=torch.int64, device="cuda")
    pix = torch.zeros(16, dtype=torch.int32, device="cuda")
    ev = velo.Events(100, n_pix, off.data_ptr(), pix.data_ptr())
    geo = velo.geometry_struct(velogen.Geometry())
    out = velo.Output(*([pix.data_ptr()] * 11))
    rc = L.velo_reconstruct_static(ctypes.byref(ev), ctypes.byref(geo.s), ctypes.byref(velo.default_params()),
                                   ctypes.byref(out), torch.cuda.current_stream().cuda_stream)
    assert rc == velo.ECAPACITY
