"""GPU parity: the CUDA library against the CPU oracle, element by element.

Cluster ids and positions, per-word labels, track hit lists and event
offsets must be identical; track states within 1e-5 relative (they are
produced by the same binary32 operations in the same order, so in practice
they are identical too).  Inputs are seeded synthetic events; no expected
value comes from the CUDA path.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2412_05041_b300 as velo
import velogen
from _compare import assert_labels, assert_same, exact_state_fraction, to_numpy

pytestmark = pytest.mark.gpu

PARAM_VALUES = dict(win_seed=0.04, win_fwd=0.04, max_slope=0.3, max_scatter_seed=0.01, max_scatter_fwd=0.02,
                    max_skipped=1, sigma_meas=0.0159, ms_theta=5e-4, chi2ndf_max=10.0, chi2ndf_max_3hit=2.0)


def params(ms_theta):
    v = dict(PARAM_VALUES, ms_theta=ms_theta)
    return velo.default_params(**v), oracle.Params(**v)


@pytest.fixture(scope="module", autouse=True)
def built():
    velo.build()
    assert torch.cuda.is_available()


def gpu_run(offsets, pixels, geometry, p, labels=True):
    off = torch.from_numpy(np.ascontiguousarray(offsets, np.uint64).view(np.int64)).cuda()
    pix = torch.from_numpy(np.ascontiguousarray(pixels, np.uint32).view(np.int32)).cuda()
    return velo.reconstruct(off, pix, geometry, p, pixel_labels=labels)


def check_batch(b, ms_theta, labels=True):
    vp, op = params(ms_theta)
    g = gpu_run(b.offsets, b.pixels, b.geometry, vp, labels)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    assert_same(g, r)
    if labels:
        assert_labels(g["pixel_cluster"].cpu().numpy(), r["pixel_cluster"], b.offsets, b.offsets)
    return g, r


def test_config1_full():
    b = velogen.generate(velogen.C1)
    g, r = check_batch(b, 0.0)
    assert len(r["track_states"]) > 3900
    assert exact_state_fraction(g, r) == 1.0


def test_config2_subset():
    b = velogen.generate(velogen.C2, n_events=300)
    g, r = check_batch(b, 5e-4)
    assert exact_state_fraction(g, r) == 1.0


def test_config2_full_size_sampled():
    """The benchmark's configuration (10k pile-up-5.5 events, one launch sequence);
    sampled events are re-generated alone and checked against the oracle one by one."""
    cfg = velogen.C2
    b = velogen.generate(cfg)
    vp, op = params(cfg.ms_theta)
    g = to_numpy(gpu_run(b.offsets, b.pixels, b.geometry, vp, labels=True))
    rng = np.random.default_rng(123)
    sample = sorted(rng.choice(cfg.n_events, size=40, replace=False).tolist()) + [0, cfg.n_events - 1]
    for e in sample:
        one = velogen.generate(cfg, n_events=1, first_event=e)
        np.testing.assert_array_equal(one.pixels, b.event(e))
        r = oracle.reconstruct(one.offsets, one.pixels, one.geometry, op)
        assert_same(g, r, events=[e])
        assert_labels(g["pixel_cluster"], r["pixel_cluster"], b.offsets, one.offsets, events=[e])
    # properties at full size
    assert (g["status"] == 0).all()
    assert g["cluster_offsets"][-1] == len(g["cluster_x"]) and g["track_offsets"][-1] == len(g["track_states"])
    assert g["track_hit_offsets"][-1] == len(g["track_hits"])
    assert (np.diff(g["cluster_offsets"].astype(np.int64)) >= 0).all()
    assert (np.diff(g["track_hit_offsets"].astype(np.int64)) >= 3).all()


def _word(q, m, r, c):
    return (q << 27) | (m << 22) | (r << 11) | c


def edge_batch():
    """Ragged events: empty, one pixel, duplicates, a bad word, a module over the
    cluster capacity, an event larger than the shared-memory tier, normal events."""
    evs = []
    evs.append(np.zeros(0, np.uint32))
    evs.append(np.array([_word(7, 3, 100, 200)], np.uint32))
    evs.append(np.array([_word(3, 2, 10, 10), _word(4, 2, 10, 10), _word(5, 2, 11, 11)], np.uint32))
    c2 = velogen.generate(velogen.C2, n_events=3, first_event=77)
    evs.append(c2.event(0))
    bad = c2.event(1).copy()
    bad[len(bad) // 2] = _word(3, 30, 5, 5)  # module 30 does not exist
    evs.append(bad)
    idx = np.arange(65536)
    evs.append(((5 << 27) | (3 << 22) | ((2 * (idx // 764)) << 11) | (2 * (idx % 764))).astype(np.uint32))
    hi = velogen.Config(seed=9, n_events=1, hi_frac=1.0, hi_min_tracks=2500, hi_max_tracks=2500)
    big = velogen.generate(hi)
    assert len(big.pixels) > 23552  # exercises the global-memory tier
    evs.append(big.pixels)
    evs.append(c2.event(2))
    evs.append(np.zeros(0, np.uint32))
    offsets = np.zeros(len(evs) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(e) for e in evs])
    return offsets, np.concatenate(evs).astype(np.uint32)


def test_edge_cases():
    offsets, pixels = edge_batch()
    vp, op = params(5e-4)
    geo = velogen.Geometry()
    g = gpu_run(offsets, pixels, geo, vp)
    r = oracle.reconstruct(offsets, pixels, geo, op)
    assert list(r["status"]) == [0, 0, 0, 0, 1, 2, 0, 0, 0]
    assert_same(g, r)
    assert_labels(g["pixel_cluster"].cpu().numpy(), r["pixel_cluster"], offsets, offsets)
    assert g["n_failed"] == 2


def test_equal_keys_order_by_id():
    """Clusters on a diagonal of the sensor share one pseudo-angle exactly (0.5
    above the beam, 2.5 below): the hits must come out in (module, key, id)
    order, equal keys by cluster id, as in the oracle."""
    words = []
    for m in (4, 5, 9):
        for i in range(60):
            rc = 800 + 3 * i  # x = y > 0: key 0.5
            words.append(_word(1 + i % 15, m, rc, rc))
            rc = 100 + 3 * i  # x = y < 0: key 2.5
            words.append(_word(2, m, rc, rc))
    rng = np.random.default_rng(3)
    words = np.array(words, np.uint32)[rng.permutation(len(words))]
    offsets = np.array([0, len(words)], np.uint64)
    vp, op = params(5e-4)
    geo = velogen.Geometry()
    g = gpu_run(offsets, words, geo, vp)
    r = oracle.reconstruct(offsets, words, geo, op)
    assert_same(g, r)
    assert_labels(g["pixel_cluster"].cpu().numpy(), r["pixel_cluster"], offsets, offsets)


def test_uneven_module_spacing():
    """Generated events on modules with uneven z spacing (every seed and
    extension lever arm differs): identical to the oracle."""
    zs = (-300.0, -280.0, -250.0, -180.0, -90.0, -40.0, 0.0, 20.0, 60.0, 130.0, 200.0, 230.0, 300.0, 390.0, 450.0,
          520.0, 600.0, 700.0)
    geo = velogen.Geometry(n_modules=len(zs), module_z=zs)
    b = velogen.generate(velogen.C2, n_events=60, first_event=500, geometry=geo)
    check_batch(b, 5e-4)


def test_bad_offsets_fail_every_event():
    b = velogen.generate(velogen.C2, n_events=4)
    off = b.offsets.copy()
    off[2], off[3] = off[3], off[2]  # not monotone
    vp, _ = params(5e-4)
    g = to_numpy(gpu_run(off, b.pixels, b.geometry, vp))
    assert (g["status"] == velo.EVT_BADWORD).all()
    assert g["n_failed"] == 4 and len(g["cluster_x"]) == 0 and len(g["track_states"]) == 0
    assert (g["pixel_cluster"] == -1).all()


def test_empty_batch():
    vp, _ = params(5e-4)
    g = to_numpy(gpu_run(np.zeros(1, np.uint64), np.zeros(0, np.uint32), velogen.Geometry(), vp))
    assert len(g["status"]) == 0 and list(g["cluster_offsets"]) == [0] and list(g["track_offsets"]) == [0]


def test_deterministic_and_split_batches_agree():
    """Same input twice gives identical bytes; a batch split in two (as replicas
    on several devices would run it) gives the same per-event results."""
    b = velogen.generate(velogen.C2, n_events=200, first_event=5000)
    vp, op = params(5e-4)
    a1 = to_numpy(gpu_run(b.offsets, b.pixels, b.geometry, vp))
    a2 = to_numpy(gpu_run(b.offsets, b.pixels, b.geometry, vp))
    for k in a1:
        np.testing.assert_array_equal(a1[k], a2[k])
    half = 77
    o1 = b.offsets[: half + 1]
    o2 = b.offsets[half:] - b.offsets[half]
    p1 = b.pixels[: int(b.offsets[half])]
    p2 = b.pixels[int(b.offsets[half]):]
    r1 = oracle.reconstruct(o1, p1, b.geometry, op)
    r2 = oracle.reconstruct(o2, p2, b.geometry, op)
    assert_same(a1, r1, events=range(half))
    assert_same(a1, r2, events=range(half, b.n_events))


def test_host_buffer_entry_point():
    b = velogen.generate(velogen.C2, n_events=120, first_event=300)
    vp, op = params(5e-4)
    H = velo.HostReconstructor(b.geometry, vp, max_events=200, max_pixels=len(b.pixels) + 1000, pixel_labels=True)
    off = torch.from_numpy(b.offsets.view(np.int64)).pin_memory()
    pix = torch.from_numpy(b.pixels.view(np.int32)).pin_memory()
    g = H.run(off, pix)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    assert_same(g, r)
    assert_labels(g["pixel_cluster"].numpy(), r["pixel_cluster"], b.offsets, b.offsets)
    # reuse of the same context with a different batch
    b2 = velogen.generate(velogen.C1, n_events=30)
    vp0, op0 = params(0.0)
    H.params = vp0
    g2 = H.run(torch.from_numpy(b2.offsets.view(np.int64)), torch.from_numpy(b2.pixels.view(np.int32)))
    assert_same(g2, oracle.reconstruct(b2.offsets, b2.pixels, b2.geometry, op0))


def _host(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).pin_memory()


def test_host_form_tracks_only():
    """Without the cluster coordinates the host form returns the same tracks,
    hit ids and offsets, and copies 12 bytes per cluster less."""
    b = velogen.generate(velogen.C2, n_events=80, first_event=700)
    vp, op = params(5e-4)
    off, pix = _host(b.offsets, np.int64), _host(b.pixels, np.int32)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    H = velo.HostReconstructor(b.geometry, vp, max_events=80, max_pixels=len(b.pixels), chunks=3)
    T = velo.HostReconstructor(b.geometry, vp, max_events=80, max_pixels=len(b.pixels), chunks=3, clusters=False)
    g, t = H.run(off, pix), T.run(off, pix)
    assert_same(g, r)
    assert "cluster_x" not in t and T.cluster_x is None
    for k, v in t.items():
        if k == "n_failed":
            assert v == g[k]
        else:
            assert torch.equal(v, g[k]), k
    nc = int(g["cluster_offsets"][-1])
    assert H.bytes_out() - T.bytes_out() == 12 * nc


def test_host_form_chunks_agree_with_oracle():
    """The pipelined host form cuts a batch into chunks of whole events; the
    results (offsets moved to batch-wide values) must not depend on the cut."""
    b = velogen.generate(velogen.C2, n_events=150, first_event=4000)
    vp, op = params(5e-4)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    H = velo.HostReconstructor(b.geometry, vp, max_events=200, max_pixels=len(b.pixels), pixel_labels=True)
    off, pix = _host(b.offsets, np.int64), _host(b.pixels, np.int32)
    for chunks in (1, 2, 3, 7, 64, 0):
        H.set_chunks(chunks)
        g = H.run(off, pix)
        assert_same(g, r)
        assert_labels(g["pixel_cluster"].numpy(), r["pixel_cluster"], b.offsets, b.offsets)
    # empty events, bad words and an overflowing module among good events, cut into chunks
    offsets, pixels = edge_batch()
    geo = velogen.Geometry()
    re = oracle.reconstruct(offsets, pixels, geo, op)
    He = velo.HostReconstructor(geo, vp, max_events=len(offsets) - 1, max_pixels=len(pixels), pixel_labels=True,
                                chunks=4)
    ge = He.run(_host(offsets, np.int64), _host(pixels, np.int32))
    assert_same(ge, re)
    assert_labels(ge["pixel_cluster"].numpy(), re["pixel_cluster"], offsets, offsets)
    assert ge["n_failed"] == 2


def test_host_form_respects_capacities():
    """Capacities in the host output behave as in the device form: exact
    capacities give the full result; one entry short copies no cluster and no
    track (nothing written past a capacity), and the totals report the sizes
    needed, while status and per-event offsets are still written."""
    b = velogen.generate(velogen.C2, n_events=40, first_event=900)
    vp, op = params(5e-4)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    H = velo.HostReconstructor(b.geometry, vp, max_events=40, max_pixels=len(b.pixels), chunks=3)
    off, pix = _host(b.offsets, np.int64), _host(b.pixels, np.int32)
    assert_same(H.run(off, pix), r)
    need = [int(v) for v in H.totals[:3]]
    H._out.cap_clusters, H._out.cap_tracks, H._out.cap_track_hits = need
    assert_same(H.run(off, pix), r)  # capacities below the bounds, but enough
    sentinel = -7
    for which in range(3):
        caps = list(need)
        caps[which] -= 1
        H._out.cap_clusters, H._out.cap_tracks, H._out.cap_track_hits = caps
        for t in (H.cluster_x, H.cluster_y, H.cluster_z, H.track_hits, H.track_states, H.track_hit_offsets):
            t.fill_(sentinel)
        g = to_numpy(H.run(off, pix))
        assert [int(v) for v in H.totals[:3]] == need
        np.testing.assert_array_equal(g["status"], r["status"])
        np.testing.assert_array_equal(g["cluster_offsets"].astype(np.uint64), r["cluster_offsets"])
        np.testing.assert_array_equal(g["track_offsets"].astype(np.uint64), r["track_offsets"])
        for t in (H.cluster_x, H.cluster_y, H.cluster_z, H.track_hits, H.track_states):
            assert (t == sentinel).all()
        assert int(H.track_hit_offsets[0]) == 0 and (H.track_hit_offsets[1:] == sentinel).all()
    H._out.cap_clusters = H._out.cap_tracks = H._out.cap_track_hits = 0
    assert_same(H.run(off, pix), r)


def test_host_form_bad_offsets_and_empty_batch():
    b = velogen.generate(velogen.C2, n_events=6)
    off = b.offsets.copy()
    off[2], off[3] = off[3], off[2]  # not monotone: every event fails, as in the device form
    vp, _ = params(5e-4)
    H = velo.HostReconstructor(b.geometry, vp, max_events=6, max_pixels=len(b.pixels), pixel_labels=True, chunks=3)
    g = to_numpy(H.run(_host(off, np.int64), _host(b.pixels, np.int32)))
    assert (g["status"] == velo.EVT_BADWORD).all()
    assert g["n_failed"] == 6 and len(g["cluster_x"]) == 0 and len(g["track_states"]) == 0
    assert (g["pixel_cluster"] == -1).all()
    g0 = to_numpy(H.run(_host(np.zeros(1, np.uint64), np.int64), torch.zeros(0, dtype=torch.int32)))
    assert len(g0["status"]) == 0 and list(g0["cluster_offsets"]) == [0] and list(g0["track_offsets"]) == [0]
    assert g0["n_failed"] == 0 and len(g0["track_hit_offsets"]) == 1


class _DevArray:
    """Zero-copy torch view of a raw device pointer (CUDA array interface)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}


def _view(ptr, n, typestr):
    if n == 0:
        return torch.empty(0)
    return torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")


def test_library_owned_result():
    import ctypes
    b = velogen.generate(velogen.C2, n_events=50, first_event=900)
    vp, op = params(5e-4)
    off = torch.from_numpy(b.offsets.view(np.int64)).cuda()
    pix = torch.from_numpy(b.pixels.view(np.int32)).cuda()
    L = velo.lib()
    ev = velo.Events(b.n_events, len(b.pixels), off.data_ptr(), pix.data_ptr())
    geo = velo.geometry_struct(b.geometry)
    res = ctypes.c_void_p()
    stream = torch.cuda.current_stream()
    velo.check(L.velo_reconstruct(ctypes.byref(ev), ctypes.byref(geo.s), ctypes.byref(vp), ctypes.byref(res),
                                  stream.cuda_stream))
    view = velo.ResultView()
    velo.check(L.velo_result_view(res, ctypes.byref(view)))
    assert view.n_events == b.n_events and view.cap_clusters == len(b.pixels)
    stream.synchronize()
    o = view.out
    tot = _view(o.totals, 4, "<i8").cpu().numpy()
    E, nc, nt, nh = b.n_events, int(tot[0]), int(tot[1]), int(tot[2])
    g = dict(status=_view(o.status, E, "<i4").cpu(), cluster_offsets=_view(o.cluster_offsets, E + 1, "<i8").cpu(),
             cluster_x=_view(o.cluster_x, nc, "<f4").cpu(), cluster_y=_view(o.cluster_y, nc, "<f4").cpu(),
             cluster_z=_view(o.cluster_z, nc, "<f4").cpu(), track_offsets=_view(o.track_offsets, E + 1, "<i8").cpu(),
             track_hit_offsets=_view(o.track_hit_offsets, nt + 1, "<i8").cpu(),
             track_hits=_view(o.track_hits, nh, "<i4").cpu(),
             track_states=_view(o.track_states, nt * velo.STATE_STRIDE, "<f4").cpu().view(-1, velo.STATE_STRIDE))
    L.velo_result_free(res)
    torch.cuda.synchronize()
    assert_same(g, oracle.reconstruct(b.offsets, b.pixels, b.geometry, op))


def test_mc_quality_matches_oracle():
    b = velogen.generate(velogen.C2, n_events=200, first_event=2000, truth=True)
    vp, op = params(5e-4)
    from oracle import mc
    g = to_numpy(gpu_run(b.offsets, b.pixels, b.geometry, vp))
    m = mc.evaluate_batch(b, g)
    assert m["efficiency"] >= 0.99 and m["ghost_rate"] <= 0.05


def test_heavy_ion_events_repeatedly_match_oracle():
    """Two heavy-ion-like events (1 PV, 10000 tracks, ~350k words: the
    clustering's (module, row) table and the tracking's CTA clusters), three
    runs: every run identical to the oracle (catches races that show only
    now and then)."""
    from dataclasses import replace
    cfg = replace(velogen.C2, seed=9, n_events=2, fixed_pvs=1, fixed_tracks=10000)
    b = velogen.generate(cfg)
    vp, op = params(cfg.ms_theta)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, op)
    for _ in range(3):
        g = gpu_run(b.offsets, b.pixels, b.geometry, vp, labels=True)
        assert_same(g, r)
        assert_labels(g["pixel_cluster"].cpu().numpy(), r["pixel_cluster"], b.offsets, b.offsets)


@pytest.mark.slow
def test_heavy_events_off_the_grid():
    """Heavy-ion-like events where the grid search of their tracking does not
    apply, next to steps where it does: a module 2 mm in front of the next one
    (at that step the seeding's lever-arm ratio 1 - a' is below 0.05) and a
    17000-track event (twelve modules of more than 8192 hits; the oracle takes
    about 35 s on it).  The window search of those steps and modules, and the
    grid in between, give results identical to the oracle."""
    from dataclasses import replace
    zs = [-300.0 + 42.0 * k for k in range(velogen.N_MODULES)]
    zs[10] = zs[11] - 2.0
    geo = velogen.Geometry(module_z=tuple(zs))
    cfg = replace(velogen.C2, seed=11, n_events=2, fixed_pvs=1, fixed_tracks=10000)
    b = velogen.generate(cfg, geometry=geo)
    assert (np.diff(b.offsets.astype(np.int64)) > 300_000).all()
    check_batch(b, cfg.ms_theta)
    cfg = replace(velogen.C2, seed=12, n_events=1, fixed_pvs=1, fixed_tracks=17000)
    b = velogen.generate(cfg)
    g, r = check_batch(b, cfg.ms_theta, labels=False)
    mod = np.asarray(r["cluster_z"])
    assert max(np.unique(mod, return_counts=True)[1]) > 8192  # clusters of the fullest module
    assert len(r["track_states"]) > 15000


def test_events_either_side_of_the_fit_rank_cap():
    """The fit ranks the kept tracks of an event of up to 1024 tracks in shared
    memory and those of a larger one through the id -> track map: events of
    about 1220 tracks (one vertex of 1200 tracks, ~16.5k clusters: the
    per-event tracking kernel) among pile-up 5.5 events, in the separate and the
    fused form, equal the oracle."""
    from dataclasses import replace
    big = velogen.generate(replace(velogen.C2, seed=31, n_events=2, fixed_pvs=1, fixed_tracks=1200))
    c2 = velogen.generate(velogen.C2, n_events=6, first_event=900)
    pixels = np.concatenate([c2.pixels[: c2.offsets[3]], big.pixels, c2.pixels[c2.offsets[3]:]])
    sizes = np.concatenate([np.diff(c2.offsets[:4].astype(np.int64)), np.diff(big.offsets.astype(np.int64)),
                            np.diff(c2.offsets[3:].astype(np.int64))])
    offsets = np.zeros(len(sizes) + 1, np.uint64)
    offsets[1:] = np.cumsum(sizes)
    vp, op = params(5e-4)
    r = oracle.reconstruct(offsets, pixels, c2.geometry, op)
    kept = np.diff(r["track_offsets"].astype(np.int64))
    nclu = np.diff(r["cluster_offsets"].astype(np.int64))
    assert (kept[3:5] > 1024).all() and (nclu[3:5] < 20000).all() and (kept[:3] < 1024).all()
    o = torch.from_numpy(offsets.view(np.int64)).cuda()
    p = torch.from_numpy(pixels.view(np.int32)).cuda()
    for tuning in (None, velo.default_tuning(fused_output=1)):
        assert_same(to_numpy(velo.reconstruct(o, p, c2.geometry, vp, tuning=tuning)), r)


def test_fp32_peak_measurement():
    """The FP32 ceiling helper returns a rate in the range a B300-class GPU can
    reach (148 SMs x 128 FMA lanes x 2 flops at 1-2.1 GHz: 38-80 TFLOP/s)."""
    import ctypes
    v = ctypes.c_double(0.0)
    assert velo.lib().velo_measure_fp32_peak(ctypes.byref(v), None) == velo.OK
    assert 10e12 < v.value < 200e12
    assert velo.lib().velo_measure_fp32_peak(None, None) == velo.EINVAL


def _sub_batch(offsets, pixels, events):
    """The listed events of a CSR batch, as a batch of their own."""
    evs = [pixels[int(offsets[e]):int(offsets[e + 1])] for e in events]
    off = np.zeros(len(evs) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in evs])
    return off, (np.concatenate(evs) if evs else np.zeros(0)).astype(np.uint32)


def test_union_find_bound_fails_its_event_only():
    """The clustering's lock-free union-find retries a link only after losing a
    race, at most union_link_attempts times.  With no attempt allowed, exactly
    the events that need a linking union (a V-shaped neighbourhood: a word
    whose left and up-right neighbours are not otherwise connected) fail with
    VELO_EVT_TIMEOUT -- no cluster, no track, labels 0xFFFFFFFF -- while every
    other event stays identical to the oracle; at the default bound every
    event is identical to the oracle."""
    evs = []
    # isolated pixels, a horizontal pair and a 2x2 block: linked without the union pass
    evs.append(np.array([_word(9, 2, 300, 300), _word(4, 5, 700, 900), _word(6, 5, 700, 901),
                         _word(3, 9, 1000, 500), _word(5, 9, 1000, 501), _word(7, 9, 1001, 500),
                         _word(8, 9, 1001, 501)], np.uint32))
    # the V: (r, c-1), (r-1, c+1), (r, c)
    evs.append(np.array([_word(5, 3, 400, 599), _word(6, 3, 399, 601), _word(7, 3, 400, 600),
                         _word(9, 7, 200, 200)], np.uint32))
    c2 = velogen.generate(velogen.C2, n_events=6, first_event=1234)
    evs += [c2.event(i) for i in range(6)]
    offsets = np.zeros(len(evs) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(e) for e in evs])
    pixels = np.concatenate(evs).astype(np.uint32)
    vp, op = params(5e-4)
    geo = velogen.Geometry()
    r = oracle.reconstruct(offsets, pixels, geo, op)
    assert (r["status"] == 0).all()
    g = to_numpy(gpu_run(offsets, pixels, geo, vp))
    assert_same(g, r)
    t = to_numpy(velo.reconstruct(torch.from_numpy(offsets.view(np.int64)).cuda(),
                                  torch.from_numpy(pixels.view(np.int32)).cuda(), geo, vp, pixel_labels=True,
                                  tuning=velo.default_tuning(union_link_attempts=0)))
    st = t["status"]
    assert st[0] == velo.EVT_OK and st[1] == velo.EVT_TIMEOUT
    assert set(st.tolist()) <= {velo.EVT_OK, velo.EVT_TIMEOUT}
    assert t["n_failed"] == int((st == velo.EVT_TIMEOUT).sum())
    for e in np.flatnonzero(st == velo.EVT_TIMEOUT):
        assert t["cluster_offsets"][e + 1] == t["cluster_offsets"][e]
        assert t["track_offsets"][e + 1] == t["track_offsets"][e]
        assert (t["pixel_cluster"][int(offsets[e]):int(offsets[e + 1])].astype(np.uint32) == 0xFFFFFFFF).all()
    good = np.flatnonzero(st == velo.EVT_OK)
    so, sp = _sub_batch(offsets, pixels, good)
    rs = oracle.reconstruct(so, sp, geo, op)
    assert_same(t, rs, events=good)
    assert_labels(t["pixel_cluster"], rs["pixel_cluster"], offsets, so, events=good)


def test_fused_fit_and_output_equal_the_separate_kernels():
    """The fit that also writes the offsets (decoupled look-back over the
    events) and the compact output gives the bytes of the separate fit, scan
    and output kernels -- on ragged events with empty, failed and heavy ones,
    and on a batch of normal events -- and the oracle's results."""
    vp, op = params(5e-4)
    geo = velogen.Geometry()
    offsets, pixels = edge_batch()
    c2 = velogen.generate(velogen.C2, n_events=200, first_event=5000)
    for off, pix in ((offsets, pixels), (c2.offsets, c2.pixels)):
        o = torch.from_numpy(np.ascontiguousarray(off, np.uint64).view(np.int64)).cuda()
        p = torch.from_numpy(np.ascontiguousarray(pix, np.uint32).view(np.int32)).cuda()
        sep = to_numpy(velo.reconstruct(o, p, geo, vp, pixel_labels=True))
        fus = to_numpy(velo.reconstruct(o, p, geo, vp, pixel_labels=True,
                                        tuning=velo.default_tuning(fused_output=1)))
        for k in sep:
            np.testing.assert_array_equal(fus[k], sep[k], err_msg=k)
        assert_same(fus, oracle.reconstruct(off, pix, geo, op))
