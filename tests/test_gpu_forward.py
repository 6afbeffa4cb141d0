"""GPU parity of forward tracking (velo_forward) with the oracle.

Downstream hit ids per layer and hit counts must be identical; the state
(q/p, chi2/ndf, slope, intercept, match distances) within 1e-5 relative
(both sides run the same binary32 operations in the same order, so in
practice it is identical).  The pixel-tracker tracks fed to the oracle come
from the oracle's own reconstruction; the library's come from the library
(the two agree exactly, which the reconstruction parity tests check).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2412_05041_b300 as velo
import velogen
from _compare import STATE_ATOL, STATE_RTOL, to_numpy
from velogen import scifi

pytestmark = pytest.mark.gpu

DOWN = scifi.Downstream()
NONE = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def built():
    velo.build()
    assert torch.cuda.is_available()


def dev(a, dt, view=None):
    a = np.ascontiguousarray(a, dt)
    if view is not None:
        a = a.view(view)
    return torch.from_numpy(a.copy() if a.size else np.zeros(1, a.dtype)[:0]).cuda()


def reco(b):
    """Library reconstruction of a generator batch (device buffers kept)."""
    R = velo.Reconstructor(b.geometry, max_events=max(b.n_events, 1), max_pixels=max(len(b.pixels), 1))
    R.run(dev(b.offsets, np.uint64, np.int64), dev(b.pixels, np.uint32, np.int32))
    R.result()
    return R


def gpu_forward(R, s, params=None, cap_tracks=None):
    F = velo.ForwardTracker(s.geometry, params, max_events=max(s.n_events, 1), max_hits=max(len(s.x), 1),
                            cap_tracks=R.sizes.cap_tracks if cap_tracks is None else cap_tracks)
    F.run(R, dev(s.offsets, np.uint64, np.int64), dev(s.layer, np.uint32, np.int32), dev(s.x, np.float32),
          dev(s.y, np.float32))
    r = to_numpy(F.result())
    return r["n_found"].astype(np.uint32), r["hits"].astype(np.uint32), r["state"]


def assert_forward_same(g, r, tracks=None):
    gn, gh, gs = g
    rn, rh, rs = r
    idx = np.arange(len(rn)) if tracks is None else np.asarray(tracks)
    np.testing.assert_array_equal(gn[idx], rn, err_msg="n_found")
    np.testing.assert_array_equal(gh[idx], rh, err_msg="downstream hits")
    np.testing.assert_allclose(gs[idx], rs, rtol=STATE_RTOL, atol=STATE_ATOL, err_msg="forward state")


def test_forward_pileup_events_match_oracle():
    """120 pile-up-5.5 events: every pixel-tracker track, its downstream hits and state."""
    b = velogen.generate(velogen.C2, n_events=120, truth=True)
    s = scifi.generate(b)
    R = reco(b)
    g = gpu_forward(R, s)
    ro = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params())
    r = oracle.forward(s.offsets, s.layer, s.x, s.y, ro, DOWN)
    assert len(r[0]) == int(R.totals[1]) > 20000
    assert_forward_same(g, r)
    assert (r[0] > 0).mean() > 0.3  # a real share of the tracks has a downstream track
    assert np.array_equal(g[2].view(np.uint32), r[2].view(np.uint32))  # in practice bit for bit


def test_forward_full_size_sampled():
    """10k pile-up-5.5 events in one launch; sampled events re-generated alone
    and checked against the oracle one by one."""
    cfg = velogen.C2
    b = velogen.generate(cfg, truth=True)
    s = scifi.generate(b)
    R = reco(b)
    g = gpu_forward(R, s)
    to = R.track_offsets.cpu().numpy()
    rng = np.random.default_rng(7)
    for e in sorted(rng.choice(cfg.n_events, size=25, replace=False).tolist()) + [0, cfg.n_events - 1]:
        one = velogen.generate(cfg, n_events=1, first_event=e, truth=True)
        so = scifi.generate(one)
        np.testing.assert_array_equal(so.x, s.x[int(s.offsets[e]):int(s.offsets[e + 1])])
        ro = oracle.reconstruct(one.offsets, one.pixels, one.geometry, oracle.Params())
        r = oracle.forward(so.offsets, so.layer, so.x, so.y, ro, DOWN)
        assert_forward_same(g, r, tracks=range(int(to[e]), int(to[e + 1])))
    # properties at full size: hit ids inside their events, counts agree with the lists
    n, h, st = g
    so_ = s.offsets.astype(np.int64)
    ev = np.repeat(np.arange(cfg.n_events), np.diff(to.astype(np.int64)))
    assert np.array_equal(n, (h != NONE).sum(1))
    nh = (so_[ev + 1] - so_[ev])[:, None]
    assert np.all((h == NONE) | (h.astype(np.int64) < nh))
    found = n > 0
    assert np.all(n[found] >= 9) and np.all(st[found, 1] <= 4.0) and np.all(st[~found] == 0)


class _Tracks:
    """A hand-built pixel-tracker result in device memory, in the layout
    velo_forward reads (cluster and track CSR arrays, totals)."""

    def __init__(self, res, cap_tracks=0):
        E = len(res["track_offsets"]) - 1
        self.keep = [dev(res["cluster_offsets"], np.uint64, np.int64), dev(res["cluster_x"], np.float32),
                     dev(res["cluster_y"], np.float32), dev(res["cluster_z"], np.float32),
                     dev(res["track_offsets"], np.uint64, np.int64),
                     dev(res["track_hit_offsets"], np.uint64, np.int64), dev(res["track_hits"], np.uint32, np.int32)]
        T = int(res["track_offsets"][-1])
        self.totals = torch.tensor([len(res["cluster_x"]), T, len(res["track_hits"]), 0], dtype=torch.int64,
                                   device="cuda")
        p = [int(t.data_ptr()) if t.numel() else 256 for t in self.keep]
        self._out = velo.Output(None, p[0], p[1], p[2], p[3], None, p[4], p[5], p[6], None,
                                int(self.totals.data_ptr()), None, 0, cap_tracks, 0)
        self.n_events = E


def run_both(res, off, layer, x, y, params=oracle.FwdParams(), cap_tracks=0):
    T = _Tracks(res, cap_tracks)
    vp = velo.default_forward_params(**{k: getattr(params, k) for k, _ in velo.ForwardParams._fields_})
    F = velo.ForwardTracker(DOWN, vp, max_events=max(T.n_events, 1), max_hits=max(len(x), 1),
                            cap_tracks=max(int(res["track_offsets"][-1]), 1))
    F.run(T, dev(off, np.uint64, np.int64), dev(layer, np.uint32, np.int32), dev(x, np.float32), dev(y, np.float32))
    g = to_numpy(F.result())
    r = oracle.forward(off, layer, x, y, res, DOWN, params)
    return (g["n_found"].astype(np.uint32), g["hits"].astype(np.uint32), g["state"]), r


def lines_result(events):
    """events: list (per event) of pixel-tracker lines ((x_b, y_b, z_b), (x_a, y_a, z_a))."""
    cx, cy, cz, co, to, tho, th = [], [], [], [0], [0], [0], []
    for lines in events:
        for (b, a) in lines:
            for (x, y, z) in (b, a):
                cx.append(x)
                cy.append(y)
                cz.append(z)
            th += [2 * (len(tho) - 1 - to[-1]), 2 * (len(tho) - 1 - to[-1]) + 1]
            tho.append(len(th))
        co.append(len(cx))
        to.append(len(tho) - 1)
    return {"cluster_offsets": np.array(co, np.uint64), "cluster_x": np.array(cx, np.float32),
            "cluster_y": np.array(cy, np.float32), "cluster_z": np.array(cz, np.float32),
            "track_offsets": np.array(to, np.uint64), "track_hit_offsets": np.array(tho, np.uint64),
            "track_hits": np.array(th, np.uint32)}


def line_hits(line, qop, layers=range(12), shift=0.0):
    (xb, yb, zb), (xa, ya, za) = line
    tx, ty = (xa - xb) / (za - zb), (ya - yb) / (za - zb)
    xm, ym = xa + tx * (DOWN.z_mag - za), ya + ty * (DOWN.z_mag - za)
    tk = tx + DOWN.kappa * qop
    return [(L, xm + tk * (DOWN.z_layers[L] - DOWN.z_mag) + shift, ym + ty * (DOWN.z_layers[L] - DOWN.z_mag))
            for L in layers]


def csr(events_hits):
    off = np.zeros(len(events_hits) + 1, np.uint64)
    off[1:] = np.cumsum([len(h) for h in events_hits])
    flat = [q for h in events_hits for q in h]
    return (off, np.array([q[0] for q in flat], np.uint32), np.array([q[1] for q in flat], np.float32),
            np.array([q[2] for q in flat], np.float32))


LINE = ((10.0, 5.0, 600.0), (11.5, 5.6, 750.0))
L2 = ((-20.0, 8.0, 600.0), (-21.2, 8.9, 750.0))


def test_constructed_cases_match_oracle():
    """The oracle's pin scenarios, one event each, in one batch: exact tracks
    of three momenta, a missing first layer, a kick outside the window, too
    few hits, a kinked segment, hit count against distance, distance ties,
    exact duplicates, two tracks, NaN and infinite coordinates, layer numbers
    past the last layer, an event without hits, an event without tracks."""
    nan, inf = float("nan"), float("inf")
    ex = line_hits(LINE, 0.1)
    cases = [
        ([LINE], line_hits(LINE, 1 / 8)), ([LINE], line_hits(LINE, -1 / 25)), ([LINE], line_hits(LINE, 1 / 50)),
        ([LINE], line_hits(LINE, 0.1, range(1, 12))),
        ([LINE], line_hits(LINE, 1 / (0.8 * 3.0))), ([LINE], line_hits(LINE, 1 / (1.2 * 3.0))),
        ([LINE], line_hits(LINE, 0.1, range(8))),
        ([LINE], line_hits(LINE, 0.1, range(8)) + line_hits(LINE, 0.1, range(8, 12), shift=1.5)),
        ([LINE], line_hits(LINE, 0.1, range(10)) + line_hits(LINE, 0.1, shift=6.0)),
        ([LINE], line_hits(LINE, 0.1, shift=5.0) + ex),
        ([LINE], ex + ex),
        ([LINE, L2], line_hits(LINE, 0.05) + line_hits(L2, -0.04)),
        ([LINE], [(L, x, nan) for (L, x, y) in ex] + [(L, nan, y) for (L, x, y) in ex[:6]]
         + [(L, inf, y) for (L, x, y) in ex[6:]] + ex),
        ([LINE], [(L + 12, x, y) for (L, x, y) in ex] + [(0xFFFFFFFF, x, y) for (L, x, y) in ex[:3]] + ex),
        ([LINE, L2], []),
        ([], ex),
        ([LINE], line_hits(LINE, 0.1, shift=24.9)), ([LINE], line_hits(LINE, 0.1, shift=-25.1)),
        ([LINE], line_hits(LINE, 0.1, range(4)) + line_hits(LINE, 0.1, range(4, 12), shift=2.9)),
    ]
    res = lines_result([c[0] for c in cases])
    g, r = run_both(res, *csr([c[1] for c in cases]))
    assert_forward_same(g, r)
    assert list(r[0][:6]) == [12, 12, 12, 11, 0, 12] and r[0][6] == 0  # the cases do what they say
    assert list(r[0][-3:-1]) == [12, 0]  # the match distance at 24.9 and 25.1 mm


@pytest.mark.parametrize("n_events,noise", [(24, (0, 5, 40, 500)), (3, (1700,))])
def test_dense_layers_and_ragged_events(n_events, noise):
    """Events of 0 to ~6000 hits (noise up to 500 per layer, several radix
    digits and bisection depths, ragged tails; the small and the large-event
    kernels) and events of ~20000 hits (hits kept in the workspace) with
    tracks in them; exact x duplicates among the noise."""
    rng = np.random.default_rng(11 + n_events)
    events, hits = [], []
    for e in range(n_events):
        n_lines = int(rng.integers(0, 12))
        lines = []
        hs = []
        for _ in range(n_lines):
            xb, yb = rng.uniform(-30, 30, 2)
            tx, ty = rng.uniform(-0.25, 0.25, 2)
            line = ((xb, yb, 500.0), (xb + 150 * tx, yb + 150 * ty, 650.0))
            lines.append(line)
            qop = rng.choice([-1, 1]) / rng.uniform(2.0, 80.0)
            hs += [(L, x + rng.normal(0, 0.08), y + rng.normal(0, 1.0)) for (L, x, y) in line_hits(line, qop)
                   if rng.random() < 0.97]
        n_noise = int(rng.choice(noise))
        for L in range(12):
            xs = rng.uniform(-3000, 3000, n_noise).astype(np.float32)
            if n_noise > 10:
                xs[: n_noise // 10] = xs[0]  # exact ties in x
            hs += [(L, float(x), float(y)) for x, y in zip(xs, rng.uniform(-2500, 2500, n_noise))]
        order = rng.permutation(len(hs))
        events.append(lines)
        hits.append([hs[i] for i in order])
    res = lines_result(events)
    g, r = run_both(res, *csr(hits))
    assert_forward_same(g, r)
    assert (r[0] > 0).sum() > (20 if n_events > 3 else 3)


def test_bad_offsets_and_overflowed_result():
    """Hit offsets that decrease: every track has no downstream track.  A
    pixel-tracker result whose totals exceed its capacity: nothing is written."""
    res = lines_result([[LINE], [L2]])
    off, layer, x, y = csr([line_hits(LINE, 0.1), line_hits(L2, -0.04)])
    T = _Tracks(res)
    F = velo.ForwardTracker(DOWN, max_events=2, max_hits=len(x), cap_tracks=2)
    F.n_found.fill_(77)
    bad = off.copy()
    bad[1] = bad[2] + 1
    F.run(T, dev(bad, np.uint64, np.int64), dev(layer, np.uint32, np.int32), dev(x, np.float32), dev(y, np.float32))
    g = to_numpy(F.result())
    assert list(g["n_found"]) == [0, 0] and np.all(g["hits"] == -1) and np.all(g["state"] == 0)
    F.run(T, dev(off, np.uint64, np.int64), dev(layer, np.uint32, np.int32), dev(x, np.float32), dev(y, np.float32))
    assert list(to_numpy(F.result())["n_found"]) == [12, 12]
    small = _Tracks(res, cap_tracks=1)  # 2 tracks in a result of capacity 1
    F.n_found.fill_(77)
    F.run(small, dev(off, np.uint64, np.int64), dev(layer, np.uint32, np.int32), dev(x, np.float32),
          dev(y, np.float32))
    torch.cuda.synchronize()
    assert F.n_found[:2].tolist() == [77, 77]


def test_empty_batch():
    res = lines_result([])
    T = _Tracks(res)
    F = velo.ForwardTracker(DOWN, max_events=1, max_hits=1, cap_tracks=1)
    e = torch.zeros(1, dtype=torch.int64, device="cuda")
    z = torch.zeros(0, dtype=torch.float32, device="cuda")
    F.run(T, e, torch.zeros(0, dtype=torch.int32, device="cuda"), z, z)
    assert F.result()["n_found"].numel() == 0


def test_track_capacity_cuts_the_output():
    """Tracks at and past cap_tracks are not written; the others are."""
    res = lines_result([[LINE, L2]])
    off, layer, x, y = csr([line_hits(LINE, 0.05) + line_hits(L2, -0.04)])
    T = _Tracks(res)
    F = velo.ForwardTracker(DOWN, max_events=1, max_hits=len(x), cap_tracks=1)
    F.run(T, dev(off, np.uint64, np.int64), dev(layer, np.uint32, np.int32), dev(x, np.float32), dev(y, np.float32))
    g = to_numpy(F.result())
    assert list(g["n_found"]) == [12] and list(g["hits"][0]) == list(range(12))
