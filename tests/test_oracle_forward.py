"""Pins of the oracle's forward tracking (pixel-tracker tracks traced to the
downstream layers through a single kick), CPU only.

The paper describes the step in words (Sec. "HLT1 details and results"):
straight to the middle of the magnet, one change of angle there, straight to
the fibre tracker, hits found and the track kept with enough hits and a low
chi2.  The pins tie the oracle's reading to geometry rather than to itself:
* a noise-free track built from a known momentum and charge is found with
  all its hits, q/p equal to the generating q/p, zero chi2 and zero match
  distances;
* the candidate rules by construction: a missing first-layer hit (found
  through the second layer), a kick outside the momentum window, too few
  hits, a kinked downstream segment (chi2 cut), and competing candidates
  settled by hit count, then match distance, then candidate id;
* Monte-Carlo invariants on generated pile-up events.
"""
import numpy as np
import pytest

import oracle
import velogen
from velogen import scifi

DOWN = scifi.Downstream()
ZL = np.array(DOWN.z_layers)
NONE = 0xFFFFFFFF


def velo_result(lines):
    """Pixel-tracker tracks of one event, each given as two clusters
    ((x_b, y_b, z_b), (x_a, y_a, z_a)) with z_b < z_a."""
    cx, cy, cz = [], [], []
    for (b, a) in lines:
        for (x, y, z) in (b, a):
            cx.append(x)
            cy.append(y)
            cz.append(z)
    n = len(lines)
    return {"cluster_offsets": np.array([0, 2 * n], np.uint64), "cluster_x": np.array(cx, np.float32),
            "cluster_y": np.array(cy, np.float32), "cluster_z": np.array(cz, np.float32),
            "track_offsets": np.array([0, n], np.uint64), "track_hit_offsets": np.arange(0, 2 * n + 1, 2, dtype=np.uint64),
            "track_hits": np.arange(2 * n, dtype=np.uint32)}


def track_hits(line, qop, layers=range(12), x_shift=None):
    """Exact downstream hits of the pixel-tracker line `line` after a kick kappa * qop."""
    (xb, yb, zb), (xa, ya, za) = line
    tx, ty = (xa - xb) / (za - zb), (ya - yb) / (za - zb)
    xm, ym = xa + tx * (DOWN.z_mag - za), ya + ty * (DOWN.z_mag - za)
    tk = tx + DOWN.kappa * qop
    out = []
    for L in layers:
        dz = ZL[L] - DOWN.z_mag
        x = xm + tk * dz + (x_shift[L] if x_shift is not None else 0.0)
        out.append((L, x, ym + ty * dz))
    return out


def run(lines, hits, params=oracle.FwdParams()):
    layer = np.array([h[0] for h in hits], np.uint32)
    x = np.array([h[1] for h in hits], np.float32)
    y = np.array([h[2] for h in hits], np.float32)
    off = np.array([0, len(hits)], np.uint64)
    return oracle.forward(off, layer, x, y, velo_result(lines), DOWN, params)


LINE = ((10.0, 5.0, 600.0), (11.5, 5.6, 750.0))  # tx = 0.01, ty = 0.004


@pytest.mark.parametrize("qop", [1.0 / 8.0, -1.0 / 25.0, 1.0 / 50.0])
def test_exact_track_found_with_its_momentum(qop):
    hits = track_hits(LINE, qop)
    n, h, st = run([LINE], hits)
    assert n[0] == 12 and list(h[0]) == list(range(12))
    assert abs(st[0][0] - qop) <= 2e-4 * abs(qop) + 1e-6   # q/p
    assert st[0][1] <= 1e-2                                 # chi2/ndf of exact points
    assert abs(st[0][4]) <= 1e-2 and abs(st[0][5]) <= 1e-2  # the lines meet at the kick plane


def test_missing_first_layer_hit_found_through_second():
    hits = track_hits(LINE, 0.1, layers=range(1, 12))
    n, h, _ = run([LINE], hits)
    assert n[0] == 11 and h[0][0] == NONE and list(h[0][1:]) == list(range(11))


def test_kick_outside_momentum_window_not_searched():
    p = oracle.FwdParams()
    hits = track_hits(LINE, 1.0 / (0.8 * p.p_min))  # momentum below p_min: the kick is outside the window
    n, _, _ = run([LINE], hits, p)
    assert n[0] == 0
    n2, _, _ = run([LINE], track_hits(LINE, 1.0 / (1.2 * p.p_min)), p)
    assert n2[0] == 12


def test_too_few_hits():
    p = oracle.FwdParams()
    hits = track_hits(LINE, 0.1, layers=range(p.min_hits - 1))
    n, _, _ = run([LINE], hits, p)
    assert n[0] == 0
    n2, _, _ = run([LINE], track_hits(LINE, 0.1, layers=range(p.min_hits)), p)
    assert n2[0] == p.min_hits


def test_kinked_segment_fails_the_chi2_cut():
    shift = np.zeros(12)
    shift[8:] = 1.5  # the last station 1.5 mm off the line: far beyond sigma_x, inside tol_x_far
    n, _, _ = run([LINE], track_hits(LINE, 0.1, x_shift=shift))
    assert n[0] == 0
    shift[8:] = 0.02  # a fraction of sigma_x
    n2, _, _ = run([LINE], track_hits(LINE, 0.1, x_shift=shift))
    assert n2[0] == 12


def test_more_hits_win_over_smaller_distance():
    """Two downstream segments in reach of one pixel-tracker track: one exact
    with 10 hits, one shifted by 6 mm at every layer (a parallel line, zero
    chi2, match distance 6 mm; outside the far-station window of the other)
    with 12.  Both candidates pass the cuts; the 12-hit one wins."""
    exact = track_hits(LINE, 0.1, layers=range(10))
    shifted = [(L, x + 6.0, y) for (L, x, y) in track_hits(LINE, 0.1)]
    n, h, st = run([LINE], exact + shifted)
    assert n[0] == 12 and list(h[0]) == list(range(10, 22))
    assert abs(abs(st[0][4]) - 6.0) < 1e-2
    n10, h10, st10 = run([LINE], exact)  # the exact segment alone passes too
    assert n10[0] == 10 and abs(st10[0][4]) < 1e-2


def test_equal_hits_smaller_distance_wins():
    exact = track_hits(LINE, 0.1)
    shifted = [(L, x + 5.0, y) for (L, x, y) in track_hits(LINE, 0.1)]
    n, h, _ = run([LINE], shifted + exact)  # the exact segment has the larger ids
    assert n[0] == 12 and list(h[0]) == list(range(12, 24))


def test_exact_tie_goes_to_smaller_candidate_id():
    """Duplicated hits: both candidates collect the same set (the nearest hit
    of every layer, ties to the smaller id), so distance and hits tie; the
    candidate with the smaller id is kept -- the hits themselves are the
    smaller ids either way."""
    exact = track_hits(LINE, 0.1)
    n, h, _ = run([LINE], exact + exact)
    assert n[0] == 12 and list(h[0]) == list(range(12))


def test_every_track_is_searched_independently():
    L2 = ((-20.0, 8.0, 600.0), (-21.2, 8.9, 750.0))
    n, h, st = run([LINE, L2], track_hits(LINE, 0.05) + track_hits(L2, -0.04))
    assert list(n) == [12, 12]
    assert list(h[0]) == list(range(12)) and list(h[1]) == list(range(12, 24))
    assert abs(st[0][0] - 0.05) < 1e-4 and abs(st[1][0] + 0.04) < 1e-4


@pytest.mark.slow
def test_generated_events_invariants():
    """Pile-up 5.5 events: tracks of particles above 5 GeV/c are found at
    >= 95 %, >= 85 % of the found ones carry their own particle's hits, and
    q/p is measured to 2 % (median)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2412_05041_b300 import truth
    b = velogen.generate(velogen.C2, n_events=12, first_event=40, truth=True)
    s = scifi.generate(b)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params())
    n, h, st = oracle.forward(s.offsets, s.layer, s.x, s.y, r, s.geometry)
    m = truth.track_matches(r, truth.cluster_truth(b, r))
    to, so, po = (a.astype(np.int64) for a in (r["track_offsets"], s.offsets, b.particle_offsets))
    ev = np.repeat(np.arange(b.n_events), np.diff(to))
    hi = [t for t in range(len(n)) if m[t] >= 0 and s.p[m[t]] > 5.0]
    found = [t for t in hi if n[t] > 0]
    assert len(found) >= 0.95 * len(hi)
    own, res = 0, []
    for t in found:
        hs = h[t][h[t] != NONE].astype(np.int64)
        if np.mean(po[ev[t]] + s.truth[so[ev[t]] + hs] == m[t]) >= 0.7:
            own += 1
            qop = s.q[m[t]] / s.p[m[t]]
            res.append(abs(st[t][0] - qop) / abs(qop))
    assert own >= 0.85 * len(found)
    assert np.median(res) <= 0.02


def test_non_finite_hits_never_taken():
    """A window test holds only for a distance that is a number: hits on the
    track's x with a NaN y, and hits with a NaN or infinite x, are never
    taken, even with the smaller ids (as distances they would tie or beat
    the real hits under a plain `>` rejection)."""
    exact = track_hits(LINE, 0.1)
    nan = float("nan")
    bad = [(L, x, nan) for (L, x, y) in exact] + [(L, nan, y) for (L, x, y) in exact[:6]] + \
          [(L, float("inf"), y) for (L, x, y) in exact[6:]]
    n, h, st = run([LINE], bad + exact)
    assert n[0] == 12 and list(h[0]) == list(range(24, 36))
    n0, _, st0 = run([LINE], exact)
    assert np.array_equal(st[0], st0[0])


def test_track_of_one_hit_has_no_line():
    """A pixel-tracker track of fewer than two hits gets no downstream track;
    the others are unaffected."""
    res = velo_result([LINE])
    res["cluster_x"] = np.append(res["cluster_x"], np.float32(3.0))
    res["cluster_y"] = np.append(res["cluster_y"], np.float32(3.0))
    res["cluster_z"] = np.append(res["cluster_z"], np.float32(700.0))
    res["cluster_offsets"] = np.array([0, 3], np.uint64)
    res["track_offsets"] = np.array([0, 2], np.uint64)
    res["track_hit_offsets"] = np.array([0, 2, 3], np.uint64)
    res["track_hits"] = np.array([0, 1, 2], np.uint32)
    hits = track_hits(LINE, 0.1)
    off = np.array([0, len(hits)], np.uint64)
    n, h, st = oracle.forward(off, np.array([q[0] for q in hits], np.uint32), np.array([q[1] for q in hits], np.float32),
                              np.array([q[2] for q in hits], np.float32), res, DOWN)
    assert list(n) == [12, 0] and np.all(h[1] == NONE) and np.all(st[1] == 0)
