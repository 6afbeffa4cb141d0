"""Pins of the oracle's pattern recognition (seeding, extension, termination,
3-hit rule, chi2/ndf cut, canonical order), CPU only.

The paper names the first stage's pattern recognition only as "simplified"
(Sec. "HLT1 details and results"); the oracle's definition is pinned here by
results that follow from geometry and the definition's rules without running
its code:
* hand-built events whose answer is fixed by construction: a seed conflict,
  contention for one hit during extension, a skipped module and termination,
  a track across the pseudo-angle wrap at phi = 0, the 3-hit chi2 rule at its
  closed-form threshold;
* exact recovery of isolated noise-free straight tracks from the generator;
* Monte-Carlo invariants on generated events (efficiency, ghost and clone
  rates) and structural invariants of every output (disjoint hits, distinct
  ascending modules, gaps <= max_skipped, cuts respected, canonical order).
"""
import numpy as np
import pytest

import oracle
import velogen
from oracle import mc

Z = -300.0 + 42.0 * np.arange(26)
P0 = oracle.Params(ms_theta=0.0)


def make_hits(points):
    """points: dict label -> (module, x, y).  Returns module/x/y arrays in id order
    (grouped by module, ascending) and label -> id."""
    labels = sorted(points, key=lambda k: (points[k][0], k))
    ids = {lab: i for i, lab in enumerate(labels)}
    module = np.array([points[k][0] for k in labels], np.uint32)
    x = np.array([points[k][1] for k in labels], np.float32)
    y = np.array([points[k][2] for k in labels], np.float32)
    return module, x, y, ids


def line(x0, y0, tx, ty, zref, mods):
    return {m: (x0 + tx * (Z[m] - zref), y0 + ty * (Z[m] - zref)) for m in mods}


def beam_line(tx, ty, zv, mods, dx=0.0, dy=0.0):
    """Straight line from (dx, dy, zv) near the beam axis: constant phi, as the
    pseudo-angle windows (centred on the previous hit) assume."""
    return {m: (dx + tx * (Z[m] - zv), dy + ty * (Z[m] - zv)) for m in mods}


def run(points, params=P0):
    module, x, y, ids = make_hits(points)
    tracks, states = oracle.track_event(module, x, y, velogen.Geometry(), params)
    return [list(map(int, t)) for t in tracks], states, ids


def test_single_straight_track():
    L = line(10.0, 4.0, 0.05, 0.02, 0.0, range(3, 12))
    pts = {f"h{m}": (m, *L[m]) for m in L}
    tracks, states, ids = run(pts)
    assert tracks == [sorted(ids.values())]
    assert states[0][18] == 2 * 9 - 4
    np.testing.assert_allclose(states[0][2], 0.05, atol=1e-6)


def test_seed_conflict_smaller_scatter_wins():
    """Two middle hits A, B on module 3 can both pair with the single h0 (module 4)
    and h2 (module 2).  A lies on the h0-h2 line, B 0.05 mm off it: A's seed has the
    smaller scatter and takes h0 and h2; B's seed is dropped and B stays unused."""
    L = line(12.0, 3.0, 0.04, 0.01, Z[3], [1, 2, 3, 4])
    pts = {"h0": (4, *L[4]), "A": (3, *L[3]), "B": (3, L[3][0] + 0.05, L[3][1]), "h2": (2, *L[2]),
           "h1m": (1, *L[1])}
    tracks, _, ids = run(pts)
    assert tracks == [sorted([ids["h1m"], ids["h2"], ids["A"], ids["h0"]])]


def test_seed_conflict_tie_goes_to_smaller_middle_id():
    """B mirrored to the other side of the line at the same distance: equal scatter,
    the smaller middle-hit id wins."""
    L = line(12.0, 3.0, 0.04, 0.0, Z[3], [1, 2, 3, 4])
    pts = {"h0": (4, *L[4]), "A": (3, L[3][0], L[3][1] + 0.03), "B": (3, L[3][0], L[3][1] - 0.03),
           "h2": (2, *L[2]), "h1m": (1, *L[1])}
    tracks, _, ids = run(pts)
    win = min(ids["A"], ids["B"])
    assert len(tracks) == 1 and win in tracks[0] and ids["h0"] in tracks[0]


def test_seed_tie_between_two_h0_goes_to_smaller_id():
    """Two h0 candidates mirrored about a line in y = 0 (y0 = +d and -d, the same
    x): the seed's scatter is exactly equal for both (negation is exact and the
    square drops the sign), so the tie rule decides: the smaller h0 id wins."""
    d = 0.0625
    pts = {"h2": (2, 20.0, 0.0), "h1": (3, 21.0, 0.0), "h0a": (4, 22.0, d), "h0b": (4, 22.0, -d)}
    tracks, _, ids = run(pts)
    assert len(tracks) == 1
    win = min(ids["h0a"], ids["h0b"])
    assert sorted(tracks[0]) == sorted([ids["h2"], ids["h1"], win])


def test_seed_lever_arms_with_uneven_module_spacing():
    """Modules 20, 30, 70 and 90 mm apart: a noise-free straight track is found
    only if the seed extrapolates with the lever arms of its own three modules
    (equal spacing would hide a swapped lever arm)."""
    zs = np.array([-300.0, -280.0, -250.0, -180.0, -90.0, 0.0, 20.0, 60.0, 130.0, 200.0, 230.0, 300.0])
    geo = velogen.Geometry(n_modules=len(zs), module_z=tuple(zs.tolist()))
    tx, ty = 0.06, 0.03
    pts = {f"h{m}": (m, np.float32(5.0 + tx * (zs[m] - zs[0])), np.float32(3.0 + ty * (zs[m] - zs[0])))
           for m in range(len(zs))}
    module, x, y, ids = make_hits(pts)
    tracks, states = oracle.track_event(module, x, y, geo, P0)
    assert [sorted(map(int, t)) for t in tracks] == [sorted(ids.values())]
    np.testing.assert_allclose(states[0][2], tx, atol=1e-6)
    np.testing.assert_allclose(states[0][3], ty, atol=1e-6)


def test_extension_contention_and_skip():
    """Tracks A and B pass within 0.05 mm of one hit on module 7; A exactly through it.
    A takes it, B counts module 7 as skipped and continues on module 6."""
    zc = Z[7]
    A = line(8.0, 8.0, 0.050, 0.050, zc, range(6, 11))
    B = line(8.05, 8.0, 0.055, 0.050, zc, range(6, 11))
    pts = {}
    for m in (10, 9, 8, 6):
        pts[f"a{m}"] = (m, *A[m])
        pts[f"b{m}"] = (m, *B[m])
    pts["h7"] = (7, *A[7])
    tracks, _, ids = run(pts)
    ta = sorted(ids[k] for k in ("a10", "a9", "a8", "h7", "a6"))
    tb = sorted(ids[k] for k in ("b10", "b9", "b8", "b6"))
    assert sorted(tracks) == sorted([ta, tb])


def test_termination_after_max_skipped():
    """Hits on 20, 19, 18, 16 and 13 of one line: the track skips 17, takes 16, misses
    15 and 14, and terminates at step 13 (16 - 13 - 1 = 2 modules missed > max_skipped = 1)."""
    L = beam_line(-0.03, 0.06, 10.0, range(13, 21))
    pts = {f"h{m}": (m, *L[m]) for m in (20, 19, 18, 16, 13)}
    tracks, _, ids = run(pts)
    assert tracks == [sorted(ids[f"h{m}"] for m in (20, 19, 18, 16))]
    # with max_skipped = 2 the hit on module 13 joins
    tracks2, _, _ = run(pts, oracle.Params(ms_theta=0.0, max_skipped=2))
    assert tracks2 == [sorted(ids.values())]


def test_pseudo_angle_wrap():
    """A track at phi ~ 0 whose y changes sign between modules: its keys sit near
    4 on one side and near 0 on the other and must still be one window."""
    L = line(20.0, -0.004, 0.02, 0.0001, Z[13], range(8, 19))
    pts = {f"h{m}": (m, *L[m]) for m in L}
    keys = [oracle.pseudo_angle(float(np.float32(v[1])), float(np.float32(v[2]))) for v in pts.values()]
    assert max(keys) > 3.99 and min(keys) < 0.01
    tracks, _, ids = run(pts)
    assert tracks == [sorted(ids.values())]


@pytest.mark.parametrize("delta,kept", [(0.035, True), (0.045, False)])
def test_three_hit_rule_closed_form(delta, kept):
    """Three hits with the middle one displaced by delta: chi2/ndf = delta^2 / (3 sigma^2)
    (2 delta^2 / (3 sigma^2) over ndf = 2).  With sigma = 0.0159 the 3-hit cut of 2.0
    sits at delta = 0.0389 mm."""
    L = line(15.0, 15.0, 0.03, 0.03, Z[5], [4, 5, 6])
    pts = {"a": (6, *L[6]), "b": (5, L[5][0] + delta, L[5][1]), "c": (4, *L[4])}
    tracks, states, _ = run(pts)
    assert (len(tracks) == 1) == kept
    if kept:
        np.testing.assert_allclose(states[0][6] / states[0][18], delta ** 2 / (3 * 0.0159 ** 2), rtol=1e-3)


def test_pseudo_angle_closed_forms():
    r2 = np.sqrt(0.5)
    cases = {(1, 0): 0.0, (r2, r2): 0.5, (0, 1): 1.0, (-r2, r2): 1.5, (-1, 0): 2.0, (-r2, -r2): 2.5,
             (0, -1): 3.0, (r2, -r2): 3.5}
    for (x, y), k in cases.items():
        assert oracle.pseudo_angle(10 * x, 10 * y) == pytest.approx(k, abs=1e-6)
    # first quadrant: k = sin(phi) / (sin(phi) + cos(phi)); monotone over the full turn
    phi = np.linspace(0, 2 * np.pi, 20001, endpoint=False)
    ks = np.array([oracle.pseudo_angle(float(np.float32(7 * np.cos(p))), float(np.float32(7 * np.sin(p)))) for p in phi])
    assert (np.diff(ks) >= 0).all() and ks.min() >= 0 and ks.max() < 4
    q1 = phi < np.pi / 2
    np.testing.assert_allclose(ks[q1], np.sin(phi[q1]) / (np.sin(phi[q1]) + np.cos(phi[q1])), atol=2e-6)


def test_isolated_straight_tracks_recovered_exactly():
    """One noise-free straight track per event with full efficiency: its clusters are
    one per crossed module, and the single reconstructed track holds exactly all of
    them whenever there are >= 3 (slope within the digitisation bound)."""
    cfg = velogen.Config(seed=21, n_events=300, fixed_pvs=1, fixed_tracks=1, ms_theta=0.0, hit_eff=1.0,
                         noise_prob=0.0)
    b = velogen.generate(cfg, truth=True)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, P0)
    n_checked = 0
    for e in range(b.n_events):
        nc = int(r["cluster_offsets"][e + 1] - r["cluster_offsets"][e])
        t0, t1 = int(r["track_offsets"][e]), int(r["track_offsets"][e + 1])
        if nc < 3:
            assert t1 == t0
            continue
        n_checked += 1
        assert t1 - t0 == 1, e
        hits = r["track_hits"][int(r["track_hit_offsets"][t0]):int(r["track_hit_offsets"][t0 + 1])]
        np.testing.assert_array_equal(hits, np.arange(nc))
        st = r["track_states"][t0]
        z = r["cluster_z"][int(r["cluster_offsets"][e]):int(r["cluster_offsets"][e + 1])]
        bound = 2 * b.geometry.pitch / (z.max() - z.min())
        assert abs(st[2] - b.particles[e][4]) <= bound and abs(st[3] - b.particles[e][5]) <= bound
    assert n_checked > 250


def check_structure(b, r, p):
    zmod = {float(np.float32(z)): i for i, z in enumerate(b.geometry.module_z)}
    for e in range(b.n_events):
        c0 = int(r["cluster_offsets"][e])
        cz = r["cluster_z"][c0:int(r["cluster_offsets"][e + 1])]
        t0, t1 = int(r["track_offsets"][e]), int(r["track_offsets"][e + 1])
        seen = set()
        firsts = []
        for t in range(t0, t1):
            h = r["track_hits"][int(r["track_hit_offsets"][t]):int(r["track_hit_offsets"][t + 1])]
            assert len(h) >= 3 and (np.diff(h.astype(np.int64)) > 0).all()
            mods = np.array([zmod[float(cz[i])] for i in h])
            assert (np.diff(mods) > 0).all() and (np.diff(mods) - 1 <= p.max_skipped).all()
            assert not (seen & set(h.tolist()))
            seen |= set(h.tolist())
            st = r["track_states"][t]
            chi2 = st[6] if p.ms_theta == 0 else st[7]
            rr = np.float32(chi2) / np.float32(2 * len(h) - 4)
            assert rr <= p.chi2ndf_max and (len(h) > 3 or rr <= p.chi2ndf_max_3hit)
            firsts.append(list(h))
        assert firsts == sorted(firsts)


def test_config1_invariants():
    b = velogen.generate(velogen.C1, truth=True)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, P0)
    m = mc.evaluate_batch(b, r)
    assert m["efficiency"] >= 0.995 and m["ghost_rate"] <= 0.005 and m["clone_rate"] <= 0.005, m
    check_structure(b, r, P0)


def test_config2_invariants():
    b = velogen.generate(velogen.C2, n_events=60, truth=True)
    p = oracle.Params()
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, p)
    m = mc.evaluate_batch(b, r)
    assert m["efficiency"] >= 0.99 and m["ghost_rate"] <= 0.05 and m["clone_rate"] <= 0.01, m
    check_structure(b, r, p)


def test_reconstruct_is_thread_count_independent():
    b = velogen.generate(velogen.C2, n_events=16)
    a = oracle.reconstruct(b.offsets, b.pixels, b.geometry, n_threads=1)
    c = oracle.reconstruct(b.offsets, b.pixels, b.geometry, n_threads=5)
    for k in a:
        np.testing.assert_array_equal(a[k], c[k])
