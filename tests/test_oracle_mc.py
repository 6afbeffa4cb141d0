"""Pins of the Monte-Carlo truth matching (oracle/mc.py) against hand-counted
events (CPU only).

The definitions being pinned (efficiency and ghost rate of the first stage's
tracking, which the paper reports for its real detector but not in figures
this project can reuse, Sec. "HLT1 details and results"):

* a cluster's truth is the particle with the largest summed charge over its
  pixels; noise counts as id -1, and ties go to the smaller id (so a tie
  between noise and a particle leaves the cluster as noise);
* a track matches particle P when at least 70 % of ALL its hits carry P;
* a particle is reconstructible with clusters on at least 3 distinct modules;
* efficiency = reconstructible particles matched by a track / reconstructible,
  ghost rate = unmatched tracks / tracks, clone rate = matches beyond the
  first of each particle / matched particles.

The two events below are written as tables of clusters (module, pixel
deposits (truth, charge)) and tracks (cluster indices).  Every figure in the
expected values was counted by hand from these tables; the comments give the
count.  Each plausible misreading changes at least one figure: ``>`` instead
of ``>=`` 70 % (track T1 sits at exactly 7 of 10), 2 modules instead of 3 or
clusters instead of distinct modules (P3: 3 clusters on 2 modules), ties to
the larger id (cluster 49), particles preferred over noise in a tie
(cluster 54), pixel counts or the largest single deposit instead of the
summed charge (clusters 57 and event 1's cluster 3), the 70 % taken over the
truth-carrying hits only (T2, T7), clone and efficiency denominators.
"""
from types import SimpleNamespace

import numpy as np

from oracle import mc

N = -1  # noise

# event 0: (module, [(truth, q), ...]) per cluster, in cluster id order
EVENT0_CLUSTERS = (
    [(m, [(0, 10)]) for m in range(10)]          # c0-c9: P0 on modules 0-9
    + [(m, [(1, 10)]) for m in range(10)]        # c10-c19: P1 on modules 0-9
    + [(m, [(2, 10)]) for m in range(10)]        # c20-c29: P2 on modules 0-9
    + [(m, [(N, 7)]) for m in range(10)]         # c30-c39: noise
    + [(4, [(3, 10)]), (4, [(3, 10)]), (5, [(3, 10)])]    # c40-c42: P3, 3 clusters on 2 modules
    + [(7, [(4, 10)]), (8, [(4, 10)]), (9, [(4, 10)])]    # c43-c45: P4 on 3 modules
    + [(0, [(5, 10)]), (1, [(5, 10)]), (2, [(5, 10)])]    # c46-c48: P5
    + [(3, [(5, 6), (6, 6)])]                              # c49: P5 / P6 tie -> P5
    + [(4, [(6, 10)]), (5, [(6, 10)])]                     # c50-c51: P6
    + [(0, [(7, 10)]), (1, [(7, 10)])]                     # c52-c53: P7
    + [(2, [(7, 5), (N, 5)])]                              # c54: P7 / noise tie -> noise
    + [(6, [(9, 10)]), (7, [(9, 10)])]                     # c55-c56: P9
    + [(8, [(8, 3), (8, 3), (8, 3), (9, 12)])]             # c57: P8 9 over 3 pixels, P9 12 in one -> P9
)
EVENT0_PARTICLES = 10
EVENT0_TRACKS = [
    list(range(0, 10)),                       # T0: P0 10/10
    [0, 1, 2, 3],                             # T0b: P0 again -> a clone
    list(range(10, 17)) + [30, 31, 32],       # T1: P1 7/10 = exactly 70 % -> P1
    list(range(20, 26)) + [33, 34, 35],       # T2: P2 6/9 -> ghost
    [40, 41, 42],                             # T3: P3 3/3 (P3 not reconstructible)
    [46, 47, 49],                             # T5: P5 3/3 (with c49 -> P5)
    [55, 56, 57],                             # T9: P9 3/3 (c57 by summed charge)
    [52, 53, 54],                             # T7: P7 2/3 -> ghost
    [36, 37, 38],                             # Tn: noise only -> ghost
]
# truths: c0-9 P0, c10-19 P1, c20-29 P2, c30-39 noise, c40-42 P3, c43-45 P4, c46-49 P5,
# c50-51 P6, c52-53 P7, c54 noise, c55-57 P9
EVENT0_CLUSTER_TRUTH = [0] * 10 + [1] * 10 + [2] * 10 + [N] * 10 + [3] * 3 + [4] * 3 + [5] * 4 + [6] * 2 + [7] * 2 \
    + [N] + [9] * 3
# modules with truth: P0, P1, P2 10; P3 {4,5}; P4 {7,8,9}; P5 {0,1,2,3}; P6 {4,5}; P7 {0,1}; P8 none;
# P9 {6,7,8} -> reconstructible P0, P1, P2, P4, P5, P9
EVENT0_RECONSTRUCTIBLE = [True, True, True, False, True, True, False, False, False, True]
EVENT0_MATCHED = [0, 0, 1, N, 3, 5, 9, N, N]

# event 1: P0 on modules 0-3, its cluster 3 shared with a single large P1 deposit
EVENT1_CLUSTERS = [
    (0, [(0, 10)]), (1, [(0, 10)]), (2, [(0, 10)]),
    (3, [(0, 8), (0, 8), (1, 15)]),           # c3: P0 16 over two pixels, P1 15 in one -> P0
    (5, [(1, 10)]), (5, [(1, 10)]), (6, [(1, 10)]),     # c4-c6: P1, 2 distinct modules
    (4, [(N, 9)]),                            # c7: noise
]
EVENT1_PARTICLES = 2
EVENT1_TRACKS = [[0, 1, 3]]                   # P0 3/3
EVENT1_RECONSTRUCTIBLE = [True, False]
EVENT1_MATCHED = [0]


def build_event(clusters):
    """Pixel words (only the charge field matters here), pixel truth, pixel
    cluster labels and the module of every cluster."""
    words, truth, label = [], [], []
    for c, (_, pixels) in enumerate(clusters):
        for t, q in pixels:
            words.append(q << 27)
            truth.append(t)
            label.append(c)
    return (np.array(words, np.uint32), np.array(truth, np.int32), np.array(label, np.uint32),
            np.array([m for m, _ in clusters], np.int64))


def match(clusters, tracks, n_particles):
    w, t, lab, mods = build_event(clusters)
    return mc.match_event(w, t, lab, len(clusters), mods, [np.array(x, np.uint32) for x in tracks], n_particles)


def test_cluster_truth_by_summed_charge_ties_to_smaller_id():
    w, t, lab, _ = build_event(EVENT0_CLUSTERS)
    np.testing.assert_array_equal(mc.cluster_truth(w, t, lab, len(EVENT0_CLUSTERS)), EVENT0_CLUSTER_TRUTH)
    w, t, lab, _ = build_event(EVENT1_CLUSTERS)
    np.testing.assert_array_equal(mc.cluster_truth(w, t, lab, len(EVENT1_CLUSTERS)), [0, 0, 0, 0, 1, 1, 1, N])


def test_cluster_truth_does_not_depend_on_pixel_order():
    w, t, lab, _ = build_event(EVENT0_CLUSTERS)
    perm = np.random.default_rng(11).permutation(len(w))
    np.testing.assert_array_equal(mc.cluster_truth(w[perm], t[perm], lab[perm], len(EVENT0_CLUSTERS)),
                                  EVENT0_CLUSTER_TRUTH)


def test_hand_counted_event_matching():
    r = match(EVENT0_CLUSTERS, EVENT0_TRACKS, EVENT0_PARTICLES)
    np.testing.assert_array_equal(r["reconstructible"], EVENT0_RECONSTRUCTIBLE)
    np.testing.assert_array_equal(r["matched"], EVENT0_MATCHED)
    r = match(EVENT1_CLUSTERS, EVENT1_TRACKS, EVENT1_PARTICLES)
    np.testing.assert_array_equal(r["reconstructible"], EVENT1_RECONSTRUCTIBLE)
    np.testing.assert_array_equal(r["matched"], EVENT1_MATCHED)


def test_hand_counted_rates():
    s = mc.summarize([match(EVENT0_CLUSTERS, EVENT0_TRACKS, EVENT0_PARTICLES)])
    # reconstructible 6 (P0 P1 P2 P4 P5 P9), of which matched 4 (P0 P1 P5 P9)
    assert s["reconstructible"] == 6 and s["efficiency"] == 4 / 6
    # 9 tracks, 3 ghosts (T2 T7 Tn); matched particles P0 P1 P3 P5 P9, one clone (T0b)
    assert s["tracks"] == 9 and s["ghost_rate"] == 3 / 9 and s["clone_rate"] == 1 / 5
    both = mc.summarize([match(EVENT0_CLUSTERS, EVENT0_TRACKS, EVENT0_PARTICLES),
                         match(EVENT1_CLUSTERS, EVENT1_TRACKS, EVENT1_PARTICLES)])
    # event 1 adds one reconstructible particle, matched, and one good track
    assert both == dict(reconstructible=7, efficiency=5 / 7, tracks=10, ghost_rate=3 / 10, clone_rate=1 / 6)


def test_evaluate_batch_on_hand_counted_events():
    """The batch form: events sliced by offsets, modules from the cluster z."""
    z = np.array([-300.0 + 42.0 * k for k in range(26)], np.float32)
    words, truth, labels, coff, cz, toff, hoff, hits, poff = [], [], [], [0], [], [0], [0], [], [0]
    for clusters, tracks, n_part in ((EVENT0_CLUSTERS, EVENT0_TRACKS, EVENT0_PARTICLES),
                                     (EVENT1_CLUSTERS, EVENT1_TRACKS, EVENT1_PARTICLES)):
        w, t, lab, mods = build_event(clusters)
        words.append(w)
        truth.append(t)
        labels.append(lab)
        coff.append(coff[-1] + len(clusters))
        cz.append(z[mods])
        for tr in tracks:
            hits.extend(tr)
            hoff.append(len(hits))
        toff.append(toff[-1] + len(tracks))
        poff.append(poff[-1] + n_part)
    pix_off = np.r_[0, np.cumsum([len(w) for w in words])].astype(np.uint64)
    batch = SimpleNamespace(n_events=2, offsets=pix_off, pixels=np.concatenate(words),
                            pixel_truth=np.concatenate(truth), particle_offsets=np.array(poff, np.uint64),
                            geometry=SimpleNamespace(module_z=z))
    result = dict(cluster_offsets=np.array(coff, np.uint64), cluster_z=np.concatenate(cz),
                  track_offsets=np.array(toff, np.uint64), track_hit_offsets=np.array(hoff, np.uint64),
                  track_hits=np.array(hits, np.uint32), pixel_cluster=np.concatenate(labels))
    assert mc.evaluate_batch(batch, result) == dict(reconstructible=7, efficiency=5 / 7, tracks=10,
                                                    ghost_rate=3 / 10, clone_rate=1 / 6)
