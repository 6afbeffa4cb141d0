"""Pins of the oracle's clustering (pixel words -> clusters), CPU only.

The oracle's clustering (8-connected components per module, ids by the
smallest (module, row, col) of each component, centroid from integer charge
sums) is checked against things that do not share its code:

* an independent breadth-first flood fill on a dense grid (every 3x3 pattern,
  random 8x8 tiles, tiles on the grid edges, duplicate words);
* the exact rational centroid of small deposits (Fractions);
* invariance under any permutation of the words of an event;
* the validation and capacity rules (bad words, too many clusters on a module).
"""
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

import oracle


def word(q, m, r, c):
    return np.uint32((q << 27) | (m << 22) | (r << 11) | c)


def bfs_clusters(pix):
    """Independent 8-connected labelling on a dense dict grid.

    pix: list of (q, m, r, c).  Returns (labels per word, clusters ordered by
    (module, smallest row*2048+col)) where each cluster is the list of word indices."""
    cells = {}
    for i, (_, m, r, c) in enumerate(pix):
        cells.setdefault((m, r, c), []).append(i)
    seen = set()
    comps = []
    for start in sorted(cells):
        if start in seen:
            continue
        comp = []
        dq = deque([start])
        seen.add(start)
        while dq:
            m, r, c = dq.popleft()
            comp.extend(cells[(m, r, c)])
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    nb = (m, r + dr, c + dc)
                    if nb in cells and nb not in seen:
                        seen.add(nb)
                        dq.append(nb)
        comps.append(comp)
    comps.sort(key=lambda comp: min((pix[i][1], pix[i][2] * 2048 + pix[i][3]) for i in comp))
    labels = np.zeros(len(pix), np.int64)
    for cid, comp in enumerate(comps):
        for i in comp:
            labels[i] = cid
    return labels, comps


def exact_centroid(pix, comp, geometry):
    qs = sum(pix[i][0] for i in comp)
    u = Fraction(sum(pix[i][0] * (2 * pix[i][3] + 1) for i in comp), 2 * qs)
    v = Fraction(sum(pix[i][0] * (2 * pix[i][2] + 1) for i in comp), 2 * qs)
    p = float(np.float32(geometry.pitch))
    x0 = float(np.float32(geometry.x0))
    y0 = float(np.float32(geometry.y0))
    return x0 + p * float(u), y0 + p * float(v)


def check_against_bfs(pix, geometry, rng=None):
    words = np.array([word(*t) for t in pix], np.uint32)
    out = oracle.cluster_event(words, geometry)
    assert out["status"] == oracle.EVT_OK
    labels, comps = bfs_clusters(pix)
    assert len(out["x"]) == len(comps)
    np.testing.assert_array_equal(out["pixel_cluster"].astype(np.int64), labels)
    for cid, comp in enumerate(comps):
        ex, ey = exact_centroid(pix, comp, geometry)
        # binary32 result of a correctly computed centroid: within a few ulp at |x| <= 42 mm
        assert abs(float(out["x"][cid]) - ex) <= 2e-5, (cid, out["x"][cid], ex)
        assert abs(float(out["y"][cid]) - ey) <= 2e-5, (cid, out["y"][cid], ey)
        m = pix[comp[0]][1]
        assert out["module"][cid] == m
        assert out["z"][cid] == np.float32(geometry.module_z[m])
    return out


def test_all_3x3_patterns(geometry):
    rng = np.random.default_rng(11)
    for pattern in range(1, 512):
        pix = []
        for b in range(9):
            if pattern >> b & 1:
                r, c = 700 + b // 3, 900 + b % 3
                pix.append((int(rng.integers(1, 16)), 5, r, c))
        # a second, isolated pixel on another module and one far away on the same module
        pix.append((7, 6, 700, 900))
        pix.append((3, 5, 710, 900))
        check_against_bfs(pix, geometry)


@pytest.mark.parametrize("density", [0.2, 0.45, 0.7])
def test_random_tiles(geometry, density):
    rng = np.random.default_rng(int(density * 100))
    for trial in range(40):
        pix = []
        for m in rng.choice(26, size=3, replace=False):
            # place one tile in the interior and one on a grid edge
            for (r0, c0) in [(int(rng.integers(10, 1500)), int(rng.integers(10, 1500))),
                             (0 if trial % 2 else 1520, 0 if trial % 3 else 1520)]:
                mask = rng.random((8, 8)) < density
                for r, c in zip(*np.nonzero(mask)):
                    pix.append((int(rng.integers(1, 16)), int(m), r0 + int(r), c0 + int(c)))
        check_against_bfs(pix, geometry)


def test_duplicate_words_join_their_cluster(geometry):
    pix = [(3, 2, 100, 100), (5, 2, 100, 100), (4, 2, 101, 101), (9, 2, 300, 300), (9, 2, 300, 300)]
    out = check_against_bfs(pix, geometry)
    assert len(out["x"]) == 2


def test_isolated_pixel_centre(geometry):
    """A single pixel's centroid is its centre: u = col + 1/2 exactly."""
    for (r, c) in [(0, 0), (1527, 1527), (764, 3), (12, 1500)]:
        out = oracle.cluster_event(np.array([word(9, 0, r, c)]), geometry)
        assert out["x"][0] == np.float32(np.float32(geometry.x0) + np.float32(geometry.pitch) * np.float32(c + 0.5))
        ex, ey = exact_centroid([(9, 0, r, c)], [0], geometry)
        assert abs(out["x"][0] - ex) <= 1e-5 and abs(out["y"][0] - ey) <= 1e-5


def test_2x2_bilinear_deposit_recovers_point(geometry):
    """A 2x2 deposit with bilinear weights has its centroid near the deposited point
    (exactly at it without charge quantisation)."""
    rng = np.random.default_rng(5)
    p = geometry.pitch
    for _ in range(200):
        c0, r0 = int(rng.integers(100, 1400)), int(rng.integers(100, 1400))
        fu, fv = rng.random(), rng.random()
        w = [(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv]
        cells = [(r0, c0), (r0, c0 + 1), (r0 + 1, c0), (r0 + 1, c0 + 1)]
        pix = [(int(np.rint(15 * wi)), 1, r, c) for wi, (r, c) in zip(w, cells) if np.rint(15 * wi) > 0]
        out = check_against_bfs(pix, geometry)
        xt = geometry.x0 + p * (c0 + 0.5 + fu)
        yt = geometry.y0 + p * (r0 + 0.5 + fv)
        # 4-bit charges: the centroid error stays well inside one pixel
        assert abs(out["x"][0] - xt) < 0.25 * p and abs(out["y"][0] - yt) < 0.25 * p


def test_permutation_invariance(geometry):
    import velogen
    b = velogen.generate(velogen.C2, n_events=3)
    rng = np.random.default_rng(3)
    for e in range(b.n_events):
        w = b.event(e)
        a = oracle.cluster_event(w, geometry)
        perm = rng.permutation(len(w))
        c = oracle.cluster_event(w[perm], geometry)
        np.testing.assert_array_equal(a["x"], c["x"])
        np.testing.assert_array_equal(a["y"], c["y"])
        np.testing.assert_array_equal(a["pixel_cluster"][perm], c["pixel_cluster"])


@pytest.mark.parametrize("bad", [
    word(0, 1, 10, 10),                      # q = 0
    word(3, 26, 10, 10),                     # module beyond the geometry
    word(3, 1, 1528, 10),                    # row beyond the grid
    word(3, 1, 10, 1528),                    # col beyond the grid
    np.uint32(0x80000000 | int(word(3, 1, 10, 10))),  # bit 31 set
])
def test_bad_word_fails_event(geometry, bad):
    words = np.array([word(3, 1, 10, 10), bad, word(3, 2, 10, 10)], np.uint32)
    out = oracle.cluster_event(words, geometry)
    assert out["status"] == oracle.EVT_BADWORD
    assert len(out["x"]) == 0
    assert (out["pixel_cluster"] == 0xFFFFFFFF).all()


def test_empty_event(geometry):
    out = oracle.cluster_event(np.zeros(0, np.uint32), geometry)
    assert out["status"] == oracle.EVT_OK and len(out["x"]) == 0


@pytest.mark.parametrize("n,expect", [(oracle.MAX_MODULE_CLUSTERS, oracle.EVT_OK),
                                      (oracle.MAX_MODULE_CLUSTERS + 1, oracle.EVT_OVERFLOW)])
def test_module_cluster_capacity(geometry, n, expect):
    idx = np.arange(n)
    r, c = 2 * (idx // 764), 2 * (idx % 764)
    words = ((5 << 27) | (3 << 22) | (r << 11) | c).astype(np.uint32)
    out = oracle.cluster_event(words, geometry)
    assert out["status"] == expect
    assert len(out["x"]) == (n if expect == oracle.EVT_OK else 0)
