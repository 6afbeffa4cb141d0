"""Brute-force pins of the oracle's triplet seeding and track extension (CPU only).

The oracle runs the search module by module over hits sorted by (key, id).
Here the same definitions are evaluated by plain enumeration instead: every
ordered triplet of hits in a tiny event (and, for extension, every hit of the
target module for every track) is tested against the cuts, the best choice is
taken by the method's lexicographic tie rules, conflicts and contention are
settled by the smallest (distance, id) claim, and the resulting tracks must
equal the oracle's output exactly.

The events are random and dense in one narrow azimuth sector (some of them
across phi = 0, where the key wraps at 4), with hit positions smeared so that
the scatter cuts decide a good share of the candidates and seeds compete for
hits.  All arithmetic is binary32, one rounding per operation in the order the
method states (Sec. "HLT1 details and results" names the simplified pattern
recognition; the rules are the oracle's stated definition).  The chi2 cuts are
opened so that every track the search builds is reported.
"""
import itertools

import numpy as np

import oracle
import velogen

F = np.float32
GEO = velogen.Geometry()
Z = np.asarray(GEO.module_z, np.float32)
P = oracle.Params(ms_theta=0.0, chi2ndf_max=1e30, chi2ndf_max_3hit=1e30)


def key_of(x, y):
    """Diamond pseudo-angle in [0, 4), binary32, written from its definition."""
    x, y = F(x), F(y)
    if y >= 0:
        return y / (x + y) if x >= 0 else F(1) + (-x) / (y - x)
    return F(2) + (-y) / ((-x) - y) if x < 0 else F(3) + x / (x - y)


def dkey(a, b):
    """Distance of two keys on the circle of circumference 4."""
    d = abs(F(a) - F(b))
    return min(d, F(4) - d)


def tiny_event(rng, mods, n_lines, n_noise, sigma, twin_frac=0.0):
    """Hits on the modules `mods`, grouped by module in ascending order (the
    cluster-id order), shuffled inside each module.  Lines come from points
    near the beam axis; a share `twin_frac` of them gets a twin about 0.1 mm
    away (so that tracks compete for hits); noise hits fill the same azimuth
    sector."""
    phi0 = rng.choice([rng.uniform(0, 2 * np.pi), -0.06])  # some sectors straddle phi = 0
    dphi = 0.12
    zc = float(Z[mods[len(mods) // 2]])
    hits = {m: [] for m in mods}
    lines = []
    for _ in range(n_lines):
        phi, r_ref = phi0 + rng.uniform(0, dphi), rng.uniform(8.0, 30.0)
        lever = rng.uniform(200.0, 600.0)  # distance of the origin upstream of the middle module
        lines.append((phi, r_ref, lever))
        if rng.random() < twin_frac:
            lines.append((phi + rng.uniform(-0.1, 0.1) / r_ref, r_ref + rng.uniform(-0.1, 0.1), lever))
    for phi, r_ref, lever in lines:
        tr = r_ref / lever
        for m in mods:
            if rng.random() < 0.1:
                continue
            r = r_ref + tr * (float(Z[m]) - zc)
            hits[m].append((r * np.cos(phi) + rng.normal(0, sigma), r * np.sin(phi) + rng.normal(0, sigma)))
    for _ in range(n_noise):
        m = int(rng.choice(mods))
        phi, r = phi0 + rng.uniform(0, dphi), rng.uniform(6.0, 35.0)
        hits[m].append((r * np.cos(phi), r * np.sin(phi)))
    module, x, y = [], [], []
    for m in sorted(mods):
        for i in rng.permutation(len(hits[m])):
            module.append(m)
            x.append(hits[m][i][0])
            y.append(hits[m][i][1])
    return np.array(module, np.uint32), np.array(x, np.float32), np.array(y, np.float32)


def brute_seeds(module, x, y, m, used):
    """Seeds with the middle hit on m: every (h0 on m+1, h1 on m, h2 on m-1)
    triplet of the event is tested; h1 and h0 must be unused.  Each h1 keeps
    its smallest (s, h0, h2); a seed claims h0 and h2 with (s, h1) and survives
    only if it holds both claims.  Survivors in the order of h1 by (key, id)."""
    n = len(module)
    key = [key_of(x[i], y[i]) for i in range(n)]
    z = Z[module]
    best = {}
    for h0, h1, h2 in itertools.product(range(n), repeat=3):
        if module[h0] != m + 1 or module[h1] != m or module[h2] != m - 1 or h0 in used or h1 in used:
            continue
        if dkey(key[h0], key[h1]) > F(P.win_seed) or dkey(key[h2], key[h1]) > F(P.win_seed):
            continue
        tx = (x[h0] - x[h2]) / (z[h0] - z[h2])
        ty = (y[h0] - y[h2]) / (z[h0] - z[h2])
        if abs(tx) > F(P.max_slope) or abs(ty) > F(P.max_slope):
            continue
        xp = x[h2] + tx * (z[h1] - z[h2])
        yp = y[h2] + ty * (z[h1] - z[h2])
        ex, ey = xp - x[h1], yp - y[h1]
        s = ex * ex + ey * ey
        if s > F(P.max_scatter_seed):
            continue
        best[h1] = min(best.get(h1, (s, h0, h2)), (s, h0, h2))
    claims = {}
    for h1, (s, h0, h2) in best.items():
        for h in (h0, h2):
            claims[h] = min(claims.get(h, (s, h1)), (s, h1))
    keep = [h1 for h1, (s, h0, h2) in best.items() if claims[h0] == (s, h1) and claims[h2] == (s, h1)]
    keep.sort(key=lambda h1: (key[h1], h1))
    return [(best[h1][1], h1, best[h1][2]) for h1 in keep]


def canonical(tracks):
    return sorted(sorted(int(h) for h in t) for t in tracks)


def oracle_tracks(module, x, y):
    tracks, _ = oracle.track_event(module, x, y, GEO, P)
    return [list(map(int, t)) for t in tracks]


def test_triplet_seeds_equal_enumeration_of_all_triplets():
    """Hits on three modules only: the oracle's tracks are exactly the seeds
    that the enumeration of all triplets leaves after conflicts."""
    rng = np.random.default_rng(20241205)
    n_seeds = n_dropped = 0
    for _ in range(150):
        m = int(rng.integers(3, 23))
        module, x, y = tiny_event(rng, [m - 1, m, m + 1], int(rng.integers(2, 7)), int(rng.integers(0, 5)),
                                  sigma=0.04)
        seeds = brute_seeds(module, x, y, m, used=set())
        assert oracle_tracks(module, x, y) == canonical(seeds)
        n_seeds += len(seeds)
        n_dropped += sum(1 for h1 in range(len(module)) if module[h1] == m) - len(seeds)
    # the cases are not trivial: many seeds, and many middle hits without one
    assert n_seeds > 300 and n_dropped > 100


def test_extension_equals_enumeration_over_the_target_module():
    """Hits on four modules m+1 .. m-2.  Step m seeds; step m-1 seeds from the
    hits left on m and m-1 with h2 on m-2; step m-2 extends the step-m tracks
    along the line through their last two hits: each track takes the unused
    hit of m-2 with the smallest (d^2, id) inside the key window and the
    distance cut, and a hit wanted by several tracks goes to the smallest
    (d^2, track index).  Tracks are indexed in creation order."""
    rng = np.random.default_rng(77)
    n_ext = n_contended = 0
    for _ in range(150):
        m = int(rng.integers(4, 24))
        module, x, y = tiny_event(rng, [m - 2, m - 1, m, m + 1], int(rng.integers(2, 7)), int(rng.integers(0, 5)),
                                  sigma=0.035, twin_frac=0.5)
        n = len(module)
        used = set()
        tracks = [list(s) for s in brute_seeds(module, x, y, m, used)]
        for t in tracks:
            used.update(t)
        n_first = len(tracks)
        later = [list(s) for s in brute_seeds(module, x, y, m - 1, used)]
        for t in later:
            used.update(t)
        tracks += later
        z = Z[module]
        zt = Z[m - 2]
        want = {}
        for t in range(n_first):
            a, b = tracks[t][-1], tracks[t][-2]  # the last hit (module m-1) and the one before
            tx = (x[a] - x[b]) / (z[a] - z[b])
            ty = (y[a] - y[b]) / (z[a] - z[b])
            xp = x[a] + tx * (zt - z[a])
            yp = y[a] + ty * (zt - z[a])
            cands = []
            for h in range(n):
                if module[h] != m - 2 or h in used or dkey(key_of(x[h], y[h]), key_of(x[a], y[a])) > F(P.win_fwd):
                    continue
                ex, ey = xp - x[h], yp - y[h]
                d2 = ex * ex + ey * ey
                if d2 <= F(P.max_scatter_fwd):
                    cands.append((d2, h))
            if cands:
                want[t] = min(cands)
        owner = {}
        for t, (d2, h) in want.items():
            owner[h] = min(owner.get(h, (d2, t)), (d2, t))
        for h, (d2, t) in owner.items():
            tracks[t].append(h)
        n_ext += len(owner)
        n_contended += len(want) - len(owner)
        assert oracle_tracks(module, x, y) == canonical(tracks)
    assert n_ext > 150 and n_contended > 5
