"""Monte-Carlo truth matching -- TEST INFRASTRUCTURE (metrics, not the hot path).

Definitions (this project's reading; the paper quotes no tracking-efficiency
figure for the first trigger stage, Sec. "HLT1 details and results"):

* pixel truth: the particle with the largest deposit on the pixel (noise = -1),
  written by the generator;
* cluster truth: the particle (or -1) with the largest summed charge over the
  cluster's pixels, ties to the smaller id -- noise counts as id -1, so a tie
  between noise and a particle leaves the cluster as noise;
* reconstructible particle: >= 3 clusters with its truth, on distinct modules;
* a track matches particle P if >= 70 % of its hits carry truth P (P >= 0);
* efficiency = reconstructible particles matched by >= 1 track / reconstructible;
* ghost rate = tracks matching no particle / tracks;
* clone rate = (matching tracks beyond the first of each particle) / matched particles.

Pinned by hand-counted events in tests/test_oracle_mc.py (every rule above
changes a hand-counted figure when misread).
"""
from __future__ import annotations

import numpy as np


def cluster_truth(words: np.ndarray, pixel_truth: np.ndarray, pixel_cluster: np.ndarray, n_clusters: int) -> np.ndarray:
    q = ((words >> 27) & 15).astype(np.int64)
    best = np.full(n_clusters, -2, np.int64)
    if n_clusters == 0:
        return best
    # sum q per (cluster, particle)
    key_c = pixel_cluster.astype(np.int64)
    key_p = pixel_truth.astype(np.int64)
    order = np.lexsort((key_p, key_c))
    c_s, p_s, q_s = key_c[order], key_p[order], q[order]
    brk = np.r_[True, (c_s[1:] != c_s[:-1]) | (p_s[1:] != p_s[:-1])]
    grp = np.cumsum(brk) - 1
    qsum = np.bincount(grp, weights=q_s).astype(np.int64)
    gc, gp = c_s[brk], p_s[brk]
    # per cluster: largest qsum, ties -> smaller particle id (groups are sorted by particle)
    bestq = np.full(n_clusters, -1, np.int64)
    for c, p, s in zip(gc, gp, qsum):
        if s > bestq[c]:
            bestq[c] = s
            best[c] = p
    return best


def match_event(words, pixel_truth, pixel_cluster, n_clusters, cluster_module, tracks, n_particles,
                min_frac: float = 0.7):
    """Returns dict(reconstructible[bool n_particles], matched_particle[per track, -1 = ghost])."""
    ct = cluster_truth(words, pixel_truth, pixel_cluster, n_clusters)
    recon = np.zeros(n_particles, bool)
    for p in range(n_particles):
        mods = np.unique(cluster_module[ct == p])
        recon[p] = len(mods) >= 3
    matched = np.full(len(tracks), -1, np.int64)
    for i, hits in enumerate(tracks):
        t = ct[np.asarray(hits, np.int64)]
        vals, cnt = np.unique(t[t >= 0], return_counts=True)
        if len(vals):
            j = int(np.argmax(cnt))
            if cnt[j] >= min_frac * len(hits):
                matched[i] = vals[j]
    return dict(reconstructible=recon, matched=matched, cluster_truth=ct)


def summarize(per_event) -> dict:
    n_rec = n_eff = n_tracks = n_ghost = n_clone = n_matched_p = 0
    for ev in per_event:
        rec = ev["reconstructible"]
        m = ev["matched"]
        n_tracks += len(m)
        n_ghost += int((m < 0).sum())
        good = m[m >= 0]
        uniq, cnt = np.unique(good, return_counts=True)
        n_matched_p += len(uniq)
        n_clone += int((cnt - 1).sum())
        n_rec += int(rec.sum())
        n_eff += int(rec[uniq].sum()) if len(uniq) else 0
    return dict(
        reconstructible=n_rec,
        efficiency=n_eff / max(n_rec, 1),
        tracks=n_tracks,
        ghost_rate=n_ghost / max(n_tracks, 1),
        clone_rate=n_clone / max(n_matched_p, 1),
    )


def evaluate_batch(batch, result, module_of_cluster=None) -> dict:
    """MC metrics of a reconstructed batch (numpy result dict in the library's layout)."""
    per = []
    z_to_mod = {float(np.float32(z)): i for i, z in enumerate(batch.geometry.module_z)}
    for e in range(batch.n_events):
        p0, p1 = int(batch.offsets[e]), int(batch.offsets[e + 1])
        c0, c1 = int(result["cluster_offsets"][e]), int(result["cluster_offsets"][e + 1])
        t0, t1 = int(result["track_offsets"][e]), int(result["track_offsets"][e + 1])
        cz = result["cluster_z"][c0:c1]
        cmod = np.array([z_to_mod[float(z)] for z in cz], np.int64)
        tracks = []
        for t in range(t0, t1):
            h0, h1 = int(result["track_hit_offsets"][t]), int(result["track_hit_offsets"][t + 1])
            tracks.append(result["track_hits"][h0:h1])
        q0, q1 = int(batch.particle_offsets[e]), int(batch.particle_offsets[e + 1])
        per.append(match_event(batch.pixels[p0:p1], batch.pixel_truth[p0:p1], result["pixel_cluster"][p0:p1],
                               c1 - c0, cmod, tracks, q1 - q0))
    return summarize(per)
