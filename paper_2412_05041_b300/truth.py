"""Monte-Carlo truth matching of reconstructed tracks (numpy; labels and metrics).

Used to label candidates for training the ghost-rejection network and to
report efficiency and ghost rate.  Definitions:
  cluster truth  the particle (or noise, -1) with the largest summed charge
                 over the cluster's pixels; ties go to the smaller id;
  matched track  >= 70 % of its hits carry one particle's truth;
  reconstructible particle  >= 3 clusters on distinct modules;
  efficiency     reconstructible particles matched by >= 1 track / reconstructible;
  ghost rate     unmatched tracks / tracks.
Particle ids are made batch-global (particle_offsets[e] + local id).
"""
from __future__ import annotations

import numpy as np


def cluster_truth(batch, result) -> np.ndarray:
    """Batch-global particle id (or -1) of every cluster of `result` (numpy dict with
    cluster_offsets, pixel_cluster)."""
    E = batch.n_events
    off = batch.offsets.astype(np.int64)
    coff = np.asarray(result["cluster_offsets"], np.int64)
    n_cl = int(coff[-1])
    ev = np.repeat(np.arange(E), np.diff(off))
    lab = np.asarray(result["pixel_cluster"]).astype(np.int64)
    ok = lab >= 0
    ok &= lab != 0xFFFFFFFF
    cl = coff[ev] + lab
    pt = batch.pixel_truth.astype(np.int64)
    gp = np.where(pt >= 0, batch.particle_offsets.astype(np.int64)[ev] + pt, -1)
    q = ((batch.pixels >> 27) & 15).astype(np.int64)
    cl, gp, q = cl[ok], gp[ok], q[ok]
    order = np.lexsort((gp, cl))
    cl, gp, q = cl[order], gp[order], q[order]
    brk = np.r_[True, (cl[1:] != cl[:-1]) | (gp[1:] != gp[:-1])]
    gi = np.cumsum(brk) - 1
    qs = np.bincount(gi, weights=q)
    gcl, ggp = cl[brk], gp[brk]
    # per cluster: the largest charge sum, ties to the smaller particle id (groups sorted by id)
    order2 = np.lexsort((ggp, -qs, gcl))
    first = np.r_[True, gcl[order2][1:] != gcl[order2][:-1]]
    truth = np.full(n_cl, -1, np.int64)
    truth[gcl[order2][first]] = ggp[order2][first]
    return truth


def track_matches(result, ctruth: np.ndarray, min_frac: float = 0.7) -> np.ndarray:
    """Batch-global matched particle id of every track (-1 = ghost)."""
    toff = np.asarray(result["track_offsets"], np.int64)
    hoff = np.asarray(result["track_hit_offsets"], np.int64)
    coff = np.asarray(result["cluster_offsets"], np.int64)
    nt = int(toff[-1])
    if nt == 0:
        return np.zeros(0, np.int64)
    ev_of_track = np.repeat(np.arange(len(toff) - 1), np.diff(toff))
    nh = np.diff(hoff[: nt + 1])
    trk = np.repeat(np.arange(nt), nh)
    hits = np.asarray(result["track_hits"]).astype(np.int64)[: int(hoff[nt])]
    p = ctruth[coff[ev_of_track][trk] + hits]
    keep = p >= 0
    trk, p = trk[keep], p[keep]
    order = np.lexsort((p, trk))
    trk, p = trk[order], p[order]
    brk = np.r_[True, (trk[1:] != trk[:-1]) | (p[1:] != p[:-1])] if len(trk) else np.zeros(0, bool)
    gi = np.cumsum(brk) - 1
    cnt = np.bincount(gi) if len(gi) else np.zeros(0, np.int64)
    gt, gpart = trk[brk], p[brk]
    o2 = np.lexsort((gpart, -cnt, gt))
    first = np.r_[True, gt[o2][1:] != gt[o2][:-1]] if len(gt) else np.zeros(0, bool)
    best_t, best_p, best_c = gt[o2][first], gpart[o2][first], cnt[o2][first]
    match = np.full(nt, -1, np.int64)
    good = best_c >= min_frac * nh[best_t]
    match[best_t[good]] = best_p[good]
    return match


def reconstructible(batch, result, ctruth: np.ndarray) -> np.ndarray:
    """Batch-global ids of particles with >= 3 clusters on distinct modules."""
    z_to_m = {float(np.float32(z)): i for i, z in enumerate(batch.geometry.module_z)}
    cz = np.asarray(result["cluster_z"], np.float32)
    mods = np.array([z_to_m[float(z)] for z in np.unique(cz)], np.int64)
    zvals = np.unique(cz)
    cm = mods[np.searchsorted(zvals, cz)] if len(cz) else np.zeros(0, np.int64)
    sel = ctruth >= 0
    pairs = np.unique(np.stack([ctruth[sel], cm[sel]], 1), axis=0) if sel.any() else np.zeros((0, 2), np.int64)
    pid, n_mod = np.unique(pairs[:, 0], return_counts=True)
    return pid[n_mod >= 3]


def metrics(batch, result) -> dict:
    ct = cluster_truth(batch, result)
    m = track_matches(result, ct)
    rec = reconstructible(batch, result, ct)
    found = np.intersect1d(rec, m[m >= 0])
    uniq, cnt = np.unique(m[m >= 0], return_counts=True)
    return dict(efficiency=len(found) / max(len(rec), 1), ghost_rate=float((m < 0).mean()) if len(m) else 0.0,
                clone_rate=float((cnt - 1).sum()) / max(len(uniq), 1), tracks=int(len(m)), reconstructible=int(len(rec)))
