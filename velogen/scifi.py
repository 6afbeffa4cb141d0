"""Seeded synthetic hits of a downstream tracker behind a dipole magnet
(input data only: none of the reconstruction arithmetic lives here).

The paper's first stage traces pixel-tracker tracks forwards to the next
tracker, straight up to the middle of the magnet, where the field is taken as
one change of angle, and straight again to the scintillating-fibre tracker
(Sec. "HLT1 details and results"); it gives no geometry.  This module invents
one, documented here and used only as a synthetic workload:

* a kick plane at z = z_mag: a particle of momentum p [GeV/c] and charge q
  leaves it with tx + kappa q / p (kappa [GeV/c rad] stands for the field
  integral), ty unchanged; straight lines on both sides;
* twelve planar layers in three stations of four (z_layers), each measuring a
  crossing as (x, y) with Gaussian resolutions sigma_x (fibres across x) and
  sigma_y (from the stereo views), inside |x| <= half_x, |y| <= half_y, with
  efficiency hit_eff; noise_per_layer uniform hits per layer and event.

Particles start from the line the pixel-tracker generator records for each
of them as it leaves the last module (no scattering downstream); p = pT
cosh(eta) with pT ~ pt_min + Exp(pt_mean), q = +-1 with equal odds.  Every
event draws from its own stream seeded by (seed, event index), independent of
the pixel-tracker generator's streams, and the hits of an event are shuffled;
a hit's id is its index in its event.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

N_LAYERS = 12


@dataclass(frozen=True)
class Downstream:
    z_mag: float = 5250.0
    z_layers: tuple = (7826.0, 7896.0, 7966.0, 8036.0, 8508.0, 8578.0, 8648.0, 8718.0,
                       9193.0, 9263.0, 9333.0, 9403.0)
    kappa: float = 1.2
    half_x: float = 3000.0
    half_y: float = 2500.0
    sigma_x: float = 0.08
    sigma_y: float = 1.0
    hit_eff: float = 0.98
    noise_per_layer: int = 20
    pt_min: float = 0.2
    pt_mean: float = 0.6


@dataclass
class ScifiBatch:
    offsets: np.ndarray          # uint64 [E + 1]
    layer: np.ndarray            # uint32 [H]
    x: np.ndarray                # float32 [H] mm
    y: np.ndarray                # float32 [H] mm
    truth: np.ndarray            # int32 [H]: particle index in its event, -1 = noise
    p: np.ndarray                # float64 [n_particles] GeV/c (batch-global particle order)
    q: np.ndarray                # int32 [n_particles]
    geometry: Downstream = field(default_factory=Downstream)

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1


def generate(batch, geometry: Downstream = Downstream()) -> ScifiBatch:
    """Downstream hits of the particles of a generator batch made with truth=True
    (streams seeded by the batch's configuration seed and event indices)."""
    if batch.particles is None:
        raise ValueError("the pixel-tracker batch must carry its particles (truth=True)")
    E = batch.n_events
    g = geometry
    zl = np.asarray(g.z_layers, np.float64)
    po = batch.particle_offsets.astype(np.int64)
    P = batch.particles
    p_all = np.zeros(len(P), np.float64)
    q_all = np.zeros(len(P), np.int32)
    layers, xs, ys, truths, counts = [], [], [], [], np.zeros(E, np.int64)
    for e in range(E):
        rng = np.random.default_rng([int(batch.seed), int(batch.first_event) + e, 0x5C1F1])
        part = P[po[e]:po[e + 1]]
        n = len(part)
        pt = g.pt_min + rng.exponential(g.pt_mean, n)
        p = pt * np.cosh(part[:, 6])
        q = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int32)
        p_all[po[e]:po[e + 1]] = p
        q_all[po[e]:po[e + 1]] = q
        x, y, z, tx, ty = part[:, 10], part[:, 11], part[:, 12], part[:, 13], part[:, 14]
        xm = x + tx * (g.z_mag - z)
        ym = y + ty * (g.z_mag - z)
        tx2 = tx + g.kappa * q / p
        dz = zl[None, :] - g.z_mag
        hx = xm[:, None] + tx2[:, None] * dz + rng.normal(0.0, g.sigma_x, (n, N_LAYERS))
        hy = ym[:, None] + ty[:, None] * dz + rng.normal(0.0, g.sigma_y, (n, N_LAYERS))
        keep = (rng.random((n, N_LAYERS)) < g.hit_eff) & (np.abs(hx) <= g.half_x) & (np.abs(hy) <= g.half_y)
        pid, lay = np.nonzero(keep)
        nx = rng.uniform(-g.half_x, g.half_x, (N_LAYERS, g.noise_per_layer))
        ny = rng.uniform(-g.half_y, g.half_y, (N_LAYERS, g.noise_per_layer))
        lay_all = np.concatenate([lay, np.repeat(np.arange(N_LAYERS), g.noise_per_layer)])
        x_all = np.concatenate([hx[pid, lay], nx.ravel()])
        y_all = np.concatenate([hy[pid, lay], ny.ravel()])
        t_all = np.concatenate([pid, np.full(N_LAYERS * g.noise_per_layer, -1)])
        perm = rng.permutation(len(lay_all))
        layers.append(lay_all[perm])
        xs.append(x_all[perm])
        ys.append(y_all[perm])
        truths.append(t_all[perm])
        counts[e] = len(perm)
    offsets = np.zeros(E + 1, np.uint64)
    offsets[1:] = np.cumsum(counts)
    cat = (lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
    return ScifiBatch(offsets, cat(layers, np.uint32), cat(xs, np.float32), cat(ys, np.float32),
                      cat(truths, np.int32), p_all, q_all, g)
