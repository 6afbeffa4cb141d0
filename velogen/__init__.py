"""Seeded synthetic VELO-like events (input data only; no reconstruction arithmetic).

Both the CPU oracle and the CUDA path read what this module writes, and this
module imports neither.  The generator itself is C++ (``velogen.cpp``), built
into ``libvelogen.so`` beside this file and called through ctypes.

The standard geometry and the workload presets follow the synthetic stand-in
for the paper's workload (pp collisions at pile-up mu ~ 5 seen by a pixel
tracker around the interaction region, Sec. "Introduction" and Sec. "Detector"):

* ``C1``  100 events, 1 PV, 40 straight tracks, no noise, no scattering.
* ``C2``  10k events, n_PV ~ Poisson(5.5), tracks/PV ~ Poisson(40),
          0.5 mrad kicks per module, 99 % hit efficiency, 1e-4 noise.
* ``C3``  as C2 with 10 % of events at n_PV ~ Poisson(15).
* ``C5``  as C2 with 5 % heavy-ion-like events (1 PV, U{2000..10000} tracks).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "velogen.cpp")
_LIB = os.path.join(_HERE, "libvelogen.so")

N_MODULES = 26
# pv, x0, y0, z0, tx, ty, eta, phi, n_modules_with_pixels, heavy_ion, then the line the
# particle leaves the pixel tracker on: x, y, z, tx, ty (after the last kink)
PARTICLE_FIELDS = 15


def module_z() -> np.ndarray:
    """z of the 26 planar modules: uniformly spaced from -300 to +750 mm (42 mm apart)."""
    return (-300.0 + 42.0 * np.arange(N_MODULES)).astype(np.float64)


@dataclass(frozen=True)
class Geometry:
    """Planar pixel modules; all lengths in mm.  1528 x 1528 cells of 55 um, centred on the beam."""
    n_modules: int = N_MODULES
    module_z: tuple = tuple(module_z().tolist())
    pitch: float = 0.055
    n_rows: int = 1528
    n_cols: int = 1528
    x0: float = -1528 * 0.055 / 2
    y0: float = -1528 * 0.055 / 2
    r_min: float = 5.1
    r_max: float = 42.0


@dataclass(frozen=True)
class Config:
    seed: int = 2
    n_events: int = 10_000
    fixed_pvs: int = 0
    fixed_tracks: int = 0
    pv_mu: float = 5.5
    heavy_frac: float = 0.0
    pv_mu_heavy: float = 15.0
    hi_frac: float = 0.0
    hi_min_tracks: int = 2000
    hi_max_tracks: int = 10000
    tracks_mu: float = 40.0
    eta_min: float = 2.0
    eta_max: float = 5.0
    pv_sigma_xy: float = 0.05
    pv_sigma_z: float = 45.0
    ms_theta: float = 5e-4
    hit_eff: float = 0.99
    noise_prob: float = 1e-4
    shuffle: int = 1


C1 = Config(seed=1, n_events=100, fixed_pvs=1, fixed_tracks=40, ms_theta=0.0, hit_eff=1.0, noise_prob=0.0)
C2 = Config(seed=2, n_events=10_000)
C3 = Config(seed=3, n_events=100_000, heavy_frac=0.10, pv_mu_heavy=15.0)
C5 = Config(seed=6, n_events=10_000, hi_frac=0.05)
PRESETS = {"C1": C1, "C2": C2, "C3": C3, "C5": C5}


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("fixed_pvs", ctypes.c_int32),
        ("fixed_tracks", ctypes.c_int32),
        ("pv_mu", ctypes.c_double),
        ("heavy_frac", ctypes.c_double),
        ("pv_mu_heavy", ctypes.c_double),
        ("hi_frac", ctypes.c_double),
        ("hi_min_tracks", ctypes.c_int32),
        ("hi_max_tracks", ctypes.c_int32),
        ("tracks_mu", ctypes.c_double),
        ("eta_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("pv_sigma_xy", ctypes.c_double),
        ("pv_sigma_z", ctypes.c_double),
        ("ms_theta", ctypes.c_double),
        ("hit_eff", ctypes.c_double),
        ("noise_prob", ctypes.c_double),
        ("shuffle", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
    ]


class _Geo(ctypes.Structure):
    _fields_ = [
        ("n_modules", ctypes.c_int32),
        ("n_rows", ctypes.c_int32),
        ("n_cols", ctypes.c_int32),
        ("module_z", ctypes.c_double * 32),
        ("pitch", ctypes.c_double),
        ("x0", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("r_min", ctypes.c_double),
        ("r_max", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile libvelogen.so in place (g++, C++17)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.velogen_run.restype = ctypes.c_void_p
        lib.velogen_run.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Geo), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
        lib.velogen_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_uint64)] * 3
        lib.velogen_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5
        lib.velogen_free.argtypes = [ctypes.c_void_p]
        lib.velogen_n_sensitive.restype = ctypes.c_uint64
        lib.velogen_n_sensitive.argtypes = [ctypes.POINTER(_Geo)]
        _lib = lib
    return _lib


def _geo_struct(g: Geometry) -> _Geo:
    s = _Geo()
    s.n_modules, s.n_rows, s.n_cols = g.n_modules, g.n_rows, g.n_cols
    for i, z in enumerate(g.module_z):
        s.module_z[i] = z
    s.pitch, s.x0, s.y0, s.r_min, s.r_max = g.pitch, g.x0, g.y0, g.r_min, g.r_max
    return s


def n_sensitive(geometry: Geometry = Geometry()) -> int:
    g = _geo_struct(geometry)
    return int(_load().velogen_n_sensitive(ctypes.byref(g)))


@dataclass
class Batch:
    """A batch of events in CSR form (host numpy arrays)."""
    offsets: np.ndarray            # uint64 [n_events + 1]
    pixels: np.ndarray             # uint32 [n_pixels]
    pixel_truth: np.ndarray | None = None       # int32 [n_pixels], -1 = noise
    particle_offsets: np.ndarray | None = None  # uint64 [n_events + 1]
    particles: np.ndarray | None = None         # float64 [n_particles, PARTICLE_FIELDS]
    geometry: Geometry = field(default_factory=Geometry)
    first_event: int = 0                        # index of the batch's first event in its stream
    seed: int = 0                               # the configuration's seed

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1

    def event(self, e: int) -> np.ndarray:
        return self.pixels[int(self.offsets[e]):int(self.offsets[e + 1])]


def generate(cfg: Config, n_events: int | None = None, first_event: int = 0, truth: bool = False,
             geometry: Geometry = Geometry(), n_threads: int = 0, pixels_out: np.ndarray | None = None) -> Batch:
    """Generate ``n_events`` events (default ``cfg.n_events``) starting at ``first_event``.

    ``pixels_out`` may be a preallocated uint32 array (e.g. a view of pinned host memory)
    that is at least as large as the batch; the words are written into it.
    """
    lib = _load()
    n = cfg.n_events if n_events is None else int(n_events)
    c = _Cfg()
    for name, _ in _Cfg._fields_:
        if name == "n_threads":
            continue
        setattr(c, name, getattr(cfg, name))
    c.n_threads = n_threads
    g = _geo_struct(geometry)
    h = lib.velogen_run(ctypes.byref(c), ctypes.byref(g), first_event, n, 1 if truth else 0)
    if not h:
        raise RuntimeError("velogen_run failed")
    try:
        ne, npx, npart = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        lib.velogen_sizes(h, ctypes.byref(ne), ctypes.byref(npx), ctypes.byref(npart))
        offsets = np.zeros(n + 1, np.uint64)
        if pixels_out is not None:
            if pixels_out.dtype != np.uint32 or pixels_out.size < npx.value or not pixels_out.flags.c_contiguous:
                raise ValueError("pixels_out too small or not contiguous uint32")
            pixels = pixels_out[: npx.value]
        else:
            pixels = np.zeros(npx.value, np.uint32)
        ptruth = np.zeros(npx.value, np.int32) if truth else None
        poff = np.zeros(n + 1, np.uint64) if truth else None
        parts = np.zeros((npart.value, PARTICLE_FIELDS), np.float64) if truth else None

        def ptr(a):
            return None if a is None else a.ctypes.data

        rc = lib.velogen_copy(h, ptr(offsets), ptr(pixels), ptr(ptruth), ptr(poff), ptr(parts))
        if rc != 0:
            raise RuntimeError(f"velogen_copy failed ({rc})")
    finally:
        lib.velogen_free(h)
    return Batch(offsets, pixels, ptruth, poff, parts, geometry, int(first_event), int(cfg.seed))


def with_events(cfg: Config, n_events: int) -> Config:
    return replace(cfg, n_events=n_events)
