"""CPU oracle for event-batched VELO-like tracking -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It defines the result the CUDA library
must reproduce (bit-exact cluster ids, cluster positions, track hit lists and
fit states, since both sides run the same binary32 operations in the same
order).  It shares no code with the CUDA library: its C++ source is
``velo_oracle.cpp`` (built into ``liboracle.so`` here, with
``-ffp-contract=off``), and this wrapper marshals numpy arrays only.

Pins (the checks that tie the oracle to something other than itself) live in
``tests/test_oracle_*.py``: clustering, fits, tracking (hand-built events and
brute-force enumeration), learned-rejection features and network, forward
tracking, and the Monte-Carlo truth matching of ``mc.py``; planted mistakes in
``tests/test_oracle_mutations.py`` check that the pins catch them.  Parity
unpinned: the absolute efficiency and ghost rate against the paper, which
prints none for this stage, and the tuned parameter values themselves.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import subprocess
from dataclasses import asdict, dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "velo_oracle.cpp")
_HDR = os.path.join(_HERE, "velo_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

STATE_STRIDE = 20
N_FEATURES = 12
MLP_HIDDEN = 32
MLP_FLOATS = 1529
FEATURE_NAMES = ("n_hits", "chi2ndf", "tx", "ty", "z_first", "z_last", "n_skipped", "mean_rx", "rms_rx", "mean_ry",
                 "rms_ry", "max_abs_r")
MAX_MODULE_CLUSTERS = 65535
EVT_OK, EVT_BADWORD, EVT_OVERFLOW = 0, 1, 2
STATE_FIELDS = ("x", "y", "tx", "ty", "z_first", "z_beam", "chi2_lsq", "chi2_kf", "kf_x", "kf_y", "kf_tx",
                "kf_ty", "kf_cxx", "kf_cxtx", "kf_ctxtx", "kf_cyy", "kf_cyty", "kf_ctyty", "ndf", "score")


@dataclass(frozen=True)
class Params:
    win_seed: float = 0.04
    win_fwd: float = 0.04
    max_slope: float = 0.3
    max_scatter_seed: float = 0.01
    max_scatter_fwd: float = 0.02
    max_skipped: int = 1
    sigma_meas: float = 0.0159
    ms_theta: float = 5e-4
    chi2ndf_max: float = 10.0
    chi2ndf_max_3hit: float = 2.0
    use_mlp: int = 0
    mlp_logit_min: float = 0.0


class _Geo(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_uint32), ("module_z", ctypes.POINTER(ctypes.c_float)),
                ("pitch_mm", ctypes.c_float), ("n_rows", ctypes.c_uint32), ("n_cols", ctypes.c_uint32),
                ("x0_mm", ctypes.c_float), ("y0_mm", ctypes.c_float)]


class _Par(ctypes.Structure):
    _fields_ = [("win_seed", ctypes.c_float), ("win_fwd", ctypes.c_float), ("max_slope", ctypes.c_float),
                ("max_scatter_seed", ctypes.c_float), ("max_scatter_fwd", ctypes.c_float),
                ("max_skipped", ctypes.c_uint32), ("sigma_meas", ctypes.c_float), ("ms_theta", ctypes.c_float),
                ("chi2ndf_max", ctypes.c_float), ("chi2ndf_max_3hit", ctypes.c_float),
                ("use_mlp", ctypes.c_uint32), ("mlp_logit_min", ctypes.c_float), ("mlp", ctypes.c_void_p)]


@dataclass(frozen=True)
class FwdParams:
    """Forward tracking (pixel-tracker tracks to the downstream layers)."""
    p_min: float = 3.0
    win_y: float = 40.0
    tol_x: float = 8.0
    tol_y: float = 40.0
    tol_x_far: float = 3.0
    sigma_x: float = 0.08
    tol_match: float = 25.0
    chi2ndf_max: float = 4.0
    min_hits: int = 9


FWD_LAYERS = 12
FWD_STATE = 6


class _Down(ctypes.Structure):
    _fields_ = [("z_mag", ctypes.c_float), ("z_layers", ctypes.c_float * FWD_LAYERS), ("kappa", ctypes.c_float)]


class _FwdPar(ctypes.Structure):
    _fields_ = [("p_min", ctypes.c_float), ("win_y", ctypes.c_float), ("tol_x", ctypes.c_float),
                ("tol_y", ctypes.c_float), ("tol_x_far", ctypes.c_float), ("sigma_x", ctypes.c_float),
                ("tol_match", ctypes.c_float), ("chi2ndf_max", ctypes.c_float), ("min_hits", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile liboracle.so in place: g++ -O2 -ffp-contract=off (no FMA contraction, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.vo_pseudo_angle.restype = ctypes.c_float
        lib.vo_pseudo_angle.argtypes = [ctypes.c_float, ctypes.c_float]
        lib.vo_cluster_event.restype = ctypes.c_int
        lib.vo_cluster_event.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(_Geo)] + [_P] * 6
        lib.vo_track_event.restype = ctypes.c_int
        lib.vo_track_event.argtypes = [ctypes.c_uint64, _P, _P, _P, ctypes.POINTER(_Geo), ctypes.POINTER(_Par),
                                       ctypes.c_uint64, _P, _P, _P, _P]
        lib.vo_fit_f32.argtypes = [ctypes.c_uint32, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P]
        lib.vo_fit_f64.argtypes = [ctypes.c_uint32, _P, _P, _P, ctypes.c_double, ctypes.c_double, _P]
        lib.vo_reconstruct.restype = ctypes.c_void_p
        lib.vo_reconstruct.argtypes = [ctypes.c_uint64, _P, _P, ctypes.POINTER(_Geo), ctypes.POINTER(_Par), ctypes.c_int]
        lib.vo_batch_sizes.argtypes = [ctypes.c_void_p, _P, _P, _P]
        lib.vo_batch_copy.argtypes = [ctypes.c_void_p] + [_P] * 11
        lib.vo_features.argtypes = [ctypes.c_uint32, _P, _P, _P, _P, _P, ctypes.c_float, _P]
        lib.vo_mlp_logit.restype = ctypes.c_float
        lib.vo_mlp_logit.argtypes = [_P, _P]
        lib.vo_batch_free.argtypes = [ctypes.c_void_p]
        lib.vo_forward_event.argtypes = [ctypes.c_uint64, _P, _P, _P, ctypes.c_uint64, _P, _P, _P, _P, _P,
                                         ctypes.POINTER(_Down), ctypes.POINTER(_FwdPar), _P, _P, _P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _GeoHolder:
    def __init__(self, geometry):
        self.z = np.ascontiguousarray(np.asarray(geometry.module_z, np.float32))
        self.s = _Geo(int(geometry.n_modules), self.z.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                      float(geometry.pitch), int(geometry.n_rows), int(geometry.n_cols), float(geometry.x0),
                      float(geometry.y0))


def _par(params: Params, mlp=None) -> _Par:
    p = _Par(**asdict(params))
    if params.use_mlp:
        if mlp is None or mlp.dtype != np.float32 or mlp.size != MLP_FLOATS or not mlp.flags.c_contiguous:
            raise ValueError("use_mlp needs a contiguous float32 model blob of MLP_FLOATS values")
        p.mlp = mlp.ctypes.data
    return p


def pseudo_angle(x: float, y: float) -> float:
    return float(_load().vo_pseudo_angle(x, y))


def cluster_event(words: np.ndarray, geometry):
    """Clusters of one event -> dict(status, x, y, z, module, pixel_cluster)."""
    lib = _load()
    w = np.ascontiguousarray(words, np.uint32)
    n = len(w)
    cx, cy, cz = (np.zeros(max(n, 1), np.float32) for _ in range(3))
    cm = np.zeros(max(n, 1), np.uint32)
    pc = np.zeros(max(n, 1), np.uint32)
    nc = ctypes.c_uint64()
    g = _GeoHolder(geometry)
    st = lib.vo_cluster_event(_ptr(w), n, ctypes.byref(g.s), _ptr(cx), _ptr(cy), _ptr(cz), _ptr(cm), _ptr(pc),
                              ctypes.byref(nc))
    k = nc.value
    return dict(status=st, x=cx[:k], y=cy[:k], z=cz[:k], module=cm[:k], pixel_cluster=pc[:n])


def track_event(module: np.ndarray, x: np.ndarray, y: np.ndarray, geometry, params: Params = Params(), mlp=None):
    """Tracks of one event from hits given in cluster-id order -> (list of hit-id arrays, states[T,20])."""
    lib = _load()
    module = np.ascontiguousarray(module, np.uint32)
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    n = len(module)
    cap = n // 3 + 1
    offs = np.zeros(cap + 1, np.uint64)
    ids = np.zeros(max(n, 1), np.uint32)
    st = np.zeros((cap, STATE_STRIDE), np.float32)
    nt = ctypes.c_uint64()
    g = _GeoHolder(geometry)
    p = _par(params, mlp)
    rc = lib.vo_track_event(n, _ptr(module), _ptr(x), _ptr(y), ctypes.byref(g.s), ctypes.byref(p), cap,
                            ctypes.byref(nt), _ptr(offs), _ptr(ids), _ptr(st))
    if rc != 0:
        raise RuntimeError("vo_track_event: capacity")
    t = nt.value
    tracks = [ids[int(offs[i]):int(offs[i + 1])].copy() for i in range(t)]
    return tracks, st[:t].copy()


def fit(x, y, z, sigma: float, ms_theta: float, dtype=np.float32) -> np.ndarray:
    """Straight-line LSQ + simplified Kalman of one track (hits ascending in z) -> state[20]."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype)
    y = np.ascontiguousarray(y, dtype)
    z = np.ascontiguousarray(z, dtype)
    out = np.zeros(STATE_STRIDE, dtype)
    f = lib.vo_fit_f32 if dtype == np.float32 else lib.vo_fit_f64
    f(len(x), _ptr(x), _ptr(y), _ptr(z), sigma, ms_theta, _ptr(out))
    return out


def reconstruct(offsets: np.ndarray, pixels: np.ndarray, geometry, params: Params = Params(), n_threads: int = 0,
                mlp=None):
    """Whole batch on the host cores -> dict of numpy arrays in the library's output layout.
    mlp: float32 model blob (MLP_FLOATS) when params.use_mlp."""
    lib = _load()
    off = np.ascontiguousarray(offsets, np.uint64)
    pix = np.ascontiguousarray(pixels, np.uint32)
    ne = len(off) - 1
    g = _GeoHolder(geometry)
    p = _par(params, mlp)
    h = lib.vo_reconstruct(ne, _ptr(off), _ptr(pix), ctypes.byref(g.s), ctypes.byref(p), n_threads)
    try:
        nc, nt, nh = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        lib.vo_batch_sizes(h, ctypes.byref(nc), ctypes.byref(nt), ctypes.byref(nh))
        out = dict(
            status=np.zeros(ne, np.int32),
            cluster_offsets=np.zeros(ne + 1, np.uint64),
            cluster_x=np.zeros(nc.value, np.float32),
            cluster_y=np.zeros(nc.value, np.float32),
            cluster_z=np.zeros(nc.value, np.float32),
            pixel_cluster=np.zeros(len(pix), np.uint32),
            track_offsets=np.zeros(ne + 1, np.uint64),
            track_hit_offsets=np.zeros(nt.value + 1, np.uint64),
            track_hits=np.zeros(nh.value, np.uint32),
            track_states=np.zeros((nt.value, STATE_STRIDE), np.float32),
            track_features=np.zeros((nt.value, N_FEATURES), np.float32),
        )
        lib.vo_batch_copy(h, *(_ptr(out[k]) for k in ("status", "cluster_offsets", "cluster_x", "cluster_y",
                                                       "cluster_z", "pixel_cluster", "track_offsets",
                                                       "track_hit_offsets", "track_hits", "track_states",
                                                       "track_features")))
    finally:
        lib.vo_batch_free(h)
    return out


def features(x, y, z, module, state, chi2ndf) -> np.ndarray:
    """The 12 candidate features of one track (hits ascending in z)."""
    lib = _load()
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    z = np.ascontiguousarray(z, np.float32)
    module = np.ascontiguousarray(module, np.uint32)
    state = np.ascontiguousarray(state, np.float32)
    out = np.zeros(N_FEATURES, np.float32)
    lib.vo_features(len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(module), _ptr(state), float(chi2ndf), _ptr(out))
    return out


def mlp_logit(mlp: np.ndarray, f: np.ndarray) -> float:
    """The network's logit for one feature vector (bfloat16 emulation, see velo_oracle.h)."""
    lib = _load()
    mlp = np.ascontiguousarray(mlp, np.float32)
    f = np.ascontiguousarray(f, np.float32)
    return float(lib.vo_mlp_logit(_ptr(mlp), _ptr(f)))


def downstream_struct(down) -> _Down:
    d = _Down()
    d.z_mag = float(down.z_mag)
    for i, z in enumerate(down.z_layers):
        d.z_layers[i] = float(z)
    d.kappa = float(down.kappa)
    return d


def forward(scifi_offsets, layer, x, y, result, down, params: FwdParams = FwdParams(), threads: int = 0):
    """Forward tracking of a batch: downstream hits in CSR (per event, ids =
    index within the event) and a reconstruction result (numpy dict with
    cluster_offsets, cluster_x/y/z, track_offsets, track_hit_offsets,
    track_hits).  Returns n_found [T], hits [T, 12] (event-local hit ids,
    0xFFFFFFFF = none), state [T, 6] = (q/p, chi2/ndf, b, a, d_x, d_y).
    Events are independent; `threads` (0 = every core) run them side by side
    (each event is one call of the C function, which releases the GIL)."""
    lib = _load()
    so = np.asarray(scifi_offsets, np.int64)
    to = np.asarray(result["track_offsets"], np.int64)
    co = np.asarray(result["cluster_offsets"], np.int64)
    hoff = np.asarray(result["track_hit_offsets"], np.uint64)
    th = np.ascontiguousarray(result["track_hits"], np.uint32)
    cx = np.ascontiguousarray(result["cluster_x"], np.float32)
    cy = np.ascontiguousarray(result["cluster_y"], np.float32)
    cz = np.ascontiguousarray(result["cluster_z"], np.float32)
    layer = np.ascontiguousarray(layer, np.uint32)
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    T = int(to[-1])
    n_found = np.zeros(max(T, 1), np.uint32)
    hits = np.full((max(T, 1), FWD_LAYERS), 0xFFFFFFFF, np.uint32)
    state = np.zeros((max(T, 1), FWD_STATE), np.float32)
    d = downstream_struct(down)
    p = _FwdPar(**asdict(params))
    def one(e):
        h0, h1, t0, t1, c0 = int(so[e]), int(so[e + 1]), int(to[e]), int(to[e + 1]), int(co[e])
        if t1 == t0:
            return
        ho = np.ascontiguousarray(hoff[t0:t1 + 1] - hoff[t0])
        tk = np.ascontiguousarray(th[int(hoff[t0]):int(hoff[t1])])
        lib.vo_forward_event(h1 - h0, _ptr(layer[h0:h1]), _ptr(x[h0:h1]), _ptr(y[h0:h1]), t1 - t0, _ptr(ho), _ptr(tk),
                             _ptr(cx[c0:]), _ptr(cy[c0:]), _ptr(cz[c0:]), ctypes.byref(d), ctypes.byref(p),
                             _ptr(n_found[t0:t1]), _ptr(hits[t0:t1]), _ptr(state[t0:t1]))

    n_thr = threads if threads > 0 else (os.cpu_count() or 1)
    if n_thr == 1 or len(to) <= 2:
        for e in range(len(to) - 1):
            one(e)
    else:
        with concurrent.futures.ThreadPoolExecutor(max_workers=n_thr) as ex:
            list(ex.map(one, range(len(to) - 1)))
    return n_found[:T], hits[:T], state[:T]
