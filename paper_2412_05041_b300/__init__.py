"""B300-native event-batched VELO-like pixel tracking (sm_103a CUDA kernels behind a C ABI).

The paper's first trigger stage reconstructs every collision event on GPUs at
the full input rate, with a simplified pattern recognition and a
parameterised Kalman filter on the pixel-tracker segment of each track
(Sec. "Introduction", Sec. "HLT1 details and results").  This package is the
thin Python layer over ``libvelo.so`` (``include/velo.h``): it marshals torch
tensors (device memory, streams) into the C structs and calls the library.
Every step of the reconstruction runs in the library's CUDA kernels; there is
no CPU fallback -- without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB_PATH, build  # noqa: F401

STATE_STRIDE = 20
MAX_MODULES = 32
STATIC_SCRATCH_BYTES = 64 << 20  # scratch array behind velo_reconstruct_static
N_FEATURES = 12
MLP_WEIGHTS = 1505
MLP_FLOATS = 1529
FEATURE_NAMES = ("n_hits", "chi2ndf", "tx", "ty", "z_first", "z_last", "n_skipped", "mean_rx", "rms_rx", "mean_ry",
                 "rms_ry", "max_abs_r")
EVT_OK, EVT_BADWORD, EVT_OVERFLOW, EVT_TIMEOUT = 0, 1, 2, 3
OK, EINVAL, ECAPACITY, ECUDA, ENOMEM = 0, 1, 2, 3, 5
STATE_FIELDS = ("x", "y", "tx", "ty", "z_first", "z_beam", "chi2_lsq", "chi2_kf", "kf_x", "kf_y", "kf_tx",
                "kf_ty", "kf_cxx", "kf_cxtx", "kf_ctxtx", "kf_cyy", "kf_cyty", "kf_ctyty", "ndf", "reserved")

_P = ctypes.c_void_p


class Geometry(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_uint32), ("module_z", ctypes.POINTER(ctypes.c_float)),
                ("pitch_mm", ctypes.c_float), ("n_rows", ctypes.c_uint32), ("n_cols", ctypes.c_uint32),
                ("x0_mm", ctypes.c_float), ("y0_mm", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("win_seed", ctypes.c_float), ("win_fwd", ctypes.c_float), ("max_slope", ctypes.c_float),
                ("max_scatter_seed", ctypes.c_float), ("max_scatter_fwd", ctypes.c_float),
                ("max_skipped", ctypes.c_uint32), ("sigma_meas", ctypes.c_float), ("ms_theta", ctypes.c_float),
                ("chi2ndf_max", ctypes.c_float), ("chi2ndf_max_3hit", ctypes.c_float),
                ("use_mlp", ctypes.c_uint32), ("mlp_logit_min", ctypes.c_float), ("mlp", _P)]


class Events(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint64), ("n_pixels", ctypes.c_uint64), ("event_offsets", _P),
                ("pixels", _P)]


class Output(ctypes.Structure):
    _fields_ = [("status", _P), ("cluster_offsets", _P), ("cluster_x", _P), ("cluster_y", _P), ("cluster_z", _P),
                ("pixel_cluster", _P), ("track_offsets", _P), ("track_hit_offsets", _P), ("track_hits", _P),
                ("track_states", _P), ("totals", _P), ("track_features", _P), ("cap_clusters", ctypes.c_uint64),
                ("cap_tracks", ctypes.c_uint64), ("cap_track_hits", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("cluster_threads", ctypes.c_uint32), ("cluster_smem_pixels", ctypes.c_uint32),
                ("track_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("wide_cluster", ctypes.c_uint32), ("fused_output", ctypes.c_uint32),
                ("union_link_attempts", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Sizes(ctypes.Structure):
    _fields_ = [("cap_clusters", ctypes.c_uint64), ("cap_tracks", ctypes.c_uint64),
                ("cap_track_hits", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64)]


class ResultView(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint64), ("n_pixels", ctypes.c_uint64), ("cap_clusters", ctypes.c_uint64),
                ("cap_tracks", ctypes.c_uint64), ("cap_track_hits", ctypes.c_uint64), ("out", Output)]


FWD_LAYERS = 12
FWD_STATE = 6
FWD_STATE_FIELDS = ("qop", "chi2ndf", "b", "a", "d_x", "d_y")


class Downstream(ctypes.Structure):
    _fields_ = [("z_mag", ctypes.c_float), ("z_layers", ctypes.c_float * FWD_LAYERS), ("kappa", ctypes.c_float)]


class ForwardParams(ctypes.Structure):
    _fields_ = [("p_min", ctypes.c_float), ("win_y", ctypes.c_float), ("tol_x", ctypes.c_float),
                ("tol_y", ctypes.c_float), ("tol_x_far", ctypes.c_float), ("sigma_x", ctypes.c_float),
                ("tol_match", ctypes.c_float), ("chi2ndf_max", ctypes.c_float), ("min_hits", ctypes.c_uint32)]


class DownstreamHits(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint64), ("n_hits", ctypes.c_uint64), ("event_offsets", _P), ("layer", _P),
                ("x", _P), ("y", _P)]


class ForwardOutput(ctypes.Structure):
    _fields_ = [("n_found", _P), ("hits", _P), ("state", _P), ("cap_tracks", ctypes.c_uint64)]


class VeloError(RuntimeError):
    pass


_lib = None

# every entry point declared in include/velo.h
EXPORTS = ("velo_params_default", "velo_query_sizes", "velo_reconstruct_into", "velo_reconstruct_into_marked",
           "velo_tuning_default", "velo_reconstruct_into_tuned", "velo_reconstruct",
           "velo_result_view", "velo_result_free", "velo_context_create", "velo_context_destroy",
           "velo_context_set_pipeline", "velo_reconstruct_host", "velo_reconstruct_static", "velo_mlp_infer", "velo_mlp_workspace_size",
           "velo_mlp_loss_grad", "velo_mlp_adam_step", "velo_forward_params_default", "velo_forward_workspace_size",
           "velo_forward", "velo_measure_fp32_peak", "velo_strerror", "velo_version")


def lib():
    """The loaded ``libvelo.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise VeloError(f"{LIB_PATH} is missing: run paper_2412_05041_b300.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        L.velo_params_default.argtypes = [ctypes.POINTER(Params)]
        L.velo_query_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(Sizes)]
        L.velo_reconstruct_into.argtypes = [ctypes.POINTER(Events), ctypes.POINTER(Geometry), ctypes.POINTER(Params),
                                            ctypes.POINTER(Output), _P, ctypes.c_uint64, _P]
        L.velo_reconstruct_into_marked.argtypes = L.velo_reconstruct_into.argtypes + [ctypes.POINTER(_P)]
        L.velo_tuning_default.argtypes = [ctypes.POINTER(Tuning)]
        L.velo_reconstruct_into_tuned.argtypes = L.velo_reconstruct_into_marked.argtypes + [ctypes.POINTER(Tuning)]
        L.velo_reconstruct.argtypes = [ctypes.POINTER(Events), ctypes.POINTER(Geometry), ctypes.POINTER(Params),
                                       ctypes.POINTER(_P), _P]
        L.velo_result_view.argtypes = [_P, ctypes.POINTER(ResultView)]
        L.velo_result_free.argtypes = [_P]
        L.velo_result_free.restype = None
        L.velo_context_create.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(_P)]
        L.velo_context_destroy.argtypes = [_P]
        L.velo_context_destroy.restype = None
        L.velo_context_set_pipeline.argtypes = [_P, ctypes.c_uint32]
        L.velo_reconstruct_host.argtypes = [_P, ctypes.POINTER(Events), ctypes.POINTER(Geometry),
                                            ctypes.POINTER(Params), ctypes.POINTER(Output), _P]
        L.velo_reconstruct_static.argtypes = [ctypes.POINTER(Events), ctypes.POINTER(Geometry),
                                              ctypes.POINTER(Params), ctypes.POINTER(Output), _P]
        L.velo_mlp_infer.argtypes = [_P, ctypes.c_uint64, _P, _P, ctypes.c_int, _P]
        L.velo_mlp_workspace_size.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.velo_mlp_loss_grad.argtypes = [_P, _P, ctypes.c_uint64, _P, _P, _P, _P, ctypes.c_uint64, _P]
        L.velo_mlp_adam_step.argtypes = [_P, _P, _P, _P, ctypes.c_uint32, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_uint32, _P]
        L.velo_forward_params_default.argtypes = [ctypes.POINTER(ForwardParams)]
        L.velo_forward_workspace_size.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.velo_forward.argtypes = [ctypes.POINTER(DownstreamHits), ctypes.POINTER(Output), ctypes.POINTER(Downstream),
                                   ctypes.POINTER(ForwardParams), ctypes.POINTER(ForwardOutput), _P, ctypes.c_uint64,
                                   _P]
        L.velo_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _P]
        L.velo_strerror.restype = ctypes.c_char_p
        L.velo_strerror.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def check(rc: int, what: str = "velo call"):
    if rc != OK:
        raise VeloError(f"{what} failed: {lib().velo_strerror(rc).decode()} ({rc})")


def default_params(**overrides) -> Params:
    p = Params()
    check(lib().velo_params_default(ctypes.byref(p)), "velo_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class _GeometryHolder:
    """Keeps the module_z array alive while a Geometry struct points at it."""

    def __init__(self, g):
        n = int(g.n_modules)
        self.z = (ctypes.c_float * n)(*[float(z) for z in g.module_z])
        self.s = Geometry(n, ctypes.cast(self.z, ctypes.POINTER(ctypes.c_float)), float(g.pitch), int(g.n_rows),
                          int(g.n_cols), float(g.x0), float(g.y0))


def geometry_struct(g) -> _GeometryHolder:
    """From any object with n_modules, module_z, pitch, n_rows, n_cols, x0, y0."""
    return _GeometryHolder(g)


def default_tuning(**overrides) -> Tuning:
    t = Tuning()
    check(lib().velo_tuning_default(ctypes.byref(t)), "velo_tuning_default")
    for k, v in overrides.items():
        setattr(t, k, v)
    return t


def query_sizes(n_events: int, n_pixels: int) -> Sizes:
    s = Sizes()
    check(lib().velo_query_sizes(n_events, n_pixels, ctypes.byref(s)), "velo_query_sizes")
    return s


def default_forward_params(**overrides) -> ForwardParams:
    p = ForwardParams()
    check(lib().velo_forward_params_default(ctypes.byref(p)), "velo_forward_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def downstream_struct(g) -> Downstream:
    """From any object with z_mag, z_layers (12), kappa."""
    d = Downstream()
    d.z_mag = float(g.z_mag)
    for i, z in enumerate(g.z_layers):
        d.z_layers[i] = float(z)
    d.kappa = float(g.kappa)
    return d


from .api import GraphReconstructor, HostReconstructor, Reconstructor, reconstruct  # noqa: E402,F401
from .forward import ForwardTracker  # noqa: E402,F401
