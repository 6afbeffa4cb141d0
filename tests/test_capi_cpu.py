"""Host-only checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every entry point include/velo.h declares, and its host-side
functions (defaults, sizes, error names, argument validation) behave."""
import ctypes
import os
import re

import pytest

import paper_2412_05041_b300 as velo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    velo.build()
    return velo.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "velo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(velo_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(velo.EXPORTS)


def test_defaults_and_strerror(L):
    p = velo.default_params()
    assert p.win_seed == pytest.approx(0.04) and p.max_skipped == 1 and p.chi2ndf_max_3hit == 2.0
    assert L.velo_strerror(velo.EINVAL) == b"invalid argument"
    assert L.velo_version() >= 100


def test_query_sizes(L):
    s = velo.query_sizes(10, 3000)
    assert s.cap_clusters == 3000 and s.cap_tracks == 1000 and s.cap_track_hits == 3000
    assert s.workspace_bytes % 256 == 0 and s.workspace_bytes > 3000 * 60
    assert velo.query_sizes(20, 3000).workspace_bytes > s.workspace_bytes
    assert L.velo_query_sizes(1 << 31, 10, ctypes.byref(velo.Sizes())) == velo.EINVAL


def test_argument_validation_before_any_device_call(L, geometry):
    g = velo.geometry_struct(geometry)
    p = velo.default_params()
    out = velo.Output(*([ctypes.c_void_p(256)] * 11))
    ev = velo.Events(1, 10, ctypes.c_void_p(256), ctypes.c_void_p(256))
    ws = ctypes.c_void_p(1 << 20)
    call = lambda e, gg, pp, o, w, nbytes: L.velo_reconstruct_into(e, gg, pp, o, w, nbytes, None)
    assert call(None, ctypes.byref(g.s), ctypes.byref(p), ctypes.byref(out), ws, 1 << 40) == velo.EINVAL
    bad = velo.default_params(win_seed=1.5)
    assert call(ctypes.byref(ev), ctypes.byref(g.s), ctypes.byref(bad), ctypes.byref(out), ws, 1 << 40) == velo.EINVAL
    bad = velo.default_params(sigma_meas=0.0)
    assert call(ctypes.byref(ev), ctypes.byref(g.s), ctypes.byref(bad), ctypes.byref(out), ws, 1 << 40) == velo.EINVAL
    gz = velo.geometry_struct(geometry)
    gz.z[3] = gz.z[2]  # not strictly ascending
    assert call(ctypes.byref(ev), ctypes.byref(gz.s), ctypes.byref(p), ctypes.byref(out), ws, 1 << 40) == velo.EINVAL
    # misaligned workspace, and a workspace that is too small
    assert call(ctypes.byref(ev), ctypes.byref(g.s), ctypes.byref(p), ctypes.byref(out), ctypes.c_void_p((1 << 20) + 8),
                1 << 40) == velo.EINVAL
    assert call(ctypes.byref(ev), ctypes.byref(g.s), ctypes.byref(p), ctypes.byref(out), ws, 100) == velo.ECAPACITY
    nul = velo.Output(*([ctypes.c_void_p(256)] * 10 + [None]))
    assert call(ctypes.byref(ev), ctypes.byref(g.s), ctypes.byref(p), ctypes.byref(nul), ws, 1 << 40) == velo.EINVAL


def test_forward_argument_validation_before_any_device_call(L):
    from velogen import scifi
    d = velo.downstream_struct(scifi.Downstream())
    p = velo.default_forward_params()
    assert (p.p_min, p.tol_x_far, p.sigma_x, p.min_hits) == (3.0, 3.0, pytest.approx(0.08), 9)
    trk = velo.Output(*([ctypes.c_void_p(256)] * 11))
    h = velo.DownstreamHits(1, 10, *([ctypes.c_void_p(256)] * 4))
    o = velo.ForwardOutput(ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256), 10)
    ws = ctypes.c_void_p(1 << 20)
    need = ctypes.c_uint64()
    assert L.velo_forward_workspace_size(1, 10, ctypes.byref(need)) == velo.OK
    assert need.value % 256 == 0 and need.value >= 10 * 24
    big = ctypes.c_uint64()
    L.velo_forward_workspace_size(1, 1000, ctypes.byref(big))
    assert big.value > need.value

    def call(hh=h, pp=p, dd=d, w=ws, nbytes=1 << 40, oo=o, tt=trk):
        return L.velo_forward(ctypes.byref(hh) if hh is not None else None, ctypes.byref(tt), ctypes.byref(dd),
                              ctypes.byref(pp), ctypes.byref(oo), w, nbytes, None)

    assert call(hh=None) == velo.EINVAL
    for k, v in (("min_hits", 2), ("min_hits", 13), ("p_min", 0.0), ("sigma_x", -1.0), ("tol_x", float("nan")),
                 ("tol_match", float("inf")), ("p_min", 1e-44)):
        assert call(pp=velo.default_forward_params(**{k: v})) == velo.EINVAL, (k, v)
    dz = velo.downstream_struct(scifi.Downstream())
    dz.z_layers[5] = dz.z_layers[4]  # not strictly ascending
    assert call(dd=dz) == velo.EINVAL
    dz = velo.downstream_struct(scifi.Downstream())
    dz.z_mag = dz.z_layers[0] + 1.0  # a layer in front of the kick plane
    assert call(dd=dz) == velo.EINVAL
    dz = velo.downstream_struct(scifi.Downstream())
    dz.kappa = 0.0
    assert call(dd=dz) == velo.EINVAL
    assert call(w=ctypes.c_void_p((1 << 20) + 16)) == velo.EINVAL  # misaligned workspace
    assert call(nbytes=need.value - 1) == velo.ECAPACITY
    no_totals = velo.Output(*([ctypes.c_void_p(256)] * 10 + [None]))
    assert call(tt=no_totals) == velo.EINVAL
    assert call(oo=velo.ForwardOutput(None, ctypes.c_void_p(256), ctypes.c_void_p(256), 10)) == velo.EINVAL


def test_no_cpu_fallback(monkeypatch, tmp_path):
    """Without the built library every call raises instead of computing elsewhere."""
    import importlib
    monkeypatch.setattr(velo, "_lib", None)
    monkeypatch.setattr(velo, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(velo.VeloError):
        velo.lib()
