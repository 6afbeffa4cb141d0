"""Element-by-element comparison of a library result with the oracle's (numpy dicts)."""
import numpy as np

# Track states are computed by the same binary32 operations in the same order
# on both sides, so they agree bit for bit in practice; the contract is a
# relative error of at most 1e-5 (absolute 1e-6 near zero).
STATE_RTOL = 1e-5
STATE_ATOL = 1e-6


def to_numpy(r: dict) -> dict:
    out = {}
    for k, v in r.items():
        if hasattr(v, "detach"):
            v = v.detach().cpu().numpy()
        out[k] = v
    return out


def assert_same(gpu: dict, ref: dict, events=None, check_labels=True):
    """gpu, ref: dicts in the library's output layout.  events: optional list of
    event indices of gpu that correspond, in order, to the events of ref."""
    g = to_numpy(gpu)
    E = len(ref["status"])
    ev = list(range(E)) if events is None else list(events)
    assert len(ev) == E
    st = g["status"].astype(np.int32)
    for j, e in enumerate(ev):
        assert st[e] == ref["status"][j], (e, st[e], ref["status"][j])
        gc0, gc1 = int(g["cluster_offsets"][e]), int(g["cluster_offsets"][e + 1])
        rc0, rc1 = int(ref["cluster_offsets"][j]), int(ref["cluster_offsets"][j + 1])
        assert gc1 - gc0 == rc1 - rc0, ("n_clusters", e, gc1 - gc0, rc1 - rc0)
        for k in ("cluster_x", "cluster_y", "cluster_z"):
            np.testing.assert_array_equal(g[k][gc0:gc1], ref[k][rc0:rc1], err_msg=f"{k} event {e}")
        gt0, gt1 = int(g["track_offsets"][e]), int(g["track_offsets"][e + 1])
        rt0, rt1 = int(ref["track_offsets"][j]), int(ref["track_offsets"][j + 1])
        assert gt1 - gt0 == rt1 - rt0, ("n_tracks", e, gt1 - gt0, rt1 - rt0)
        gh = g["track_hit_offsets"].astype(np.int64)
        rh = ref["track_hit_offsets"].astype(np.int64)
        for a, b in zip(range(gt0, gt1), range(rt0, rt1)):
            ga = g["track_hits"][gh[a]:gh[a + 1]].astype(np.uint32)
            rb = ref["track_hits"][rh[b]:rh[b + 1]].astype(np.uint32)
            np.testing.assert_array_equal(ga, rb, err_msg=f"track hits event {e} track {a - gt0}")
        np.testing.assert_allclose(g["track_states"][gt0:gt1], ref["track_states"][rt0:rt1], rtol=STATE_RTOL,
                                   atol=STATE_ATOL, err_msg=f"states event {e}")
    return True


def assert_labels(gpu_labels, ref_labels, gpu_offsets, ref_offsets, events=None):
    g = np.asarray(gpu_labels).astype(np.uint32)
    r = np.asarray(ref_labels).astype(np.uint32)
    E = len(ref_offsets) - 1
    ev = list(range(E)) if events is None else list(events)
    for j, e in enumerate(ev):
        a0, a1 = int(gpu_offsets[e]), int(gpu_offsets[e + 1])
        b0, b1 = int(ref_offsets[j]), int(ref_offsets[j + 1])
        np.testing.assert_array_equal(g[a0:a1], r[b0:b1], err_msg=f"pixel labels event {e}")


def exact_state_fraction(gpu, ref):
    g = to_numpy(gpu)["track_states"]
    return float((g == ref["track_states"]).mean()) if len(g) else 1.0
