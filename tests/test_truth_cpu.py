"""The library's truth matching (used for training labels and reported
efficiencies) against the oracle's independent implementation, and the model
file format."""
import numpy as np

import oracle
import velogen
from oracle import mc
from paper_2412_05041_b300 import mlp, truth


def test_truth_metrics_agree_with_oracle_matching():
    b = velogen.generate(velogen.C2, n_events=25, first_event=40, truth=True)
    r = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params())
    a = truth.metrics(b, r)
    o = mc.evaluate_batch(b, r)
    assert a["reconstructible"] == o["reconstructible"] and a["tracks"] == o["tracks"]
    for k in ("efficiency", "ghost_rate", "clone_rate"):
        assert abs(a[k] - o[k]) < 1e-12, (k, a[k], o[k])


def test_model_file_roundtrip(tmp_path):
    blob = np.arange(mlp.MLP_FLOATS, dtype=np.float32) * 0.5
    p = tmp_path / "m.bin"
    mlp.save(str(p), blob, -1.25)
    b2, thr = mlp.load(str(p))
    np.testing.assert_array_equal(blob, b2)
    assert thr == -1.25


def test_downstream_hits_regenerate_per_event():
    """Every event's downstream hits come from its own stream (seed, event
    index): an event generated alone equals its slice of a batch, and two
    batches of the same configuration are identical."""
    import numpy as np
    import velogen
    from velogen import scifi
    b = velogen.generate(velogen.C2, n_events=6, first_event=100, truth=True)
    s = scifi.generate(b)
    again = scifi.generate(velogen.generate(velogen.C2, n_events=6, first_event=100, truth=True))
    for k in ("offsets", "layer", "x", "y", "truth"):
        assert np.array_equal(getattr(s, k), getattr(again, k))
    for e in (0, 3, 5):
        one = scifi.generate(velogen.generate(velogen.C2, n_events=1, first_event=100 + e, truth=True))
        h0, h1 = int(s.offsets[e]), int(s.offsets[e + 1])
        assert np.array_equal(one.x, s.x[h0:h1]) and np.array_equal(one.layer, s.layer[h0:h1])
    assert ((s.layer >= 0) & (s.layer < scifi.N_LAYERS)).all()
    assert (np.abs(s.x) <= s.geometry.half_x).all() and (np.abs(s.y) <= s.geometry.half_y).all()
