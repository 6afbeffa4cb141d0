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
