"""Pins of the learned ghost rejection's reference arithmetic, CPU only.

* the float64 backward of ``oracle.mlp`` against central finite differences;
* the bfloat16 rounding of the C++ oracle against torch's bfloat16 conversion
  (round to nearest even), and its logit within the bfloat16 error of the
  float64 forward;
* the candidate features against closed forms: a noise-free line has zero
  residuals; the residual mean and RMS equal numpy's on a track with known
  offsets; skipped modules and z ends come from the hit pattern.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp

Z = -300.0 + 42.0 * np.arange(26)


def random_blob(rng):
    w = rng.normal(0, 0.4, mlp.N_WEIGHTS)
    mean = rng.normal(0, 1, 12)
    inv_std = rng.uniform(0.5, 2.0, 12)
    return mlp.pack(mean, inv_std, w)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.5, mlp.N_WEIGHTS)
    X = rng.normal(0, 1, (40, 12))
    y = (rng.random(40) < 0.4).astype(np.float64)
    L, g = mlp.backward(w, X, y)
    h = 1e-6
    idx = rng.choice(mlp.N_WEIGHTS, 120, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(mlp.forward(wp, X)[0], y) - mlp.loss(mlp.forward(wm, X)[0], y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_bf16_rounding_is_round_to_nearest_even():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 10, 2000), rng.normal(0, 1e-3, 500), [0.0, -0.0, 1.0, 1.00390625, 1.01171875]])
    v = v.astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    # exact ties (the lower 16 bits 0x8000) go to the even neighbour: 1 + 2^-8 rounds
    # down to 1, 1 + 3 * 2^-8 up to 1 + 2^-6
    assert ref[-2] == 1.0 and ref[-1] == 1.015625
    # a network whose only path is one input -> one hidden unit -> logit exposes bf16(x)
    for x, r in zip(np.concatenate([v[:300], v[-5:]]), np.concatenate([ref[:300], ref[-5:]])):
        blob = np.zeros(mlp.N_FLOATS, np.float32)
        p = mlp.unpack(blob)
        p["inv_std"][0] = 1.0
        p["W1"][0, 0] = 1.0  # bf16(1) = 1
        p["W2"][0, 0] = 1.0
        p["W3"][0] = 1.0
        f = np.zeros(12, np.float32)
        f[0] = abs(x)
        got = oracle.mlp_logit(blob, f)
        # h1 = bf16(relu(bf16(|x|))) = bf16(|x|); h2 = h1; logit = h1
        assert got == abs(float(torch.tensor(abs(float(x))).to(torch.bfloat16).float()))


def test_logit_within_bf16_error_of_float64_forward():
    rng = np.random.default_rng(2)
    for _ in range(20):
        blob = random_blob(rng)
        p = mlp.unpack(blob)
        w = blob[24:].astype(np.float64)
        for _ in range(20):
            f = rng.normal(0, 1, 12).astype(np.float32)
            xn = (f.astype(np.float64) - p["mean"]) * p["inv_std"]
            z64 = mlp.forward(w, xn[None, :])[0][0]
            z = oracle.mlp_logit(blob, f)
            # three bf16 roundings (inputs, weights, h1) of relative size 2^-8 each
            scale = 1.0 + np.abs(p["W3"]).sum() * 4
            assert abs(z - z64) <= 0.05 * scale, (z, z64)


def test_features_of_exact_line():
    mods = np.array([5, 6, 7, 9, 10, 11], np.uint32)
    z = Z[mods].astype(np.float32)
    x = (0.03 * (z + 20)).astype(np.float32)
    y = (-0.05 * (z + 20)).astype(np.float32)
    st = oracle.fit(x, y, z, 0.0159, 0.0)
    f = oracle.features(x, y, z, mods, st, 0.5)
    assert f[0] == 6 and f[1] == np.float32(0.5) and f[4] == z[0] and f[5] == z[-1]
    assert f[6] == 1  # module 8 missed
    assert f[2] == st[2] and f[3] == st[3]
    assert np.all(np.abs(f[7:]) < 1e-4)


def test_features_residual_statistics():
    rng = np.random.default_rng(3)
    for _ in range(50):
        n = int(rng.integers(3, 15))
        mods = np.sort(rng.choice(26, n, replace=False)).astype(np.uint32)
        z = Z[mods].astype(np.float32)
        x = (rng.uniform(-20, 20) + rng.uniform(-0.2, 0.2) * (z - z[0]) + rng.normal(0, 0.02, n)).astype(np.float32)
        y = (rng.uniform(-20, 20) + rng.uniform(-0.2, 0.2) * (z - z[0]) + rng.normal(0, 0.02, n)).astype(np.float32)
        st = oracle.fit(x, y, z, 0.0159, 5e-4)
        f = oracle.features(x, y, z, mods, st, 1.25)
        dz = z.astype(np.float64) - z[0]
        rx = x - st[0] - st[2] * dz
        ry = y - st[1] - st[3] * dz
        np.testing.assert_allclose(f[[7, 8, 9, 10]], [rx.mean(), np.sqrt((rx ** 2).mean()), ry.mean(),
                                                      np.sqrt((ry ** 2).mean())], atol=2e-5)
        np.testing.assert_allclose(f[11], max(np.abs(rx).max(), np.abs(ry).max()), atol=2e-5)
        assert f[6] == (mods[-1] - mods[0] + 1) - n
        assert f[8] >= abs(f[7]) - 1e-7 and f[10] >= abs(f[9]) - 1e-7


def test_learned_rejection_replaces_three_hit_rule():
    """With a network whose logit is a constant, every candidate passes (or none
    does) the learned rule; the loose chi2 cut still applies."""
    import velogen
    b = velogen.generate(velogen.C2, n_events=3)
    blob = np.zeros(mlp.N_FLOATS, np.float32)
    mlp.unpack(blob)["b3"][0] = 1.0  # logit = 1 for every candidate
    keep_all = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params(use_mlp=1, mlp_logit_min=0.5),
                                  mlp=blob)
    plain_loose = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params(chi2ndf_max_3hit=10.0))
    np.testing.assert_array_equal(keep_all["track_hits"], plain_loose["track_hits"])
    assert (keep_all["track_states"][:, 19] == 1.0).all()
    none = oracle.reconstruct(b.offsets, b.pixels, b.geometry, oracle.Params(use_mlp=1, mlp_logit_min=1.5), mlp=blob)
    assert len(none["track_states"]) == 0
