"""Pins of the oracle's track fit (straight-line least squares and the simplified
Kalman filter that the paper names as the first stage's track fit, Sec. "HLT1
details and results"), CPU only.

Each pin checks the oracle against an independent solution:
* least squares vs numpy.polyfit (float64 build of the same oracle code);
* the Kalman filter with no process noise vs least squares (two different
  algorithms that must meet: the filter starts from the last two hits with
  no prior, so both minimise the same chi2);
* the Kalman filter with process noise vs the batch generalised-least-squares
  solution of the same random-walk model, solved by numpy.linalg.lstsq --
  state, covariance and the chi2 sum of normalised innovations;
* closed forms: chi2 of three points with a displaced middle point, the
  closest approach to the beam of a line through the z axis;
* the float32 build stays within float32 rounding of the float64 build.
"""
import numpy as np
import pytest

import oracle

Z = -300.0 + 42.0 * np.arange(26)


def rand_track(rng, n, sigma=0.0159, first=None):
    k0 = int(rng.integers(0, 26 - n + 1)) if first is None else first
    z = Z[k0:k0 + n].copy()
    x = rng.uniform(-30, 30) + rng.uniform(-0.3, 0.3) * (z - z[0]) + rng.normal(0, sigma, n)
    y = rng.uniform(-30, 30) + rng.uniform(-0.3, 0.3) * (z - z[0]) + rng.normal(0, sigma, n)
    return x, y, z


@pytest.mark.parametrize("n", [3, 4, 7, 12, 26])
def test_lsq_matches_polyfit(n):
    rng = np.random.default_rng(n)
    sigma = 0.0159
    for _ in range(50):
        x, y, z = rand_track(rng, n)
        st = oracle.fit(x, y, z, sigma, 0.0, dtype=np.float64)
        dz = z - z[0]
        bx, ax = np.polyfit(dz, x, 1)
        by, ay = np.polyfit(dz, y, 1)
        np.testing.assert_allclose([st[0], st[1], st[2], st[3]], [ax, ay, bx, by], rtol=1e-9, atol=1e-11)
        chi2 = (((x - ax - bx * dz) / sigma) ** 2).sum() + (((y - ay - by * dz) / sigma) ** 2).sum()
        np.testing.assert_allclose(st[6], chi2, rtol=1e-7, atol=1e-12)
        assert st[4] == z[0] and st[18] == 2 * n - 4


@pytest.mark.parametrize("n", [3, 5, 10, 26])
def test_kalman_without_noise_equals_lsq(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(30):
        x, y, z = rand_track(rng, n)
        st = oracle.fit(x, y, z, 0.0159, 0.0, dtype=np.float64)
        np.testing.assert_allclose(st[8:12], st[0:4], rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(st[7], st[6], rtol=1e-9, atol=1e-12)


def gls_reference(z, m, sigma, theta):
    """Batch solution of the model the filter runs (downstream -> upstream):
    X_i = X_{i+1} + T_{i+1} (z_i - z_{i+1}),  T_i = T_{i+1} + w_i,  w_i ~ N(0, theta^2),
    flat prior on (X_{n-1}, T_{n-1}), measurements m_i = X_i + N(0, sigma^2)."""
    n = len(z)
    npar = 2 + (n - 1)
    coefX = {n - 1: np.eye(npar)[0]}
    coefT = {n - 1: np.eye(npar)[1]}
    for k, i in enumerate(range(n - 2, -1, -1)):
        coefX[i] = coefX[i + 1] + coefT[i + 1] * (z[i] - z[i + 1])
        coefT[i] = coefT[i + 1] + np.eye(npar)[2 + k]
    rows, rhs = [], []
    for i in range(n):
        rows.append(coefX[i] / sigma)
        rhs.append(m[i] / sigma)
    for k in range(n - 1):
        rows.append(np.eye(npar)[2 + k] / theta)
        rhs.append(0.0)
    A, b = np.array(rows), np.array(rhs)
    beta, *_ = np.linalg.lstsq(A, b, rcond=None)
    cov = np.linalg.inv(A.T @ A)
    G = np.stack([coefX[0], coefT[0]])
    state = G @ beta
    C = G @ cov @ G.T
    chi2 = float(((A @ beta - b) ** 2).sum())
    return state, C, chi2


@pytest.mark.parametrize("n", [3, 4, 8, 15])
def test_kalman_with_scattering_equals_gls(n):
    rng = np.random.default_rng(7 + n)
    sigma, theta = 0.0159, 5e-4
    for _ in range(30):
        x, y, z = rand_track(rng, n)
        st = oracle.fit(x, y, z, sigma, theta, dtype=np.float64)
        sx, Cx, chx = gls_reference(z, x, sigma, theta)
        sy, Cy, chy = gls_reference(z, y, sigma, theta)
        np.testing.assert_allclose([st[8], st[10]], sx, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose([st[9], st[11]], sy, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose([st[12], st[13], st[14]], [Cx[0, 0], Cx[0, 1], Cx[1, 1]], rtol=1e-6, atol=1e-14)
        np.testing.assert_allclose([st[15], st[16], st[17]], [Cy[0, 0], Cy[0, 1], Cy[1, 1]], rtol=1e-6, atol=1e-14)
        np.testing.assert_allclose(st[7], chx + chy, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("delta", [0.01, 0.035, 0.05])
def test_three_point_chi2_closed_form(delta):
    """Points (z, x) = (0, 0), (42, delta), (84, 0): the fit line is x = delta/3,
    residuals (-1, 2, -1) delta/3, so chi2 = 2 delta^2 / (3 sigma^2)."""
    sigma = 0.0159
    z = Z[4:7]
    x = np.array([5.0, 5.0 + delta, 5.0])
    y = np.array([7.0, 7.0, 7.0])
    st = oracle.fit(x, y, z, sigma, 0.0, dtype=np.float64)
    np.testing.assert_allclose(st[6], 2 * delta ** 2 / (3 * sigma ** 2), rtol=1e-9)
    np.testing.assert_allclose(st[0], 5.0 + delta / 3, rtol=1e-12)
    assert abs(st[2]) < 1e-12


def test_z_beam_of_line_through_axis():
    rng = np.random.default_rng(3)
    for _ in range(50):
        zv = rng.uniform(-100, 100)
        tx, ty = rng.uniform(-0.2, 0.2, 2)
        z = Z[10:18]
        st = oracle.fit(tx * (z - zv), ty * (z - zv), z, 0.0159, 0.0, dtype=np.float64)
        np.testing.assert_allclose(st[5], zv, atol=1e-7)
        assert st[6] < 1e-18


def test_float32_close_to_float64():
    rng = np.random.default_rng(9)
    for n in (3, 6, 12, 20):
        for _ in range(30):
            x, y, z = rand_track(rng, n)
            a = oracle.fit(x, y, z, 0.0159, 5e-4, dtype=np.float64)
            b = oracle.fit(x.astype(np.float32), y.astype(np.float32), z.astype(np.float32), 0.0159, 5e-4)
            # positions ~30 mm (ulp 2e-6 mm); the closed-form sums lose a few more bits to
            # cancellation in S0*Sxz - Sz*Sx than the filter does (still < 1e-2 sigma)
            np.testing.assert_allclose(b[[0, 1]], a[[0, 1]], atol=1e-4)
            np.testing.assert_allclose(b[[8, 9]], a[[8, 9]], atol=2e-5)
            np.testing.assert_allclose(b[[2, 3, 10, 11]], a[[2, 3, 10, 11]], atol=2e-6)
            np.testing.assert_allclose(b[[12, 14, 15, 17]], a[[12, 14, 15, 17]], rtol=1e-3)
            np.testing.assert_allclose(b[[6, 7]], a[[6, 7]], rtol=1e-3, atol=1e-3)
