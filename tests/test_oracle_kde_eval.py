"""Pins of the oracle's density estimate, Eq. (1) with the Gaussian kernel of Eq. (2),
against facts outside it: a library density, moments and integrals of fhat, the
convolution identity for the integral of fhat^2, and a 40-digit brute force."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
import synthdata


def _trapz(y, x):
    return float(np.sum((y[1:] + y[:-1]) * np.diff(x)) / 2.0)


def test_single_point_is_the_normal_density():
    from scipy.stats import norm
    t = np.linspace(-4.0, 6.0, 41)
    got = oracle.kde_eval([1.25], 0.7, t)
    assert np.allclose(got, norm.pdf(t, loc=1.25, scale=0.7), rtol=1e-14, atol=0)


def test_matches_scipy_gaussian_kde():
    from scipy.stats import gaussian_kde
    x = synthdata.normal_mixture(11, 300, [0.4, 0.6], [-1.0, 2.0], [0.5, 1.0])
    h = 0.37
    # gaussian_kde's kernel has standard deviation factor * std(x, ddof=1)
    kde = gaussian_kde(x, bw_method=h / np.std(x, ddof=1))
    t = np.linspace(-4.0, 6.0, 77)
    assert np.allclose(oracle.kde_eval(x, h, t), kde(t), rtol=1e-11, atol=0)


def test_integrates_to_one_with_the_sample_mean_and_inflated_variance():
    x = synthdata.student_t3(12, 200)
    h = 0.45
    t = np.linspace(x.min() - 14 * h, x.max() + 14 * h, 400001)
    f = oracle.kde_eval(x, h, t)
    assert abs(_trapz(f, t) - 1.0) < 1e-9
    mean = _trapz(t * f, t)
    assert abs(mean - x.mean()) < 1e-7 * (1 + abs(x.mean()))
    var = _trapz((t - x.mean()) ** 2 * f, t)
    assert abs(var - (np.mean((x - x.mean()) ** 2) + h * h)) < 1e-6 * var


def test_integral_of_square_is_a_pair_sum():
    """int fhat^2 = n^-2 sum_ij phi_{h sqrt 2}(X_i - X_j): Gaussians convolve."""
    x = synthdata.normal(13, 60) * 1.3
    h = 0.3
    t = np.linspace(x.min() - 12 * h, x.max() + 12 * h, 200001)
    lhs = _trapz(oracle.kde_eval(x, h, t) ** 2, t)
    s = h * math.sqrt(2.0)
    d = x[:, None] - x[None, :]
    rhs = np.exp(-0.5 * (d / s) ** 2).sum() / (s * math.sqrt(2 * math.pi)) / x.size ** 2
    assert abs(lhs - rhs) < 1e-9 * rhs


def test_brute_force_40_digits():
    mp.mp.dps = 40
    x = synthdata.uniform(14, 9) * 3.0
    t = [-0.5, 0.1, 1.7, 3.3]
    h = 0.21
    got = oracle.kde_eval(x, h, t)
    for j, tj in enumerate(t):
        ref = mp.fsum(mp.npdf(mp.mpf(tj), mu=mp.mpf(xi), sigma=mp.mpf(h)) for xi in x) / len(x)
        assert abs(got[j] - float(ref)) <= 1e-15 * float(ref) + 1e-300


def test_thread_count_does_not_change_bits():
    x = synthdata.normal(15, 5000)
    t = np.linspace(-3, 3, 333)
    a = oracle.kde_eval(x, 0.2, t, threads=1)
    b = oracle.kde_eval(x, 0.2, t, threads=7)
    assert np.array_equal(a, b)


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.kde_eval([1.0], 0.0, [0.0])
    with pytest.raises(ValueError):
        oracle.kde_eval([], 1.0, [0.0])
