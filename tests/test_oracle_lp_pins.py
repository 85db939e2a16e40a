"""Pins of the oracle's structure similarity loss (GS-LIVM, arXiv 2410.17084, Eq. 11):
L_p = mean over scan points of min_k (|P_j - p_k| - mean(S_k)).

Mistakes each test is meant to catch: the minimum taken over the distance alone (the
text's "nearest Gaussian") instead of over distance minus mean scale, the scale's sum
instead of its mean, a squared distance, a sum instead of a mean.
"""
import numpy as np
import pytest
from scipy.spatial.distance import cdist


def test_single_gaussian_closed_form(oracle):
    P = np.float32([[1, 2, 2], [0, 0, 0], [3, 4, 0]])
    loss, best, arg = oracle.structure_loss(P, np.float32([[0, 0, 0]]), np.float32([[0.3, 0.6, 0.9]]))
    assert np.allclose(best, [3 - 0.6, -0.6, 5 - 0.6], atol=1e-7)
    assert loss == pytest.approx((2.4 - 0.6 + 4.4) / 3, abs=1e-7)
    assert np.all(arg == 0)


def test_larger_scale_wins_over_nearer_centre(oracle):
    """A farther Gaussian with a larger mean scale gives the smaller value."""
    P = np.float32([[0, 0, 0]])
    g = np.float32([[1, 0, 0], [2, 0, 0]])
    s = np.float32([[0.1, 0.1, 0.1], [1.5, 1.5, 1.5]])
    loss, best, arg = oracle.structure_loss(P, g, s)
    assert arg[0] == 1 and best[0] == pytest.approx(0.5, abs=1e-7)


def test_brute_force_matches_dense_distances(oracle):
    rng = np.random.default_rng(21)
    P = rng.uniform(-5, 5, (300, 3)).astype(np.float32)
    g = rng.uniform(-5, 5, (400, 3)).astype(np.float32)
    s = rng.uniform(0, 0.3, (400, 3)).astype(np.float32)
    loss, best, arg = oracle.structure_loss(P, g, s)
    V = cdist(P.astype(np.float64), g.astype(np.float64)) - s.astype(np.float64).mean(1)[None, :]
    assert np.allclose(best, V.min(1), rtol=0, atol=1e-12)
    assert np.array_equal(arg, V.argmin(1))
    assert loss == pytest.approx(V.min(1).mean(), rel=1e-12)


def test_scale_covariance(oracle):
    """Scaling every coordinate and every Gaussian scale by c scales L_p by c."""
    rng = np.random.default_rng(22)
    P = rng.uniform(-1, 1, (50, 3)).astype(np.float32)
    g = rng.uniform(-1, 1, (60, 3)).astype(np.float32)
    s = rng.uniform(0, 0.1, (60, 3)).astype(np.float32)
    l1 = oracle.structure_loss(P, g, s)[0]
    l4 = oracle.structure_loss(P * 4, g * 4, s * 4)[0]
    assert l4 == pytest.approx(4 * l1, rel=1e-6)
