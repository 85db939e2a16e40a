"""Pins of the oracle's full posterior covariance Sigma* of the query nodes (GS-LIVM,
arXiv 2410.17084, Eq. 3; the Sigma* that the supplementary Alg. 3 forms in full) against
closed forms and an independent dense computation.

Mistakes each test is meant to catch: a missing prior term k(x*_q, x*_q'), the two node
indices swapped (u/v), a missing transpose, the noise added to K**, a covariance that is
not symmetric or not positive semi-definite.
"""
import math

import numpy as np
import pytest

S = 0.5


def grid(G, s=S):
    return -s / 2 + (np.arange(G) + 0.5) * s / G


def _nodes(G):
    u = grid(G)
    return np.array([(u[i], u[j]) for i in range(G) for j in range(G)])


def test_one_point_closed_form(oracle):
    """n = 1: Sigma*_qr = sf2 e(q, r) - sf2^2 k_q k_r / (sf2 + sn2), with k_q the
    normalised kernel between node q and the point and e(q, r) that between two nodes."""
    lam, sf2, sn2, G = 12.5, 1.3, 4e-4, 4
    c0 = np.float32([0.25, 0.25, 0.25])
    x = (0.0625, -0.125)
    P = (np.float32([[x[0], x[1], 0.03125]]) + c0).astype(np.float32)
    st, ax, mu, cov = oracle.solve_voxel_fullcov(P, c0, S, G, lam, sf2, sn2, 0, 2)
    assert st == 0
    nd = _nodes(G)
    kq = np.exp(-lam * ((nd[:, 0] - x[0]) ** 2 + (nd[:, 1] - x[1]) ** 2))
    e = np.exp(-lam * ((nd[:, None, 0] - nd[None, :, 0]) ** 2 + (nd[:, None, 1] - nd[None, :, 1]) ** 2))
    ref = sf2 * e - sf2 ** 2 * np.outer(kq, kq) / (sf2 + sn2)
    assert np.allclose(cov, ref, rtol=1e-12, atol=1e-15)


def test_dense_brute_force_and_structure(oracle):
    rng = np.random.default_rng(11)
    n, G, lam, sf2, sn2 = 25, 5, 12.5, 1.0, 1e-3
    c0 = np.float32([-0.75, 0.25, 1.25])
    u = rng.uniform(-0.24, 0.24, (n, 2))
    h = 0.1 * u[:, 0] ** 2 + 0.03 * u[:, 1] + rng.normal(0, 0.01, n)
    P = (np.stack([u[:, 0], u[:, 1], h], 1) + c0).astype(np.float32)
    st, ax, mu, cov = oracle.solve_voxel_fullcov(P, c0, S, G, lam, sf2, sn2, 1, 2)
    assert st == 0
    X = P[:, :2].astype(np.float64) - c0[:2].astype(np.float64)
    nd = _nodes(G)
    K = sf2 * np.exp(-lam * ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    Ks = sf2 * np.exp(-lam * ((X[:, None, :] - nd[None, :, :]) ** 2).sum(-1))  # n x Q
    Kss = sf2 * np.exp(-lam * ((nd[:, None, :] - nd[None, :, :]) ** 2).sum(-1))
    ref = Kss - Ks.T @ np.linalg.solve(K + sn2 * np.eye(n), Ks)
    assert np.allclose(cov, ref, rtol=1e-9, atol=1e-12)
    assert np.allclose(cov, cov.T, rtol=0, atol=1e-14)
    assert np.linalg.eigvalsh(cov).min() > -1e-10
    # its diagonal is the variance of the diagonal-only solve
    st2, ax2, mu2, var2 = oracle.solve_voxel(P, c0, S, G, lam, sf2, sn2, 1, 2)
    assert np.allclose(np.diag(cov), var2, rtol=1e-12, atol=1e-15)
    assert np.allclose(mu, mu2, rtol=0, atol=1e-14)


def test_far_from_data_is_the_prior(oracle):
    """Points far outside the kernel's reach leave the prior covariance K**."""
    lam, sf2, sn2, G = 2000.0, 1.0, 4e-4, 3
    c0 = np.float32([0.25, 0.25, 0.25])
    P = (np.float32([[0.2499, 0.2499, 0.0], [-0.2499, 0.2499, 0.01]]) + c0).astype(np.float32)
    st, ax, mu, cov = oracle.solve_voxel_fullcov(P, c0, S, G, lam, sf2, sn2, 0, 2)
    nd = _nodes(G)
    Kss = sf2 * np.exp(-lam * ((nd[:, None, :] - nd[None, :, :]) ** 2).sum(-1))
    # the node nearest a point (0.1667, 0.1667) is 0.083 m away: k ~ exp(-2000 * 0.0139)
    assert np.allclose(cov, Kss, rtol=0, atol=1e-10)
    assert math.isclose(cov[0, 0], sf2)
