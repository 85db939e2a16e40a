"""Pins of the oracle's per-point-noise solve and of its voxel state machine (GS-LIVM,
arXiv 2410.17084, Sec. 3.3: types (a)-(d), variance feedback, convergence threshold eta)
against closed forms, an independent dense solve and the transition rules.

Mistakes each test is meant to catch: the noise of the wrong point on the diagonal, the
noise left in the kernel column of the input variance, a sign error in the posterior
variance, fed-back noise not replacing the sensor's, a converged voxel still solved, a
voxel below tau solved, the threshold compared with the wrong variance.
"""
import math

import numpy as np
import pytest

S = 0.5


def grid(G, s=S):
    return -s / 2 + (np.arange(G) + 0.5) * s / G


@pytest.mark.parametrize("mean_mode", [0, 1])
def test_repeated_input_closed_form(oracle, mean_mode):
    """n observations of f at one input x with noises d_i: a scalar Gaussian with prior
    variance sf2 observed n times, so the posterior at x has precision 1/sf2 + sum 1/d_i
    and mean m + V sum (f_i - m)/d_i.  A node u with c = k(u, x) sees
    f(u) = (c/sf2) f(x) + independent residual of variance sf2 - c^2/sf2."""
    lam, sf2 = 12.5, 0.8
    x = (0.0625, -0.09375)
    f = np.array([0.03125, -0.015625, 0.046875, 0.0078125, 0.0])
    d = np.array([4e-4, 1e-3, 2.5e-4, 7e-3, 5e-4])
    c0 = np.float32([0.25, 0.25, 0.25])
    P = np.stack([np.full(5, x[0]), np.full(5, x[1]), f], 1) + c0
    P = P.astype(np.float32)
    fl = P[:, 2].astype(np.float64) - c0[2]  # the targets as stored in FP32
    G = 6
    st, ax, mu, var, pvar = oracle.solve_voxel_hetero(P, c0, S, G, lam, sf2, d,
                                                      mean_mode=mean_mode, axis_override=2)
    assert st == 0 and ax == 2
    m = fl.mean() if mean_mode == 1 else 0.0
    V = 1.0 / (1.0 / sf2 + np.sum(1.0 / d))
    mx = m + V * np.sum((fl - m) / d)
    xl = (float(P[0, 0]) - c0[0], float(P[0, 1]) - c0[1])
    assert np.allclose(pvar, V, rtol=1e-10, atol=0)
    u = grid(G)
    for i in range(G):
        for j in range(G):
            c = sf2 * math.exp(-lam * ((xl[0] - u[i]) ** 2 + (xl[1] - u[j]) ** 2))
            a = c / sf2
            assert mu[i * G + j] == pytest.approx(m + a * (mx - m), rel=1e-10, abs=1e-14)
            assert var[i * G + j] == pytest.approx(sf2 - c * c / sf2 + a * a * V, rel=1e-10,
                                                   abs=1e-14)


def _quadric_voxel(rng, n):
    u = rng.uniform(-0.24, 0.24, size=(n, 2))
    h = 0.2 * u[:, 0] ** 2 - 0.1 * u[:, 0] * u[:, 1] + 0.05 * u[:, 1] + rng.normal(0, 0.01, n)
    c0 = np.float32([1.25, -0.75, 0.25])
    return (np.stack([u[:, 0], u[:, 1], h], 1) + c0).astype(np.float32), c0


def test_constant_noise_reduces_to_the_homoscedastic_solve(oracle):
    rng = np.random.default_rng(5)
    P, c0 = _quadric_voxel(rng, 40)
    G, lam, sf2, sn2 = 9, 12.5, 1.0, 4e-4
    st0, ax0, mu0, var0 = oracle.solve_voxel(P, c0, S, G, lam, sf2, sn2, mean_mode=1)
    st, ax, mu, var, pvar = oracle.solve_voxel_hetero(P, c0, S, G, lam, sf2,
                                                      np.full(40, sn2), mean_mode=1)
    assert st == st0 == 0 and ax == ax0
    assert np.allclose(mu, mu0, rtol=0, atol=1e-13)
    assert np.allclose(var, var0, rtol=1e-11, atol=1e-15)


def test_dense_solve_brute_force(oracle):
    """Posterior mean and variance at the nodes and at the inputs against a dense LU
    solve written here from Eq. 3 with A = K + diag(d)."""
    rng = np.random.default_rng(6)
    n = 30
    P, c0 = _quadric_voxel(rng, n)
    d = rng.uniform(1e-4, 5e-3, n)
    G, lam, sf2 = 5, 12.5, 1.3
    st, ax, mu, var, pvar = oracle.solve_voxel_hetero(P, c0, S, G, lam, sf2, d, mean_mode=1,
                                                      axis_override=2)
    assert st == 0
    X = P[:, :2].astype(np.float64) - c0[:2].astype(np.float64)
    f = P[:, 2].astype(np.float64) - float(c0[2])
    m = f.mean()
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    K = sf2 * np.exp(-lam * D2)
    A = K + np.diag(d)
    alpha = np.linalg.solve(A, f - m)
    pv = np.array([sf2 - K[i] @ np.linalg.solve(A, K[i]) for i in range(n)])
    assert np.allclose(pvar, pv, rtol=1e-9, atol=1e-15)
    assert np.all(pvar <= d * (1 + 1e-12)) and np.all(pvar >= 0)
    u = grid(G)
    for i in range(G):
        for j in range(G):
            k = sf2 * np.exp(-lam * ((X[:, 0] - u[i]) ** 2 + (X[:, 1] - u[j]) ** 2))
            assert mu[i * G + j] == pytest.approx(m + k @ alpha, rel=1e-9, abs=1e-13)
            assert var[i * G + j] == pytest.approx(sf2 - k @ np.linalg.solve(A, k), rel=1e-9,
                                                   abs=1e-13)


def test_smaller_noise_pulls_the_mean_toward_that_point(oracle):
    """Two points at one input: the posterior mean there moves toward the observation
    whose noise is smaller."""
    c0 = np.float32([0.25, 0.25, 0.25])
    P = (np.float32([[0, 0, 0.02], [0, 0, -0.02]]) + c0).astype(np.float32)
    G = 1  # the single node sits at the voxel centre, where the points are
    r1 = oracle.solve_voxel_hetero(P, c0, S, G, 12.5, 1.0, np.array([1e-4, 1e-2]), 0, 2)
    r2 = oracle.solve_voxel_hetero(P, c0, S, G, 12.5, 1.0, np.array([1e-2, 1e-4]), 0, 2)
    assert r1[2][0] > 0.015 and r2[2][0] < -0.015
    assert r1[4][0] == pytest.approx(r1[4][1])


def _plane_scan(rng, n, lo, hi, z=0.1):
    """n points of the plane z = const over [lo, hi]^2 (x, y), metres."""
    xy = rng.uniform(lo, hi, size=(n, 2))
    return np.concatenate([xy, np.full((n, 1), z) + rng.normal(0, 0.005, (n, 1))], 1).astype(np.float32)


def test_state_machine_transitions(oracle):
    """Types and feedback over three scans of a plane patch (0.5 m voxels):
    voxel (0,0,0) is covered everywhere (converges at its first solve), voxel (1,0,0)
    only along one edge strip (stays active), voxel (2,0,0) gets too few points (a)."""
    rng = np.random.default_rng(7)
    G, lam, sf2, sn2, tau, eta, floor = 9, 12.5, 1.0, 4e-4, 10, 0.3, 4e-6
    st = oracle.VoxelStore(0.5, max_points=64, sensor_var=sn2)
    full = _plane_scan(rng, 40, 0.01, 0.49)
    strip = np.concatenate([rng.uniform(0.51, 0.56, (20, 1)), rng.uniform(0.01, 0.49, (20, 1)),
                            np.full((20, 1), 0.1)], 1).astype(np.float32)
    few = np.float32([[1.2, 0.2, 0.1]] * 3)
    r = st.process_scan(np.concatenate([full, strip, few]), G, lam, sf2, tau, eta, floor)
    by = {x["key"]: x for x in r}
    a, b, c = by[(0, 0, 0)], by[(1, 0, 0)], by[(2, 0, 0)]
    assert [x["key"] for x in r] == [(0, 0, 0), (1, 0, 0), (2, 0, 0)]
    assert a["type_before"] == 1 and b["type_before"] == 1 and c["type_before"] == 0
    assert a["status"] == 0 and a["mean_var"] <= eta * sf2 and a["type_after"] == 3
    assert b["status"] == 0 and b["mean_var"] > eta * sf2 and b["type_after"] == 2
    assert c["status"] == 1 and c["type_after"] == 0
    # fed back: every stored point of a solved voxel carries its posterior variance
    for x in (a, b):
        nz = np.array(st.noise[x["key"]])
        assert np.array_equal(nz, np.maximum(x["pvar"].astype(np.float32), np.float32(floor)))
        assert np.all(nz < sn2)
    # second scan: more strip points, more points in the converged and the small voxel
    strip2 = np.concatenate([rng.uniform(0.56, 0.7, (25, 1)), rng.uniform(0.01, 0.49, (25, 1)),
                             np.full((25, 1), 0.1)], 1).astype(np.float32)
    few2 = np.float32([[1.3, 0.3, 0.1]] * 8)
    nz_b = list(st.noise[(1, 0, 0)])
    r = st.process_scan(np.concatenate([full[:5], strip2, few2]), G, lam, sf2, tau, eta, floor)
    by = {x["key"]: x for x in r}
    a, b, c = by[(0, 0, 0)], by[(1, 0, 0)], by[(2, 0, 0)]
    assert a["type_before"] == 3 and a["status"] == oracle.CONVERGED and a["type_after"] == 3
    assert b["type_before"] == 2 and b["status"] == 0
    # old points carry their fed-back variance, new ones the sensor's
    assert np.array_equal(b["noise"], np.array(nz_b + [float(np.float32(sn2))] * 25))
    assert c["type_before"] == 1 and c["status"] == 0  # 11 points now: solved
    # a converged voxel's points are stored all the same
    assert len(st.buckets[(0, 0, 0)]) == 45


def test_threshold_uses_mean_over_nodes(oracle):
    """The convergence test compares the mean of the G x G predicted variances with
    eta * sf2: doubling sf2 (kernel and threshold scale together) keeps the decision."""
    rng = np.random.default_rng(8)
    pts = _plane_scan(rng, 30, 0.01, 0.49)
    dec = []
    for sf2 in (1.0, 2.0):
        st = oracle.VoxelStore(0.5, max_points=64, sensor_var=4e-4 * sf2)
        r = st.process_scan(pts, 9, 12.5, sf2, 10, 0.3, 0.0)
        assert r[0]["mean_var"] == pytest.approx(float(np.mean(r[0]["var"])))
        dec.append((r[0]["type_after"], r[0]["mean_var"] / sf2))
    assert dec[0][0] == dec[1][0] and dec[0][1] == pytest.approx(dec[1][1], rel=1e-6)
