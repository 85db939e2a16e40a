"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics,
not by the oracle itself (GS-LIVM, arXiv 2410.17084, Sec. 3.1-3.2).

Each test targets a plausible mistake: a dropped noise term, a wrong sign, a swapped
parameter axis, a transposed factor, a wrong grid offset or a mis-sorted eigenpair.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

S = 0.5  # voxel side used by the synthetic configs


def grid(G, s=S):
    return -s / 2 + (np.arange(G) + 0.5) * s / G


def one_voxel(local, centre=(0.25, 0.25, 0.25)):
    c = np.asarray(centre, dtype=np.float32)
    return (np.asarray(local, dtype=np.float64) + c).astype(np.float32), c


# --------------------------------------------------------------------------
# Eq. 3 closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lam,sf2,sn2", [(12.5, 1.0, 4e-4), (1.0, 1.0, 1e-2), (50.0, 2.5, 0.3)])
def test_one_point_posterior(oracle, lam, sf2, sn2):
    """n = 1, zero prior mean: mu = sf2 k f1 / (sf2 + s2), var = sf2 - sf2^2 k^2/(sf2+s2)."""
    x1 = (0.0625, -0.125)
    f1 = 0.09375
    P, c = one_voxel([[x1[0], x1[1], f1]])
    G = 8
    st, ax, mu, var = oracle.solve_voxel(P, c, S, G, lam, sf2, sn2, mean_mode=0, axis_override=2)
    assert st == 0 and ax == 2
    u = grid(G)
    for i in range(G):
        for j in range(G):
            k = math.exp(-lam * ((x1[0] - u[i]) ** 2 + (x1[1] - u[j]) ** 2))
            mu_ref = sf2 * k * f1 / (sf2 + sn2)
            var_ref = sf2 - (sf2 * k) ** 2 / (sf2 + sn2)
            assert mu[i * G + j] == pytest.approx(mu_ref, rel=1e-12, abs=1e-15)
            assert var[i * G + j] == pytest.approx(var_ref, rel=1e-12, abs=1e-15)


def test_two_point_posterior(oracle):
    """n = 2: A^-1 = [[s+s2, -s r], [-s r, s+s2]] / ((s+s2)^2 - s^2 r^2)."""
    lam, sf2, sn2 = 12.5, 1.0, 4e-4
    xa, xb = (0.0, 0.0), (0.125, 0.0625)
    fa, fb = 0.03125, -0.015625
    P, c = one_voxel([[xa[0], xa[1], fa], [xb[0], xb[1], fb]])
    G = 4
    st, ax, mu, var = oracle.solve_voxel(P, c, S, G, lam, sf2, sn2, mean_mode=0, axis_override=2)
    assert st == 0
    r = math.exp(-lam * ((xa[0] - xb[0]) ** 2 + (xa[1] - xb[1]) ** 2))
    s = sf2
    det = (s + sn2) ** 2 - (s * r) ** 2
    Ainv = np.array([[s + sn2, -s * r], [-s * r, s + sn2]]) / det
    u = grid(G)
    for i in range(G):
        for j in range(G):
            k = np.array([sf2 * math.exp(-lam * ((x[0] - u[i]) ** 2 + (x[1] - u[j]) ** 2))
                          for x in (xa, xb)])
            assert mu[i * G + j] == pytest.approx(k @ Ainv @ np.array([fa, fb]), rel=1e-11,
                                                  abs=1e-15)
            assert var[i * G + j] == pytest.approx(sf2 - k @ Ainv @ k, rel=1e-11, abs=1e-15)


def _exact_posterior(x, f, q, lam, sf2, sn2, mean_mode):
    """Gauss-Jordan in exact rational arithmetic on the double-rounded Gram entries."""
    n = len(f)
    m = Fraction(0)
    if mean_mode == 1:
        m = sum(Fraction(v) for v in f) / n
    A = [[Fraction(sf2 * math.exp(-lam * ((x[i][0] - x[j][0]) ** 2 + (x[i][1] - x[j][1]) ** 2)))
          + (Fraction(sn2) if i == j else 0) for j in range(n)] for i in range(n)]
    inv = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv[col], inv[piv] = inv[piv], inv[col]
        p = A[col][col]
        A[col] = [v / p for v in A[col]]
        inv[col] = [v / p for v in inv[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                fct = A[r][col]
                A[r] = [a - fct * b for a, b in zip(A[r], A[col])]
                inv[r] = [a - fct * b for a, b in zip(inv[r], inv[col])]
    k = [Fraction(sf2 * math.exp(-lam * ((x[i][0] - q[0]) ** 2 + (x[i][1] - q[1]) ** 2)))
         for i in range(n)]
    fm = [Fraction(v) - m for v in f]
    mu = m + sum(k[i] * inv[i][j] * fm[j] for i in range(n) for j in range(n))
    var = Fraction(sf2) - sum(k[i] * inv[i][j] * k[j] for i in range(n) for j in range(n))
    return float(mu), float(var)


@pytest.mark.parametrize("n,mean_mode", [(1, 1), (2, 0), (3, 1), (4, 0), (4, 1)])
def test_brute_force_tiny_voxels(oracle, n, mean_mode):
    """Cholesky + substitutions against an exact rational inverse for n <= 4."""
    rng = np.random.default_rng(100 + n)
    lam, sf2, sn2 = 12.5, 1.0, 4e-4
    loc = rng.uniform(-0.25, 0.25, (n, 3)).astype(np.float32)
    P, c = one_voxel(loc, centre=(0.75, -0.25, 1.25))
    x = [(float(p[0]) - float(c[0]), float(p[1]) - float(c[1])) for p in P]
    f = [float(p[2]) - float(c[2]) for p in P]
    G = 3
    st, ax, mu, var = oracle.solve_voxel(P, c, S, G, lam, sf2, sn2, mean_mode=mean_mode,
                                         axis_override=2)
    u = grid(G)
    for i in range(G):
        for j in range(G):
            mref, vref = _exact_posterior(x, f, (u[i], u[j]), lam, sf2, sn2, mean_mode)
            assert mu[i * G + j] == pytest.approx(mref, rel=1e-10, abs=1e-13)
            assert var[i * G + j] == pytest.approx(vref, rel=1e-8, abs=1e-13)


# --------------------------------------------------------------------------
# Limits and invariants of the GP posterior
# --------------------------------------------------------------------------
def test_noise_to_zero_interpolates(oracle):
    """As sigma^2 -> 0 the posterior interpolates: mu(x_i) = f_i and var(x_i) = 0 at
    training points that sit exactly on query nodes."""
    G = 8
    u = grid(G)  # multiples of 1/32: exact in FP32
    rng = np.random.default_rng(7)
    idx = rng.choice(G * G, 12, replace=False)
    loc = np.array([[u[q // G], u[q % G], rng.uniform(-0.1, 0.1)] for q in idx])
    P, c = one_voxel(loc)
    st, ax, mu, var = oracle.solve_voxel(P, c, S, G, 12.5, 1.0, 1e-12, mean_mode=1,
                                         axis_override=2)
    assert st == 0
    f = P[:, 2].astype(np.float64) - float(c[2])
    for t, q in enumerate(idx):
        assert mu[q] == pytest.approx(f[t], abs=1e-7)
        assert var[q] == pytest.approx(0.0, abs=1e-9)


def test_variance_bounds_and_far_field(oracle):
    """0 <= var <= sf2 everywhere; far from all data (lambda d^2 >> 1) the posterior
    returns to the prior: mu -> m, var -> sf2."""
    rng = np.random.default_rng(3)
    n = 20
    loc = np.c_[rng.uniform(-0.25, -0.2, (n, 2)), rng.uniform(-0.05, 0.05, n)]
    P, c = one_voxel(loc)
    G = 10
    sf2 = 1.7
    st, ax, mu, var = oracle.solve_voxel(P, c, S, G, 800.0, sf2, 1e-3, mean_mode=1,
                                         axis_override=2)
    assert st == 0
    assert np.all(var >= 0) and np.all(var <= sf2 * (1 + 1e-12))
    m = np.mean(P[:, 2].astype(np.float64) - float(c[2]))
    far = G * G - 1  # node (+0.225, +0.225): distance > 0.4, lambda d^2 > 128
    assert mu[far] == pytest.approx(m, abs=1e-12)
    assert var[far] == pytest.approx(sf2, rel=1e-12)


def test_constant_targets_give_constant_mean(oracle):
    """With the data-mean prior, constant f makes f - m vanish and mu == m everywhere."""
    rng = np.random.default_rng(5)
    loc = np.c_[rng.uniform(-0.25, 0.25, (30, 2)), np.full(30, 0.0625)]
    P, c = one_voxel(loc)
    st, ax, mu, var = oracle.solve_voxel(P, c, S, 9, 12.5, 1.0, 4e-4, mean_mode=1,
                                         axis_override=2)
    assert np.allclose(mu, 0.0625, atol=1e-13, rtol=0)


def test_permutation_invariance(oracle):
    rng = np.random.default_rng(11)
    loc = np.c_[rng.uniform(-0.25, 0.25, (40, 2)), rng.uniform(-0.05, 0.05, 40)]
    P, c = one_voxel(loc)
    perm = rng.permutation(40)
    _, _, mu1, v1 = oracle.solve_voxel(P, c, S, 10, 12.5, 1.0, 4e-4)
    _, _, mu2, v2 = oracle.solve_voxel(P[perm], c, S, 10, 12.5, 1.0, 4e-4)
    assert np.allclose(mu1, mu2, rtol=0, atol=1e-12)
    assert np.allclose(v1, v2, rtol=1e-9, atol=1e-14)


def test_translation_invariance(oracle):
    """Moving the voxel and its points by whole voxels changes nothing (exact inputs)."""
    rng = np.random.default_rng(12)
    loc = np.round(np.c_[rng.uniform(-0.25, 0.25, (25, 2)), rng.uniform(-0.05, 0.05, 25)]
                   * 4096) / 4096
    P, c = one_voxel(loc)
    shift = np.float32([16.0, -8.0, 4.0])
    _, ax1, mu1, v1 = oracle.solve_voxel(P, c, S, 10, 12.5, 1.0, 4e-4)
    _, ax2, mu2, v2 = oracle.solve_voxel(P + shift, c + shift, S, 10, 12.5, 1.0, 4e-4)
    assert ax1 == ax2
    assert np.array_equal(mu1, mu2) and np.array_equal(v1, v2)


def test_axis_relabelling_consistency(oracle):
    """A surface valued along X with parameters (y, z) is the same regression as the
    surface valued along Z with parameters (x, y) (Alg. 1 switch cases X and Z)."""
    rng = np.random.default_rng(13)
    loc = np.c_[rng.uniform(-0.25, 0.25, (30, 2)), 0.02 * rng.standard_normal(30)]
    Pz, c = one_voxel(loc)
    # X-valued copy: x' = value, y' = first parameter, z' = second parameter
    Px = np.ascontiguousarray(Pz[:, [2, 0, 1]])
    cx = np.ascontiguousarray(c[[2, 0, 1]])
    Py = np.ascontiguousarray(Pz[:, [1, 2, 0]])  # Y-valued: (z', x') parameters
    cy = np.ascontiguousarray(c[[1, 2, 0]])
    sz = oracle.solve_voxel(Pz, c, S, 10, 12.5, 1.0, 4e-4)
    sx = oracle.solve_voxel(Px, cx, S, 10, 12.5, 1.0, 4e-4)
    sy = oracle.solve_voxel(Py, cy, S, 10, 12.5, 1.0, 4e-4)
    assert (sz[1], sx[1], sy[1]) == (2, 0, 1)
    for other in (sx, sy):
        assert np.allclose(sz[2], other[2], rtol=0, atol=1e-12)
        assert np.allclose(sz[3], other[3], rtol=1e-9, atol=1e-14)


def test_value_axis_is_normal_direction(oracle):
    rng = np.random.default_rng(14)
    for axis in range(3):
        loc = np.zeros((50, 3))
        p1, p2 = (axis + 1) % 3, (axis + 2) % 3
        loc[:, p1] = rng.uniform(-0.25, 0.25, 50)
        loc[:, p2] = rng.uniform(-0.25, 0.25, 50)
        loc[:, axis] = 0.2 * loc[:, p1] - 0.1 * loc[:, p2] + 0.01 * rng.standard_normal(50)
        P, c = one_voxel(loc)
        ax, nrm, ev = oracle.pca_axis(P)
        assert ax == axis
        assert np.argmax(np.abs(nrm)) == axis
        assert ev[0] < 1e-2 * ev[1]


def test_gram_spd_and_pivot_failure(oracle):
    """Cholesky succeeds on every synthetic Gram; a negative noise making the 1x1 Gram
    non-positive is reported as NOT_SPD."""
    from paper_2410_17084_b300 import synth
    b = synth.plane_batch(50, seed=9)
    out = oracle.solve_batch(b.xyz, b.offsets, b.centres, b.lam, b.sf2, b.sn2, b.size, b.G,
                             b.tau)
    assert np.all(out["status"] == 0)
    P, c = one_voxel([[0.0, 0.0, 0.0]])
    st, *_ = oracle.solve_voxel(P, c, S, 4, 12.5, 1.0, -1.5, axis_override=2)
    assert st == oracle.NOT_SPD


# --------------------------------------------------------------------------
# 3x3 eigen solver and Gaussian initialisation (Sec. 3.2, Eq. 5-8)
# --------------------------------------------------------------------------
def _smith_eigenvalues(A):
    """Trigonometric closed form for the eigenvalues of a symmetric 3x3 (Smith 1961)."""
    p1 = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
    q = np.trace(A) / 3
    p2 = (A[0, 0] - q) ** 2 + (A[1, 1] - q) ** 2 + (A[2, 2] - q) ** 2 + 2 * p1
    p = math.sqrt(p2 / 6)
    B = (A - q * np.eye(3)) / p
    r = np.linalg.det(B) / 2
    r = min(1.0, max(-1.0, r))
    phi = math.acos(r) / 3
    e1 = q + 2 * p * math.cos(phi)
    e3 = q + 2 * p * math.cos(phi + 2 * math.pi / 3)
    return sorted([e1, 3 * q - e1 - e3, e3])


def test_eig3_matches_closed_form(oracle):
    rng = np.random.default_rng(21)
    for _ in range(50):
        M = rng.standard_normal((3, 3))
        A = M @ M.T
        ev, V = oracle.eig3(A)
        assert np.allclose(sorted(ev), _smith_eigenvalues(A), rtol=1e-12, atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)
        assert np.allclose(A @ V, V * ev[None, :], atol=1e-11)


def test_init_planar_grid_closed_form(oracle):
    """Flat mean field, equal weights: each subgrid is an n_r x n_r planar lattice of
    spacing h, so Phi has eigenvalues h^2 (n_r^2 - 1) / 12 (twice) and 0."""
    n_s, n_r = 3, 3
    G = n_s * n_r
    h = S / G
    mean = np.full(G * G, 0.03)
    var = np.full(G * G, 2e-4)
    c = np.float32([0.25, 0.25, 0.25])
    pos, scale, quat, phi = oracle.init_voxel(mean, var, 2, c, S, G, n_s, n_r, 1.0)
    lam = h * h * (n_r * n_r - 1) / 12
    assert np.allclose(scale[:, 0], math.sqrt(lam), rtol=1e-12)
    assert np.allclose(scale[:, 1], math.sqrt(lam), rtol=1e-12)
    assert np.allclose(scale[:, 2], 1e-4 * S, rtol=1e-12)  # floored normal axis
    u = grid(G)
    for g in range(n_s * n_s):
        bi, bj = divmod(g, n_s)
        cx = u[bi * n_r:(bi + 1) * n_r].mean()
        cy = u[bj * n_r:(bj + 1) * n_r].mean()
        assert np.allclose(pos[g], [0.25 + cx, 0.25 + cy, 0.25 + 0.03], atol=1e-14)
        # normal (third column of R) along the value axis Z
        w, x, y, z = quat[g]
        R = _rot(quat[g])
        assert abs(abs(R[2, 2]) - 1) < 1e-12


def _rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_init_tilted_plane_recovers_rotation(oracle, axis):
    """Mean field mu = a u + b v on equal weights: Phi = c M^T M with M rows (1,0,a),
    (0,1,b) in (p1, p2, value) order, eigenvalues c (1 + a^2 + b^2), c and 0, and the
    normal (-a, -b, 1) / norm as the third rotation column."""
    n_s, n_r = 2, 4
    G = n_s * n_r
    a, b = 0.3, -0.7
    u = grid(G)
    mean = np.array([a * u[i] + b * u[j] for i in range(G) for j in range(G)])
    var = np.full(G * G, 1e-4)
    c = np.float32([0.25, -0.25, 0.75])
    pos, scale, quat, phi = oracle.init_voxel(mean, var, axis, c, S, G, n_s, n_r, 1.0)
    h = S / G
    cc = h * h * (n_r * n_r - 1) / 12
    p1, p2 = (axis + 1) % 3, (axis + 2) % 3
    nrm = np.zeros(3)
    nrm[p1], nrm[p2], nrm[axis] = -a, -b, 1.0
    nrm /= np.linalg.norm(nrm)
    for g in range(n_s * n_s):
        assert scale[g, 0] == pytest.approx(math.sqrt(cc * (1 + a * a + b * b)), rel=1e-11)
        assert scale[g, 1] == pytest.approx(math.sqrt(cc), rel=1e-11)
        assert scale[g, 2] == pytest.approx(1e-4 * S, rel=1e-12)
        R = _rot(quat[g])
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        assert abs(abs(R[:, 2] @ nrm) - 1) < 1e-12
        # round trip of Eq. 5 on the two unfloored axes
        S2 = np.diag([scale[g, 0] ** 2, scale[g, 1] ** 2, 0.0])
        assert np.allclose(R @ S2 @ R.T, phi[g], atol=1e-14)


def test_init_weight_scale_invariance(oracle):
    rng = np.random.default_rng(31)
    G, n_s, n_r = 9, 3, 3
    mean = rng.uniform(-0.05, 0.05, G * G)
    var = rng.uniform(1e-5, 1e-3, G * G)
    c = np.float32([1.25, 0.75, -0.25])
    o1 = oracle.init_voxel(mean, var, 1, c, S, G, n_s, n_r, 1.0)
    o2 = oracle.init_voxel(mean, var * 7.0, 1, c, S, G, n_s, n_r, 1.0)
    for x, y in zip(o1, o2):
        assert np.allclose(x, y, rtol=1e-10, atol=1e-15)


def test_init_weights_follow_inverse_variance(oracle):
    """Eq. 6: one node with a much smaller variance pulls the position onto itself."""
    G, n_s, n_r = 4, 1, 4
    mean = np.zeros(G * G)
    var = np.full(G * G, 1.0)
    var[5] = 1e-5  # node (1, 1)
    c = np.float32([0.25, 0.25, 0.25])
    pos, *_ = oracle.init_voxel(mean, var, 2, c, S, G, n_s, n_r, 1.0)
    u = grid(G)
    w = 1.0 / var
    ref = np.array([(w * np.repeat(u, G)).sum(), (w * np.tile(u, G)).sum()]) / w.sum()
    assert np.allclose(pos[0, :2] - 0.25, ref, atol=1e-15)
    assert abs(pos[0, 0] - 0.25 - u[1]) < 2e-5


def test_init_paper_mode(oracle):
    """init_mode 1 is Eq. 8 as printed: S = diag(Phi), R = identity."""
    rng = np.random.default_rng(32)
    G, n_s, n_r = 6, 2, 3
    mean = rng.uniform(-0.05, 0.05, G * G)
    var = rng.uniform(1e-5, 1e-3, G * G)
    c = np.float32([0.25, 0.25, 0.25])
    pos, scale, quat, phi = oracle.init_voxel(mean, var, 0, c, S, G, n_s, n_r, 1.0,
                                              init_mode=1)
    for g in range(n_s * n_s):
        assert np.array_equal(scale[g], np.diag(phi[g]))
        assert np.array_equal(quat[g], [1.0, 0.0, 0.0, 0.0])


# --------------------------------------------------------------------------
# ALG.HASH and ALG.STORE (supplementary Alg. 2)
# --------------------------------------------------------------------------
def test_voxel_keys_floor_in_fp32(oracle):
    xs = np.float32([0.0, 0.49999997, 0.5, -1e-7, -0.5, -0.50000006, 123.456, -77.25])
    xyz = np.stack([xs, -xs, xs * 3], 1).astype(np.float32)
    k = oracle.voxel_keys(xyz, 0.5)
    ref = np.floor(xyz / np.float32(0.5)).astype(np.int32)
    assert np.array_equal(k, ref)
    assert k[3, 0] == -1 and k[2, 0] == 1 and k[0, 0] == 0


def test_store_dedups_touched_and_caps_buckets(oracle):
    st = oracle.VoxelStore(0.5, max_points=5)
    pts = np.float32([[0.1, 0.1, 0.1]] * 7 + [[0.6, 0.1, 0.1]] + [[0.1, 0.1, 0.1]])
    touched = st.insert_scan(pts)
    assert touched == [(0, 0, 0), (1, 0, 0)]
    assert st.total[(0, 0, 0)] == 8 and len(st.buckets[(0, 0, 0)]) == 5
    touched2 = st.insert_scan(np.float32([[0.6, 0.1, 0.1], [-0.1, 0.1, 0.1]]))
    assert touched2 == [(1, 0, 0), (-1, 0, 0)]
