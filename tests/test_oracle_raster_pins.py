"""Pins of the oracle's Gaussian rasteriser (GS-LIVM Eq. 9: front-to-back alpha blending of
colour, plus depth and silhouette images) against closed forms and symmetries.

Mistakes each test is meant to catch: back-to-front blending, a missing transmittance
factor, the dilation 0.3 I left out, the quaternion read as (x, y, z, w), a transposed
projected covariance, the early-termination rule off by one Gaussian, no near-plane cull,
a depth key whose FP32 rounding (or wrong row of the camera rotation) misorders layers.
"""
import math

import numpy as np
import pytest

I3 = np.eye(3)
Z3 = np.zeros(3)


def _one(oracle, pos, scale, quat, op, col, W=33, H=33, f=40.0, near=0.2):
    return oracle.rasterize(np.float32([pos]).reshape(-1, 3), np.float32([scale]).reshape(-1, 3),
                            np.float32([quat]).reshape(-1, 4), np.float32(op).reshape(-1),
                            np.float32([col]).reshape(-1, 3), I3, Z3, f, f, W / 2, H / 2, W, H, near)


def test_single_gaussian_closed_form(oracle):
    z0, s, op, f = 2.0, 0.05, 0.8, 40.0
    C, D, S, amb = _one(oracle, [0, 0, z0], [s, s, s], [1, 0, 0, 0], op, [0.2, 0.5, 0.9])
    s, op = float(np.float32(s)), float(np.float32(op))  # the inputs are FP32
    a = (f * s / z0) ** 2 + 0.3  # projected variance per axis in pixels^2
    r = math.ceil(3 * math.sqrt(a))
    for (x, y) in [(16, 16), (17, 16), (16, 19), (14, 18), (16 + r - 1, 16)]:
        dx, dy = x + 0.5 - 16.5, y + 0.5 - 16.5
        al = min(0.99, op * math.exp(-0.5 * (dx * dx + dy * dy) / a))
        if al < 1 / 255:
            al = 0.0
        assert S[y, x] == pytest.approx(al, rel=1e-9, abs=1e-12)
        assert D[y, x] == pytest.approx(z0 * al, rel=1e-9, abs=1e-12)
        assert np.allclose(C[y, x], np.array([0.2, 0.5, 0.9], dtype=np.float32) * al, rtol=1e-6)


def test_three_sigma_square_cut(oracle):
    """Beyond the 3-sigma square nothing is drawn, though alpha would exceed 1/255 there."""
    z0, s, op, f, W = 2.0, 0.5, 0.99, 40.0, 71
    C, D, S, amb = _one(oracle, [0, 0, z0], [s, s, s], [1, 0, 0, 0], op, [1, 1, 1], W=W, H=W)
    a = (f * float(np.float32(s)) / z0) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(a))
    c = W / 2
    inside, outside = int(c + r - 1), int(c + r + 1)
    val = lambda x: float(np.float32(op)) * math.exp(-0.5 * (x + 0.5 - c) ** 2 / a)
    row = int(c)
    assert S[row, inside] == pytest.approx(val(inside), rel=1e-9)
    assert S[row, outside] == 0.0 and val(outside) > 1 / 255


def test_front_to_back_any_input_order(oracle):
    P = np.float32([[0, 0, 3.0], [0, 0, 2.0]])
    sc = np.float32([[0.2, 0.2, 0.2]] * 2)
    q = np.float32([[1, 0, 0, 0]] * 2)
    op = np.float32([0.9, 0.6])
    col = np.float32([[1, 0, 0], [0, 1, 0]])
    # principal point on the centre of pixel (16, 16)
    C1, D1, S1, _ = oracle.rasterize(P, sc, q, op, col, I3, Z3, 40, 40, 16.5, 16.5, 32, 32)
    C2, D2, S2, _ = oracle.rasterize(P[::-1], sc[::-1], q, op[::-1], col[::-1], I3, Z3, 40, 40, 16.5, 16.5, 32, 32)
    assert np.array_equal(C1, C2) and np.array_equal(D1, D2)
    # at the image centre both alphas are at their opacities: near (green, 0.6) first
    a_near, a_far = float(np.float32(0.6)), float(np.float32(0.9))
    assert np.allclose(C1[16, 16], [a_far * (1 - a_near), a_near, 0], rtol=0, atol=1e-12)
    assert S1[16, 16] == pytest.approx(a_near + a_far * (1 - a_near), abs=1e-12)


def test_early_termination_keeps_the_gaussian_at_the_threshold(oracle):
    """Opaque layers (alpha = 0.99): T goes 1 -> 0.01 -> 1e-4 (kept, not below) and
    stops before the third, so S = 0.99 + 0.99 * 0.01 exactly at a layer's centre."""
    P = np.float32([[0, 0, 2.0], [0, 0, 2.5], [0, 0, 3.0]])
    sc = np.float32([[0.5, 0.5, 0.5]] * 3)
    C, D, S, amb = oracle.rasterize(P, sc, np.float32([[1, 0, 0, 0]] * 3), np.float32([1, 1, 1]),
                                    np.float32([[1, 1, 1]] * 3), I3, Z3, 40, 40, 16.5, 16.5, 32, 32)
    assert S[16, 16] == pytest.approx(0.99 + 0.99 * 0.01, abs=1e-12)
    assert D[16, 16] == pytest.approx(2.0 * 0.99 + 2.5 * 0.99 * 0.01, abs=1e-12)


def test_near_plane_cull(oracle):
    C, D, S, amb = _one(oracle, [0, 0, 0.15], [0.05] * 3, [1, 0, 0, 0], 0.9, [1, 1, 1])
    assert S.max() == 0.0


def test_rotation_about_the_view_axis_transposes(oracle):
    """An elongated Gaussian turned 90 degrees about the optical axis (quaternion
    (cos 45, 0, 0, sin 45), w first) renders the transposed image."""
    a = _one(oracle, [0, 0, 2], [0.15, 0.03, 0.01], [1, 0, 0, 0], 0.9, [1, 1, 1], W=32, H=32)[2]
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    b = _one(oracle, [0, 0, 2], [0.15, 0.03, 0.01], [c, 0, 0, s], 0.9, [1, 1, 1], W=32, H=32)[2]
    assert a[16, 21] > 0.1 and a[21, 16] < 1e-3  # elongated along x before the turn
    assert np.allclose(b, a.T, atol=1e-7)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_depth_order_is_the_exact_depth_order(oracle, seed):
    """The order of blending is the order of the exact (FP64) camera depths, although the
    oracle sorts and culls on a depth key rounded to FP32: twenty Gaussians on the optical
    axis of a randomly turned and shifted camera, depths 0.01 apart (far above the key's
    rounding), given in random order.  At the centre pixel every alpha is the opacity 0.8,
    so T = 0.2^k after k layers and blending stops before the sixth (0.2^6 < 1e-4): the
    depth image there is sum_k z_(k) 0.8 0.2^k over the five nearest exact depths, a value
    that any other order of those five changes by more than 1e-4."""
    rng = np.random.default_rng(seed)
    Rc, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Rc) < 0:
        Rc[:, 0] = -Rc[:, 0]
    tc = rng.uniform(-2, 2, 3)
    z = 5.0 + 0.01 * rng.permutation(20)
    t = np.stack([np.zeros(20), np.zeros(20), z], axis=1)   # camera frame, on the axis
    P = np.float32((t - tc) @ Rc)                             # world points, rounded to FP32
    zx = P.astype(np.float64) @ Rc[2] + tc[2]                 # their exact camera depths
    sc = np.float32([[0.3, 0.3, 0.3]] * 20)
    q = np.float32([[1, 0, 0, 0]] * 20)
    op = np.float32([0.8] * 20)
    col = np.float32([[1, 1, 1]] * 20)
    W = H = 33
    C, D, S, amb = oracle.rasterize(P, sc, q, op, col, Rc, tc, 40, 40, W / 2, H / 2, W, H)
    a = float(np.float32(0.8))
    near5 = np.sort(zx)[:5]
    w = a * (1 - a) ** np.arange(5)
    assert amb[16, 16] == 0
    assert S[16, 16] == pytest.approx(w.sum(), abs=1e-9)
    assert D[16, 16] == pytest.approx(float(near5 @ w), abs=1e-9)
    # the same value from the shuffled inputs in another order
    perm = rng.permutation(20)
    _, D2, _, _ = oracle.rasterize(P[perm], sc, q, op, col, Rc, tc, 40, 40, W / 2, H / 2, W, H)
    assert D2[16, 16] == D[16, 16]
