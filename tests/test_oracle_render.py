"""Pins of the oracle's Gaussian splatting (§3.1): the projected covariance
of an isotropic Gaussian against its closed form (f s / z)^2 + 0.3, front-to-
back compositing of two Gaussians on one ray, invariance to the input order,
invisibility of transparent and behind-camera Gaussians, the 90-degree roll
of the camera rolling the image, and the transmittance cut-off."""
import math

import numpy as np

import oracle

F, W = 100.0, 64
VIEW = np.array([[1.0, 0, 0, -0.5], [0, 1.0, 0, -0.5], [0, 0, 1.0, 2.0]])   # camera 2 units in front of (0.5, 0.5, 0)


def iso(s2):
    return [s2, 0, 0, s2, 0, s2]


def test_isotropic_gaussian_profile():
    s2 = 4e-4
    z = 2.5                                    # camera depth of a point at world z = 0.5
    sig2 = (F * math.sqrt(s2) / z) ** 2 + 0.3
    o = 0.7
    img, T = oracle.render([[0.5, 0.5, 0.5]], [iso(s2)], [[1.0, 0.5, 0.25]], [o], VIEW, F, F, 31.5, 31.5, W, W)
    # the projected centre sits on pixel (31, 31)'s centre
    assert abs(img[31, 31, 0] - o) < 1e-14 and abs(T[31, 31] - (1 - o)) < 1e-14
    for dpx in (1, 2, 3):
        a = o * math.exp(-0.5 * dpx * dpx / sig2)
        if a >= 1 / 255:
            assert abs(img[31, 31 + dpx, 0] - a) < 1e-12
            assert abs(img[31 + dpx, 31, 1] - 0.5 * a) < 1e-12


def test_front_to_back_compositing_and_order():
    mean = [[0.5, 0.5, 0.5], [0.5, 0.5, 0.2]]          # the second is farther (camera depth 2.2 vs 2.5?)
    # camera depth = z + 2: the second Gaussian (z = 0.2) is nearer (2.2) than the first (2.5)
    col = [[1, 0, 0], [0, 1, 0]]
    op = [0.6, 0.5]
    cov = [iso(1e-4), iso(1e-4)]
    bg = (0.0, 0.0, 1.0)
    img, _ = oracle.render(mean, cov, col, op, VIEW, F, F, 31.5, 31.5, W, W, bg)
    a_near, a_far = 0.5, 0.6
    expect = np.array([0.0, a_near, 0.0]) + (1 - a_near) * np.array([a_far, 0.0, 0.0]) + (1 - a_near) * (1 - a_far) * np.array(bg)
    np.testing.assert_allclose(img[31, 31], expect, atol=1e-14)
    img2, _ = oracle.render(mean[::-1], cov[::-1], col[::-1], op[::-1], VIEW, F, F, 31.5, 31.5, W, W, bg)
    np.testing.assert_array_equal(img, img2)


def test_transparent_and_hidden_gaussians_leave_the_background():
    rng = np.random.default_rng(0)
    mean = 0.3 + 0.4 * rng.random((50, 3))
    cov = [iso(2e-4)] * 50
    col = rng.random((50, 3))
    bg = (0.2, 0.3, 0.4)
    img, T = oracle.render(mean, cov, col, np.zeros(50), VIEW, F, F, 32, 32, W, W, bg)
    assert np.all(img == np.array(bg)) and np.all(T == 1.0)
    behind = mean.copy()
    behind[:, 2] = -1.9                                # camera depth 0.1 < 0.2
    img, T = oracle.render(behind, cov, col, np.ones(50) * 0.9, VIEW, F, F, 32, 32, W, W, bg)
    assert np.all(T == 1.0)


def test_camera_roll_rolls_the_image():
    rng = np.random.default_rng(1)
    n = 40
    mean = 0.35 + 0.3 * rng.random((n, 3))
    A = rng.standard_normal((n, 3, 3)) * 0.01
    S = A @ A.transpose(0, 2, 1) + 1e-5 * np.eye(3)
    cov = np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)
    col = rng.random((n, 3))
    op = rng.uniform(0.2, 0.9, n)
    img, _ = oracle.render(mean, cov, col, op, VIEW, F, F, 32, 32, W, W)
    # roll the camera by +90 degrees about its optical axis: (x, y) -> (-y, x) in camera coordinates
    Rz = np.array([[0, -1.0, 0], [1.0, 0, 0], [0, 0, 1.0]])
    v2 = np.concatenate([Rz @ VIEW[:, :3], (Rz @ VIEW[:, 3])[:, None]], 1)
    img2, _ = oracle.render(mean, cov, col, op, v2, F, F, 32, 32, W, W)
    # camera-frame point (x, y) -> (-y, x): pixel (row r, col c) -> (row c, col W-1-r)
    np.testing.assert_allclose(img2, np.rot90(img, k=-1), atol=1e-12)


def test_transmittance_cut_off():
    # three opaque Gaussians on one ray: alpha clamps to 0.99; after two the
    # transmittance is 1e-4, and the third would take it to 1e-6 < 1e-4, so
    # the pixel stops before the third
    mean = [[0.5, 0.5, 0.5], [0.5, 0.5, 0.6], [0.5, 0.5, 0.7]]
    img, T = oracle.render(mean, [iso(1e-4)] * 3, [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [1.0, 1.0, 1.0], VIEW, F, F,
                           31.5, 31.5, W, W)
    np.testing.assert_allclose(img[31, 31], [0.99, 0.99 * 0.01, 0.0], atol=1e-14)
    assert abs(T[31, 31] - 1e-4) < 1e-15


def test_order_ambiguity_bound_is_the_swap_of_two_layers():
    """Two Gaussians at exactly the same camera depth on one ray: ties keep
    the input order, so giving them in both orders composites both orders.
    The two images differ by alpha_1 alpha_2 (col_1 - col_2) per channel in
    front of full transmittance, the transmittance is the same, and the
    ambiguity bound at that pixel is the largest channel of that difference."""
    mean = [[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]]
    col = [[1.0, 0.2, 0.0], [0.0, 0.6, 0.3]]
    op = [0.6, 0.5]
    cov = [iso(1e-4), iso(2e-4)]
    bg = (0.1, 0.1, 0.1)
    a, Ta, amb = oracle.render(mean, cov, col, op, VIEW, F, F, 31.5, 31.5, W, W, bg, tie_eps=2.0 ** -21)
    b, Tb, _ = oracle.render(mean[::-1], cov[::-1], col[::-1], op[::-1], VIEW, F, F, 31.5, 31.5, W, W, bg,
                             tie_eps=2.0 ** -21)
    a1, a2 = 0.6, 0.5                       # both centred on pixel (31, 31)
    np.testing.assert_allclose(a[31, 31] - b[31, 31], a1 * a2 * (np.array(col[0]) - np.array(col[1])), atol=1e-14)
    np.testing.assert_allclose(Ta, Tb, atol=1e-15)
    assert abs(amb[31, 31] - a1 * a2 * 1.0) < 1e-14
    # wherever the two orders differ, the bound covers the difference
    diff = np.abs(a - b).max(axis=2)
    assert np.all(diff <= amb + 1e-14) and amb.max() > 0
    # without a tolerance the bound is off and the image is unchanged
    c, _ = oracle.render(mean, cov, col, op, VIEW, F, F, 31.5, 31.5, W, W, bg)
    np.testing.assert_array_equal(a, c)


def test_order_ambiguity_bound_at_the_near_plane():
    """A Gaussian whose camera depth is the near plane itself (0.2) may be
    drawn or not by an implementation that rounds its depth: the bound at
    its centre is its alpha in front of full transmittance; distinct depths
    far apart give no bound."""
    near = [[0.5, 0.5, -1.8]]               # camera depth exactly 0.2
    img, T, amb = oracle.render(near, [iso(1e-6)], [[1.0, 1.0, 1.0]], [0.7], VIEW, F, F, 31.5, 31.5, W, W,
                                tie_eps=2.0 ** -21)
    assert np.all(T == 1.0)                 # t_z > 0.2 is false: not drawn
    assert abs(amb[31, 31] - 0.7) < 1e-14
    far = [[0.5, 0.5, 0.5], [0.5, 0.5, 0.1]]
    _, _, amb2 = oracle.render(far, [iso(1e-4)] * 2, [[1, 0, 0], [0, 1, 0]], [0.6, 0.5], VIEW, F, F, 31.5, 31.5, W,
                               W, tie_eps=2.0 ** -21)
    assert np.all(amb2 == 0.0)
