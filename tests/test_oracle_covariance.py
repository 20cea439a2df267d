"""Pins of the oracle's deformed Gaussian covariance F Sigma F^T (§3.1, §3.2)
against invariants: rotations keep the spectrum, det scales by J^2, a
diagonal stretch scales entries by s_i s_j, successive deformations compose,
and Sigma = (F R S)(F R S)^T for a kernel built from rotation and scales."""
import numpy as np

import oracle


def _rot(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _pack(S):
    return np.array([S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]])


def test_rotation_keeps_spectrum_and_stretch_scales_determinant():
    rng = np.random.default_rng(1)
    for _ in range(20):
        R0 = _rot(rng)
        s = rng.uniform(0.1, 2.0, 3)
        S0 = R0 @ np.diag(s ** 2) @ R0.T
        out = oracle.sym33(oracle.covariance(_rot(rng)[None], _pack(S0)[None]))[0]
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(out)), np.sort(s ** 2), rtol=1e-12)
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        out = oracle.sym33(oracle.covariance(F[None], _pack(S0)[None]))[0]
        np.testing.assert_allclose(np.linalg.det(out), np.linalg.det(F) ** 2 * np.prod(s ** 2), rtol=1e-10)
        np.testing.assert_allclose(out, out.T, atol=0)


def test_diagonal_stretch_and_composition():
    rng = np.random.default_rng(2)
    S0 = rng.standard_normal((3, 3))
    S0 = S0 @ S0.T
    d = np.array([1.5, 0.5, 2.0])
    out = oracle.sym33(oracle.covariance(np.diag(d)[None], _pack(S0)[None]))[0]
    np.testing.assert_allclose(out, S0 * np.outer(d, d), rtol=1e-14)
    F1, F2 = np.eye(3) + 0.2 * rng.standard_normal((2, 3, 3))
    once = oracle.covariance(F1[None], _pack(S0)[None])
    twice = oracle.covariance(F2[None], once)
    both = oracle.covariance((F2 @ F1)[None], _pack(S0)[None])
    np.testing.assert_allclose(twice, both, rtol=1e-12, atol=1e-15)


def test_kernel_from_rotation_and_scales():
    rng = np.random.default_rng(3)
    n = 32
    F = np.eye(3) + 0.1 * rng.standard_normal((n, 3, 3))
    Rs = np.array([_rot(rng) for _ in range(n)])
    sc = rng.uniform(0.01, 0.1, (n, 3))
    M = Rs * sc[:, None, :]
    S0 = np.array([_pack(m @ m.T) for m in M])
    FM = F @ M
    expect = FM @ FM.transpose(0, 2, 1)
    np.testing.assert_allclose(oracle.sym33(oracle.covariance(F, S0)), expect, rtol=1e-12, atol=1e-18)
