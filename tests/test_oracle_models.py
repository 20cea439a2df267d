"""Pins of the oracle's further constitutive models (App. A, App. B.1,
App. B.2): each Kirchhoff stress equals P F^T with P the central difference of
its strain energy, the stress is frame-indifferent and zero at rest, and the
volume-only plasticity models keep or clamp det F."""
import numpy as np
import pytest

import oracle

MU, LAM = 1.3e3, 2.1e3


def energy(model, F, mu, lam):
    J = np.linalg.det(F)
    if model == 2:
        E = 0.5 * (F.T @ F - np.eye(3))
        return mu * np.sum(E * E) + 0.5 * lam * (J - 1) ** 2
    if model == 3:
        eps = np.log(np.linalg.svd(F, compute_uv=False))
        return mu * np.sum(eps ** 2) + 0.5 * lam * np.sum(eps) ** 2
    if model == 4:
        return 0.5 * lam * (J - 1) ** 2
    if model == 5:
        kappa = 2 * mu / 3 + lam
        return kappa * (J + 1 / J - 2)
    raise ValueError(model)


def fd_piola(model, F, h=1e-6):
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, j] += h
            Fm[i, j] -= h
            P[i, j] = (energy(model, Fp, MU, LAM) - energy(model, Fm, MU, LAM)) / (2 * h)
    return P


def rand_F(rng, scale=0.25):
    while True:
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        if np.linalg.det(F) > 0.3:
            return F


@pytest.mark.parametrize("model", [2, 3, 4, 5])
def test_stress_is_the_energy_derivative(model):
    rng = np.random.default_rng(10 + model)
    for _ in range(10):
        F = rand_F(rng)
        tau = oracle.kirchhoff(model, F, MU, LAM)
        ref = fd_piola(model, F) @ F.T
        assert np.abs(tau - ref).max() < 1e-6 * max(np.abs(ref).max(), 1.0)
        np.testing.assert_allclose(tau, tau.T, atol=1e-9 * np.abs(tau).max())


@pytest.mark.parametrize("model", [2, 3, 4, 5])
def test_rest_and_frame_indifference_and_linearity(model):
    assert np.abs(oracle.kirchhoff(model, np.eye(3), MU, LAM)).max() < 1e-12
    rng = np.random.default_rng(20 + model)
    F = rand_F(rng)
    A = rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(A)
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    t = oracle.kirchhoff(model, F, MU, LAM)
    np.testing.assert_allclose(oracle.kirchhoff(model, Q @ F, MU, LAM), Q @ t @ Q.T, atol=1e-9 * np.abs(t).max())
    t2 = oracle.kirchhoff(model, F, 2 * MU, 0.0) + oracle.kirchhoff(model, F, 0.0, 2 * LAM)
    np.testing.assert_allclose(t2, 2 * t, atol=1e-9 * np.abs(t).max())


def test_fluid_plasticity_keeps_volume():
    rng = np.random.default_rng(30)
    for _ in range(10):
        F = rand_F(rng, 0.4)
        Fn, case = oracle.return_map(3, F, MU, LAM, 0.0, 30.0)
        c = np.linalg.det(F) ** (1 / 3)
        np.testing.assert_allclose(Fn, c * np.eye(3), rtol=1e-14)
        assert oracle.return_map(3, Fn, MU, LAM, 0.0, 30.0)[0] == pytest.approx(Fn, rel=1e-14)


@pytest.mark.parametrize("J,expect", [(2.0, 1.2), (1.1, 1.1), (0.8, 0.8), (0.01, 0.05)])
def test_sigma_plasticity_clamps_volume(J, expect):
    rng = np.random.default_rng(31)
    F = rand_F(rng)
    F *= (J / np.linalg.det(F)) ** (1 / 3)
    Fn, _ = oracle.return_map(4, F, MU, LAM, 0.0, 30.0)
    np.testing.assert_allclose(Fn, expect ** (1 / 3) * np.eye(3), rtol=1e-12)
