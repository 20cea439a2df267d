"""Pins of the oracle's BGDO stage 2 (§4.3, Algorithm 1, App. F) against
closed forms: the stress-gradient of a model linear in E, central differences
through the Lame map, rest and rigid-rotation key frames, the fixed-weight
limits and the per-material average."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _cloud(n, seed, spread=0.06):
    rng = np.random.default_rng(seed)
    return 0.5 + spread * (rng.random((n, 3)) - 0.5) * 2


def _mat(n, E, elastic=0, plastic=0, nu=0.3):
    return oracle.Material(np.full(n, (1 / 64) ** 3), 100.0, np.log(E), nu, 1e3, 30.0, elastic, plastic)


@pytest.mark.parametrize("elastic", [0, 1])
def test_stress_gradient_equals_stress_norm(elastic):
    # tau is linear in (mu, lambda) and both scale with E at fixed nu (App. B.1),
    # so d|tau|/dlogE = |tau| exactly.
    rng = np.random.default_rng(3 + elastic)
    n = 40
    F = np.eye(3) + 0.1 * rng.standard_normal((n, 3, 3))
    s = oracle.new_state(_cloud(n, 1), F=F)
    m = _mat(n, np.exp(rng.uniform(np.log(1e3), np.log(1e6), n)), elastic)
    r = oracle.bgdo(oracle.Cfg(32, 1 / 32, 1e-5), [s], m, delta_pre_step=True)
    norms = []
    for p in range(n):
        mu, lam = oracle.lame(np.exp(m.logE[p]), 0.3)
        norms.append(np.linalg.norm(oracle.kirchhoff(elastic, F[p], mu, lam)))
    np.testing.assert_allclose(r["g_tau"][0], norms, rtol=1e-12)


@pytest.mark.parametrize("elastic", [0, 1])
def test_stress_gradient_matches_central_difference(elastic):
    rng = np.random.default_rng(11)
    F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    if np.linalg.det(F) < 0.2:
        F[:, 0] *= -1
    nu, logE, h = 0.27, np.log(4.2e4), 1e-5

    def snorm(le):
        mu, lam = oracle.lame(np.exp(le), nu)
        return np.linalg.norm(oracle.kirchhoff(elastic, F, mu, lam))
    fd = (snorm(logE + h) - snorm(logE - h)) / (2 * h)
    s = oracle.new_state(_cloud(1, 2), F=F[None])
    m = _mat(1, np.exp(logE), elastic, nu=nu)
    r = oracle.bgdo(oracle.Cfg(32, 1 / 32, 1e-5), [s], m, delta_pre_step=True)
    assert abs(r["g_tau"][0, 0] - fd) <= 1e-7 * abs(fd)


def test_rest_state_gives_the_deformation_target_term_only():
    # F = I, uniform velocity, no gravity, away from walls: tau = 0, F' = I, so
    # G = -(1 - eta)(0 - delta_target) with eta = 0.1 log(1 + E) for E < e^10.
    n = 64
    E = 1e3
    s = oracle.new_state(_cloud(n, 5), v=np.tile([0.3, -0.2, 0.1], (n, 1)))
    cfg = oracle.Cfg(32, 1 / 32, 1e-4, gravity=(0, 0, 0))
    r = oracle.bgdo(cfg, [s, s, s], _mat(n, E))
    eta = 0.1 * np.log(1 + E)
    assert np.all(r["g_tau"] == 0)
    assert np.max(np.abs(r["delta"])) < 1e-12
    np.testing.assert_allclose(r["G"], 0.1 * (1 - eta), rtol=1e-10)
    np.testing.assert_allclose(r["log_E"], np.log(E) - 0.1 * (1 - eta), rtol=1e-12)


def test_rigid_rotation_key_frame():
    # F = R, v = w x (x - c), C = [w]_x: fixed-corotated tau = 0 and one substep
    # reproduces C, so F' = (I + dt [w]_x) R and delta = |F' - I|_F.
    n = 80
    rng = np.random.default_rng(8)
    x = _cloud(n, 9)
    c = np.array([0.5, 0.5, 0.5])
    w = np.array([1.5, -2.0, 0.7])
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, cq, d = q
    R = np.array([[a * a + b * b - cq * cq - d * d, 2 * (b * cq - a * d), 2 * (b * d + a * cq)],
                  [2 * (b * cq + a * d), a * a - b * b + cq * cq - d * d, 2 * (cq * d - a * b)],
                  [2 * (b * d - a * cq), 2 * (cq * d + a * b), a * a - b * b - cq * cq + d * d]])
    s = oracle.new_state(x, v=(x - c) @ W.T, C=np.tile(W, (n, 1, 1)), F=np.tile(R, (n, 1, 1)))
    dt = 1e-3
    cfg = oracle.Cfg(32, 1 / 32, dt, gravity=(0, 0, 0))
    r = oracle.bgdo(cfg, [s], _mat(n, 5e3), w=0.25)
    expect = np.linalg.norm((np.eye(3) + dt * W) @ R - np.eye(3))
    assert np.max(np.abs(r["g_tau"])) < 1e-8
    np.testing.assert_allclose(r["delta"][0], expect, rtol=1e-9)
    np.testing.assert_allclose(r["G"], 0.25 * np.log1p(np.abs(r["g_tau"][0])) - 0.75 * (expect - 0.1), rtol=1e-9)


def test_fixed_weights_select_one_signal_and_keys_average():
    n = 48
    rng = np.random.default_rng(21)
    cfg = oracle.Cfg(32, 1 / 32, 1e-4)
    keys = [oracle.new_state(_cloud(n, 30 + k), v=0.2 * rng.standard_normal((n, 3)),
                             F=np.eye(3) + 0.05 * rng.standard_normal((n, 3, 3))) for k in range(3)]
    m = _mat(n, 2e4)
    r1 = oracle.bgdo(cfg, keys, m, w=1.0)
    r0 = oracle.bgdo(cfg, keys, m, w=0.0)
    np.testing.assert_allclose(r1["G"], np.mean(np.log1p(r1["g_tau"]), axis=0), rtol=1e-12)
    np.testing.assert_allclose(r0["G"], -np.mean(r0["delta"] - 0.1, axis=0), rtol=1e-12, atol=1e-15)
    # key frames are independent pseudo steps: the mean of single-key updates
    single = [oracle.bgdo(cfg, [k], m)["G"] for k in keys]
    np.testing.assert_allclose(oracle.bgdo(cfg, keys, m)["G"], np.mean(single, axis=0), rtol=1e-12)
    # the pre-step reading measures the key frame's own F
    rp = oracle.bgdo(cfg, keys, m, delta_pre_step=True)
    np.testing.assert_allclose(rp["delta"][1], np.linalg.norm(keys[1]["F"] - np.eye(3), axis=(1, 2)), rtol=1e-13)


def test_eta_saturates_for_stiff_materials():
    # E > e^10: eta = 1 and G = log(1 + |tau|) > 0 (stiffness is reduced)
    n = 16
    rng = np.random.default_rng(4)
    s = oracle.new_state(_cloud(n, 3), F=np.eye(3) + 0.02 * rng.standard_normal((n, 3, 3)))
    r = oracle.bgdo(oracle.Cfg(32, 1 / 32, 1e-6), [s], _mat(n, 3e8), delta_pre_step=True)
    np.testing.assert_allclose(r["G"], np.log1p(r["g_tau"][0]), rtol=1e-12)
    assert np.all(r["G"] > 0)


def test_per_material_average():
    n = 60
    rng = np.random.default_rng(6)
    s = oracle.new_state(_cloud(n, 7), F=np.eye(3) + 0.05 * rng.standard_normal((n, 3, 3)))
    label = rng.integers(0, 3, n)
    m = _mat(n, np.exp(rng.uniform(7, 11, n)))
    cfg = oracle.Cfg(32, 1 / 32, 1e-4)
    per_p = oracle.bgdo(cfg, [s], m)["G"]
    per_m = oracle.bgdo(cfg, [s], m, label=label, per_material=True)["G"]
    for k in range(3):
        np.testing.assert_allclose(per_m[label == k], per_p[label == k].mean(), rtol=1e-12)
