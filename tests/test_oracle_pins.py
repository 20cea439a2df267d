"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, special cases, brute force), never against itself.

Each test names the passage it pins.  A plausible slip in the oracle (a
dropped term, a wrong sign, a transposed operand, a wrong constant) fails at
least one of them.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ----------------------------------------------------------------------------
# interpolation kernel (quadratic B-spline reading of N in the §4.2 equation)
# ----------------------------------------------------------------------------

def cardinal_quadratic_bspline(t):
    """Textbook piecewise definition of the centred quadratic B-spline."""
    t = abs(t)
    if t < 0.5:
        return 0.75 - t * t
    if t < 1.5:
        return 0.5 * (1.5 - t) ** 2
    return 0.0


def test_bspline_matches_textbook_and_moments(orc):
    for fx in np.linspace(0.5, 1.4999, 37):
        w, dw = orc.bspline(fx)
        for i in range(3):
            assert w[i] == pytest.approx(cardinal_quadratic_bspline(fx - i), abs=1e-15)
            h = 1e-6
            fd = (cardinal_quadratic_bspline(fx + h - i) - cardinal_quadratic_bspline(fx - h - i)) / (2 * h)
            assert dw[i] == pytest.approx(fd, abs=2e-6)   # O(h) at the C1 knots
        d = np.arange(3) - fx
        assert w.sum() == pytest.approx(1.0, abs=1e-15)               # partition of unity
        assert (w * d).sum() == pytest.approx(0.0, abs=1e-15)          # linear reproduction
        assert (w * d * d).sum() == pytest.approx(0.25, abs=1e-15)     # D_p = dx^2/4: the 4/dx^2 of §4.2
        assert dw.sum() == pytest.approx(0.0, abs=1e-14)
        assert (dw * d).sum() == pytest.approx(1.0, abs=1e-14)         # sum grad w (x_i)^T = I


# ----------------------------------------------------------------------------
# SVD / polar decomposition
# ----------------------------------------------------------------------------

def higham_polar(F, iters=60):
    """Scaled Newton iteration X <- (g X + X^{-T}/g)/2 (Higham 1986); an
    algorithm independent of the oracle's Jacobi SVD."""
    X = F.copy()
    for _ in range(iters):
        Xi = np.linalg.inv(X).T
        g = (np.linalg.norm(Xi) / np.linalg.norm(X)) ** 0.5
        Xn = 0.5 * (g * X + Xi / g)
        if np.linalg.norm(Xn - X) < 1e-15:
            X = Xn
            break
        X = Xn
    return X


def svd_cases(rng):
    cases = [np.eye(3), np.diag([2.0, 2.0, 0.5]), np.diag([1.0, 1.0, 1.0 + 1e-12]), np.diag([1.3, 0.0, 0.7]),
             np.diag([1.2, 0.8, -0.9]), np.zeros((3, 3)) + np.diag([1e-9, 1e-9, 1e-9])]
    for _ in range(30):
        cases.append(np.eye(3) + 0.3 * rng.standard_normal((3, 3)))
    for _ in range(10):
        cases.append(rand_rot(rng) @ np.diag(rng.uniform(0.5, 1.5, 3)) @ rand_rot(rng).T)
    cases.append(rand_rot(rng) @ np.diag([1.0, 1.0, -1.0]) @ rand_rot(rng))
    cases.append(rand_rot(rng) @ np.diag([0.9, 0.9, 1.1]) @ rand_rot(rng).T)
    return cases


def test_svd_reconstruction_and_convention(orc):
    rng = np.random.default_rng(1)
    for F in svd_cases(rng):
        U, S, V = orc.svd(F)
        scale = max(1.0, np.abs(F).max())
        assert np.abs(U @ np.diag(S) @ V.T - F).max() < 1e-12 * scale
        assert np.abs(U.T @ U - np.eye(3)).max() < 1e-12
        assert np.abs(V.T @ V - np.eye(3)).max() < 1e-12
        assert np.linalg.det(U) == pytest.approx(1.0, abs=1e-12)
        assert np.linalg.det(V) == pytest.approx(1.0, abs=1e-12)
        ref = np.linalg.svd(F, compute_uv=False)
        assert np.allclose(np.abs(S), ref, atol=1e-12 * scale)        # |sigma| = library singular values
        assert S[0] >= S[1] - 1e-12 and S[1] >= abs(S[2]) - 1e-12
        d = np.linalg.det(F)
        if abs(d) > 1e-12:
            assert np.sign(S[2]) == np.sign(d)                         # last sigma carries sign(det F)


def test_polar_matches_newton_iteration(orc):
    rng = np.random.default_rng(2)
    for F in svd_cases(rng):
        if np.linalg.det(F) <= 1e-6:
            continue
        R = orc.polar(F)
        assert np.abs(R - higham_polar(F)).max() < 1e-10
        S = R.T @ F
        assert np.abs(S - S.T).max() < 1e-10                          # F = R S, S symmetric
        assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)


# ----------------------------------------------------------------------------
# elasticity (App. A and App. B.1)
# ----------------------------------------------------------------------------

def energy_fcr(F, mu, lam):
    """Fixed-corotated energy of Stomakhin et al. 2012: mu sum(s_i-1)^2 + lam/2 (J-1)^2."""
    s = np.linalg.svd(F, compute_uv=False)
    J = np.linalg.det(F)
    if J < 0:
        s[-1] = -s[-1]
    return mu * np.sum((s - 1.0) ** 2) + 0.5 * lam * (J - 1.0) ** 2


def energy_nh(F, mu, lam):
    """Neo-Hookean energy: mu/2 (tr F^T F - 3) - mu log J + lam/2 (log J)^2."""
    J = np.linalg.det(F)
    return 0.5 * mu * (np.sum(F * F) - 3.0) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2


def fd_pk1(energy, F, mu, lam, h=1e-6):
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            P[i, j] = (energy(F + E, mu, lam) - energy(F - E, mu, lam)) / (2 * h)
    return P


@pytest.mark.parametrize("model,energy", [(0, energy_fcr), (1, energy_nh)])
def test_kirchhoff_is_energy_derivative_times_Ft(orc, model, energy):
    rng = np.random.default_rng(3 + model)
    mu, lam = 3.7, 5.3
    for _ in range(25):
        F = rand_rot(rng) @ np.diag(rng.uniform(0.6, 1.4, 3)) @ rand_rot(rng).T
        tau = orc.kirchhoff(model, F, mu, lam)
        ref = fd_pk1(energy, F, mu, lam) @ F.T
        assert np.abs(tau - ref).max() < 1e-7 * max(1.0, np.abs(ref).max())
        assert np.abs(tau - tau.T).max() < 1e-12                        # symmetric: no spurious torque


@pytest.mark.parametrize("model", [0, 1])
def test_rest_state_is_stress_free_and_rotation_invariant(orc, model):
    assert np.abs(orc.kirchhoff(model, np.eye(3), 1e4, 2e4)).max() == 0.0
    rng = np.random.default_rng(5)
    for _ in range(10):
        Q = rand_rot(rng)
        assert np.abs(orc.kirchhoff(model, Q, 1e4, 2e4)).max() < 1e-9          # rigid rotation: no stress
        F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
        F = F if np.linalg.det(F) > 0 else -F
        t1 = orc.kirchhoff(model, Q @ F, 3.0, 4.0)
        t2 = Q @ orc.kirchhoff(model, F, 3.0, 4.0) @ Q.T
        assert np.abs(t1 - t2).max() < 1e-12


def test_lame_parameters_reproduce_E_and_nu_in_uniaxial_stress(orc):
    """App. B.1 (mu, lambda from E, nu): small uniaxial stretch eps with lateral
    contraction -nu eps must give axial stress E eps and zero lateral stress
    (the definitions of Young's modulus and Poisson's ratio)."""
    for E, nu in [(1e4, 0.3), (5e3, 0.2), (1e5, 0.4)]:
        mu, lam = orc.lame(E, nu)
        eps = 1e-7
        F = np.diag([1 + eps, 1 - nu * eps, 1 - nu * eps])
        for model in (0, 1):
            tau = orc.kirchhoff(model, F, mu, lam)
            assert tau[0, 0] / eps == pytest.approx(E, rel=1e-5)
            assert abs(tau[1, 1] / eps) < 1e-4 * E
            assert abs(tau[2, 2] / eps) < 1e-4 * E


def test_stress_linear_in_E(orc):
    """App. B.1: tau is linear in E at fixed F and nu."""
    rng = np.random.default_rng(6)
    F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    F = F if np.linalg.det(F) > 0 else -F
    for model in (0, 1):
        a = orc.kirchhoff(model, F, *orc.lame(1e4, 0.3))
        b = orc.kirchhoff(model, F, *orc.lame(3e4, 0.3))
        assert np.abs(b - 3 * a).max() < 1e-9 * np.abs(b).max()


# ----------------------------------------------------------------------------
# plasticity (App. A eq. von_mises / drucker_prager; App. B.2)
# ----------------------------------------------------------------------------

def log_strain(F):
    s = np.linalg.svd(F, compute_uv=False)
    return np.log(s)


def test_dp_alpha_at_30_degrees(orc):
    # sin 30 = 1/2:  sqrt(2/3) * 2 * (1/2) / (3 - 1/2) = sqrt(2/3) * 2/5
    assert orc.dp_alpha(30.0) == pytest.approx(math.sqrt(2.0 / 3.0) * 0.4, rel=1e-14)


def test_von_mises_projects_onto_yield_surface(orc):
    rng = np.random.default_rng(7)
    mu, lam = orc.lame(1e4, 0.3)
    sy = 1e3
    n_proj = 0
    for _ in range(40):
        F = rand_rot(rng) @ np.diag(np.exp(rng.normal(0, 0.3, 3))) @ rand_rot(rng).T
        Fn, case = orc.return_map(1, F, mu, lam, sy, 30.0)
        e = log_strain(F)
        dev = np.linalg.norm(e - e.mean())
        if dev <= sy / (2 * mu):
            assert case == 0 and np.array_equal(Fn, F)
            continue
        n_proj += 1
        assert case == 1
        en = log_strain(Fn)
        assert np.linalg.norm(en - en.mean()) == pytest.approx(sy / (2 * mu), rel=1e-10)   # on the surface
        assert np.linalg.det(Fn) == pytest.approx(np.linalg.det(F), rel=1e-10)            # volume kept
        Fnn, c2 = orc.return_map(1, Fn, mu, lam, sy, 30.0)
        assert np.abs(Fnn - Fn).max() < 1e-9                                             # idempotent
        Q1, Q2 = rand_rot(rng), rand_rot(rng)                                             # isotropic
        Fr, _ = orc.return_map(1, Q1 @ F @ Q2, mu, lam, sy, 30.0)
        assert np.abs(Fr - Q1 @ Fn @ Q2).max() < 1e-10
    assert n_proj > 10


def test_drucker_prager_cases(orc):
    rng = np.random.default_rng(8)
    mu, lam = orc.lame(1e4, 0.3)
    alpha = orc.dp_alpha(30.0)
    kap = (3 * lam + 2 * mu) / (2 * mu) * alpha
    seen = set()
    for _ in range(80):
        F = rand_rot(rng) @ np.diag(np.exp(rng.normal(-0.05, 0.2, 3))) @ rand_rot(rng).T
        e = log_strain(F)
        Fn, case = orc.return_map(2, F, mu, lam, 0.0, 30.0)
        seen.add(case)
        if e.sum() > 0:                              # expansion: cone tip, Sigma = I
            assert case == 2
            assert np.allclose(np.linalg.svd(Fn, compute_uv=False), 1.0, atol=1e-12)
            assert np.linalg.det(Fn) == pytest.approx(1.0, abs=1e-12)
        elif np.linalg.norm(e - e.mean()) + kap * e.sum() <= 0:
            assert case == 0 and np.array_equal(Fn, F)
        else:
            assert case == 1
            en = log_strain(Fn)
            # on the cone |eps_hat| + kappa tr(eps) = 0, trace (volume) kept
            assert np.linalg.norm(en - en.mean()) == pytest.approx(-kap * en.sum(), rel=1e-9)
            assert en.sum() == pytest.approx(e.sum(), rel=1e-10)
            Fnn, _ = orc.return_map(2, Fn, mu, lam, 0.0, 30.0)
            assert np.abs(Fnn - Fn).max() < 1e-9
    assert seen == {0, 1, 2}


# ----------------------------------------------------------------------------
# transfers: P2G / grid update / G2P (§4.2 equation; App. A)
# ----------------------------------------------------------------------------

def small_setup(orc, n=6, res=16, seed=0, walls=(0,) * 6, gravity=(0.0, 0.0, 0.0), dt=1e-3, model=(0, 0),
                Fnoise=0.1, Cnoise=1.0):
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    cfg = orc.Cfg(res, dx, dt, gravity, bound=3, walls=walls)
    x = rng.uniform(0.4, 0.6, (n, 3))
    F = np.array([np.eye(3) + Fnoise * rng.standard_normal((3, 3)) for _ in range(n)])
    st = orc.new_state(x, rng.standard_normal((n, 3)), Cnoise * rng.standard_normal((n, 3, 3)), F)
    mat = orc.Material(rng.uniform(0.5, 1.5, n) * dx ** 3 / 8, rng.uniform(1, 3, n), np.log(rng.uniform(1e2, 1e3, n)),
                       rng.uniform(0.2, 0.4, n), rng.uniform(50, 100, n), 30.0, model[0], model[1])
    return cfg, st, mat


def node_positions(cfg):
    I = np.stack(np.meshgrid(*[np.arange(r) for r in cfg.res], indexing="ij"), -1)
    return I * cfg.dx


def test_p2g_conserves_mass_and_linear_momentum(orc):
    cfg, st, mat = small_setup(orc, n=12)
    gm, gmv = orc.p2g(cfg, st, mat)
    assert gm.sum() == pytest.approx(mat.mass.sum(), rel=1e-14)
    # the C and stress terms vanish in the sum because sum_i w (x_i - x_p) = 0
    ref = (mat.mass[:, None] * st["v"]).sum(0)
    assert np.abs(gmv.reshape(-1, 3).sum(0) - ref).max() < 1e-13 * np.abs(mat.mass).sum()


def test_p2g_first_moment_is_affine_momentum_minus_stress_impulse(orc):
    """sum_i m_i v_i (x_i - x_p)^T = (m_p C_p - 4 dt V_p tau_p / dx^2) dx^2/4
    = m_p C_p dx^2/4 - dt V_p tau_p for one particle: pins the 4/dx^2 factor and
    the sign of the stress term of the §4.2 equation (a compressed particle
    pushes momentum outward)."""
    for model in (0, 1):
        cfg, st, mat = small_setup(orc, n=1, model=(model, 0), seed=11)
        st["F"][0] = np.diag([0.9, 0.95, 0.92])                                       # compressed
        gm, gmv = orc.p2g(cfg, st, mat)
        X = node_positions(cfg).reshape(-1, 3) - st["x"][0]
        M = gmv.reshape(-1, 3).T @ X
        tau = orc.kirchhoff(model, st["F"][0], *orc.lame(np.exp(mat.logE[0]), mat.nu[0]))
        ref = mat.mass[0] * st["C"][0] * cfg.dx ** 2 / 4 - cfg.dt * mat.vol[0] * tau
        assert np.abs(M - ref).max() < 1e-12 * np.abs(ref).max()
        st["C"][0] = 0.0
        st["v"][0] = 0.0
        gm, gmv = orc.p2g(cfg, st, mat)
        assert np.sum(gmv.reshape(-1, 3) * X) > 0                                    # outward push


def test_grid_update_gravity_and_walls(orc):
    res = 8
    cfg = orc.Cfg(res, 1 / res, 0.01, (0.0, -9.8, 0.0), bound=3)       # floor sticky, others slip
    gm = np.zeros((res,) * 3)
    gmv = np.zeros((res,) * 3 + (3,))
    for I, u in [((4, 4, 4), (1.0, 2.0, 3.0)), ((1, 4, 4), (-1.0, 2.0, 3.0)), ((6, 4, 4), (-1.0, 2.0, 3.0)),
                 ((4, 1, 4), (1.0, 2.0, 3.0)), ((4, 4, 7), (1.0, 2.0, 3.0)), ((4, 4, 0), (1.0, 2.0, 3.0))]:
        gm[I] = 2.0
        gmv[I] = 2.0 * np.array(u)
    gv = orc.grid_update(cfg, gm, gmv)
    g = 0.01 * -9.8
    assert np.allclose(gv[4, 4, 4], [1.0, 2.0 + g, 3.0])
    assert np.allclose(gv[1, 4, 4], [0.0, 2.0 + g, 3.0])       # x- slip, outward: cut
    assert np.allclose(gv[6, 4, 4], [-1.0, 2.0 + g, 3.0])      # x+ slip, inward: kept
    assert np.allclose(gv[4, 1, 4], [0.0, 0.0, 0.0])           # sticky floor
    assert np.allclose(gv[4, 4, 7], [1.0, 2.0 + g, 0.0])       # z+ slip, v_z > 0 outward: cut
    assert np.allclose(gv[4, 4, 0], [1.0, 2.0 + g, 3.0])       # z- slip, v_z > 0 inward: kept
    assert np.all(gv[0, 0, 0] == 0.0)                          # empty node


def test_grid_update_slip_cuts_outward_normal(orc):
    res = 8
    cfg = orc.Cfg(res, 1 / res, 0.01, (0.0, 0.0, 0.0), bound=3)
    gm = np.zeros((res,) * 3)
    gmv = np.zeros((res,) * 3 + (3,))
    gm[4, 4, 6] = 1.0
    gmv[4, 4, 6] = (1.0, 2.0, 3.0)                             # z+ band, v_z outward
    gv = orc.grid_update(cfg, gm, gmv)
    assert np.allclose(gv[4, 4, 6], [1.0, 2.0, 0.0])


def test_free_fall_closed_form(orc):
    """Uniform velocity, F = I, no walls reached: v_n = v_0 + n dt g and
    x_n = x_0 + n dt v_0 + dt^2 g n(n+1)/2 (grid velocity updated first, then
    positions: symplectic Euler), F and C stay I and 0."""
    res, n_sub, dt = 32, 40, 1e-3
    cfg = orc.Cfg(res, 1 / res, dt, (0.0, -9.8, 0.0), bound=3)
    rng = np.random.default_rng(9)
    x0 = rng.uniform(0.4, 0.6, (50, 3))
    v0 = np.array([0.3, 0.5, -0.2])
    st = orc.new_state(x0, np.tile(v0, (50, 1)))
    mat = orc.Material(np.full(50, 1e-5), 1.0, np.log(10.0), 0.3, 0.0, 30.0, 0, 0)   # soft: CFL 0.1
    out = orc.run(cfg, st, mat, n_sub)
    g = np.array([0.0, -9.8, 0.0])
    assert np.abs(out["v"] - (v0 + n_sub * dt * g)).max() < 1e-12
    xr = x0 + n_sub * dt * v0 + dt * dt * g * n_sub * (n_sub + 1) / 2
    assert np.abs(out["x"] - xr).max() < 1e-13
    assert np.abs(out["C"]).max() < 1e-10
    assert np.abs(out["F"] - np.eye(3)).max() < 1e-13


def test_rigid_rotation_reproduced_by_one_transfer(orc):
    """APIC with a quadratic B-spline reproduces linear fields: v = w x (x-c),
    C = [w]_x survive one P2G -> G2P round trip exactly (F = I, tau = 0)."""
    res, dt = 32, 1e-4
    cfg = orc.Cfg(res, 1 / res, dt, (0.0, 0.0, 0.0), bound=3, walls=(0,) * 6)
    rng = np.random.default_rng(10)
    x = rng.uniform(0.4, 0.6, (64, 3))
    c = np.array([0.5, 0.5, 0.5])
    w = np.array([0.7, -1.1, 0.4])
    Wx = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    st = orc.new_state(x, np.cross(w, x - c), np.tile(Wx, (64, 1, 1)))
    mat = orc.Material(np.full(64, 1e-5), 1.0, np.log(1e4), 0.3, 0.0, 30.0, 0, 0)
    out = orc.substep(cfg, st, mat)
    assert np.abs(out["v"] - np.cross(w, x - c)).max() < 1e-13
    assert np.abs(out["C"] - Wx).max() < 1e-11
    assert np.abs(out["x"] - (x + dt * np.cross(w, x - c))).max() < 1e-15


def angular_momentum(st, mat, dx):
    """particle angular momentum incl. the APIC affine part m (dx^2/4) eps:C^T"""
    L = np.cross(st["x"], mat.mass[:, None] * st["v"]).sum(0)
    C = st["C"]
    aff = np.stack([C[:, 2, 1] - C[:, 1, 2], C[:, 0, 2] - C[:, 2, 0], C[:, 1, 0] - C[:, 0, 1]], axis=1)
    return L + (mat.mass[:, None] * aff).sum(0) * dx * dx / 4


def test_angular_and_linear_momentum_conserved_over_substeps(orc):
    """No gravity, no walls: a spinning, deformed elastic cube keeps total
    linear and (APIC) angular momentum; the stress adds no torque because
    tau is symmetric."""
    res = 32
    dx = 1 / res
    cfg = orc.Cfg(res, dx, 2e-4, (0.0, 0.0, 0.0), bound=3, walls=(0,) * 6)
    rng = np.random.default_rng(12)
    x = rng.uniform(0.42, 0.58, (300, 3))
    w = np.array([3.0, -2.0, 5.0])
    v = np.cross(w, x - 0.5) + 0.1 * rng.standard_normal((300, 3))
    F = np.array([np.eye(3) + 0.05 * rng.standard_normal((3, 3)) for _ in range(300)])
    st = orc.new_state(x, v, None, F)
    for model in (0, 1):
        mat = orc.Material(np.full(300, (dx / 2) ** 3), 10.0, np.log(1e3), 0.3, 0.0, 30.0, model, 0)
        L0 = angular_momentum(st, mat, dx)
        P0 = (mat.mass[:, None] * st["v"]).sum(0)
        out = orc.run(cfg, st, mat, 60)
        assert np.abs(out["F"] - F).max() > 1e-3                      # it did deform
        L1 = angular_momentum(out, mat, dx)
        P1 = (mat.mass[:, None] * out["v"]).sum(0)
        assert np.abs(L1 - L0).max() < 1e-11 * np.abs(L0).max()
        assert np.abs(P1 - P0).max() < 1e-11 * np.abs(mat.mass).sum()


def test_out_of_domain_is_an_error(orc):
    cfg = orc.Cfg(16, 1 / 16, 1e-3)
    st = orc.new_state(np.array([[0.01, 0.5, 0.5]]))
    mat = orc.Material([1e-5], 1.0, np.log(1e4), 0.3, 0.0, 30.0, 0, 0)
    with pytest.raises(orc.OracleError):
        orc.substep(cfg, st, mat)
