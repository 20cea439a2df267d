"""Pins of the oracle's hand-written adjoint against brute-force FP64 central
finite differences of the oracle's own forward (which the forward pins tie to
the paper).  Covers every piece of the substep: weights, P2G with stress,
grid update with walls, G2P, F update and the return maps, plus the
trajectory driver with loss frames."""
import numpy as np
import pytest


def setup_case(orc, model, n=6, res=16, seed=0):
    rng = np.random.default_rng(seed)
    dx = 1.0 / res
    cfg = orc.Cfg(res, dx, 2e-3, (0.0, -9.8, 0.0), bound=3)
    x = rng.uniform(0.35, 0.65, (n, 3))
    x[0, 1] = 0.17 + 0.003                       # one particle's stencil reaches the sticky floor band
    x[1, 0] = 0.80                               # and one reaches the x+ slip band
    el, pl = model
    if pl == 1:     # large deviatoric stretch so von Mises yields
        F = np.array([np.diag([1.25, 0.85, 0.95]) + 0.05 * rng.standard_normal((3, 3)) for _ in range(n)])
    elif pl == 2:   # mix of compression (projection) and expansion (cone tip)
        F = np.array([np.diag([0.8, 1.1, 0.95]) + 0.05 * rng.standard_normal((3, 3)) for _ in range(n)])
        F[-1] = np.diag([1.05, 1.04, 1.06]) + 0.01 * rng.standard_normal((3, 3))
    else:
        F = np.array([np.eye(3) + 0.1 * rng.standard_normal((3, 3)) for _ in range(n)])
    st = orc.new_state(x, rng.standard_normal((n, 3)), 3.0 * rng.standard_normal((n, 3, 3)), F)
    mat = orc.Material(rng.uniform(0.5, 1.5, n) * (dx / 2) ** 3, 100.0, np.log(rng.uniform(20, 60, n)),
                       rng.uniform(0.2, 0.4, n), rng.uniform(1.0, 4.0, n), 30.0, el, pl)
    return cfg, st, mat, rng


def objective(orc, cfg, st, mat, c):
    return float(np.sum(orc.pack(orc.substep(cfg, st, mat)) * c))


@pytest.mark.parametrize("model", [(0, 0), (1, 0), (0, 1), (0, 2), (2, 0), (3, 0), (4, 0), (5, 0), (0, 3), (0, 4),
                                   (3, 2), (4, 3)],
                         ids=["fcr", "nh", "fcr_vm", "fcr_dp", "stvk", "hencky", "fluid", "volume", "fcr_fluidplastic",
                              "fcr_sigmaplastic", "hencky_dp", "fluid_fluidplastic"])
def test_substep_adjoint_matches_central_differences(orc, model):
    cfg, st, mat, rng = setup_case(orc, model, seed=sum(model) * 7 + model[0])
    n = len(st["x"])
    c = rng.standard_normal((n, 24))
    adj_in, g = orc.substep_adjoint(cfg, st, mat, c)
    if model[1]:   # make sure the plastic branch was exercised
        cases = set()
        s1 = orc.substep(cfg, st, mat)
        for p in range(n):
            mu, lam = orc.lame(np.exp(mat.logE[p]), mat.nu[p])
            # the substep's pre-plastic F is (I + dt C') F, C' = the new C
            G = (np.eye(3) + cfg.dt * s1["C"][p]) @ st["F"][p]
            cases.add(orc.return_map(model[1], G, mu, lam, mat.yield_stress[p], 30.0)[1])
        assert 1 in cases
    packed = orc.pack(st)
    worst = 0.0
    for p in range(n):
        for k in range(24):
            h = 1e-7 if k < 3 else 1e-6
            sp, sm = packed.copy(), packed.copy()
            sp[p, k] += h
            sm[p, k] -= h
            fd = (objective(orc, cfg, orc.unpack(sp), mat, c) - objective(orc, cfg, orc.unpack(sm), mat, c)) / (2 * h)
            err = abs(fd - adj_in[p, k]) / (abs(fd) + 1e-3 * np.abs(adj_in).max() + 1e-30)
            worst = max(worst, err)
    assert worst < 2e-5
    # central-difference roundoff: about eps |f| / h per evaluation pair
    f0 = abs(objective(orc, cfg, st, mat, c))
    for j, attr in enumerate(["logE", "nu", "yield_stress"]):
        for p in range(n):
            h = 1e-6
            fd_floor = 8 * np.finfo(float).eps * f0 / h
            a = getattr(mat, attr).copy()
            ap, am = a.copy(), a.copy()
            ap[p] += h
            am[p] -= h
            fp = objective(orc, cfg, st, mat.with_params(**{attr: ap}), c)
            fm = objective(orc, cfg, st, mat.with_params(**{attr: am}), c)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[p, j]) <= 2e-5 * (abs(fd) + 1e-3 * np.abs(g[:, j]).max()) + fd_floor + 1e-12, \
                (attr, p, fd, g[p, j])


def test_yield_gradient_is_nonzero_only_for_plastic_particles(orc):
    cfg, st, mat, rng = setup_case(orc, (0, 0), seed=3)
    _, g = orc.substep_adjoint(cfg, st, mat, rng.standard_normal((len(st["x"]), 24)))
    assert np.all(g[:, 2] == 0.0)


def test_trajectory_gradient_matches_central_differences(orc):
    """Loss = 1/(F N) sum_f sum_p |x_p(t_f) - x_hat_p(t_f)|^2 over 3 frames of a
    20-substep run of 8 particles; gradient w.r.t. per-particle log E and nu."""
    rng = np.random.default_rng(21)
    res, n = 16, 8
    cfg = orc.Cfg(res, 1.0 / res, 1e-3, (0.0, -9.8, 0.0), bound=3)
    x = 0.5 + 0.04 * rng.standard_normal((n, 3))
    st = orc.new_state(x, np.tile([0.0, -0.5, 0.0], (n, 1)) + 0.1 * rng.standard_normal((n, 3)), None,
                       np.array([np.eye(3) + 0.05 * rng.standard_normal((3, 3)) for _ in range(n)]))
    mat = orc.Material(np.full(n, (0.5 / res) ** 3), 100.0, np.log(rng.uniform(5.0, 15.0, n)),
                       rng.uniform(0.2, 0.4, n), 0.0, 30.0, 0, 0)
    frames = [5, 12, 20]
    target = rng.uniform(0.45, 0.55, (3, n, 3))

    def loss(m):
        _, tape = orc.run(cfg, st, m, 20, tape=True)
        fx = tape[frames][:, :, 0:3]
        return orc.trajectory_loss(fx, target), tape

    (L, dLdx), tape = loss(mat)
    adj0, g = orc.backward(cfg, mat, tape, frames, dLdx)
    for j, attr in enumerate(["logE", "nu"]):
        for p in range(n):
            h = 1e-4      # the loss is O(1e-2) and its gradient O(1e-7): a smaller h drowns in roundoff
            a = getattr(mat, attr)
            ap, am = a.copy(), a.copy()
            ap[p] += h
            am[p] -= h
            fd = (loss(mat.with_params(**{attr: ap}))[0][0] - loss(mat.with_params(**{attr: am}))[0][0]) / (2 * h)
            assert abs(fd - g[p, j]) <= 1e-5 * (abs(fd) + 1e-3 * np.abs(g[:, j]).max()), (attr, p, fd, g[p, j])
    # adjoint of the initial positions
    for p in range(n):
        for d in range(3):
            h = 1e-6
            sp, sm = {k: v.copy() for k, v in st.items()}, {k: v.copy() for k, v in st.items()}
            sp["x"][p, d] += h
            sm["x"][p, d] -= h

            def lx(s):
                _, tp = orc.run(cfg, s, mat, 20, tape=True)
                return orc.trajectory_loss(tp[frames][:, :, 0:3], target)[0]

            fd = (lx(sp) - lx(sm)) / (2 * h)
            assert abs(fd - adj0[p, d]) <= 1e-5 * (abs(fd) + 1e-3 * np.abs(adj0[:, :3]).max())
