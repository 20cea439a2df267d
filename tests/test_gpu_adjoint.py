"""GPU reverse pass (hand-written adjoint with checkpoint recompute) against
the FP64 oracle's adjoint and against FP64 central finite differences.  Each
side runs its own forward from the same seeded inputs and forms its own loss
gradient; nothing the CUDA path computes is fed to the oracle.

Tolerance: gradients within 1e-3 relative, ||g_gpu - g_ref||_2 / ||g_ref||_2
per parameter kind."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_01723_gb300 import scenes  # noqa: E402

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def sim_mod():
    from __graft_entry__ import build
    build()
    from paper_2602_01723_gb300 import sim
    return sim


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def mixed_state(sc, seed=3, fs=0.08):
    rng = np.random.default_rng(seed)
    v = (sc.v + 0.3 * rng.standard_normal((sc.n, 3))).astype(np.float32)
    C = (2.0 * rng.standard_normal((sc.n, 3, 3))).astype(np.float32)
    F = np.array([np.eye(3) + fs * rng.standard_normal((3, 3)) for _ in range(sc.n)], dtype=np.float32)
    return v, C, F


def one_substep_case(orc, sim_mod, sc, v, C, F, params=None, seed=0):
    """Adjoint of one substep seeded by a random dL/dx of the new positions."""
    rng = np.random.default_rng(seed)
    cx = rng.standard_normal((sc.n, 3)).astype(np.float32)
    s = sim_mod.Simulator.from_scene(sc, ckpt_every=20)
    s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F, params=params)
    s.step(1, record=True)
    g, a0 = s.backward([1], torch.as_tensor(cx[None]), want_state0=True)
    g = g.double().cpu().numpy()
    a0 = a0.double().cpu().numpy()
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, params)
    adj_out = np.zeros((sc.n, 24))
    adj_out[:, 0:3] = cx
    ai, gr = orc.substep_adjoint(cfg, orc.new_state(sc.x, v, C, F), mat, adj_out)
    return g, a0, gr, ai


@pytest.mark.parametrize("kind", ["fcr", "nh", "fcr_vm", "fcr_dp"])
def test_one_substep_adjoint_matches_oracle(orc, sim_mod, kind):
    sc = scenes.ball_512()
    el, pl = {"fcr": (0, 0), "nh": (1, 0), "fcr_vm": (0, 1), "fcr_dp": (0, 2)}[kind]
    sc.materials = [scenes.material(el, pl, 5e3, 0.3, 100.0, yield_stress=30.0, friction_angle_deg=30.0)]
    sc.params = None
    fs = 0.15 if pl else 0.05
    v, C, F = mixed_state(sc, fs=fs)
    g, a0, gr, ai = one_substep_case(orc, sim_mod, sc, v, C, F)
    assert rel(a0[:, 0:3], ai[:, 0:3]) < GRAD_TOL
    assert rel(a0[:, 3:6], ai[:, 3:6]) < GRAD_TOL
    assert rel(a0[:, 6:15], ai[:, 6:15]) < GRAD_TOL
    assert rel(a0[:, 15:24], ai[:, 15:24]) < GRAD_TOL
    assert rel(g[:, 0], gr[:, 0]) < GRAD_TOL      # d / d log E
    assert rel(g[:, 1], gr[:, 1]) < GRAD_TOL      # d / d nu
    # (a one-substep position loss does not depend on the yield stress: the
    # return map changes only the stored F; the multi-substep test covers it)


def frame_loss_gradients(orc, sim_mod, sc, params, n_sub, frames, target, C=None, F=None, **sim_kw):
    """The frame MSE loss L = 1/(F N) sum |x_f - target_f|^2 differentiated on
    both sides: the GPU records its forward, reads the frame positions and
    runs its reverse pass; the oracle runs its own FP64 forward with a tape
    and its own adjoint.  Returns (g_gpu, g_oracle), each (n, 3)."""
    s = sim_mod.Simulator.from_scene(sc, **sim_kw)
    s.load(sc.x, sc.vol, sc.mat_id, v=sc.v, C=C, F=F, params=params)
    xs, prev = [], 0
    for f in frames:
        s.step(f - prev, record=True)
        xs.append(s.positions().double().cpu().numpy())
        prev = f
    s.step(n_sub - prev, record=True)
    nf = len(frames)
    dLdx = 2.0 * (np.stack(xs) - target) / (nf * sc.n)
    g = s.backward(frames, torch.as_tensor(dLdx, dtype=torch.float32)).double().cpu().numpy()
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, params)
    _, tape = orc.run(cfg, orc.new_state(sc.x, sc.v, C, F), mat, n_sub, tape=True)
    _, dLdx_ref = orc.trajectory_loss(tape[frames][:, :, 0:3], target)
    _, g_ref = orc.backward(cfg, mat, tape, frames, dLdx_ref)
    return g, g_ref


@pytest.mark.parametrize("tape_grid", [0, 1])
def test_multi_substep_adjoint_all_models(orc, sim_mod, tape_grid):
    """30 substeps of a mixed-material ball (FCR, NH, von Mises, Drucker-
    Prager), checkpoint every 20 (two segments), frames at 10, 20, 30; log E,
    nu and yield-stress gradients.  tape_grid 0: the reverse substeps read the
    binning and grid kept by the segment's recompute; 1: they rebuild them."""
    sc = scenes.ball_512()
    sc.materials = [scenes.material(0, 0, 5e3, 0.3, 100.0), scenes.material(1, 0, 5e3, 0.3, 100.0),
                    scenes.material(0, 1, 5e3, 0.3, 100.0, yield_stress=20.0),
                    scenes.material(0, 2, 5e3, 0.3, 100.0, friction_angle_deg=30.0)]
    sc.mat_id = (np.arange(sc.n) % 4).astype(np.int32)
    rng = np.random.default_rng(5)
    params = np.stack([np.log(5e3) + 0.3 * rng.standard_normal(sc.n), rng.uniform(0.2, 0.4, sc.n),
                       rng.uniform(10.0, 30.0, sc.n)], axis=1).astype(np.float32)
    sc.v = (sc.v + 2.0 * rng.standard_normal((sc.n, 3))).astype(np.float32)    # shear: plastic flow
    frames = [10, 20, 30]
    target = sc.x[None].astype(np.float64) + 0.01 * rng.standard_normal((3, sc.n, 3))
    g, g_ref = frame_loss_gradients(orc, sim_mod, sc, params, 30, frames, target, tape_grid=tape_grid)
    for j in range(3):
        assert np.abs(g_ref[:, j]).max() > 0
        assert rel(g[:, j], g_ref[:, j]) < GRAD_TOL, (j, rel(g[:, j], g_ref[:, j]))


def seeded_cotangent_gradients(orc, sim_mod, sc, params, n_sub, frames, cot, **sim_kw):
    """Parameter gradients of sum_f <cot_f, x(t_f)> on both sides: the same
    seeded cotangents cot (n_frames, n, 3) enter the GPU reverse pass and the
    oracle's FP64 reverse pass.  Neither side's positions enter the other's
    cotangents, so the comparison checks the checkpointed reverse pass itself,
    independently of how well any particular loss is conditioned.  Returns
    (g_gpu, g_oracle, x_gpu, x_oracle) with x at the last substep."""
    s = sim_mod.Simulator.from_scene(sc, **sim_kw)
    s.load(sc.x, sc.vol, sc.mat_id, v=sc.v, instance=sc.instance, params=params)
    s.step(n_sub, record=True)
    x_gpu = s.positions().double().cpu().numpy()
    g = s.backward(frames, torch.as_tensor(cot, dtype=torch.float32)).double().cpu().numpy()
    assert s.stats()["device_error"] == 0
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, params)
    _, tape = orc.run(cfg, orc.new_state(sc.x, sc.v), mat, n_sub, tape=True)
    _, g_ref = orc.backward(cfg, mat, tape, frames, cot)
    return g, g_ref, x_gpu, tape[n_sub][:, 0:3]


def test_ball_512_seeded_cotangents_400_substeps(orc, sim_mod):
    """The differentiable workload's 512-particle, 16^3 copy as configured:
    400 substeps of 1e-4 with the floor contact from about substep 130,
    checkpoint every 20 (20 segments, the overlapped recompute), ten frames
    every 40 substeps, at the initial guess log E = log 5e3, nu = 0.3.  Both
    reverse passes take the same seeded cotangents; the GPU's d/d log E and
    d/d nu match the FP64 adjoint within 1e-3 relative per kind."""
    sc = scenes.ball_512()
    frames = [int(f) for f in sc.frame_sub]
    assert frames == list(range(40, 401, 40)) and sc.ckpt_every == 20 and sc.n_substeps == 400
    cot = np.random.default_rng(400).standard_normal((len(frames), sc.n, 3))
    g, g_ref, x_gpu, x_ref = seeded_cotangent_gradients(orc, sim_mod, sc, sc.params, sc.n_substeps, frames, cot)
    print("ball_512, 400 substeps, seeded cotangents: x %.3g dx, d/dlogE %.3g, d/dnu %.3g"
          % (np.abs(x_gpu - x_ref).max() / sc.dx, rel(g[:, 0], g_ref[:, 0]), rel(g[:, 1], g_ref[:, 1])))
    assert np.abs(x_gpu - x_ref).max() < 1e-4 * sc.dx      # the trajectory both adjoints run along
    for j in range(2):
        assert np.abs(g_ref[:, j]).max() > 0
        assert rel(g[:, j], g_ref[:, j]) < GRAD_TOL, (j, rel(g[:, j], g_ref[:, j]))


def test_converging_cloud_with_overflow_items_seeded_cotangents(orc, sim_mod):
    """A cloud of 8,192 particles converging at 60/s (lists of 160 per block
    from the load, several times that many particles per block within 60
    substeps) puts particles in overflow entries during the recorded forward.
    With checkpoints every 20 substeps and seeded cotangents at substeps 20,
    40 and 60, d/d log E and d/d nu match the FP64 adjoint within 1e-3."""
    rng = np.random.default_rng(91)
    n, R = 8192, 32
    dx = 1.0 / R
    x = rng.uniform(0.2, 0.8, (n, 3)).astype(np.float32)
    v = (-60.0 * (x.astype(np.float64) - 0.5)).astype(np.float32)
    sc = scenes.Scene("converging_cloud", R, 1e-4, 60, x, v, np.full(n, (0.5 * dx) ** 3, np.float32),
                      np.zeros(n, np.int32), [scenes.material(0, 0, 1e2, 0.3, 1.0)], gravity=(0.0, 0.0, 0.0),
                      ckpt_every=20)
    frames = [20, 40, 60]
    cot = np.random.default_rng(92).standard_normal((len(frames), n, 3))
    g, g_ref, x_gpu, x_ref = seeded_cotangent_gradients(orc, sim_mod, sc, None, 60, frames, cot)
    s = sim_mod.Simulator.from_scene(sc)
    s.load(sc.x, sc.vol, sc.mat_id, v=sc.v)
    s.step(60, record=True)
    s.backward(frames, torch.as_tensor(cot, dtype=torch.float32))
    st = s.stats()
    s.close()
    print("converging cloud, 60 substeps: %d overflow placements, x %.3g dx, d/dlogE %.3g, d/dnu %.3g"
          % (st["overflow_particles"], np.abs(x_gpu - x_ref).max() / dx, rel(g[:, 0], g_ref[:, 0]),
             rel(g[:, 1], g_ref[:, 1])))
    assert st["list_capacity"] == 160 and st["overflow_particles"] > 0, st
    assert np.abs(x_gpu - x_ref).max() < 1e-4 * dx
    for j in range(2):
        assert np.abs(g_ref[:, j]).max() > 0
        assert rel(g[:, j], g_ref[:, j]) < GRAD_TOL, (j, rel(g[:, j], g_ref[:, j]))


def test_recording_in_two_calls_with_odd_checkpoint_interval(orc, sim_mod):
    """The recorded forward copies each checkpoint after the substep that
    completes it, inside one run per call.  With a checkpoint every 7
    substeps the copies fall inside graph-replayed substep pairs, and a
    recording made of two calls (90 and 80 substeps) starts its second run
    between checkpoints.  Seeded cotangents at substeps 90 and 170 (the ball
    meets the floor near substep 130, so the stress, and with it E and nu,
    shapes the trajectory): d/d log E and d/d nu match the FP64 adjoint
    within 1e-3."""
    sc = scenes.ball_512()
    frames = [90, 170]
    cot = np.random.default_rng(745).standard_normal((len(frames), sc.n, 3))
    s = sim_mod.Simulator.from_scene(sc, ckpt_every=7)
    s.load(sc.x, sc.vol, sc.mat_id, v=sc.v, params=sc.params)
    s.step(90, record=True)
    s.step(80, record=True)
    g = s.backward(frames, torch.as_tensor(cot, dtype=torch.float32)).double().cpu().numpy()
    assert s.stats()["recorded"] == 170 and s.stats()["device_error"] == 0
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.params)
    _, tape = orc.run(cfg, orc.new_state(sc.x, sc.v), mat, 170, tape=True)
    _, g_ref = orc.backward(cfg, mat, tape, frames, cot)
    print("ball_512, 90 + 80 recorded substeps, checkpoint every 7: d/dlogE %.3g, d/dnu %.3g"
          % (rel(g[:, 0], g_ref[:, 0]), rel(g[:, 1], g_ref[:, 1])))
    for j in range(2):
        assert np.abs(g_ref[:, j]).max() > 0
        assert rel(g[:, j], g_ref[:, j]) < GRAD_TOL, (j, rel(g[:, j], g_ref[:, j]))


def test_ball_512_trajectory_gradient(orc, sim_mod):
    """The 512-particle, 16^3 copy of the differentiable ball: 400 substeps,
    checkpoint every 20, loss frames every 40 substeps, target from the seeded
    ground-truth parameters.  (1) the oracle's FP64 gradient against FP64
    central differences of its own loss, within 1e-3; (2) the GPU gradient of
    this loss end to end (its own FP32 forward, its own dL/dx, its reverse
    pass) against the FP64 one, within 1e-3 per kind.  The loss is about
    3e-9: the frame positions lie within about 5e-5 of the target, so
    dL/dx = 2 (x - x_target)/(F N) is a small difference of positions and
    amplifies the forward's position error by about the ratio of dx to
    |x - x_target|.  With the positions held in fixed point the forward stays
    within about 5e-6 dx of the oracle over the 400 substeps, and the
    end-to-end gradient within about 2e-4."""
    sc = scenes.ball_512()
    frames = [int(f) for f in sc.frame_sub]
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    st0 = orc.new_state(sc.x, sc.v)
    mat_true = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.extra["params_true"])
    _, tape_t = orc.run(cfg, st0, mat_true, sc.n_substeps, tape=True)
    target = tape_t[frames][:, :, 0:3]
    g, g64 = frame_loss_gradients(orc, sim_mod, sc, sc.params, sc.n_substeps, frames, target)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.params)
    for p in np.argsort(-np.abs(g64[:, 0]))[:2]:
        h = 1e-3
        fl = []
        for sgn in (1, -1):
            le = mat.logE.copy()
            le[p] += sgn * h
            _, tp = orc.run(cfg, st0, mat.with_params(logE=le), sc.n_substeps, tape=True)
            fl.append(orc.trajectory_loss(tp[frames][:, :, 0:3], target)[0])
        fd = (fl[0] - fl[1]) / (2 * h)
        assert abs(g64[p, 0] - fd) < 1e-3 * abs(fd), (p, g64[p, 0], fd)
    print("ground-truth loss, GPU vs FP64 gradient: d/dlogE %.3g, d/dnu %.3g"
          % (rel(g[:, 0], g64[:, 0]), rel(g[:, 1], g64[:, 1])))
    assert rel(g[:, 0], g64[:, 0]) < GRAD_TOL
    assert rel(g[:, 1], g64[:, 1]) < GRAD_TOL


def test_ball_50k_full_size_gradient(orc, sim_mod):
    """The 50k-particle, 64^3 ball at full size: 100 substeps (5 checkpoint
    segments), frames at 60 and 100, from a slightly stressed seeded start
    (|F - I| ~ 0.02): before the floor contact a ball in free fall carries no
    stress and its log-E gradient is rounding noise, so the stressed start
    makes the gradient physical from the first substep.  The target is
    offset from the start (a well-conditioned loss)."""
    sc = scenes.ball_50k()
    v, C, F = scenes.key_frames(sc, 1, k_seed=65, vs=0.1, cs=1.0, fs=0.02)[0]
    sc.v = v
    frames = [60, 100]
    rng = np.random.default_rng(7)
    target = sc.x[None].astype(np.float64) + np.array([0.0, -0.01, 0.0]) + 0.002 * rng.standard_normal((2, sc.n, 3))
    g, g_ref = frame_loss_gradients(orc, sim_mod, sc, sc.params, 100, frames, target, C=C, F=F)
    assert np.abs(g_ref[:, 0]).max() > 0
    assert rel(g[:, 0], g_ref[:, 0]) < GRAD_TOL
    assert rel(g[:, 1], g_ref[:, 1]) < GRAD_TOL


def test_backward_leaves_the_recorded_state_unchanged(sim_mod):
    sc = scenes.ball_512()
    s = sim_mod.Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(30, record=True)
    x_before = s.positions().clone()
    s.backward([10, 30], torch.ones((2, sc.n, 3), device="cuda"))
    assert torch.equal(s.positions(), x_before)
    s.step(5, record=True)                        # recording continues contiguously
    s.backward([35], torch.ones((1, sc.n, 3), device="cuda"))
    s.close()


def test_backward_argument_errors(sim_mod):
    from paper_2602_01723_gb300 import _lib as L
    sc = scenes.ball_512()
    s = sim_mod.Simulator.from_scene(sc)
    s.load_scene(sc)
    with pytest.raises(L.MpmError):
        s.backward([1], torch.ones((1, sc.n, 3), device="cuda"))     # nothing recorded
    s.step(10, record=True)
    with pytest.raises(L.MpmError):
        s.backward([11], torch.ones((1, sc.n, 3), device="cuda"))    # frame beyond the recording
    s.step(3)                                                        # unrecorded step breaks the recording
    with pytest.raises(L.MpmError):
        s.step(1, record=True)
    s.close()
    for bad in (-1, 2):                                              # tape_grid is 0 or 1
        with pytest.raises(L.MpmError):
            sim_mod.Simulator.from_scene(sc, tape_grid=bad)


def test_grid_tape_overflow_reruns_with_whole_pool_slots(orc, sim_mod):
    """The grid tape sizes each recorded state's grid slot from the active
    blocks seen when it is allocated.  A context first differentiates a
    compact 512-particle ball on a 64^3 grid (small slots), then the same
    number of particles spread over [0.15, 0.85]^3 (about twenty times the
    active blocks): its states overflow their slots, the reverse pass runs
    again with slots of the whole pool, and the gradients of the spread
    scene match the FP64 oracle.  30 substeps, checkpoint every 10 (the
    overlapped segment steps run), frames at 10, 20, 30, stressed start."""
    R, dx, dt, n = 64, 1.0 / 64, 1e-4, 512
    mats = [scenes.material(0, 0, 5e3, 0.3, 100.0)]
    rng = np.random.default_rng(11)
    xa, h = scenes._jittered_ball(n, (0.5, 0.3, 0.5), 0.05, rng)
    xb = rng.uniform(0.15, 0.85, (n, 3)).astype(np.float32)
    F = (np.eye(3)[None] + 0.02 * rng.standard_normal((n, 3, 3))).reshape(n, 9)
    C = (0.5 * rng.standard_normal((n, 9)))
    params = np.stack([np.log(5e3) + 0.3 * rng.standard_normal(n), rng.uniform(0.2, 0.4, n), np.zeros(n)],
                      axis=1).astype(np.float32)
    vol = np.full(n, (0.5 * dx) ** 3, np.float32)
    mid = np.zeros(n, np.int32)
    frames = [10, 20, 30]
    s = sim_mod.Simulator(R, dx, dt, (0.0, -9.8, 0.0), mats, ckpt_every=10)

    def grads(x, target):
        s.load(x.astype(np.float32), vol, mid, v=np.zeros((n, 3), np.float32), C=C.astype(np.float32),
               F=F.astype(np.float32), params=params)
        xs, prev = [], 0
        for f in frames:
            s.step(f - prev, record=True)
            xs.append(s.positions().double().cpu().numpy())
            prev = f
        dLdx = 2.0 * (np.stack(xs) - target) / (len(frames) * n)
        return s.backward(frames, torch.as_tensor(dLdx, dtype=torch.float32)).double().cpu().numpy()

    grads(xa, xa[None] + 0.001)
    st_a = s.stats()
    assert 0 < st_a["tape_grid_blocks"] < st_a["pool_blocks"] and st_a["tape_grid_reruns"] == 0, st_a
    target = xb[None] + np.array([0.0, -0.001, 0.0]) + 0.001 * rng.standard_normal((3, n, 3))
    g = grads(xb, target)
    st_b = s.stats()
    assert st_b["tape_grid_reruns"] == 1 and st_b["tape_grid_blocks"] == st_b["pool_blocks"], st_b
    s.close()
    cfg = orc.Cfg((R, R, R), dx, dt, (0.0, -9.8, 0.0))
    mat = orc.Material.from_table(vol, mid, mats, params)
    _, tape = orc.run(cfg, orc.new_state(xb, np.zeros((n, 3), np.float32), C.astype(np.float32), F.astype(np.float32)),
                      mat, 30, tape=True)
    _, dLdx_ref = orc.trajectory_loss(tape[frames][:, :, 0:3], target)
    _, g_ref = orc.backward(cfg, mat, tape, frames, dLdx_ref)
    for j in range(2):
        assert np.abs(g_ref[:, j]).max() > 0
        assert rel(g[:, j], g_ref[:, j]) < GRAD_TOL, (j, rel(g[:, j], g_ref[:, j]))


def test_reverse_pass_without_graphs_matches_graph_replay(sim_mod):
    """The reverse pass launched directly (the recompute of the previous
    segment forked onto the side stream with events, no captured graphs)
    gives the gradients of the graph-replayed reverse pass, for both tape
    modes: 40 substeps of the 512-particle ball, checkpoint every 10 (four
    segments), frames at 20 and 40, from a stressed seeded start."""
    sc = scenes.ball_512()
    v, C, F = scenes.key_frames(sc, 1, k_seed=66, vs=0.1, cs=1.0, fs=0.02)[0]
    dev = torch.device("cuda")
    init = {"x": torch.as_tensor(sc.x, device=dev), "v": torch.as_tensor(v, device=dev),
            "C": torch.as_tensor(C, device=dev), "F": torch.as_tensor(F, device=dev),
            "vol": torch.as_tensor(sc.vol, device=dev), "mat_id": torch.as_tensor(sc.mat_id, device=dev)}
    target = init["x"][None] + 0.002
    out = {}
    for tape_grid in (0, 1):
        for use_graph in (True, False):
            s = sim_mod.Simulator.from_scene(sc, ckpt_every=10, tape_grid=tape_grid)
            s.set_tuning(1, 128, use_graph)
            p = torch.as_tensor(sc.params, device=dev).clone().requires_grad_(True)
            xs = sim_mod.trajectory(p, s, init, [20, 40])
            (g,) = torch.autograd.grad(((xs - target) ** 2).sum(), p)
            s.sync()
            out[(tape_grid, use_graph)] = g.double().cpu().numpy()
            s.close()
    ref = out[(0, True)]
    assert np.abs(ref[:, 0]).max() > 0
    for k, g in out.items():
        for j in range(2):
            assert rel(g[:, j], ref[:, j]) < GRAD_TOL, (k, j, rel(g[:, j], ref[:, j]))


@pytest.mark.parametrize("tape_grid", [0, 1])
def test_fwd_bwd_captured_in_one_cuda_graph_both_tape_modes(sim_mod, tape_grid):
    """A whole fwd+bwd of the 512-particle ball (40 substeps, checkpoint
    every 10) captured by the caller with torch.cuda.graph, for both tape
    modes, replayed twice: the gradients of the run outside the capture."""
    sc = scenes.ball_512()
    v, C, F = scenes.key_frames(sc, 1, k_seed=67, vs=0.1, cs=1.0, fs=0.02)[0]
    dev = torch.device("cuda")
    init = {"x": torch.as_tensor(sc.x, device=dev), "v": torch.as_tensor(v, device=dev),
            "C": torch.as_tensor(C, device=dev), "F": torch.as_tensor(F, device=dev),
            "vol": torch.as_tensor(sc.vol, device=dev), "mat_id": torch.as_tensor(sc.mat_id, device=dev)}
    target = init["x"][None] + 0.002
    s = sim_mod.Simulator.from_scene(sc, ckpt_every=10, tape_grid=tape_grid)
    p = torch.as_tensor(sc.params, device=dev).clone().requires_grad_(True)

    def fb():
        xs = sim_mod.trajectory(p, s, init, [20, 40])
        (g,) = torch.autograd.grad(((xs - target) ** 2).sum(), p)
        return g

    ref = fb().double().cpu().numpy()
    fb()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = fb()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        r = out.double().cpu().numpy()
        for j in range(2):
            assert rel(r[:, j], ref[:, j]) < GRAD_TOL, (j, rel(r[:, j], ref[:, j]))
    s.sync()
    assert s.stats()["device_error"] == 0
    s.close()
