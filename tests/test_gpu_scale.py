"""GPU tests of the batched form (64 instances, each on its own 64^3 grid),
the 2M-particle 256^3 block-sparse scene, CUDA-graph replay, the autotuner
and the per-material gradient reduction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_01723_gb300 import scenes  # noqa: E402


@pytest.fixture(scope="module")
def sim_mod():
    from __graft_entry__ import build
    build()
    from paper_2602_01723_gb300 import sim
    return sim


def test_graph_replay_matches_direct_launches(sim_mod):
    sc = scenes.cube_8k()
    out = []
    for g in (False, True):
        s = sim_mod.Simulator.from_scene(sc)
        s.set_tuning(1, 128, g)
        s.load_scene(sc)
        s.step(50)
        s.sync()
        out.append(s.positions().cpu().numpy())
        s.close()
    assert np.abs(out[0] - out[1]).max() < 1e-6 * sc.dx


def test_autotuner_picks_a_valid_setting_and_restores_the_state(sim_mod):
    sc = scenes.cube_8k()
    s = sim_mod.Simulator.from_scene(sc)
    s.load_scene(sc)
    x0 = s.positions().clone()
    r = s.autotune(10)
    assert r["scatter"] in (1, 2) and r["chunk"] in (32, 64, 96, 128) and r["best_us"] > 0
    assert torch.equal(s.positions(), x0)
    s.step(20)
    s.sync()
    s.close()


def test_batch_of_64_matches_single_instance_runs(sim_mod):
    """Instance b of the batch equals the same particles run alone (up to the
    order of floating-point reductions)."""
    sc = scenes.batch_64()
    s = sim_mod.Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(60)
    s.sync()
    xb = s.positions().cpu().numpy()
    st = s.stats()
    assert st["device_error"] == 0
    s.close()
    for b in (0, 17, 63):
        idx = np.nonzero(sc.instance == b)[0]
        s1 = sim_mod.Simulator(sc.grid_res, sc.dx, sc.dt, sc.gravity, [sc.materials[b]])
        s1.load(sc.x[idx], sc.vol[idx], np.zeros(len(idx), np.int32), v=sc.v[idx])
        s1.step(60)
        s1.sync()
        x1 = s1.positions().cpu().numpy()
        s1.close()
        assert np.abs(x1 - xb[idx]).max() < 1e-5 * sc.dx, b


def test_batch_gradients_per_instance(orc, sim_mod):
    """Per-instance (log E, nu, yield) gradients of the batched reverse pass:
    the per-material reduction equals a segmented sum of the per-particle
    gradients, and instance b's gradient equals the single-instance one.
    Frames at 70 and 90 substeps: after the floor contact (from substep ~53),
    where the gradients are physical rather than rounding noise."""
    sc = scenes.batch_64()
    frames = [70, 90]
    rng = np.random.default_rng(1)
    target = torch.as_tensor(sc.x[None] + 0.005 * rng.standard_normal((2, sc.n, 3)), dtype=torch.float32,
                             device="cuda")
    s = sim_mod.Simulator.from_scene(sc)
    init = {"x": sc.x, "v": sc.v, "vol": sc.vol, "mat_id": sc.mat_id, "instance": sc.instance}
    params = torch.tensor(np.stack([np.log([m["E"] for m in sc.materials]), [m["nu"] for m in sc.materials],
                                    [m["yield_stress"] for m in sc.materials]], axis=1)[sc.mat_id],
                          dtype=torch.float32, device="cuda", requires_grad=True)
    xs = sim_mod.trajectory(params, s, init, frames)
    loss = ((xs - target) ** 2).sum()
    loss.backward()
    per_inst = s.reduce_by_material(params.grad).cpu().numpy()
    ref = np.zeros((len(sc.materials), 3))
    np.add.at(ref, sc.mat_id, params.grad.double().cpu().numpy())
    assert np.abs(per_inst - ref).max() < 1e-4 * np.abs(ref).max()
    s.close()
    b = 5
    idx = np.nonzero(sc.instance == b)[0]
    s1 = sim_mod.Simulator(sc.grid_res, sc.dx, sc.dt, sc.gravity, [sc.materials[b]])
    p1 = params.detach()[idx].clone().requires_grad_(True)
    xs1 = sim_mod.trajectory(p1, s1, {"x": sc.x[idx], "v": sc.v[idx], "vol": sc.vol[idx],
                                      "mat_id": np.zeros(len(idx), np.int32)}, frames)
    ((xs1 - target[:, idx]) ** 2).sum().backward()
    g1 = p1.grad.double().cpu().numpy().sum(0)
    assert np.abs(g1 - per_inst[b]).max() < 1e-3 * np.abs(g1).max()
    s1.close()


def test_large_2m_block_sparse(orc, sim_mod):
    """2M particles on the 256^3 block-sparse grid: the P2G grid of a stressed
    seeded key frame against the oracle (dense FP64 grid) over all nodes;
    then 100 substeps from the scene's own start, with the active-block count
    against the grid's 262,144 blocks and the device memory used."""
    sc = scenes.large_2m()
    v, C, F = scenes.key_frames(sc, 1, k_seed=47, vs=0.5, cs=2.0, fs=0.05)[0]
    free0, total = torch.cuda.mem_get_info()
    s = sim_mod.Simulator.from_scene(sc)
    s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F)
    m, mv = s.debug_p2g()
    m = m[0].double().cpu().numpy()
    mv = mv[0].double().cpu().numpy()
    s.load_scene(sc)
    s.step(100)
    s.sync()
    free1, _ = torch.cuda.mem_get_info()
    st = s.stats()
    assert st["device_error"] == 0
    assert st["active_blocks"] < 0.2 * (256 // 4) ** 3
    used_gb = (free0 - free1) / 2 ** 30
    assert used_gb < 8.0, used_gb
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials)
    gm, gmv = orc.p2g(cfg, orc.new_state(sc.x, v, C, F), mat)
    floor = np.abs(gm).max() * 9.8 * sc.dt
    em = np.abs(m - gm).max() / max(np.abs(gm).max(), floor)
    emv = np.abs(mv - gmv).max() / max(np.abs(gmv).max(), floor)
    assert em < 1e-5 and emv < 1e-5, (em, emv)


def test_large_2m_per_object_gradient_matches_central_differences(sim_mod):
    """The 2M-particle scene's fwd+bwd at full size (256^3 block-sparse,
    checkpoint every 25, per-object gradients).  The oracle cannot run 2M
    particles, so this checks a property that holds at any size: the gradient
    of the loss with respect to one object's log E (the per-material sum of
    the per-particle gradients) equals the central difference of the loss
    itself, each side a full-size FP32 forward.  100 substeps (four
    segments), frames at 50 and 100, from a stressed seeded start so that the
    stress gradient is physical before the floor contact; objects 0 (elastic)
    and 4 (plasticine, below its yield strain here).  The sand objects are
    left out: their cone-tip projection switches under a finite step."""
    sc = scenes.large_2m()
    v, C, F = scenes.key_frames(sc, 1, k_seed=48, vs=0.1, cs=1.0, fs=0.02)[0]
    params = np.stack([np.log([m["E"] for m in sc.materials]), [m["nu"] for m in sc.materials],
                       [m["yield_stress"] for m in sc.materials]], axis=1)[sc.mat_id].astype(np.float32)
    frames = [50, 100]
    rng = np.random.default_rng(2)
    target = sc.x[None].astype(np.float64) + np.array([0.0, -0.005, 0.0]) + 0.002 * rng.standard_normal((2, sc.n, 3))
    s = sim_mod.Simulator.from_scene(sc)

    def run(p, record):
        s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F, params=p)
        xs, prev = [], 0
        for f in frames:
            s.step(f - prev, record=record)
            xs.append(s.positions().double().cpu().numpy())
            prev = f
        return np.stack(xs)

    def loss(xs):
        return float(((xs - target) ** 2).sum() / (len(frames) * sc.n))

    xs = run(params, True)
    dLdx = 2.0 * (xs - target) / (len(frames) * sc.n)
    g = s.backward(frames, torch.as_tensor(dLdx, dtype=torch.float32, device="cuda"))
    g_obj = s.reduce_by_material(g).double().cpu().numpy()
    assert s.stats()["device_error"] == 0
    h = 0.05
    for o in (0, 4):
        lv = []
        for sgn in (1.0, -1.0):
            p = params.copy()
            p[sc.mat_id == o, 0] += sgn * h
            lv.append(loss(run(p, False)))
        fd = (lv[0] - lv[1]) / (2 * h)
        assert abs(fd) > 0
        assert abs(g_obj[o, 0] - fd) < 0.03 * abs(fd), (o, g_obj[o, 0], fd)
    s.close()


def test_batched_fwd_bwd_captured_in_one_cuda_graph(sim_mod):
    """The 64-instance batch's whole fwd+bwd (load, recorded forward, frame
    positions, loss, reverse pass, per-instance reduction) captured in one
    CUDA graph with torch.cuda.graph and replayed: after two runs outside the
    capture (which allocate the checkpoints, tapes and adjoint buffers), the
    library launches straight into the caller's graph, with no allocation and
    no synchronisation.  Two replays give the per-instance gradients of the
    runs outside the capture (up to the order of floating-point reductions),
    and no device error is raised."""
    sc = scenes.batch_64()
    dev = torch.device("cuda")
    s = sim_mod.Simulator.from_scene(sc)
    init = {"x": torch.as_tensor(sc.x, device=dev), "v": torch.as_tensor(sc.v, device=dev),
            "vol": torch.as_tensor(sc.vol, device=dev),
            "mat_id": torch.as_tensor(sc.mat_id, dtype=torch.int32, device=dev),
            "instance": torch.as_tensor(sc.instance, dtype=torch.int32, device=dev)}
    params = torch.tensor(np.stack([np.log([m["E"] for m in sc.materials]), [m["nu"] for m in sc.materials],
                                    [m["yield_stress"] for m in sc.materials]], axis=1)[sc.mat_id],
                          dtype=torch.float32, device=dev, requires_grad=True)
    frames = [70, 90, 130, 200]
    target = init["x"][None] + 0.005

    def fb():
        xs = sim_mod.trajectory(params, s, init, frames)
        (g,) = torch.autograd.grad(((xs - target) ** 2).sum(), params)
        return s.reduce_by_material(g)

    ref = fb().double().cpu().numpy()
    fb()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = fb()
    reps = []
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        reps.append(out.double().cpu().numpy())
    s.sync()
    assert s.stats()["device_error"] == 0
    for r in reps:
        assert np.isfinite(r).all()
        assert np.abs(r - ref).max() < 1e-3 * np.abs(ref).max(), np.abs(r - ref).max() / np.abs(ref).max()
    s.close()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _smallest_of_each_kind(sc):
    """Instance ids of the smallest fixed-corotated, Neo-Hookean, plasticine
    (von Mises) and sand (Drucker-Prager) instance of a batched scene.  The
    plasticine one is the smallest whose yield strain sigma_y / (2 mu) is
    below 0.05, so that it yields within the run and its yield-stress
    gradient is not zero."""
    counts = np.bincount(sc.instance, minlength=sc.n_instances)
    kinds = {}
    for b in np.argsort(counts, kind="stable"):
        m = sc.materials[b]
        k = ("nh" if m["elastic"] == 1 else "fcr") if m["plastic"] == 0 else ("vm" if m["plastic"] == 1 else "dp")
        if k == "vm" and m["yield_stress"] / (m["E"] / (1.0 + m["nu"])) > 0.05:
            continue
        kinds.setdefault(k, int(b))
    return kinds


def test_batch_64_instances_match_the_oracle(orc, sim_mod):
    """The 64-instance batch (1.47M particles, each instance on its own 64^3
    grid) as one context: 200 substeps, recorded, then the reverse pass of
    seeded cotangents at the ten frames (every 20 substeps) and the
    per-instance reduction.  For the smallest instance of each material kind
    the oracle runs that instance alone on its own grid (the instances are
    independent problems, §4.2: one parameter set per instance label):
    positions after 200 substeps within 1e-4 dx, per-particle gradients and
    the per-instance sums within 1e-3 relative per parameter kind."""
    sc = scenes.batch_64()
    frames = [int(f) for f in sc.frame_sub]
    cot = np.random.default_rng(64).standard_normal((len(frames), sc.n, 3)).astype(np.float32)
    s = sim_mod.Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(sc.n_substeps, record=True)
    x = s.positions().double().cpu().numpy()
    g = s.backward(frames, torch.as_tensor(cot))
    g_inst = s.reduce_by_material(g).double().cpu().numpy()
    g = g.double().cpu().numpy()
    assert s.stats()["device_error"] == 0
    s.close()
    for kind, b in sorted(_smallest_of_each_kind(sc).items()):
        idx = np.nonzero(sc.instance == b)[0]
        cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
        mat = orc.Material.from_table(sc.vol[idx], np.zeros(len(idx), np.int32), [sc.materials[b]])
        _, tape = orc.run(cfg, orc.new_state(sc.x[idx], sc.v[idx]), mat, sc.n_substeps, tape=True)
        ex = np.abs(x[idx] - tape[sc.n_substeps][:, 0:3]).max() / sc.dx
        _, g_ref = orc.backward(cfg, mat, tape, frames, cot[:, idx].astype(np.float64))
        kinds = [0, 1, 2] if kind == "vm" else [0, 1]
        eg = [_rel(g[idx, j], g_ref[:, j]) for j in kinds]
        es = [abs(g_inst[b, j] - g_ref[:, j].sum()) / np.abs(g_ref[:, j]).sum() for j in kinds]
        print("instance %d (%s, %d particles): x %.3g dx, grads %s, sums %s"
              % (b, kind, len(idx), ex, ["%.3g" % e for e in eg], ["%.3g" % e for e in es]))
        assert ex < 1e-4, (kind, ex)
        for j, e in zip(kinds, eg):
            assert np.abs(g_ref[:, j]).max() > 0
            assert e < 1e-3, (kind, j, e)
        assert max(es) < 1e-3, (kind, es)


def test_large_sparse_scene_on_the_256_grid_matches_the_oracle(orc, sim_mod):
    """The 8-object large scene with 20,000 particles (2,500 per object) on
    the full 256^3 block-sparse grid, dt 2e-5, checkpoint every 25: 100
    substeps from a slightly stressed seeded start (so that the stress
    gradient is physical before any contact), recorded, then the reverse pass
    of seeded cotangents at substeps 25, 50, 75, 100 and the per-object
    reduction by material id.  The plasticine objects' yield stress is
    lowered to 100 (yield strain 0.013), so that they yield from the stressed
    start and their yield-stress gradient is not zero.  The oracle holds the
    256^3 grid densely in FP64.  Positions within 1e-4 dx; per-particle
    gradients and per-object sums within 1e-3 relative per parameter kind."""
    sc = scenes.large_2m(20_000)
    for m in sc.materials:
        if m["plastic"] == scenes.PLASTIC_VM:
            m["yield_stress"] = 100.0
    v, C, F = scenes.key_frames(sc, 1, k_seed=49, vs=0.1, cs=1.0, fs=0.02)[0]
    params = np.stack([np.log([m["E"] for m in sc.materials]), [m["nu"] for m in sc.materials],
                       [m["yield_stress"] for m in sc.materials]], axis=1)[sc.mat_id].astype(np.float32)
    frames = [25, 50, 75, 100]
    cot = np.random.default_rng(256).standard_normal((len(frames), sc.n, 3)).astype(np.float32)
    s = sim_mod.Simulator.from_scene(sc)
    assert s.grid_res == (256, 256, 256)
    s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F, params=params)
    s.step(100, record=True)
    x = s.positions().double().cpu().numpy()
    g = s.backward(frames, torch.as_tensor(cot))
    g_obj = s.reduce_by_material(g).double().cpu().numpy()
    g = g.double().cpu().numpy()
    st = s.stats()
    assert st["device_error"] == 0 and st["active_blocks"] < 0.01 * (256 // 4) ** 3, st
    s.close()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, params)
    _, tape = orc.run(cfg, orc.new_state(sc.x, v, C, F), mat, 100, tape=True)
    _, g_ref = orc.backward(cfg, mat, tape, frames, cot.astype(np.float64))
    ex = np.abs(x - tape[100][:, 0:3]).max() / sc.dx
    ref_obj = np.zeros((len(sc.materials), 3))
    np.add.at(ref_obj, sc.mat_id, g_ref)
    eg = [_rel(g[:, j], g_ref[:, j]) for j in range(3)]
    eo = [_rel(g_obj[:, j], ref_obj[:, j]) for j in range(3)]
    print("large scene 20k on 256^3: x %.3g dx, grads %s, per object %s"
          % (ex, ["%.3g" % e for e in eg], ["%.3g" % e for e in eo]))
    assert ex < 1e-4, ex
    for j in range(3):
        assert np.abs(g_ref[:, j]).max() > 0
        assert eg[j] < 1e-3 and eo[j] < 1e-3, (j, eg[j], eo[j])
