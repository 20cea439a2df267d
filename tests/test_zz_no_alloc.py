"""mpm_substep_noalloc: the one-substep entry point for callers that cannot
allocate device memory (its grid lives in a fixed-size device array inside
libmpm).  Checked through the C ABI against the context-based entry points
(mpm_load_particles + mpm_step(1) + mpm_get_particles) on two calls in a row,
so that stale scratch from the first call would show up in the second.

This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _scene():
    from paper_2602_01723_gb300 import scenes
    sc = scenes.cube_8k()
    sc.materials = [scenes.material(0, 0, 1e4, 0.3, 10.0), scenes.material(1, 0, 2e4, 0.3, 10.0),
                    scenes.material(0, 1, 1e4, 0.3, 10.0, yield_stress=50.0), scenes.material(0, 2, 1e4, 0.25, 10.0)]
    sc.mat_id = (np.arange(sc.n) % 4).astype(np.int32)
    rng = np.random.default_rng(17)
    v = (0.5 * rng.standard_normal((sc.n, 3))).astype(np.float32)
    C = (3.0 * rng.standard_normal((sc.n, 3, 3))).astype(np.float32)
    F = np.array([np.eye(3) + 0.05 * rng.standard_normal((3, 3)) for _ in range(sc.n)], dtype=np.float32)
    return sc, v, C, F


def _materials(table):
    from paper_2602_01723_gb300 import _lib as L
    arr = (L.mpm_material * len(table))()
    for i, t in enumerate(table):
        arr[i] = L.mpm_material(t["elastic"], t["plastic"], t["E"], t["nu"], t["rho"], t["yield_stress"],
                                t["friction_angle_deg"])
    return arr


def _noalloc(sc, state, res=None):
    from paper_2602_01723_gb300 import _lib as L
    dev = torch.device("cuda")
    x = torch.as_tensor(state["x"], device=dev).contiguous()
    v = torch.as_tensor(state["v"], device=dev).contiguous()
    C = torch.as_tensor(state["C"], device=dev).reshape(-1, 9).contiguous()
    F = torch.as_tensor(state["F"], device=dev).reshape(-1, 9).contiguous()
    vol = torch.as_tensor(sc.vol, device=dev).contiguous()
    mid = torch.as_tensor(sc.mat_id, dtype=torch.int32, device=dev).contiguous()
    out = [torch.empty_like(x), torch.empty_like(v), torch.empty_like(C), torch.empty_like(F)]
    r = res or (sc.grid_res,) * 3
    st = L.lib().mpm_substep_noalloc((ctypes.c_int32 * 3)(*r), sc.dx, sc.dt, (ctypes.c_float * 3)(*sc.gravity),
                                     _materials(sc.materials), len(sc.materials), None, sc.n, _p(x), _p(v), _p(C),
                                     _p(F), _p(vol), _p(mid), *[_p(o) for o in out],
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, {"x": out[0].cpu().numpy(), "v": out[1].cpu().numpy(), "C": out[2].cpu().numpy().reshape(-1, 3, 3),
                "F": out[3].cpu().numpy().reshape(-1, 3, 3)}


def _context_step(sc, state):
    from paper_2602_01723_gb300.sim import Simulator
    s = Simulator.from_scene(sc)
    s.load(state["x"], sc.vol, sc.mat_id, v=state["v"], C=state["C"], F=state["F"])
    s.step(1)
    s.sync()
    out = {k: t.cpu().numpy() for k, t in s.get().items()}
    s.close()
    return out


def _errors(a, b, sc):
    return (np.abs(a["x"] - b["x"]).max() / sc.dx, np.abs(a["v"] - b["v"]).max() / np.abs(b["v"]).max(),
            np.abs(a["C"] - b["C"]).max() / np.abs(b["C"]).max(), np.abs(a["F"] - b["F"]).max())


# the suite's one-substep tolerances against the FP64 oracle: positions
# 1e-4 dx, v and C 1e-5 relative, F 2e-5 absolute
TOL = (1e-4, 1e-5, 1e-5, 2e-5)


def _oracle_step(sc, state):
    import oracle
    cfg = oracle.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = oracle.Material.from_table(sc.vol, sc.mat_id, sc.materials)
    st = oracle.new_state(*[np.asarray(state[k], dtype=np.float64) for k in ("x", "v", "C", "F")])
    return oracle.substep(cfg, st, mat)


def _close(noalloc, context, ref, sc):
    e_ref = _errors(noalloc, ref, sc)
    e_ctx = _errors(noalloc, context, sc)
    msg = "vs oracle %s, vs context path %s" % (["%.3g" % e for e in e_ref], ["%.3g" % e for e in e_ctx])
    assert all(e < t for e, t in zip(e_ref, TOL)), msg
    # both FP32 paths are within TOL of the oracle, so they differ by < 2 TOL
    assert all(e < 2 * t for e, t in zip(e_ctx, TOL)), msg


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    from __graft_entry__ import build
    build()
    sc, v, C, F = _scene()
    s0 = {"x": sc.x, "v": v, "C": C, "F": F}
    st, n1 = _noalloc(sc, s0)
    assert st == 0
    _close(n1, _context_step(sc, s0), _oracle_step(sc, s0), sc)
    st, n2 = _noalloc(sc, n1)          # second call: the scratch holds the first call's grid
    assert st == 0
    # against the oracle's own two substeps from the seeded state (two
    # substeps' error: within twice the one-substep bound), and against the
    # context path applied to the same input
    ref2 = _oracle_step(sc, _oracle_step(sc, s0))
    e_ref = _errors(n2, ref2, sc)
    assert all(e < 2 * t for e, t in zip(e_ref, TOL)), e_ref
    e_ctx = _errors(n2, _context_step(sc, n1), sc)
    assert all(e < 2 * t for e, t in zip(e_ctx, TOL)), e_ctx


def test_noalloc_rejects_grids_beyond_its_scratch():
    from __graft_entry__ import build
    from paper_2602_01723_gb300 import _lib as L
    build()
    sc, v, C, F = _scene()
    st, _ = _noalloc(sc, {"x": sc.x, "v": v, "C": C, "F": F}, res=(128, 128, 32))
    assert st == 8   # MPM_ERR_CAPACITY: 128*128*32 nodes > MPM_NOALLOC_MAX_NODES
    assert L.STATUS_NAMES[st] == "MPM_ERR_CAPACITY"


def test_noalloc_error_word_does_not_leak_into_the_next_call():
    """The scratch's error word is shared by every call, like its grid.  A
    first call with one particle outside the grid (x = 0.01, whose stencil
    would start at node -1) returns MPM_ERR_OUT_OF_DOMAIN; the next call, with
    the valid seeded state on the same stream, returns MPM_OK and matches the
    oracle: each call clears the error word before it runs."""
    from __graft_entry__ import build
    build()
    sc, v, C, F = _scene()
    bad_x = sc.x.copy()
    bad_x[5] = [0.01, 0.5, 0.5]
    st, _ = _noalloc(sc, {"x": bad_x, "v": v, "C": C, "F": F})
    assert st == 4                                    # MPM_ERR_OUT_OF_DOMAIN
    s0 = {"x": sc.x, "v": v, "C": C, "F": F}
    st, n1 = _noalloc(sc, s0)
    assert st == 0
    e_ref = _errors(n1, _oracle_step(sc, s0), sc)
    assert all(e < t for e, t in zip(e_ref, TOL)), e_ref
