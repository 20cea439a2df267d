"""GPU parity of the MCIS fill sampling (§4.1 steps 1-4) against the FP64
oracle on the same seeded inputs: exact nearest-surface distances below the
cut-off, weights (both in FP64; 1e-14 relative covers one rounding of exp),
and the drawn candidate indices, which are integer decisions taken on both
sides from integer cumulative weights (bit-exact).  At full size the oracle
checks a sample of candidates one by one and every draw is checked against
the GPU's own weights."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2602_01723_gb300 import scenes  # noqa: E402

SIGMA, EPS = 0.02, 1e-6
CUT = SIGMA * math.sqrt(2 * math.log(1 / EPS))


@pytest.fixture(scope="module")
def sim_mod():
    from __graft_entry__ import build
    build()
    from paper_2602_01723_gb300 import sim
    return sim


def run_gpu(sim_mod, c, host=False):
    if host:
        import ctypes
        from paper_2602_01723_gb300 import _lib as L
        nc, nd = int(c["cand_off"][-1]), int(c["draw_off"][-1])
        d, w, p = np.zeros(nc), np.zeros(nc), np.zeros(nd, dtype=np.int64)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        surf = np.ascontiguousarray(c["surf"], np.float32)
        cand = np.ascontiguousarray(c["cand"], np.float32)
        u = np.ascontiguousarray(c["u"], np.float64)
        L.mpm_mcis(c["surf_off"], vp(surf), c["cand_off"], vp(cand), c["draw_off"], vp(u), SIGMA, EPS, vp(d), vp(w),
                   vp(p), ctypes.c_void_p(0))
        return {"d": d, "w": w, "picked": p}
    out = sim_mod.mcis(c["surf_off"], c["surf"], c["cand_off"], c["cand"], c["draw_off"], c["u"], SIGMA, EPS)
    return {k: v.cpu().numpy() for k, v in out.items()}


def check(got, ref):
    near = ref["d"] < CUT
    assert near.any()
    np.testing.assert_allclose(got["d"][near], ref["d"][near], rtol=1e-15, atol=0)
    np.testing.assert_allclose(got["w"], ref["w"], rtol=1e-14, atol=0)
    np.testing.assert_array_equal(got["picked"], ref["picked"])


@pytest.mark.parametrize("host", [False, True])
def test_mcis_matches_the_oracle(orc, sim_mod, host):
    c = scenes.mcis_case((700, 500, 600), (3000, 2500, 2000), (400, 300, 200), k_seed=71)
    ref = orc.mcis(c["surf_off"], c["surf"], c["cand_off"], c["cand"], c["draw_off"], c["u"], SIGMA, EPS)
    check(run_gpu(sim_mod, c, host), ref)


def test_mcis_edge_cases(orc, sim_mod):
    """An object with no candidates, one with no surface points (all weights
    eps: draws are floor(u M)), one candidate on a surface point, and
    coordinates slightly outside the unit cube."""
    rng = np.random.default_rng(5)
    surf = np.array([[0.5, 0.5, 0.5], [1.01, 0.2, 0.2], [-0.01, 0.3, 0.3]], np.float32)
    cand = np.concatenate([[[0.5, 0.5, 0.5], [0.99, 0.2, 0.2], [0.02, 0.3, 0.31]],
                           0.4 + 0.2 * rng.random((50, 3))]).astype(np.float32)
    c = {"surf_off": np.array([0, 3, 3, 3]), "surf": surf, "cand_off": np.array([0, 53, 53, 60]),
         "cand": np.concatenate([cand, 0.1 + 0.1 * rng.random((7, 3)).astype(np.float32)]),
         "draw_off": np.array([0, 40, 45, 60]), "u": rng.random(60)}
    ref = orc.mcis(c["surf_off"], c["surf"], c["cand_off"], c["cand"], c["draw_off"], c["u"], SIGMA, EPS)
    got = run_gpu(sim_mod, c)
    assert got["w"][0] == 1.0 and np.all(got["picked"][40:45] == -1)
    np.testing.assert_array_equal(got["picked"][45:], 53 + np.floor(c["u"][45:] * 7).astype(np.int64))
    near = ref["d"] < CUT
    np.testing.assert_allclose(got["d"][near], ref["d"][near], rtol=1e-15)
    np.testing.assert_allclose(got["w"], ref["w"], rtol=1e-14)
    np.testing.assert_array_equal(got["picked"], ref["picked"])


def test_mcis_full_size_three_objects(orc, sim_mod):
    """The three objects of the 300k scene at full size (108k surface points,
    750k candidates, 192k draws): 1,500 sampled candidates against the
    oracle's brute force over their object's surface, and every draw against
    the inverse CDF of the GPU's own weights."""
    c = scenes.mcis_case()
    got = run_gpu(sim_mod, c)
    rng = np.random.default_rng(9)
    so, co, do = c["surf_off"], c["cand_off"], c["draw_off"]
    for k in range(3):
        idx = co[k] + rng.choice(co[k + 1] - co[k], 500, replace=False)
        sub = orc.mcis([0, so[k + 1] - so[k]], c["surf"][so[k]:so[k + 1]], [0, 500], c["cand"][idx], [0, 0], [],
                       SIGMA, EPS)
        near = sub["d"] < CUT
        np.testing.assert_allclose(got["d"][idx][near], sub["d"][near], rtol=1e-15)
        np.testing.assert_allclose(got["w"][idx], sub["w"], rtol=1e-14)
        # draws: the inverse CDF of the GPU weights, in exact integers
        wq = np.floor(got["w"][co[k]:co[k + 1]] * 2.0 ** 40 + 0.5).astype(np.int64)
        cum = np.cumsum(wq)
        t = np.floor(c["u"][do[k]:do[k + 1]] * float(cum[-1])).astype(np.int64)
        expect = co[k] + np.minimum(np.searchsorted(cum, t, side="right"), len(cum) - 1)
        np.testing.assert_array_equal(got["picked"][do[k]:do[k + 1]], expect)
