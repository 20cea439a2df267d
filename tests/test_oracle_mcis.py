"""Pins of the oracle's MCIS fill sampling (§4.1 steps 1-4): nearest-surface
distances against scipy's k-d tree (an independent algorithm), the weight at
points where its value is known (1 on the surface, 1/2 at sigma sqrt(2 ln 2),
eps beyond the cut-off), exact draws for equal weights, draw frequencies
against the normalized weights, and the independence of objects."""
import math

import numpy as np
import pytest

import oracle

SIGMA, EPS = 0.02, 1e-6


def test_distances_match_a_kd_tree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    surf = [rng.random((300, 3)), 0.5 + 0.1 * rng.random((200, 3))]
    cand = [rng.random((400, 3)), 0.45 + 0.2 * rng.random((300, 3))]
    r = oracle.mcis([0, 300, 500], np.concatenate(surf), [0, 400, 700], np.concatenate(cand), [0, 0, 0], [])
    for k in range(2):
        ref, _ = spatial.cKDTree(surf[k]).query(cand[k])
        got = r["d"][[0, 400][k]:[400, 700][k]]
        np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)


def test_weight_at_known_distances():
    surf = np.array([[0.5, 0.5, 0.5]])
    half = SIGMA * math.sqrt(2 * math.log(2))
    cut = SIGMA * math.sqrt(2 * math.log(1 / EPS))
    cand = np.array([[0.5, 0.5, 0.5], [0.5 + half, 0.5, 0.5], [0.5, 0.5 + 1.5 * cut, 0.5], [0.9, 0.1, 0.5]])
    r = oracle.mcis([0, 1], surf, [0, 4], cand, [0, 0], [])
    assert r["w"][0] == 1.0
    assert abs(r["w"][1] - 0.5) < 1e-15
    assert r["w"][2] == EPS and r["w"][3] == EPS
    # monotone in the distance
    dists = np.linspace(0, cut, 50)
    c2 = np.stack([0.5 + dists, np.full(50, 0.5), np.full(50, 0.5)], 1)
    w = oracle.mcis([0, 1], surf, [0, 50], c2, [0, 0], [])["w"]
    assert np.all(np.diff(w) <= 0)


def test_equal_weights_draw_floor_u_m():
    # every candidate beyond the cut-off: all weights eps, so draw i picks floor(u_i M)
    rng = np.random.default_rng(2)
    M = 1000
    cand = 0.1 + 0.05 * rng.random((M, 3))
    u = rng.random(5000)
    r = oracle.mcis([0, 1], [[0.9, 0.9, 0.9]], [0, M], cand, [0, 5000], u)
    np.testing.assert_array_equal(r["picked"], np.floor(u * M).astype(np.int64))


def test_draw_frequencies_follow_the_weights():
    rng = np.random.default_rng(3)
    surf = np.array([[0.5, 0.5, 0.5]])
    cand = 0.5 + np.array([[0.0, 0, 0], [0.01, 0, 0], [0.02, 0, 0], [0.03, 0, 0], [0.2, 0, 0]])
    n = 200000
    r = oracle.mcis([0, 1], surf, [0, 5], cand, [0, n], rng.random(n))
    p = r["w"] / r["w"].sum()
    freq = np.bincount(r["picked"], minlength=5) / n
    sd = np.sqrt(p * (1 - p) / n)
    assert np.all(np.abs(freq - p) < 5 * sd + 1e-6), (freq, p)
    assert r["cum"][-1] == sum(int(math.floor(w * 2 ** 40 + 0.5)) for w in r["w"])


def test_objects_are_independent_and_empty_objects_pick_nothing():
    rng = np.random.default_rng(4)
    surf = np.concatenate([0.2 + 0.01 * rng.random((20, 3)), 0.8 + 0.01 * rng.random((20, 3))])
    cand = np.concatenate([0.2 + 0.02 * rng.random((30, 3)), 0.8 + 0.02 * rng.random((30, 3))])
    r = oracle.mcis([0, 20, 40, 40], surf, [0, 30, 60, 60], cand, [0, 10, 20, 23], rng.random(23))
    assert np.all((r["picked"][:10] >= 0) & (r["picked"][:10] < 30))
    assert np.all((r["picked"][10:20] >= 30) & (r["picked"][10:20] < 60))
    assert np.all(r["picked"][20:] == -1)
    # object 0's candidates never see object 1's surface
    alone = oracle.mcis([0, 20], surf[:20], [0, 30], cand[:30], [0, 0], [])
    np.testing.assert_array_equal(alone["d"], r["d"][:30])
