"""Seeded synthetic particle scenes shaped like the paper's workloads.

This module only draws inputs: positions, velocities, particle volumes,
material ids, a material table and optional per-particle parameters.  It holds
none of the simulation arithmetic, imports neither the CUDA binding nor the
oracle, and is the one module both sides consume.

The paper's 3DGS scenes (PhysGaussian, Physics3D, PhysDreamer data and the
multi-object set, §5.1 "Datasets") are not available; these generators stand in
for them.  Every scene sits in the unit cube (App. C.1 normalises each scene to
1x1x1), and each object is a Gaussian-splat-like surface shell plus interior
points on a half-cell lattice, as the Instance-aware Particle Filling of §4.1
produces.

Seeds: ``numpy.random.Generator(PCG64(2602_01723 + k))`` for workload k.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 2602_01723

ELASTIC_FCR, ELASTIC_NH = 0, 1
PLASTIC_NONE, PLASTIC_VM, PLASTIC_DP = 0, 1, 2


def material(elastic=ELASTIC_FCR, plastic=PLASTIC_NONE, E=1e4, nu=0.3, rho=1.0, yield_stress=0.0,
             friction_angle_deg=30.0):
    return dict(elastic=int(elastic), plastic=int(plastic), E=float(E), nu=float(nu), rho=float(rho),
                yield_stress=float(yield_stress), friction_angle_deg=float(friction_angle_deg))


@dataclasses.dataclass
class Scene:
    name: str
    grid_res: int
    dt: float
    n_substeps: int
    x: np.ndarray                      # (n,3) float32
    v: np.ndarray                      # (n,3) float32
    vol: np.ndarray                    # (n,) float32
    mat_id: np.ndarray                 # (n,) int32 index into materials
    materials: List[dict]
    params: Optional[np.ndarray] = None     # (n,3) float32 per-particle (logE, nu, yield) or None
    instance: Optional[np.ndarray] = None   # (n,) int32 instance id (batched scenes)
    n_instances: int = 1
    gravity: tuple = (0.0, -9.8, 0.0)
    ckpt_every: int = 0
    frame_sub: Optional[np.ndarray] = None  # substep index of each loss frame
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self):
        return int(self.x.shape[0])

    @property
    def dx(self):
        return 1.0 / self.grid_res


def _rng(k):
    return np.random.Generator(np.random.PCG64(SEED_BASE + k))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# --------------------------------------------------------------------------
# shapes: inside tests and uniform surface samples with unit normals
# --------------------------------------------------------------------------

class Sphere:
    def __init__(self, c, r):
        self.c, self.r = np.asarray(c, float), float(r)

    def bbox(self):
        return self.c - self.r, self.c + self.r

    def inside(self, p):
        return np.linalg.norm(p - self.c, axis=1) < self.r

    def area(self):
        return 4 * math.pi * self.r ** 2

    def volume(self):
        return 4.0 / 3.0 * math.pi * self.r ** 3

    def surface(self, n, rng):
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return self.c + self.r * d, d


class Torus:
    """Torus lying flat (axis along y): major radius R, tube radius r."""

    def __init__(self, c, R, r):
        self.c, self.R, self.r = np.asarray(c, float), float(R), float(r)

    def bbox(self):
        e = np.array([self.R + self.r, self.r, self.R + self.r])
        return self.c - e, self.c + e

    def inside(self, p):
        q = p - self.c
        rho = np.sqrt(q[:, 0] ** 2 + q[:, 2] ** 2)
        return (rho - self.R) ** 2 + q[:, 1] ** 2 < self.r ** 2

    def area(self):
        return 4 * math.pi ** 2 * self.R * self.r

    def volume(self):
        return 2 * math.pi ** 2 * self.R * self.r ** 2

    def surface(self, n, rng):
        out_u, out_v = [], []
        got = 0
        while got < n:
            m = 2 * (n - got) + 16
            u = rng.uniform(0, 2 * math.pi, m)
            v = rng.uniform(0, 2 * math.pi, m)
            keep = rng.uniform(0, 1, m) < (self.R + self.r * np.cos(v)) / (self.R + self.r)
            out_u.append(u[keep]); out_v.append(v[keep]); got += int(keep.sum())
        u = np.concatenate(out_u)[:n]; v = np.concatenate(out_v)[:n]
        nrm = np.stack([np.cos(v) * np.cos(u), np.sin(v), np.cos(v) * np.sin(u)], axis=1)
        ring = np.stack([np.cos(u), np.zeros_like(u), np.sin(u)], axis=1)
        return self.c + self.R * ring + self.r * nrm, nrm


class Box:
    def __init__(self, c, half):
        self.c, self.h = np.asarray(c, float), float(half)

    def bbox(self):
        return self.c - self.h, self.c + self.h

    def inside(self, p):
        return np.all(np.abs(p - self.c) < self.h, axis=1)

    def area(self):
        return 24 * self.h ** 2

    def volume(self):
        return 8 * self.h ** 3

    def surface(self, n, rng):
        face = rng.integers(0, 6, n)
        ax, sgn = face // 2, np.where(face % 2 == 0, -1.0, 1.0)
        uv = rng.uniform(-self.h, self.h, (n, 3))
        uv[np.arange(n), ax] = sgn * self.h
        nrm = np.zeros((n, 3))
        nrm[np.arange(n), ax] = sgn
        return self.c + uv, nrm


def _lattice_inside(shape, h, jitter, rng):
    lo, hi = shape.bbox()
    axes = [np.arange(lo[d] + 0.5 * h, hi[d], h) for d in range(3)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    g = g[shape.inside(g)]
    return g + rng.uniform(-jitter, jitter, g.shape)


def _shell(shape, n, sigma_n, rng):
    p, nrm = shape.surface(n, rng)
    return p + nrm * rng.normal(0.0, sigma_n, (n, 1))


def shell_plus_interior(shapes, n_total, dx, rng):
    """Interior lattice at spacing dx/2 with +-dx/8 jitter inside each shape,
    plus surface-shell points split by area so that the total is exactly
    n_total (interior subsampled when it alone exceeds 85% of n_total).
    Returns (points, object index)."""
    h = dx / 2.0
    interiors = [_lattice_inside(s, h, dx / 8.0, rng) for s in shapes]
    n_int = sum(len(a) for a in interiors)
    cap = int(0.85 * n_total)
    if n_int > cap:
        keep = rng.choice(n_int, cap, replace=False)
        allp = np.concatenate(interiors)
        owner = np.concatenate([np.full(len(a), i) for i, a in enumerate(interiors)])
        keep.sort()
        interiors = [allp[keep][owner[keep] == i] for i in range(len(shapes))]
        n_int = cap
    n_shell = n_total - n_int
    areas = np.array([s.area() for s in shapes])
    split = np.floor(n_shell * areas / areas.sum()).astype(int)
    split[-1] += n_shell - split.sum()
    pts, obj = [], []
    for i, s in enumerate(shapes):
        sh = _shell(s, int(split[i]), 0.1 * dx, rng)
        pts += [interiors[i], sh]
        obj += [np.full(len(interiors[i]), i), np.full(len(sh), i)]
    return np.concatenate(pts), np.concatenate(obj).astype(np.int32)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def cube_8k() -> Scene:
    """8,192 particles: 16^3 strata of side 0.0125 tiling [0.4,0.6]^3, two
    uniform points per stratum; 32^3 grid, dt 1e-4, 100 substeps;
    fixed-corotated E 1e4, nu 0.3, rho 1, V_p = (dx/2)^3; at rest; sticky floor."""
    rng = _rng(1)
    R = 32
    s = 0.2 / 16
    idx = np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = np.repeat(0.4 + idx * s, 2, axis=0) + rng.uniform(0, s, (idx.shape[0] * 2, 3))
    n = len(x)
    return Scene("cube_8k", R, 1e-4, 100, _f32(x), _f32(np.zeros((n, 3))), _f32(np.full(n, (0.5 / R) ** 3)),
                 np.zeros(n, np.int32), [material(ELASTIC_FCR, PLASTIC_NONE, 1e4, 0.3, 1.0)])


def three_objects_300k(n_total=300_000) -> Scene:
    """300k particles in three objects on a 128^3 grid (sphere: elastic with
    E log-uniform in [1e3,1e5]; torus: plasticine, von Mises yield 1e3; box:
    sand, Drucker-Prager 30 deg), dt 5e-5, 2,000 substeps, v0 = (0,-1,0)."""
    rng = _rng(2)
    R = 128
    dx = 1.0 / R
    shapes = [Sphere((0.2, 0.20, 0.5), 0.10), Torus((0.5, 0.14, 0.5), 0.10, 0.04), Box((0.8, 0.18, 0.5), 0.08)]
    x, obj = shell_plus_interior(shapes, n_total, dx, rng)
    E_sphere = float(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
    mats = [material(ELASTIC_FCR, PLASTIC_NONE, E_sphere, 0.3, 100.0),
            material(ELASTIC_FCR, PLASTIC_VM, 1e4, 0.3, 100.0, yield_stress=1e3),
            material(ELASTIC_FCR, PLASTIC_DP, 1e4, 0.3, 100.0, friction_angle_deg=30.0)]
    n = len(x)
    v = np.tile([0.0, -1.0, 0.0], (n, 1))
    return Scene("three_objects_300k", R, 5e-5, 2000, _f32(x), _f32(v), _f32(np.full(n, (0.5 * dx) ** 3)),
                 obj, mats)


def _jittered_ball(n, center, radius, rng):
    h = (4.0 / 3.0 * math.pi * radius ** 3 / n) ** (1.0 / 3.0)
    c = np.asarray(center)
    k = int(math.ceil(radius / h)) + 1
    ax = np.arange(-k, k + 1) * h
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = g + rng.uniform(-h / 2, h / 2, g.shape)
    g = g[np.linalg.norm(g, axis=1) < radius]
    g = g[rng.permutation(len(g))]
    if len(g) >= n:
        g = g[:n]
    else:
        extra = []
        while sum(len(e) for e in extra) < n - len(g):
            q = rng.uniform(-radius, radius, (2 * n, 3))
            extra.append(q[np.linalg.norm(q, axis=1) < radius])
        g = np.concatenate([g] + extra)[:n]
    return c + g, h


def _diff_ball(name, n, R, center, k_seed, n_sub=400):
    rng = _rng(k_seed)
    x, h = _jittered_ball(n, center, 0.15, rng)
    gt = np.stack([rng.normal(np.log(5e3), 0.5, n), rng.uniform(0.2, 0.4, n), np.zeros(n)], axis=1)
    guess = np.stack([np.full(n, np.log(5e3)), np.full(n, 0.3), np.zeros(n)], axis=1)
    v = np.tile([0.0, -1.0, 0.0], (n, 1))
    frames = np.arange(1, 11) * (n_sub // 10)
    sc = Scene(name, R, 1e-4, n_sub, _f32(x), _f32(v), _f32(np.full(n, h ** 3)), np.zeros(n, np.int32),
               [material(ELASTIC_FCR, PLASTIC_NONE, 5e3, 0.3, 100.0)], params=_f32(guess), ckpt_every=20,
               frame_sub=frames.astype(np.int32))
    sc.extra["params_true"] = _f32(gt)
    return sc


def ball_50k() -> Scene:
    """50k particles in a jittered ball r 0.15 at (0.5,0.21,0.5); 64^3 grid;
    400 substeps of 1e-4; checkpoint every 20; per-particle ground truth
    log E ~ N(log 5e3, 0.5), nu ~ U(0.2,0.4); guess log 5e3, 0.3; loss frames
    every 40 substeps."""
    return _diff_ball("ball_50k", 50_000, 64, (0.5, 0.21, 0.5), 3)


def ball_512() -> Scene:
    """512-particle, 16^3 copy of ball_50k for finite-difference checks."""
    return _diff_ball("ball_512", 512, 16, (0.5, 0.36, 0.5), 13)


def _object_scene(name, k_seed, R, counts, dt, n_sub, placements, mats_for, floor_gap):
    rng = _rng(k_seed)
    dx = 1.0 / R
    xs, objs, inst = [], [], []
    cycle = [Sphere, Torus, Box]
    for b, nb in enumerate(counts):
        # size the shape so the half-cell interior holds about 65% of nb
        vol = 0.65 * nb * (dx / 2) ** 3
        kind = cycle[b % 3]
        c = placements[b]
        if kind is Sphere:
            shape = Sphere(c, (vol * 3 / (4 * math.pi)) ** (1 / 3))
        elif kind is Torus:
            r = (vol / (2 * math.pi ** 2 * 2.5)) ** (1 / 3)
            shape = Torus(c, 2.5 * r, r)
        else:
            shape = Box(c, 0.5 * vol ** (1 / 3))
        lo, _ = shape.bbox()
        shape.c = shape.c + np.array([0.0, floor_gap - lo[1], 0.0])    # bottom at y = floor_gap
        p, _ = shell_plus_interior([shape], int(nb), dx, rng)
        xs.append(p); inst.append(np.full(len(p), b, np.int32))
    x = np.concatenate(xs)
    instance = np.concatenate(inst)
    mats = mats_for(rng, len(counts))
    n = len(x)
    v = np.zeros((n, 3))
    return x, v, instance, mats, dx


def batch_64() -> Scene:
    """64 instances, each on its own 64^3 grid, particle counts uniform in
    2k..40k, shapes cycling sphere/torus/box; per-instance material type
    uniform over {FCR, Neo-Hookean, plasticine, sand}, E log-U[1e3,1e5],
    nu U(0.2,0.4), yield log-U[3e2,3e3], rho 100; bottoms at y 0.06,
    v0 = (0,-1,0); 200 substeps of 1e-4."""
    rng = _rng(4)
    B = 64
    counts = rng.integers(2000, 40001, B)
    R = 64

    def mats_for(r, nb):
        out = []
        kinds = r.integers(0, 4, nb)
        for b in range(nb):
            E = float(np.exp(r.uniform(np.log(1e3), np.log(1e5))))
            nu = float(r.uniform(0.2, 0.4))
            ys = float(np.exp(r.uniform(np.log(3e2), np.log(3e3))))
            k = int(kinds[b])
            el = ELASTIC_NH if k == 1 else ELASTIC_FCR
            pl = {0: PLASTIC_NONE, 1: PLASTIC_NONE, 2: PLASTIC_VM, 3: PLASTIC_DP}[k]
            out.append(material(el, pl, E, nu, 100.0, yield_stress=ys, friction_angle_deg=30.0))
        return out

    place = [(0.5, 0.5, 0.5)] * B
    x, v, inst, mats, dx = _object_scene("batch_64", 4, R, counts, 1e-4, 200, place, mats_for, 0.06)
    n = len(x)
    v[:, 1] = -1.0
    frames = (np.arange(1, 11) * 20).astype(np.int32)
    sc = Scene("batch_64", R, 1e-4, 200, _f32(x), _f32(v), _f32(np.full(n, (0.5 * dx) ** 3)), inst.copy(), mats,
               instance=inst, n_instances=B, frame_sub=frames, ckpt_every=20)
    # target parameters: a second seeded draw of the same ranges
    sc.extra["materials_target"] = mats_for(_rng(104), B)
    return sc


def large_2m(n_total=2_000_000) -> Scene:
    """2M particles from 8 shell-plus-interior objects on a 256^3 grid
    (block-sparse, 4^3 tiles), 500 substeps of 2e-5, checkpoint every 25,
    materials cycling elastic / plasticine / sand, rho 100; bottoms at
    y 0.02, v0 = (0,-1,0)."""
    R = 256
    counts = np.full(8, n_total // 8)
    counts[-1] += n_total - counts.sum()
    place = [(0.2 + 0.2 * (b % 4), 0.0, 0.3 + 0.4 * (b // 4)) for b in range(8)]

    def mats_for(r, nb):
        out = []
        for b in range(nb):
            k = b % 3
            pl = [PLASTIC_NONE, PLASTIC_VM, PLASTIC_DP][k]
            out.append(material(ELASTIC_FCR, pl, 1e4 if k else 3e4, 0.3, 100.0, yield_stress=1e3,
                                friction_angle_deg=30.0))
        return out

    x, v, inst, mats, dx = _object_scene("large_2m", 5, R, counts, 2e-5, 500, place, mats_for, 0.02)
    n = len(x)
    v[:, 1] = -1.0
    return Scene("large_2m", R, 2e-5, 500, _f32(x), _f32(v), _f32(np.full(n, (0.5 * dx) ** 3)), inst.copy(), mats,
                 ckpt_every=25, frame_sub=(np.arange(1, 11) * 50).astype(np.int32))


WORKLOADS = {
    "cube_8k": cube_8k,
    "three_objects_300k": three_objects_300k,
    "ball_50k": ball_50k,
    "ball_512": ball_512,
    "batch_64": batch_64,
    "large_2m": large_2m,
}


def key_frames(sc: Scene, n_keys=3, k_seed=40, vs=0.5, cs=5.0, fs=0.05):
    """n_keys synthetic key-frame states (v, C, F) at the scene's positions:
    the scene velocity plus N(0, vs^2) noise, an affine field N(0, cs^2) and a
    deformation gradient R_z(0.3 k) (I + N(0, fs^2)).  They stand in for the
    snapshots a forward run would store (Algorithm 1, Stage 1)."""
    rng = _rng(k_seed)
    n = sc.n
    out = []
    for k in range(n_keys):
        th = 0.3 * k
        Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
        v = sc.v + vs * rng.standard_normal((n, 3))
        C = cs * rng.standard_normal((n, 3, 3))
        F = np.einsum("ij,njk->nik", Rz, np.eye(3) + fs * rng.standard_normal((n, 3, 3)))
        out.append((_f32(v), _f32(C), _f32(F)))
    return out


def gaussian_covariances(sc: Scene, k_seed=50):
    """A Gaussian kernel per particle, Sigma = R S S^T R^T (§3.1) with a
    uniformly random rotation R and flat splat scales S = diag(a, b, 0.1 a')
    where a, b ~ U(0.3, 1) dx/2 (surface-like 3DGS kernels).  Returned as
    (n, 6) float32 xx xy xz yy yz zz."""
    rng = _rng(k_seed)
    n = sc.n
    half = 0.5 * sc.dx
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    a, b, c, d = q.T
    R = np.stack([np.stack([a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)], -1),
                  np.stack([2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)], -1),
                  np.stack([2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d], -1)], 1)
    s = np.stack([rng.uniform(0.3, 1.0, n) * half, rng.uniform(0.3, 1.0, n) * half,
                  0.1 * rng.uniform(0.3, 1.0, n) * half], 1)
    M = R * s[:, None, :]
    S = M @ M.transpose(0, 2, 1)
    return _f32(np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1))


def mcis_case(n_surface=(36_000, 36_000, 36_000), n_cand=(250_000, 250_000, 250_000),
              n_draw=(64_000, 64_000, 64_000), k_seed=70):
    """Inputs of the MCIS fill (§4.1) for the three objects of the 300k scene:
    per object its surface proxy C_k (uniform surface samples with a normal
    offset N(0, (0.1 dx)^2), dx = 1/128, like the splat shells), candidates
    uniform in its bounding box kept where the shape's own inside test holds
    (a stand-in for the occupancy selection, which precedes MCIS), and one
    uniform in [0, 1) per draw.  Returns dict(surf_off, surf, cand_off, cand,
    draw_off, u)."""
    rng = _rng(k_seed)
    dx = 1.0 / 128
    shapes = [Sphere((0.2, 0.20, 0.5), 0.10), Torus((0.5, 0.14, 0.5), 0.10, 0.04), Box((0.8, 0.18, 0.5), 0.08)]
    surf, cand = [], []
    for k, sh in enumerate(shapes):
        surf.append(_shell(sh, n_surface[k], 0.1 * dx, rng))
        lo, hi = sh.bbox()
        got = []
        need = n_cand[k]
        while need > 0:
            q = lo + (hi - lo) * rng.random((2 * need + 64, 3))
            q = q[sh.inside(q)][:need]
            got.append(q)
            need -= len(q)
        cand.append(np.concatenate(got))
    off = lambda parts: np.concatenate([[0], np.cumsum([len(a) for a in parts])]).astype(np.int64)
    return {"surf_off": off(surf), "surf": _f32(np.concatenate(surf)), "cand_off": off(cand),
            "cand": _f32(np.concatenate(cand)), "draw_off": np.concatenate([[0], np.cumsum(n_draw)]).astype(np.int64),
            "u": rng.random(int(sum(n_draw)))}


def gaussian_appearance(sc: Scene, k_seed=80, transparent=None):
    """Per particle an RGB colour U(0, 1)^3 and an opacity U(0.3, 1) (splat
    appearance); particles flagged in `transparent` get opacity 0, as the
    filled interior points of §4.1 step 6."""
    rng = _rng(k_seed)
    col = rng.random((sc.n, 3))
    op = rng.uniform(0.3, 1.0, sc.n)
    if transparent is not None:
        op[np.asarray(transparent)] = 0.0
    return _f32(col), _f32(op)


def camera(width, height, eye=(0.5, 0.45, -1.0), target=(0.5, 0.25, 0.5), fov_deg=40.0):
    """A pinhole camera looking from `eye` at `target` (y up): the row-major
    3x4 world-to-camera transform [R | T] with camera z along the view
    direction and image y down, and fx, fy, cx, cy in pixels."""
    e, t = np.asarray(eye, float), np.asarray(target, float)
    z = t - e
    z /= np.linalg.norm(z)
    x = np.cross(np.array([0.0, -1.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    T = -R @ e
    f = 0.5 * height / math.tan(math.radians(fov_deg) / 2)
    return np.concatenate([R, T[:, None]], 1), f, f, 0.5 * width, 0.5 * height
