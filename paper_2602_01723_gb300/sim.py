"""Python front end of libmpm: a Simulator that owns one mpm_ctx, and the
torch.autograd.Function that differentiates a trajectory loss through the
library's hand-written adjoint.  PyTorch supplies device memory and streams
only; every step of the simulation runs in libmpm's kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L


def _stream(s=None):
    s = s if s is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(a, dtype, device, width=None):
    if a is None:
        return None
    t = torch.as_tensor(a, dtype=dtype)
    if width is not None:
        t = t.reshape(-1, width)
    return t.to(device).contiguous()


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Simulator:
    """One simulation context (one or more independent grids)."""

    def __init__(self, grid_res, dx, dt, gravity, materials, n_instances=1, walls=None, bound=3, ckpt_every=20,
                 chunk=0, max_active_blocks=0, max_particles=0, scatter=1, tape_grid=0, device="cuda"):
        if np.isscalar(grid_res):
            grid_res = (grid_res,) * 3
        self.grid_res = tuple(int(r) for r in grid_res)
        self.dx, self.dt = float(dx), float(dt)
        self.device = torch.device(device)
        opt = L.mpm_default_options()
        opt.n_instances = int(n_instances)
        opt.bound = int(bound)
        if walls is not None:
            for i, w in enumerate(walls):
                opt.walls[i] = int(w)
        opt.ckpt_every = int(ckpt_every)
        opt.chunk = int(chunk)
        opt.scatter = int(scatter)
        opt.tape_grid = int(tape_grid)
        opt.max_active_blocks = int(max_active_blocks)
        opt.max_particles = int(max_particles)
        self.n_instances = int(n_instances)
        self.materials = list(materials)
        with torch.cuda.device(self.device):
            self.ctx = L.mpm_create(self.grid_res, self.dx, self.dt, gravity, self.materials, opt)
        self.n = 0

    @classmethod
    def from_scene(cls, sc, **kw):
        kw.setdefault("n_instances", sc.n_instances)
        kw.setdefault("ckpt_every", sc.ckpt_every or 20)
        return cls(sc.grid_res, sc.dx, sc.dt, sc.gravity, sc.materials, **kw)

    def load_scene(self, sc, params=None, stream=None):
        return self.load(sc.x, sc.vol, sc.mat_id, v=sc.v, instance=sc.instance,
                         params=sc.params if params is None else params, stream=stream)

    def load(self, x, vol, material_id, v=None, C=None, F=None, instance=None, params=None, stream=None):
        dv = self.device
        x = _dev(x, torch.float32, dv, 3)
        n = x.shape[0]
        args = [x, _dev(v, torch.float32, dv, 3), _dev(C, torch.float32, dv, 9), _dev(F, torch.float32, dv, 9),
                _dev(vol, torch.float32, dv), _dev(material_id, torch.int32, dv), _dev(instance, torch.int32, dv),
                _dev(params, torch.float32, dv, 3)]
        L.mpm_load_particles(self.ctx, n, *[_p(a) for a in args], _stream(stream))
        self.n = n
        return self

    def step(self, n_substeps, record=False, stream=None):
        L.mpm_step(self.ctx, int(n_substeps), int(bool(record)), _stream(stream))

    def get(self, stream=None):
        n = self.n
        out = {"x": torch.empty((n, 3), device=self.device), "v": torch.empty((n, 3), device=self.device),
               "C": torch.empty((n, 3, 3), device=self.device), "F": torch.empty((n, 3, 3), device=self.device)}
        L.mpm_get_particles(self.ctx, _p(out["x"]), _p(out["v"]), _p(out["C"]), _p(out["F"]), _stream(stream))
        return out

    def positions(self, out=None, stream=None):
        out = torch.empty((self.n, 3), device=self.device) if out is None else out
        L.mpm_get_particles(self.ctx, _p(out), None, None, None, _stream(stream))
        return out

    def sync(self, stream=None):
        L.mpm_sync(self.ctx, _stream(stream))

    def stats(self, stream=None):
        return L.mpm_stats(self.ctx, _stream(stream))

    def trace(self, enable):
        return L.mpm_trace(self.ctx, enable)

    def reduce_by_material(self, per_particle, stream=None):
        out = torch.empty((len(self.materials), 3), device=self.device)
        per_particle = per_particle.contiguous()
        L.mpm_reduce_by_material(self.ctx, _p(per_particle), _p(out), _stream(stream))
        return out

    def set_tuning(self, scatter=1, chunk=128, use_graph=True):
        L.mpm_set_tuning(self.ctx, scatter, chunk, use_graph)

    def autotune(self, n_substeps=20, stream=None):
        return L.mpm_autotune(self.ctx, n_substeps, _stream(stream))

    def record_reset(self):
        L.mpm_record_reset(self.ctx)

    def backward(self, frame_sub, dL_dx, want_state0=False, stream=None):
        dL_dx = _dev(dL_dx, torch.float32, self.device).reshape(len(frame_sub), self.n, 3).contiguous()
        g = torch.empty((self.n, 3), device=self.device)
        a0 = torch.empty((self.n, 24), device=self.device) if want_state0 else None
        L.mpm_backward(self.ctx, list(frame_sub), _p(dL_dx), _p(g), _p(a0), _stream(stream))
        return (g, a0) if want_state0 else g

    def load_covariance(self, cov0, stream=None):
        """Rest covariance Sigma of each particle's Gaussian kernel, (n, 6)
        xx xy xz yy yz zz (§3.1)."""
        cov0 = _dev(cov0, torch.float32, self.device, 6)
        L.mpm_load_covariance(self.ctx, _p(cov0), _stream(stream))
        self._cov0 = cov0    # keep alive until the stream has copied it

    def covariance(self, out=None, stream=None):
        """Deformed covariance F Sigma F^T of every particle, (n, 6) (§3.2)."""
        out = torch.empty((self.n, 6), device=self.device) if out is None else out
        L.mpm_get_covariance(self.ctx, _p(out), _stream(stream))
        return out

    def snapshot(self, slot, stream=None):
        """Stores the current state as BGDO key frame `slot` (Algorithm 1, Stage 1)."""
        L.mpm_snapshot(self.ctx, slot, _stream(stream))

    def bgdo(self, slots, delta_target=0.1, w=None, per_material=False, delta_pre_step=False, signals=False,
             stream=None):
        """BGDO stage 2 from the key frames in `slots` (§4.3, Algorithm 1,
        App. F).  Returns the per-particle update G, the updated log E
        (log E - G) and, with signals=True, the per-key g_tau and delta."""
        n, K, dv = self.n, len(slots), self.device
        out = {"G": torch.empty(n, device=dv), "log_E": torch.empty(n, device=dv)}
        if signals:
            out["g_tau"] = torch.empty((K, n), device=dv)
            out["delta"] = torch.empty((K, n), device=dv)
        L.mpm_bgdo(self.ctx, list(slots), delta_target, w, per_material, delta_pre_step, _p(out["G"]),
                   _p(out["log_E"]), _p(out.get("g_tau")), _p(out.get("delta")), _stream(stream))
        return out

    def debug_p2g(self, stream=None):
        nn = self.n_instances * self.grid_res[0] * self.grid_res[1] * self.grid_res[2]
        m = torch.empty(nn, device=self.device)
        mv = torch.empty(nn * 3, device=self.device)
        L.mpm_debug_p2g(self.ctx, _p(m), _p(mv), _stream(stream))
        shape = (self.n_instances,) + self.grid_res
        return m.reshape(shape), mv.reshape(shape + (3,))

    def close(self):
        if getattr(self, "ctx", None):
            L.mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trajectory(torch.autograd.Function):
    """Positions at loss frames as a differentiable function of per-particle
    material parameters (log E, nu, yield stress), through libmpm's
    hand-written adjoint with checkpoint recompute.

    forward(params (n,3), sim, init, frame_sub) loads the initial state
    `init` (dict with x, vol, mat_id and optionally v, C, F, instance) with
    `params`, runs a recorded forward pass and returns x at the frames,
    shape (n_frames, n, 3).  backward returns dL/dparams (n,3)."""

    @staticmethod
    def forward(ctx, params, sim, init, frame_sub):
        frame_sub = [int(f) for f in frame_sub]
        if sorted(frame_sub) != frame_sub or (frame_sub and frame_sub[0] < 0):
            raise ValueError("frame_sub must be non-decreasing and >= 0")
        sim.load(init["x"], init["vol"], init["mat_id"], v=init.get("v"), C=init.get("C"), F=init.get("F"),
                 instance=init.get("instance"), params=params.detach())
        frames, prev = [], 0
        for f in frame_sub:
            if f > prev:
                sim.step(f - prev, record=True)
            frames.append(sim.positions())
            prev = f
        ctx.sim = sim
        ctx.frame_sub = frame_sub
        return torch.stack(frames)

    @staticmethod
    def backward(ctx, grad_frames):
        g = ctx.sim.backward(ctx.frame_sub, grad_frames.contiguous())
        return g, None, None, None


def trajectory(params, sim, init, frame_sub):
    return Trajectory.apply(params, sim, init, frame_sub)


def mcis(surf_off, surf, cand_off, cand, draw_off, u, sigma=0.02, eps=1e-6, device="cuda", stream=None):
    """MCIS fill sampling (§4.1 steps 1-4) on the GPU: objects as contiguous
    ranges (offsets of n_obj + 1), uniforms u per draw.  Returns dict(d, w,
    picked) as device tensors (float64, float64, int64)."""
    dv = torch.device(device)
    surf = _dev(surf, torch.float32, dv, 3)
    cand = _dev(cand, torch.float32, dv, 3)
    u = _dev(u, torch.float64, dv)
    nc, nd = int(cand_off[-1]), int(draw_off[-1])
    out = {"d": torch.empty(nc, dtype=torch.float64, device=dv), "w": torch.empty(nc, dtype=torch.float64, device=dv),
           "picked": torch.empty(nd, dtype=torch.int64, device=dv)}
    L.mpm_mcis(surf_off, _p(surf), cand_off, _p(cand), draw_off, _p(u), sigma, eps, _p(out["d"]), _p(out["w"]),
               _p(out["picked"]), _stream(stream))
    return out


def render(mean, cov, color, opacity, view, fx, fy, cx, cy, width, height, bg=(0.0, 0.0, 0.0), device="cuda",
           stream=None):
    """Splat the Gaussians into an image (§3.1) on the GPU.  view: 3x4
    world-to-camera [R | T].  Returns (image (H, W, 3), transmittance (H, W))
    as device tensors."""
    dv = torch.device(device)
    mean = _dev(mean, torch.float32, dv, 3)
    n = mean.shape[0]
    cov = _dev(cov, torch.float32, dv, 6)
    color = _dev(color, torch.float32, dv, 3)
    opacity = _dev(opacity, torch.float32, dv)
    img = torch.empty((height, width, 3), device=dv)
    tr = torch.empty((height, width), device=dv)
    view = np.asarray(view, dtype=np.float64).reshape(-1)
    L.mpm_render(n, _p(mean), _p(cov), _p(color), _p(opacity), view, fx, fy, cx, cy, width, height, bg, _p(img),
                 _p(tr), _stream(stream))
    return img, tr
