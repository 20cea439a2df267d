"""FP64 CPU oracle of the MLS-MPM substep and its adjoint (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline and reference legs of ``bench.py`` may import this package.  The product path
(``paper_2602_01723_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``mpm_oracle.c`` (plain C, double precision, scalar
loops); this module only compiles it with gcc and marshals numpy arrays.

State layout: ``x (n,3)``, ``v (n,3)``, ``C (n,3,3)``, ``F (n,3,3)``, float64,
row-major 3x3.  A packed state row is ``[x(3) v(3) C(9) F(9)]`` (24 doubles).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmpm_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


_P = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


class _Cfg(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int * 3), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("gravity", ctypes.c_double * 3), ("bound", ctypes.c_int), ("wall", ctypes.c_int * 6)]


class _Mat(ctypes.Structure):
    _fields_ = [("mass", _P), ("vol", _P), ("logE", _P), ("nu", _P), ("yield_", _P), ("phi_deg", _P),
                ("elastic", _PI), ("plastic", _PI)]


class _BgdoOpt(ctypes.Structure):
    _fields_ = [("delta_target", ctypes.c_double), ("w", ctypes.c_double), ("per_material", ctypes.c_int),
                ("delta_pre_step", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_bspline.argtypes = [ctypes.c_double, _P, _P]
            L.orc_lame.argtypes = [ctypes.c_double, ctypes.c_double, _P, _P]
            L.orc_svd.argtypes = [_P, _P, _P, _P]
            L.orc_polar.argtypes = [_P, _P]
            L.orc_kirchhoff.argtypes = [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, _P]
            L.orc_return_map.argtypes = [ctypes.c_int, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _P]
            L.orc_dp_alpha.argtypes = [ctypes.c_double]
            L.orc_dp_alpha.restype = ctypes.c_double
            cp, mp = ctypes.POINTER(_Cfg), ctypes.POINTER(_Mat)
            L.orc_p2g.argtypes = [cp, ctypes.c_long, _P, _P, _P, _P, mp, _P, _P]
            L.orc_grid_update.argtypes = [cp, _P, _P, _P]
            L.orc_g2p.argtypes = [cp, ctypes.c_long, _P, _P, _P, _P, mp, _P]
            L.orc_substep.argtypes = [cp, ctypes.c_long, _P, _P, _P, _P, mp]
            L.orc_run.argtypes = [cp, ctypes.c_long, _P, _P, _P, _P, mp, ctypes.c_int, _P]
            L.orc_substep_adjoint.argtypes = [cp, ctypes.c_long, _P, mp, _P, _P, _P]
            L.orc_backward.argtypes = [cp, ctypes.c_long, mp, ctypes.c_int, _P, ctypes.c_int, _PI, _P, _P, _P]
            L.orc_covariance.argtypes = [ctypes.c_long, _P, _P, _P]
            L.orc_render.argtypes = [ctypes.c_long, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                     ctypes.c_double, _P]
            _PL = ctypes.POINTER(ctypes.c_long)
            L.orc_mcis.argtypes = [ctypes.c_int, _PL, _P, _PL, _P, _PL, _P, ctypes.c_double, ctypes.c_double, _P, _P,
                                   ctypes.POINTER(ctypes.c_longlong), _PL]
            L.orc_bgdo.argtypes = [cp, ctypes.c_long, ctypes.c_int, _P, mp, _PI, ctypes.c_int,
                                   ctypes.POINTER(_BgdoOpt), _P, _P, _P]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_P)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------------------
# configuration / material / state containers
# --------------------------------------------------------------------------

WALL_OPEN, WALL_SLIP, WALL_STICKY = 0, 1, 2
DEFAULT_WALLS = (WALL_SLIP, WALL_SLIP, WALL_STICKY, WALL_SLIP, WALL_SLIP, WALL_SLIP)


class Cfg:
    def __init__(self, res, dx, dt, gravity=(0.0, -9.8, 0.0), bound=3, walls=DEFAULT_WALLS):
        if np.isscalar(res):
            res = (res, res, res)
        self.res = tuple(int(r) for r in res)
        self.dx, self.dt = float(dx), float(dt)
        self.gravity = tuple(float(g) for g in gravity)
        self.bound = int(bound)
        self.walls = tuple(int(w) for w in walls)
        self._c = _Cfg((ctypes.c_int * 3)(*self.res), self.dx, self.dt, (ctypes.c_double * 3)(*self.gravity),
                       self.bound, (ctypes.c_int * 6)(*self.walls))

    @property
    def ptr(self):
        return ctypes.byref(self._c)

    @property
    def n_nodes(self):
        return self.res[0] * self.res[1] * self.res[2]


class Material:
    """Per-particle material arrays.  mass = rho * vol (reading: m_p = rho V_p)."""

    def __init__(self, vol, rho, logE, nu, yield_stress, phi_deg, elastic, plastic):
        n = len(vol)
        bc = lambda a, dt=np.float64: np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=dt), (n,)).copy())
        self.vol = bc(vol)
        self.rho = bc(rho)
        self.mass = self.rho * self.vol
        self.logE, self.nu = bc(logE), bc(nu)
        self.yield_stress, self.phi_deg = bc(yield_stress), bc(phi_deg)
        self.elastic, self.plastic = bc(elastic, np.int32), bc(plastic, np.int32)
        self._c = _Mat(_d(self.mass), _d(self.vol), _d(self.logE), _d(self.nu), _d(self.yield_stress),
                       _d(self.phi_deg), self.elastic.ctypes.data_as(_PI), self.plastic.ctypes.data_as(_PI))

    @property
    def ptr(self):
        return ctypes.byref(self._c)

    @property
    def n(self):
        return len(self.vol)

    def with_params(self, logE=None, nu=None, yield_stress=None):
        return Material(self.vol, self.rho, self.logE if logE is None else logE, self.nu if nu is None else nu,
                        self.yield_stress if yield_stress is None else yield_stress, self.phi_deg, self.elastic,
                        self.plastic)

    def subset(self, idx):
        return Material(self.vol[idx], self.rho[idx], self.logE[idx], self.nu[idx], self.yield_stress[idx],
                        self.phi_deg[idx], self.elastic[idx], self.plastic[idx])

    @staticmethod
    def from_table(vol, mat_id, table, params=None):
        """table: sequence of dicts with keys elastic, plastic, E, nu, rho,
        yield_stress, friction_angle_deg.  params (n,3) = per-particle
        (logE, nu, yield) overriding the table when given."""
        mat_id = np.asarray(mat_id)
        col = lambda k: np.array([float(t[k]) for t in table])[mat_id]
        logE, nu, ys = np.log(col("E")), col("nu"), col("yield_stress")
        if params is not None:
            params = np.asarray(params, dtype=np.float64)
            logE, nu, ys = params[:, 0], params[:, 1], params[:, 2]
        return Material(vol, col("rho"), logE, nu, ys, col("friction_angle_deg"),
                        col("elastic").astype(np.int32), col("plastic").astype(np.int32))


def new_state(x, v=None, C=None, F=None):
    x = _f64(x, (-1, 3)).copy()
    n = len(x)
    v = np.zeros((n, 3)) if v is None else _f64(v, (n, 3)).copy()
    C = np.zeros((n, 3, 3)) if C is None else _f64(C, (n, 3, 3)).copy()
    F = np.tile(np.eye(3), (n, 1, 1)) if F is None else _f64(F, (n, 3, 3)).copy()
    return {"x": x, "v": v, "C": C, "F": F}


def copy_state(s):
    return {k: np.array(a, dtype=np.float64, copy=True) for k, a in s.items()}


def pack(s):
    n = len(s["x"])
    return np.concatenate([s["x"], s["v"], s["C"].reshape(n, 9), s["F"].reshape(n, 9)], axis=1)


def unpack(a):
    a = np.asarray(a)
    n = a.shape[0]
    return {"x": a[:, 0:3].copy(), "v": a[:, 3:6].copy(), "C": a[:, 6:15].reshape(n, 3, 3).copy(),
            "F": a[:, 15:24].reshape(n, 3, 3).copy()}


def _check(st):
    if st == 1:
        raise OracleError("particle outside the grid stencil range")
    if st == 2:
        raise OracleError("non-finite state or J <= 0 for Neo-Hookean")
    if st != 0:
        raise OracleError("oracle status %d" % st)


# --------------------------------------------------------------------------
# unit functions
# --------------------------------------------------------------------------

def bspline(fx):
    w, dw = np.zeros(3), np.zeros(3)
    lib().orc_bspline(float(fx), _d(w), _d(dw))
    return w, dw


def lame(E, nu):
    mu, lam = ctypes.c_double(), ctypes.c_double()
    lib().orc_lame(float(E), float(nu), ctypes.byref(mu), ctypes.byref(lam))
    return mu.value, lam.value


def dp_alpha(phi_deg):
    return lib().orc_dp_alpha(float(phi_deg))


def svd(F):
    F = _f64(F, (3, 3))
    U, S, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().orc_svd(_d(F), _d(U), _d(S), _d(V))
    return U, S, V


def polar(F):
    F = _f64(F, (3, 3))
    R = np.zeros((3, 3))
    lib().orc_polar(_d(F), _d(R))
    return R


def kirchhoff(model, F, mu, lam):
    F = _f64(F, (3, 3))
    tau = np.zeros((3, 3))
    _check(lib().orc_kirchhoff(int(model), _d(F), float(mu), float(lam), _d(tau)))
    return tau


def return_map(model, F, mu, lam, yield_stress, phi_deg):
    """Returns (F_new, case) with case 0 elastic, 1 projected, 2 cone tip."""
    F = _f64(F, (3, 3))
    out = np.zeros((3, 3))
    c = lib().orc_return_map(int(model), _d(F), float(mu), float(lam), float(yield_stress), float(phi_deg),
                             _d(out))
    return out, c


# --------------------------------------------------------------------------
# substep pieces and drivers
# --------------------------------------------------------------------------

def _state_ptrs(s):
    for k in ("x", "v", "C", "F"):
        if not (s[k].dtype == np.float64 and s[k].flags.c_contiguous):
            s[k] = np.ascontiguousarray(s[k], dtype=np.float64)
    return _d(s["x"]), _d(s["v"]), _d(s["C"]), _d(s["F"])


def p2g(cfg: Cfg, state, mat: Material):
    """Dense grid mass (R0,R1,R2) and momentum (R0,R1,R2,3) after P2G."""
    s = copy_state(state)
    gm = np.zeros(cfg.n_nodes)
    gmv = np.zeros(3 * cfg.n_nodes)
    _check(lib().orc_p2g(cfg.ptr, len(s["x"]), *_state_ptrs(s), mat.ptr, _d(gm), _d(gmv)))
    return gm.reshape(cfg.res), gmv.reshape(cfg.res + (3,))


def grid_update(cfg: Cfg, gm, gmv):
    gm = _f64(gm, (-1,))
    gmv = _f64(gmv, (-1,))
    gv = np.zeros(3 * cfg.n_nodes)
    lib().orc_grid_update(cfg.ptr, _d(gm), _d(gmv), _d(gv))
    return gv.reshape(cfg.res + (3,))


def g2p(cfg: Cfg, state, mat: Material, gv):
    s = copy_state(state)
    gv = _f64(gv, (-1,))
    _check(lib().orc_g2p(cfg.ptr, len(s["x"]), *_state_ptrs(s), mat.ptr, _d(gv)))
    return s


def substep(cfg: Cfg, state, mat: Material):
    s = copy_state(state)
    _check(lib().orc_substep(cfg.ptr, len(s["x"]), *_state_ptrs(s), mat.ptr))
    return s


def run(cfg: Cfg, state, mat: Material, n_sub: int, tape: bool = False):
    """Runs n_sub substeps.  With tape=True also returns the (n_sub+1, n, 24)
    packed states after 0..n_sub substeps."""
    s = copy_state(state)
    n = len(s["x"])
    t = np.zeros((n_sub + 1, n, 24)) if tape else None
    _check(lib().orc_run(cfg.ptr, n, *_state_ptrs(s), mat.ptr, int(n_sub), _d(t) if tape else None))
    return (s, t) if tape else s


def substep_adjoint(cfg: Cfg, state, mat: Material, adj_out):
    """Adjoint of one substep: returns (adj_in (n,24), g_param (n,3))."""
    st = _f64(pack(state))
    n = st.shape[0]
    ao = _f64(adj_out, (n, 24))
    ai = np.zeros((n, 24))
    g = np.zeros((n, 3))
    _check(lib().orc_substep_adjoint(cfg.ptr, n, _d(st), mat.ptr, _d(ao), _d(ai), _d(g)))
    return ai, g


def backward(cfg: Cfg, mat: Material, tape, frame_sub, dLdx):
    """Trajectory adjoint from a tape of run(..., tape=True).

    frame_sub: substep index of each frame; dLdx: (n_frames, n, 3).
    Returns (adj0 (n,24), g_param (n,3) = dL/d(logE, nu, yield))."""
    tape = _f64(tape)
    n_sub = tape.shape[0] - 1
    n = tape.shape[1]
    fs = np.ascontiguousarray(np.asarray(frame_sub, dtype=np.int32))
    dl = _f64(dLdx, (len(fs), n, 3))
    adj0 = np.zeros((n, 24))
    g = np.zeros((n, 3))
    _check(lib().orc_backward(cfg.ptr, n, mat.ptr, n_sub, _d(tape), len(fs), fs.ctypes.data_as(_PI), _d(dl),
                              _d(adj0), _d(g)))
    return adj0, g


def trajectory_loss(frames_x, target_x):
    """L = 1/(F N) sum_f sum_p |x_p(t_f) - x_hat_p(t_f)|^2 and dL/dx per frame."""
    fx = np.asarray(frames_x, dtype=np.float64)
    tx = np.asarray(target_x, dtype=np.float64)
    nf, n = fx.shape[0], fx.shape[1]
    d = fx - tx
    return float(np.sum(d * d) / (nf * n)), 2.0 * d / (nf * n)


def bgdo(cfg: Cfg, keys, mat: Material, label=None, delta_target=0.1, w=None, per_material=False,
         delta_pre_step=False):
    """BGDO stage 2 (§4.3, Algorithm 1, App. F) from key-frame states.

    keys: list of states (dicts).  w=None takes eta = min(1, 0.1 log(1+E)).
    Returns dict(G (n,), log_E (n,) = logE - G, g_tau (K,n), delta (K,n))."""
    K = len(keys)
    n = len(keys[0]["x"])
    kp = _f64(np.stack([pack(k) for k in keys]))
    lab = np.ascontiguousarray(np.zeros(n, np.int32) if label is None else np.asarray(label, dtype=np.int32))
    n_lab = int(lab.max()) + 1 if n else 0
    opt = _BgdoOpt(float(delta_target), -1.0 if w is None else float(w), int(bool(per_material)),
                   int(bool(delta_pre_step)))
    G = np.zeros(n)
    gt = np.zeros((K, n))
    dl = np.zeros((K, n))
    _check(lib().orc_bgdo(cfg.ptr, n, K, _d(kp), mat.ptr, lab.ctypes.data_as(_PI), n_lab, ctypes.byref(opt),
                          _d(G), _d(gt), _d(dl)))
    return {"G": G, "log_E": mat.logE - G, "g_tau": gt, "delta": dl}


def covariance(F, cov0):
    """Sigma(t) = F Sigma F^T per particle (§3.2); cov as (n,6) xx xy xz yy yz zz."""
    F = _f64(F, (-1, 3, 3))
    n = len(F)
    c0 = _f64(cov0, (n, 6))
    out = np.zeros((n, 6))
    lib().orc_covariance(n, _d(F), _d(c0), _d(out))
    return out


def sym33(c):
    """(n,6) xx xy xz yy yz zz -> (n,3,3)."""
    c = np.asarray(c, dtype=np.float64).reshape(-1, 6)
    return np.stack([c[:, [0, 1, 2]], c[:, [1, 3, 4]], c[:, [2, 4, 5]]], axis=1)


MCIS_WSCALE = 2.0 ** 40


def mcis(surf_off, surf, cand_off, cand, draw_off, u, sigma=0.02, eps=1e-6):
    """MCIS steps 1-4 (§4.1) per object over contiguous ranges.  Returns
    dict(d, w, cum (inclusive integer cumulative weights per object), picked
    (global candidate index of every draw, -1 for an object without
    candidates))."""
    L = lib()
    to_l = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    so, co, do = to_l(surf_off), to_l(cand_off), to_l(draw_off)
    sf = _f64(surf, (-1, 3))
    cf = _f64(cand, (-1, 3))
    uu = _f64(u, (-1,))
    n_obj = len(so) - 1
    nc = int(co[-1])
    d, w = np.zeros(nc), np.zeros(nc)
    cum = np.zeros(nc, dtype=np.int64)
    picked = np.zeros(int(do[-1]), dtype=np.int64)
    PL = ctypes.POINTER(ctypes.c_long)
    L.orc_mcis(n_obj, so.ctypes.data_as(PL), _d(sf), co.ctypes.data_as(PL), _d(cf), do.ctypes.data_as(PL), _d(uu),
               float(sigma), float(eps), _d(d), _d(w), cum.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
               picked.ctypes.data_as(PL))
    return {"d": d, "w": w, "cum": cum, "picked": picked}


def render(mean, cov, col, opac, view, fx, fy, cx, cy, W, H, bg=(0.0, 0.0, 0.0), tie_eps=None):
    """Splat the Gaussians (§3.1) into an H x W x 3 image; view is the 3x4
    [R | T] world-to-camera transform.  Returns (image, transmittance), and
    with tie_eps also the per-pixel order-ambiguity bound: how far reordering
    layers whose depths agree within tie_eps times the magnitude of their
    depth's terms (or drawing or dropping one that near the near plane) can
    move the pixel's colour."""
    mean = _f64(mean, (-1, 3))
    n = len(mean)
    cv, cl, op = _f64(cov, (n, 6)), _f64(col, (n, 3)), _f64(opac, (n,))
    vw, b = _f64(view, (12,)), _f64(bg, (3,))
    img = np.zeros((H, W, 3))
    T = np.zeros((H, W))
    amb = np.zeros((H, W)) if tie_eps is not None else None
    lib().orc_render(n, _d(mean), _d(cv), _d(cl), _d(op), _d(vw), float(fx), float(fy), float(cx), float(cy), int(W),
                     int(H), _d(b), _d(img), _d(T), float(tie_eps or 0.0), _d(amb) if amb is not None else None)
    return (img, T) if amb is None else (img, T, amb)
