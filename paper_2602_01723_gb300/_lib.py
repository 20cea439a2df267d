"""ctypes binding of libmpm (include/mpm.h).  Same names as the C ABI; only
argument marshalling happens here.  Importing this module fails loudly when
the library has not been built: there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "libmpm.so")

MPM_OK = 0
STATUS_NAMES = {0: "MPM_OK", 1: "MPM_ERR_INVALID_ARG", 2: "MPM_ERR_OOM", 3: "MPM_ERR_CUDA",
                4: "MPM_ERR_OUT_OF_DOMAIN", 5: "MPM_ERR_NONFINITE", 6: "MPM_ERR_TIMEOUT", 7: "MPM_ERR_STATE",
                8: "MPM_ERR_CAPACITY", 9: "MPM_ERR_CFL"}


class MpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class mpm_material(ctypes.Structure):
    _fields_ = [("elastic", ctypes.c_int32), ("plastic", ctypes.c_int32), ("E", ctypes.c_float),
                ("nu", ctypes.c_float), ("rho", ctypes.c_float), ("yield_stress", ctypes.c_float),
                ("friction_angle_deg", ctypes.c_float)]


class mpm_options(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("bound", ctypes.c_int32), ("walls", ctypes.c_int32 * 6),
                ("max_particles", ctypes.c_int64), ("max_active_blocks", ctypes.c_int64),
                ("ckpt_every", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("scatter", ctypes.c_int32), ("tape_grid", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class mpm_bgdo_options(ctypes.Structure):
    _fields_ = [("delta_target", ctypes.c_float), ("w", ctypes.c_float), ("per_material", ctypes.c_int32),
                ("delta_pre_step", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


MPM_MAX_SNAPSHOTS = 8

_ctx_p = ctypes.c_void_p
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes); every symbol include/mpm.h declares
SIGNATURES = {
    "mpm_default_options": (ctypes.c_int, [ctypes.POINTER(mpm_options)]),
    "mpm_create": (ctypes.c_int, [_i32p, ctypes.c_float, ctypes.c_float, _f32p, ctypes.POINTER(mpm_material),
                                  ctypes.c_int32, ctypes.POINTER(mpm_options), ctypes.POINTER(_ctx_p)]),
    "mpm_load_particles": (ctypes.c_int, [_ctx_p, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mpm_step": (ctypes.c_int, [_ctx_p, ctypes.c_int32, ctypes.c_int32, _vp]),
    "mpm_get_particles": (ctypes.c_int, [_ctx_p, _vp, _vp, _vp, _vp, _vp]),
    "mpm_backward": (ctypes.c_int, [_ctx_p, ctypes.c_int32, _i32p, _vp, _vp, _vp, _vp]),
    "mpm_record_reset": (ctypes.c_int, [_ctx_p]),
    "mpm_sync": (ctypes.c_int, [_ctx_p, _vp]),
    "mpm_stats": (ctypes.c_int, [_ctx_p, _i64p, _vp]),
    "mpm_last_error": (ctypes.c_char_p, [_ctx_p]),
    "mpm_destroy": (ctypes.c_int, [_ctx_p]),
    "mpm_debug_p2g": (ctypes.c_int, [_ctx_p, _vp, _vp, _vp]),
    "mpm_trace": (ctypes.c_int, [_ctx_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _i64p]),
    "mpm_reduce_by_material": (ctypes.c_int, [_ctx_p, _vp, _vp, _vp]),
    "mpm_snapshot": (ctypes.c_int, [_ctx_p, ctypes.c_int32, _vp]),
    "mpm_bgdo_default_options": (ctypes.c_int, [ctypes.POINTER(mpm_bgdo_options)]),
    "mpm_bgdo": (ctypes.c_int, [_ctx_p, ctypes.c_int32, _i32p, ctypes.POINTER(mpm_bgdo_options), _vp, _vp, _vp,
                                _vp, _vp]),
    "mpm_load_covariance": (ctypes.c_int, [_ctx_p, _vp, _vp]),
    "mpm_get_covariance": (ctypes.c_int, [_ctx_p, _vp, _vp]),
    "mpm_mcis": (ctypes.c_int, [ctypes.c_int32, _i64p, _vp, _i64p, _vp, _i64p, _vp, ctypes.c_double, ctypes.c_double,
                                _vp, _vp, _vp, _vp]),
    "mpm_mcis_last_error": (ctypes.c_char_p, []),
    "mpm_render": (ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp, _vp, _f32p, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_int32, _f32p, _vp, _vp, _vp]),
    "mpm_render_last_error": (ctypes.c_char_p, []),
    "mpm_set_tuning": (ctypes.c_int, [_ctx_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mpm_autotune": (ctypes.c_int, [_ctx_p, ctypes.c_int32, _i32p, _vp]),
    "mpm_substep_noalloc": (ctypes.c_int, [_i32p, ctypes.c_float, ctypes.c_float, _f32p, ctypes.POINTER(mpm_material),
                                           ctypes.c_int32, ctypes.POINTER(mpm_options), ctypes.c_int64,
                                           _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}

_lib = None


def lib():
    """Loads libmpm.so (raising when it is missing or lacks a symbol)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO):
            raise ImportError("libmpm.so is not built (%s); run paper_2602_01723_gb300.build.build() or "
                              "__graft_entry__.build()" % SO)
        L = ctypes.CDLL(SO)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status, ctx=None):
    if status != MPM_OK:
        msg = lib().mpm_last_error(ctx)
        raise MpmError(status, msg.decode() if msg else "")
    return status


# thin same-name wrappers -----------------------------------------------------

def mpm_default_options():
    o = mpm_options()
    check(lib().mpm_default_options(ctypes.byref(o)))
    return o


def mpm_create(grid_res, dx, dt, gravity, table, opt=None):
    res = (ctypes.c_int32 * 3)(*[int(r) for r in grid_res])
    g = (ctypes.c_float * 3)(*[float(v) for v in gravity])
    mats = (mpm_material * len(table))()
    for i, t in enumerate(table):
        mats[i] = mpm_material(int(t["elastic"]), int(t["plastic"]), float(t["E"]), float(t["nu"]),
                               float(t["rho"]), float(t.get("yield_stress", 0.0)),
                               float(t.get("friction_angle_deg", 30.0)))
    out = _ctx_p()
    st = lib().mpm_create(res, float(dx), float(dt), g, mats, len(table),
                          ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
    check(st, None)
    return out


def mpm_load_particles(ctx, n, x, v, C, F, vol, material_id, instance, params, stream):
    check(lib().mpm_load_particles(ctx, int(n), x, v, C, F, vol, material_id, instance, params, stream), ctx)


def mpm_step(ctx, n_substeps, record, stream):
    check(lib().mpm_step(ctx, int(n_substeps), int(record), stream), ctx)


def mpm_get_particles(ctx, x, v, C, F, stream):
    check(lib().mpm_get_particles(ctx, x, v, C, F, stream), ctx)


def mpm_backward(ctx, frame_substep, dL_dx, dL_dparams, dL_dstate0, stream):
    fs = (ctypes.c_int32 * len(frame_substep))(*[int(f) for f in frame_substep])
    check(lib().mpm_backward(ctx, len(frame_substep), fs, dL_dx, dL_dparams, dL_dstate0, stream), ctx)


def mpm_record_reset(ctx):
    check(lib().mpm_record_reset(ctx), ctx)


def mpm_sync(ctx, stream):
    check(lib().mpm_sync(ctx, stream), ctx)


def mpm_stats(ctx, stream):
    c = (ctypes.c_int64 * 16)()
    check(lib().mpm_stats(ctx, c, stream), ctx)
    keys = ["particles", "occupied_blocks", "active_blocks", "chunks", "fp64_svd_fallbacks", "recorded",
            "device_error", "pool_blocks", "launches", "tape_grid_blocks", "tape_grid_reruns", "overflow_particles",
            "list_capacity", "list_blocks"]
    return dict(zip(keys, list(c)))


def mpm_trace(ctx, enable):
    """Returns {variant: (ms, launches)} recorded since the last call, then
    switches tracing on or off."""
    ms = (ctypes.c_double * 3)()
    cnt = (ctypes.c_int64 * 3)()
    check(lib().mpm_trace(ctx, int(enable), ms, cnt), ctx)
    return {"p2g": (ms[0], cnt[0]), "fused": (ms[1], cnt[1]), "g2p": (ms[2], cnt[2])}


def mpm_last_error(ctx):
    m = lib().mpm_last_error(ctx)
    return m.decode() if m else ""


def mpm_destroy(ctx):
    if ctx:
        check(lib().mpm_destroy(ctx))


def mpm_reduce_by_material(ctx, per_particle, per_material, stream):
    check(lib().mpm_reduce_by_material(ctx, per_particle, per_material, stream), ctx)


def mpm_set_tuning(ctx, scatter, chunk, use_graph):
    check(lib().mpm_set_tuning(ctx, int(scatter), int(chunk), int(use_graph)), ctx)


def mpm_autotune(ctx, n_substeps, stream):
    out = (ctypes.c_int32 * 3)()
    check(lib().mpm_autotune(ctx, int(n_substeps), out, stream), ctx)
    return {"scatter": out[0], "chunk": out[1], "best_us": out[2]}


def mpm_debug_p2g(ctx, m, mv, stream):
    check(lib().mpm_debug_p2g(ctx, m, mv, stream), ctx)


def mpm_snapshot(ctx, slot, stream):
    check(lib().mpm_snapshot(ctx, int(slot), stream), ctx)


def mpm_bgdo(ctx, slots, delta_target, w, per_material, delta_pre_step, G, log_E, g_tau, delta, stream):
    o = mpm_bgdo_options()
    check(lib().mpm_bgdo_default_options(ctypes.byref(o)))
    o.delta_target = float(delta_target)
    o.w = -1.0 if w is None else float(w)
    o.per_material = int(bool(per_material))
    o.delta_pre_step = int(bool(delta_pre_step))
    sl = (ctypes.c_int32 * len(slots))(*[int(k) for k in slots])
    check(lib().mpm_bgdo(ctx, len(slots), sl, ctypes.byref(o), G, log_E, g_tau, delta, stream), ctx)


def mpm_load_covariance(ctx, cov0, stream):
    check(lib().mpm_load_covariance(ctx, cov0, stream), ctx)


def mpm_get_covariance(ctx, cov, stream):
    check(lib().mpm_get_covariance(ctx, cov, stream), ctx)


def mpm_mcis(surf_off, surf, cand_off, cand, draw_off, u, sigma, eps, d, w, picked, stream):
    n_obj = len(surf_off) - 1
    so = (ctypes.c_int64 * len(surf_off))(*[int(v) for v in surf_off])
    co = (ctypes.c_int64 * len(cand_off))(*[int(v) for v in cand_off])
    do = (ctypes.c_int64 * len(draw_off))(*[int(v) for v in draw_off])
    st = lib().mpm_mcis(n_obj, so, surf, co, cand, do, u, float(sigma), float(eps), d, w, picked, stream)
    if st != 0:
        raise MpmError(st, (lib().mpm_mcis_last_error() or b"").decode())


def mpm_render(n, mean, cov, color, opacity, view, fx, fy, cx, cy, width, height, bg, image, trans, stream):
    v = (ctypes.c_float * 12)(*[float(a) for a in view])
    b = (ctypes.c_float * 3)(*[float(a) for a in bg])
    st = lib().mpm_render(int(n), mean, cov, color, opacity, v, float(fx), float(fy), float(cx), float(cy),
                          int(width), int(height), b, image, trans, stream)
    if st != 0:
        raise MpmError(st, (lib().mpm_render_last_error() or b"").decode())
