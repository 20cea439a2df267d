#!/usr/bin/env python
"""Benchmark of the MLS-MPM substep (libmpm) on one node.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (the configuration the headline metric is quoted on): the
300,000-particle three-object scene (sphere elastic, torus plasticine, box
sand) on a 128^3 grid, dt 5e-5, synthetic seeded inputs.  One step = one full
2,000-substep forward simulation from the initial state, which is resident in
HBM when the timed region starts; L2 is flushed (a 256 MiB write) between
timed steps, outside the timed events.  With N > 1 (torchrun, one process per
GPU, NCCL) every rank runs its own replica (weak scaling; the single scene is
not sharded), and rank 0 prints one JSON line with the max-over-ranks time.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-substeps/sec fwd and fwd+bwd at 1 GB300; HBM roofline %; err vs FP64"
UNIT = "particle-substeps/s"
WORKLOAD = "three_objects_300k"
# algorithmic bytes per particle-substep of the forward substep: the particle
# state read once and written once (2 x 96 B), the material word (4 B) and the
# grid (about 6 B per particle: 16 B written and read per active node, ~0.19
# active nodes per particle)
FWD_BYTES_PER_PS = 200.0
ORACLE_SAMPLE_SUBSTEPS = 30
REF_STEP_SUBSTEPS = 4
FB_WORKLOAD = "ball_50k"
# fwd+bwd algorithmic bytes per particle-substep: the forward (200 B), the
# recompute of the checkpoint segment with the tape write (~200 B), and the
# reverse substep (tape state read by the recomputed P2G, the G2P adjoint and
# the P2G adjoint, adjoint state in and out, parameter gradients: ~480 B)
FB_BYTES_PER_PS = 880.0
# BGDO stage 2 per particle and key frame: one pseudo substep (200 B) and the
# signal pass (key-frame F and Lame pair 44 B, post-step F 36 B, G read and
# written 8 B); the copy of the key frame is not counted
BGDO_BYTES_PER_PK = 288.0
# deformed covariance per particle: F (36 B) and rest covariance (24 B) read,
# covariance (24 B) written
COV_BYTES_PER_P = 84.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_peak_clock_mhz():
    """Maximum SM clock: from MEASURED_PEAKS.json, else the GB300's 2070 MHz."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("sm_max_mhz"):
            return float(d["sm_max_mhz"])
    return 2070.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    import torch
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", 0))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return dist, dist.get_rank(), dist.get_world_size(), local
    torch.cuda.set_device(0)
    return None, 0, 1, 0


def max_over_ranks(local_ms, dist, device=None):
    """The slowest rank's time: whole-job throughput divides by it."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_units(n_units, rank, world):
    """Contiguous, near-equal shard [lo, hi) of n_units independent problems
    (instances of a batch) for one rank; no data moves between shards."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def oracle_rate(sc, n_sub):
    """Timed FP64 oracle on the first n_sub substeps of the workload."""
    import oracle as orc
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.params)
    st = orc.new_state(sc.x, sc.v)
    t0 = time.perf_counter()
    out = orc.run(cfg, st, mat, n_sub)
    t = time.perf_counter() - t0
    return sc.n * n_sub / t, t, out


def _oracle_instance_rate(job):
    """One batch instance alone on the oracle (a worker of the all-core
    baseline; runs in a spawned process)."""
    idx, n_sub = job
    from paper_2602_01723_gb300 import scenes
    import oracle as orc
    sc = scenes.batch_64()
    sel = sc.instance == idx
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol[sel], sc.mat_id[sel] * 0, [sc.materials[idx]])
    orc.run(cfg, orc.new_state(sc.x[sel], sc.v[sel]), mat, n_sub)
    return int(sel.sum()) * n_sub


def oracle_all_cores(n_inst=32, n_sub=10):
    """The oracle as it stands on all host cores: independent instances of
    the 64-instance batch (each its own problem on its own grid), one process
    per core (spawned), over a bounded sample."""
    import multiprocessing as mp
    import oracle as orc
    orc.build()
    cores = min(os.cpu_count() or 1, n_inst)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_instance_rate, [(0, 1)] * cores)          # workers up, libraries loaded
        t0 = time.perf_counter()
        units = sum(pool.map(_oracle_instance_rate, [(i, n_sub) for i in range(n_inst)]))
        t = time.perf_counter() - t0
    return {"value": units / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d substeps of each of the first %d instances of the 64-instance batch, one process per "
                      "core, FP64, %.1f s" % (n_sub, n_inst, t)}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle timed on the host cores."""
    if "RANK" in os.environ and int(os.environ["RANK"]) != 0:
        return
    from paper_2602_01723_gb300 import scenes
    import oracle as orc
    orc.build()
    sc = scenes.WORKLOADS[WORKLOAD]()
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.params)
    st = orc.new_state(sc.x, sc.v)
    for _ in range(args.warmup):
        st = orc.run(cfg, st, mat, REF_STEP_SUBSTEPS)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = orc.run(cfg, st, mat, REF_STEP_SUBSTEPS)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sc.n * REF_STEP_SUBSTEPS * args.steps / tot
    sample = "%d substeps of the %d-particle scene per step, FP64, 1 thread" % (REF_STEP_SUBSTEPS, sc.n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "particles": sc.n, "grid": sc.grid_res,
                                            "dt": sc.dt, "substeps_per_step": REF_STEP_SUBSTEPS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    dist, rank, world, local = dist_setup(args.gpus)
    from __graft_entry__ import build
    if rank == 0 or dist is None:
        build()
    if dist is not None:
        dist.barrier()
        build()
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import Simulator, _p, _stream
    from paper_2602_01723_gb300 import _lib as L

    dev = torch.device("cuda", torch.cuda.current_device())
    sc = scenes.WORKLOADS[WORKLOAD]()
    n, S = sc.n, sc.n_substeps
    sim = Simulator.from_scene(sc)
    # initial state resident on the device
    x0 = torch.as_tensor(sc.x, device=dev).contiguous()
    v0 = torch.as_tensor(sc.v, device=dev).contiguous()
    vol = torch.as_tensor(sc.vol, device=dev).contiguous()
    mid = torch.as_tensor(sc.mat_id, dtype=torch.int32, device=dev).contiguous()
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    sim.n = n

    def one_step():
        L.mpm_load_particles(sim.ctx, n, _p(x0), _p(v0), None, None, _p(vol), _p(mid), None, None, _stream())
        sim.step(S)

    for _ in range(args.warmup):
        one_step()
    sim.sync()
    torch.cuda.synchronize()

    l0 = sim.stats()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                 # L2 flush between timed steps, outside the events
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    sim.sync()
    launches = sim.stats()["launches"] - l0
    # the same steps again with CUDA events around every launch of the
    # substep kernel (graph replay is off while tracing): the dominant
    # kernel's average duration for the roofline
    sim.trace(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        one_step()
    sim.sync()
    tr = sim.trace(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = world * n * S * args.steps / (tot_ms * 1e-3)

    # roofline of the dominant kernel: the fused G2P + update + P2G kernel
    fused_ms, fused_n = tr["fused"]
    peak, peak_kind = load_peaks()
    avg_fused_s = fused_ms * 1e-3 / max(fused_n, 1)
    achieved = FWD_BYTES_PER_PS * n / avg_fused_s / 1e9
    # DRAM bytes per launch from the committed ncu capture, only while the
    # kernel sources are the ones that capture measured
    traffic = inst = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        from paper_2602_01723_gb300.profiling import source_hash
        with open(prof) as f:
            t = json.load(f).get("k_substep_fused_three_objects_300k")
        if t and t.get("source_hash") == source_hash() and t.get("particles") == n:
            traffic = t["bytes_per_launch"]
            inst = t.get("warp_instructions_per_launch")
    # the same kernel against the issue ceiling: warp instructions per launch
    # (same capture) over the launch time, against one instruction per cycle
    # per scheduler (4 per SM) at the maximum SM clock
    issue = None
    if traffic is not None and inst:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak_issue = sms * 4 * load_peak_clock_mhz() * 1e6
        issue = {"warp_instructions_per_launch": inst, "achieved": inst / avg_fused_s, "peak": peak_issue,
                 "unit": "warp instructions/s", "frac": inst / avg_fused_s / peak_issue,
                 "peak_kind": "SMs x 4 schedulers x maximum SM clock"}

    # end to end through the C ABI with host (pinned) buffers
    xh = torch.as_tensor(sc.x).pin_memory()
    vh = torch.as_tensor(sc.v).pin_memory()
    volh = torch.as_tensor(sc.vol).pin_memory()
    midh = torch.as_tensor(sc.mat_id, dtype=torch.int32).pin_memory()
    xout = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for k in range(max(1, min(args.steps, 3))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.mpm_load_particles(sim.ctx, n, _p(xh), _p(vh), None, None, _p(volh), _p(midh), None, None, _stream())
        sim.step(S)
        L.mpm_get_particles(sim.ctx, _p(xout), None, None, None, _stream())
        sim.sync()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_v = world * n * S / (statistics.mean(e2e_ms) * 1e-3)
    h2d = n * (12 + 12 + 4 + 4)
    d2h = n * 12

    # error against the FP64 oracle, both sides from the same seeded inputs:
    # (1) the P2G grid (all nodes) of a stressed key frame of the scene;
    # (2) positions after the oracle's timed sample of free-running substeps
    #     from the scene's start (the CPU baseline run below)
    err = {}
    cpu = None
    if rank == 0:
        import oracle as orc
        cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
        mat = orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, sc.params)
        kv, kC, kF = scenes.key_frames(sc, 1, k_seed=46, vs=0.5, cs=2.0, fs=0.1)[0]
        sim.load(sc.x, sc.vol, sc.mat_id, v=kv, C=kC, F=kF)
        m, mv = sim.debug_p2g()
        gm, gmv = orc.p2g(cfg, orc.new_state(sc.x, kv, kC, kF), mat)
        floor = np.abs(gm).max() * 9.8 * sc.dt
        err["grid_m_rel"] = float(np.abs(m[0].double().cpu().numpy() - gm).max() / max(np.abs(gm).max(), floor))
        err["grid_mv_rel"] = float(np.abs(mv[0].double().cpu().numpy() - gmv).max() / max(np.abs(gmv).max(), floor))
        cpu = oracle_rate(sc, ORACLE_SAMPLE_SUBSTEPS)
        sim.load_scene(sc)
        sim.step(ORACLE_SAMPLE_SUBSTEPS)
        xg = sim.positions().double().cpu().numpy()
        err["x_after_%d_substeps_max_dx" % ORACLE_SAMPLE_SUBSTEPS] = float(np.abs(xg - cpu[2]["x"]).max() / sc.dx)
        err["note"] = ("FP32 GPU vs FP64 oracle from the same seeded inputs: P2G of a stressed key frame, and "
                       "free-running positions after %d substeps" % ORACLE_SAMPLE_SUBSTEPS)

    fb = fwd_bwd(args, dev, flush, world, dist)
    bg = guarded(bgdo_leg, args, sim, sc, (x0, v0, vol, mid), flush)
    mc = guarded(mcis_leg, args, dev, flush)
    cf = guarded(configs_leg, args, dev, flush)
    rd = guarded(render_leg, args, sim, sc, dev, flush)
    if rank == 0:
        # every leg's result against the FP64 oracle, outside the timed regions
        errs = guarded(fp64_errors, dev)
        for leg, key in ((fb, "fwd_bwd"), (bg, "bgdo"), (mc, "mcis"), (rd, "render")):
            leg["err_vs_fp64"] = errs.get(key, errs)
        for name in ("cube_8k", "batch_64", "large_2m"):
            if name in cf:
                cf[name]["err_vs_fp64"] = errs.get(name, errs)
        cpu_all = guarded(oracle_all_cores)

    if rank == 0:
        cpu_v, cpu_t = cpu[0], cpu[1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded shell + interior scene; the paper's 3DGS scenes are not available)",
            "config": {"workload": WORKLOAD, "particles": n, "grid": sc.grid_res, "dt": sc.dt,
                       "substeps_per_step": S, "materials": "elastic FCR / von Mises / Drucker-Prager",
                       "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_substep<fused>", "avg_launch_us": avg_fused_s * 1e6,
                         "launches": fused_n, "bytes_per_particle_substep": FWD_BYTES_PER_PS,
                         "peak_kind": peak_kind,
                         "timing": "CUDA events around each launch on the launching stream, over a second pass "
                                   "of the timed steps", "issue": issue},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d substeps of the %d-particle scene, FP64 oracle, 1 thread, %.1f s"
                                       % (ORACLE_SAMPLE_SUBSTEPS, n, cpu_t)},
            "cpu_baseline_all_cores": cpu_all,
            "clocks": clk.summary(),
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "err_vs_fp64": err,
            "fwd_bwd": fb,
            "bgdo": bg,
            "configs": cf,
            "mcis": mc,
            "render": rd,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def guarded(leg, *a):
    """Runs one auxiliary leg; a failure is reported in its place (with the
    exception) instead of losing the whole line."""
    try:
        return leg(*a)
    except Exception as e:  # noqa: BLE001 -- reported, not hidden
        import torch
        try:
            torch.cuda.synchronize()
        except Exception:  # noqa: BLE001
            pass
        return {"error": "%s: %s" % (type(e).__name__, e)}


def bgdo_leg(args, sim, sc, init, flush):
    """One BGDO iteration on the same scene (§4.3, Algorithm 1): stage 1 is
    the full forward with key frames at substeps 0, S/2 and S; stage 2 the
    three pseudo substeps and the log-E update.  Also times the export of the
    deformed Gaussian covariances F Sigma F^T (§3.2)."""
    import torch
    from paper_2602_01723_gb300 import _lib as L
    from paper_2602_01723_gb300.sim import _p, _stream
    x0, v0, vol, mid = init
    n, S = sc.n, sc.n_substeps

    def stage1():
        L.mpm_load_particles(sim.ctx, n, _p(x0), _p(v0), None, None, _p(vol), _p(mid), None, None, _stream())
        sim.snapshot(0)
        sim.step(S // 2)
        sim.snapshot(1)
        sim.step(S - S // 2)
        sim.snapshot(2)

    def timed(fn, reps):
        ms = []
        for k in range(reps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    stage1()
    sim.bgdo([0, 1, 2])
    sim.sync()
    s1 = timed(stage1, max(1, min(args.steps, 2)))
    out = {}

    def stage2():
        out.update(sim.bgdo([0, 1, 2]))
    s2 = timed(stage2, max(3, args.steps))
    sim.sync()
    peak, _ = load_peaks()
    pk = n * 3 / (s2 * 1e-3)
    cov0 = torch.zeros((n, 6), device=x0.device)
    cov0[:, 0] = cov0[:, 3] = cov0[:, 5] = 1e-6
    sim.load_covariance(cov0)
    cov = torch.empty((n, 6), device=x0.device)
    reps = 20

    def cov_burst():
        for _ in range(reps):
            sim.covariance(out=cov)
    cms = timed(cov_burst, max(3, args.steps)) / reps
    return {"workload": sc.name, "particles": n, "keys": 3, "stage1_ms": s1, "stage2_ms": s2,
            "iteration_ms": s1 + s2, "particle_keys_per_s": pk,
            "stage2_bytes_per_particle_key": BGDO_BYTES_PER_PK,
            "stage2_hbm_frac": pk * BGDO_BYTES_PER_PK / 1e9 / peak,
            "G_finite": bool(torch.isfinite(out["G"]).all().item()),
            "covariance": {"us": cms * 1e3, "timing": "%d back-to-back exports between events" % reps,
                           "bytes_per_particle": COV_BYTES_PER_P,
                           "hbm_frac": n * COV_BYTES_PER_P / (cms * 1e-3) / 1e9 / peak},
            "note": "CUDA events, medians; stage 1 includes the three snapshot copies"}


def one_graph_fwd_bwd(sim, prm0, init, frames, target, flush, units, ref):
    """The whole fwd+bwd (load, recorded forward, frame positions, loss,
    reverse pass, per-material reduction) captured once into one CUDA graph
    with torch.cuda.graph, then replayed: CUDA events around each replay."""
    import torch
    from paper_2602_01723_gb300.sim import trajectory
    p = prm0.clone().requires_grad_(True)

    def fbg():
        xs = trajectory(p, sim, init, frames)
        (g,) = torch.autograd.grad(((xs - target) ** 2).sum(), p)
        return sim.reduce_by_material(g)
    fbg()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = fbg()
    ms = []
    for k in range(3):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    sim.sync()
    t = statistics.median(ms)
    rel = float((out - ref).abs().max() / ref.abs().max())
    del graph
    return {"ms": t, "value": units / (t * 1e-3), "unit": UNIT, "max_rel_diff_vs_eager": rel}


def configs_leg(args, dev, flush):
    """Forward throughput of the other workload shapes (the 8k cube, the
    64-instance batch on its own 64^3 grids, the 2M-particle 256^3
    block-sparse scene), each a full run of its substeps from the resident
    initial state; fwd+bwd of the batch (10-frame loss, per-instance
    parameter gradients) and of the 2M scene (10-frame loss, per-object
    gradients, checkpoint every 25), with the device memory in use
    afterwards."""
    import numpy as np
    import torch
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import Simulator, trajectory
    from paper_2602_01723_gb300 import _lib as L
    from paper_2602_01723_gb300.sim import _p, _stream
    out = {}
    for name in ("cube_8k", "batch_64", "large_2m"):
        sc = scenes.WORKLOADS[name]()
        free0, total = torch.cuda.mem_get_info()
        sim = Simulator.from_scene(sc)
        n, S = sc.n, sc.n_substeps
        x0, v0 = torch.as_tensor(sc.x, device=dev), torch.as_tensor(sc.v, device=dev)
        vol = torch.as_tensor(sc.vol, device=dev)
        mid = torch.as_tensor(sc.mat_id, dtype=torch.int32, device=dev)
        inst = None if sc.instance is None else torch.as_tensor(sc.instance, dtype=torch.int32, device=dev)
        prm = None if sc.params is None else torch.as_tensor(sc.params, device=dev)
        sim.n = n

        def run():
            L.mpm_load_particles(sim.ctx, n, _p(x0), _p(v0), None, None, _p(vol), _p(mid), _p(inst), _p(prm),
                                 _stream())
            sim.step(S)
        tuned = None
        if name == "batch_64":
            # the batch runs with autotuned tile sizes (scatter strategy, chunk)
            L.mpm_load_particles(sim.ctx, n, _p(x0), _p(v0), None, None, _p(vol), _p(mid), _p(inst), _p(prm),
                                 _stream())
            tuned = sim.autotune(20)
        run()
        sim.sync()
        ms = []
        for k in range(max(2, min(args.steps, 3))):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        out[name] = {"particles": n, "substeps": S, "ms": t, "value": n * S / (t * 1e-3), "unit": UNIT,
                     "autotuned": tuned,
                     "hbm_frac": n * S / (t * 1e-3) * FWD_BYTES_PER_PS / 1e9 / load_peaks()[0]}
        if name in ("batch_64", "large_2m"):
            frames = [int(f) for f in (np.linspace(S / 10, S, 10) if sc.frame_sub is None else sc.frame_sub)]
            init = {"x": x0, "v": v0, "vol": vol, "mat_id": mid, "instance": inst}
            prm0 = torch.tensor(np.stack([np.log([m["E"] for m in sc.materials]), [m["nu"] for m in sc.materials],
                                          [m["yield_stress"] for m in sc.materials]], 1)[sc.mat_id],
                                dtype=torch.float32, device=dev)
            target = x0[None] + 0.005

            def fb():
                p = prm0.clone().requires_grad_(True)
                xs = trajectory(p, sim, init, frames)
                ((xs - target) ** 2).sum().backward()
                return sim.reduce_by_material(p.grad)
            fb()
            torch.cuda.synchronize()
            fms = []
            for k in range(2):
                flush.fill_(float(k))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g = fb()
                e1.record()
                torch.cuda.synchronize()
                fms.append(e0.elapsed_time(e1))
            tf = statistics.median(fms)
            one_graph = None
            if name == "batch_64":
                try:
                    one_graph = one_graph_fwd_bwd(sim, prm0, init, frames, target, flush, n * S, fb())
                except Exception as e:  # noqa: BLE001 -- reported in the line
                    one_graph = {"error": "%s: %s" % (type(e).__name__, e)}
            free1, _ = torch.cuda.mem_get_info()
            out[name]["fwd_bwd"] = {"ms": tf, "value": n * S / (tf * 1e-3), "unit": UNIT,
                                    "ckpt_every": int(sc.ckpt_every or 20), "frames": len(frames),
                                    "grads_finite": bool(torch.isfinite(g).all().item()),
                                    "grads": "per instance" if sc.n_instances > 1 else "per object (material id)",
                                    "one_cuda_graph": one_graph,
                                    "device_memory_gb": (free0 - free1) / 1e9,
                                    "device_memory": "cudaMemGetInfo after the fwd+bwd runs minus before the context "
                                                     "was created: the context (state, grids, checkpoints, tapes, "
                                                     "adjoint buffers) and the run's torch tensors"}
        sim.close()
    out["note"] = "CUDA events, medians; L2 flushed between runs; inputs resident on the device"
    return out


def mcis_leg(args, dev, flush):
    """MCIS fill sampling (§4.1) for the three objects of the same scene:
    108k surface points, 750k candidates, 192k draws, inputs resident on the
    device; CUDA events around the whole call (binning, nearest-surface
    search, weights, scans, draws)."""
    import torch
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import mcis
    c = scenes.mcis_case()
    surf = torch.as_tensor(c["surf"], device=dev)
    cand = torch.as_tensor(c["cand"], device=dev)
    u = torch.as_tensor(c["u"], device=dev)
    mcis(c["surf_off"], surf, c["cand_off"], cand, c["draw_off"], u)
    ms = []
    for k in range(max(3, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = mcis(c["surf_off"], surf, c["cand_off"], cand, c["draw_off"], u)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    nc = int(c["cand_off"][-1])
    return {"surface_points": int(c["surf_off"][-1]), "candidates": nc, "draws": int(c["draw_off"][-1]),
            "ms": t, "candidates_per_s": nc / (t * 1e-3),
            "picked_valid": bool(((out["picked"] >= 0) & (out["picked"] < nc)).all().item()),
            "note": "CUDA events, median; includes the stream-ordered scratch allocation"}


def render_leg(args, sim, sc, dev, flush):
    """Splatting (§3.1) of the same scene's 300k Gaussians, deformed by a
    stressed key frame (F Sigma F^T from the library), into a 1024 x 768
    image; CUDA events around the whole call (projection, tile keys, radix
    sort, compositing)."""
    import torch
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import render
    v, C, F = scenes.key_frames(sc, 1, k_seed=81, fs=0.05)[0]
    sim.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F)
    sim.load_covariance(scenes.gaussian_covariances(sc))
    cov = sim.covariance()
    col, op = scenes.gaussian_appearance(sc)
    mean = torch.as_tensor(sc.x, device=dev)
    col_d, op_d = torch.as_tensor(col, device=dev), torch.as_tensor(op, device=dev)
    W, H = 1024, 768
    view, fx, fy, cx, cy = scenes.camera(W, H)
    render(mean, cov, col_d, op_d, view, fx, fy, cx, cy, W, H)
    ms = []
    for k in range(max(3, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        img, T = render(mean, cov, col_d, op_d, view, fx, fy, cx, cy, W, H)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    return {"gaussians": sc.n, "width": W, "height": H, "ms": t, "gaussians_per_s": sc.n / (t * 1e-3),
            "coverage": float((T < 0.5).float().mean().item()),
            "note": "CUDA events, median; includes the scratch allocation and the host read of the key count"}


def fp64_errors(dev):
    """The error of each leg's result against the FP64 oracle.  Both sides
    start from the same seeded inputs; nothing the GPU computes is given to
    the oracle.  Norms: positions max |dx| / dx; gradients
    ||g - g_ref||_2 / ||g_ref||_2 per parameter kind; grids max |diff| over
    max(|ref|, |m_ref| |g| dt); BGDO, MCIS and splat per-element maxima."""
    import numpy as np
    import torch
    import oracle as orc
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import Simulator, mcis, render
    orc.build()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    out = {}

    def setup(sc, params=None):
        return (orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity),
                orc.Material.from_table(sc.vol, sc.mat_id, sc.materials, params))

    # cube_8k: the configured 100-substep run
    sc = scenes.cube_8k()
    s = Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(sc.n_substeps)
    xg = s.positions().double().cpu().numpy()
    s.close()
    cfg, mat = setup(sc)
    ref = orc.run(cfg, orc.new_state(sc.x, sc.v), mat, sc.n_substeps)
    out["cube_8k"] = {"x_max_dx": float(np.abs(xg - ref["x"]).max() / sc.dx), "substeps": sc.n_substeps}

    # batch_64: the whole batch on the GPU for its 200 substeps; its smallest
    # instance alone on the oracle
    sc = scenes.batch_64()
    s = Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(sc.n_substeps)
    xg = s.positions().double().cpu().numpy()
    s.close()
    b = int(np.argmin(np.bincount(sc.instance, minlength=sc.n_instances)))
    sel = sc.instance == b
    cfg = orc.Cfg(sc.grid_res, sc.dx, sc.dt, sc.gravity)
    mat = orc.Material.from_table(sc.vol[sel], sc.mat_id[sel] * 0, [sc.materials[b]])
    ref = orc.run(cfg, orc.new_state(sc.x[sel], sc.v[sel]), mat, sc.n_substeps)
    out["batch_64"] = {"x_max_dx": float(np.abs(xg[sel] - ref["x"]).max() / sc.dx), "instance": b,
                       "particles": int(sel.sum()), "substeps": sc.n_substeps}

    # large_2m: the P2G grid of a stressed seeded key frame, all 2M particles
    # on the 256^3 grid, every node
    sc = scenes.large_2m()
    v, C, F = scenes.key_frames(sc, 1, k_seed=47, vs=0.5, cs=2.0, fs=0.05)[0]
    s = Simulator.from_scene(sc)
    s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F)
    m, mv = s.debug_p2g()
    m, mv = m[0].double().cpu().numpy(), mv[0].double().cpu().numpy()
    s.close()
    cfg, mat = setup(sc)
    gm, gmv = orc.p2g(cfg, orc.new_state(sc.x, v, C, F), mat)
    floor = np.abs(gm).max() * 9.8 * sc.dt
    out["large_2m"] = {"grid_m_rel": float(np.abs(m - gm).max() / max(np.abs(gm).max(), floor)),
                       "grid_mv_rel": float(np.abs(mv - gmv).max() / max(np.abs(gmv).max(), floor))}
    del m, mv, gm, gmv

    # fwd_bwd: the differentiable ball's 512-particle copy as configured (400
    # substeps, checkpoint 20, ten frames), the same seeded cotangents on both
    # sides
    sc = scenes.ball_512()
    frames = [int(f) for f in sc.frame_sub]
    cot = np.random.default_rng(400).standard_normal((len(frames), sc.n, 3))
    s = Simulator.from_scene(sc)
    s.load_scene(sc)
    s.step(sc.n_substeps, record=True)
    xg = s.positions().double().cpu().numpy()
    g = s.backward(frames, torch.as_tensor(cot, dtype=torch.float32)).double().cpu().numpy()
    s.close()
    cfg, mat = setup(sc, sc.params)
    _, tape = orc.run(cfg, orc.new_state(sc.x, sc.v), mat, sc.n_substeps, tape=True)
    _, gr = orc.backward(cfg, mat, tape, frames, cot)
    out["fwd_bwd"] = {"workload": "ball_512 (the 512-particle, 16^3 copy)",
                      "grad_logE_rel": rel(g[:, 0], gr[:, 0]), "grad_nu_rel": rel(g[:, 1], gr[:, 1]),
                      "x_max_dx": float(np.abs(xg - tape[-1][:, 0:3]).max() / sc.dx),
                      "cotangents": "seeded N(0, 1), the same on both sides"}

    # bgdo: stage 2 from three seeded key frames of the 300k scene, every particle
    sc = scenes.three_objects_300k()
    keys = scenes.key_frames(sc, 3, k_seed=42, cs=2.0, fs=0.03)
    s = Simulator.from_scene(sc)
    for k, (v, C, F) in enumerate(keys):
        s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F)
        s.snapshot(k)
    got = {k: t.double().cpu().numpy() for k, t in s.bgdo([0, 1, 2], signals=True).items()}
    s.close()
    cfg, mat = setup(sc)
    ref = orc.bgdo(cfg, [orc.new_state(sc.x, v, C, F) for v, C, F in keys], mat, label=sc.mat_id)
    out["bgdo"] = {"G_max_abs": float(np.abs(got["G"] - ref["G"]).max()),
                   "g_tau_max_rel": float((np.abs(got["g_tau"] - ref["g_tau"]) / np.maximum(np.abs(ref["g_tau"]), 1e-30)).max()),
                   "delta_max_abs": float(np.abs(got["delta"] - ref["delta"]).max()),
                   "sample": "every particle, three seeded key frames"}

    # mcis: 1,500 sampled candidates against the oracle's brute force over
    # their object's surface; every draw against the inverse CDF of the GPU's
    # weights (exact integers)
    c = scenes.mcis_case()
    r = mcis(c["surf_off"], c["surf"], c["cand_off"], c["cand"], c["draw_off"], c["u"])
    gd, gw, gp = (r[k].cpu().numpy() for k in ("d", "w", "picked"))
    so, co, do = c["surf_off"], c["cand_off"], c["draw_off"]
    rng = np.random.default_rng(9)
    cut = 0.02 * np.sqrt(2 * np.log(1e6))
    ed = ew = 0.0
    draws_ok = True
    for k in range(3):
        idx = co[k] + rng.choice(co[k + 1] - co[k], 500, replace=False)
        sub = orc.mcis([0, so[k + 1] - so[k]], c["surf"][so[k]:so[k + 1]], [0, 500], c["cand"][idx], [0, 0], [])
        near = sub["d"] < cut
        ed = max(ed, float((np.abs(gd[idx][near] - sub["d"][near]) / sub["d"][near].clip(1e-300)).max()))
        ew = max(ew, float((np.abs(gw[idx] - sub["w"]) / sub["w"]).max()))
        wq = np.floor(gw[co[k]:co[k + 1]] * 2.0 ** 40 + 0.5).astype(np.int64)
        cum = np.cumsum(wq)
        t = np.floor(c["u"][do[k]:do[k + 1]] * float(cum[-1])).astype(np.int64)
        expect = co[k] + np.minimum(np.searchsorted(cum, t, side="right"), len(cum) - 1)
        draws_ok = draws_ok and bool(np.array_equal(gp[do[k]:do[k + 1]], expect))
    out["mcis"] = {"d_max_rel": ed, "w_max_rel": ew, "draws_exact": draws_ok,
                   "sample": "1,500 candidates (500 per object); all 192k draws"}

    # render: a tile-aligned 64 x 64 crop of the 1024 x 768 splat of the same
    # deformed Gaussians; per pixel the excess over the order-ambiguity bound
    sc = scenes.three_objects_300k()
    v, C, F = scenes.key_frames(sc, 1, k_seed=81, fs=0.05)[0]
    cov = orc.covariance(F, scenes.gaussian_covariances(sc)).astype(np.float32)
    col, op = scenes.gaussian_appearance(sc)
    W, H = 1024, 768
    view, fx, fy, cx, cy = scenes.camera(W, H)
    img, _ = render(sc.x, cov, col, op, view, fx, fy, cx, cy, W, H)
    x0, y0 = 464, 400
    ref, _, amb = orc.render(sc.x, cov, col, op, view, fx, fy, cx - x0, cy - y0, 64, 64, tie_eps=2.0 ** -21)
    e = np.abs(img.cpu().numpy()[y0:y0 + 64, x0:x0 + 64] - ref).max(axis=2)
    out["render"] = {"pixel_max_abs": float(e.max()), "pixel_max_abs_beyond_order_bound": float((e - amb).max()),
                     "pixels_beyond_2e-4_and_bound": int(((e - amb) > 2e-4).sum()), "crop": "64 x 64 at (464, 400)"}
    return out


def fwd_bwd(args, dev, flush, world, dist):
    """fwd+bwd throughput on the 50k-particle differentiable ball: one step =
    a recorded 400-substep forward (checkpoint every 20) plus the reverse pass
    for the 10-frame position MSE against a target run with the seeded
    ground-truth parameters."""
    import numpy as np
    import torch
    from paper_2602_01723_gb300 import scenes
    from paper_2602_01723_gb300.sim import Simulator, trajectory

    sc = scenes.WORKLOADS[FB_WORKLOAD]()
    n, S = sc.n, sc.n_substeps
    frames = [int(f) for f in sc.frame_sub]
    sim = Simulator.from_scene(sc)
    init = {"x": torch.as_tensor(sc.x, device=dev), "v": torch.as_tensor(sc.v, device=dev),
            "vol": torch.as_tensor(sc.vol, device=dev),
            "mat_id": torch.as_tensor(sc.mat_id, dtype=torch.int32, device=dev)}
    with torch.no_grad():
        target = trajectory(torch.as_tensor(sc.extra["params_true"], device=dev), sim, init, frames).clone()
    guess = torch.as_tensor(sc.params, device=dev)

    def one_step():
        params = guess.clone().requires_grad_(True)
        xs = trajectory(params, sim, init, frames)
        loss = ((xs - target) ** 2).sum() / (len(frames) * n)
        loss.backward()
        return params.grad

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l0 = sim.stats()["launches"]
    ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g = one_step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = sim.stats()["launches"] - l0
    tot = max_over_ranks(sum(ms), dist, dev)
    value = world * n * S * args.steps / (tot * 1e-3)
    peak, _ = load_peaks()
    sim.close()
    return {"value": value, "unit": UNIT, "workload": FB_WORKLOAD, "particles": n, "grid": sc.grid_res,
            "substeps_per_step": S, "ckpt_every": sc.ckpt_every, "frames": len(frames),
            "ms_per_step": tot / args.steps, "bytes_per_particle_substep": FB_BYTES_PER_PS,
            "hbm_frac": value * FB_BYTES_PER_PS / 1e9 / world / peak, "gpu_launches": int(launches),
            "grad_finite": bool(torch.isfinite(g).all().item()),
            "note": "device time of recorded forward + reverse pass, CUDA events; L2 flushed between steps"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
