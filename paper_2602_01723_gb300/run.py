"""Runs one of the seeded workloads on the GPU through libmpm.

    python -m paper_2602_01723_gb300.run --workload three_objects_300k --substeps 10

Prints the context counters afterwards.  Used for ad-hoc runs and as the
command under ncu for the kernel profiles."""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="three_objects_300k")
    ap.add_argument("--substeps", type=int, default=10)
    ap.add_argument("--scatter", type=int, default=1)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--record", action="store_true", help="record checkpoints for a reverse pass")
    ap.add_argument("--backward", action="store_true",
                    help="record the run, then time the reverse pass of a loss on the final positions")
    ap.add_argument("--mcis", action="store_true",
                    help="instead: MCIS fill sampling of the three objects (750k candidates), twice")
    ap.add_argument("--render", action="store_true",
                    help="instead: splat the scene's Gaussians (deformed by a stressed key frame) at 1024x768, twice")
    args = ap.parse_args()
    if args.mcis or args.render:
        return other(args)

    import torch
    from . import scenes
    from .build import build
    from .sim import Simulator

    build()
    sc = scenes.WORKLOADS[args.workload]()
    s = Simulator.from_scene(sc, scatter=args.scatter, chunk=args.chunk)
    s.load_scene(sc)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t0 = time.perf_counter()
    e[0].record()
    s.step(args.substeps, record=args.record or args.backward)
    e[1].record()
    if args.backward:
        s.backward([args.substeps], torch.ones((1, s.n, 3), device="cuda"))
    e[2].record()
    s.sync()
    dt = time.perf_counter() - t0
    st = s.stats()
    st["workload"] = args.workload
    st["substeps"] = args.substeps
    st["wall_s"] = dt
    st["forward_ms"] = e[0].elapsed_time(e[1])
    if args.backward:
        st["backward_ms"] = e[1].elapsed_time(e[2])
    print(json.dumps(st))
    s.close()


def other(args):
    """One MCIS run or one splat, repeated once (the second run is the warm one)."""
    import torch
    from . import scenes
    from .build import build
    from .sim import Simulator, mcis, render

    build()
    out = {}
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.mcis:
            case = scenes.mcis_case()
            torch.cuda.synchronize()
            e0.record()
            r = mcis(case["surf_off"], case["surf"], case["cand_off"], case["cand"], case["draw_off"], case["u"])
            e1.record()
            torch.cuda.synchronize()
            out = {"what": "mcis", "candidates": int(case["cand_off"][-1]), "ms": e0.elapsed_time(e1),
                   "picked_valid": bool((r["picked"] >= 0).all().item())}
        else:
            sc = scenes.WORKLOADS[args.workload]()
            s = Simulator.from_scene(sc)
            v, C, F = scenes.key_frames(sc, 1, k_seed=81, fs=0.05)[0]
            s.load(sc.x, sc.vol, sc.mat_id, v=v, C=C, F=F)
            s.load_covariance(scenes.gaussian_covariances(sc))
            cov = s.covariance()
            col, op = scenes.gaussian_appearance(sc)
            dev = torch.device("cuda")
            mean = torch.as_tensor(sc.x, device=dev)
            W, H = 1024, 768
            view, fx, fy, cx, cy = scenes.camera(W, H)
            torch.cuda.synchronize()
            e0.record()
            img, T = render(mean, cov, torch.as_tensor(col, device=dev), torch.as_tensor(op, device=dev), view,
                            fx, fy, cx, cy, W, H)
            e1.record()
            torch.cuda.synchronize()
            s.close()
            out = {"what": "render", "gaussians": sc.n, "ms": e0.elapsed_time(e1),
                   "coverage": float((T < 0.5).float().mean().item())}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
