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
    args = ap.parse_args()

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


if __name__ == "__main__":
    main()
