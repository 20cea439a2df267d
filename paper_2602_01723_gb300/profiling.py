"""Summaries of Nsight Compute output for profiles/.

    python -m paper_2602_01723_gb300.profiling launches LAUNCHES.csv OUT.md --cmd "..."
    python -m paper_2602_01723_gb300.profiling kernel REPORT.ncu-rep OUT.md --cmd "..." \
        [--traffic-key KEY --particles N]

`launches` turns an `ncu --metrics gpu__time_duration.sum --csv` launch list
into a per-kernel table (launches, total time, share).  `kernel` extracts the
figures used for the roofline from a `--set full` report (duration, DRAM
bytes, issue and stall counters).  With --traffic-key it also stores the
DRAM bytes per launch in profiles/traffic.json, tagged with a hash of the
CUDA sources, so that bench.py reports the traffic only while the kernel is
unchanged."""
from __future__ import annotations

import argparse
import collections
import csv
import hashlib
import io
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


# the files the substep kernel's device code is compiled from
KERNEL_SOURCES = ("mpm_forward.cu", "mpm_math.cuh", "mpm_dev.cuh")


def strip_comments(src: str) -> str:
    """C++ source without its // and /* */ comments (string and character
    literals kept), so that a comment edit leaves the hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return "".join(out)


def source_hash() -> str:
    """sha256 over the sources of the substep kernel's device code, comments
    stripped and runs of white space taken as one space."""
    h = hashlib.sha256()
    csrc = os.path.join(HERE, "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode() + b"\0" + " ".join(strip_comments(fh.read()).split()).encode())
    return h.hexdigest()[:16]


def _ns(value, unit):
    v = float(value.replace(",", ""))
    return v * {"nsecond": 1.0, "usecond": 1e3, "msecond": 1e6, "second": 1e9}.get(unit, 1.0)


def launches(csv_path, out_md, cmd):
    rows = list(csv.reader(open(csv_path)))
    hdr = None
    agg = collections.OrderedDict()
    for r in rows:
        if "Kernel Name" in r:
            hdr = r
            continue
        if hdr and len(r) == len(hdr):
            d = dict(zip(hdr, r))
            if d.get("Metric Name") != "gpu__time_duration.sum":
                continue
            name = d["Kernel Name"].split("(")[0]
            a = agg.setdefault(name, [0, 0.0])
            a[0] += 1
            a[1] += _ns(d["Metric Value"], d["Metric Unit"])
    tot = sum(v[1] for v in agg.values()) or 1.0
    lines = ["# Launch list", "", "Command:", "", "```", cmd, "```", "",
             "Per-launch times are cold-cache and serialised (ncu); compare shares, not absolutes.", "",
             "| kernel | launches | total (us) | per launch (us) | share |", "|---|---|---|---|---|"]
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        lines.append("| `%s` | %d | %.1f | %.1f | %.1f%% |" % (k, n, t / 1e3, t / 1e3 / n, 100 * t / tot))
    with open(out_md, "w") as f:
        f.write("\n".join(lines) + "\n")


WANT = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("lts__throughput.avg.pct_of_peak_sustained_elapsed", "L2 throughput % of peak"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput % of peak"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % (occupancy)"),
    ("sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active", "FMA pipe %"),
    ("sm__inst_executed_pipe_xu.avg.pct_of_peak_sustained_active", "XU (MUFU) pipe %"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("smsp__inst_executed_op_shared_atom.sum", "shared atomic instructions"),
    ("l1tex__t_requests_pipe_lsu_mem_global_op_red.sum", "global reduction requests"),
    ("launch__registers_per_thread", "registers / thread"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
]


def kernel(rep, out_md, cmd, traffic_key=None, particles=None):
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units = rows[0], rows[1]
    idx = {h: i for i, h in enumerate(hdr)}
    lines = ["# Kernel profile", "", "Command:", "", "```", cmd, "```", ""]
    per_launch, inst = [], []
    for r in rows[2:]:
        name = r[idx["Kernel Name"]] if "Kernel Name" in idx else "?"
        lines += ["## `%s`" % name, "", "| metric | value | unit |", "|---|---|---|"]
        for m, label in WANT:
            if m in idx:
                lines.append("| %s (`%s`) | %s | %s |" % (label, m, r[idx[m]], units[idx[m]]))
        stalls = []
        for h, i in idx.items():
            if h.startswith("smsp__average_warps_issue_stalled_") and h.endswith("_per_issue_active.ratio"):
                try:
                    v = float(r[i])
                except ValueError:
                    continue
                stalls.append((v, h[len("smsp__average_warps_issue_stalled_"):-len("_per_issue_active.ratio")]))
        stalls.sort(reverse=True)
        lines += ["", "Top stall reasons (cycles per issued instruction): " +
                  ", ".join("%s %.2f" % (n, v) for v, n in stalls[:6]), ""]
        rd = _bytes(r[idx["dram__bytes_read.sum"]], units[idx["dram__bytes_read.sum"]])
        wr = _bytes(r[idx["dram__bytes_write.sum"]], units[idx["dram__bytes_write.sum"]])
        per_launch.append(rd + wr)
        if "smsp__inst_executed.sum" in idx:
            inst.append(float(r[idx["smsp__inst_executed.sum"]].replace(",", "")))
    with open(out_md, "w") as f:
        f.write("\n".join(lines) + "\n")
    if traffic_key and per_launch:
        d = {}
        if os.path.exists(TRAFFIC):
            with open(TRAFFIC) as f:
                d = json.load(f)
        b = sum(per_launch) / len(per_launch)
        d[traffic_key] = {"bytes_per_launch": b, "source_hash": source_hash(), "launches": len(per_launch),
                          "particles": particles, "note": "dram__bytes_read.sum + dram__bytes_write.sum, "
                          "ncu --set full (cold L2 per replay)", "hashed_sources": list(KERNEL_SOURCES)}
        if inst:
            d[traffic_key]["warp_instructions_per_launch"] = sum(inst) / len(inst)
        with open(TRAFFIC, "w") as f:
            json.dump(d, f, indent=1)


def _bytes(v, unit):
    x = float(v.replace(",", ""))
    return x * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="what", required=True)
    a = sub.add_parser("launches")
    a.add_argument("csv")
    a.add_argument("out")
    a.add_argument("--cmd", required=True)
    b = sub.add_parser("kernel")
    b.add_argument("rep")
    b.add_argument("out")
    b.add_argument("--cmd", required=True)
    b.add_argument("--traffic-key")
    b.add_argument("--particles", type=int)
    args = ap.parse_args()
    if args.what == "launches":
        launches(args.csv, args.out, args.cmd)
    else:
        kernel(args.rep, args.out, args.cmd, args.traffic_key, args.particles)


if __name__ == "__main__":
    main()
