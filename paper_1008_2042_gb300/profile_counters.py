"""Per-launch Nsight Compute counters of the projector P and the adjoint P^T on every
multigrid level of the paper-scale workload (512x512x70 voxels, 512x384 imager, 40 views),
written to profiles/kernels.json.

    python -m paper_1008_2042_gb300.profile_counters [--out profiles/kernels.json]

For each kernel and level the single-launch case of ``profile_case`` runs once without the
profiler, then under ``ncu`` with a handful of counters on one launch (the second of the
process, after one untimed call). Recorded per launch: DRAM bytes read and written, warp
and thread instructions executed, L1 throughput and issue activity (percent of peak), the
L2 hit rate and the device time under the profiler (serialised, cold caches: a share, not
a timing). The sha256 of the kernel's sources is stored with each record, and bench.py uses
a record only while the sources still hash to it.

The public P launch (plain epilogue) stands for the reconstruction's P launches (residual
and scaled-direction epilogues), which walk the same rays; the public P^T launch is the
reconstruction's.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")

KERNEL_SOURCES = {
    "k_project": ("project.cu", "project.cuh", "project_kernel.cuh", "project_trace.cu"),
    "k_backproject": ("backproject.cu",),
}
OPS = {"k_project": "project", "k_backproject": "backproject"}
METRICS = ("dram__bytes_read.sum", "dram__bytes_write.sum", "smsp__inst_executed.sum",
           "smsp__thread_inst_executed.sum", "gpu__time_duration.sum",
           "l1tex__throughput.avg.pct_of_peak_sustained_active",
           "smsp__issue_active.avg.pct_of_peak_sustained_active", "lts__t_sector_hit_rate.pct")
LEVELS = (0, 1, 2)


def kernel_sources_sha(kernel: str) -> str:
    """sha256 over the CUDA sources that define a kernel (its files and the internal header)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel] + ("cbct_internal.cuh",):
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _case(kernel: str, level: int):
    return [sys.executable, "-m", "paper_1008_2042_gb300.profile_case", "--op", OPS[kernel],
            "--level", str(level), "--repeat", "1"]


def _ncu_command(kernel: str, level: int, log: str):
    return ["ncu", "--metrics", ",".join(METRICS), "--clock-control", "none", "--print-units", "base",
            "-k", f"regex:{kernel}", "-s", "1", "-c", "1", "--csv", "--log-file", log] + _case(kernel, level)


def _parse(log: str) -> dict:
    with open(log) as fh:
        text = fh.read()
    start = text.find('"ID"')
    rows = list(csv.DictReader(io.StringIO(text[start:])))
    out = {}
    for r in rows:
        v = r["Metric Value"].replace(",", "")
        try:
            out[r["Metric Name"]] = float(v)
        except ValueError:
            pass
        out["kernel_name"] = r["Kernel Name"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "kernels.json"))
    ap.add_argument("--logdir", default=os.path.join(HERE, "_build", "ncu"), help="where the raw ncu CSV logs go")
    a = ap.parse_args(argv)
    os.makedirs(a.logdir, exist_ok=True)
    rec = {"_comment": "Per-launch Nsight Compute counters of P and P^T on every multigrid level of the paper-scale "
                       "workload (one launch per level); written by paper_1008_2042_gb300/profile_counters.py, used "
                       "by bench.py while the kernel sources hash to sources_sha256."}
    for kernel in KERNEL_SOURCES:
        levels = {}
        for lev in LEVELS:
            subprocess.run(_case(kernel, lev), check=True, cwd=ROOT, stdout=subprocess.DEVNULL)
            log = os.path.join(a.logdir, f"counters_{kernel}_l{lev}.csv")
            subprocess.run(_ncu_command(kernel, lev, log), check=True, cwd=ROOT, stdout=subprocess.DEVNULL)
            m = _parse(log)
            levels[str(lev)] = {
                "kernel_name": m.get("kernel_name"),
                "dram_read_bytes": m.get("dram__bytes_read.sum"),
                "dram_write_bytes": m.get("dram__bytes_write.sum"),
                "warp_inst": m.get("smsp__inst_executed.sum"),
                "thread_inst": m.get("smsp__thread_inst_executed.sum"),
                "ncu_duration_ns": m.get("gpu__time_duration.sum"),
                "l1_throughput_pct": m.get("l1tex__throughput.avg.pct_of_peak_sustained_active"),
                "issue_active_pct": m.get("smsp__issue_active.avg.pct_of_peak_sustained_active"),
                "l2_hit_pct": m.get("lts__t_sector_hit_rate.pct"),
            }
            print(kernel, lev, levels[str(lev)], flush=True)
        rec[kernel] = {"sources_sha256": kernel_sources_sha(kernel), "levels": levels,
                       "command": " ".join(_ncu_command(kernel, 0, "<log>")[:-len(_case(kernel, 0))])
                       + " python -m paper_1008_2042_gb300.profile_case --op " + OPS[kernel]
                       + " --level <L> --repeat 1"}
    with open(a.out, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
