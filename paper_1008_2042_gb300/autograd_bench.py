"""Throughput of the differentiable batch: forward P and backward P^T through the
autograd wrapper for 8 volumes of 256x256x64 voxels (1.0 mm), 60 views, 256x192 imager
(1.5 mm), loss ½‖P f − y‖².

    python -m paper_1008_2042_gb300.autograd_bench [--batch 8] [--steps 5] [--warmup 3]

Prints one JSON line: volumes/s and ray-voxel updates/s of forward + backward (device time,
CUDA events; inputs resident on the GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

import paper_1008_2042_gb300 as cb  # noqa: E402
from paper_1008_2042_gb300 import autograd, build  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)
    build.build()
    geom = synth.Geometry(nx=256, ny=256, nz=64, dx=1.0, dy=1.0, dz=1.0, nu=256, nv=192, du=1.5, dv=1.5,
                          n_views=60)
    g = cb.Geometry(geom)
    import numpy as np
    fs = np.stack([synth.voxelize(geom, synth.random_ellipsoids(geom, 1004 + b, n=8)) for b in range(a.batch)])
    f = torch.tensor(fs, dtype=torch.float32, device="cuda")
    y = torch.rand((a.batch,) + geom.proj_shape, device="cuda") * 3.0
    nnz = cb.count_nnz(g)

    def step():
        x = f.clone().requires_grad_(True)
        loss = 0.5 * ((autograd.project(g, x) - y) ** 2).sum()
        loss.backward()
        return x.grad

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    vols = a.batch * a.steps
    print(json.dumps({"workload": f"{a.batch} x 256x256x64, 60 views, 256x192 imager, forward P + backward P^T",
                      "volumes_per_s": vols / secs, "updates_per_s": 2 * nnz * vols / secs,
                      "ms_per_batch": 1e3 * secs / a.steps, "nnz_per_P": nnz}))
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
