"""Runs one operator of the library on a fixed workload a few times — the target for
Nsight Compute captures and quick timings of a single kernel.

    python -m paper_1008_2042_gb300.profile_case --op project --shape paper --repeat 3

--op: project | backproject | tf_analyze | tf_synth | tf_shrink (fused W, T_mu, W^T, H) | tf_shrink_z (the
     same on the z-fastest layout the reconstruction iterates in) | reconstruct
--shape: paper (512x512x70, 512x384 imager, 40 views) | small (64x64x16, 128x32, 40 views)
         | iso256 (256x256x64 at 1 mm, 256x192 imager at 1.5 mm, 60 views)
--level: multigrid level of the operator's grid (0 = finest; project/backproject only)
Prints the mean device time per call (CUDA events) after one untimed call.
"""
from __future__ import annotations

import argparse
import dataclasses
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

import paper_1008_2042_gb300 as cb  # noqa: E402
from paper_1008_2042_gb300 import build as cuda_build  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="project",
                    choices=("project", "backproject", "tf_analyze", "tf_synth", "tf_shrink", "tf_shrink_z", "reconstruct"))
    ap.add_argument("--shape", default="paper", choices=("paper", "small", "iso256"))
    ap.add_argument("--views", type=int, default=40)
    ap.add_argument("--level", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=3)
    a = ap.parse_args(argv)

    cuda_build.build()
    if a.shape == "paper":
        geom = synth.config_paper(a.views)
    elif a.shape == "iso256":
        geom = synth.Geometry(nx=256, ny=256, nz=64, dx=1.0, dy=1.0, dz=1.0, nu=256, nv=192, du=1.5, dv=1.5,
                              n_views=a.views if a.views != 40 else 60)
    else:
        geom = synth.config_small(a.views)
    geom = geom.level(a.level) if a.level else geom
    dev = torch.device("cuda")
    g = cb.Geometry(geom)
    rng = torch.Generator(device=dev).manual_seed(1)
    f = torch.rand(geom.vol_shape, device=dev, generator=rng)
    y = torch.rand(geom.proj_shape, device=dev, generator=rng)
    alpha = None
    f_out = torch.empty_like(f)
    if a.op == "tf_shrink_z":  # (ny, nx, nz): z fastest, as inside the iteration
        f = torch.rand((geom.ny, geom.nx, geom.nz), device=dev, generator=rng)
        f_out = torch.empty_like(f)
    if a.op == "tf_synth":
        alpha = cb.tf_analyze(f)

    def run():
        if a.op == "project":
            cb.project(g, f)
        elif a.op == "backproject":
            cb.backproject(g, y)
        elif a.op == "tf_analyze":
            cb.tf_analyze(f)
        elif a.op == "tf_synth":
            cb.tf_synthesize_shrink(alpha, 1e-3, True)
        elif a.op in ("tf_shrink", "tf_shrink_z"):
            cb.tf_shrink(f, 1e-3, True, out=f_out)
        else:
            cb.reconstruct(g, y, 5e-4, 1, [1])

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.repeat):
        run()
    e1.record()
    torch.cuda.synchronize()
    print(f"{a.op} {a.shape} level {a.level}: {e0.elapsed_time(e1) / a.repeat:.3f} ms per call")
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
