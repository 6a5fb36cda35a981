"""Serving benchmark: a seeded stream of reconstruction requests through the request
server, mixed precision and many requests at once, against the plain FP32 path that runs
one request at a time on the same GPU.

Workload (synthetic, seeded): 200 requests; volume uniformly one of 128x128x32 (2.0 mm
voxels, 128x48 imager at 3.0 mm), 256x256x64 (1.0 mm, 256x192 at 1.5 mm) and 512x512x70
(0.5x0.5x2.5 mm, 512x384 at 0.776 mm); views uniform in 20..120 over 360 degrees;
incident photons per ray log-uniform in [1e4, 1e5]; 3-level multigrid with 5/10/15
iterations (coarsest first), 3 CGLS updates each, mu = 5e-4. One seeded ellipsoid
phantom per volume shape; each request projects it with its own views (the library's
projector) and draws its own Poisson noise.

Two arms over the same request list:
* plain: FP32 CGLS vectors, one request on the device at a time, no graphs;
* served: BF16 CGLS vectors, up to 16 requests on the device, each captured as a CUDA graph,
  admitted under the L2 bound, smaller requests on higher-priority streams (also run
  without the priorities, Poisson arrivals only, to show what they trade);
* served by age: the same, with the oldest admitted request on the highest-priority
  streams and the others filling what it leaves idle, re-ranked after every A2 iteration.
Each arm runs twice: all requests submitted at once (throughput: requests per second of
makespan) and with Poisson arrivals at a fraction of the plain arm's measured capacity
(latency: p50 / p99 of completion minus submission). Every served volume is compared with
the plain arm's volume of the same request (relative L2). Prints one JSON line.

Usage: python -m paper_1008_2042_gb300.serve_bench [--requests 200] [--load 0.8]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

SHAPES = {
    "128x128x32": dict(nx=128, ny=128, nz=32, dx=2.0, dy=2.0, dz=2.0, nu=128, nv=48, du=3.0, dv=3.0),
    "256x256x64": dict(nx=256, ny=256, nz=64, dx=1.0, dy=1.0, dz=1.0, nu=256, nv=192, du=1.5, dv=1.5),
    "512x512x70": dict(nx=512, ny=512, nz=70, dx=0.5, dy=0.5, dz=2.5, nu=512, nv=384, du=0.776, dv=0.776),
}
LEVELS, ITERS, MU = 3, [5, 10, 15], 5e-4


def make_trace(n: int, seed: int = 1005):
    """The request list: shape, views, photons and an arrival offset on a unit-rate
    Poisson clock (exponential gaps of mean 1), all from one seeded generator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names = list(SHAPES)
    out, t = [], 0.0
    for i in range(n):
        t += rng.exponential(1.0)
        out.append({"shape": names[int(rng.integers(0, len(names)))],
                    "views": int(rng.integers(20, 121)),
                    "photons": float(10.0 ** rng.uniform(4.0, 5.0)),
                    "arrival": t, "seed": seed * 1000 + i})
    return out


def percentile(xs, q):
    """q-th percentile with linear interpolation between order statistics."""
    return float(np.percentile(np.asarray(xs, np.float64), q))


def geometry(shape: str, views: int):
    import synth
    return synth.Geometry(n_views=views, **SHAPES[shape])


def prepare_inputs(cb, trace, device="cuda"):
    """Pinned host projections for every request (not timed)."""
    import torch
    import synth
    phantoms = {}
    for name in SHAPES:
        g = geometry(name, 1)
        ell = synth.torso_ellipsoids(g, 1002) if name == "512x512x70" else synth.random_ellipsoids(g, 1001)
        phantoms[name] = torch.tensor(synth.voxelize(g, ell), dtype=torch.float32, device=device)
    ys = []
    for r in trace:
        geom = geometry(r["shape"], r["views"])
        with cb.Geometry(geom) as g:
            p = cb.project(g, phantoms[r["shape"]])
        gen = torch.Generator(device=device)
        gen.manual_seed(r["seed"])
        counts = torch.poisson(r["photons"] * torch.exp(-p.double()), generator=gen)
        y = -torch.log(torch.clamp(counts, min=1.0) / r["photons"])
        ys.append(y.float().cpu().pin_memory())
    torch.cuda.synchronize()
    return ys


def run_arm(cb, trace, ys, outs, *, storage, max_active, use_graphs, rate=None, priority="size"):
    """Submits every request (all at once when rate is None, else at its arrival time on
    a Poisson clock of `rate` requests per second) and waits for all. Returns makespan and
    per-request latencies (seconds, server clock)."""
    with cb.Server(max_active=max_active, use_graphs=use_graphs, priority=priority) as srv:
        t_start = time.perf_counter()
        ids = []
        for r, y, o in zip(trace, ys, outs):
            if rate is not None:
                delay = r["arrival"] / rate - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
            ids.append(srv.submit(geometry(r["shape"], r["views"]), y, MU, LEVELS, ITERS, o, storage=storage))
        infos = [srv.wait(i) for i in ids]
        stats = srv.stats()
    lat = [i["t_done"] - i["t_submit"] for i in infos]
    first = min(i["t_submit"] for i in infos)
    makespan = max(i["t_done"] for i in infos) - first
    by_shape = {s: [l for l, r in zip(lat, trace) if r["shape"] == s] for s in SHAPES}
    return {"makespan_s": makespan, "recon_per_s": len(infos) / makespan,
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99), "mean_s": float(np.mean(lat)),
            "p50_by_shape_s": {s: percentile(v, 50) for s, v in by_shape.items() if v},
            "max_active_seen": stats["max_active_seen"], "max_device_gb": stats["max_bytes_seen"] / 1e9,
            "bypassed": stats["bypassed"]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--load", type=float, default=0.8, help="arrival rate as a fraction of the plain arm's capacity")
    ap.add_argument("--max-active", type=int, default=16)
    args = ap.parse_args(argv)

    import torch
    from paper_1008_2042_gb300 import build
    build.build()
    import paper_1008_2042_gb300 as cb

    trace = make_trace(args.requests)
    ys = prepare_inputs(cb, trace)
    out_plain = [torch.empty(geometry(r["shape"], 1).vol_shape, dtype=torch.float32).pin_memory() for r in trace]
    out_served = [torch.empty_like(o).pin_memory() for o in out_plain]

    # warm-up: one request of each shape through both configurations
    warm = [next(r for r in trace if r["shape"] == s) for s in SHAPES]
    wy = [ys[trace.index(r)] for r in warm]
    wo = [torch.empty_like(out_plain[trace.index(r)]).pin_memory() for r in warm]
    run_arm(cb, warm, wy, wo, storage="f32", max_active=1, use_graphs=False)
    run_arm(cb, warm, wy, wo, storage="bf16", max_active=args.max_active, use_graphs=True)
    run_arm(cb, warm, wy, wo, storage="bf16", max_active=args.max_active, use_graphs=False, priority="age")

    plain_sat = run_arm(cb, trace, ys, out_plain, storage="f32", max_active=1, use_graphs=False)
    served_sat = run_arm(cb, trace, ys, out_served, storage="bf16", max_active=args.max_active, use_graphs=True)
    errs = [float(np.linalg.norm(s.numpy().astype(np.float64) - p.numpy()) / max(np.linalg.norm(p.numpy()), 1e-30))
            for s, p in zip(out_served, out_plain)]
    rate = args.load * plain_sat["recon_per_s"]
    plain_open = run_arm(cb, trace, ys, out_plain, storage="f32", max_active=1, use_graphs=False, rate=rate)
    served_open = run_arm(cb, trace, ys, out_served, storage="bf16", max_active=args.max_active, use_graphs=True,
                          rate=rate)
    served_open_flat = run_arm(cb, trace, ys, out_served, storage="bf16", max_active=args.max_active,
                               use_graphs=True, rate=rate, priority="none")
    out_age = [torch.empty_like(o).pin_memory() for o in out_plain]
    age_sat = run_arm(cb, trace, ys, out_age, storage="bf16", max_active=args.max_active, use_graphs=False,
                      priority="age")
    age_open = run_arm(cb, trace, ys, out_age, storage="bf16", max_active=args.max_active, use_graphs=False,
                       rate=rate, priority="age")
    errs_age = [float(np.linalg.norm(a.numpy().astype(np.float64) - s.numpy()) / max(np.linalg.norm(s.numpy()), 1e-30))
                for a, s in zip(out_age, out_served)]
    counts = {s: sum(r["shape"] == s for r in trace) for s in SHAPES}
    line = {
        "metric": "served reconstructions per second and latency",
        "requests": len(trace), "shapes": counts,
        "views_range": [min(r["views"] for r in trace), max(r["views"] for r in trace)],
        "levels": LEVELS, "iters_per_level": ITERS, "n_cgls": 3, "mu": MU,
        "plain_f32_one_at_a_time": {"all_at_once": plain_sat, "poisson": plain_open},
        "served_bf16_concurrent": {"all_at_once": served_sat, "poisson": served_open,
                                   "poisson_without_size_priority": served_open_flat},
        "served_bf16_age_priority": {"all_at_once": age_sat, "poisson": age_open,
                                     "rel_l2_vs_size_priority_max": max(errs_age)},
        "throughput_ratio_age_vs_plain": age_sat["recon_per_s"] / plain_sat["recon_per_s"],
        "poisson_rate_per_s": rate, "load_vs_plain_capacity": args.load,
        "throughput_ratio_served_vs_plain": served_sat["recon_per_s"] / plain_sat["recon_per_s"],
        "rel_l2_served_bf16_vs_plain_f32": {"max": max(errs), "median": percentile(errs, 50)},
        "data": "synthetic: seeded ellipsoid phantoms per shape, per-request views and Poisson noise",
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
