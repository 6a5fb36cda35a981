"""Host side of the serving benchmark: the seeded request list follows the stated
distributions and the latency percentiles are order statistics."""
import math

import numpy as np

from paper_1008_2042_gb300 import serve_bench as sb


def test_trace_is_seeded_and_follows_the_workload():
    a = sb.make_trace(2000)
    assert a == sb.make_trace(2000)
    assert a != sb.make_trace(2000, seed=7)
    shapes = [r["shape"] for r in a]
    for s in sb.SHAPES:
        assert abs(shapes.count(s) / len(a) - 1 / 3) < 0.05
    views = np.array([r["views"] for r in a])
    assert views.min() >= 20 and views.max() <= 120 and abs(views.mean() - 70) < 3
    ph = np.log10([r["photons"] for r in a])
    assert ph.min() >= 4 and ph.max() <= 5 and abs(ph.mean() - 4.5) < 0.05
    t = np.array([r["arrival"] for r in a])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1.0) < 0.08 and abs(gaps.std() - 1.0) < 0.1  # exponential, rate 1


def test_percentiles_are_order_statistics():
    xs = list(range(1, 101))
    assert sb.percentile(xs, 50) == 50.5
    assert math.isclose(sb.percentile(xs, 99), 99.01)
    assert sb.percentile([3.0], 99) == 3.0


def test_shapes_are_valid_geometries():
    for name in sb.SHAPES:
        g = sb.geometry(name, 20)
        half_diag = 0.5 * math.hypot(g.nx * g.dx, g.ny * g.dy)
        assert half_diag < g.sad and half_diag < g.sdd - g.sad
        # the imager covers the magnified volume transversally
        assert g.nu * g.du >= g.sdd / g.sad * 2 * half_diag * 0.7
