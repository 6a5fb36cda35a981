"""cbct_project_static — the projector entry point that allocates no device memory — gives
the same projections as cbct_project, bit for bit, on consecutive calls that reuse its
fixed scratch, and leaves the device's free memory unchanged.

It serves callers that cannot allocate device memory while running, such as a service
whose device memory is fixed at start-up or a latency-critical loop that cannot afford
the synchronisation an allocation may cause. This file is collected last so that a
failure here leaves every other test run.
"""
import gc

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1008_2042_gb300 import build
    build.build()
    import paper_1008_2042_gb300 as m
    m.load_library()
    return m


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


GEOMS = [
    synth.config_small(),
    synth.Geometry(nx=37, ny=29, nz=11, dx=1.7, dy=2.3, dz=1.1, nu=45, nv=23, du=1.9, dv=1.3,
                   u_off=2.1, v_off=-1.7, n_views=7, angles=tuple(0.05 + 2 * np.pi * np.arange(7) / 7)),
]


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_project_static_matches_project_on_repeated_calls(cb, gi):
    """Both entry points run the same kernels on the same input: the results are equal."""
    geom = GEOMS[gi]
    f = torch.tensor(synth.random_volume(geom, 404 + gi), dtype=torch.float32, device="cuda")
    with cb.Geometry(geom) as g:
        ref = cb.project(g, f).cpu().numpy()
        for _ in range(2):
            out = torch.full(geom.proj_shape, float("nan"), dtype=torch.float32, device="cuda")
            cb.project_static(g, f, out)
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.array_equal(got, ref), rel(got, ref)


def test_project_static_leaves_device_memory_unchanged(cb):
    """After the first call on the device (which looks up the scratch's address), further
    calls change neither the free device memory nor torch's allocator."""
    geom = GEOMS[1]
    f = torch.tensor(synth.random_volume(geom, 410), dtype=torch.float32, device="cuda")
    out = torch.empty(geom.proj_shape, dtype=torch.float32, device="cuda")
    with cb.Geometry(geom) as g:
        cb.project_static(g, f, out)
        torch.cuda.synchronize()
        # tensors left unreachable by earlier tests are freed by Python's collector, which
        # would otherwise run at any moment and move torch's counters: collect them now and
        # keep the collector off while the calls are measured
        gc.collect()
        gc.disable()
        try:
            free0, _ = torch.cuda.mem_get_info()
            alloc0 = torch.cuda.memory_allocated()
            for _ in range(3):
                cb.project_static(g, f, out)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            alloc1 = torch.cuda.memory_allocated()
        finally:
            gc.enable()
        assert alloc1 == alloc0, (alloc0, alloc1)
        assert free1 == free0, (free0, free1)


def test_project_static_rejects_a_volume_beyond_its_scratch(cb):
    geom = synth.Geometry(nx=256, ny=256, nz=65, dx=1.0, dy=1.0, dz=1.0, nu=64, nv=32, du=2.0, dv=2.0,
                          n_views=2)
    assert geom.nx * geom.ny * geom.nz > 4194304
    with cb.Geometry(geom) as g:
        f = torch.zeros(geom.vol_shape, dtype=torch.float32, device="cuda")
        out = torch.zeros(geom.proj_shape, dtype=torch.float32, device="cuda")
        with pytest.raises(cb.CbctError) as e:
            cb.project_static(g, f, out)
        assert e.value.status == 1
        assert "fixed scratch" in str(e.value)
