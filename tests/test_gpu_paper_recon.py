"""End-to-end parity of the reconstruction at the paper-scale workload.

Workload: 512x512x70 voxels of 0.5x0.5x2.5 mm, 512x384 imager at 0.776 mm, 40 views, the
seeded 30-ellipsoid torso (seed 1002) with Poisson noise at 5e4 photons per ray (seed
2002), mu = 5e-4, a 3-level multigrid (128x128x18 -> 256x256x35 -> 512x512x70, Section
2.2.3) around Algorithm A2 (Section 2.1) with 3 CGLS updates (Appendix 1). The data y
are the FP64 oracle's projection of the phantom with that noise, so the whole chain on
the device, from y to the volume, meets the oracle at the benchmark's size.

The iteration split is reduced to 2/2/2 (coarsest first) so that the oracle finishes in
about two minutes on 16 host cores; every launch shape of the benchmark's reconstruction
runs (each level's P, P^T, fused regularisation step and CGLS updates, and both
prolongations). Bar: relative L2 <= 1e-3 against the FP64 oracle, for FP32 storage and
for the BF16 and FP16 storage of the CGLS residual and projected direction.

The same test also checks the library's P of the phantom against the oracle's over the
whole stack (relative L2 <= 1e-4): the benchmark synthesises its y with the library's P
of this phantom and this noise seed, so its input is this test's input to within that
bar.
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MU = 5e-4
LEVELS = 3
ITERS = [2, 2, 2]
PHOTONS = 5e4


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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def paper_case():
    geom = synth.config_paper(40)
    f_true = synth.voxelize(geom, synth.torso_ellipsoids(geom, 1002))
    t0 = time.perf_counter()
    p_ideal = oracle.project(geom, f_true)
    y = synth.noisy_line_integrals(p_ideal, PHOTONS, 2002)
    ref = oracle.reconstruct(geom, y, MU, LEVELS, ITERS)
    print(f"\noracle: y and the {ITERS} reconstruction in {time.perf_counter() - t0:.0f} s "
          f"on {oracle.num_threads()} threads")
    return geom, f_true, p_ideal, y, ref


def test_paper_projection_of_phantom_matches_oracle(cb, paper_case):
    geom, f_true, p_ideal, _, _ = paper_case
    with cb.Geometry(geom) as g:
        p = cb.project(g, dev(f_true)).cpu().numpy()
    e = rel(p, p_ideal)
    print(f"\nP of the torso phantom, whole stack: relative L2 {e:.2e}")
    assert e <= 1e-4, e


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_paper_reconstruction_matches_oracle(cb, paper_case, storage):
    geom, f_true, _, y, ref = paper_case
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), MU, LEVELS, ITERS, storage=storage).cpu().numpy()
    e = rel(out, ref)
    print(f"\nreconstruction {geom.nx}x{geom.ny}x{geom.nz}, 40 views, {ITERS}, {storage}: "
          f"relative L2 against the FP64 oracle {e:.2e}")
    assert e <= 1e-3, (storage, e)
    assert out.min() >= 0.0
    # a reconstruction moving toward the phantom from the zero start
    assert rel(ref, f_true) < 1.0


def test_paper_reconstruction_80_views_matches_oracle(cb):
    """The workload's second view count: 80 views, one A2 iteration per level (every level's
    launch shapes run; the oracle needs about two minutes), FP32, relative L2 <= 1e-3."""
    geom = synth.config_paper(80)
    f_true = synth.voxelize(geom, synth.torso_ellipsoids(geom, 1002))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), PHOTONS, 2002)
    iters = [1, 1, 1]
    ref = oracle.reconstruct(geom, y, MU, LEVELS, iters)
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), MU, LEVELS, iters).cpu().numpy()
    e = rel(out, ref)
    print(f"\nreconstruction {geom.nx}x{geom.ny}x{geom.nz}, 80 views, {iters}, f32: relative L2 against the "
          f"FP64 oracle {e:.2e}")
    assert e <= 1e-3, e
