"""Reduced-precision storage: projections and frame coefficients held as bfloat16 or
binary16 with FP32 arithmetic and FP64 inner products, through the typed C-ABI entry
points and the storage option of the reconstruction.

Bars:
* typed P and W store exactly the FP32 result rounded once to nearest-even, so they
  equal the FP32 call cast to the type, and lie within one rounding of the FP64 oracle
  (u |x| with unit roundoff u = 2^-8 for bfloat16, 2^-11 for binary16, or half the
  subnormal spacing below the smallest normal), plus the FP32 bar;
* typed P^T and synthesis widen exactly, so they equal the FP32 calls on the widened
  input and match the oracle on the same (rounded) input within the FP32 bars;
* the reconstruction with 16-bit CGLS vectors matches the oracle that rounds at the same
  points within relative L2 1e-3, and the plain FP64 oracle within 1e-3 as well. The
  error against the plain FP64 oracle is printed for every storage type.

Workload of the reconstruction: 64x64x16 voxels of 1 mm, 6 seeded ellipsoids, 80 views of
a 128x32 imager at 0.8 mm, Poisson noise at 1e4 photons per ray, one level, 20 iterations.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}
# half the spacing of the subnormals: the rounding error bound below the smallest normal
TINY = {"bf16": 2.0 ** -134, "f16": 2.0 ** -25}
TORCH = {"bf16": torch.bfloat16, "f16": torch.float16}


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


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32).to(dtype).to("cuda")


def widened(x, st):
    """x rounded to the storage type on the CPU (torch's cast), as float64."""
    return torch.tensor(np.asarray(x, np.float32)).to(TORCH[st]).to(torch.float64).numpy()


GEOMS = [
    synth.config_small(),
    synth.Geometry(nx=37, ny=29, nz=11, dx=1.7, dy=2.3, dz=1.1, nu=45, nv=23, du=1.9, dv=1.3,
                   u_off=2.1, v_off=-1.7, n_views=7, angles=tuple(0.05 + 2 * np.pi * np.arange(7) / 7)),
]


@pytest.mark.parametrize("st", ["bf16", "f16"])
@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_project_typed_output_is_one_rounding(cb, st, gi):
    geom = GEOMS[gi]
    f = synth.random_volume(geom, 501 + gi)
    with cb.Geometry(geom) as g:
        fd = dev(f)
        g32 = cb.project(g, fd)
        g16 = cb.project(g, fd, dtype=TORCH[st])
        assert g16.dtype == TORCH[st]
        assert torch.equal(g16, g32.to(TORCH[st]))  # the FP32 result, rounded once (RNE)
    ref = oracle.project(geom, f)
    got = g16.to(torch.float64).cpu().numpy()
    bound = U[st] * np.abs(ref) + TINY[st] + 1e-5 * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)


@pytest.mark.parametrize("st", ["bf16", "f16"])
@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_backproject_typed_input(cb, st, gi):
    geom = GEOMS[gi]
    y = widened(synth.random_projections(geom, 601 + gi), st)
    with cb.Geometry(geom) as g:
        y16 = dev(y, TORCH[st])
        b16 = cb.backproject(g, y16)
        b32 = cb.backproject(g, y16.float())
        assert torch.equal(b16, b32)  # widening is exact
    ref = oracle.backproject(geom, y)
    assert rel(b16.cpu().numpy(), ref) <= 1e-4, rel(b16.cpu().numpy(), ref)


TF_SHAPES = [(16, 64, 64), (11, 29, 37)]


@pytest.mark.parametrize("st", ["bf16", "f16"])
@pytest.mark.parametrize("shape", TF_SHAPES)
def test_tf_analyze_typed_output_is_one_rounding(cb, st, shape):
    f = np.random.default_rng(7).standard_normal(shape) * 0.02
    fd = dev(f)
    a32 = cb.tf_analyze(fd)
    a16 = cb.tf_analyze(fd, dtype=TORCH[st])
    assert a16.dtype == TORCH[st]
    assert torch.equal(a16, a32.to(TORCH[st]))
    ref = oracle.tf_analyze(f)
    got = a16.to(torch.float64).cpu().numpy()
    bound = U[st] * np.abs(ref) + TINY[st] + 1e-6 * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)


@pytest.mark.parametrize("st", ["bf16", "f16"])
@pytest.mark.parametrize("shape", TF_SHAPES)
@pytest.mark.parametrize("positive", [False, True])
def test_tf_synthesize_shrink_typed_input(cb, st, shape, positive):
    rng = np.random.default_rng(8)
    alpha = widened(rng.standard_normal((27,) + shape) * 0.01, st)
    mu = float(np.median(np.sqrt((alpha[1:] ** 2).sum(0))))
    a16 = dev(alpha, TORCH[st])
    out16 = cb.tf_synthesize_shrink(a16, mu, positive)
    out32 = cb.tf_synthesize_shrink(a16.float(), mu, positive)
    assert torch.equal(out16, out32)
    ref = oracle.tf_synthesize_shrink(alpha, mu, positive)
    scale = np.linalg.norm(oracle.tf_synthesize_shrink(alpha, mu, False))
    assert np.linalg.norm(out16.cpu().numpy() - ref) <= 1e-5 * scale


@pytest.fixture(scope="module")
def low_dose_case():
    geom = synth.config_small(80)
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e4, 1003)
    mu, iters = 5e-4, [20]
    refs = {st: oracle.reconstruct(geom, y, mu, 1, iters, storage=st) for st in ("f64", "bf16", "f16")}
    return geom, f_true, y, mu, iters, refs


@pytest.mark.parametrize("st", ["f32", "bf16", "f16"])
def test_reconstruct_storage_parity(cb, low_dose_case, st):
    geom, f_true, y, mu, iters, refs = low_dose_case
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), mu, 1, iters, storage=st).cpu().numpy()
    same_rounding = refs["f64" if st == "f32" else st]
    e_same, e_fp64 = rel(out, same_rounding), rel(out, refs["f64"])
    print(f"\nstorage {st}: rel-L2 vs oracle with the same rounding {e_same:.3e}, "
          f"vs plain FP64 oracle {e_fp64:.3e}, oracle's own 16-bit effect "
          f"{rel(same_rounding, refs['f64']):.3e}, vs phantom {rel(out, f_true):.3e}")
    assert e_same <= 1e-3, e_same
    assert e_fp64 <= 1e-3, e_fp64
    assert out.min() >= 0.0


def test_reconstruct_multigrid_f16_storage(cb):
    """Three levels with binary16 CGLS vectors: the scaled q keeps every level finite and
    the result tracks the FP64 oracle."""
    geom = synth.config_small()
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e5, 2001)
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), 5e-4, 3, [3, 4, 5], storage="f16").cpu().numpy()
    ref = oracle.reconstruct(geom, y, 5e-4, 3, [3, 4, 5], storage="f16")
    assert np.isfinite(out).all()
    assert rel(out, ref) <= 1e-3, rel(out, ref)


def test_unknown_storage_is_rejected(cb):
    import ctypes
    geom = synth.config_small()
    lib = cb.load_library()
    with cb.Geometry(geom) as g:
        y = torch.zeros(geom.proj_shape, device="cuda")
        f = torch.zeros(geom.vol_shape, device="cuda")
        it = (ctypes.c_int * 1)(1)
        opts = cb.ReconOpts(3, 1, 1, 7)
        st = lib.cbct_reconstruct_ex(ctypes.c_void_p(y.data_ptr()), g.handle, 1e-3, 0.0, 1, it, ctypes.byref(opts),
                                     None, 0, ctypes.c_void_p(f.data_ptr()), None)
        assert st == 1
        assert lib.cbct_project_ex(g.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(y.data_ptr()), 9,
                                   None) == 1
