"""Parity of the CUDA operators (through the C ABI) with the FP64 oracle, element by
element on seeded inputs: P and P^T within relative L2 1e-4, W and the shrink/synthesis
within 1e-5, the multigrid transfers within 1e-6."""
import dataclasses

import numpy as np
import pytest

import oracle
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


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


GEOMS = {
    "small": synth.config_small(),
    # odd sizes (ragged tiles in every kernel), anisotropic voxels, offsets, rotated start
    "odd": synth.Geometry(nx=37, ny=29, nz=11, dx=1.7, dy=2.3, dz=1.1, nu=45, nv=23, du=1.9, dv=1.3,
                          u_off=2.1, v_off=-1.7, n_views=7,
                          angles=tuple(0.05 + 2 * np.pi * np.arange(7) / 7)),
    # steep cone: many z crossings per ray, rays leaving through top and bottom
    "cone": synth.Geometry(nx=24, ny=24, nz=12, dx=3.0, dy=3.0, dz=2.0, nu=40, nv=70, du=3.0, dv=6.0,
                           n_views=5, angles=tuple(0.3 + 1.1 * np.arange(5))),
    # one voxel
    "one": synth.Geometry(nx=1, ny=1, nz=1, dx=10.0, dy=10.0, dz=10.0, nu=8, nv=6, du=2.0, dv=2.0,
                          n_views=3, angles=(0.1, 1.0, 2.5)),
    # nv larger than one block of rows; imager wider than 128
    "tall": synth.Geometry(nx=40, ny=36, nz=20, dx=1.5, dy=1.5, dz=1.5, nu=150, nv=140, du=0.8, dv=0.7,
                           n_views=4, angles=(0.2, 0.9, 2.2, 4.0)),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_project_parity(cb, name):
    geom = GEOMS[name]
    f = synth.random_volume(geom, 101)
    with cb.Geometry(geom) as g:
        p = cb.project(g, dev(f)).cpu().numpy()
    ref = oracle.project(geom, f)
    assert rel(p, ref) <= 1e-4, rel(p, ref)


# traces of about 200 columns: several groups of every size, with a ragged last group
GROUP_GEOMS = {
    "odd": GEOMS["odd"],
    "cone": GEOMS["cone"],
    "long": synth.Geometry(nx=101, ny=90, nz=9, dx=1.0, dy=1.1, dz=2.0, nu=60, nv=26, du=1.9, dv=1.6,
                           u_off=0.7, v_off=-0.4, n_views=3, angles=(0.15, 1.9, 3.7)),
}


@pytest.fixture
def forced_group(cb):
    yield cb.set_project_group
    cb.set_project_group(0)


@pytest.mark.parametrize("sg", [16, 24, 32, 40, 48, 56, 64, 80, 96])
def test_project_parity_every_group_size(cb, forced_group, sg):
    """Every compiled column-group size of the projector against the oracle, and against
    the automatic choice to FP32 rounding (the groups only re-associate the sums)."""
    assert sg in cb.PROJECT_GROUP_SIZES
    for name, geom in GROUP_GEOMS.items():
        f = synth.random_volume(geom, 103)
        with cb.Geometry(geom) as g:
            forced_group(0)
            auto = cb.project(g, dev(f)).cpu().numpy()
            forced_group(sg)
            p = cb.project(g, dev(f)).cpu().numpy()
        ref = oracle.project(geom, f)
        assert rel(p, ref) <= 1e-4, (name, rel(p, ref))
        assert rel(p, auto) <= 2e-6, (name, rel(p, auto))


@pytest.mark.parametrize("sg", [16, 56, 96])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_reconstruct_parity_forced_group_sizes(cb, forced_group, sg, storage):
    """The CGLS projector modes (scaled direction, residual; FP32 and BF16 storage) under
    forced group sizes: a short reconstruction against the oracle."""
    geom = GROUP_GEOMS["long"]
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 104))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e5, 105)
    forced_group(sg)
    with cb.Geometry(geom) as g:
        x = cb.reconstruct(g, dev(y), 5e-4, 1, [6], storage=storage).cpu().numpy()
    ref = oracle.reconstruct(geom, y, 5e-4, 1, [6], storage=0 if storage == "f32" else storage)
    assert rel(x, ref) <= 1e-3, rel(x, ref)


def test_project_group_choice(cb, forced_group):
    """The automatic choice is a compiled size; forcing names a compiled size or 0; a forced
    size whose shared memory does not fit leaves that grid on the automatic choice."""
    geom = synth.config_paper(40)
    with cb.Geometry(geom) as g:
        auto = [cb.project_group(g, lv) for lv in range(3)]
        assert all(a in cb.PROJECT_GROUP_SIZES for a in auto)
        forced_group(24)
        assert cb.project_group(g, 0) == 24
        with pytest.raises(cb.CbctError) as e:
            forced_group(33)
        assert e.value.status == 1
        assert cb.project_group(g, 0) == 24  # an invalid call changes nothing
        forced_group(0)
        assert [cb.project_group(g, lv) for lv in range(3)] == auto
    big = LARGEST_NZ
    with cb.Geometry(big) as g:
        forced_group(0)
        a = cb.project_group(g, 0)
        forced_group(96)  # 96 columns of 1024-voxel lines exceed the shared memory
        assert cb.project_group(g, 0) == a


LARGEST_NZ = synth.Geometry(nx=256, ny=256, nz=1024, dx=1.0, dy=1.0, dz=0.2, nu=64, nv=40, du=1.5, dv=1.5,
                            n_views=2, angles=(0.1, 1.7))


@pytest.mark.parametrize("name", list(GEOMS))
def test_backproject_parity(cb, name):
    geom = GEOMS[name]
    y = synth.random_projections(geom, 102)
    with cb.Geometry(geom) as g:
        b = cb.backproject(g, dev(y)).cpu().numpy()
    ref = oracle.backproject(geom, y)
    assert rel(b, ref) <= 1e-4, rel(b, ref)


def test_project_phantom_parity(cb):
    geom = synth.config_small()
    f = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    with cb.Geometry(geom) as g:
        p = cb.project(g, dev(f)).cpu().numpy()
    ref = oracle.project(geom, f)
    assert rel(p, ref) <= 1e-5, rel(p, ref)


@pytest.mark.parametrize("name", ["small", "odd", "cone"])
def test_gpu_adjoint_identity(cb, name):
    geom = GEOMS[name]
    f = synth.random_volume(geom, 103)
    y = synth.random_projections(geom, 104)
    with cb.Geometry(geom) as g:
        pf = cb.project(g, dev(f)).cpu().numpy().astype(np.float64)
        bty = cb.backproject(g, dev(y)).cpu().numpy().astype(np.float64)
    f32 = f.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    lhs, rhs = np.vdot(pf, y32), np.vdot(f32, bty)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


def test_count_nnz_matches_oracle(cb):
    for geom in (GEOMS["small"], GEOMS["odd"], GEOMS["cone"]):
        with cb.Geometry(geom) as g:
            n_gpu = cb.count_nnz(g)
        n_ref = oracle.count_nnz(geom)
        assert abs(n_gpu - n_ref) <= 5e-3 * n_ref, (n_gpu, n_ref)


def test_count_nnz_levels(cb):
    geom = synth.config_small()
    with cb.Geometry(geom) as g:
        for lev in (1, 2):
            n_gpu = cb.count_nnz(g, lev)
            n_ref = oracle.count_nnz(geom.level(lev))
            assert abs(n_gpu - n_ref) <= 5e-3 * n_ref, (lev, n_gpu, n_ref)


TF_SHAPES = [(16, 64, 64), (5, 6, 7), (1, 4, 3), (2, 3, 5), (9, 17, 33), (3, 70, 40), (4, 19, 61)]


@pytest.mark.parametrize("shape", TF_SHAPES)
def test_tf_analyze_parity(cb, shape):
    f = np.random.default_rng(5).standard_normal(shape)
    a = cb.tf_analyze(dev(f)).cpu().numpy()
    ref = oracle.tf_analyze(f)
    assert rel(a, ref) <= 1e-5, rel(a, ref)
    scale = np.linalg.norm(ref)
    for i in range(27):  # every channel, relative to the whole transform (a channel can be 0)
        assert np.linalg.norm(a[i] - ref[i]) <= 1e-5 * max(np.linalg.norm(ref[i]), 1e-3 * scale), i


@pytest.mark.parametrize("shape", TF_SHAPES)
@pytest.mark.parametrize("positive", [False, True])
def test_tf_synthesize_shrink_parity(cb, shape, positive):
    rng = np.random.default_rng(6)
    alpha = rng.standard_normal((27,) + shape) * 0.01
    # threshold near the median high-pass norm: about half the voxels are zeroed
    mu = float(np.median(np.sqrt((alpha[1:] ** 2).sum(0))))
    out = cb.tf_synthesize_shrink(dev(alpha), mu, positive).cpu().numpy()
    ref = oracle.tf_synthesize_shrink(alpha, mu, positive)
    assert rel(out, ref) <= 1e-5, rel(out, ref)


# the fused step's tile width along the contiguous (last) axis is chosen per launch from
# 24, 32 and 36: these cover each width (70 = 3 x 24 - 2, 35 = 36 - 1, 64 = 2 x 32) and a
# long marching axis split into several blocks
FUSED_SHAPES = TF_SHAPES + [(6, 9, 70), (5, 4, 35), (300, 3, 5)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("positive", [False, True])
def test_tf_shrink_fused_parity(cb, shape, positive):
    """The fused regularisation step H(W^T T_mu W f) against the oracle's three steps."""
    f = np.random.default_rng(10).standard_normal(shape)
    mu = float(np.median(np.sqrt((oracle.tf_analyze(f)[1:] ** 2).sum(0))))
    out = cb.tf_shrink(dev(f), mu, positive).cpu().numpy()
    alpha = oracle.tf_analyze(f)
    ref = oracle.tf_synthesize_shrink(alpha, mu, positive)
    # H is a projection (1-Lipschitz): measure against the output's size before H, which
    # stays meaningful when H zeroes most voxels of a tiny random volume
    scale = np.linalg.norm(oracle.tf_synthesize_shrink(alpha, mu, False))
    assert np.linalg.norm(out - ref) <= 1e-5 * scale, np.linalg.norm(out - ref) / scale


@pytest.mark.parametrize("layout", ["x_fastest", "z_fastest"])
def test_tf_shrink_on_nonnegative_phantom(cb, layout):
    """On a reconstruction-like volume (the seeded ellipsoid phantom, mu = 5e-4, H on) H
    zeroes few voxels, so the plain relative-L2 bar of the frame transforms applies to the
    fused step and to the public shrink + synthesis alike."""
    geom = synth.config_small()
    f = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    if layout == "z_fastest":
        f = np.ascontiguousarray(f.transpose(1, 2, 0))
    mu = 5e-4
    alpha = oracle.tf_analyze(f)
    ref = oracle.tf_synthesize_shrink(alpha, mu, True)
    out = cb.tf_shrink(dev(f), mu, True).cpu().numpy()
    assert rel(out, ref) <= 1e-5, rel(out, ref)
    out2 = cb.tf_synthesize_shrink(dev(alpha), mu, True).cpu().numpy()
    assert rel(out2, ref) <= 1e-5, rel(out2, ref)


def test_tf_round_trip_identity(cb):
    f = np.random.default_rng(7).standard_normal((16, 64, 64))
    ft = dev(f)
    back = cb.tf_synthesize_shrink(cb.tf_analyze(ft), 0.0, False).cpu().numpy()
    assert rel(back, f) <= 1e-6


def test_prolong_parity(cb):
    fc = np.random.default_rng(8).uniform(0, 1, (9, 16, 12))
    cs, fs, fshape = (2.0, 2.0, 5.0), (1.0, 1.0, 2.5), (18, 32, 24)
    out = cb.prolong(dev(fc), cs, fshape, fs).cpu().numpy()
    ref = oracle.prolong(fc, cs, fshape, fs)
    assert rel(out, ref) <= 1e-6, rel(out, ref)
    # odd fine sizes (non-nested grids), as on the paper's 70 -> 35 -> 18 slices
    out = cb.prolong(dev(fc), cs, (17, 31, 23), fs).cpu().numpy()
    ref = oracle.prolong(fc, cs, (17, 31, 23), fs)
    assert rel(out, ref) <= 1e-6, rel(out, ref)


def test_restrict_parity(cb):
    ff = np.random.default_rng(9).uniform(0, 1, (17, 31, 24))
    out = cb.restrict(dev(ff), (1.0, 1.0, 2.0), (9, 16, 12), (2.0, 2.0, 4.0)).cpu().numpy()
    ref = oracle.restrict(ff, (1.0, 1.0, 2.0), (9, 16, 12), (2.0, 2.0, 4.0))
    assert rel(out, ref) <= 1e-6, rel(out, ref)


@pytest.mark.parametrize("name", ["small", "odd", "tall"])
def test_backproject_eq3_parity(cb, name):
    """The paper's own backprojector, Eq. (3), against the oracle's restatement."""
    geom = GEOMS[name]
    y = synth.random_projections(geom, 105)
    with cb.Geometry(geom) as g:
        b = cb.backproject_eq3(g, dev(y)).cpu().numpy()
    ref = oracle.backproject_eq3(geom, y)
    assert rel(b, ref) <= 1e-4, rel(b, ref)


def test_batched_operators_equal_single_calls(cb):
    geom = GEOMS["odd"]
    fs = np.stack([synth.random_volume(geom, 200 + b) for b in range(3)])
    ys = np.stack([synth.random_projections(geom, 300 + b) for b in range(3)])
    with cb.Geometry(geom) as g:
        pb = cb.project_batch(g, dev(fs)).cpu().numpy()
        bb = cb.backproject_batch(g, dev(ys)).cpu().numpy()
        for b in range(3):
            assert np.array_equal(pb[b], cb.project(g, dev(fs[b])).cpu().numpy())
            assert np.array_equal(bb[b], cb.backproject(g, dev(ys[b])).cpu().numpy())
