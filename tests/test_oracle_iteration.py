"""Pins of the oracle's CGLS (Appendix 1), Algorithm A2 (Section 2.1) and the multigrid
transfer operators (Section 2.2.3) against exact least-squares solutions, invariants and
special cases."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_geom(n_views=6):
    # 4x4x2 voxels seen by 6 views of 8x6 pixels: 288 rays, 32 unknowns, full column rank
    return synth.Geometry(nx=4, ny=4, nz=2, dx=8.0, dy=8.0, dz=8.0, nu=8, nv=6, du=6.0, dv=6.0,
                          n_views=n_views, angles=tuple(0.2 + 2 * np.pi * np.arange(n_views) / n_views))


def _small_geom():
    return synth.Geometry(nx=8, ny=8, nz=8, dx=4.0, dy=4.0, dz=4.0, nu=12, nv=10, du=4.0, dv=4.0,
                          n_views=5, angles=tuple(0.3 + 2 * np.pi * np.arange(5) / 5))


@pytest.mark.parametrize("n_iter", [1, 2, 3, 5])
def test_cgls_equals_krylov_least_squares(n_iter):
    geom = _small_geom()
    A = dense.system_matrix(geom)
    rng = np.random.default_rng(n_iter)
    y = A @ rng.uniform(0, 1, A.shape[1]) + 0.01 * rng.standard_normal(A.shape[0])
    x0 = rng.uniform(0, 0.5, A.shape[1])
    x = oracle.cgls(geom, y.reshape(geom.proj_shape), x0.reshape(geom.vol_shape), n_iter).ravel()
    ref = dense.krylov_lsq(A, y, x0, n_iter)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_cgls_residual_is_non_increasing():
    geom = synth.config_small(n_views=10)
    f = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = oracle.project(geom, f)
    _, res = oracle.cgls(geom, y, np.zeros(geom.vol_shape), 6, return_resid=True)
    assert np.all(np.diff(res) <= 1e-12 * res[0]), res
    assert res[-1] < 0.2 * res[0]


def test_cgls_reaches_least_squares_solution_on_full_rank_system():
    geom = _tiny_geom()
    A = dense.system_matrix(geom)
    assert np.linalg.matrix_rank(A) == A.shape[1]
    rng = np.random.default_rng(7)
    y = rng.uniform(0, 10, A.shape[0])
    x = oracle.cgls(geom, y.reshape(geom.proj_shape), np.zeros(geom.vol_shape), 3 * A.shape[1]).ravel()
    ref, *_ = np.linalg.lstsq(A, y, rcond=None)
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)


def test_a2_without_regularisation_reaches_least_squares():
    """mu = 0 makes D^T T_mu D the identity (tight frame); with H off and enough CGLS
    steps every outer iteration lands on the least-squares solution, momentum or not."""
    geom = _tiny_geom()
    A = dense.system_matrix(geom)
    y = np.random.default_rng(8).uniform(0, 10, A.shape[0])
    ref, *_ = np.linalg.lstsq(A, y, rcond=None)
    for momentum in (False, True):
        f = oracle.a2(geom, y.reshape(geom.proj_shape), 0.0, 3, n_cgls=3 * A.shape[1],
                      positivity=False, momentum=momentum).ravel()
        assert np.linalg.norm(f - ref) <= 1e-7 * np.linalg.norm(ref)


def test_a2_fixed_point_at_consistent_constant_volume():
    """Consistent data of a positive constant volume: CGLS sees a zero residual, the
    constant has no high-pass coefficients and is positive, so A2 never moves."""
    geom = _small_geom()
    f_true = np.full(geom.vol_shape, 0.02)
    y = oracle.project(geom, f_true)
    f = oracle.a2(geom, y, 5e-4, 4, n_cgls=3, f0=f_true)
    assert np.abs(f - f_true).max() <= 1e-15


def test_a2_momentum_accelerates_a1():
    """Section 2.1: A2 is A1 plus momentum and converges faster. With mu = 0, H off and
    one CGLS step per outer iteration, A1 is steepest descent with exact line search."""
    geom = synth.config_small(n_views=8)
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = oracle.project(geom, f_true)
    res = {}
    for momentum in (False, True):
        f = oracle.a2(geom, y, 0.0, 25, n_cgls=1, positivity=False, momentum=momentum)
        res[momentum] = np.linalg.norm(oracle.project(geom, f) - y)
    assert res[True] < 0.7 * res[False], res


def _golden_momentum():
    """(t^(k), c_k) for k = 0..7 from the golden file (hand-evaluated recurrence)."""
    rows = []
    with open(os.path.join(GOLDEN, "a2_momentum.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, t, c = line.split()
                rows.append((int(k), float(t), float(c)))
    assert [r[0] for r in rows] == list(range(len(rows)))
    return np.array([r[1] for r in rows]), np.array([r[2] for r in rows])


def test_a2_momentum_schedule_matches_hand_evaluated_recurrence():
    """Section 2.1, Algorithm A2: the coefficient each iteration of the C iteration
    applies equals (t^(k-1) - 1) / t^(k) of the paper's recurrence, evaluated by hand."""
    _, c_ref = _golden_momentum()
    geom = _small_geom()
    y = oracle.project(geom, np.full(geom.vol_shape, 0.01))
    _, c = oracle.a2(geom, y, 5e-4, len(c_ref), n_cgls=1, return_coefficients=True)
    assert np.abs(c - c_ref).max() <= 1e-15, (c, c_ref)
    _, c1 = oracle.a2(geom, y, 5e-4, 4, n_cgls=1, momentum=False, return_coefficients=True)
    assert not c1.any()  # A1: no momentum


def test_a2_applies_the_momentum_point_as_stated():
    """With the data step removed (no CGLS update) and H off, A2 is the accelerated
    shrinkage iteration f^(k+1) = W^T T_mu W (f^(k) + c_k (f^(k) - f^(k-1))), f^(-1) =
    f^(0); built here from the pinned frame operators and the golden c_k, so a shifted
    coefficient index or a sign error in the momentum point fails."""
    _, c_ref = _golden_momentum()
    geom = _small_geom()
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.0, 0.04, geom.vol_shape)
    mu = 4e-3
    y = np.zeros(geom.proj_shape)
    n = 6
    f, c = oracle.a2(geom, y, mu, n, n_cgls=0, positivity=False, f0=f0, return_coefficients=True)
    prev, cur = f0.copy(), f0.copy()
    for k in range(n):
        v = cur + c_ref[k] * (cur - prev)
        prev, cur = cur, oracle.tf_synthesize(oracle.tf_shrink(oracle.tf_analyze(v), mu))
    assert np.abs(f - cur).max() <= 1e-13 * np.abs(cur).max()
    # the momentum terms matter here: without them the result differs
    f_a1 = oracle.a2(geom, y, mu, n, n_cgls=0, positivity=False, f0=f0, momentum=False)
    assert np.abs(f_a1 - cur).max() > 1e-6 * np.abs(cur).max()


@pytest.mark.parametrize("momentum,positivity", [(True, True), (False, True), (True, False)])
def test_a2_equals_dense_restatement(momentum, positivity):
    """The C iteration against an independent dense-matrix restatement (slab-clipped
    system matrix, per-axis circulant frame filters, dense CGLS)."""
    geom = _small_geom()
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 21, n=4, vmax=0.04))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e4, 22)
    A = dense.system_matrix(geom)
    for mu in (0.0, 2e-3):
        f = oracle.a2(geom, y, mu, 5, n_cgls=2, positivity=positivity, momentum=momentum)
        ref = dense.a2_dense(A, y, geom.vol_shape, mu, 5, 2, positivity, momentum)
        assert np.linalg.norm(f - ref) <= 1e-12 * np.linalg.norm(ref), (mu, np.linalg.norm(f - ref))


@pytest.mark.parametrize("shape,levels,iters", [((8, 8, 8), 3, [2, 3, 2]), ((10, 16, 12), 2, [3, 2])])
def test_multigrid_equals_dense_restatement(shape, levels, iters):
    """The whole cascade of Section 2.2.3 (coarsest first, prolongation between levels,
    odd coarse sizes included) against the dense restatement."""
    nz, ny, nx = shape
    geom = synth.Geometry(nx=nx, ny=ny, nz=nz, dx=4.0, dy=4.0, dz=4.0, nu=16, nv=12, du=4.0, dv=4.0,
                          n_views=6, angles=tuple(0.3 + 2 * np.pi * np.arange(6) / 6))
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 31, n=4, vmax=0.04))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e4, 32)
    out = oracle.reconstruct(geom, y, 1e-3, levels, iters)
    ref = dense.reconstruct_dense(geom, y, 1e-3, levels, iters)
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref), np.linalg.norm(out - ref)


def test_a2_shrinkage_lowers_frame_sparsity_measure():
    """With mu > 0 the result's high-pass energy is below the unregularised one."""
    geom = synth.config_small(n_views=10)
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e4, 3)
    hp = {}
    for mu in (0.0, 2e-3):
        f = oracle.a2(geom, y, mu, 4, n_cgls=3)
        a = oracle.tf_analyze(f)
        hp[mu] = np.sqrt((a[1:] ** 2).sum(0)).sum()
    assert hp[2e-3] < 0.8 * hp[0.0], hp


def test_prolong_is_exact_on_linear_functions_inside_the_hull():
    cshape, cs = (5, 6, 7), (2.0, 3.0, 4.0)
    fshape, fs = (10, 12, 14), (1.0, 1.5, 2.0)
    cz = -cshape[0] * cs[2] / 2 + (np.arange(cshape[0]) + 0.5) * cs[2]
    cy = -cshape[1] * cs[1] / 2 + (np.arange(cshape[1]) + 0.5) * cs[1]
    cx = -cshape[2] * cs[0] / 2 + (np.arange(cshape[2]) + 0.5) * cs[0]
    lin = lambda z, y, x: 0.3 + 0.1 * x - 0.2 * y + 0.05 * z
    fc = lin(cz[:, None, None], cy[None, :, None], cx[None, None, :])
    ff = oracle.prolong(fc, cs, fshape, fs)
    fz = -fshape[0] * fs[2] / 2 + (np.arange(fshape[0]) + 0.5) * fs[2]
    fy = -fshape[1] * fs[1] / 2 + (np.arange(fshape[1]) + 0.5) * fs[1]
    fx = -fshape[2] * fs[0] / 2 + (np.arange(fshape[2]) + 0.5) * fs[0]
    ref = lin(fz[:, None, None], fy[None, :, None], fx[None, None, :])
    inside = ((np.abs(fz) <= cz.max())[:, None, None] & (np.abs(fy) <= cy.max())[None, :, None]
              & (np.abs(fx) <= cx.max())[None, None, :])
    assert np.abs(ff - ref)[inside].max() < 1e-13
    assert np.abs(oracle.prolong(np.full(cshape, 0.7), cs, fshape, fs) - 0.7).max() < 1e-15


def test_restrict_of_constant_and_prolong_of_restrict_shapes():
    ff = np.full((7, 9, 10), 1.25)
    fc = oracle.restrict(ff, (1.0, 1.0, 1.0), (4, 5, 5), (2.0, 2.0, 2.0))
    assert np.abs(fc - 1.25).max() < 1e-15


def test_restrict_of_linear_function_on_aligned_grids():
    """Each coarse voxel holds 2x2x2 fine centres whose centroid is its own centre, so a
    linear function restricts to its values at the coarse centres."""
    lin = lambda z, y, x: 0.3 + 0.1 * x - 0.2 * y + 0.05 * z
    fshape, fs = (6, 8, 10), (1.0, 1.5, 2.0)      # (nz, ny, nx); spacings (dx, dy, dz)
    cshape, cs = (3, 4, 5), (2.0, 3.0, 4.0)
    c = lambda n, h: -n * h / 2 + (np.arange(n) + 0.5) * h
    ff = lin(c(fshape[0], fs[2])[:, None, None], c(fshape[1], fs[1])[None, :, None], c(fshape[2], fs[0])[None, None, :])
    ref = lin(c(cshape[0], cs[2])[:, None, None], c(cshape[1], cs[1])[None, :, None], c(cshape[2], cs[0])[None, None, :])
    assert np.abs(oracle.restrict(ff, fs, cshape, cs) - ref).max() < 1e-14


def test_restrict_of_linear_function_on_a_ragged_grid():
    """7 fine voxels of 1 mm (centres -3..3) under 4 coarse voxels of 2 mm (boxes
    [-4,-2), [-2,0), [0,2), [2,4)): the coarse voxels hold the centres {-3}, {-2,-1},
    {0,1}, {2,3}, whose means are -3, -1.5, 0.5, 2.5. A linear function of x restricts
    to its values there; a shifted or reversed coarse index fails."""
    x = np.arange(7) - 3.0
    ff = np.broadcast_to(0.2 + 0.7 * x, (2, 2, 7)).copy()
    fc = oracle.restrict(ff, (1.0, 1.0, 1.0), (1, 1, 4), (2.0, 2.0, 2.0))
    assert np.abs(fc[0, 0] - (0.2 + 0.7 * np.array([-3.0, -1.5, 0.5, 2.5]))).max() < 1e-15


def test_multigrid_single_level_equals_a2():
    geom = synth.config_small(n_views=6)
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = oracle.project(geom, f_true)
    r1 = oracle.reconstruct(geom, y, 5e-4, 1, [3])
    r2 = oracle.a2(geom, y, 5e-4, 3)
    assert np.array_equal(r1, r2)


def test_multigrid_two_levels_starts_from_prolonged_coarse_solution():
    geom = synth.config_small(n_views=6)
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = oracle.project(geom, f_true)
    coarse = geom.level(1)
    fc = oracle.a2(coarse, y, 5e-4, 2)
    ref = oracle.prolong(fc, (coarse.dx, coarse.dy, coarse.dz), geom.vol_shape, (geom.dx, geom.dy, geom.dz))
    out = oracle.reconstruct(geom, y, 5e-4, 2, [2, 0])
    assert np.array_equal(out, ref)
    # and refining from it lowers the data residual further
    out2 = oracle.reconstruct(geom, y, 5e-4, 2, [2, 2])
    assert np.linalg.norm(oracle.project(geom, out2) - y) < np.linalg.norm(oracle.project(geom, out) - y)
