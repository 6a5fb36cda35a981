"""Pins of the FP64 oracle's projector P and adjoint P^T against things other than itself:
an independent brute-force system matrix, closed-form chords, the adjoint identity of
Eq. (A1), the paper's Eq. (3) and the paper's non-zero count (Section 2.2.2)."""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_geoms():
    base = synth.Geometry(nx=8, ny=8, nz=8, dx=4.0, dy=4.0, dz=4.0, nu=12, nv=10, du=4.0,
                          dv=4.0, n_views=6)
    return [
        base,
        # odd sizes, anisotropic voxels, detector offsets, rotated start angle
        dataclasses.replace(base, nx=7, ny=9, nz=5, dx=3.0, dy=5.0, dz=2.5, nu=11, nv=7,
                            u_off=1.3, v_off=-0.7,
                            angles=tuple(0.1 + 2 * np.pi * np.arange(6) / 6), n_views=6),
        # strong cone angle: detector spans far above/below the volume
        dataclasses.replace(base, nz=4, dz=8.0, nv=16, dv=9.0, n_views=4),
    ]


def _chord_box(S, D, lo, hi):
    """Length of segment S->D inside the box [lo, hi] (written out per axis)."""
    d = D - S
    t0, t1 = 0.0, 1.0
    for a in range(3):
        if abs(d[a]) < 1e-300:
            if not (lo[a] <= S[a] < hi[a]):
                return 0.0
            continue
        ta, tb = sorted(((lo[a] - S[a]) / d[a], (hi[a] - S[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(t1 - t0, 0.0) * float(np.linalg.norm(d))


def _rays(geom):
    """Source and pixel-centre positions of all rays, ordered (k, iv, iu)."""
    out = []
    for k, th in enumerate(geom.view_angles()):
        c, s = math.cos(th), math.sin(th)
        S = np.array([geom.sad * c, geom.sad * s, 0.0])
        C = -(geom.sdd - geom.sad) * np.array([c, s, 0.0])
        eu = np.array([-s, c, 0.0])
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                u = geom.u_off + (iu - (geom.nu - 1) / 2) * geom.du
                v = geom.v_off + (iv - (geom.nv - 1) / 2) * geom.dv
                out.append((S, C + u * eu + np.array([0.0, 0.0, v])))
    return out


@pytest.mark.parametrize("gi", range(3))
def test_siddon_equals_bruteforce_matrix(gi):
    geom = _small_geoms()[gi]
    A = dense.system_matrix(geom)
    f = synth.random_volume(geom, 11 + gi)
    y = synth.random_projections(geom, 21 + gi)
    p = oracle.project(geom, f).ravel()
    ref = A @ f.ravel()
    assert np.linalg.norm(p - ref) <= 1e-12 * np.linalg.norm(ref)
    bt = oracle.backproject(geom, y).ravel()
    refT = A.T @ y.ravel()
    assert np.linalg.norm(bt - refT) <= 1e-12 * np.linalg.norm(refT)
    assert oracle.count_nnz(geom) == int((A > 1e-9 * min(geom.dx, geom.dy, geom.dz)).sum())


def test_unit_volume_gives_box_chord():
    geom = synth.config_small(n_views=8)
    p = oracle.project(geom, np.ones(geom.vol_shape)).ravel()
    lo = -0.5 * np.array([geom.nx * geom.dx, geom.ny * geom.dy, geom.nz * geom.dz])
    ref = np.array([_chord_box(S, D, lo, -lo) for S, D in _rays(geom)])
    assert np.abs(p - ref).max() <= 1e-10
    assert (ref > 0).mean() > 0.5  # most rays cross the volume


def test_voxel_aligned_block_gives_exact_chord():
    geom = dataclasses.replace(synth.config_small(n_views=5), angles=tuple(0.3 + np.arange(5)))
    f = np.zeros(geom.vol_shape)
    f[3:11, 20:37, 5:50] = 0.017
    p = oracle.project(geom, f).ravel()
    x0, y0, z0 = -geom.nx * geom.dx / 2, -geom.ny * geom.dy / 2, -geom.nz * geom.dz / 2
    lo = np.array([x0 + 5 * geom.dx, y0 + 20 * geom.dy, z0 + 3 * geom.dz])
    hi = np.array([x0 + 50 * geom.dx, y0 + 37 * geom.dy, z0 + 11 * geom.dz])
    ref = 0.017 * np.array([_chord_box(S, D, lo, hi) for S, D in _rays(geom)])
    assert np.abs(p - ref).max() <= 1e-12
    assert (ref > 0).sum() > 1000


def _ellipsoid_chord(S, D, e):
    """Analytic chord of segment S->D through a solid ellipsoid (quadratic roots)."""
    c, s = math.cos(e.phi), math.sin(e.phi)
    R = np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])
    ax = np.array([e.ax, e.ay, e.az])
    p0 = R @ (S - np.array([e.cx, e.cy, e.cz])) / ax
    dd = R @ (D - S) / ax
    a, b, cc = dd @ dd, 2 * p0 @ dd, p0 @ p0 - 1.0
    disc = b * b - 4 * a * cc
    if disc <= 0:
        return 0.0
    r = math.sqrt(disc)
    t0, t1 = max((-b - r) / (2 * a), 0.0), min((-b + r) / (2 * a), 1.0)
    return max(t1 - t0, 0.0) * float(np.linalg.norm(D - S))


def test_ellipsoid_chord_converges_under_refinement():
    e = synth.Ellipsoid(3.0, -2.0, 1.0, 20.0, 13.0, 9.0, 0.4, 0.02)
    errs = []
    for n, h in ((16, 4.0), (32, 2.0), (64, 1.0)):
        geom = synth.Geometry(nx=n, ny=n, nz=n // 2, dx=h, dy=h, dz=h, nu=48, nv=32, du=2.0,
                              dv=2.0, n_views=3, angles=(0.2, 1.3, 2.5))
        f = synth.voxelize(geom, [e])
        p = oracle.project(geom, f).ravel()
        ref = np.array([e.value * _ellipsoid_chord(S, D, e) for S, D in _rays(geom)])
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    # voxelisation error is O(h): every halving of the voxel size about halves it
    assert errs[1] < 0.65 * errs[0] and errs[2] < 0.65 * errs[1], errs
    assert errs[2] < 0.08, errs


def test_adjoint_identity_fp64():
    geom = synth.config_small(n_views=40)
    f = synth.random_volume(geom, 5)
    y = synth.random_projections(geom, 6)
    lhs = float(np.vdot(oracle.project(geom, f), y))
    rhs = float(np.vdot(f, oracle.backproject(geom, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_sampled_backprojection_matches_scatter():
    geom = synth.Geometry(nx=32, ny=24, nz=8, dx=2.0, dy=2.0, dz=3.0, nu=64, nv=16, du=1.6,
                          dv=2.0, n_views=10)
    y = synth.random_projections(geom, 8)
    full = oracle.backproject(geom, y).ravel()
    rng = np.random.default_rng(0)
    sel = rng.choice(full.size, 300, replace=False)
    part = oracle.backproject_voxels(geom, y, sel)
    assert np.abs(part - full[sel]).max() <= 1e-11 * np.abs(full).max()


def test_eq3_backprojector_agrees_with_exact_adjoint_for_dense_rays():
    """Appendix 2: with many rays per voxel the exact transpose of the Siddon weights
    applied to a constant imager approaches Eq. (3) (volume x ray density)."""
    geom = synth.Geometry(nx=12, ny=12, nz=6, dx=4.0, dy=4.0, dz=4.0, nu=320, nv=160, du=0.25,
                          dv=0.25, n_views=4, angles=(0.1, 0.9, 2.0, 4.0))
    ones = np.ones(geom.proj_shape)
    exact = oracle.backproject(geom, ones)
    eq3 = oracle.backproject_eq3(geom, ones)
    rel = np.abs(exact - eq3) / eq3
    # voxels whose shadow stays on the imager in every view (the imager is 80 mm wide)
    x, y, _ = synth.voxel_centres(geom)
    covered = np.broadcast_to(np.hypot(x[None, None, :], y[None, :, None]) < 20.0, rel.shape)
    assert np.median(rel[covered]) < 0.005, np.median(rel[covered])
    assert rel[covered].max() < 0.02, rel[covered].max()


def _golden_paper_numbers():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                vals[line[0]] = [float(v) for v in line[1:]]
    return vals


@pytest.mark.slow
def test_nonzero_count_matches_paper_order_of_magnitude():
    """Section 2.2.2: ~4e9 non-zeros for the clinical geometry of Section 3. The volume
    and imager are square in x/y, so views 0..9 (one quadrant) give a quarter of the total."""
    g = _golden_paper_numbers()
    nx, ny, nz, dx, dy, dz = g["vol"]
    nu, nv, wu, wv = g["imager"]
    sad, sdd = g["sad_sdd"]
    K = int(g["views"][0])
    geom = synth.Geometry(nx=int(nx), ny=int(ny), nz=int(nz), dx=dx, dy=dy, dz=dz,
                          nu=int(nu), nv=int(nv), du=wu / nu, dv=wv / nv, sad=sad, sdd=sdd,
                          n_views=K // 4, angles=tuple(2 * np.pi * np.arange(K // 4) / K))
    nnz = 4 * oracle.count_nnz(geom)
    assert 0.5 * g["nnz_clinical"][0] <= nnz <= 2.0 * g["nnz_clinical"][0], nnz


def test_sampled_projection_matches_full_projection():
    geom = synth.Geometry(nx=32, ny=24, nz=8, dx=2.0, dy=2.0, dz=3.0, nu=64, nv=16, du=1.6,
                          dv=2.0, n_views=10)
    f = synth.random_volume(geom, 9)
    full = oracle.project(geom, f).ravel()
    sel = np.random.default_rng(1).choice(full.size, 300, replace=False)
    assert np.array_equal(oracle.project_rays(geom, f, sel), full[sel])
