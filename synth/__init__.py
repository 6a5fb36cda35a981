"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds only input generation: scan geometries, ellipsoid phantoms and the
Poisson noise model of the measured line integrals. It contains none of the
reconstruction method's arithmetic (no projector, no frame transform, no iteration), so
the FP64 oracle and the CUDA path can both be fed from it without sharing any code.

The paper's own data (the NCAT digital phantom, the Catphan scans and the patient scan
of Section 3) are not available; seeded ellipsoid phantoms in the paper's scan geometry
(Section 3: source-to-axis 100 cm, source-to-imager 150 cm, circular orbit, flat imager,
40 views over a full turn) stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Circular-orbit cone-beam geometry with a flat imager (Section 2.1, Fig. 1).

    Lengths in mm, angles in radians. The volume is centred on the rotation axis (z);
    voxel (ix, iy, iz) is the half-open box starting at (-nx*dx/2 + ix*dx, ...). View k
    places the source at sad*(cos t, sin t, 0) and the imager centre at
    -(sdd - sad)*(cos t, sin t, 0); the imager u axis is (-sin t, cos t, 0) and its v
    axis is z. Pixel (iu, iv) is centred at u = u_off + (iu - (nu-1)/2)*du,
    v = v_off + (iv - (nv-1)/2)*dv. ``angles`` None means n_views angles evenly spaced
    over 2*pi starting at 0.
    """

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    nu: int
    nv: int
    du: float
    dv: float
    sad: float = 1000.0
    sdd: float = 1500.0
    n_views: int = 40
    u_off: float = 0.0
    v_off: float = 0.0
    angles: Optional[tuple] = None

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            a = np.asarray(self.angles, dtype=np.float64)
            assert a.shape == (self.n_views,)
            return a
        return 2.0 * np.pi * np.arange(self.n_views, dtype=np.float64) / self.n_views

    @property
    def vol_shape(self):
        """numpy shape of a volume, x fastest: (nz, ny, nx)."""
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self):
        """numpy shape of a projection stack, u fastest: (n_views, nv, nu)."""
        return (self.n_views, self.nv, self.nu)

    def level(self, ell: int) -> "Geometry":
        """Grid of multigrid level ell (0 = finest): ceil(n / 2**ell) voxels per axis at
        2**ell times the spacing, same centre; the imager is not coarsened."""
        s = 2 ** ell
        return dataclasses.replace(
            self,
            nx=-(-self.nx // s), ny=-(-self.ny // s), nz=-(-self.nz // s),
            dx=self.dx * s, dy=self.dy * s, dz=self.dz * s)


# ---------------------------------------------------------------------------------------
# Workload shapes (synthetic stand-ins for the paper's Section 3 workloads)
# ---------------------------------------------------------------------------------------

def config_small(n_views: int = 40) -> Geometry:
    """64x64x16 voxels of 1.0 mm; 128x32 imager at 0.8 mm; 40 views (small parity case)."""
    return Geometry(nx=64, ny=64, nz=16, dx=1.0, dy=1.0, dz=1.0,
                    nu=128, nv=32, du=0.8, dv=0.8, n_views=n_views)


def config_paper(n_views: int = 40) -> Geometry:
    """512x512x70 voxels of 0.5x0.5x2.5 mm; 512x384 imager at 0.776 mm; 40 or 80 views."""
    return Geometry(nx=512, ny=512, nz=70, dx=0.5, dy=0.5, dz=2.5,
                    nu=512, nv=384, du=0.776, dv=0.776, n_views=n_views)


# ---------------------------------------------------------------------------------------
# Ellipsoid phantoms
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Ellipsoid:
    """Solid ellipsoid: centre (mm), semi-axes (mm), rotation phi about z (rad), value (/mm)."""
    cx: float
    cy: float
    cz: float
    ax: float
    ay: float
    az: float
    phi: float
    value: float


def voxel_centres(geom: Geometry):
    """1-D voxel-centre coordinates (x, y, z) in mm."""
    x = -geom.nx * geom.dx / 2 + (np.arange(geom.nx) + 0.5) * geom.dx
    y = -geom.ny * geom.dy / 2 + (np.arange(geom.ny) + 0.5) * geom.dy
    z = -geom.nz * geom.dz / 2 + (np.arange(geom.nz) + 0.5) * geom.dz
    return x, y, z


def voxelize(geom: Geometry, ellipsoids: Sequence[Ellipsoid]) -> np.ndarray:
    """Sample the phantom at voxel centres; later ellipsoids overwrite earlier ones.

    Returns float64 (nz, ny, nx). Each ellipsoid is evaluated only inside its bounding box."""
    x, y, z = voxel_centres(geom)
    f = np.zeros(geom.vol_shape, dtype=np.float64)
    for e in ellipsoids:
        c, s = math.cos(e.phi), math.sin(e.phi)
        hx = math.hypot(e.ax * c, e.ay * s)
        hy = math.hypot(e.ax * s, e.ay * c)
        sel = [np.nonzero(np.abs(v - cen) <= h + 1e-9)[0]
               for v, cen, h in ((z, e.cz, e.az), (y, e.cy, hy), (x, e.cx, hx))]
        if any(len(q) == 0 for q in sel):
            continue
        (z0, z1), (y0, y1), (x0, x1) = [(q[0], q[-1] + 1) for q in sel]
        Z, Y, X = np.meshgrid(z[z0:z1], y[y0:y1], x[x0:x1], indexing="ij")
        xr = (X - e.cx) * c + (Y - e.cy) * s
        yr = -(X - e.cx) * s + (Y - e.cy) * c
        zr = Z - e.cz
        inside = (xr / e.ax) ** 2 + (yr / e.ay) ** 2 + (zr / e.az) ** 2 <= 1.0
        f[z0:z1, y0:y1, x0:x1][inside] = e.value
    return f


def random_ellipsoids(geom: Geometry, seed: int, n: int = 6, vmax: float = 0.03):
    """n ellipsoids: centres uniform in the inner 70 % of the box, semi-axes uniform in
    5-25 mm (clipped to the box half-extent), random rotation about z, values uniform in
    [0, vmax] /mm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hx, hy, hz = geom.nx * geom.dx / 2, geom.ny * geom.dy / 2, geom.nz * geom.dz / 2
    out = []
    for _ in range(n):
        cx, cy, cz = (rng.uniform(-0.7, 0.7) * h for h in (hx, hy, hz))
        ax, ay, az = (min(rng.uniform(5.0, 25.0), h) for h in (hx, hy, hz))
        out.append(Ellipsoid(cx, cy, cz, ax, ay, az, rng.uniform(0, np.pi), rng.uniform(0.0, vmax)))
    return out


def torso_ellipsoids(geom: Geometry, seed: int):
    """A 30-ellipsoid torso: body (0.02 /mm), two lungs (0.005 /mm) and 27 bones, spine
    and ribs (0.04 /mm), scaled to the volume's transverse extent."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hx, hy, hz = geom.nx * geom.dx / 2, geom.ny * geom.dy / 2, geom.nz * geom.dz / 2
    e = [Ellipsoid(0, 0, 0, 0.85 * hx, 0.62 * hy, 1.2 * hz, 0.0, 0.02)]
    for sgn in (-1, 1):
        e.append(Ellipsoid(sgn * 0.38 * hx, 0.05 * hy, 0.0, 0.28 * hx, 0.38 * hy, 1.1 * hz,
                           sgn * 0.15, 0.005))
    # spine: 3 vertebral bodies along z behind the centre
    for k in range(3):
        e.append(Ellipsoid(0.0, -0.42 * hy, (k - 1) * 0.6 * hz, 0.09 * hx, 0.08 * hy,
                           0.25 * hz, 0.0, 0.04))
    # sternum
    e.append(Ellipsoid(0.0, 0.5 * hy, 0.0, 0.08 * hx, 0.03 * hy, 0.9 * hz, 0.0, 0.04))
    # 23 rib cross-sections around the body outline, jittered
    for k in range(23):
        a = 2 * np.pi * (k + 0.5) / 23 + rng.uniform(-0.05, 0.05)
        rx, ry = 0.78 * hx * np.cos(a), 0.55 * hy * np.sin(a)
        e.append(Ellipsoid(rx, ry, rng.uniform(-0.5, 0.5) * hz, rng.uniform(0.015, 0.03) * hx,
                           rng.uniform(0.012, 0.025) * hy, rng.uniform(0.15, 0.4) * hz,
                           a, 0.04))
    assert len(e) == 30
    return e


def random_volume(geom: Geometry, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform volume (nz, ny, nx), float64 — for operator parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=geom.vol_shape)


def random_projections(geom: Geometry, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform projection stack (n_views, nv, nu), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=geom.proj_shape)


# ---------------------------------------------------------------------------------------
# Measurement model (data simulation, not part of the method)
# ---------------------------------------------------------------------------------------

def noisy_line_integrals(p: np.ndarray, photons: float, seed: int) -> np.ndarray:
    """Poisson transmission noise on ideal line integrals p (1/mm * mm):
    N ~ Poisson(photons * exp(-p)), y = -ln(max(N, 1) / photons). float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.poisson(photons * np.exp(-np.asarray(p, dtype=np.float64)))
    return -np.log(np.maximum(counts, 1) / photons)


def default_level_iters(levels: int, total: int) -> list:
    """Split ``total`` outer iterations over ``levels`` grids in the ratio 1:2:...:levels
    (coarsest first) — the 5/10/15 proportions of Section 3.1 — rounding so they sum to
    ``total``."""
    w = np.arange(1, levels + 1, dtype=np.float64)
    raw = total * w / w.sum()
    it = np.floor(raw).astype(int)
    rem = total - it.sum()
    order = np.argsort(-(raw - it))
    for j in range(rem):
        it[order[j]] += 1
    return [int(v) for v in it]
