"""P/P^T as a torch.autograd.Function on the differentiable batch workload: 8 seeded
ellipsoid volumes of 256x256x64 voxels (1.0 mm), 60 views on a 256x192 imager (1.5 mm).
The gradient of ½‖P f − y‖² is checked against central finite differences at 32 random
voxels and against the FP64 oracle's P^T (P f − y)."""
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


def batch_geometry():
    return synth.Geometry(nx=256, ny=256, nz=64, dx=1.0, dy=1.0, dz=1.0, nu=256, nv=192, du=1.5, dv=1.5,
                          n_views=60)


@pytest.fixture(scope="module")
def batch_case():
    geom = batch_geometry()
    fs = np.stack([synth.voxelize(geom, synth.random_ellipsoids(geom, 1004 + b, n=8)) for b in range(8)])
    return geom, fs


def test_gradient_matches_oracle_and_finite_differences(cb, batch_case):
    from paper_1008_2042_gb300 import autograd
    geom, fs = batch_case
    with cb.Geometry(geom) as g:
        f = torch.tensor(fs, dtype=torch.float32, device="cuda")
        # seeded synthetic data in the range of the line integrals (not fitted exactly)
        ys = np.stack([synth.random_projections(geom, 2004 + b, 0.0, 3.0) for b in range(8)])
        y = torch.tensor(ys, dtype=torch.float32, device="cuda")
        x = f.clone().requires_grad_(True)
        loss = 0.5 * ((autograd.project(g, x) - y).double() ** 2).sum()
        loss.backward()
        grad = x.grad.detach().cpu().numpy()

        # oracle gradient of item 0: P^T (P f - y), FP64
        y0 = ys[0].astype(np.float32).astype(np.float64)
        ref = oracle.backproject(geom, oracle.project(geom, fs[0].astype(np.float32).astype(np.float64)) - y0)
        err = np.linalg.norm(grad[0] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, err

        # central differences at 32 voxels of item 3 (the loss is quadratic: exact up to rounding)
        rng = np.random.default_rng(4)
        idx = rng.choice(geom.nx * geom.ny * geom.nz, 32, replace=False)
        f3 = f[3].clone()
        y3 = y[3]
        h = 1.0
        for j in idx:
            z, rem = divmod(int(j), geom.ny * geom.nx)
            yy, xx = divmod(rem, geom.nx)
            vals = []
            for sgn in (1.0, -1.0):
                fp = f3.clone()
                fp[z, yy, xx] += sgn * h
                with torch.no_grad():
                    vals.append(0.5 * ((cb.project(g, fp) - y3).double() ** 2).sum().item())
            fd = (vals[0] - vals[1]) / (2 * h)
            gj = grad[3, z, yy, xx]
            assert abs(fd - gj) <= 1e-3 * max(abs(gj), 1e-3 * np.abs(grad[3]).max()), (j, fd, gj)


def test_batch_items_are_independent(cb, batch_case):
    from paper_1008_2042_gb300 import autograd
    geom, fs = batch_case
    with cb.Geometry(geom) as g:
        f = torch.tensor(fs[:3], dtype=torch.float32, device="cuda", requires_grad=True)
        autograd.project(g, f).pow(2).sum().backward()
        for b in range(3):
            fb = torch.tensor(fs[b], dtype=torch.float32, device="cuda", requires_grad=True)
            autograd.project(g, fb).pow(2).sum().backward()
            assert torch.equal(fb.grad, f.grad[b])
