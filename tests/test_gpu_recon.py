"""Parity of the CUDA iteration (CGLS, A2, multigrid) with the FP64 oracle through the C
ABI, at the small configuration (64x64x16, 40 views, 20 iterations) within relative L2
1e-3, plus error behaviour of the boundary."""
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


@pytest.fixture(scope="module")
def small_case():
    """The small workload: 6 seeded ellipsoids, Poisson noise at 1e5 photons per ray."""
    geom = synth.config_small()
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, 1001))
    y = synth.noisy_line_integrals(oracle.project(geom, f_true), 1e5, 2001)
    return geom, f_true, y


def test_cgls_parity(cb, small_case):
    geom, f_true, y = small_case
    x0 = np.full(geom.vol_shape, 0.005)
    with cb.Geometry(geom) as g:
        for n in (1, 3):
            x = cb.cgls(g, dev(y), dev(x0), n).cpu().numpy()
            ref = oracle.cgls(geom, y, x0, n)
            assert rel(x, ref) <= 1e-4, (n, rel(x, ref))


def test_reconstruct_small_config_parity(cb, small_case):
    geom, f_true, y = small_case
    mu = 5e-4
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), mu, 1, [20]).cpu().numpy()
    ref = oracle.reconstruct(geom, y, mu, 1, [20])
    assert rel(out, ref) <= 1e-3, rel(out, ref)
    assert out.min() >= 0.0
    # the reconstruction is a reconstruction: close to the phantom
    assert rel(ref, f_true) < 0.5


@pytest.mark.parametrize("momentum,positivity", [(False, True), (True, False)])
def test_reconstruct_variants_parity(cb, small_case, momentum, positivity):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), 1e-3, 1, [6], momentum=momentum, positivity=positivity,
                             n_cgls=2).cpu().numpy()
    ref = oracle.reconstruct(geom, y, 1e-3, 1, [6], n_cgls=2, momentum=momentum, positivity=positivity)
    assert rel(out, ref) <= 1e-3, rel(out, ref)


def test_multigrid_parity(cb, small_case):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), 5e-4, 3, [3, 4, 5]).cpu().numpy()
    ref = oracle.reconstruct(geom, y, 5e-4, 3, [3, 4, 5])
    assert rel(out, ref) <= 1e-3, rel(out, ref)


def test_caller_workspace_gives_same_result(cb, small_case):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        a = cb.reconstruct(g, dev(y), 5e-4, 2, [2, 3]).cpu().numpy()
        ws = torch.empty(cb.reconstruct_workspace_size(g), dtype=torch.uint8, device="cuda")
        b = cb.reconstruct(g, dev(y), 5e-4, 2, [2, 3], workspace=ws).cpu().numpy()
    assert np.array_equal(a, b)


def test_zero_iterations_give_zero(cb, small_case):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        out = cb.reconstruct(g, dev(y), 5e-4, 2, [0, 0]).cpu().numpy()
    assert not out.any()


def test_lambda_is_unsupported_and_nan_is_reported(cb, small_case):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        with pytest.raises(cb.CbctError) as e:
            cb.reconstruct(g, dev(y), 5e-4, 1, [1], lam=0.5)
        assert e.value.status == 5
        bad = y.copy()
        bad[3, 4, 5] = np.nan
        with pytest.raises(cb.CbctError) as e:
            cb.reconstruct(g, dev(bad), 5e-4, 1, [1])
        assert e.value.status == 4
        # the handle stays usable after an error
        out = cb.reconstruct(g, dev(y), 5e-4, 1, [1]).cpu().numpy()
        assert np.isfinite(out).all()


def test_shape_errors_are_raised_before_launch(cb, small_case):
    geom, _, y = small_case
    with cb.Geometry(geom) as g:
        with pytest.raises(ValueError):
            cb.project(g, torch.zeros((2, 2, 2), device="cuda"))
        with pytest.raises(TypeError):
            cb.project(g, torch.zeros(geom.vol_shape, device="cuda", dtype=torch.float64))
