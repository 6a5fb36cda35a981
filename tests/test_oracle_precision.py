"""Pins of the oracle's reduced-precision variant (no counterpart in the paper): the
rounding to bfloat16 / binary16 against a brute-force nearest-even search over every
code of the format and against numpy's binary16 cast, and the CGLS that holds r and q
in those formats against a dense-matrix restatement that rounds by the brute-force
search."""
import numpy as np
import pytest

import oracle
import synth
from oracle import dense

CODES = {"bf16": 1, "f16": 2}


def _samples(fmt, rng):
    vals, _ = dense.format_codes(fmt)
    mids = 0.5 * (vals[:-1] + vals[1:])          # every tie between neighbours
    if fmt == "f16":
        mags = 10.0 ** rng.uniform(-9, 5, 20000)   # subnormals .. overflow
        edge = [65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -25, 3 * 2.0 ** -25, 2.0 ** -24]
    else:
        mags = 10.0 ** rng.uniform(-42, 38.6, 20000)
        edge = [2.0 ** -133, 2.0 ** -134, 3 * 2.0 ** -134, 3.3e38, 3.4e38, -3.4e38]
    return np.concatenate([rng.standard_normal(20000) * mags, mids, edge])


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_rounding_matches_brute_force_nearest_even(fmt):
    x = _samples(fmt, np.random.default_rng(11))
    got = oracle.round_storage(x, CODES[fmt])
    want = dense.round_nearest_even(x, fmt)
    assert np.array_equal(got, want)


def test_binary16_rounding_matches_numpy_cast():
    x = _samples("f16", np.random.default_rng(12))
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(oracle.round_storage(x, 2), want)


def test_brute_force_search_knows_the_formats():
    """Independent facts about the formats: largest finite values, smallest subnormals
    and the number of finite non-negative codes."""
    v16, _ = dense.format_codes("f16")
    vb, _ = dense.format_codes("bf16")
    assert v16[-1] == 65504.0 and v16[v16 > 0][0] == 2.0 ** -24
    assert vb[-1] == (2 - 2 ** -7) * 2.0 ** 127 and vb[vb > 0][0] == 2.0 ** -133
    assert (v16 >= 0).sum() == 0x7C00 and (vb >= 0).sum() == 0x7F80
    # bfloat16 spacing at 1 is 2^-7: ties go to the even code
    assert dense.round_nearest_even(1 + 2 ** -8, "bf16") == 1.0
    assert dense.round_nearest_even(1 + 3 * 2 ** -8, "bf16") == 1 + 2 ** -6
    assert np.isinf(dense.round_nearest_even(65520.0, "f16"))


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_cgls_storage_matches_dense_restatement(fmt):
    geom = synth.Geometry(nx=6, ny=5, nz=4, dx=2.0, dy=2.2, dz=1.5, nu=12, nv=6, du=2.5, dv=2.0, n_views=5)
    A = dense.system_matrix(geom)
    f = synth.random_volume(geom, 3)
    y = (A @ f.ravel()).reshape(geom.proj_shape) + 0.01 * np.random.default_rng(1).standard_normal(geom.proj_shape)
    x0 = np.full(geom.vol_shape, 0.01)
    for n in (1, 4):
        got = oracle.cgls(geom, y, x0, n, storage=fmt)
        want = dense.cgls_dense(A, y.ravel(), x0.ravel(), n, storage=fmt)
        assert np.linalg.norm(got.ravel() - want) <= 1e-12 * np.linalg.norm(want)
        # the rounding is felt, and it stays a perturbation of the FP64 iterate
        plain = oracle.cgls(geom, y, x0, n)
        d = np.linalg.norm(got - plain) / np.linalg.norm(plain)
        assert 0 < d < 50 * {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[fmt]

