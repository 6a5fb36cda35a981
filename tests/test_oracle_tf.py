"""Pins of the oracle's tight-frame analysis W, synthesis W^T and shrinkage T_mu
(Section 2.1, Eq. (2)) against the printed filter taps and closed forms."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [(5, 6, 7), (8, 8, 8), (1, 4, 3), (2, 3, 5), (3, 1, 2)]


def _printed_filters():
    """The paper's filters from the golden file: dict name -> taps at offsets -1, 0, 1."""
    out = {}
    with open(os.path.join(GOLDEN, "tf_filters.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                a, b = float(line[1]), float(line[2])
                out[line[0]] = math.sqrt(a) / b * np.array([float(t) for t in line[3:6]])
    return out


@pytest.mark.parametrize("shape", SHAPES)
def test_tight_frame_identity(shape):
    f = np.random.default_rng(1).standard_normal(shape)
    back = oracle.tf_synthesize(oracle.tf_analyze(f))
    assert np.abs(back - f).max() <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_parseval(shape):
    f = np.random.default_rng(2).standard_normal(shape)
    a = oracle.tf_analyze(f)
    assert abs(np.linalg.norm(a) - np.linalg.norm(f)) <= 1e-12 * np.linalg.norm(f)


def test_synthesis_is_transpose():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((4, 5, 6))
    a = rng.standard_normal((27, 4, 5, 6))
    lhs = np.vdot(oracle.tf_analyze(f), a)
    rhs = np.vdot(f, oracle.tf_synthesize(a))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_constant_volume_has_only_lowpass():
    a = oracle.tf_analyze(np.full((6, 5, 7), 0.37))
    assert np.abs(a[0] - 0.37).max() < 1e-14
    assert np.abs(a[1:]).max() < 1e-14


def test_impulse_response_equals_printed_filters():
    """alpha_i = psi_i conv delta_p, so alpha_i(p + k) = h_l(k_x) h_m(k_y) h_n(k_z) with
    i = l + 3m + 9n and the printed taps (Section 2.1)."""
    h = _printed_filters()
    H = [h["h0"], h["h1"], h["h2"]]
    f = np.zeros((7, 7, 7))
    f[3, 3, 3] = 1.0
    a = oracle.tf_analyze(f)
    for i in range(27):
        l, m, n = i % 3, (i // 3) % 3, i // 9
        expect = np.einsum("c,b,a->cba", H[n], H[m], H[l])  # offsets -1, 0, 1 on z, y, x
        assert np.abs(a[i, 2:5, 2:5, 2:5] - expect).max() < 1e-15, i
        mask = np.ones((7, 7, 7), bool)
        mask[2:5, 2:5, 2:5] = False
        assert np.abs(a[i][mask]).max() == 0.0


def test_h1_of_a_ramp_is_a_scaled_central_difference():
    """Section 4: h1 acts as a central difference; on f = x it gives sqrt(2)/2 per unit slope."""
    x = np.arange(10, dtype=np.float64)
    f = np.broadcast_to(x[None, None, :], (4, 5, 10)).copy()
    a = oracle.tf_analyze(f)
    assert np.abs(a[1][:, :, 1:-1] - math.sqrt(2) / 2).max() < 1e-14  # l=1, m=n=0
    assert np.abs(a[2][:, :, 1:-1]).max() < 1e-14                     # h2 kills linears


def test_zero_threshold_is_identity():
    f = np.random.default_rng(4).standard_normal((5, 6, 7))
    out = oracle.tf_synthesize_shrink(oracle.tf_analyze(f), 0.0, False)
    assert np.abs(out - f).max() <= 1e-12


def test_huge_threshold_keeps_lowpass_smoothing():
    """mu -> inf removes all high-pass channels: W^T keeps psi_0 * psi_0, i.e. the
    autocorrelation of h0, [1, 4, 6, 4, 1] / 16 along each axis (periodic)."""
    rng = np.random.default_rng(5)
    f = rng.standard_normal((6, 7, 8))
    out = oracle.tf_synthesize_shrink(oracle.tf_analyze(f), 1e30, False)
    k = np.array([1, 4, 6, 4, 1]) / 16.0
    ref = f.copy()
    for ax in range(3):
        ref = sum(k[j] * np.roll(ref, j - 2, axis=ax) for j in range(5))
    assert np.abs(out - ref).max() <= 1e-12


def test_vector_shrinkage_formula():
    """Eq. (2) on a hand-built coefficient field: norm 2 mu -> factor 1/2; norm <= mu -> 0;
    alpha_0 untouched; zero norm gives zero (no division by zero)."""
    mu = 0.3
    a = np.zeros((27, 1, 1, 4))
    a[0] = 5.0
    a[1:, 0, 0, 0] = 2 * mu / math.sqrt(26)     # norm 2 mu
    a[1:, 0, 0, 1] = mu / math.sqrt(26)         # norm exactly mu
    a[1:, 0, 0, 2] = 0.5 * mu / math.sqrt(26)   # norm below mu
    out = oracle.tf_shrink(a, mu)
    assert np.allclose(out[0], 5.0, rtol=0, atol=0)
    assert np.allclose(out[1:, 0, 0, 0], mu / math.sqrt(26), rtol=1e-14, atol=0)
    assert np.abs(out[1:, 0, 0, 1:]).max() <= 1e-17
    assert np.all(np.isfinite(out))


def test_positivity():
    f = np.array([-1.0, 0.0, 2.0, -1e-300])
    assert np.array_equal(oracle.positivity(f), np.array([0.0, 0.0, 2.0, 0.0]))


def test_sampled_regularisation_step_matches_the_three_steps():
    f = np.random.default_rng(21).standard_normal((6, 9, 11))
    alpha = oracle.tf_analyze(f)
    mu = float(np.median(np.sqrt((alpha[1:] ** 2).sum(0))))
    for positive in (False, True):
        full = oracle.tf_synthesize_shrink(alpha, mu, positive).ravel()
        sel = np.arange(full.size)
        assert np.abs(oracle.tf_shrink_voxels(f, mu, positive, sel) - full).max() <= 1e-12 * np.abs(full).max()
