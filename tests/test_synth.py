"""The seeded input generators are deterministic and produce the stated shapes."""
import numpy as np

import synth


def test_phantoms_are_seeded_and_shaped():
    g = synth.config_small()
    a = synth.voxelize(g, synth.random_ellipsoids(g, 1001))
    b = synth.voxelize(g, synth.random_ellipsoids(g, 1001))
    assert a.shape == (16, 64, 64) and np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() <= 0.03 and (a > 0).mean() > 0.02
    t = synth.torso_ellipsoids(synth.config_paper(), 1002)
    assert len(t) == 30
    vals = sorted({e.value for e in t})
    assert vals == [0.005, 0.02, 0.04]


def test_noise_model_is_seeded():
    p = np.linspace(0.0, 4.0, 1000)
    y1 = synth.noisy_line_integrals(p, 1e5, 3)
    y2 = synth.noisy_line_integrals(p, 1e5, 3)
    assert np.array_equal(y1, y2)
    assert np.abs(y1 - p).max() < 0.2


def test_iteration_split_follows_paper_ratio():
    assert synth.default_level_iters(3, 30) == [5, 10, 15]
    assert synth.default_level_iters(3, 50) == [8, 17, 25]
    assert synth.default_level_iters(1, 20) == [20]


def test_multigrid_level_shapes():
    g = synth.config_paper()
    assert g.level(1).vol_shape == (35, 256, 256)
    assert g.level(2).vol_shape == (18, 128, 128)
    assert g.level(2).dz == 10.0 and g.level(2).nu == g.nu
