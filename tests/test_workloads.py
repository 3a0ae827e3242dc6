"""Synthetic input recipes: shapes, dtypes, seeds, unit power, tilt spans."""
import math

import numpy as np

import workloads as W


def test_configs_shapes_and_recipe():
    c1 = W.config_c1(1)
    assert (c1.nx, c1.ny, c1.N, c1.D, c1.iters) == (256, 256, 16, 10, 20)
    assert c1.noll == list(range(2, 12))
    assert c1.amp.dtype == np.float32 and c1.coeff.dtype == np.float32
    assert abs(float(np.sum(c1.amp.astype(np.float64) ** 2)) - 1.0) < 1e-5
    R = 128.0
    assert np.abs(c1.coeff[:, :2]).max() <= 0.4 * math.pi * R * (1 + 1e-6)
    assert np.all(c1.coeff[:, 2] == 0.0)          # defocus 0
    assert np.all(c1.target == 1.0)
    c2 = W.config_c2(1)
    assert (c2.nx, c2.ny, c2.N, c2.D, c2.iters) == (1024, 1024, 400, 10, 50)
    assert np.abs(c2.coeff[:, :2]).max() <= 0.45 * math.pi * 512 * (1 + 1e-6)
    # 50 patches: at most 50 distinct aberration rows
    assert len({tuple(r) for r in c2.coeff[:, 2:]}) <= 50
    c3 = W.config_c3(1)
    assert (c3.nx, c3.ny, c3.N, c3.D, c3.iters) == (1920, 1152, 2000, 11, 100)
    assert sorted(set(np.round(c3.coeff[:, 2], 4))) == [-20.0, -10.0, 0.0, 10.0, 20.0]
    assert c3.target.min() >= 0.5 and c3.target.max() <= 1.0
    assert np.allclose(c3.amp, c3.amp.flat[0])


def test_seeded_and_distinct():
    a, b, c = W.config_c1(1), W.config_c1(1), W.config_c1(2)
    assert np.array_equal(a.coeff, b.coeff) and np.array_equal(a.phase0, b.phase0)
    assert not np.array_equal(a.coeff, c.coeff)


def test_c5_batch_mix():
    hs = W.config_c5(1, count=64)
    assert len(hs) == 64
    for h in hs:
        assert (h.nx, h.ny) in W.C5_SIZES
        assert 10 <= h.N <= 5000
        assert h.D in (5, 10, 11) and h.coeff.shape == (h.N, h.D)
