"""Pins for the 4D-TV oracle: closed forms on piecewise-constant fields and finite
differences (no GPU)."""
import math

import numpy as np

from oracle import tv4d


def test_spatial_closed_forms():
    dims = (3, 4, 5)
    V = 60
    c = np.full(V, 0.7)
    val, g = tv4d.spatial(c, dims, eps=1e-8)
    assert math.isclose(val, math.sqrt(1e-8), rel_tol=1e-12)
    np.testing.assert_array_equal(g, 0.0)
    # a step of height h across the x axis between x = 1 and x = 2: the 3*4 voxels at x = 1
    # see |d| = h, the rest sqrt(eps)
    s = np.zeros(dims)
    s[:, :, 2:] = 0.5
    val, _ = tv4d.spatial(s.reshape(-1), dims, eps=1e-8)
    ref = (12 * math.sqrt(0.25 + 1e-8) + 48 * math.sqrt(1e-8)) / V
    assert math.isclose(val, ref, rel_tol=1e-12)


def test_temporal_closed_form():
    prev = [np.zeros(10), np.ones(10)]
    cur = np.full(10, 3.0)
    val, _ = tv4d.temporal(cur, prev, eps=0.0)
    a0, a1 = math.exp(-2), math.exp(-1)
    assert math.isclose(val, (a0 * 30 + a1 * 20) / (a0 + a1), rel_tol=1e-14)
    assert tv4d.temporal(cur, [])[0] == 0.0


def test_gradients_finite_difference():
    rng = np.random.default_rng(1)
    dims = (3, 4, 2)
    s = rng.standard_normal(24)
    prev = [rng.standard_normal(24) for _ in range(3)]
    reg = tv4d.regulariser(dims, prev, eps=1e-3)
    _, g = reg(s)
    d = rng.standard_normal(24)
    h = 1e-6
    fd = (reg(s + h * d)[0] - reg(s - h * d)[0]) / (2 * h)
    assert abs(fd - g @ d) < 1e-8 * max(1.0, abs(fd))
