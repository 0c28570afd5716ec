"""Pins for the oracle's primitive ops against brute force, library special cases,
adjoint identities and finite differences (no GPU)."""
import itertools

import numpy as np
import pytest
import scipy.ndimage
import torch

from oracle import network as net


def _brute_conv(x, W, b, stride):
    """Seven nested loops over output voxel, output channel, taps and input channel."""
    Dz, Dy, Dx, Ci = x.shape
    Co, K = W.shape[0], W.shape[1]
    pad = (K - 1) // 2
    O = [(d + 2 * pad - K) // stride + 1 for d in (Dz, Dy, Dx)]
    y = np.zeros((*O, Co))
    for oz in range(O[0]):
        for oy in range(O[1]):
            for ox in range(O[2]):
                for co in range(Co):
                    acc = b[co]
                    for kz in range(K):
                        for ky in range(K):
                            for kx in range(K):
                                iz, iy, ix = (stride * oz + kz - pad, stride * oy + ky - pad,
                                              stride * ox + kx - pad)
                                if 0 <= iz < Dz and 0 <= iy < Dy and 0 <= ix < Dx:
                                    for ci in range(Ci):
                                        acc += W[co, kz, ky, kx, ci] * x[iz, iy, ix, ci]
                    y[oz, oy, ox, co] = acc
    return y


@pytest.mark.parametrize("shape,ci,co,k,s", [((5, 4, 3), 2, 3, 3, 1), ((5, 4, 3), 2, 3, 3, 2),
                                             ((4, 6, 5), 3, 2, 1, 1), ((7, 3, 2), 1, 2, 3, 2)])
def test_conv_matches_brute_force(shape, ci, co, k, s):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((*shape, ci))
    W = rng.standard_normal((co, k, k, k, ci))
    b = rng.standard_normal(co)
    np.testing.assert_allclose(net.conv3d(x, W, b, s), _brute_conv(x, W, b, s), rtol=1e-12,
                               atol=1e-12)


def test_conv_matches_scipy_correlate():
    """Stride 1, 3x3x3 = sum over input channels of zero-padded 3D correlations; stride 2 is
    its subsample at even indices."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 5, 7, 3))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = np.zeros((6, 5, 7, 4))
    for co in range(4):
        ref[..., co] = b[co] + sum(
            scipy.ndimage.correlate(x[..., c], W[co, ..., c], mode="constant", cval=0.0)
            for c in range(3))
    np.testing.assert_allclose(net.conv3d(x, W, b, 1), ref, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(net.conv3d(x, W, b, 2), ref[::2, ::2, ::2], rtol=1e-11,
                               atol=1e-11)


@pytest.mark.parametrize("k,s", [(3, 1), (3, 2), (1, 1)])
def test_conv_backward_is_adjoint(k, s):
    """<conv(x), y> = <x, conv^T(y)> and <conv_W(x), y> = <W, dW(x, y)> (zero bias);
    db is the sum of y."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 6, 3, 4))
    W = rng.standard_normal((3, k, k, k, 4))
    z = np.zeros(3)
    y0 = net.conv3d(x, W, z, s)
    dy = rng.standard_normal(y0.shape)
    dx, dW, db = net.conv3d_backward(x, W, s, dy)
    assert abs((y0 * dy).sum() - (x * dx).sum()) < 1e-10 * abs((y0 * dy).sum())
    assert abs((y0 * dy).sum() - (W * dW).sum()) < 1e-10 * abs((y0 * dy).sum())
    np.testing.assert_allclose(db, dy.reshape(-1, 3).sum(0), rtol=1e-13)


def test_layernorm_matches_torch_and_invariants():
    rng = np.random.default_rng(4)
    z = rng.standard_normal((3, 4, 5, 6)) * 2 + 1
    g, bta = rng.standard_normal(6), rng.standard_normal(6)
    y, (xh, rstd) = net.layernorm(z, g, bta)
    ref = torch.nn.functional.layer_norm(torch.from_numpy(z), (6,), torch.from_numpy(g),
                                         torch.from_numpy(bta), eps=1e-5).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(xh.mean(-1), 0, atol=1e-13)
    var = z.var(-1)
    np.testing.assert_allclose((xh ** 2).mean(-1), var / (var + 1e-5), rtol=1e-12)


def test_layernorm_backward_finite_difference():
    rng = np.random.default_rng(5)
    z = rng.standard_normal((2, 3, 2, 5))
    g, bta = rng.standard_normal(5), rng.standard_normal(5)
    dy = rng.standard_normal(z.shape)
    _, cache = net.layernorm(z, g, bta)
    dz, dg, db = net.layernorm_backward(dy, cache, g)
    h = 1e-6
    for arr, grad in ((z, dz), (g, dg), (bta, db)):
        d = rng.standard_normal(arr.shape)
        arr += h * d
        fp = (net.layernorm(z, g, bta)[0] * dy).sum()
        arr -= 2 * h * d
        fm = (net.layernorm(z, g, bta)[0] * dy).sum()
        arr += h * d
        fd = (fp - fm) / (2 * h)
        assert abs(fd - (grad * d).sum()) < 1e-7 * max(1.0, abs(fd))


def test_lrelu():
    t = np.array([-2.0, -0.0, 0.0, 3.0])
    np.testing.assert_array_equal(net.lrelu(t), [-0.4, 0.0, 0.0, 3.0])
    np.testing.assert_array_equal(net.lrelu_backward(np.ones(4), t), [0.2, 0.2, 0.2, 1.0])


@pytest.mark.parametrize("sin,sout", [((3, 4, 2), (6, 8, 4)), ((2, 3, 4), (3, 5, 7)),
                                      ((1, 2, 3), (2, 3, 5))])
def test_upsample_matches_torch(sin, sout):
    rng = np.random.default_rng(6)
    u = rng.standard_normal((*sin, 3))
    ref = torch.nn.functional.interpolate(
        torch.from_numpy(u).permute(3, 0, 1, 2)[None], size=sout, mode="trilinear",
        align_corners=False)[0].permute(1, 2, 3, 0).numpy()
    np.testing.assert_allclose(net.upsample(u, sout), ref, rtol=1e-12, atol=1e-12)


def test_upsample_index_maps_and_fields():
    i0, i1, w = net.up_axis_map(4, 8)
    np.testing.assert_array_equal(i0, [0, 0, 0, 1, 1, 2, 2, 3])
    np.testing.assert_array_equal(i1, [1, 1, 1, 2, 2, 3, 3, 3])
    np.testing.assert_array_equal(w, [0.0, 0.25, 0.75, 0.25, 0.75, 0.25, 0.75, 0.25])
    # a constant field is reproduced exactly
    c = np.full((3, 2, 4, 2), 1.75)
    np.testing.assert_array_equal(net.upsample(c, (6, 4, 8)), np.full((6, 4, 8, 2), 1.75))
    # a field linear in x is reproduced exactly away from the clamped borders
    x = np.arange(5, dtype=np.float64)
    lin = np.broadcast_to(x[None, None, :, None], (2, 2, 5, 1)).copy()
    out = net.upsample(lin, (4, 4, 10))
    xo = (np.arange(10) + 0.5) / 2 - 0.5
    np.testing.assert_allclose(out[0, 0, 1:9, 0], xo[1:9], rtol=0, atol=1e-15)


def test_upsample_backward_is_adjoint():
    rng = np.random.default_rng(7)
    for sin, sout in (((3, 2, 4), (6, 4, 8)), ((3, 3, 2), (5, 6, 3))):
        u = rng.standard_normal((*sin, 2))
        dy = rng.standard_normal((*sout, 2))
        lhs = (net.upsample(u, sout) * dy).sum()
        rhs = (u * net.upsample_backward(dy, sin)).sum()
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
