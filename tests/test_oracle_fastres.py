"""Pins of the paper-form 3D-FastResUNet oracle (Sec. III-D, flagged variant).

The primitives are checked against NumPy loops and the independently pinned NumPy oracle of
the residual U-Net; the blocks against closed forms on inputs that make them constant; the
gradient against central finite differences of the whole network; the layout against a
count worked out by hand.
"""
import numpy as np
import pytest
import torch

from oracle import fastres as fr
from oracle import network as onet

R = np.random.default_rng(7)


def t5(x):
    """(Dz, Dy, Dx, C) NumPy -> (1, C, Dz, Dy, Dx) tensor."""
    return torch.as_tensor(x).permute(3, 0, 1, 2).unsqueeze(0)


def n4(t):
    return t[0].permute(1, 2, 3, 0).detach().numpy()


def brute_depthwise(x, W, b, s, d):
    Dz, Dy, Dx, C = x.shape
    O = [(v - 1) // s + 1 for v in (Dz, Dy, Dx)]
    y = np.zeros((*O, C))
    for oz in range(O[0]):
        for oy in range(O[1]):
            for ox in range(O[2]):
                for c in range(C):
                    acc = b[c]
                    for kz in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                iz, iy, ix = (s * oz + d * (kz - 1), s * oy + d * (ky - 1),
                                              s * ox + d * (kx - 1))
                                if 0 <= iz < Dz and 0 <= iy < Dy and 0 <= ix < Dx:
                                    acc += W[c, kz, ky, kx] * x[iz, iy, ix, c]
                    y[oz, oy, ox, c] = acc
    return y


@pytest.mark.parametrize("s,d", [(1, 1), (2, 1), (1, 2), (1, 3), (2, 2)])
def test_depthwise_matches_brute_force(s, d):
    x = R.normal(size=(5, 4, 7, 3))
    W = R.normal(size=(3, 3, 3, 3))
    b = R.normal(size=3)
    P = {"q.W": torch.as_tensor(W), "q.b": torch.as_tensor(b)}
    got = n4(fr.depthwise(P, "q", t5(x), s, d))
    np.testing.assert_allclose(got, brute_depthwise(x, W, b, s, d), rtol=1e-12, atol=1e-12)


def test_depthwise_is_dense_with_diagonal_weights():
    x = R.normal(size=(4, 6, 5, 4))
    W = R.normal(size=(4, 3, 3, 3))
    b = R.normal(size=4)
    Wd = np.zeros((4, 3, 3, 3, 4))
    for c in range(4):
        Wd[c, ..., c] = W[c]
    P = {"q.W": torch.as_tensor(W), "q.b": torch.as_tensor(b)}
    for s in (1, 2):
        np.testing.assert_allclose(n4(fr.depthwise(P, "q", t5(x), s)),
                                   onet.conv3d(x, Wd, b, s), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k,s", [(3, 1), (3, 2), (1, 1), (1, 2)])
def test_dense_matches_numpy_conv(k, s):
    x = R.normal(size=(5, 6, 3, 4))
    W = R.normal(size=(3, k, k, k, 4))
    b = R.normal(size=3)
    P = {"q.W": torch.as_tensor(W), "q.b": torch.as_tensor(b)}
    np.testing.assert_allclose(n4(fr.dense(P, "q", t5(x), s)), onet.conv3d(x, W, b, s),
                               rtol=1e-12, atol=1e-12)


def test_layernorm_and_up_match_numpy_oracle():
    z = R.normal(size=(3, 4, 5, 6))
    g, beta = R.normal(size=6), R.normal(size=6)
    P = {"n.g": torch.as_tensor(g), "n.beta": torch.as_tensor(beta)}
    np.testing.assert_allclose(n4(fr.layernorm(P, "n", t5(z))), onet.layernorm(z, g, beta)[0],
                               rtol=1e-12, atol=1e-12)
    u = R.normal(size=(2, 3, 3, 2))
    np.testing.assert_allclose(n4(fr.up(t5(u), (3, 5, 6))), onet.upsample(u, (3, 5, 6)),
                               rtol=1e-12, atol=1e-12)


def sig(t):
    return 1.0 / (1.0 + np.exp(-t))


def test_se_on_channel_constant_input():
    C, h = 8, fr.se_hidden(8)
    v = R.normal(size=C)
    x = np.broadcast_to(v, (3, 4, 5, C)).copy()
    W1, b1 = R.normal(size=(h, 1, 1, 1, C)), R.normal(size=h)
    W2, b2 = R.normal(size=(C, 1, 1, 1, h)), R.normal(size=C)
    P = {k: torch.as_tensor(a) for k, a in
         {"s.fc1.W": W1, "s.fc1.b": b1, "s.fc2.W": W2, "s.fc2.b": b2}.items()}
    scale = sig(W2.reshape(C, h) @ np.maximum(W1.reshape(h, C) @ v + b1, 0) + b2)
    np.testing.assert_allclose(n4(fr.se(P, "s", t5(x))), x * scale, rtol=1e-12)


def test_gate_with_zero_projections():
    cx, cg = 6, 4
    f = fr.gate_inner(cx)
    x = R.normal(size=(4, 4, 6, cx))
    g = R.normal(size=(2, 2, 3, cg))
    bx, bg, wp, bp = R.normal(size=f), R.normal(size=f), R.normal(size=f), 0.3
    P = {"a.x.W": np.zeros((f, 1, 1, 1, cx)), "a.x.b": bx, "a.g.W": np.zeros((f, 1, 1, 1, cg)),
         "a.g.b": bg, "a.psi.W": wp.reshape(1, 1, 1, 1, f), "a.psi.b": np.array([bp])}
    P = {k: torch.as_tensor(a) for k, a in P.items()}
    psi = sig(wp @ np.maximum(bx + bg, 0) + bp)
    np.testing.assert_allclose(n4(fr.gate(P, "a", t5(x), t5(g))), x * psi, rtol=1e-12)


def test_aspp_closed_form_on_constant_branches():
    """Zero depthwise weights make every tensor constant over the voxels, so the ASPP output
    is act(LN(proj([b0, b1, b2, b3]))) of per-branch vectors (concat order pinned)."""
    C = 8
    cb = fr.aspp_branch(C)
    spec_names = [e for e in fr._aspp("p", C)]
    P = {}
    for name, shape, kind, fan, in spec_names:
        a = R.normal(size=shape)
        if name.endswith(".dw.W"):
            a = np.zeros(shape)
        P[name] = a
    x = R.normal(size=(4, 6, 5, C))
    Pt = {k: torch.as_tensor(a) for k, a in P.items()}
    got = n4(fr.aspp(Pt, "p", t5(x)))

    def lr(t):
        return np.where(t > 0, t, 0.2 * t)

    def pw(name, v):
        W = P[name + ".W"]
        return W.reshape(W.shape[0], -1) @ v + P[name + ".b"]

    def ln(name, z):
        mu, var = z.mean(), z.var()
        return (z - mu) / np.sqrt(var + 1e-5) * P[name + ".g"] + P[name + ".beta"]

    d = lr(ln("p.down.ln", pw("p.down.pw", P["p.down.dw.b"])))
    b0 = lr(pw("p.b0", d))
    b1 = lr(pw("p.b1.pw", P["p.b1.dw.b"]))
    b2 = lr(pw("p.b2.pw", P["p.b2.dw.b"]))
    b3 = lr(pw("p.b3", d))
    want = lr(ln("p.ln", pw("p.proj", np.concatenate([b0, b1, b2, b3]))))
    assert got.shape == (2, 3, 3, C) and cb * 4 == P["p.proj.W"].shape[-1]
    np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=1e-10, atol=1e-12)


SMALL = fr.FastSpec((5, 6, 4), 2, (4, 8), 2)


def test_layout_count_by_hand_and_contiguous():
    lay = fr.param_layout(SMALL)
    assert fr.param_count(SMALL) == 3859   # worked out module by module
    off = 0
    for name, shape, kind, fan, o, cnt in lay:
        assert o == off and cnt == int(np.prod(shape))
        off += cnt
    assert lay[0][0] == "stem.W" and lay[-1][0] == "tail.b"
    names = [e[0] for e in lay]
    assert names.index("se1.fc1.W") < names.index("enc1.a.dw.W") < names.index("aspp.down.dw.W")
    assert names.index("att1.x.W") < names.index("dec1.a.dw.W") < names.index("att0.x.W")
    assert "enc0.p.W" not in names and "enc1.p.W" in names


def _theta(spec, seed):
    rng = np.random.default_rng(seed)
    th = np.zeros(fr.param_count(spec))
    for name, shape, kind, fan, o, cnt in fr.param_layout(spec):
        if kind == onet.KIND_CONV_W:
            th[o:o + cnt] = rng.normal(size=cnt) * np.sqrt(2.0 / fan)
        elif kind == onet.KIND_LN_G:
            th[o:o + cnt] = 1.0 + 0.1 * rng.normal(size=cnt)
        else:
            th[o:o + cnt] = 0.1 * rng.normal(size=cnt)
    return th


def test_tail_closed_form_and_output_range():
    th = _theta(SMALL, 1)
    Z = R.normal(size=(120, 2))
    out = fr.forward(SMALL, th, Z)
    assert np.all((out > 0) & (out < 1))
    lay = {e[0]: e for e in fr.param_layout(SMALL)}
    o = lay["tail.W"][4]
    th[o:o + lay["tail.W"][5]] = 0.0
    th[lay["tail.b"][4]] = 0.7
    np.testing.assert_allclose(fr.forward(SMALL, th, Z), sig(0.7), rtol=1e-14)


def test_gradient_matches_finite_differences():
    th = _theta(SMALL, 2)
    Z = R.normal(size=(120, 2))
    w = R.normal(size=120)
    out, kept = fr.forward(SMALL, th, Z, keep=True)
    g = fr.backward(SMALL, kept, w)
    for k in range(3):
        d = R.normal(size=th.size)
        h = 1e-7   # the truncation error is O(h^2) with large third derivatives (sigmoids)
        fp = w @ fr.forward(SMALL, th + h * d, Z)
        fm = w @ fr.forward(SMALL, th - h * d, Z)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)


def test_dip_step_uses_the_variant():
    from oracle import dip
    th = _theta(SMALL, 3)
    Z = R.normal(size=(120, 2))
    J = R.normal(size=(16, 120))
    Jn, _ = dip.normalise_columns(J)
    dv = R.normal(size=16)
    st = dip.AdamState.fresh(th.size)
    res = dip.dip_step(SMALL, Jn, Z, dv, th, st, 1e-3)
    ds = fr.forward(SMALL, th, Z)
    np.testing.assert_array_equal(res.dsigma, ds)
    r = Jn @ ds - dv
    assert res.loss == pytest.approx(r @ r / 16, rel=1e-14)


@pytest.mark.parametrize("grid,L,widths", [((4, 3, 5), 1, (8,)), ((6, 5, 4), 3, (8, 16, 16))])
def test_gradient_matches_finite_differences_other_depths(grid, L, widths):
    """One stage (the bottleneck one level below the stem's) and three stages (levels down to
    one voxel): the gradient is the derivative of the forward at these depths too."""
    spec = fr.FastSpec(grid, L, widths, 2)
    th = _theta(spec, 4)
    n = grid[0] * grid[1] * grid[2]
    Z = R.normal(size=(n, 2))
    w = R.normal(size=n)
    out, kept = fr.forward(spec, th, Z, keep=True)
    assert out.shape == (n,) and np.all((out > 0) & (out < 1))
    g = fr.backward(spec, kept, w)
    d = R.normal(size=th.size)
    h = 1e-7
    fd = (w @ fr.forward(spec, th + h * d, Z) - w @ fr.forward(spec, th - h * d, Z)) / (2 * h)
    assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))
    names = [e[0] for e in fr.param_layout(spec)]
    assert sum(nm.endswith(".a.dw.W") for nm in names) == 2 * L   # L encoder + L decoder blocks
    assert sum(nm.endswith(".psi.W") for nm in names) == L
