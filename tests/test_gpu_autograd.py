"""The torch.autograd.Function wrappers (paper_2507_14046_gb300.autograd): every op's
hand-written backward kernel, reached through torch.autograd, against finite differences
and against the FP64 oracle's gradient; and a stem block (conv -> LayerNorm -> LeakyReLU)
composed by autograd against the oracle's backward of the same block.

Finite differences: the convolution, the up-sampling and the J product are linear in each
argument, so a central difference with a unit step is exact up to rounding; LayerNorm
without the activation is smooth and is checked with a small step in FP32 at a looser bar
(with LeakyReLU the comparison with the oracle's backward stands alone).
"""
import numpy as np
import pytest

from oracle import network as onet
from tests.problems import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _fd(f, args, i, d, h):
    """Central difference of f along direction d in argument i (FP32 evaluation, FP64 sum)."""
    ap = list(args)
    am = list(args)
    ap[i] = args[i] + h * d
    am[i] = args[i] - h * d
    with torch.no_grad():
        return (f(*ap).double().sum().item() - f(*am).double().sum().item()) / (2 * h)


@pytest.mark.parametrize("din,ci,co,k,s,tc", [((6, 7, 9), 8, 16, 3, 1, False),
                                              ((7, 5, 6), 16, 8, 3, 2, False),
                                              ((5, 6, 4), 24, 16, 1, 1, False),
                                              ((8, 8, 12), 16, 16, 3, 1, True),
                                              ((6, 10, 8), 32, 16, 3, 1, True)])
def test_conv3d_function(d2ip, din, ci, co, k, s, tc):
    from paper_2507_14046_gb300 import autograd as AG
    rng = np.random.default_rng(ci * 7 + co + k + s)
    B = 2
    x = rng.standard_normal((B, *din, ci)).astype(np.float32)
    blk = co * k ** 3 * ci + co
    wb = (rng.standard_normal((B, blk)) * 0.2).astype(np.float32)
    if tc:  # the tensor-core form rounds x and W to BF16: compare on BF16-exact values
        x = torch.from_numpy(x).bfloat16().float().numpy()
        wb[:, :blk - co] = torch.from_numpy(wb[:, :blk - co]).bfloat16().float().numpy()
    X = _dev(x).requires_grad_()
    Wb = _dev(wb).requires_grad_()
    y = AG.conv3d(X, Wb, co, k, s, tc)
    w = rng.standard_normal(tuple(y.shape)).astype(np.float32)
    if tc:
        w = torch.from_numpy(w).bfloat16().float().numpy()
    (y * _dev(w)).sum().backward()
    tol = 1e-4 if tc else 1e-5
    for b in range(B):
        W = wb[b, :blk - co].reshape(co, k, k, k, ci).astype(np.float64)
        ry = onet.conv3d(x[b].astype(np.float64), W, wb[b, blk - co:].astype(np.float64), s)
        assert rel(y[b].detach().cpu().numpy(), ry) < tol
        gx, gW, gb = onet.conv3d_backward(x[b].astype(np.float64), W, s, w[b].astype(np.float64))
        assert rel(X.grad[b].cpu().numpy(), gx) < tol
        assert rel(Wb.grad[b, :blk - co].cpu().numpy(), gW.reshape(-1)) < tol
        assert rel(Wb.grad[b, blk - co:].cpu().numpy(), gb) < tol
    if not tc:  # linear in each argument: unit-step central differences are exact
        f = lambda a, bb: (AG.conv3d(a, bb, co, k, s) * _dev(w))  # noqa: E731
        for i, g in ((0, X.grad), (1, Wb.grad)):
            d = torch.randn_like(g)
            fd = _fd(f, (X.detach(), Wb.detach()), i, d, 1.0)
            assert abs(fd - (g.double() * d.double()).sum().item()) <= 1e-4 * max(1.0, abs(fd))


@pytest.mark.parametrize("c,resid,act", [(16, False, 1), (32, True, 1), (8, True, 0)])
def test_layernorm_act_function(d2ip, c, resid, act):
    from paper_2507_14046_gb300 import autograd as AG
    rng = np.random.default_rng(c + resid + act)
    B, d = 2, (5, 6, 7)
    z = rng.standard_normal((B, *d, c)).astype(np.float32)
    gb = np.concatenate([1 + 0.3 * rng.standard_normal((B, c)), 0.3 * rng.standard_normal((B, c))],
                        axis=1).astype(np.float32)
    t = rng.standard_normal((B, *d, c)).astype(np.float32) if resid else None
    Z = _dev(z).requires_grad_()
    G = _dev(gb).requires_grad_()
    T = _dev(t).requires_grad_() if resid else None
    y = AG.layernorm_act(Z, G, T, act)
    w = rng.standard_normal(tuple(y.shape)).astype(np.float32)
    (y * _dev(w)).sum().backward()
    for b in range(B):
        g, beta = gb[b, :c].astype(np.float64), gb[b, c:].astype(np.float64)
        pre, cache = onet.layernorm(z[b].astype(np.float64), g, beta)
        if resid:
            pre = pre + t[b]
        ry = onet.lrelu(pre) if act else pre
        assert rel(y[b].detach().cpu().numpy(), ry) < 1e-5
        dpre = onet.lrelu_backward(w[b].astype(np.float64), pre) if act else w[b].astype(np.float64)
        dz, dg, dbeta = onet.layernorm_backward(dpre, cache, g)
        assert rel(Z.grad[b].cpu().numpy(), dz) < 1e-5
        assert rel(G.grad[b, :c].cpu().numpy(), dg) < 1e-5
        assert rel(G.grad[b, c:].cpu().numpy(), dbeta) < 1e-5
        if resid:
            assert rel(T.grad[b].cpu().numpy(), dpre) < 1e-5
    if act:  # a finite difference across LeakyReLU kinks measures the step, not the gradient
        return
    f = lambda a, gg: AG.layernorm_act(a, gg, T.detach() if resid else None, act) * _dev(w)  # noqa
    for i, g in ((0, Z.grad), (1, G.grad)):
        d = torch.randn_like(g)
        fd = _fd(f, (Z.detach(), G.detach()), i, d, 1e-2)
        assert abs(fd - (g.double() * d.double()).sum().item()) <= 2e-2 * max(1.0, abs(fd))


@pytest.mark.parametrize("low,out,cu,cs", [((3, 4, 5), (6, 8, 10), 8, 4), ((3, 2, 4), (5, 4, 7), 4, 0)])
def test_upsample_concat_function(d2ip, low, out, cu, cs):
    from paper_2507_14046_gb300 import autograd as AG
    rng = np.random.default_rng(cu + cs)
    B = 2
    u = rng.standard_normal((B, *low, cu)).astype(np.float32)
    sk = rng.standard_normal((B, *out, cs)).astype(np.float32) if cs else None
    U = _dev(u).requires_grad_()
    S = _dev(sk).requires_grad_() if cs else None
    cat = AG.upsample_concat(U, S, out)
    w = rng.standard_normal(tuple(cat.shape)).astype(np.float32)
    (cat * _dev(w)).sum().backward()
    for b in range(B):
        ref = onet.upsample_backward(w[b, ..., :cu].astype(np.float64), low)
        assert rel(U.grad[b].cpu().numpy(), ref) < 1e-5
        if cs:
            np.testing.assert_array_equal(S.grad[b].cpu().numpy(), w[b, ..., cu:])
    f = lambda a: AG.upsample_concat(a, S.detach() if cs else None, out) * _dev(w)  # noqa
    d = torch.randn_like(U)
    fd = _fd(f, (U.detach(),), 0, d, 1.0)
    assert abs(fd - (U.grad.double() * d.double()).sum().item()) <= 1e-4 * max(1.0, abs(fd))


def test_sensitivity_residual_function(d2ip):
    from paper_2507_14046_gb300 import autograd as AG
    rng = np.random.default_rng(3)
    m, n, B = 208, 2048, 3
    J = _dev(rng.standard_normal((m, n)))
    x = _dev(rng.standard_normal((B, n))).requires_grad_()
    dv = _dev(rng.standard_normal((B, m)))
    r = AG.sensitivity_residual(J, x, dv)
    w = rng.standard_normal((B, m)).astype(np.float32)
    (r * _dev(w)).sum().backward()
    Jn = J.double().cpu().numpy()
    assert rel(r.detach().cpu().numpy(),
               x.detach().double().cpu().numpy() @ Jn.T - dv.double().cpu().numpy()) < 1e-5
    assert rel(x.grad.cpu().numpy(), w.astype(np.float64) @ Jn) < 1e-5


def test_stem_block_composed_by_autograd(d2ip):
    """act(LN(conv3(Z))) built from the Functions; torch.autograd's gradient of <w, y> with
    respect to the conv and LayerNorm parameters equals the oracle's hand-written backward."""
    from paper_2507_14046_gb300 import autograd as AG
    rng = np.random.default_rng(11)
    d, ci, co = (8, 8, 8), 8, 16
    z = (0.1 * rng.standard_normal((1, *d, ci))).astype(np.float32)
    blk = co * 27 * ci + co
    wb = (rng.standard_normal((1, blk)) * np.sqrt(2.0 / (27 * ci))).astype(np.float32)
    gb = np.concatenate([np.ones((1, co)), np.zeros((1, co))], axis=1).astype(np.float32)
    Wb, G = _dev(wb).requires_grad_(), _dev(gb).requires_grad_()
    y = AG.layernorm_act(AG.conv3d(_dev(z), Wb, co, 3, 1), G, None, 1)
    w = rng.standard_normal(tuple(y.shape)).astype(np.float32)
    (y * _dev(w)).sum().backward()
    P = {"s.W": wb[0, :blk - co].reshape(co, 3, 3, 3, ci).astype(np.float64),
         "s.b": wb[0, blk - co:].astype(np.float64), "n.g": np.ones(co), "n.beta": np.zeros(co)}
    out, cache = onet._conv_ln_act_fwd(P, "s", "n", z[0].astype(np.float64), 1)
    assert rel(y[0].detach().cpu().numpy(), out) < 1e-5
    Gd = {}
    onet._conv_ln_act_bwd(P, Gd, "s", "n", 1, cache, w[0].astype(np.float64))
    assert rel(Wb.grad[0, :blk - co].cpu().numpy(), Gd["s.W"].reshape(-1)) < 1e-5
    assert rel(Wb.grad[0, blk - co:].cpu().numpy(), Gd["s.b"]) < 1e-5
    assert rel(G.grad[0, :co].cpu().numpy(), Gd["n.g"]) < 1e-5
    assert rel(G.grad[0, co:].cpu().numpy(), Gd["n.beta"]) < 1e-5
