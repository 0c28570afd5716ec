"""Per-op parity of the CUDA kernels (called through the C ABI) against the FP64 oracle.

Bar: norm-wise relative error <= 1e-5 for FP32 arithmetic; index work (resampling maps)
is checked through exact special cases.  Shapes span several tiles and ragged tails.
"""
import numpy as np
import pytest

from oracle import dip, network as onet
from tests.problems import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _stream():
    return torch.cuda.current_stream().cuda_stream


CONV_CASES = [((9, 7, 11), 8, 16, 3, 1), ((9, 7, 11), 16, 32, 3, 2), ((5, 6, 7), 24, 8, 1, 1),
              ((8, 16, 16), 8, 8, 3, 1), ((4, 4, 4), 64, 64, 3, 1), ((7, 5, 3), 48, 16, 3, 1),
              ((6, 9, 5), 32, 64, 3, 2), ((3, 3, 3), 96, 32, 1, 1), ((16, 32, 32), 16, 1, 1, 1),
              ((8, 8, 8), 128, 128, 3, 1)]


@pytest.mark.parametrize("din,ci,co,k,s", CONV_CASES)
def test_conv_forward_dgrad_wgrad(d2ip, din, ci, co, k, s):
    rng = np.random.default_rng(hash((din, ci, co, k, s)) % 2**32)
    B = 2
    x = rng.standard_normal((B, *din, ci)).astype(np.float32)
    blk = co * k ** 3 * ci + co
    wb = (rng.standard_normal((B, blk)) * 0.2).astype(np.float32)
    W = [wb[b, :co * k ** 3 * ci].reshape(co, k, k, k, ci).astype(np.float64) for b in range(B)]
    bias = [wb[b, co * k ** 3 * ci:].astype(np.float64) for b in range(B)]
    ref = [onet.conv3d(x[b].astype(np.float64), W[b], bias[b], s) for b in range(B)]
    dout = ref[0].shape[:3]
    xd, wd = _dev(x), _dev(wb)
    y = torch.zeros((B, *dout, co), device="cuda")
    # weights and bias of problem b sit at b * blk (w_batch_stride = blk)
    d2ip.d2ip_conv3d_forward(xd, wd, int(wd.data_ptr()) + 4 * co * k ** 3 * ci, y, B, *din, ci,
                             co, k, s, blk, _stream())
    torch.cuda.synchronize()
    for b in range(B):
        assert rel(y[b].cpu().numpy(), ref[b]) < TOL
    # backward
    dy = rng.standard_normal((B, *dout, co)).astype(np.float32)
    grads = [onet.conv3d_backward(x[b].astype(np.float64), W[b], s, dy[b].astype(np.float64))
             for b in range(B)]
    dyd = _dev(dy)
    dx = torch.zeros_like(xd)
    d2ip.d2ip_conv3d_dgrad(dyd, wd, dx, B, *din, ci, co, k, s, blk, 0, _stream())
    ws_bytes = d2ip.d2ip_conv3d_wgrad_workspace(B, *din, ci, co, k, s)
    ws = torch.empty(ws_bytes // 4 + 1, device="cuda")
    dW = torch.zeros((B, blk), device="cuda")
    d2ip.d2ip_conv3d_wgrad(xd, dyd, dW, B, *din, ci, co, k, s, blk, 0, ws, ws_bytes, _stream())
    torch.cuda.synchronize()
    for b in range(B):
        gdx, gdW, gdb = grads[b]
        assert rel(dx[b].cpu().numpy(), gdx) < TOL
        assert rel(dW[b, :co * k ** 3 * ci].cpu().numpy(), gdW.reshape(-1)) < TOL
        assert rel(dW[b, co * k ** 3 * ci:].cpu().numpy(), gdb) < TOL
    # accumulate mode adds
    d2ip.d2ip_conv3d_dgrad(dyd, wd, dx, B, *din, ci, co, k, s, blk, 1, _stream())
    torch.cuda.synchronize()
    assert rel(dx[0].cpu().numpy(), 2 * grads[0][0]) < TOL


@pytest.mark.parametrize("nvox,c,resid", [(1000, 8, False), (777, 16, True), (513, 32, True),
                                          (300, 64, False), (129, 128, True), (2048, 24, True)])
def test_layernorm_act_forward_backward(d2ip, nvox, c, resid):
    rng = np.random.default_rng(nvox + c)
    B = 2
    z = (rng.standard_normal((B, nvox, c)) * 1.5 + 0.3).astype(np.float32)
    gb = np.concatenate([1 + 0.3 * rng.standard_normal((B, c)), 0.2 * rng.standard_normal((B, c))],
                        axis=1).astype(np.float32)
    r = rng.standard_normal((B, nvox, c)).astype(np.float32) if resid else None
    zd, gbd = _dev(z), _dev(gb)
    rd = _dev(r) if resid else None
    y, xh = torch.zeros_like(zd), torch.zeros_like(zd)
    rs = torch.zeros((B, nvox), device="cuda")
    d2ip.d2ip_layernorm_act_forward(zd, gbd, rd, y, xh, rs, B, nvox, c, 1, 2 * c, _stream())
    dy = rng.standard_normal((B, nvox, c)).astype(np.float32)
    dyd = _dev(dy)
    dz, dt = torch.zeros_like(zd), torch.zeros_like(zd)
    dgb = torch.zeros((B, 2 * c), device="cuda")
    wsb = d2ip.d2ip_layernorm_workspace(B, nvox, c)
    ws = torch.empty(wsb // 4 + 1, device="cuda")
    d2ip.d2ip_layernorm_act_backward(dyd, y, xh, rs, gbd, dz, dt, dgb, B, nvox, c, 2 * c, 0, ws,
                                     wsb, _stream())
    torch.cuda.synchronize()
    for b in range(B):
        g, be = gb[b, :c].astype(np.float64), gb[b, c:].astype(np.float64)
        lnout, cache = onet.layernorm(z[b].astype(np.float64), g, be)
        t = lnout + (r[b] if resid else 0.0)
        assert rel(y[b].cpu().numpy(), onet.lrelu(t)) < TOL
        assert rel(xh[b].cpu().numpy(), cache[0]) < TOL
        dpre = onet.lrelu_backward(dy[b].astype(np.float64), t)
        rdz, rdg, rdb = onet.layernorm_backward(dpre, cache, g)
        assert rel(dt[b].cpu().numpy(), dpre) < TOL
        assert rel(dz[b].cpu().numpy(), rdz) < TOL
        assert rel(dgb[b, :c].cpu().numpy(), rdg) < TOL
        assert rel(dgb[b, c:].cpu().numpy(), rdb) < TOL


@pytest.mark.parametrize("low,out,cu,cs", [((4, 8, 8), (8, 16, 16), 16, 8),
                                           ((3, 2, 4), (5, 4, 7), 8, 4),
                                           ((1, 2, 3), (2, 3, 5), 4, 0),
                                           ((16, 32, 32), (32, 64, 64), 32, 16),
                                           ((1, 3, 5), (2, 6, 10), 8, 8),
                                           ((3, 5, 7), (6, 10, 14), 12, 0)])
def test_upsample_concat(d2ip, low, out, cu, cs):
    rng = np.random.default_rng(sum(low))
    B = 2
    u = rng.standard_normal((B, *low, cu)).astype(np.float32)
    sk = rng.standard_normal((B, *out, cs)).astype(np.float32)
    cat = torch.zeros((B, *out, cu + cs), device="cuda")
    ud, skd = _dev(u), _dev(sk) if cs else None
    d2ip.d2ip_upsample_concat_forward(ud, skd, cat, B, *low, *out, cu, cs, _stream())
    dcat = rng.standard_normal((B, *out, cu + cs)).astype(np.float32)
    dl = torch.zeros_like(ud)
    ds = torch.zeros((B, *out, cs), device="cuda") if cs else None
    d2ip.d2ip_upsample_concat_backward(_dev(dcat), dl, ds, B, *low, *out, cu, cs, _stream())
    torch.cuda.synchronize()
    for b in range(B):
        ref = onet.upsample(u[b].astype(np.float64), out)
        c = cat[b].cpu().numpy()
        assert rel(c[..., :cu], ref) < TOL
        np.testing.assert_array_equal(c[..., cu:], sk[b])
        assert rel(dl[b].cpu().numpy(),
                   onet.upsample_backward(dcat[b, ..., :cu].astype(np.float64), low)) < TOL
        if cs:
            np.testing.assert_array_equal(ds[b].cpu().numpy(), dcat[b, ..., cu:])


def test_upsample_constant_field_exact(d2ip):
    u = np.full((1, 3, 4, 5, 4), 0.625, dtype=np.float32)
    cat = torch.zeros((1, 6, 8, 10, 4), device="cuda")
    d2ip.d2ip_upsample_concat_forward(_dev(u), None, cat, 1, 3, 4, 5, 6, 8, 10, 4, 0, _stream())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cat.cpu().numpy(), 0.625)


@pytest.mark.parametrize("m,n,B", [(208, 2048, 1), (416, 16384, 3), (624, 4999, 9),
                                   (416, 55296, 13), (3, 1030, 17)])
def test_sensitivity_products_and_normalisation(d2ip, m, n, B):
    rng = np.random.default_rng(m + n)
    J = rng.standard_normal((m, n)).astype(np.float32) * 3
    Jd = _dev(J)
    cn = torch.zeros(n, dtype=torch.float64, device="cuda")
    d2ip.d2ip_normalize_columns(Jd, cn, m, n, _stream())
    Jn, c = dip.normalise_columns(J)
    x = rng.standard_normal((B, n)).astype(np.float32)
    dv = rng.standard_normal((B, m)).astype(np.float32)
    r = torch.zeros((B, m), device="cuda")
    loss = torch.zeros(B, dtype=torch.float64, device="cuda")
    wsb = d2ip.d2ip_sensitivity_workspace(B, m, n)
    ws = torch.empty(wsb // 4 + 1, device="cuda")
    d2ip.d2ip_sensitivity_residual(Jd, _dev(x), _dev(dv), r, loss, B, m, n, ws, wsb, _stream())
    g = torch.zeros((B, n), device="cuda")
    d2ip.d2ip_sensitivity_adjoint(Jd, r, g, 2.0 / m, B, m, n, _stream())
    torch.cuda.synchronize()
    np.testing.assert_allclose(cn.cpu().numpy(), c, rtol=1e-12)
    assert rel(Jd.cpu().numpy(), Jn) < 1e-7
    for b in range(B):
        rr, L = dip.data_term(Jn, x[b].astype(np.float64), dv[b].astype(np.float64))
        assert rel(r[b].cpu().numpy(), rr) < TOL
        assert abs(loss[b].item() - L) <= TOL * L
        gref = dip.data_term_grad(Jn, r[b].cpu().numpy().astype(np.float64))
        assert rel(g[b].cpu().numpy(), gref) < TOL


def test_adam_matches_oracle(d2ip):
    rng = np.random.default_rng(3)
    n = 100003
    th = rng.standard_normal(n).astype(np.float32)
    st = dip.AdamState.fresh(n)
    thr = th.astype(np.float64)
    td, md, vd = _dev(th), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    for t in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        thr = dip.adam_step(thr, g.astype(np.float64), st, 1e-3)
        d2ip.d2ip_adam_update(td, _dev(g), md, vd, n, 1e-3, 0.9, 0.999, 1e-8, t, _stream())
    torch.cuda.synchronize()
    assert rel(td.cpu().numpy(), thr) < TOL
    assert rel(md.cpu().numpy(), st.m) < TOL
    assert rel(vd.cpu().numpy(), st.v) < TOL


def test_bad_arguments_are_rejected(d2ip):
    with pytest.raises(d2ip.D2IPError) as e:
        d2ip.d2ip_conv3d_forward(1, 1, 1, 1, 1, 4, 4, 4, 8, 8, 5, 1, 0, None)
    assert e.value.status == -2
    with pytest.raises(d2ip.D2IPError) as e:
        d2ip.d2ip_layernorm_act_forward(1, 1, None, 1, 1, 1, 1, 10, 6, 1, 0, None)
    assert e.value.status == -2
