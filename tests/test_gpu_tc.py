"""Parity of the tcgen05 (BF16 x BF16 -> FP32) implicit-GEMM convolution against the FP64
oracle evaluated on the same BF16-rounded inputs, so the only difference left is the FP32
accumulation order inside the tensor cores.  Shapes cover every channel chunk width
(16/32/64 channels -> 32/64/128-byte swizzle), several chunks per tap, stride 2, 1x1x1,
ragged grids and a batch of problems with their own weights."""
import numpy as np
import pytest

from oracle import network as onet
from tests.problems import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-4  # products of BF16 values are exact; FP32 accumulation order differs


def bf16_round(a):
    """Round float32 to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _faces(a):
    """The elements on the six outer faces of a (Z, Y, X, C) volume (the zero-padded halo)."""
    m = np.zeros(a.shape[:3], dtype=bool)
    m[0], m[-1] = True, True
    m[:, 0], m[:, -1] = True, True
    m[:, :, 0], m[:, :, -1] = True, True
    return a[m]


def _elementwise(got, ref):
    """Every element within TOL of the largest magnitude, and the outer faces on their own:
    a single wrong halo voxel cannot hide in a norm-wise error."""
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
    fg, fr = _faces(got), _faces(ref)
    assert np.abs(fg - fr).max() <= TOL * max(np.abs(fr).max(), 1e-30)


def _err_word(ws):
    base = ws.data_ptr()
    off = (-base) % 1024
    return int(ws.view(torch.uint8)[off:off + 4].view(torch.int32).item())


TC_CASES = [((16, 8, 8), 16, 16, 3, 1), ((7, 9, 11), 32, 16, 3, 1), ((4, 8, 8), 64, 64, 3, 1),
            ((6, 9, 5), 16, 32, 3, 2), ((16, 16, 8), 48, 16, 3, 1), ((8, 8, 8), 96, 32, 1, 1),
            ((8, 16, 16), 128, 128, 3, 1), ((5, 6, 7), 192, 64, 3, 1), ((8, 8, 8), 64, 128, 3, 2),
            ((16, 32, 32), 16, 32, 3, 2), ((9, 7, 11), 32, 64, 3, 2)]


@pytest.mark.parametrize("din,ci,co,k,s", TC_CASES)
def test_tc_conv_forward_and_dgrad(d2ip, din, ci, co, k, s):
    rng = np.random.default_rng(ci * 131 + co + s)
    B = 2
    stream = torch.cuda.current_stream().cuda_stream
    x = bf16_round(rng.standard_normal((B, *din, ci)).astype(np.float32))
    nw = co * k ** 3 * ci
    wb = (rng.standard_normal((B, nw + co)) * 0.1).astype(np.float32)
    wb[:, :nw] = bf16_round(wb[:, :nw])
    W = [wb[b, :nw].reshape(co, k, k, k, ci).astype(np.float64) for b in range(B)]
    bias = [wb[b, nw:].astype(np.float64) for b in range(B)]
    ref = [onet.conv3d(x[b].astype(np.float64), W[b], bias[b], s) for b in range(B)]
    dout = ref[0].shape[:3]
    wsb = d2ip.d2ip_conv3d_tc_workspace(B, *din, ci, co, k, s)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    xd, wd = _dev(x), _dev(wb)
    y = torch.zeros((B, *dout, co), device="cuda")
    d2ip.d2ip_conv3d_forward_tc(xd, wd, int(wd.data_ptr()) + 4 * nw, y, B, *din, ci, co, k, s,
                                nw + co, ws, wsb, stream)
    torch.cuda.synchronize()
    assert _err_word(ws) == 0
    errs = [rel(y[b].cpu().numpy(), ref[b]) for b in range(B)]
    print("tc forward rel err", errs)
    assert max(errs) < TOL
    for b in range(B):
        _elementwise(y[b].cpu().numpy(), ref[b])
    if k == 1 and s != 1:
        return
    dy = bf16_round(rng.standard_normal((B, *dout, co)).astype(np.float32))
    dx = torch.zeros_like(xd)
    wsb2 = d2ip.d2ip_conv3d_tc_workspace(B, *din, ci, co, k, s)
    d2ip.d2ip_conv3d_dgrad_tc(_dev(dy), wd, dx, B, *din, ci, co, k, s, nw + co, 0, ws, wsb2,
                              stream)
    torch.cuda.synchronize()
    assert _err_word(ws) == 0
    for b in range(B):
        gdx = onet.conv3d_backward(x[b].astype(np.float64), W[b], s, dy[b].astype(np.float64))[0]
        assert rel(dx[b].cpu().numpy(), gdx) < TOL
        _elementwise(dx[b].cpu().numpy(), gdx)


def test_tc_rejects_unsupported_shapes(d2ip):
    assert d2ip.d2ip_conv3d_tc_workspace(1, 4, 4, 4, 8, 16, 3, 1) == -1
    with pytest.raises(d2ip.D2IPError) as e:
        d2ip.d2ip_conv3d_dgrad_tc(1, 1, 1, 1, 4, 4, 4, 16, 24, 3, 1, 0, 0, 1, 1 << 20, None)
    assert e.value.status == -2


WG_CASES = [((16, 8, 8), 16, 16, 3), ((7, 9, 11), 32, 16, 3), ((4, 8, 8), 64, 64, 3),
            ((16, 16, 8), 48, 16, 3), ((8, 16, 16), 16, 32, 3), ((5, 6, 7), 192, 64, 3),
            ((8, 8, 8), 128, 128, 3), ((6, 5, 9), 96, 32, 3), ((9, 7, 11), 48, 16, 1),
            ((8, 8, 8), 96, 32, 1), ((4, 8, 16), 192, 64, 1)]


@pytest.mark.parametrize("din,ci,co,k", WG_CASES)
def test_tc_weight_gradient(d2ip, din, ci, co, k):
    rng = np.random.default_rng(ci * 7 + co + k)
    B = 2
    stream = torch.cuda.current_stream().cuda_stream
    x = bf16_round(rng.standard_normal((B, *din, ci)).astype(np.float32))
    dy = bf16_round(rng.standard_normal((B, *din, co)).astype(np.float32))
    nw = co * k ** 3 * ci
    wsb = d2ip.d2ip_conv3d_wgrad_tc_workspace(B, *din, ci, co, k)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")
    out = torch.full((B, nw + co), float("nan"), device="cuda")
    d2ip.d2ip_conv3d_wgrad_tc(_dev(x), _dev(dy), out, B, *din, ci, co, k, nw + co, 0, ws, wsb,
                              stream)
    torch.cuda.synchronize()
    assert _err_word(ws) == 0
    W0 = np.zeros((co, k, k, k, ci))
    for b in range(B):
        _, gW, gb = onet.conv3d_backward(x[b].astype(np.float64), W0, 1, dy[b].astype(np.float64))
        o = out[b].cpu().numpy()
        e = rel(o[:nw], gW.reshape(-1))
        print("tc wgrad rel err", e)
        assert e < TOL
        assert rel(o[nw:], gb) < 1e-5
