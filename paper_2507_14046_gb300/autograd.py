"""torch.autograd.Function wrappers of the library's op-level C calls: each op's forward and
hand-written backward are the CUDA kernels behind the C ABI; this module only allocates the
outputs (torch tensors on the caller's device) and passes pointers.

Layouts are those of the C ABI: activations channels-last [B][Dz][Dy][Dx][C] (float32,
contiguous, on the GPU); a convolution's parameters per problem as one row Wb[B][Co*K^3*Ci +
Co] (W[co][kz][ky][kx][ci], then the bias); LayerNorm parameters gb[B][2C] (gamma, then beta).
The J products treat J and the measurements as data (no gradient).

    y = conv3d(x, Wb, co, ksize, stride)            # FP32 SIMT kernels
    y = conv3d(x, Wb, co, ksize, stride, tc=True)   # tcgen05, BF16 operands, FP32 accumulation
    y = layernorm_act(z, gb, resid=None, act=1)
    cat = upsample_concat(low, skip, out_dims)
    r = sensitivity_residual(J, x, dv)              # r = J x - dv;  dL/dx = J^T dL/dr
"""
from __future__ import annotations

import torch

from . import binding as B


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _need(t, name):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")


def _out_dims(d, k, s):
    p = (k - 1) // 2
    return tuple((v + 2 * p - k) // s + 1 for v in d)


class _Conv3d(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, Wb, co, k, s, tc):
        _need(x, "x")
        _need(Wb, "Wb")
        b, dz, dy, dx, ci = x.shape
        if Wb.shape != (b, co * k ** 3 * ci + co):
            raise ValueError("Wb must be [B, co*k^3*ci + co]")
        out = torch.empty((b, *_out_dims((dz, dy, dx), k, s), co), device=x.device)
        wbias = Wb.data_ptr() + 4 * co * k ** 3 * ci
        if tc:
            nws = B.d2ip_conv3d_tc_workspace(b, dz, dy, dx, ci, co, k, s)
            ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=x.device)
            B.d2ip_conv3d_forward_tc(x, Wb, wbias, out, b, dz, dy, dx, ci, co, k, s,
                                     Wb.stride(0), ws, nws, _stream())
        else:
            B.d2ip_conv3d_forward(x, Wb, wbias, out, b, dz, dy, dx, ci, co, k, s, Wb.stride(0),
                                  _stream())
        ctx.save_for_backward(x, Wb)
        ctx.cfg = (co, k, s, tc)
        return out

    @staticmethod
    def backward(ctx, gy):
        x, Wb = ctx.saved_tensors
        co, k, s, tc = ctx.cfg
        gy = gy.contiguous()
        b, dz, dy, dx, ci = x.shape
        gx = gW = None
        if ctx.needs_input_grad[0]:
            gx = torch.empty_like(x)
            if tc:
                nws = B.d2ip_conv3d_tc_workspace(b, dz, dy, dx, ci, co, k, s)
                ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=x.device)
                B.d2ip_conv3d_dgrad_tc(gy, Wb, gx, b, dz, dy, dx, ci, co, k, s, Wb.stride(0), 0,
                                       ws, nws, _stream())
            else:
                B.d2ip_conv3d_dgrad(gy, Wb, gx, b, dz, dy, dx, ci, co, k, s, Wb.stride(0), 0,
                                    _stream())
        if ctx.needs_input_grad[1]:
            gW = torch.empty_like(Wb)
            if tc and s == 1:
                nws = B.d2ip_conv3d_wgrad_tc_workspace(b, dz, dy, dx, ci, co, k)
                ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=x.device)
                B.d2ip_conv3d_wgrad_tc(x, gy, gW, b, dz, dy, dx, ci, co, k, gW.stride(0), 0, ws,
                                       nws, _stream())
            else:
                nws = B.d2ip_conv3d_wgrad_workspace(b, dz, dy, dx, ci, co, k, s)
                ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=x.device)
                B.d2ip_conv3d_wgrad(x, gy, gW, b, dz, dy, dx, ci, co, k, s, gW.stride(0), 0, ws,
                                    nws, _stream())
        return gx, gW, None, None, None, None


def conv3d(x, Wb, co, ksize=3, stride=1, tc=False):
    """y[b] = conv(x[b], W_b) + b_b, zero padding (k-1)/2, output ceil(D/stride)."""
    return _Conv3d.apply(x, Wb, co, ksize, stride, tc)


class _LayerNormAct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, gb, resid, act):
        _need(z, "z")
        _need(gb, "gb")
        b, *d, c = z.shape
        nvox = int(torch.tensor(d).prod())
        if resid is not None:
            _need(resid, "resid")
        y = torch.empty_like(z)
        xh = torch.empty_like(z)
        rs = torch.empty((b, nvox), device=z.device)
        B.d2ip_layernorm_act_forward(z, gb, resid, y, xh, rs, b, nvox, c, act, gb.stride(0),
                                     _stream())
        ctx.save_for_backward(y, xh, rs, gb)
        ctx.cfg = (act, resid is not None, nvox)
        return y

    @staticmethod
    def backward(ctx, gy):
        y, xh, rs, gb = ctx.saved_tensors
        act, has_resid, nvox = ctx.cfg
        gy = gy.contiguous()
        b, *d, c = y.shape
        gz = torch.empty_like(y)
        gt = torch.empty_like(y) if has_resid else None
        ggb = torch.empty_like(gb)
        nws = B.d2ip_layernorm_workspace(b, nvox, c)
        ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=y.device)
        B.d2ip_layernorm_act_backward(gy, y if act else None, xh, rs, gb, gz, gt, ggb, b, nvox,
                                      c, gb.stride(0), 0, ws, nws, _stream())
        return gz, ggb, gt, None


def layernorm_act(z, gb, resid=None, act=1):
    """act(LN(z) * gamma + beta (+ resid)) over the channels of each voxel; act 1 = LeakyReLU
    (0.2), 0 = none."""
    return _LayerNormAct.apply(z, gb, resid, act)


class _UpsampleConcat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, low, skip, out_dims):
        _need(low, "low")
        b, lz, ly, lx, cu = low.shape
        cs = 0
        if skip is not None:
            _need(skip, "skip")
            cs = skip.shape[-1]
        oz, oy, ox = out_dims
        cat = torch.empty((b, oz, oy, ox, cu + cs), device=low.device)
        B.d2ip_upsample_concat_forward(low, skip, cat, b, lz, ly, lx, oz, oy, ox, cu, cs,
                                       _stream())
        ctx.cfg = (tuple(low.shape), cs, tuple(out_dims))
        return cat

    @staticmethod
    def backward(ctx, gcat):
        (b, lz, ly, lx, cu), cs, (oz, oy, ox) = ctx.cfg
        gcat = gcat.contiguous()
        glow = torch.empty((b, lz, ly, lx, cu), device=gcat.device)
        gskip = torch.empty((b, oz, oy, ox, cs), device=gcat.device) if cs else None
        B.d2ip_upsample_concat_backward(gcat, glow, gskip, b, lz, ly, lx, oz, oy, ox, cu, cs,
                                        _stream())
        return glow, gskip, None


def upsample_concat(low, skip, out_dims):
    """[trilinear(low -> out_dims), skip] along the channels (skip may be None)."""
    return _UpsampleConcat.apply(low, skip, out_dims)


class _SensitivityResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, x, dv):
        for t, n in ((J, "J"), (x, "x"), (dv, "dv")):
            _need(t, n)
        m, n = J.shape
        b = x.shape[0]
        r = torch.empty((b, m), device=x.device)
        nws = B.d2ip_sensitivity_workspace(b, m, n)
        ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=x.device)
        B.d2ip_sensitivity_residual(J, x, dv, r, None, b, m, n, ws, nws, _stream())
        ctx.save_for_backward(J)
        return r

    @staticmethod
    def backward(ctx, gr):
        (J,) = ctx.saved_tensors
        m, n = J.shape
        gr = gr.contiguous()
        gx = torch.empty((gr.shape[0], n), device=gr.device)
        B.d2ip_sensitivity_adjoint(J, gr, gx, 1.0, gr.shape[0], m, n, _stream())
        return None, gx, None


def sensitivity_residual(J, x, dv):
    """r[b] = J x[b] - dv[b] (x [B, n], dv [B, m]); J and dv are data (no gradient)."""
    return _SensitivityResidual.apply(J, x, dv)
