"""Oracle: the paper-form 3D-FastResUNet (Sec. III-D) as a flagged network variant, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. III-D names the parts of the network and their order but gives no widths, kernel
sizes, dilation rates or attention form.  Those are filled in here by a reading (the
simplified residual U-Net of ``oracle.network`` stays the default network):

* DWSep(ci -> co, s): depthwise 3x3x3 (per channel, stride s, dilation 1, zero padding 1,
  bias) followed by a pointwise 1x1x1 convolution ci -> co with bias (the depthwise
  separable convolution the section cites).  DW_d: the depthwise part with dilation d and
  zero padding d.
* LN and act (LeakyReLU 0.2) as in ``oracle.network``.
* ResConv3D(ci -> co, s): h = act(LN_a(DWSep_a(x; ci -> co, s)));
  out = act(LN_b(DWSep_b(h; co -> co, 1)) + P(x)), P = identity when ci == co and s == 1,
  else a 1x1x1 convolution ci -> co with stride s.
* SE(C) (squeeze-and-excitation): s = sigmoid(FC2(relu(FC1(mean over voxels of x)))),
  FC1: C -> max(C/4, 1), FC2: back to C (each with bias, written as 1x1x1 convolutions on a
  one-voxel volume); y = x * s per channel.
* Encoder: stem = act(LN(conv3(c_in -> w0))); for l = 0..L-1:
  e_l = ResConv3D(SE(previous), in -> w_l, stride 1 for l = 0 else 2), previous = e_l
  (three pairs of SE units and ResConv3D blocks for L = 3).
* Bottleneck at level L: d = act(LN(DWSep(e_{L-1}; C -> C, s = 2))), C = w_{L-1}, then
  ASPP(C) with four branches of width Cb = max(C/2, 1), each followed by act:
  a 1x1x1 convolution, DW_2 then 1x1x1, DW_3 then 1x1x1, and the global mean through a
  1x1x1 convolution broadcast to every voxel; the branches are concatenated in that order
  and b = act(LN(conv1(4 Cb -> C))).
* Decoder, l = L-1 .. 0, g = b for l = L-1 else d_{l+1} (C_g channels, one level coarser):
  attention gate on the skip e_l (additive attention, F = max(w_l/2, 1) inner channels):
  q = relu(conv1_x(e_l) + Up(conv1_g(g))), psi = sigmoid(conv1_psi(q; F -> 1)),
  a_l = e_l * psi (per voxel); then d_l = ResConv3D(concat[Up(g), a_l] -> w_l, s = 1)
  (upsampled first, then the gated skip).  Three attention units and three decoder
  ResConv3D blocks for L = 3: six ResConv3D blocks in all.
* Tail: sigmoid(conv1(d_0; w0 -> 1)) (the Conv3D + sigmoid tail).
* Up: trilinear with half-pixel centres to the finer level's size (as ``oracle.network``).
* Parameters: one flat arena in module order (the order above; within a gate x, g, psi;
  within ASPP the down DWSep and its LN, the four branches, the projection and its LN);
  dense weights W[co][kz][ky][kx][ci] then b[co], depthwise weights W[c][kz][ky][kx] then
  b[c], LayerNorm gamma[c] then beta[c].

The forward pass is written with plain PyTorch CPU operations in float64 (the convolution,
LayerNorm and interpolation primitives are pinned against NumPy loops in the tests); the
gradient is reverse-mode differentiation of that forward (exact up to rounding).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
import torch.nn.functional as F

from .network import KIND_CONV_B, KIND_CONV_W, KIND_LN_B, KIND_LN_G, LN_EPS, SLOPE, NetSpec


@dataclass(frozen=True)
class FastSpec(NetSpec):
    """Grid, L (encoder stages), widths w_0..w_{L-1}, c_in; the bottleneck sits at level L."""


def se_hidden(c: int) -> int:
    return max(c // 4, 1)


def gate_inner(c: int) -> int:
    return max(c // 2, 1)


def aspp_branch(c: int) -> int:
    return max(c // 2, 1)


# ------------------------------------------------------------------------------------
# parameter layout
# ------------------------------------------------------------------------------------

def _dense(name, ci, co, k):
    fan = ci * k ** 3
    return [(name + ".W", (co, k, k, k, ci), KIND_CONV_W, fan),
            (name + ".b", (co,), KIND_CONV_B, fan)]


def _dw(name, c):
    return [(name + ".W", (c, 3, 3, 3), KIND_CONV_W, 27), (name + ".b", (c,), KIND_CONV_B, 27)]


def _ln(name, c):
    return [(name + ".g", (c,), KIND_LN_G, c), (name + ".beta", (c,), KIND_LN_B, c)]


def _dwsep(name, ci, co):
    return _dw(name + ".dw", ci) + _dense(name + ".pw", ci, co, 1)


def _res(name, ci, co, s):
    e = _dwsep(name + ".a", ci, co) + _ln(name + ".lna", co)
    e += _dwsep(name + ".b", co, co) + _ln(name + ".lnb", co)
    if ci != co or s != 1:
        e += _dense(name + ".p", ci, co, 1)
    return e


def _se(name, c):
    h = se_hidden(c)
    return _dense(name + ".fc1", c, h, 1) + _dense(name + ".fc2", h, c, 1)


def _gate(name, cx, cg):
    f = gate_inner(cx)
    return _dense(name + ".x", cx, f, 1) + _dense(name + ".g", cg, f, 1) + \
        _dense(name + ".psi", f, 1, 1)


def _aspp(name, c):
    cb = aspp_branch(c)
    e = _dwsep(name + ".down", c, c) + _ln(name + ".down.ln", c)
    e += _dense(name + ".b0", c, cb, 1)
    e += _dw(name + ".b1.dw", c) + _dense(name + ".b1.pw", c, cb, 1)
    e += _dw(name + ".b2.dw", c) + _dense(name + ".b2.pw", c, cb, 1)
    e += _dense(name + ".b3", c, cb, 1)
    e += _dense(name + ".proj", 4 * cb, c, 1) + _ln(name + ".ln", c)
    return e


def _g_channels(spec, l):
    """Channels of the gating signal of decoder stage l."""
    return spec.widths[spec.levels - 1] if l == spec.levels - 1 else spec.widths[l + 1]


def param_layout(spec: FastSpec):
    """[(name, shape, kind, fan_in, offset, count)] in module order."""
    w, L = spec.widths, spec.levels
    ent = _dense("stem", spec.c_in, w[0], 3) + _ln("stem.ln", w[0])
    for l in range(L):
        cin = w[0] if l == 0 else w[l - 1]
        ent += _se(f"se{l}", cin)
        ent += _res(f"enc{l}", cin, w[l], 1 if l == 0 else 2)
    ent += _aspp("aspp", w[L - 1])
    for l in range(L - 1, -1, -1):
        cg = _g_channels(spec, l)
        ent += _gate(f"att{l}", w[l], cg)
        ent += _res(f"dec{l}", cg + w[l], w[l], 1)
    ent += _dense("tail", w[0], 1, 1)
    out, off = [], 0
    for name, shape, kind, fan_in in ent:
        cnt = int(np.prod(shape))
        out.append((name, shape, kind, fan_in, off, cnt))
        off += cnt
    return out


def param_count(spec: FastSpec) -> int:
    lay = param_layout(spec)
    return lay[-1][4] + lay[-1][5]


def table(spec: FastSpec):
    """(kind, offset, count, fan_in) rows, the parameter table of the C ABI."""
    return [(k, o, c, f) for _, _, k, f, o, c in param_layout(spec)]


# ------------------------------------------------------------------------------------
# primitives (tensors are (1, C, Dz, Dy, Dx) float64)
# ------------------------------------------------------------------------------------

def dense(P, name, x, stride=1):
    W = P[name + ".W"]
    k = W.shape[1]
    return F.conv3d(x, W.permute(0, 4, 1, 2, 3), P[name + ".b"], stride=stride,
                    padding=(k - 1) // 2)


def depthwise(P, name, x, stride=1, dilation=1):
    W = P[name + ".W"]
    return F.conv3d(x, W.unsqueeze(1), P[name + ".b"], stride=stride, padding=dilation,
                    dilation=dilation, groups=W.shape[0])


def layernorm(P, name, z):
    mu = z.mean(dim=1, keepdim=True)
    var = ((z - mu) ** 2).mean(dim=1, keepdim=True)
    xh = (z - mu) / torch.sqrt(var + LN_EPS)
    return xh * P[name + ".g"].view(1, -1, 1, 1, 1) + P[name + ".beta"].view(1, -1, 1, 1, 1)


def act(t):
    return F.leaky_relu(t, SLOPE)


def up(x, dims):
    return F.interpolate(x, size=tuple(dims), mode="trilinear", align_corners=False)


def dwsep(P, name, x, stride=1):
    return dense(P, name + ".pw", depthwise(P, name + ".dw", x, stride))


def res(P, name, x, stride):
    h = act(layernorm(P, name + ".lna", dwsep(P, name + ".a", x, stride)))
    zb = layernorm(P, name + ".lnb", dwsep(P, name + ".b", h))
    p = dense(P, name + ".p", x, stride) if (name + ".p.W") in P else x
    return act(zb + p)


def se(P, name, x):
    s = x.mean(dim=(2, 3, 4), keepdim=True)
    s = torch.sigmoid(dense(P, name + ".fc2", torch.relu(dense(P, name + ".fc1", s))))
    return x * s


def gate(P, name, x, g):
    q = torch.relu(dense(P, name + ".x", x) + up(dense(P, name + ".g", g), x.shape[2:]))
    return x * torch.sigmoid(dense(P, name + ".psi", q))


def aspp(P, name, x):
    d = act(layernorm(P, name + ".down.ln", dwsep(P, name + ".down", x, 2)))
    b0 = act(dense(P, name + ".b0", d))
    b1 = act(dense(P, name + ".b1.pw", depthwise(P, name + ".b1.dw", d, 1, 2)))
    b2 = act(dense(P, name + ".b2.pw", depthwise(P, name + ".b2.dw", d, 1, 3)))
    pooled = act(dense(P, name + ".b3", d.mean(dim=(2, 3, 4), keepdim=True)))
    b3 = pooled.expand(-1, -1, *d.shape[2:])
    cat = torch.cat([b0, b1, b2, b3], dim=1)
    return act(layernorm(P, name + ".ln", dense(P, name + ".proj", cat)))


# ------------------------------------------------------------------------------------
# network
# ------------------------------------------------------------------------------------

def unpack(spec: FastSpec, theta: torch.Tensor) -> dict:
    return {name: theta[off:off + cnt].view(shape)
            for name, shape, _, _, off, cnt in param_layout(spec)}


def forward_t(spec: FastSpec, theta: torch.Tensor, Zin) -> torch.Tensor:
    """Delta sigma = V(phi(theta | Z)) as a float64 tensor of length n (Eq. 2)."""
    P = unpack(spec, theta)
    L = spec.levels
    z = torch.as_tensor(np.asarray(Zin, dtype=np.float64)).reshape(*spec.dims(0), spec.c_in)
    x = z.permute(3, 0, 1, 2).unsqueeze(0)
    cur = act(layernorm(P, "stem.ln", dense(P, "stem", x)))
    e = []
    for l in range(L):
        cur = res(P, f"enc{l}", se(P, f"se{l}", cur), 1 if l == 0 else 2)
        e.append(cur)
    g = aspp(P, "aspp", e[L - 1])
    for l in range(L - 1, -1, -1):
        a = gate(P, f"att{l}", e[l], g)
        g = res(P, f"dec{l}", torch.cat([up(g, e[l].shape[2:]), a], dim=1), 1)
    y = torch.sigmoid(dense(P, "tail", g))
    return y.reshape(-1)


def forward(spec: FastSpec, theta, Zin, keep=False):
    """Same interface as ``oracle.network.forward``: the length-n output (NumPy), and with
    ``keep`` the state ``backward`` needs."""
    th = torch.tensor(np.asarray(theta, dtype=np.float64), requires_grad=keep)
    with torch.set_grad_enabled(keep):
        out = forward_t(spec, th, Zin)
    o = out.detach().numpy().copy()
    return (o, (th, out)) if keep else o


def backward(spec: FastSpec, kept, dsigma):
    """Gradient of <dsigma, Delta sigma> with respect to the flat theta."""
    th, out = kept
    (g,) = torch.autograd.grad(out, th, torch.as_tensor(np.asarray(dsigma, np.float64)))
    return g.numpy().copy()
