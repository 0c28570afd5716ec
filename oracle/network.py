"""Oracle: the residual 3D U-Net phi(theta | Z) of Eq. 2 and its backward pass, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper describes 3D-FastResUNet (Sec. III-D) as a U-Net of 3D convolutions with residual
connections and LayerNorm; the fitting path built here uses the simplified residual U-Net
of its synthetic workloads.  Concrete reading (stated once, used everywhere):

* conv3(ci->co, s): 3x3x3, stride s, zero padding 1, bias; output size ceil(D/s) per axis.
  conv1(ci->co): 1x1x1 with bias.
* LN: LayerNorm over the channel vector of each voxel, eps 1e-5, affine gamma/beta.
* act: LeakyReLU with slope 0.2.
* ResBlock(ci->co): h = act(LN_a(conv3_a(x))); h = LN_b(conv3_b(h)); out = act(h + P(x)),
  P = identity when ci == co, else conv1.
* stem: act(LN(conv3(c_in -> w0))); encoder level 0: ResBlock(w0 -> w0);
  encoder level l > 0: act(LN(conv3(w_{l-1} -> w_l, s=2))) then ResBlock(w_l -> w_l).
* decoder l = L-2 .. 0: u = Up(previous level output -> size of level l);
  ResBlock(concat[u, e_l] -> w_l) (channels: upsampled first, then skip).
* tail: conv1(w0 -> 1), linear (no sigmoid: the truth values are negative).
* Up: trilinear, half-pixel centres (PyTorch align_corners=False) to an explicit size:
  src = (o + 1/2) * S_in / S_out - 1/2 clamped below at 0, i0 = floor(src),
  i1 = min(i0 + 1, S_in - 1), weight of i1 = src - i0.
* Volumes are (Z, Y, X, C) arrays (channels fastest); the output is vectorised as
  q = (z*Y + y)*X + x (the operator V of Eq. 2).
* Flat parameter arena, in module order; per conv W[co][kz][ky][kx][ci] then b[co];
  per LN gamma[c] then beta[c].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LN_EPS = 1e-5
SLOPE = 0.2

KIND_CONV_W, KIND_CONV_B, KIND_LN_G, KIND_LN_B = 0, 1, 2, 3


@dataclass(frozen=True)
class NetSpec:
    grid: tuple[int, int, int]      # (X, Y, Z)
    levels: int
    widths: tuple[int, ...]
    c_in: int = 8

    def dims(self, level: int) -> tuple[int, int, int]:
        """(Z, Y, X) of a level: each stride-2 conv maps D -> ceil(D / 2)."""
        X, Y, Z = self.grid
        d = (Z, Y, X)
        for _ in range(level):
            d = tuple((v + 1) // 2 for v in d)
        return d


# ------------------------------------------------------------------------------------
# parameter layout
# ------------------------------------------------------------------------------------

def _conv_entries(name, ci, co, k):
    return [(name + ".W", (co, k, k, k, ci), KIND_CONV_W, ci * k * k * k),
            (name + ".b", (co,), KIND_CONV_B, ci * k * k * k)]


def _ln_entries(name, c):
    return [(name + ".g", (c,), KIND_LN_G, c), (name + ".beta", (c,), KIND_LN_B, c)]


def _res_entries(name, ci, co):
    e = _conv_entries(name + ".a", ci, co, 3) + _ln_entries(name + ".lna", co)
    e += _conv_entries(name + ".b", co, co, 3) + _ln_entries(name + ".lnb", co)
    if ci != co:
        e += _conv_entries(name + ".p", ci, co, 1)
    return e


def param_layout(spec: NetSpec):
    """[(name, shape, kind, fan_in, offset, count)] in module order."""
    w, L = spec.widths, spec.levels
    ent = _conv_entries("stem", spec.c_in, w[0], 3) + _ln_entries("stem.ln", w[0])
    ent += _res_entries("enc0", w[0], w[0])
    for l in range(1, L):
        ent += _conv_entries(f"down{l}", w[l - 1], w[l], 3) + _ln_entries(f"down{l}.ln", w[l])
        ent += _res_entries(f"enc{l}", w[l], w[l])
    for l in range(L - 2, -1, -1):
        ent += _res_entries(f"dec{l}", w[l + 1] + w[l], w[l])
    ent += _conv_entries("tail", w[0], 1, 1)
    out, off = [], 0
    for name, shape, kind, fan_in in ent:
        cnt = int(np.prod(shape))
        out.append((name, shape, kind, fan_in, off, cnt))
        off += cnt
    return out


def param_count(spec: NetSpec) -> int:
    lay = param_layout(spec)
    return lay[-1][4] + lay[-1][5]


def unpack(spec: NetSpec, theta: np.ndarray) -> dict:
    return {name: theta[off:off + cnt].reshape(shape)
            for name, shape, _, _, off, cnt in param_layout(spec)}


def pack(spec: NetSpec, tensors: dict) -> np.ndarray:
    out = np.zeros(param_count(spec), dtype=np.float64)
    for name, shape, _, _, off, cnt in param_layout(spec):
        out[off:off + cnt] = np.asarray(tensors[name], dtype=np.float64).reshape(-1)
    return out


# ------------------------------------------------------------------------------------
# primitive ops (forward and exact adjoint)
# ------------------------------------------------------------------------------------

def conv3d(x, W, b, stride):
    """y[o] = b + sum over taps k and input channels c of W[:, k, c] x[s*o + k - pad, c].

    x: (Dz, Dy, Dx, Ci); W: (Co, K, K, K, Ci); zero padding (K-1)/2.  The channel sum of
    each tap is one matrix product.
    """
    K = W.shape[1]
    pad = (K - 1) // 2
    Dz, Dy, Dx, _ = x.shape
    O = [(d + 2 * pad - K) // stride + 1 for d in (Dz, Dy, Dx)]
    xp = np.pad(x, ((pad, pad), (pad, pad), (pad, pad), (0, 0)))
    y = np.broadcast_to(b, (*O, W.shape[0])).copy()
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                patch = xp[kz:kz + stride * (O[0] - 1) + 1:stride,
                           ky:ky + stride * (O[1] - 1) + 1:stride,
                           kx:kx + stride * (O[2] - 1) + 1:stride]
                y += patch @ W[:, kz, ky, kx, :].T
    return y


def conv3d_backward(x, W, stride, dy):
    """Adjoint of ``conv3d`` in (x, W, b): returns (dx, dW, db)."""
    K = W.shape[1]
    pad = (K - 1) // 2
    O = dy.shape[:3]
    xp = np.pad(x, ((pad, pad), (pad, pad), (pad, pad), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    Co = W.shape[0]
    dy2 = dy.reshape(-1, Co)
    for kz in range(K):
        for ky in range(K):
            for kx in range(K):
                sl = (slice(kz, kz + stride * (O[0] - 1) + 1, stride),
                      slice(ky, ky + stride * (O[1] - 1) + 1, stride),
                      slice(kx, kx + stride * (O[2] - 1) + 1, stride))
                patch = xp[sl].reshape(-1, xp.shape[3])
                dW[:, kz, ky, kx, :] = dy2.T @ patch
                dxp[sl] += dy @ W[:, kz, ky, kx, :]
    Dz, Dy, Dx, _ = x.shape
    dx = dxp[pad:pad + Dz, pad:pad + Dy, pad:pad + Dx]
    db = dy2.sum(axis=0)
    return dx, dW, db


def layernorm(z, g, beta):
    """Per-voxel LayerNorm over channels: xhat = (z - mean) / sqrt(var + eps) (biased var)."""
    mu = z.mean(axis=-1, keepdims=True)
    var = ((z - mu) ** 2).mean(axis=-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + LN_EPS)
    xhat = (z - mu) * rstd
    return xhat * g + beta, (xhat, rstd)


def layernorm_backward(dy, cache, g):
    """Exact derivative of ``layernorm``: returns (dz, dgamma, dbeta)."""
    xhat, rstd = cache
    C = xhat.shape[-1]
    dxh = dy * g
    dz = rstd * (dxh - dxh.mean(axis=-1, keepdims=True)
                 - xhat * (dxh * xhat).mean(axis=-1, keepdims=True))
    red = tuple(range(dy.ndim - 1))
    del C
    return dz, (dy * xhat).sum(axis=red), dy.sum(axis=red)


def lrelu(t):
    return np.where(t > 0, t, SLOPE * t)


def lrelu_backward(da, t):
    return np.where(t > 0, da, SLOPE * da)


def up_axis_map(s_in: int, s_out: int):
    """Per-output (i0, i1, w1) of half-pixel linear interpolation along one axis.

    src = (o + 1/2) s_in / s_out - 1/2 = ((2o+1) s_in - s_out) / (2 s_out), clamped at 0;
    the integer form keeps the index map exact.
    """
    o = np.arange(s_out)
    num = (2 * o + 1) * s_in - s_out
    num = np.maximum(num, 0)
    den = 2 * s_out
    i0 = num // den
    w1 = (num - i0 * den) / den
    i1 = np.minimum(i0 + 1, s_in - 1)
    return i0, i1, w1.astype(np.float64)


def upsample(u, out_dims):
    """Trilinear resampling of u (Sz, Sy, Sx, C) to out_dims = (Oz, Oy, Ox): each output is
    the sum over the 8 corners of the product of the three axis weights times the input."""
    maps = [up_axis_map(s, o) for s, o in zip(u.shape[:3], out_dims)]
    (z0, z1, wz), (y0, y1, wy), (x0, x1, wx) = maps
    out = np.zeros((*out_dims, u.shape[3]))
    for iz, fz in ((z0, 1 - wz), (z1, wz)):
        for iy, fy in ((y0, 1 - wy), (y1, wy)):
            for ix, fx in ((x0, 1 - wx), (x1, wx)):
                w = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
                out += w[..., None] * u[iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return out


def upsample_backward(dy, in_dims):
    """Adjoint of ``upsample``: scatter-add each output gradient to its 8 corners."""
    out_dims = dy.shape[:3]
    maps = [up_axis_map(s, o) for s, o in zip(in_dims, out_dims)]
    (z0, z1, wz), (y0, y1, wy), (x0, x1, wx) = maps
    du = np.zeros((*in_dims, dy.shape[3]))
    for iz, fz in ((z0, 1 - wz), (z1, wz)):
        for iy, fy in ((y0, 1 - wy), (y1, wy)):
            for ix, fx in ((x0, 1 - wx), (x1, wx)):
                w = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
                Iz, Iy, Ix = np.broadcast_arrays(iz[:, None, None], iy[None, :, None],
                                                 ix[None, None, :])
                np.add.at(du, (Iz, Iy, Ix), w[..., None] * dy)
    return du


# ------------------------------------------------------------------------------------
# blocks
# ------------------------------------------------------------------------------------

def _conv_ln_act_fwd(P, name, ln, x, stride):
    z = conv3d(x, P[name + ".W"], P[name + ".b"], stride)
    y, lc = layernorm(z, P[ln + ".g"], P[ln + ".beta"])
    return lrelu(y), (x, lc, y)


def _conv_ln_act_bwd(P, G, name, ln, stride, cache, da):
    x, lc, y = cache
    dy = lrelu_backward(da, y)
    dz, G[ln + ".g"], G[ln + ".beta"] = layernorm_backward(dy, lc, P[ln + ".g"])
    dx, G[name + ".W"], G[name + ".b"] = conv3d_backward(x, P[name + ".W"], stride, dz)
    return dx


def _res_fwd(P, name, x):
    h1, c1 = _conv_ln_act_fwd(P, name + ".a", name + ".lna", x, 1)
    zb = conv3d(h1, P[name + ".b.W"], P[name + ".b.b"], 1)
    h2, lcb = layernorm(zb, P[name + ".lnb.g"], P[name + ".lnb.beta"])
    proj = (name + ".p.W") in P
    p = conv3d(x, P[name + ".p.W"], P[name + ".p.b"], 1) if proj else x
    t = h2 + p
    return lrelu(t), (x, c1, h1, lcb, t, proj)


def _res_bwd(P, G, name, cache, dout):
    x, c1, h1, lcb, t, proj = cache
    dt = lrelu_backward(dout, t)
    dzb, G[name + ".lnb.g"], G[name + ".lnb.beta"] = layernorm_backward(dt, lcb,
                                                                        P[name + ".lnb.g"])
    dh1, G[name + ".b.W"], G[name + ".b.b"] = conv3d_backward(h1, P[name + ".b.W"], 1, dzb)
    dx = _conv_ln_act_bwd(P, G, name + ".a", name + ".lna", 1, c1, dh1)
    if proj:
        dxp, G[name + ".p.W"], G[name + ".p.b"] = conv3d_backward(x, P[name + ".p.W"], 1, dt)
        dx = dx + dxp
    else:
        dx = dx + dt
    return dx


# ------------------------------------------------------------------------------------
# network
# ------------------------------------------------------------------------------------

def forward(spec: NetSpec, theta, Zin, keep=False):
    """Delta sigma = V(phi(theta | Z)) (Eq. 2).  Zin: (n, c_in) or (Z, Y, X, c_in).

    Returns the length-n vector (and the cache for ``backward`` when ``keep``)."""
    P = unpack(spec, np.asarray(theta, dtype=np.float64))
    L = spec.levels
    x0 = np.asarray(Zin, dtype=np.float64).reshape(*spec.dims(0), spec.c_in)
    cache = {}
    s, cache["stem"] = _conv_ln_act_fwd(P, "stem", "stem.ln", x0, 1)
    e = [None] * L
    e[0], cache["enc0"] = _res_fwd(P, "enc0", s)
    for l in range(1, L):
        d, cache[f"down{l}"] = _conv_ln_act_fwd(P, f"down{l}", f"down{l}.ln", e[l - 1], 2)
        e[l], cache[f"enc{l}"] = _res_fwd(P, f"enc{l}", d)
    cur = e[L - 1]
    for l in range(L - 2, -1, -1):
        u = upsample(cur, spec.dims(l))
        cat = np.concatenate([u, e[l]], axis=-1)
        cache[f"up{l}"] = (cur.shape[:3], u.shape[3])
        cur, cache[f"dec{l}"] = _res_fwd(P, f"dec{l}", cat)
    y = conv3d(cur, P["tail.W"], P["tail.b"], 1)
    cache["tail"] = cur
    out = y.reshape(-1)
    return (out, (P, cache)) if keep else out


def backward(spec: NetSpec, kept, dsigma):
    """Gradient of <dsigma, Delta sigma> with respect to the flat theta (chain rule in
    reverse module order).  ``kept`` is the second value of ``forward(..., keep=True)``."""
    P, cache = kept
    L = spec.levels
    G = {}
    cur = cache["tail"]
    dy = np.asarray(dsigma, dtype=np.float64).reshape(*spec.dims(0), 1)
    dcur, G["tail.W"], G["tail.b"] = conv3d_backward(cur, P["tail.W"], 1, dy)
    de = [None] * L
    for l in range(0, L - 1):
        dcat = _res_bwd(P, G, f"dec{l}", cache[f"dec{l}"], dcur)
        in_dims, cu = cache[f"up{l}"]
        de[l] = dcat[..., cu:].copy()
        dcur = upsample_backward(dcat[..., :cu], in_dims)
        # dcur is the gradient of the previous decoder level output (or e_{L-1})
        if l + 1 == L - 1:
            de[L - 1] = dcur
    if L == 1:
        de[0] = dcur
    for l in range(L - 1, 0, -1):
        dd = _res_bwd(P, G, f"enc{l}", cache[f"enc{l}"], de[l])
        dprev = _conv_ln_act_bwd(P, G, f"down{l}", f"down{l}.ln", 2, cache[f"down{l}"], dd)
        de[l - 1] = de[l - 1] + dprev
    ds = _res_bwd(P, G, "enc0", cache["enc0"], de[0])
    _conv_ln_act_bwd(P, G, "stem", "stem.ln", 1, cache["stem"], ds)
    return pack(spec, G)
