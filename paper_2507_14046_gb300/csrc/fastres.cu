// The paper-form 3D-FastResUNet variant (Sec. III-D) as a node list: construction in
// parameter order, buffer binding, and the forward and backward launch sequences.
//
// Reading of the architecture (the section names the parts but no sizes):
//  DWSep(ci -> co, s) = depthwise 3x3x3 (stride s) then pointwise 1x1x1;
//  ResConv3D(ci -> co, s): act(LN_b(DWSep_b(act(LN_a(DWSep_a(x))))) + P(x)), P a 1x1x1
//    convolution with stride s when ci != co or s != 1, else the identity;
//  SE(C): x * sigmoid(FC2(relu(FC1(mean_voxels x)))), FC1 C -> max(C/4, 1);
//  encoder: stem act(LN(conv3(c_in -> w0))), then per level l SE and ResConv3D(-> w_l,
//    stride 2 for l > 0);
//  bottleneck: act(LN(DWSep(e_{L-1}, s = 2))) then ASPP with branches 1x1x1, depthwise
//    dilation 2 and 3 (each then 1x1x1) and the broadcast global mean, each of width
//    max(C/2, 1) and LeakyReLU, concatenated, projected by 1x1x1 to C, act(LN);
//  decoder l = L-1..0: additive attention gate on the skip e_l with inner width max(w_l/2, 1):
//    e_l * sigmoid(psi(relu(Wx e_l + Up(Wg g)))), then ResConv3D([Up(g), gated skip] -> w_l);
//  tail: sigmoid(conv1(w0 -> 1)).
// Parameters are laid out in that module order (weights then bias; LN gamma then beta).
#include <algorithm>

#include "common.cuh"
#include "fastres.cuh"
#include "../../include/d2ip.h"

namespace d2ip {
namespace {

struct FrBuilder {
  FastNet& n;
  std::vector<long long>& table;
  long long off = 0;

  long long rows(int kind, long long count, long long fan) {
    const long long o = off;
    table.insert(table.end(), {(long long)kind, off, count, fan});
    off += count;
    return o;
  }
  long long dense_params(int ci, int co, int k) {
    const long long fan = (long long)ci * k * k * k;
    const long long o = rows(D2IP_PARAM_CONV_W, (long long)co * k * k * k * ci, fan);
    rows(D2IP_PARAM_CONV_B, co, fan);
    return o;
  }
  long long dw_params(int C) {
    const long long o = rows(D2IP_PARAM_CONV_W, 27LL * C, 27);
    rows(D2IP_PARAM_CONV_B, C, 27);
    return o;
  }
  long long ln_params(int C) {
    const long long o = rows(D2IP_PARAM_LN_GAMMA, C, C);
    rows(D2IP_PARAM_LN_BETA, C, C);
    return o;
  }

  int val(int lvl, int C) {
    FrVal v;
    v.lvl = lvl;
    v.C = C;
    n.vals.push_back(v);
    return (int)n.vals.size() - 1;
  }
  int node(FrNode nd, int lvl, int C) {
    nd.out = val(lvl, C);
    n.nodes.push_back(nd);
    return nd.out;
  }
  int lvl(int x) const { return n.vals[x].lvl; }
  int ch(int x) const { return n.vals[x].C; }
  int one() const { return (int)n.dims.size() - 1; }

  int conv3(int x, int co, long long w) {
    FrNode d;
    d.kind = kFrConv3;
    d.in0 = x;
    d.ci = ch(x);
    d.co = co;
    d.w_off = w;
    return node(d, lvl(x), co);
  }
  int pw(int x, int co, int s, long long w) {
    FrNode d;
    d.kind = kFrPw;
    d.in0 = x;
    d.ci = ch(x);
    d.co = co;
    d.s = s;
    d.w_off = w;
    return node(d, lvl(x) + (s == 2 ? 1 : 0), co);
  }
  int dw(int x, int s, int dil, long long w) {
    FrNode d;
    d.kind = kFrDw;
    d.in0 = x;
    d.ci = d.co = ch(x);
    d.s = s;
    d.d = dil;
    d.w_off = w;
    return node(d, lvl(x) + (s == 2 ? 1 : 0), ch(x));
  }
  int ln(int z, long long g, int resid = -1) {
    FrNode d;
    d.kind = kFrLn;
    d.in0 = z;
    d.resid = resid;
    d.w_off = g;
    return node(d, lvl(z), ch(z));
  }
  int act(int x, int kind) {
    FrNode d;
    d.kind = kFrAct;
    d.in0 = x;
    d.act = kind;
    return node(d, lvl(x), ch(x));
  }
  int two(int kind, int a, int b, int out_lvl, int C) {
    FrNode d;
    d.kind = kind;
    d.in0 = a;
    d.in1 = b;
    return node(d, out_lvl, C);
  }
  int pool(int x) {
    FrNode d;
    d.kind = kFrPool;
    d.in0 = x;
    return node(d, one(), ch(x));
  }
  int bcast(int x, int to_lvl) {
    FrNode d;
    d.kind = kFrBcast;
    d.in0 = x;
    return node(d, to_lvl, ch(x));
  }
  int up(int x, int to_lvl) {
    FrNode d;
    d.kind = kFrUp;
    d.in0 = x;
    return node(d, to_lvl, ch(x));
  }
  int concat(const std::vector<int>& parts) {
    int C = 0;
    for (int p : parts) C += ch(p);
    const int out = val(lvl(parts[0]), C);
    int o = 0;
    for (int p : parts) {
      FrNode d;
      d.kind = kFrSlice;
      d.in0 = p;
      d.out = out;
      d.off = o;
      o += ch(p);
      n.nodes.push_back(d);
    }
    return out;
  }

  int dwsep(int x, int co, int s, long long wdw, long long wpw) {
    return pw(dw(x, s, 1, wdw), co, 1, wpw);
  }
  int res(int x, int co, int s) {
    const int ci = ch(x);
    const long long a_dw = dw_params(ci), a_pw = dense_params(ci, co, 1), lna = ln_params(co);
    const long long b_dw = dw_params(co), b_pw = dense_params(co, co, 1), lnb = ln_params(co);
    const bool proj = ci != co || s != 1;
    const long long p = proj ? dense_params(ci, co, 1) : -1;
    const int h = ln(dwsep(x, co, s, a_dw, a_pw), lna);
    const int zb = dwsep(h, co, 1, b_dw, b_pw);
    const int r = proj ? pw(x, co, s, p) : x;
    return ln(zb, lnb, r);
  }
  int se(int x) {
    const int C = ch(x), h = std::max(C / 4, 1);
    const long long f1 = dense_params(C, h, 1), f2 = dense_params(h, C, 1);
    const int s = act(pw(act(pw(pool(x), h, 1, f1), kActRelu), C, 1, f2), kActSigmoid);
    return two(kFrCscale, x, s, lvl(x), C);
  }
  int gate(int x, int g) {
    const int F = std::max(ch(x) / 2, 1);
    const long long wx = dense_params(ch(x), F, 1), wg = dense_params(ch(g), F, 1),
                    wp = dense_params(F, 1, 1);
    const int px = pw(x, F, 1, wx);
    const int ug = up(pw(g, F, 1, wg), lvl(x));
    const int q = act(two(kFrAdd, px, ug, lvl(x), F), kActRelu);
    const int psi = act(pw(q, 1, 1, wp), kActSigmoid);
    return two(kFrVscale, x, psi, lvl(x), ch(x));
  }
  int aspp(int x) {
    const int C = ch(x), cb = std::max(C / 2, 1);
    const long long d_dw = dw_params(C), d_pw = dense_params(C, C, 1), d_ln = ln_params(C);
    const long long w0 = dense_params(C, cb, 1);
    const long long w1d = dw_params(C), w1p = dense_params(C, cb, 1);
    const long long w2d = dw_params(C), w2p = dense_params(C, cb, 1);
    const long long w3 = dense_params(C, cb, 1);
    const long long wpr = dense_params(4 * cb, C, 1), lnp = ln_params(C);
    const int d = ln(dwsep(x, C, 2, d_dw, d_pw), d_ln);
    const int b0 = act(pw(d, cb, 1, w0), kActLeaky);
    const int b1 = act(pw(dw(d, 1, 2, w1d), cb, 1, w1p), kActLeaky);
    const int b2 = act(pw(dw(d, 1, 3, w2d), cb, 1, w2p), kActLeaky);
    const int b3 = bcast(act(pw(pool(d), cb, 1, w3), kActLeaky), lvl(d));
    return ln(pw(concat({b0, b1, b2, b3}), C, 1, wpr), lnp);
  }
};

long long nv(const FastNet& n, int v) { return n.dims[n.vals[v].lvl].count(); }

}  // namespace

bool fastres_supported(int L, const int* w, int c_in) {
  if (L < 1 || L > 6 || c_in < 1 || c_in > 256) return false;
  for (int l = 0; l < L; ++l)
    if (w[l] < 8 || w[l] % 8 || w[l] > 128) return false;
  return true;
}

void FastNet::build(Dims3 grid, int L, const std::vector<int>& w, int c_in,
                    std::vector<long long>& table, long long& P) {
  dims.assign(1, grid);
  for (int l = 1; l <= L; ++l) dims.push_back(conv_out_dims(dims[l - 1], 3, 2));
  dims.push_back(Dims3{1, 1, 1});
  vals.clear();
  nodes.clear();
  table.clear();
  FrBuilder b{*this, table};
  FrVal z;
  z.lvl = 0;
  z.C = c_in;
  z.grad = false;
  vals.push_back(z);
  const long long w_stem = b.dense_params(c_in, w[0], 3), ln_stem = b.ln_params(w[0]);
  int cur = b.ln(b.conv3(0, w[0], w_stem), ln_stem);
  std::vector<int> e(L);
  for (int l = 0; l < L; ++l) {
    cur = b.se(cur);
    e[l] = cur = b.res(cur, w[l], l == 0 ? 1 : 2);
  }
  int g = b.aspp(e[L - 1]);
  for (int l = L - 1; l >= 0; --l) {
    const int a = b.gate(e[l], g);
    const int cat = b.two(kFrUpcat, g, a, l, b.ch(g) + w[l]);
    g = b.res(cat, w[l], 1);
  }
  const long long wt = b.dense_params(w[0], 1, 1);
  b.act(b.pw(g, 1, 1, wt), kActSigmoid);
  P = b.off;
  // backward order = reverse node order: the first node to produce a value's gradient writes
  // it, later ones add into it
  std::vector<char> written(vals.size(), 0);
  auto mark = [&](int v, bool& acc) {
    if (v < 0 || !vals[v].grad) return;
    acc = written[v] != 0;
    written[v] = 1;
  };
  for (int i = (int)nodes.size() - 1; i >= 0; --i) {
    FrNode& nd = nodes[i];
    mark(nd.in0, nd.acc0);
    if (nd.in1 >= 0) mark(nd.in1, nd.acc1);
    if (nd.resid >= 0) mark(nd.resid, nd.accr);
  }
}

long long FastNet::arena_floats(int batch) const {
  const auto r = [](long long f) { return (f + 63) / 64 * 64; };
  long long tot = 0, tmpf = 0, wsf = 0;
  for (size_t v = 1; v + 1 < vals.size(); ++v) {
    const long long f = r((long long)batch * nv(*this, (int)v) * vals[v].C);
    tot += 2 * f;
    tmpf = std::max(tmpf, f);
  }
  for (const FrNode& nd : nodes) {
    const Dims3 din = dims[vals[nd.in0].lvl];
    const long long n_in = din.count();
    long long w = 0;
    switch (nd.kind) {
      case kFrConv3:
        w = conv3d_wgrad_chunks(din, 3, 1) * ((long long)nd.co * 27 * nd.ci + nd.co);
        break;
      case kFrPw:
        w = pw_wgrad_rows(din, nd.s) * ((long long)nd.co * nd.ci + nd.co);
        break;
      case kFrDw:
        w = dw_wgrad_rows(din, nd.s) * 28LL * nd.ci;
        break;
      case kFrLn:
        w = layernorm_bwd_blocks(n_in, vals[nd.in0].C) * 2LL * vals[nd.in0].C;
        tot += r((long long)batch * n_in * (vals[nd.in0].C + 1));
        break;
      case kFrPool:
      case kFrCscale:
        w = vox_sum_rows(n_in) * vals[nd.in0].C;
        break;
      case kFrBcast:
        w = vox_sum_rows(nv(*this, nd.out)) * vals[nd.in0].C;
        break;
      default:
        break;
    }
    wsf = std::max(wsf, (long long)batch * w);
  }
  return tot + r(wsf) + 2 * r(tmpf);
}

void FastNet::bind(float* base, int batch, float* zin, float* dsigma, float* gds) {
  B = batch;
  const auto r = [](long long f) { return (f + 63) / 64 * 64; };
  float* p = base;
  vals[0].v = zin;
  tmp_floats = 0;
  for (size_t v = 1; v + 1 < vals.size(); ++v) {
    const long long f = r((long long)B * nv(*this, (int)v) * vals[v].C);
    vals[v].v = p;
    p += f;
    vals[v].g = p;
    p += f;
    tmp_floats = std::max(tmp_floats, f);
  }
  vals.back().v = dsigma;
  vals.back().g = gds;
  long long wsf = 0;
  for (FrNode& nd : nodes) {
    if (nd.kind == kFrLn) {
      const long long n_in = nv(*this, nd.in0);
      nd.xh = p;
      nd.rs = p + (long long)B * n_in * vals[nd.in0].C;
      p += r((long long)B * n_in * (vals[nd.in0].C + 1));
    }
  }
  // the workspace size is recomputed the same way as in arena_floats
  const long long total = arena_floats(B);
  const long long used = p - base;
  wsf = total - used - 2 * r(tmp_floats);
  ws_floats = wsf;
  ws = p;
  p += wsf;
  tmp = p;
  p += r(tmp_floats);
  tmp2 = p;
}

namespace {

struct Tr {
  const FrRun& r;
  void beg(int k, double w) const {
    if (r.beg) r.beg(r.user, k, w);
  }
  void fin() const {
    if (r.fin) r.fin(r.user);
  }
};

}  // namespace

cudaError_t FastNet::forward(const FrRun& R) const {
  const Tr t{R};
  cudaStream_t st = R.stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  for (const FrNode& nd : nodes) {
    const FrVal &x = vals[nd.in0], &y = vals[nd.out];
    const Dims3 din = dims[x.lvl], dout = dims[y.lvl];
    const long long nin = din.count(), nout = dout.count();
    const float* W = R.theta + nd.w_off;
    switch (nd.kind) {
      case kFrConv3:
        t.beg(D2IP_KCLASS_CONV_FWD, 2.0 * B * nout * 27 * nd.ci * nd.co);
        ok(conv3d_fwd_f32(x.v, W, W + 27LL * nd.co * nd.ci, y.v, B, din, nd.ci, nd.co, 3, 1,
                          nin * nd.ci, nout * nd.co, R.Pp, st));
        t.fin();
        break;
      case kFrPw:
        t.beg(D2IP_KCLASS_CONV_FWD, 2.0 * B * nout * nd.ci * nd.co);
        ok(pw_fwd_f32(x.v, W, y.v, B, din, nd.ci, nd.co, nd.s, R.Pp, 0, st));
        t.fin();
        break;
      case kFrDw:
        t.beg(D2IP_KCLASS_CONV_FWD, 2.0 * B * nout * 27 * nd.ci);
        ok(dw_fwd_f32(x.v, W, y.v, B, din, nd.ci, nd.s, nd.d, R.Pp, st));
        t.fin();
        break;
      case kFrLn:
        t.beg(D2IP_KCLASS_LN_FWD, 4.0 * B * nin * (x.C * (nd.resid >= 0 ? 4 : 3) + 1));
        ok(layernorm_act_fwd_f32(x.v, W, nd.resid >= 0 ? vals[nd.resid].v : nullptr, y.v, nd.xh,
                                 nd.rs, B, nin, x.C, 1, R.Pp, st));
        t.fin();
        break;
      case kFrAct:
        t.beg(D2IP_KCLASS_MISC, 8.0 * B * nin * x.C);
        ok(act_fwd_f32(x.v, y.v, (long long)B * nin * x.C, nd.act, st));
        t.fin();
        break;
      case kFrAdd:
        t.beg(D2IP_KCLASS_MISC, 12.0 * B * nin * x.C);
        ok(add2_f32(x.v, vals[nd.in1].v, y.v, (long long)B * nin * x.C, st));
        t.fin();
        break;
      case kFrPool: {
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nin * x.C);
        const long long rows = vox_sum_rows(nin);
        ok(vox_sum_partial_f32(x.v, nullptr, ws, B, nin, x.C, 1.0f / (float)nin, st));
        ok(reduce_rows_f32(ws, y.v, B, rows, x.C, x.C, 0, st));
        t.fin();
        break;
      }
      case kFrBcast:
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nout * x.C);
        ok(bcast_f32(x.v, y.v, B, nout, x.C, 1.0f, 0, st));
        t.fin();
        break;
      case kFrCscale:
        t.beg(D2IP_KCLASS_MISC, 8.0 * B * nin * x.C);
        ok(cscale_f32(x.v, vals[nd.in1].v, y.v, B, nin, x.C, 0, st));
        t.fin();
        break;
      case kFrVscale:
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nin * (2.0 * x.C + 1));
        ok(vscale_f32(x.v, vals[nd.in1].v, y.v, (long long)B * nin, x.C, 0, st));
        t.fin();
        break;
      case kFrUp:
        t.beg(D2IP_KCLASS_UP_FWD, 4.0 * B * (nin + nout) * x.C);
        ok(upsample_concat_fwd_f32(x.v, nullptr, y.v, B, din, dout, x.C, 0, st));
        t.fin();
        break;
      case kFrUpcat: {
        const FrVal& s = vals[nd.in1];
        t.beg(D2IP_KCLASS_UP_FWD, 4.0 * B * (nin * x.C + nout * (x.C + 2.0 * s.C)));
        ok(upsample_concat_fwd_f32(x.v, s.v, y.v, B, din, dout, x.C, s.C, st));
        t.fin();
        break;
      }
      case kFrSlice:
        t.beg(D2IP_KCLASS_MISC, 8.0 * B * nin * x.C);
        ok(slice_f32(x.v, x.C, 0, y.v, y.C, nd.off, x.C, (long long)B * nin, 0, st));
        t.fin();
        break;
      default:
        ok(cudaErrorInvalidValue);
    }
  }
  return e;
}

cudaError_t FastNet::backward(const FrRun& R) const {
  const Tr t{R};
  cudaStream_t st = R.stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  for (int i = (int)nodes.size() - 1; i >= 0; --i) {
    const FrNode& nd = nodes[i];
    const FrVal &x = vals[nd.in0], &y = vals[nd.out];
    const Dims3 din = dims[x.lvl], dout = dims[y.lvl];
    const long long nin = din.count(), nout = dout.count();
    const float* W = R.theta + nd.w_off;
    float* G = R.grad + nd.w_off;
    const int a0 = nd.acc0 ? 1 : 0, a1 = nd.acc1 ? 1 : 0;
    switch (nd.kind) {
      case kFrConv3: {
        const double fl = 2.0 * B * nout * 27 * nd.ci * nd.co;
        if (x.grad) {
          t.beg(D2IP_KCLASS_CONV_DGRAD, fl);
          ok(conv3d_dgrad_f32(y.g, W, x.g, B, din, nd.ci, nd.co, 3, 1, nout * nd.co,
                              nin * nd.ci, R.Pp, a0, st));
          t.fin();
        }
        t.beg(D2IP_KCLASS_CONV_WGRAD, fl);
        ok(conv3d_wgrad_partial_f32(x.v, y.g, ws, B, din, nd.ci, nd.co, 3, 1, nin * nd.ci,
                                    nout * nd.co, st));
        ok(reduce_rows_f32(ws, G, B, conv3d_wgrad_chunks(din, 3, 1),
                           27LL * nd.co * nd.ci + nd.co, R.Pp, 0, st));
        t.fin();
        break;
      }
      case kFrPw: {
        const double fl = 2.0 * B * nout * nd.ci * nd.co;
        t.beg(D2IP_KCLASS_CONV_DGRAD, fl);
        ok(pw_dgrad_f32(y.g, W, x.g, B, din, nd.ci, nd.co, nd.s, R.Pp, a0, st));
        t.fin();
        t.beg(D2IP_KCLASS_CONV_WGRAD, fl);
        ok(pw_wgrad_partial_f32(x.v, y.g, ws, B, din, nd.ci, nd.co, nd.s, st));
        ok(reduce_rows_f32(ws, G, B, pw_wgrad_rows(din, nd.s), (long long)nd.co * nd.ci + nd.co,
                           R.Pp, 0, st));
        t.fin();
        break;
      }
      case kFrDw: {
        const double fl = 2.0 * B * nout * 27 * nd.ci;
        t.beg(D2IP_KCLASS_CONV_DGRAD, fl);
        ok(dw_dgrad_f32(y.g, W, x.g, B, din, nd.ci, nd.s, nd.d, R.Pp, a0, st));
        t.fin();
        t.beg(D2IP_KCLASS_CONV_WGRAD, fl);
        ok(dw_wgrad_partial_f32(x.v, y.g, ws, B, din, nd.ci, nd.s, nd.d, st));
        ok(reduce_rows_f32(ws, G, B, dw_wgrad_rows(din, nd.s), 28LL * nd.ci, R.Pp, 0, st));
        t.fin();
        break;
      }
      case kFrLn: {
        const bool res = nd.resid >= 0;
        float* dz = a0 ? tmp : x.g;
        float* dt = res ? (nd.accr ? tmp2 : vals[nd.resid].g) : nullptr;
        const long long cnt = (long long)B * nin * x.C;
        t.beg(D2IP_KCLASS_LN_BWD, 4.0 * B * nin * (x.C * (res ? 5 : 4) + 1));
        ok(layernorm_act_bwd_f32(y.g, y.v, nd.xh, nd.rs, W, dz, dt, ws, B, nin, x.C, R.Pp, st));
        ok(reduce_rows_f32(ws, G, B, layernorm_bwd_blocks(nin, x.C), 2LL * x.C, R.Pp, 0, st));
        if (a0) ok(accum_f32(x.g, tmp, cnt, 1, st));
        if (res && nd.accr) ok(accum_f32(vals[nd.resid].g, tmp2, cnt, 1, st));
        t.fin();
        break;
      }
      case kFrAct:
        t.beg(D2IP_KCLASS_MISC, 12.0 * B * nin * x.C);
        ok(act_bwd_f32(y.v, y.g, x.g, (long long)B * nin * x.C, nd.act, a0, st));
        t.fin();
        break;
      case kFrAdd: {
        const long long cnt = (long long)B * nin * x.C;
        t.beg(D2IP_KCLASS_MISC, 16.0 * cnt);
        ok(accum_f32(x.g, y.g, cnt, a0, st));
        ok(accum_f32(vals[nd.in1].g, y.g, cnt, a1, st));
        t.fin();
        break;
      }
      case kFrPool:
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nin * x.C);
        ok(bcast_f32(y.g, x.g, B, nin, x.C, 1.0f / (float)nin, a0, st));
        t.fin();
        break;
      case kFrBcast: {
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nout * x.C);
        ok(vox_sum_partial_f32(y.g, nullptr, ws, B, nout, x.C, 1.0f, st));
        ok(reduce_rows_f32(ws, x.g, B, vox_sum_rows(nout), x.C, x.C, a0, st));
        t.fin();
        break;
      }
      case kFrCscale: {
        const FrVal& s = vals[nd.in1];
        t.beg(D2IP_KCLASS_MISC, 16.0 * B * nin * x.C);
        ok(cscale_f32(y.g, s.v, x.g, B, nin, x.C, a0, st));
        ok(vox_sum_partial_f32(y.g, x.v, ws, B, nin, x.C, 1.0f, st));
        ok(reduce_rows_f32(ws, s.g, B, vox_sum_rows(nin), x.C, x.C, a1, st));
        t.fin();
        break;
      }
      case kFrVscale: {
        const FrVal& p = vals[nd.in1];
        t.beg(D2IP_KCLASS_MISC, 4.0 * B * nin * (4.0 * x.C + 2));
        ok(vscale_f32(y.g, p.v, x.g, (long long)B * nin, x.C, a0, st));
        ok(vdot_f32(y.g, x.v, p.g, (long long)B * nin, x.C, a1, st));
        t.fin();
        break;
      }
      case kFrUp: {
        t.beg(D2IP_KCLASS_UP_BWD, 4.0 * B * (nin + nout) * x.C);
        float* dl = a0 ? tmp : x.g;
        ok(upsample_concat_bwd_f32(y.g, dl, nullptr, B, din, dout, x.C, 0, st));
        if (a0) ok(accum_f32(x.g, tmp, (long long)B * nin * x.C, 1, st));
        t.fin();
        break;
      }
      case kFrUpcat: {
        const FrVal& s = vals[nd.in1];
        t.beg(D2IP_KCLASS_UP_BWD, 4.0 * B * (nin * x.C + nout * (x.C + 2.0 * s.C)));
        float* dl = a0 ? tmp : x.g;
        float* dsk = a1 ? tmp2 : s.g;
        ok(upsample_concat_bwd_f32(y.g, dl, dsk, B, din, dout, x.C, s.C, st));
        if (a0) ok(accum_f32(x.g, tmp, (long long)B * nin * x.C, 1, st));
        if (a1) ok(accum_f32(s.g, tmp2, (long long)B * nout * s.C, 1, st));
        t.fin();
        break;
      }
      case kFrSlice:
        t.beg(D2IP_KCLASS_MISC, 8.0 * B * nin * x.C);
        ok(slice_f32(y.g, y.C, nd.off, x.g, x.C, 0, x.C, (long long)B * nin, a0, st));
        t.fin();
        break;
      default:
        ok(cudaErrorInvalidValue);
    }
  }
  return e;
}

}  // namespace d2ip
