// LayerNorm(+residual)(+LeakyReLU) forward/backward, trilinear up + concat and its adjoint,
// the data term (J x - dv, J^T r, FP64 loss), FP64 column normalisation of J, ERR, Adam.
#include <cmath>

#include "common.cuh"

namespace d2ip {
namespace {

// ------------------------------------------------------------------------------------
// LayerNorm over the channel vector of a voxel.  A group of GP lanes (power of two)
// serves one voxel; lane l holds channels 4l .. 4l+3 (C <= 4*GP, C % 4 == 0).
// ------------------------------------------------------------------------------------
template <int GP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = GP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GP);
  return v;
}

// Four consecutive floats from an address that need not be 16-byte aligned (LayerNorm
// parameters sit at arbitrary offsets of the parameter arena).
__device__ __forceinline__ float4 ld4_any(const float* p) {
  return make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
}

template <int GP>
__global__ void __launch_bounds__(256)
ln_fwd_kernel(const float* __restrict__ z, const float* __restrict__ gamma,
              const float* __restrict__ resid, float* __restrict__ y, float* __restrict__ xhat,
              float* __restrict__ rstd, long long nvox, int C, int act, long long g_bs,
              __nv_bfloat16* __restrict__ ybf, int sp) {
  const int b = blockIdx.y;
  const long long off = (long long)b * nvox * C;
  const float* beta = gamma + b * g_bs + C;
  gamma += b * g_bs;
  const int lane = threadIdx.x % GP;
  const long long vox = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / GP;
  const int c = lane * 4;
  const bool on = vox < nvox && c < C;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (on) v = *reinterpret_cast<const float4*>(z + off + vox * C + c);
  const float inv_c = 1.0f / (float)C;
  const float mean = group_sum<GP>(v.x + v.y + v.z + v.w) * inv_c;
  float4 d = make_float4(v.x - mean, v.y - mean, v.z - mean, v.w - mean);
  if (!on) d = make_float4(0.f, 0.f, 0.f, 0.f);
  const float var = group_sum<GP>(d.x * d.x + d.y * d.y + d.z * d.z + d.w * d.w) * inv_c;
  const float rs = 1.0f / sqrtf(var + kLnEps);
  if (!on) return;
  const float4 g = ld4_any(gamma + c);
  const float4 be = ld4_any(beta + c);
  float4 xh = make_float4(d.x * rs, d.y * rs, d.z * rs, d.w * rs);
  float4 o = make_float4(fmaf(xh.x, g.x, be.x), fmaf(xh.y, g.y, be.y), fmaf(xh.z, g.z, be.z),
                         fmaf(xh.w, g.w, be.w));
  if (resid) {
    const float4 r = *reinterpret_cast<const float4*>(resid + off + vox * C + c);
    o.x += r.x;
    o.y += r.y;
    o.z += r.z;
    o.w += r.w;
  }
  if (act) {
    o.x = o.x > 0.f ? o.x : kLeakySlope * o.x;
    o.y = o.y > 0.f ? o.y : kLeakySlope * o.y;
    o.z = o.z > 0.f ? o.z : kLeakySlope * o.z;
    o.w = o.w > 0.f ? o.w : kLeakySlope * o.w;
  }
  *reinterpret_cast<float4*>(y + off + vox * C + c) = o;
  if (ybf) stage_bf16x4(ybf + (off + vox * C) * sp, C, c, o, sp);  // next conv's BF16 input
  *reinterpret_cast<float4*>(xhat + off + vox * C + c) = xh;
  if (lane == 0) rstd[(long long)b * nvox + vox] = rs;
}

// dpre = dy * act'(.) (mask from the stored activation output), dz = LN backward of dpre
// (FP32 into dz and/or BF16 staging into dzbf; either may be null), dt = dpre (optional);
// per-block partial sums of (dgamma, dbeta).
template <int GP>
__global__ void __launch_bounds__(256)
ln_bwd_kernel(const float* __restrict__ dy, const float* __restrict__ act_out,
              const float* __restrict__ xhat, const float* __restrict__ rstd,
              const float* __restrict__ gamma, float* __restrict__ dz, float* __restrict__ dt,
              float* __restrict__ part, long long nvox, int C, long long g_bs,
              __nv_bfloat16* __restrict__ dzbf, __nv_bfloat16* __restrict__ dtbf, int sp) {
  constexpr int kGroups = 256 / GP;
  __shared__ float red[kGroups][2 * 4 * GP];
  const int b = blockIdx.y;
  const long long off = (long long)b * nvox * C;
  gamma += b * g_bs;
  const int lane = threadIdx.x % GP;
  const int grp = threadIdx.x / GP;
  const int c = lane * 4;
  const bool con = c < C;
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  if (con) g = ld4_any(gamma + c);
  const float inv_c = 1.0f / (float)C;
  float ag[4] = {0.f, 0.f, 0.f, 0.f}, ab[4] = {0.f, 0.f, 0.f, 0.f};
  const long long step = (long long)gridDim.x * kGroups;
  for (long long base = (long long)blockIdx.x * kGroups; base < nvox; base += step) {
    const long long vox = base + grp;
    const bool on = vox < nvox && con;
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f), xh = d;
    float rs = 0.f;
    if (on) {
      d = *reinterpret_cast<const float4*>(dy + off + vox * C + c);
      xh = *reinterpret_cast<const float4*>(xhat + off + vox * C + c);
      rs = rstd[(long long)b * nvox + vox];
      if (act_out) {
        const float4 a = *reinterpret_cast<const float4*>(act_out + off + vox * C + c);
        d.x = a.x > 0.f ? d.x : kLeakySlope * d.x;
        d.y = a.y > 0.f ? d.y : kLeakySlope * d.y;
        d.z = a.z > 0.f ? d.z : kLeakySlope * d.z;
        d.w = a.w > 0.f ? d.w : kLeakySlope * d.w;
      }
      if (dt) *reinterpret_cast<float4*>(dt + off + vox * C + c) = d;
      if (dtbf) stage_bf16x4(dtbf + (off + vox * C) * sp, C, c, d, sp);
    }
    const float4 dx = make_float4(d.x * g.x, d.y * g.y, d.z * g.z, d.w * g.w);
    const float s1 = group_sum<GP>(dx.x + dx.y + dx.z + dx.w) * inv_c;
    const float s2 =
        group_sum<GP>(dx.x * xh.x + dx.y * xh.y + dx.z * xh.z + dx.w * xh.w) * inv_c;
    if (on) {
      float4 o;
      o.x = rs * (dx.x - s1 - xh.x * s2);
      o.y = rs * (dx.y - s1 - xh.y * s2);
      o.z = rs * (dx.z - s1 - xh.z * s2);
      o.w = rs * (dx.w - s1 - xh.w * s2);
      if (dz) *reinterpret_cast<float4*>(dz + off + vox * C + c) = o;
      if (dzbf) stage_bf16x4(dzbf + (off + vox * C) * sp, C, c, o, sp);
      ag[0] += d.x * xh.x;
      ag[1] += d.y * xh.y;
      ag[2] += d.z * xh.z;
      ag[3] += d.w * xh.w;
      ab[0] += d.x;
      ab[1] += d.y;
      ab[2] += d.z;
      ab[3] += d.w;
    }
  }
  for (int i = 0; i < 4; ++i) {
    red[grp][c + i] = ag[i];
    red[grp][4 * GP + c + i] = ab[i];
  }
  __syncthreads();
  float* out = part + ((long long)b * gridDim.x + blockIdx.x) * 2 * C;
  for (int ch = threadIdx.x; ch < 2 * C; ch += blockDim.x) {
    const int col = ch < C ? ch : 4 * GP + (ch - C);
    float s = 0.f;
    for (int q = 0; q < kGroups; ++q) s += red[q][col];
    out[ch] = s;
  }
}

inline int lanes_for(int C) {
  const int g = (C + 3) / 4;
  int p = 1;
  while (p < g) p <<= 1;
  return p;
}

// ------------------------------------------------------------------------------------
// trilinear resampling, half-pixel centres, explicit target size
// ------------------------------------------------------------------------------------
struct AxisW {
  int i0, i1;
  float w1;
};

// src = ((2o+1) s_in - s_out) / (2 s_out), clamped at 0: integer form, exact index map.
// Sizes stay far below 2^15, so 32-bit arithmetic is exact.
__device__ __forceinline__ AxisW axis_map(int o, int s_in, int s_out) {
  int num = (2 * o + 1) * s_in - s_out;
  if (num < 0) num = 0;
  const int den = 2 * s_out;
  AxisW a;
  a.i0 = num / den;
  a.w1 = (float)(num - a.i0 * den) / (float)den;
  a.i1 = a.i0 + 1 < s_in ? a.i0 + 1 : s_in - 1;
  return a;
}

// One thread per (output voxel, group of 4 channels) of cat = [up(low), skip].
__global__ void up_concat_fwd_kernel(const float* __restrict__ low,
                                     const float* __restrict__ skip, float* __restrict__ cat,
                                     Dims3 dl, Dims3 dout, int Cu, int Cs,
                                     __nv_bfloat16* __restrict__ catbf, int sp) {
  const int b = blockIdx.y;
  const int Ct = Cu + Cs, G = Ct / 4;
  const long long nout = dout.count();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nout * G) return;
  const long long vox = e / G;
  const int c = (int)(e % G) * 4;
  float4 val;
  if (c >= Cu) {
    val = *reinterpret_cast<const float4*>(skip + ((long long)b * nout + vox) * Cs + (c - Cu));
  } else {
    const int ox = (int)(vox % dout.x);
    const int r = (int)(vox / dout.x);
    const int oy = r % dout.y, oz = r / dout.y;
    const AxisW az = axis_map(oz, dl.z, dout.z), ay = axis_map(oy, dl.y, dout.y),
                ax = axis_map(ox, dl.x, dout.x);
    const float* L = low + (long long)b * dl.count() * Cu + c;
    const int zs[2] = {az.i0, az.i1}, ys[2] = {ay.i0, ay.i1}, xs[2] = {ax.i0, ax.i1};
    const float wz[2] = {1.f - az.w1, az.w1}, wy[2] = {1.f - ay.w1, ay.w1},
                wx[2] = {1.f - ax.w1, ax.w1};
    val = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float w = wz[i] * wy[j] * wx[k];
          const float4 v = *reinterpret_cast<const float4*>(
              L + (((long long)zs[i] * dl.y + ys[j]) * dl.x + xs[k]) * Cu);
          val.x += w * v.x;
          val.y += w * v.y;
          val.z += w * v.z;
          val.w += w * v.w;
        }
  }
  if (cat) *reinterpret_cast<float4*>(cat + ((long long)b * nout + vox) * Ct + c) = val;
  if (catbf) stage_bf16x4(catbf + ((long long)b * nout + vox) * Ct * sp, Ct, c, val, sp);
}

// Factor-2 form (every output extent twice the input's): a thread takes one input voxel i
// and one group of 4 channels and writes the 2 x 2 x 2 outputs 2i + a.  Along an axis output
// 2i reads (i - 1, i) with weights (1/4, 3/4) and 2i + 1 reads (i, i + 1) with (3/4, 1/4);
// the neighbours are loaded with clamped indices, which reproduces the clamped map at the
// borders.  Groups past Cu copy the skip channels of the 8 outputs.
__global__ void __launch_bounds__(256)
up2_concat_fwd_kernel(const float* __restrict__ low, const float* __restrict__ skip,
                      float* __restrict__ cat, Dims3 dl, Dims3 dout, int Cu, int Cs,
                      __nv_bfloat16* __restrict__ catbf, int sp) {
  const int b = blockIdx.y;
  const int Ct = Cu + Cs, G = Ct / 4;
  const long long nl = dl.count();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nl * G) return;
  const long long vox = e / G;
  const int c = (int)(e % G) * 4;
  const int ix = (int)(vox % dl.x);
  const int rr = (int)(vox / dl.x);
  const int iy = rr % dl.y, iz = rr / dl.y;
  const long long nout = dout.count();
  float* C = cat ? cat + (long long)b * nout * Ct + c : nullptr;
  __nv_bfloat16* Cb = catbf ? catbf + (long long)b * nout * Ct * sp : nullptr;
  auto put = [&](int a, int bb, int cc, float4 v) {
    const long long o = ((long long)(2 * iz + a) * dout.y + (2 * iy + bb)) * dout.x + (2 * ix + cc);
    if (C) *reinterpret_cast<float4*>(C + o * Ct) = v;
    if (Cb) stage_bf16x4(Cb + o * Ct * sp, Ct, c, v, sp);
  };
  if (c >= Cu) {  // skip channels of the 8 outputs
    const float* S = skip + (long long)b * nout * Cs + (c - Cu);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const long long o =
              ((long long)(2 * iz + a) * dout.y + (2 * iy + bb)) * dout.x + (2 * ix + cc);
          put(a, bb, cc, *reinterpret_cast<const float4*>(S + o * Cs));
        }
    return;
  }
  const float* L = low + (long long)b * nl * Cu + c;
  const int zs[3] = {iz > 0 ? iz - 1 : 0, iz, iz + 1 < dl.z ? iz + 1 : dl.z - 1};
  const int ys[3] = {iy > 0 ? iy - 1 : 0, iy, iy + 1 < dl.y ? iy + 1 : dl.y - 1};
  const int xs[3] = {ix > 0 ? ix - 1 : 0, ix, ix + 1 < dl.x ? ix + 1 : dl.x - 1};
  // along x first: for each (z, y) neighbour row the two x outputs
  float4 rx[3][3][2];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 v[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        v[i] = *reinterpret_cast<const float4*>(
            L + (((long long)zs[k] * dl.y + ys[j]) * dl.x + xs[i]) * Cu);
      rx[k][j][0] = make_float4(0.25f * v[0].x + 0.75f * v[1].x, 0.25f * v[0].y + 0.75f * v[1].y,
                                0.25f * v[0].z + 0.75f * v[1].z, 0.25f * v[0].w + 0.75f * v[1].w);
      rx[k][j][1] = make_float4(0.75f * v[1].x + 0.25f * v[2].x, 0.75f * v[1].y + 0.25f * v[2].y,
                                0.75f * v[1].z + 0.25f * v[2].z, 0.75f * v[1].w + 0.25f * v[2].w);
    }
  const float w[2][2] = {{0.25f, 0.75f}, {0.75f, 0.25f}};  // [output parity][first, second]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
          for (int dy = 0; dy < 2; ++dy) {
            const float wv = w[a][dz] * w[bb][dy];
            const float4 t = rx[a + dz][bb + dy][cc];
            o.x = fmaf(wv, t.x, o.x);
            o.y = fmaf(wv, t.y, o.y);
            o.z = fmaf(wv, t.z, o.z);
            o.w = fmaf(wv, t.w, o.w);
          }
        put(a, bb, cc, o);
      }
}

// Output positions along one axis that read input index i, with their weights.
__device__ __forceinline__ int axis_sources(int i, int s_in, int s_out, int* os, float* ws) {
  // outputs o with i0(o) or i1(o) == i satisfy (i - 1/2) r - 1/2 < o < (i + 3/2) r - 1/2,
  // r = s_out / s_in; scan that window (widened by one) with the exact map
  int lo = ((2 * i - 1) * s_out - s_in) / (2 * s_in) - 1;
  int hi = ((2 * i + 3) * s_out - s_in) / (2 * s_in) + 1;
  if (lo < 0) lo = 0;
  if (hi > s_out - 1) hi = s_out - 1;
  int n = 0;
  for (int o = lo; o <= hi && n < 8; ++o) {
    const AxisW a = axis_map(o, s_in, s_out);
    float w = 0.f;
    if (a.i0 == i) w += 1.f - a.w1;
    if (a.i1 == i) w += a.w1;
    if (a.i0 == i || a.i1 == i) {
      os[n] = o;
      ws[n] = w;
      ++n;
    }
  }
  return n;
}

// One thread per (low voxel, group of 4 up-sampled channels): gather of the adjoint.
__global__ void up_bwd_kernel(const float* __restrict__ dcat, float* __restrict__ dlow,
                              Dims3 dl, Dims3 dout, int Cu, int Cs) {
  const int b = blockIdx.y;
  const int Ct = Cu + Cs, G = Cu / 4;
  const long long nl = dl.count();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nl * G) return;
  const long long vox = e / G;
  const int c = (int)(e % G) * 4;
  const int ix = (int)(vox % dl.x);
  const int r = (int)(vox / dl.x);
  const int iy = r % dl.y, iz = r / dl.y;
  int oz[8], oy[8], ox[8];
  float wz[8], wy[8], wx[8];
  const int nz = axis_sources(iz, dl.z, dout.z, oz, wz);
  const int ny = axis_sources(iy, dl.y, dout.y, oy, wy);
  const int nx = axis_sources(ix, dl.x, dout.x, ox, wx);
  const float* D = dcat + (long long)b * dout.count() * Ct + c;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int a = 0; a < nz; ++a)
    for (int q = 0; q < ny; ++q)
      for (int k = 0; k < nx; ++k) {
        const float w = wz[a] * wy[q] * wx[k];
        const float4 v = *reinterpret_cast<const float4*>(
            D + (((long long)oz[a] * dout.y + oy[q]) * dout.x + ox[k]) * Ct);
        acc.x += w * v.x;
        acc.y += w * v.y;
        acc.z += w * v.z;
        acc.w += w * v.w;
      }
  *reinterpret_cast<float4*>(dlow + ((long long)b * nl + vox) * Cu + c) = acc;
}

// Factor-2 form of the adjoint (every output extent twice the low one).  Along an axis low
// index i receives from the outputs 2i-1, 2i, 2i+1, 2i+2 with weights 1/4, 3/4, 3/4, 1/4
// (the transpose of the forward's 1/4-3/4 stencil); at the borders the clamped neighbour
// folds the outer weight onto the inner one (i = 0: 2i gets 1; i = n-1: 2i+1 gets 1) and the
// taps past the edge get 0.  A thread takes two neighbouring low voxels along x (six output
// columns instead of eight) and one group of 4 channels; taps are unrolled.
__global__ void __launch_bounds__(256) up2_bwd_kernel(const float* __restrict__ dcat,
                                                      float* __restrict__ dlow, Dims3 dl,
                                                      Dims3 dout, int Cu, int Cs) {
  const int b = blockIdx.y;
  const int Ct = Cu + Cs, G = Cu / 4;
  const int hx = (dl.x + 1) / 2;  // pairs along x
  const long long npair = (long long)dl.z * dl.y * hx;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npair * G) return;
  const long long pr = e / G;
  const int c = (int)(e % G) * 4;
  const int px = (int)(pr % hx);
  const int r = (int)(pr / hx);
  const int iy = r % dl.y, iz = r / dl.y;
  const int ix0 = 2 * px;
  auto axis = [](int i, int n, float* w) {
    w[0] = i >= 1 ? 0.25f : 0.f;
    w[1] = i == 0 ? 1.f : 0.75f;
    w[2] = i == n - 1 ? 1.f : 0.75f;
    w[3] = i <= n - 2 ? 0.25f : 0.f;
  };
  float wz[4], wy[4], wa[4], wb[4];
  axis(iz, dl.z, wz);
  axis(iy, dl.y, wy);
  axis(ix0, dl.x, wa);
  const bool two = ix0 + 1 < dl.x;
  axis(ix0 + 1, dl.x, wb);
  // output x columns 2*ix0 - 1 .. 2*ix0 + 4: the first voxel uses columns 0..3, the second 2..5
  float wxa[6] = {wa[0], wa[1], wa[2], wa[3], 0.f, 0.f};
  float wxb[6] = {0.f, 0.f, wb[0], wb[1], wb[2], wb[3]};
  const float* D = dcat + (long long)b * dout.count() * Ct + c;
  float4 A = make_float4(0.f, 0.f, 0.f, 0.f), Bv = A;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int oz = 2 * iz - 1 + a;
    if (wz[a] == 0.f) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int oy = 2 * iy - 1 + q;
      if (wy[q] == 0.f) continue;
      const float wzy = wz[a] * wy[q];
      const float* row = D + ((long long)oz * dout.y + oy) * dout.x * Ct;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int ox = 2 * ix0 - 1 + k;
        if (ox < 0 || ox >= dout.x) continue;
        const float ka = wxa[k], kb = two ? wxb[k] : 0.f;
        if (ka == 0.f && kb == 0.f) continue;
        const float4 v = *reinterpret_cast<const float4*>(row + (long long)ox * Ct);
        const float fa = wzy * ka, fb = wzy * kb;
        A.x += fa * v.x;
        A.y += fa * v.y;
        A.z += fa * v.z;
        A.w += fa * v.w;
        Bv.x += fb * v.x;
        Bv.y += fb * v.y;
        Bv.z += fb * v.z;
        Bv.w += fb * v.w;
      }
    }
  }
  float* O = dlow + ((long long)b * dl.count() + ((long long)iz * dl.y + iy) * dl.x + ix0) * Cu + c;
  *reinterpret_cast<float4*>(O) = A;
  if (two) *reinterpret_cast<float4*>(O + Cu) = Bv;
}

// The same factor-2 adjoint through shared memory: a CTA takes 8 x 4 x 2 low voxels and 8
// channels, loads the 18 x 10 x 6 output voxels they read (zeros outside the grid), and
// applies the transposed stencil one axis at a time (z, then y, then x).  Each output value
// is read about twice instead of eight times, and a low value costs 4 + 4 + 4 weighted taps
// per staged line instead of 64 scattered loads.
constexpr int kU2X = 8, kU2Y = 4, kU2Z = 2;
__device__ __forceinline__ float up2_adj_w(int i, int n, int a) {  // tap a: output 2i - 1 + a
  return a == 0 ? (i >= 1 ? 0.25f : 0.f)
       : a == 1 ? (i == 0 ? 1.f : 0.75f)
       : a == 2 ? (i == n - 1 ? 1.f : 0.75f)
                : (i <= n - 2 ? 0.25f : 0.f);
}
__device__ __forceinline__ void fma4(float4& o, float w, const float4& v) {
  o.x = fmaf(w, v.x, o.x), o.y = fmaf(w, v.y, o.y), o.z = fmaf(w, v.z, o.z), o.w = fmaf(w, v.w, o.w);
}

__global__ void __launch_bounds__(256) up2_bwd_tile_kernel(const float* __restrict__ dcat,
                                                           float* __restrict__ dlow, Dims3 dl,
                                                           Dims3 dout, int Cu, int Ct) {
  constexpr int FX = 2 * kU2X + 2, FY = 2 * kU2Y + 2, FZ = 2 * kU2Z + 2;
  __shared__ float4 F[FZ][FY][FX][2];   // output tile (8 channels: two float4)
  __shared__ float4 T1[kU2Z][FY][FX][2];  // after the z pass
  float4 (*T2)[kU2Y][FX][2] = reinterpret_cast<float4 (*)[kU2Y][FX][2]>(&F[0][0][0][0]);
  const int b = blockIdx.y;
  const int ncg = Cu / 8;
  const int cg = blockIdx.x % ncg, tile = blockIdx.x / ncg;  // channel groups of a tile adjacent
  const int tx = (dl.x + kU2X - 1) / kU2X, ty = (dl.y + kU2Y - 1) / kU2Y;
  const int lx0 = (tile % tx) * kU2X, ly0 = ((tile / tx) % ty) * kU2Y,
            lz0 = (tile / (tx * ty)) * kU2Z;
  const int c0 = cg * 8;
  const float* D = dcat + (long long)b * dout.count() * Ct + c0;
  for (int e = threadIdx.x; e < FZ * FY * FX * 2; e += blockDim.x) {
    const int h = e & 1, fx = (e >> 1) % FX, fy = (e >> 1) / FX % FY, fz = (e >> 1) / (FX * FY);
    const int ox = 2 * lx0 - 1 + fx, oy = 2 * ly0 - 1 + fy, oz = 2 * lz0 - 1 + fz;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ox >= 0 && ox < dout.x && oy >= 0 && oy < dout.y && oz >= 0 && oz < dout.z)
      v = *reinterpret_cast<const float4*>(
          D + (((long long)oz * dout.y + oy) * dout.x + ox) * Ct + 4 * h);
    F[fz][fy][fx][h] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kU2Z * FY * FX * 2; e += blockDim.x) {  // z
    const int h = e & 1, fx = (e >> 1) % FX, fy = (e >> 1) / FX % FY, lz = (e >> 1) / (FX * FY);
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a) fma4(o, up2_adj_w(lz0 + lz, dl.z, a), F[2 * lz + a][fy][fx][h]);
    T1[lz][fy][fx][h] = o;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kU2Z * kU2Y * FX * 2; e += blockDim.x) {  // y (into F's space)
    const int h = e & 1, fx = (e >> 1) % FX, ly = (e >> 1) / FX % kU2Y, lz = (e >> 1) / (FX * kU2Y);
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a) fma4(o, up2_adj_w(ly0 + ly, dl.y, a), T1[lz][2 * ly + a][fx][h]);
    T2[lz][ly][fx][h] = o;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kU2Z * kU2Y * kU2X * 2; e += blockDim.x) {  // x, then store
    const int h = e & 1, lx = (e >> 1) % kU2X, ly = (e >> 1) / kU2X % kU2Y,
              lz = (e >> 1) / (kU2X * kU2Y);
    const int ix = lx0 + lx, iy = ly0 + ly, iz = lz0 + lz;
    if (ix >= dl.x || iy >= dl.y || iz >= dl.z) continue;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a) fma4(o, up2_adj_w(ix, dl.x, a), T2[lz][ly][2 * lx + a][h]);
    *reinterpret_cast<float4*>(
        dlow + ((long long)b * dl.count() + ((long long)iz * dl.y + iy) * dl.x + ix) * Cu + c0 +
        4 * h) = o;
  }
}

__global__ void split_skip_kernel(const float* __restrict__ dcat, float* __restrict__ dskip,
                                  long long nout, int Cu, int Cs) {
  const int b = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nout * Cs) return;
  const long long vox = e / Cs;
  const int c = (int)(e % Cs);
  dskip[((long long)b * nout + vox) * Cs + c] =
      dcat[((long long)b * nout + vox) * (Cu + Cs) + Cu + c];
}

__global__ void add_kernel(float* __restrict__ y, const float* __restrict__ x, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

// ------------------------------------------------------------------------------------
// data term
// ------------------------------------------------------------------------------------
constexpr int kJB = 8;  // problems per block in the J kernels
constexpr int kJtmulMaxSmem = 200 * 1024;

// r[b][i] = sum_j J[i][j] x[b][j] - dv[b][i], in two deterministic stages.  Stage 1: a block
// takes 1024 columns (4 per thread, float4) of kJRows rows for kJB problems and writes the
// block's partial sums; stage 2 adds the column chunks in order and subtracts dv.
constexpr int kJRows = 4;
constexpr int kJCols = 1024;
constexpr int kTCols = 64, kTB = 16;  // transposed-J (BF16) forms: columns per block, problems

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float4 load4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

template <typename JT>
__global__ void __launch_bounds__(256)
jmul_part_kernel(const JT* __restrict__ J, const float* __restrict__ x,
                 float* __restrict__ part, int B, int m, int n, long long x_bs) {
  __shared__ float red[8][kJRows * kJB];
  const int chunk = blockIdx.x;
  const int i0 = blockIdx.y * kJRows;
  const int b0 = blockIdx.z * kJB;
  const int nb = B - b0 < kJB ? B - b0 : kJB;
  const int nr = m - i0 < kJRows ? m - i0 : kJRows;
  float acc[kJRows][kJB];
#pragma unroll
  for (int r = 0; r < kJRows; ++r)
#pragma unroll
    for (int q = 0; q < kJB; ++q) acc[r][q] = 0.f;
  const int j = chunk * kJCols + threadIdx.x * 4;
  if (j + 3 < n && (n & 3) == 0) {
    float4 xv[kJB];
#pragma unroll
    for (int q = 0; q < kJB; ++q)
      xv[q] = q < nb ? *reinterpret_cast<const float4*>(x + (long long)(b0 + q) * x_bs + j)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kJRows; ++r) {
      if (r >= nr) break;
      const float4 a = load4(J + (long long)(i0 + r) * n + j);
#pragma unroll
      for (int q = 0; q < kJB; ++q)
        acc[r][q] = fmaf(a.x, xv[q].x, fmaf(a.y, xv[q].y, fmaf(a.z, xv[q].z,
                                                            fmaf(a.w, xv[q].w, acc[r][q]))));
    }
  } else {
    for (int jj = j; jj < j + 4 && jj < n; ++jj)
      for (int r = 0; r < nr; ++r) {
        const float a = to_f32(J[(long long)(i0 + r) * n + jj]);
        for (int q = 0; q < nb; ++q) acc[r][q] = fmaf(a, x[(long long)(b0 + q) * x_bs + jj], acc[r][q]);
      }
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
#pragma unroll
  for (int r = 0; r < kJRows; ++r)
#pragma unroll
    for (int q = 0; q < kJB; ++q) {
      float v = acc[r][q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) red[w][r * kJB + q] = v;
    }
  __syncthreads();
  if (threadIdx.x < kJRows * kJB) {
    const int r = threadIdx.x / kJB, q = threadIdx.x % kJB;
    if (r < nr && q < nb) {
      float v = 0.f;
      for (int k = 0; k < 8; ++k) v += red[k][threadIdx.x];
      part[((long long)chunk * B + b0 + q) * m + i0 + r] = v;
    }
  }
}

// r[e] = sum_c part[c][e] - dv[e]: 32 columns x 8 chunk groups per block, the groups' sums
// added in order.
__global__ void __launch_bounds__(256)
jmul_final_many_kernel(const float* __restrict__ part, const float* __restrict__ dv,
                       float* __restrict__ r, long long N, int nchunks) {
  __shared__ float red[8][33];
  const int col = threadIdx.x % 32, grp = threadIdx.x / 32;
  const long long e = (long long)blockIdx.x * 32 + col;
  float s0 = 0.f, s1 = 0.f;
  if (e < N) {
    int c = grp;
    for (; c + 8 < nchunks; c += 16) {
      s0 += part[(long long)c * N + e];
      s1 += part[(long long)(c + 8) * N + e];
    }
    if (c < nchunks) s0 += part[(long long)c * N + e];
  }
  red[grp][col] = s0 + s1;
  __syncthreads();
  if (grp == 0 && e < N) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += red[q][col];
    r[e] = s - dv[e];
  }
}


template <typename JT>
__global__ void __launch_bounds__(256)
jtmul_kernel(const JT* __restrict__ J, const float* __restrict__ r, float* __restrict__ g,
             float scale, int B, int m, int n, long long g_bs) {
  extern __shared__ float rs[];  // [kJB][m]
  const int b0 = blockIdx.y * kJB;
  const int nb = B - b0 < kJB ? B - b0 : kJB;
  for (int e = threadIdx.x; e < nb * m; e += blockDim.x) rs[e] = r[(long long)b0 * m + e];
  __syncthreads();
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float acc[kJB];
#pragma unroll
  for (int q = 0; q < kJB; ++q) acc[q] = 0.f;
  for (int i = 0; i < m; ++i) {
    const float a = to_f32(J[(long long)i * n + j]);
#pragma unroll
    for (int q = 0; q < kJB; ++q)
      if (q < nb) acc[q] = fmaf(a, rs[q * m + i], acc[q]);
  }
  for (int q = 0; q < nb; ++q) g[(long long)(b0 + q) * g_bs + j] = scale * acc[q];
}

__global__ void __launch_bounds__(1024)
loss_kernel(const float* __restrict__ r, double* __restrict__ loss, double* __restrict__ trace,
            int* __restrict__ trace_pos, int trace_cap, int* __restrict__ adam_t,
            int* __restrict__ status, int B, int m, const double* __restrict__ reg_part,
            int reg_blocks) {
  // one warp per problem (problems w, w + nw, ...): lanes add i = lane, lane + 32, ... in
  // order, then a fixed butterfly over the lanes
  __shared__ int bad_s;
  const int pos = trace_pos ? *trace_pos : 0;
  const int slot = trace_cap > 0 ? pos % trace_cap : 0;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  if (threadIdx.x == 0) bad_s = 0;
  __syncthreads();
  for (int b = warp; b < B; b += nw) {
    double s = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double v = (double)r[(long long)b * m + i];
      s += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      double L = s / (double)m;
      if (reg_part)
        for (int k = 0; k < reg_blocks; ++k) L += reg_part[(long long)b * reg_blocks + k];
      loss[b] = L;
      if (trace) trace[(long long)slot * B + b] = L;
      if (!isfinite(L)) atomicOr(&bad_s, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (trace_pos) *trace_pos = pos + 1;
    if (adam_t) *adam_t += 1;
    if (bad_s && status) *status |= 1;
  }
}

// 4D-TV regulariser (Sec. III-E).  Per voxel v of frame i (previous outputs h_0..h_{i-1}):
//   spatial  (1/V) sqrt(d_x^2 + d_y^2 + d_z^2 + eps), forward differences, 0 past the far face;
//   temporal (1/sum a) sum_j a_j sqrt((s - h_j)^2 + eps), a_j = exp(-(i - j)).
// g[v] += lam_s' dR_s/ds[v] + lam_t' dR_t/ds[v] with lam_s' = lam*lam_s, lam_t' = lam*lam_t;
// part[b][block] = the block's share of lam_s' R_s + lam_t' R_t (FP64, fixed order).
__device__ __forceinline__ float tv_mag(const float* s, int x, int y, int z, Dims3 d, float eps,
                                        float* dxo, float* dyo, float* dzo) {
  const long long v = ((long long)z * d.y + y) * d.x + x;
  const float c = s[v];
  const float dx = x + 1 < d.x ? s[v + 1] - c : 0.f;
  const float dy = y + 1 < d.y ? s[v + d.x] - c : 0.f;
  const float dz = z + 1 < d.z ? s[v + (long long)d.x * d.y] - c : 0.f;
  *dxo = dx;
  *dyo = dy;
  *dzo = dz;
  return sqrtf(dx * dx + dy * dy + dz * dz + eps);
}

// d mag(u) / d s[u + e_axis] = (its forward difference along axis) / mag(u).
__device__ __forceinline__ float bx_over(const float* s, int x, int y, int z, Dims3 d, float eps,
                                         int axis) {
  float dx, dy, dz;
  const float m = tv_mag(s, x, y, z, d, eps, &dx, &dy, &dz);
  return (axis == 0 ? dx : axis == 1 ? dy : dz) / m;
}

__global__ void __launch_bounds__(256)
tv4d_kernel(const float* __restrict__ ds, const float* __restrict__ hist,
            const int* __restrict__ nprev_dev, float* __restrict__ g, double* __restrict__ part,
            Dims3 d, long long hist_bs, float lam_s, float lam_t, float eps) {
  __shared__ double red[256];
  const int b = blockIdx.y;
  const long long n = d.count();
  const float* s = ds + (long long)b * n;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double val = 0.0;
  if (v < n) {
    const int x = (int)(v % d.x), y = (int)((v / d.x) % d.y), z = (int)(v / ((long long)d.x * d.y));
    float ax, ay, az;
    const float mag = tv_mag(s, x, y, z, d, eps, &ax, &ay, &az);
    float grad = -(ax + ay + az) / mag;  // d mag(v) / d s[v]
    // the backward neighbours' magnitudes also contain s[v]
    if (x > 0) grad += bx_over(s, x - 1, y, z, d, eps, 0);
    if (y > 0) grad += bx_over(s, x, y - 1, z, d, eps, 1);
    if (z > 0) grad += bx_over(s, x, y, z - 1, d, eps, 2);
    float gt = 0.f, vt = 0.f;
    const int np = nprev_dev ? *nprev_dev : 0;
    if (np > 0) {
      float asum = 0.f;
      for (int j = 0; j < np; ++j) {
        const float a = expf(-(float)(np - j));
        const float diff = s[v] - hist[(long long)b * hist_bs + (long long)j * n + v];
        const float q = sqrtf(diff * diff + eps);
        asum += a;
        vt += a * q;
        gt += a * diff / q;
      }
      gt /= asum;
      vt /= asum;
    }
    g[(long long)b * n + v] += lam_s * grad + lam_t * gt;
    val = (double)lam_s * mag + (double)lam_t * vt;
  }
  red[threadIdx.x] = val;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)b * gridDim.x + blockIdx.x] = red[0];
}

__global__ void colnorm_kernel(float* __restrict__ J, double* __restrict__ cn, int m, int n) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) {
    const double v = (double)J[(long long)i * n + j];
    s += v * v;
  }
  const double c = sqrt(s);
  cn[j] = c;
  if (c > 0.0)
    for (int i = 0; i < m; ++i) J[(long long)i * n + j] = (float)((double)J[(long long)i * n + j] / c);
}

__global__ void err_kernel(const float* __restrict__ est, const float* __restrict__ truth,
                           double* __restrict__ out, long long n) {
  __shared__ double ra[256], rb[256];
  const int b = blockIdx.x;
  double a = 0.0, t = 0.0;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) {
    const double e = (double)est[b * n + j], g = (double)truth[b * n + j];
    a += (e - g) * (e - g);
    t += g * g;
  }
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ra[threadIdx.x] += ra[threadIdx.x + o];
      rb[threadIdx.x] += rb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = sqrt(ra[0] / rb[0]);
}

__global__ void __launch_bounds__(256)
adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
            float* __restrict__ v, long long count, float lr, float b1f, float b2f, float o1,
            float o2, float lnb1, float lnb2, float eps, const int* __restrict__ t_dev,
            int t_host) {
  // beta and (1 - beta) come rounded to float from double, so (1 - 0.999) keeps full float
  // precision.  The bias corrections 1 - beta^t = -expm1(t ln beta), with ln beta formed in
  // double on the host: about 2e-7 relative error, with no FP64 work on the device.
  const float tf = (float)(t_dev ? *t_dev : t_host);
  const float ibc1 = -1.f / expm1f(tf * lnb1), ibc2 = -1.f / expm1f(tf * lnb2);
  auto upd = [&](float gi, float& mi, float& vi, float& th) {
    mi = fmaf(b1f, mi, o1 * gi);
    vi = fmaf(b2f, vi, o2 * gi * gi);
    th -= lr * (mi * ibc1) / (sqrtf(vi * ibc2) + eps);
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = (count & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(g) |
                     reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  if (vec) {  // four parameters per thread and step, the same arithmetic per element
    for (long long i = i0; i < count / 4; i += stride) {
      const float4 gi = reinterpret_cast<const float4*>(g)[i];
      float4 mi = reinterpret_cast<float4*>(m)[i], vi = reinterpret_cast<float4*>(v)[i],
             th = reinterpret_cast<float4*>(theta)[i];
      upd(gi.x, mi.x, vi.x, th.x);
      upd(gi.y, mi.y, vi.y, th.y);
      upd(gi.z, mi.z, vi.z, th.z);
      upd(gi.w, mi.w, vi.w, th.w);
      reinterpret_cast<float4*>(m)[i] = mi;
      reinterpret_cast<float4*>(v)[i] = vi;
      reinterpret_cast<float4*>(theta)[i] = th;
    }
    return;
  }
  for (long long i = i0; i < count; i += stride) {
    float mi = m[i], vi = v[i], th = theta[i];
    upd(g[i], mi, vi, th);
    m[i] = mi;
    v[i] = vi;
    theta[i] = th;
  }
}

}  // namespace

int tv4d_blocks(long long n) { return (int)ceil_div(n, 256); }

__global__ void set_int_kernel(int* p, int v) { *p = v; }

cudaError_t set_device_int(int* p, int v, cudaStream_t stream) {
  set_int_kernel<<<1, 1, 0, stream>>>(p, v);
  return cudaGetLastError();
}

cudaError_t tv4d_f32(const float* ds, const float* hist, const int* nprev_dev, float* g,
                     double* part, int B, Dims3 d, long long hist_bs, float lam_s, float lam_t,
                     float eps, cudaStream_t stream) {
  dim3 grid((unsigned)tv4d_blocks(d.count()), B);
  tv4d_kernel<<<grid, 256, 0, stream>>>(ds, hist, nprev_dev, g, part, d, hist_bs, lam_s, lam_t,
                                        eps);
  return cudaGetLastError();
}

int layernorm_bwd_blocks(long long nvox, int C) {
  const int gp = lanes_for(C);
  const long long need = ceil_div(nvox, 256 / gp);
  return (int)(need < 256 ? need : 256);
}

cudaError_t layernorm_act_fwd_f32(const float* z, const float* gamma, const float* resid,
                                  float* y, float* xhat, float* rstd, int B, long long nvox,
                                  int C, int act, long long g_bs, cudaStream_t stream,
                                  __nv_bfloat16* ybf, int sp) {
  if (C % 4 != 0 || C > 128) return cudaErrorInvalidValue;
  const int gp = lanes_for(C);
  dim3 grid((unsigned)ceil_div(nvox * gp, 256), B);
#define D2IP_LNF(G) \
  ln_fwd_kernel<G><<<grid, 256, 0, stream>>>(z, gamma, resid, y, xhat, rstd, nvox, C, act, g_bs, \
                                             ybf, sp)
  switch (gp) {
    case 1: D2IP_LNF(1); break;
    case 2: D2IP_LNF(2); break;
    case 4: D2IP_LNF(4); break;
    case 8: D2IP_LNF(8); break;
    case 16: D2IP_LNF(16); break;
    default: D2IP_LNF(32); break;
  }
#undef D2IP_LNF
  return cudaGetLastError();
}

cudaError_t layernorm_act_bwd_f32(const float* dy, const float* act_out, const float* xhat,
                                  const float* rstd, const float* gamma, float* dz, float* dt,
                                  float* part, int B, long long nvox, int C, long long g_bs,
                                  cudaStream_t stream, __nv_bfloat16* dzbf,
                                  __nv_bfloat16* dtbf, int sp) {
  if (C % 4 != 0 || C > 128) return cudaErrorInvalidValue;
  const int gp = lanes_for(C);
  dim3 grid(layernorm_bwd_blocks(nvox, C), B);
#define D2IP_LNB(G)                                                                          \
  ln_bwd_kernel<G><<<grid, 256, 0, stream>>>(dy, act_out, xhat, rstd, gamma, dz, dt, part, \
                                             nvox, C, g_bs, dzbf, dtbf, sp)
  switch (gp) {
    case 1: D2IP_LNB(1); break;
    case 2: D2IP_LNB(2); break;
    case 4: D2IP_LNB(4); break;
    case 8: D2IP_LNB(8); break;
    case 16: D2IP_LNB(16); break;
    default: D2IP_LNB(32); break;
  }
#undef D2IP_LNB
  return cudaGetLastError();
}

cudaError_t upsample_concat_fwd_f32(const float* low, const float* skip, float* cat, int B,
                                    Dims3 dlow, Dims3 dout, int Cu, int Cs,
                                    cudaStream_t stream, __nv_bfloat16* catbf, int sp) {
  if (Cu % 4 || Cs % 4 || (!cat && !catbf)) return cudaErrorInvalidValue;
  const long long total = dout.count() * ((Cu + Cs) / 4);
  dim3 grid((unsigned)ceil_div(total, 256), B);
  if (dout.x == 2 * dlow.x && dout.y == 2 * dlow.y && dout.z == 2 * dlow.z) {
    dim3 g2((unsigned)ceil_div(dlow.count() * ((Cu + Cs) / 4), 256), B);
    up2_concat_fwd_kernel<<<g2, 256, 0, stream>>>(low, skip, cat, dlow, dout, Cu, Cs, catbf,
                                                  sp);
    return cudaGetLastError();
  }
  up_concat_fwd_kernel<<<grid, 256, 0, stream>>>(low, skip, cat, dlow, dout, Cu, Cs, catbf, sp);
  return cudaGetLastError();
}

cudaError_t upsample_concat_bwd_f32(const float* dcat, float* dlow, float* dskip, int B,
                                    Dims3 dlow_dims, Dims3 dout, int Cu, int Cs,
                                    cudaStream_t stream) {
  if (Cu % 4 || Cs % 4) return cudaErrorInvalidValue;
  if (dout.x == 2 * dlow_dims.x && dout.y == 2 * dlow_dims.y && dout.z == 2 * dlow_dims.z &&
      Cu % 8 == 0) {
    const long long tiles = ceil_div(dlow_dims.x, kU2X) * ceil_div(dlow_dims.y, kU2Y) *
                            ceil_div(dlow_dims.z, kU2Z);
    dim3 g2((unsigned)(tiles * (Cu / 8)), B);
    up2_bwd_tile_kernel<<<g2, 256, 0, stream>>>(dcat, dlow, dlow_dims, dout, Cu, Cu + Cs);
  } else if (dout.x == 2 * dlow_dims.x && dout.y == 2 * dlow_dims.y &&
             dout.z == 2 * dlow_dims.z) {
    const long long pairs = (long long)dlow_dims.z * dlow_dims.y * ((dlow_dims.x + 1) / 2);
    dim3 g2((unsigned)ceil_div(pairs * (Cu / 4), 256), B);
    up2_bwd_kernel<<<g2, 256, 0, stream>>>(dcat, dlow, dlow_dims, dout, Cu, Cs);
  } else {
    dim3 g1((unsigned)ceil_div(dlow_dims.count() * (Cu / 4), 256), B);
    up_bwd_kernel<<<g1, 256, 0, stream>>>(dcat, dlow, dlow_dims, dout, Cu, Cs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !dskip || Cs == 0) return e;
  dim3 g2((unsigned)ceil_div(dout.count() * Cs, 256), B);
  split_skip_kernel<<<g2, 256, 0, stream>>>(dcat, dskip, dout.count(), Cu, Cs);
  return cudaGetLastError();
}

cudaError_t add_inplace_f32(float* y, const float* x, long long count, cudaStream_t stream) {
  add_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, stream>>>(y, x, count);
  return cudaGetLastError();
}

int jmul_chunks(int n) {
  const long long a = ceil_div(n, kJCols), b = ceil_div(n, kTCols);
  return (int)(a > b ? a : b);
}

template <typename JT>
cudaError_t jmul_impl(const JT* J, const float* x, const float* dv, float* r, float* part, int B,
                      int m, int n, long long x_bs, cudaStream_t stream) {
  const int nch = jmul_chunks(n);
  dim3 grid(nch, (unsigned)ceil_div(m, kJRows), (unsigned)ceil_div(B, kJB));
  jmul_part_kernel<JT><<<grid, 256, 0, stream>>>(J, x, part, B, m, n, x_bs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  jmul_final_many_kernel<<<(unsigned)ceil_div((long long)B * m, 32), 256, 0, stream>>>(
      part, dv, r, (long long)B * m, nch);
  return cudaGetLastError();
}

cudaError_t jmul_residual_f32(const float* J, const float* x, const float* dv, float* r,
                              float* part, int B, int m, int n, long long x_bs,
                              cudaStream_t stream) {
  return jmul_impl(J, x, dv, r, part, B, m, n, x_bs, stream);
}

// ---- BF16 paths: J stored transposed, Jt[n][m] (BF16) ------------------------------
// r[b][i] = sum_j Jt[j][i] x[b][j] - dv[b][i]: a block takes kTCols columns j for up to kTB
// problems; thread t owns the row pairs i = 2 p, 2 p + 1 (p = t + 256 s) and adds j in order;
// per-block partial sums, then the chunks in order (jmul_final_kernel).  SPLIT: J is the sum
// of two BF16 copies, Jt (hi) + Jlo (lo = bf16(J - hi)), added in FP32 before the product.
template <int SLOTS, bool SPLIT>
__global__ void __launch_bounds__(256)
jmul_t_kernel(const __nv_bfloat16* __restrict__ Jt, const __nv_bfloat16* __restrict__ Jlo,
              const float* __restrict__ x, float* __restrict__ part, int B, int m, int n,
              long long x_bs) {
  __shared__ __align__(16) float xs[kTB][kTCols];
  const int chunk = blockIdx.x, b0 = blockIdx.y * kTB;
  const int nb = B - b0 < kTB ? B - b0 : kTB;
  const int j0 = chunk * kTCols;
  const int nj = n - j0 < kTCols ? n - j0 : kTCols;
  for (int e = threadIdx.x; e < kTB * kTCols; e += blockDim.x) {
    const int q = e / kTCols, jj = e % kTCols;
    xs[q][jj] = (q < nb && jj < nj) ? x[(long long)(b0 + q) * x_bs + j0 + jj] : 0.f;
  }
  __syncthreads();
  float acc[SLOTS][2][kTB];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s)
#pragma unroll
    for (int q = 0; q < kTB; ++q) acc[s][0][q] = acc[s][1][q] = 0.f;
  const int np = m / 2;
  // four columns per step: their J pairs from global memory, x from shared memory as float4
  // (columns past n carry x = 0 and read row n - 1, which exists)
  for (int jj = 0; jj < nj; jj += 4) {
    const __nv_bfloat162* rows[4];
    const __nv_bfloat162* rlo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jr = j0 + jj + u < n ? j0 + jj + u : n - 1;
      rows[u] = reinterpret_cast<const __nv_bfloat162*>(Jt + (long long)jr * m);
      if (SPLIT) rlo[u] = reinterpret_cast<const __nv_bfloat162*>(Jlo + (long long)jr * m);
    }
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int pi = threadIdx.x + 256 * s;
      if (pi >= np) break;
      float2 a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = __bfloat1622float2(rows[u][pi]);
        if (SPLIT) {
          const float2 l = __bfloat1622float2(rlo[u][pi]);
          a[u].x += l.x, a[u].y += l.y;
        }
      }
#pragma unroll
      for (int q = 0; q < kTB; ++q) {
        const float4 xv = *reinterpret_cast<const float4*>(&xs[q][jj]);
        acc[s][0][q] = fmaf(a[3].x, xv.w, fmaf(a[2].x, xv.z, fmaf(a[1].x, xv.y, fmaf(a[0].x, xv.x, acc[s][0][q]))));
        acc[s][1][q] = fmaf(a[3].y, xv.w, fmaf(a[2].y, xv.z, fmaf(a[1].y, xv.y, fmaf(a[0].y, xv.x, acc[s][1][q]))));
      }
    }
  }
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int pi = threadIdx.x + 256 * s;
    if (pi >= np) break;
#pragma unroll
    for (int q = 0; q < kTB; ++q)
      if (q < nb) {
        float* o = part + ((long long)chunk * B + b0 + q) * m + 2 * pi;
        o[0] = acc[s][0][q];
        o[1] = acc[s][1][q];
      }
  }
}

// g[b][j] = scale sum_i Jt[j][i] r[b][i]: a thread per column j (kJtRows per block) keeps
// the kTB problems' sums; the block stages r and, chunk by chunk along i, a tile of Jt rows
// (coalesced) in shared memory; i is added in order.  SPLIT: the tile holds hi + lo in FP32.
constexpr int kJtRows = 128, kJtChunk = 64;

template <bool SPLIT>
struct JtTile {  // element type and padded row of the shared-memory J tile
  using T = __nv_bfloat16;
  static constexpr int kLd = kJtChunk + 8;  // 144 bytes
};
template <>
struct JtTile<true> {
  using T = float;
  static constexpr int kLd = kJtChunk + 4;  // 272 bytes
};

template <bool SPLIT>
__global__ void __launch_bounds__(kJtRows)
jtmul_t_kernel(const __nv_bfloat16* __restrict__ Jt, const __nv_bfloat16* __restrict__ Jlo,
               const float* __restrict__ r, float* __restrict__ g, float scale, int B, int m,
               int n, long long g_bs) {
  extern __shared__ float rs[];  // [kTB][m], then two J tiles
  using TT = typename JtTile<SPLIT>::T;
  constexpr int kLd = JtTile<SPLIT>::kLd;
  constexpr int kPer = kJtRows * (kJtChunk / 4) / kJtRows;  // 4-element pieces per thread
  TT* jt0 = reinterpret_cast<TT*>(rs + kTB * m);  // [2][kJtRows][kLd]
  const int b0 = blockIdx.y * kTB;
  const int nb = B - b0 < kTB ? B - b0 : kTB;
  for (int e = threadIdx.x; e < kTB * m; e += blockDim.x)
    rs[e] = e < nb * m ? r[(long long)b0 * m + e] : 0.f;
  const long long j0 = (long long)blockIdx.x * kJtRows;
  const long long j = j0 + threadIdx.x;
  float acc[kTB];
#pragma unroll
  for (int q = 0; q < kTB; ++q) acc[q] = 0.f;
  // tile of chunk i0: rows j0 .. j0 + 127, columns i0 .. i0 + 63, 8-byte pieces; the next
  // chunk's pieces are loaded into registers while the current tile is used
  uint2 pre[kPer], prel[kPer];
  auto load = [&](int i0) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = threadIdx.x + kJtRows * k;
      const int row = e / (kJtChunk / 4), c4 = (e % (kJtChunk / 4)) * 4;
      const bool in = j0 + row < n && i0 + c4 < m;
      pre[k] = in ? *reinterpret_cast<const uint2*>(Jt + (j0 + row) * m + i0 + c4)
                  : make_uint2(0u, 0u);
      if (SPLIT)
        prel[k] = in ? *reinterpret_cast<const uint2*>(Jlo + (j0 + row) * m + i0 + c4)
                     : make_uint2(0u, 0u);
    }
  };
  auto f4 = [](uint2 u) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  };
  auto store = [&](TT* jt) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = threadIdx.x + kJtRows * k;
      const int row = e / (kJtChunk / 4), c4 = (e % (kJtChunk / 4)) * 4;
      if constexpr (SPLIT) {
        const float4 h = f4(pre[k]), l = f4(prel[k]);
        *reinterpret_cast<float4*>(jt + row * kLd + c4) =
            make_float4(h.x + l.x, h.y + l.y, h.z + l.z, h.w + l.w);
      } else {
        *reinterpret_cast<uint2*>(jt + row * kLd + c4) = pre[k];
      }
    }
  };
  load(0);
  store(jt0);
  int buf = 0;
  for (int i0 = 0; i0 < m; i0 += kJtChunk) {
    const int ni = m - i0 < kJtChunk ? m - i0 : kJtChunk;  // a multiple of 4
    __syncthreads();  // tile `buf` complete; the other one no longer read
    const bool more = i0 + kJtChunk < m;
    if (more) load(i0 + kJtChunk);
    const TT* jt = jt0 + buf * (kJtRows * kLd);
    for (int c = 0; c < ni; c += 4) {
      float4 a;
      if constexpr (SPLIT)
        a = *reinterpret_cast<const float4*>(jt + threadIdx.x * kLd + c);
      else
        a = f4(*reinterpret_cast<const uint2*>(jt + threadIdx.x * kLd + c));
#pragma unroll
      for (int q = 0; q < kTB; ++q) {
        const float4 rv = *reinterpret_cast<const float4*>(rs + q * m + i0 + c);
        acc[q] = fmaf(a.x, rv.x, fmaf(a.y, rv.y, fmaf(a.z, rv.z, fmaf(a.w, rv.w, acc[q]))));
      }
    }
    if (more) store(jt0 + (buf ^ 1) * (kJtRows * kLd));
    buf ^= 1;
  }
  if (j < n) {
#pragma unroll
    for (int q = 0; q < kTB; ++q)
      if (q < nb) g[(long long)(b0 + q) * g_bs + j] = scale * acc[q];
  }
}

// J [m][n] FP32 -> Jt [n][m] BF16 through 32 x 32 shared-memory tiles; Jlo (optional)
// receives bf16(J - Jt), the low part of the split form.
__global__ void transpose_bf16_kernel(const float* __restrict__ J, __nv_bfloat16* __restrict__ Jt,
                                      __nv_bfloat16* __restrict__ Jlo, int m, int n) {
  __shared__ float t[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = i0 + k, j = j0 + threadIdx.x;
    t[k][threadIdx.x] = (i < m && j < n) ? J[(long long)i * n + j] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int j = j0 + k, i = i0 + threadIdx.x;
    if (i < m && j < n) {
      const float v = t[threadIdx.x][k];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      Jt[(long long)j * m + i] = h;
      if (Jlo) Jlo[(long long)j * m + i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

cudaError_t jmul_residual_bf16(const __nv_bfloat16* Jt, const float* x, const float* dv, float* r,
                               float* part, int B, int m, int n, long long x_bs,
                               cudaStream_t stream, const __nv_bfloat16* Jlo) {
  if (m % 4 || m > 1024) return cudaErrorInvalidValue;
  const int nch = (int)ceil_div(n, kTCols);
  dim3 grid((unsigned)nch, (unsigned)ceil_div(B, kTB));
  if (m / 2 <= 256) {
    if (Jlo)
      jmul_t_kernel<1, true><<<grid, 256, 0, stream>>>(Jt, Jlo, x, part, B, m, n, x_bs);
    else
      jmul_t_kernel<1, false><<<grid, 256, 0, stream>>>(Jt, Jlo, x, part, B, m, n, x_bs);
  } else {
    if (Jlo)
      jmul_t_kernel<2, true><<<grid, 256, 0, stream>>>(Jt, Jlo, x, part, B, m, n, x_bs);
    else
      jmul_t_kernel<2, false><<<grid, 256, 0, stream>>>(Jt, Jlo, x, part, B, m, n, x_bs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  jmul_final_many_kernel<<<(unsigned)ceil_div((long long)B * m, 32), 256, 0, stream>>>(
      part, dv, r, (long long)B * m, nch);
  return cudaGetLastError();
}

template <typename JT>
cudaError_t jtmul_impl(const JT* J, const float* r, float* g, float scale, int B, int m, int n,
                       long long g_bs, cudaStream_t stream) {
  const size_t smem = (size_t)kJB * m * sizeof(float);
  if (smem > (size_t)kJtmulMaxSmem) return cudaErrorInvalidValue;
  dim3 grid((unsigned)ceil_div(n, 256), (unsigned)ceil_div(B, kJB));
  jtmul_kernel<JT><<<grid, 256, smem, stream>>>(J, r, g, scale, B, m, n, g_bs);
  return cudaGetLastError();
}

cudaError_t jtmul_f32(const float* J, const float* r, float* g, float scale, int B, int m,
                      int n, long long g_bs, cudaStream_t stream) {
  return jtmul_impl(J, r, g, scale, B, m, n, g_bs, stream);
}

cudaError_t jtmul_bf16(const __nv_bfloat16* Jt, const float* r, float* g, float scale, int B,
                       int m, int n, long long g_bs, cudaStream_t stream,
                       const __nv_bfloat16* Jlo) {
  const size_t tile = Jlo ? (size_t)JtTile<true>::kLd * 4 : (size_t)JtTile<false>::kLd * 2;
  const size_t smem = (size_t)kTB * m * sizeof(float) + 2 * (size_t)kJtRows * tile;
  if (m % 4 || smem > (size_t)kJtmulMaxSmem) return cudaErrorInvalidValue;
  dim3 grid((unsigned)ceil_div(n, kJtRows), (unsigned)ceil_div(B, kTB));
  if (Jlo)
    jtmul_t_kernel<true><<<grid, kJtRows, smem, stream>>>(Jt, Jlo, r, g, scale, B, m, n, g_bs);
  else
    jtmul_t_kernel<false><<<grid, kJtRows, smem, stream>>>(Jt, Jlo, r, g, scale, B, m, n, g_bs);
  return cudaGetLastError();
}

cudaError_t transpose_bf16(const float* J, __nv_bfloat16* Jt, int m, int n, cudaStream_t stream,
                           __nv_bfloat16* Jlo) {
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(m, 32));
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, stream>>>(J, Jt, Jlo, m, n);
  return cudaGetLastError();
}

__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                               long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

cudaError_t convert_bf16(const float* x, __nv_bfloat16* y, long long n, cudaStream_t stream) {
  to_bf16_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, stream>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t prepare_pointwise_kernels() {
  cudaError_t e = cudaFuncSetAttribute(jtmul_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kJtmulMaxSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(jtmul_t_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kJtmulMaxSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(jtmul_t_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kJtmulMaxSmem);
}

cudaError_t residual_loss_f64(const float* r, double* loss, double* trace, int* trace_pos,
                              int trace_cap, int* adam_t, int* status, int B, int m,
                              cudaStream_t stream, const double* reg_part, int reg_blocks) {
  const int threads = 32 * (B < 32 ? (B > 0 ? B : 1) : 32);
  loss_kernel<<<1, threads, 0, stream>>>(r, loss, trace, trace_pos, trace_cap, adam_t, status, B,
                                         m, reg_part, reg_blocks);
  return cudaGetLastError();
}

cudaError_t normalize_columns_f64(float* J, double* colnorm, int m, int n,
                                  cudaStream_t stream) {
  colnorm_kernel<<<(unsigned)ceil_div(n, 128), 128, 0, stream>>>(J, colnorm, m, n);
  return cudaGetLastError();
}

cudaError_t err_ratio_f64(const float* est, const float* truth, double* out, int B,
                          long long n, cudaStream_t stream) {
  err_kernel<<<B, 256, 0, stream>>>(est, truth, out, n);
  return cudaGetLastError();
}

cudaError_t adam_step_f32(float* theta, const float* g, float* m, float* v, long long count,
                          double lr, double beta1, double beta2, double eps, const int* t_dev,
                          int t_host, cudaStream_t stream) {
  // four parameters per thread when aligned; a grid-stride loop past 16 blocks per SM
  long long blocks = ceil_div(ceil_div(count, 4), 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  adam_kernel<<<(unsigned)blocks, 256, 0, stream>>>(
      theta, g, m, v, count, (float)lr, (float)beta1, (float)beta2, (float)(1.0 - beta1),
      (float)(1.0 - beta2), (float)std::log(beta1), (float)std::log(beta2), (float)eps, t_dev,
      t_host);
  return cudaGetLastError();
}

}  // namespace d2ip

// ------------------------------------------------------------------------------------
// 1x1x1 convolution to a single output channel (the network's last layer):
// y[v] = b + sum_c w[c] h[v][c]; backward dh[v][c] = w[c] g[v] with the weight partials
// sum_v g[v] h[v][c] and sum_v g[v] per block of kOneVox voxels (fixed-order sums).
// ------------------------------------------------------------------------------------
namespace d2ip {
namespace {

constexpr int kOneThreads = 256, kOneVpt = 8, kOneVox = kOneThreads * kOneVpt;

template <int C>
__global__ void __launch_bounds__(kOneThreads)
co1_fwd_kernel(const float* __restrict__ h, const float* __restrict__ wb, float* __restrict__ y,
               long long nvox, long long w_bs) {
  const int b = blockIdx.y;
  const long long v = (long long)blockIdx.x * kOneThreads + threadIdx.x;
  if (v >= nvox) return;
  const float* w = wb + (long long)b * w_bs;
  const float4* hv = reinterpret_cast<const float4*>(h + ((long long)b * nvox + v) * C);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < C / 4; ++c) {
    const float4 a = hv[c];
    s = fmaf(a.x, __ldg(w + 4 * c), s);
    s = fmaf(a.y, __ldg(w + 4 * c + 1), s);
    s = fmaf(a.z, __ldg(w + 4 * c + 2), s);
    s = fmaf(a.w, __ldg(w + 4 * c + 3), s);
  }
  y[(long long)b * nvox + v] = s + __ldg(w + C);
}

template <int C>
__global__ void __launch_bounds__(kOneThreads)
co1_bwd_kernel(const float* __restrict__ h, const float* __restrict__ g,
               const float* __restrict__ wb, float* __restrict__ dh, float* __restrict__ part,
               long long nvox, long long w_bs, int nblk, int accumulate) {
  __shared__ float red[kOneThreads][C + 1];
  const int b = blockIdx.y;
  const float* w = wb + (long long)b * w_bs;
  float wr[C];
#pragma unroll
  for (int c = 0; c < C; ++c) wr[c] = __ldg(w + c);
  float acc[C + 1];
#pragma unroll
  for (int c = 0; c <= C; ++c) acc[c] = 0.f;
  const long long v0 = (long long)blockIdx.x * kOneVox;
  for (int i = 0; i < kOneVpt; ++i) {
    const long long v = v0 + (long long)i * kOneThreads + threadIdx.x;
    if (v >= nvox) break;
    const long long o = (long long)b * nvox + v;
    const float gv = g[o];
    const float4* hv = reinterpret_cast<const float4*>(h + o * C);
    float4* dv = reinterpret_cast<float4*>(dh + o * C);
#pragma unroll
    for (int c = 0; c < C / 4; ++c) {
      const float4 a = hv[c];
      acc[4 * c] = fmaf(gv, a.x, acc[4 * c]);
      acc[4 * c + 1] = fmaf(gv, a.y, acc[4 * c + 1]);
      acc[4 * c + 2] = fmaf(gv, a.z, acc[4 * c + 2]);
      acc[4 * c + 3] = fmaf(gv, a.w, acc[4 * c + 3]);
      float4 d = make_float4(wr[4 * c] * gv, wr[4 * c + 1] * gv, wr[4 * c + 2] * gv,
                             wr[4 * c + 3] * gv);
      if (accumulate) {
        const float4 p = dv[c];
        d.x += p.x, d.y += p.y, d.z += p.z, d.w += p.w;
      }
      dv[c] = d;
    }
    acc[C] += gv;
  }
#pragma unroll
  for (int c = 0; c <= C; ++c) red[threadIdx.x][c] = acc[c];
  __syncthreads();
  if (threadIdx.x <= C) {
    float s = 0.f;
    for (int t = 0; t < kOneThreads; ++t) s += red[t][threadIdx.x];
    part[((long long)b * nblk + blockIdx.x) * (C + 1) + threadIdx.x] = s;
  }
}

}  // namespace

bool conv1x1_co1_supported(int C) { return C == 4 || C == 8 || C == 16 || C == 32; }

long long conv1x1_co1_blocks(long long nvox) { return ceil_div(nvox, kOneVox); }

cudaError_t conv1x1_co1_fwd_f32(const float* h, const float* wb, float* y, int B, long long nvox,
                                int C, long long w_bs, cudaStream_t stream) {
  dim3 grid((unsigned)ceil_div(nvox, kOneThreads), B);
  switch (C) {
    case 4: co1_fwd_kernel<4><<<grid, kOneThreads, 0, stream>>>(h, wb, y, nvox, w_bs); break;
    case 8: co1_fwd_kernel<8><<<grid, kOneThreads, 0, stream>>>(h, wb, y, nvox, w_bs); break;
    case 16: co1_fwd_kernel<16><<<grid, kOneThreads, 0, stream>>>(h, wb, y, nvox, w_bs); break;
    case 32: co1_fwd_kernel<32><<<grid, kOneThreads, 0, stream>>>(h, wb, y, nvox, w_bs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t conv1x1_co1_bwd_f32(const float* h, const float* g, const float* wb, float* dh,
                                float* part, int B, long long nvox, int C, long long w_bs,
                                int accumulate, cudaStream_t stream) {
  const int nblk = (int)conv1x1_co1_blocks(nvox);
  dim3 grid((unsigned)nblk, B);
#define D2IP_CO1B(C_)                                                                  \
  co1_bwd_kernel<C_><<<grid, kOneThreads, 0, stream>>>(h, g, wb, dh, part, nvox, w_bs, nblk, \
                                                       accumulate)
  switch (C) {
    case 4: D2IP_CO1B(4); break;
    case 8: D2IP_CO1B(8); break;
    case 16: D2IP_CO1B(16); break;
    case 32: D2IP_CO1B(32); break;
    default: return cudaErrorInvalidValue;
  }
#undef D2IP_CO1B
  return cudaGetLastError();
}

}  // namespace d2ip
