// Kernels of the paper-form 3D-FastResUNet variant (Sec. III-D): depthwise 3x3x3 and
// pointwise 1x1x1 convolutions (the depthwise separable convolution), elementwise
// activations, voxel sums and broadcasts (squeeze-and-excitation, the ASPP pooling branch),
// channel and voxel scaling (SE, attention gates) and channel slices (concatenation).
//
// Tensors are channels-last [B][voxels][C] (the layout of every other kernel of the
// library); weights are read per problem at a batch stride w_bs.  Every reduction runs in a
// fixed order (partial rows per voxel chunk, then reduce_rows_f32), so results are
// deterministic.  `acc` selects y += f(...) instead of y = f(...).
#include "common.cuh"
#include "fastres.cuh"

namespace d2ip {
namespace {

constexpr int kPwV = 32;       // voxels per pointwise forward / data-gradient block
constexpr int kPwK = 32;       // input channels per staged weight tile of the forward
constexpr int kPwPairs = 4096; // (co, ci) pairs per weight-gradient block (16 per thread)
constexpr int kSumV = 256;     // voxels per voxel-sum partial row
constexpr int kRowTarget = 608;  // partial rows aimed at per weight gradient (4 per SM)

// Voxels per partial row of a weight gradient: a multiple of 32 between 32 and `cap`, chosen
// so that about kRowTarget rows (blocks) cover the volume.
long long wgrad_chunk(long long nout, long long cap) {
  long long c = ceil_div(ceil_div(nout, kRowTarget), 32) * 32;
  return c < 32 ? 32 : (c > cap ? cap : c);
}

__device__ __forceinline__ long long strided_voxel(long long q, Dims3 dout, Dims3 din, int s) {
  if (s == 1) return q;
  const long long yx = (long long)dout.y * dout.x;
  const int qz = (int)(q / yx);
  const long long r = q - qz * yx;
  const int qy = (int)(r / dout.x), qx = (int)(r - (long long)qy * dout.x);
  return ((long long)(s * qz) * din.y + s * qy) * din.x + s * qx;
}

// y[q][o] (=|+=) b[o] + sum_i W[o][i] x[in(q)][i], in(q) the voxel s*q of din.  The block
// stages its vb input rows (row stride ci + 1: no bank conflicts between voxels) and the
// weights transposed, kPwK input channels at a time, so a warp reads consecutive outputs'
// weights.  vb * co <= 1024: each thread keeps the sums of up to 4 (voxel, output) pairs;
// the channel sum runs in order.
__global__ void __launch_bounds__(256) pw_fwd_kernel(const float* __restrict__ x,
                                                     const float* __restrict__ W, float* y,
                                                     Dims3 din, Dims3 dout, int ci, int co, int s,
                                                     long long w_bs, int acc, int vb) {
  extern __shared__ float sm[];  // xs[vb][ci + 1], wt[kPwK][co]
  float* xs = sm;
  float* wt = sm + vb * (ci + 1);
  const int b = blockIdx.y;
  const long long nout = dout.count(), q0 = (long long)blockIdx.x * vb;
  x += (long long)b * din.count() * ci;
  y += (long long)b * nout * co;
  W += (long long)b * w_bs;
  const float* bias = W + (long long)co * ci;
  for (int i = threadIdx.x; i < vb * ci; i += blockDim.x) {
    const int v = i / ci, c = i - v * ci;
    const long long q = q0 + v;
    xs[v * (ci + 1) + c] = q < nout ? x[strided_voxel(q, dout, din, s) * ci + c] : 0.f;
  }
  const int npair = vb * co;
  float a[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = threadIdx.x + 256 * j;
    a[j] = o < npair ? bias[o % co] : 0.f;
  }
  for (int k0 = 0; k0 < ci; k0 += kPwK) {
    const int kn = min(kPwK, ci - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < kn * co; i += blockDim.x) {
      const int k = i / co, c = i - k * co;
      wt[i] = W[(long long)c * ci + k0 + k];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = threadIdx.x + 256 * j;
      if (o >= npair) continue;
      const int v = o / co, c = o - v * co;
      const float* xv = xs + v * (ci + 1) + k0;
      float t = a[j];
      for (int k = 0; k < kn; ++k) t = fmaf(wt[k * co + c], xv[k], t);
      a[j] = t;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = threadIdx.x + 256 * j;
    if (o >= npair) continue;
    const int v = o / co, c = o - v * co;
    const long long q = q0 + v;
    if (q >= nout) continue;
    float* d = y + q * co + c;
    *d = acc ? *d + a[j] : a[j];
  }
}

// dx[in(q)][i] (+)= sum_o W[o][i] dy[q][o]  (voxels not sampled by a stride-2 layer get no
// contribution; the launcher clears them first when acc = 0).
__global__ void __launch_bounds__(256) pw_dgrad_kernel(const float* __restrict__ dy,
                                                       const float* __restrict__ W, float* dx,
                                                       Dims3 din, Dims3 dout, int ci, int co,
                                                       int s, long long w_bs, int acc) {
  extern __shared__ float ds[];  // [kPwV][co]
  const int b = blockIdx.y;
  const long long nout = dout.count(), q0 = (long long)blockIdx.x * kPwV;
  dy += (long long)b * nout * co;
  dx += (long long)b * din.count() * ci;
  W += (long long)b * w_bs;
  for (int i = threadIdx.x; i < kPwV * co; i += blockDim.x) {
    const long long q = q0 + i / co;
    ds[i] = q < nout ? dy[q0 * co + i] : 0.f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < kPwV * ci; o += blockDim.x) {
    const int v = o / ci, c = o - v * ci;
    const long long q = q0 + v;
    if (q >= nout) continue;
    const float* dv = ds + v * co;
    float a = 0.f;
    for (int k = 0; k < co; ++k) a = fmaf(W[(long long)k * ci + c], dv[k], a);
    float* d = dx + strided_voxel(q, dout, din, s) * ci + c;
    *d = acc ? *d + a : a;
  }
}

// part[b][chunk][p], p < co*ci: sum over the chunk's voxels of dy[q][o] x[in(q)][i]
// (p = o*ci + i); p >= co*ci: sum of dy[q][p - co*ci] (the bias).  One block covers a voxel
// chunk and a tile of kPwPairs pairs, each thread 16 pairs.
__global__ void __launch_bounds__(256) pw_wgrad_kernel(const float* __restrict__ x,
                                                       const float* __restrict__ dy, float* part,
                                                       Dims3 din, Dims3 dout, int ci, int co,
                                                       int s, long long rows, long long chv) {
  extern __shared__ float sm[];  // xs[kPwV][ci] then dys[kPwV][co]
  float* xs = sm;
  float* dys = sm + kPwV * ci;
  const int b = blockIdx.z;
  const long long nout = dout.count(), chunk = blockIdx.x;
  const long long npairs = (long long)co * ci + co;
  const long long p0 = (long long)blockIdx.y * kPwPairs;
  x += (long long)b * din.count() * ci;
  dy += (long long)b * nout * co;
  float a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = 0.f;
  const long long v_end = min(nout, (chunk + 1) * chv);
  for (long long t0 = chunk * chv; t0 < v_end; t0 += kPwV) {
    __syncthreads();
    for (int i = threadIdx.x; i < kPwV * ci; i += blockDim.x) {
      const long long q = t0 + i / ci;
      xs[i] = q < v_end ? x[strided_voxel(q, dout, din, s) * ci + i % ci] : 0.f;
    }
    for (int i = threadIdx.x; i < kPwV * co; i += blockDim.x) {
      const long long q = t0 + i / co;
      dys[i] = q < v_end ? dy[t0 * co + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long p = p0 + threadIdx.x + 256LL * j;
      if (p >= npairs || p >= p0 + kPwPairs) continue;
      float acc = a[j];
      if (p < (long long)co * ci) {
        const int o = (int)(p / ci), i = (int)(p - (long long)o * ci);
        for (int v = 0; v < kPwV; ++v) acc = fmaf(dys[v * co + o], xs[v * ci + i], acc);
      } else {
        const int o = (int)(p - (long long)co * ci);
        for (int v = 0; v < kPwV; ++v) acc += dys[v * co + o];
      }
      a[j] = acc;
    }
  }
  float* row = part + ((long long)b * rows + chunk) * npairs;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const long long p = p0 + threadIdx.x + 256LL * j;
    if (p < npairs && p < p0 + kPwPairs) row[p] = a[j];
  }
}

// Depthwise 3x3x3, stride s, dilation d, zero padding d: y[q][c] = b[c] +
// sum_t W[c][t] x[s*q + d*(t - 1)][c].  One thread per (voxel, channel).
__global__ void __launch_bounds__(256) dw_fwd_kernel(const float* __restrict__ x,
                                                     const float* __restrict__ W, float* y,
                                                     Dims3 din, Dims3 dout, int C, int s, int d,
                                                     long long w_bs) {
  const int b = blockIdx.y;
  const long long nout = dout.count();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nout * C) return;
  const int c = (int)(idx % C);
  const long long q = idx / C;
  const long long yx = (long long)dout.y * dout.x;
  const int oz = (int)(q / yx), oy = (int)((q - oz * yx) / dout.x),
            ox = (int)(q - oz * yx - (long long)oy * dout.x);
  x += (long long)b * din.count() * C;
  W += (long long)b * w_bs;
  const float* w = W + (long long)c * 27;
  float a = W[(long long)C * 27 + c];
  for (int kz = 0; kz < 3; ++kz) {
    const int iz = s * oz + d * (kz - 1);
    if (iz < 0 || iz >= din.z) continue;
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = s * oy + d * (ky - 1);
      if (iy < 0 || iy >= din.y) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = s * ox + d * (kx - 1);
        if (ix < 0 || ix >= din.x) continue;
        a = fmaf(w[(kz * 3 + ky) * 3 + kx], x[(((long long)iz * din.y + iy) * din.x + ix) * C + c],
                 a);
      }
    }
  }
  y[(long long)b * nout * C + idx] = a;
}

// dx[p][c] (+)= sum over taps t and outputs q with s*q + d*(t - 1) = p of W[c][t] dy[q][c].
__global__ void __launch_bounds__(256) dw_dgrad_kernel(const float* __restrict__ dy,
                                                       const float* __restrict__ W, float* dx,
                                                       Dims3 din, Dims3 dout, int C, int s, int d,
                                                       long long w_bs, int acc) {
  const int b = blockIdx.y;
  const long long nin = din.count();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nin * C) return;
  const int c = (int)(idx % C);
  const long long p = idx / C;
  const long long yx = (long long)din.y * din.x;
  const int pz = (int)(p / yx), py = (int)((p - pz * yx) / din.x),
            px = (int)(p - pz * yx - (long long)py * din.x);
  dy += (long long)b * dout.count() * C;
  W += (long long)b * w_bs;
  const float* w = W + (long long)c * 27;
  float a = 0.f;
  for (int kz = 0; kz < 3; ++kz) {
    const int tz = pz - d * (kz - 1);
    if (tz < 0 || tz % s) continue;
    const int oz = tz / s;
    if (oz >= dout.z) continue;
    for (int ky = 0; ky < 3; ++ky) {
      const int ty = py - d * (ky - 1);
      if (ty < 0 || ty % s) continue;
      const int oy = ty / s;
      if (oy >= dout.y) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int tx = px - d * (kx - 1);
        if (tx < 0 || tx % s) continue;
        const int ox = tx / s;
        if (ox >= dout.x) continue;
        a = fmaf(w[(kz * 3 + ky) * 3 + kx],
                 dy[(((long long)oz * dout.y + oy) * dout.x + ox) * C + c], a);
      }
    }
  }
  float* o = dx + (long long)b * nin * C + idx;
  *o = acc ? *o + a : a;
}

// part[b][chunk][28 C]: per chunk of chv output voxels, W part [c][27] then bias [c].
// Thread (channel c, voxel lane vl) sums its voxels; lanes are then added in order.
__global__ void __launch_bounds__(256) dw_wgrad_kernel(const float* __restrict__ x,
                                                       const float* __restrict__ dy, float* part,
                                                       Dims3 din, Dims3 dout, int C, int s, int d,
                                                       long long rows, long long chv) {
  __shared__ float red[256 * 28];
  const int b = blockIdx.y;
  const long long chunk = blockIdx.x, nout = dout.count();
  const int nvl = 256 / C;
  const int c = threadIdx.x % C, vl = threadIdx.x / C;
  x += (long long)b * din.count() * C;
  dy += (long long)b * nout * C;
  float a[28];
#pragma unroll
  for (int t = 0; t < 28; ++t) a[t] = 0.f;
  if (vl < nvl) {
    const long long yx = (long long)dout.y * dout.x;
    const long long v_end = min(nout, (chunk + 1) * chv);
    for (long long q = chunk * chv + vl; q < v_end; q += nvl) {
      const int oz = (int)(q / yx), oy = (int)((q - oz * yx) / dout.x),
                ox = (int)(q - oz * yx - (long long)oy * dout.x);
      const float g = dy[q * C + c];
      a[27] += g;
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const int kz = t / 9, ky = (t / 3) % 3, kx = t % 3;
        const int iz = s * oz + d * (kz - 1), iy = s * oy + d * (ky - 1),
                  ix = s * ox + d * (kx - 1);
        if (iz >= 0 && iz < din.z && iy >= 0 && iy < din.y && ix >= 0 && ix < din.x)
          a[t] = fmaf(g, x[(((long long)iz * din.y + iy) * din.x + ix) * C + c], a[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < 28; ++t) red[(vl * C + c) * 28 + t] = a[t];
  }
  __syncthreads();
  float* row = part + ((long long)b * rows + chunk) * 28LL * C;
  for (int i = threadIdx.x; i < 28 * C; i += blockDim.x) {
    const int cc = i / 28, t = i - cc * 28;
    float sum = 0.f;
    for (int l = 0; l < nvl; ++l) sum += red[(l * C + cc) * 28 + t];
    if (t < 27)
      row[(long long)cc * 27 + t] = sum;
    else
      row[27LL * C + cc] = sum;
  }
}

__device__ __forceinline__ float act_f(float v, int kind) {
  if (kind == kActLeaky) return v > 0.f ? v : kLeakySlope * v;
  if (kind == kActRelu) return v > 0.f ? v : 0.f;
  return 1.f / (1.f + expf(-v));
}

// derivative from the output y (leaky / relu keep the sign of their input)
__device__ __forceinline__ float act_d(float y, int kind) {
  if (kind == kActLeaky) return y > 0.f ? 1.f : kLeakySlope;
  if (kind == kActRelu) return y > 0.f ? 1.f : 0.f;
  return y * (1.f - y);
}

__global__ void act_fwd_kernel(const float* __restrict__ x, float* y, long long n, int kind) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = act_f(x[i], kind);
}

__global__ void act_bwd_kernel(const float* __restrict__ y, const float* __restrict__ dy,
                               float* dx, long long n, int kind, int acc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = dy[i] * act_d(y[i], kind);
  dx[i] = acc ? dx[i] + g : g;
}

__global__ void add2_kernel(const float* __restrict__ a, const float* __restrict__ b, float* y,
                            long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] + b[i];
}

__global__ void accum_kernel(float* dst, const float* __restrict__ src, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// part[b][chunk][c] = scale * sum over the chunk's voxels of x[q][c] (* y[q][c] when y).
// Block: 32 channels x 8 voxel lanes; lanes added in order.
__global__ void __launch_bounds__(256) vox_sum_kernel(const float* __restrict__ x,
                                                      const float* __restrict__ y, float* part,
                                                      long long nvox, int C, float scale,
                                                      long long rows) {
  __shared__ float red[8][32];
  const int b = blockIdx.z;
  const int c = blockIdx.y * 32 + (threadIdx.x & 31), vl = threadIdx.x >> 5;
  const long long chunk = blockIdx.x;
  x += (long long)b * nvox * C;
  if (y) y += (long long)b * nvox * C;
  float a = 0.f;
  if (c < C) {
    const long long v_end = min(nvox, (chunk + 1) * kSumV);
    for (long long q = chunk * kSumV + vl; q < v_end; q += 8) {
      const float v = x[q * C + c];
      a += y ? v * y[q * C + c] : v;
    }
  }
  red[vl][threadIdx.x & 31] = a;
  __syncthreads();
  if (vl == 0 && c < C) {
    float s = 0.f;
    for (int l = 0; l < 8; ++l) s += red[l][threadIdx.x];
    part[((long long)b * rows + chunk) * C + c] = scale * s;
  }
}

// y[b][q][c] (=|+=) scale * x[b][c]
__global__ void bcast_kernel(const float* __restrict__ x, float* y, long long nvox, int C,
                             float scale, int acc, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long per = nvox * C;
  const long long b = i / per;
  const float v = scale * x[b * C + i % C];
  y[i] = acc ? y[i] + v : v;
}

// y[b][q][c] = x[b][q][c] * s[b][c]    (dx form: dx (=|+=) dy * s)
__global__ void cscale_kernel(const float* __restrict__ x, const float* __restrict__ s, float* y,
                              long long nvox, int C, int acc, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long b = i / (nvox * C);
  const float v = x[i] * s[b * C + i % C];
  y[i] = acc ? y[i] + v : v;
}

// y[q][c] = x[q][c] * psi[q]  (over all problems' voxels; dx form with acc)
__global__ void vscale_kernel(const float* __restrict__ x, const float* __restrict__ psi,
                              float* y, int C, int acc, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float v = x[i] * psi[i / C];
  y[i] = acc ? y[i] + v : v;
}

// dpsi[q] (=|+=) sum_c dy[q][c] x[q][c]: one warp per voxel, channels in lane order then a
// fixed butterfly.
__global__ void vdot_kernel(const float* __restrict__ dy, const float* __restrict__ x,
                            float* dpsi, int C, int acc, long long nvox) {
  const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nvox) return;
  float a = 0.f;
  for (int c = lane; c < C; c += 32) a = fmaf(dy[q * C + c], x[q * C + c], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) dpsi[q] = acc ? dpsi[q] + a : a;
}

// dst[q][dst_off + c] (=|+=) src[q][src_off + c], c < width
__global__ void slice_kernel(const float* __restrict__ src, int src_C, int src_off, float* dst,
                             int dst_C, int dst_off, int width, int acc, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long q = i / width;
  const int c = (int)(i - q * width);
  const float v = src[q * src_C + src_off + c];
  float* d = dst + q * dst_C + dst_off + c;
  *d = acc ? *d + v : v;
}

unsigned blocks(long long n) { return (unsigned)ceil_div(n, 256); }

}  // namespace

// voxels per pointwise forward block: vb * co <= 1024 (4 sums per thread), at most kPwV
int pw_vb(int co) { return co >= 1024 ? 1 : (1024 / co < kPwV ? 1024 / co : kPwV); }

bool pw_supported(int ci, int co) {
  return ci >= 1 && co >= 1 && co <= 1024 &&
         ((long long)pw_vb(co) * (ci + 1) + (long long)kPwK * co) * 4 <= 48 * 1024 &&
         (long long)kPwV * (ci + co) * 4 <= 48 * 1024;
}

cudaError_t pw_fwd_f32(const float* x, const float* W, float* y, int B, Dims3 din, int ci,
                       int co, int s, long long w_bs, int acc, cudaStream_t st) {
  if (!pw_supported(ci, co) || (s != 1 && s != 2)) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 1, s);
  const int vb = pw_vb(co);
  dim3 grid((unsigned)ceil_div(dout.count(), vb), B);
  const size_t smem = ((size_t)vb * (ci + 1) + (size_t)kPwK * co) * sizeof(float);
  pw_fwd_kernel<<<grid, 256, smem, st>>>(x, W, y, din, dout, ci, co, s, w_bs, acc, vb);
  return cudaGetLastError();
}

cudaError_t pw_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din, int ci,
                         int co, int s, long long w_bs, int acc, cudaStream_t st) {
  if (!pw_supported(ci, co) || (s != 1 && s != 2)) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 1, s);
  if (s != 1 && !acc) {
    cudaError_t e = cudaMemsetAsync(dx, 0, sizeof(float) * B * din.count() * ci, st);
    if (e != cudaSuccess) return e;
    acc = 1;
  }
  dim3 grid((unsigned)ceil_div(dout.count(), kPwV), B);
  pw_dgrad_kernel<<<grid, 256, kPwV * co * sizeof(float), st>>>(dy, W, dx, din, dout, ci, co,
                                                                  s, w_bs, acc);
  return cudaGetLastError();
}

long long pw_wgrad_rows(Dims3 din, int s) {
  const long long n = conv_out_dims(din, 1, s).count();
  return ceil_div(n, wgrad_chunk(n, 256));
}

cudaError_t pw_wgrad_partial_f32(const float* x, const float* dy, float* part, int B, Dims3 din,
                                 int ci, int co, int s, cudaStream_t st) {
  if (!pw_supported(ci, co) || (s != 1 && s != 2)) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 1, s);
  const long long rows = pw_wgrad_rows(din, s);
  const long long chv = wgrad_chunk(dout.count(), 256);
  const long long npairs = (long long)co * ci + co;
  dim3 grid((unsigned)rows, (unsigned)ceil_div(npairs, kPwPairs), B);
  pw_wgrad_kernel<<<grid, 256, kPwV * (ci + co) * sizeof(float), st>>>(x, dy, part, din, dout,
                                                                         ci, co, s, rows, chv);
  return cudaGetLastError();
}

cudaError_t dw_fwd_f32(const float* x, const float* W, float* y, int B, Dims3 din, int C, int s,
                       int d, long long w_bs, cudaStream_t st) {
  if (C < 1 || C > 256 || (s != 1 && s != 2) || d < 1) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 3, s);
  dim3 grid(blocks(dout.count() * C), B);
  dw_fwd_kernel<<<grid, 256, 0, st>>>(x, W, y, din, dout, C, s, d, w_bs);
  return cudaGetLastError();
}

cudaError_t dw_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din, int C,
                         int s, int d, long long w_bs, int acc, cudaStream_t st) {
  if (C < 1 || C > 256 || (s != 1 && s != 2) || d < 1) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 3, s);
  dim3 grid(blocks(din.count() * C), B);
  dw_dgrad_kernel<<<grid, 256, 0, st>>>(dy, W, dx, din, dout, C, s, d, w_bs, acc);
  return cudaGetLastError();
}

long long dw_wgrad_rows(Dims3 din, int s) {
  const long long n = conv_out_dims(din, 3, s).count();
  return ceil_div(n, wgrad_chunk(n, 512));
}

cudaError_t dw_wgrad_partial_f32(const float* x, const float* dy, float* part, int B, Dims3 din,
                                 int C, int s, int d, cudaStream_t st) {
  if (C < 1 || C > 256 || (s != 1 && s != 2) || d < 1) return cudaErrorInvalidValue;
  const Dims3 dout = conv_out_dims(din, 3, s);
  const long long rows = dw_wgrad_rows(din, s);
  dim3 grid((unsigned)rows, B);
  dw_wgrad_kernel<<<grid, 256, 0, st>>>(x, dy, part, din, dout, C, s, d, rows,
                                        wgrad_chunk(dout.count(), 512));
  return cudaGetLastError();
}

cudaError_t act_fwd_f32(const float* x, float* y, long long n, int kind, cudaStream_t st) {
  act_fwd_kernel<<<blocks(n), 256, 0, st>>>(x, y, n, kind);
  return cudaGetLastError();
}

cudaError_t act_bwd_f32(const float* y, const float* dy, float* dx, long long n, int kind,
                        int acc, cudaStream_t st) {
  act_bwd_kernel<<<blocks(n), 256, 0, st>>>(y, dy, dx, n, kind, acc);
  return cudaGetLastError();
}

cudaError_t add2_f32(const float* a, const float* b, float* y, long long n, cudaStream_t st) {
  add2_kernel<<<blocks(n), 256, 0, st>>>(a, b, y, n);
  return cudaGetLastError();
}

cudaError_t accum_f32(float* dst, const float* src, long long n, int acc, cudaStream_t st) {
  if (!acc) return cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
  accum_kernel<<<blocks(n), 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

long long vox_sum_rows(long long nvox) { return ceil_div(nvox, kSumV); }

cudaError_t vox_sum_partial_f32(const float* x, const float* y, float* part, int B,
                                long long nvox, int C, float scale, cudaStream_t st) {
  const long long rows = vox_sum_rows(nvox);
  dim3 grid((unsigned)rows, (unsigned)ceil_div(C, 32), B);
  vox_sum_kernel<<<grid, 256, 0, st>>>(x, y, part, nvox, C, scale, rows);
  return cudaGetLastError();
}

cudaError_t bcast_f32(const float* x, float* y, int B, long long nvox, int C, float scale,
                      int acc, cudaStream_t st) {
  const long long total = (long long)B * nvox * C;
  bcast_kernel<<<blocks(total), 256, 0, st>>>(x, y, nvox, C, scale, acc, total);
  return cudaGetLastError();
}

cudaError_t cscale_f32(const float* x, const float* s, float* y, int B, long long nvox, int C,
                       int acc, cudaStream_t st) {
  const long long total = (long long)B * nvox * C;
  cscale_kernel<<<blocks(total), 256, 0, st>>>(x, s, y, nvox, C, acc, total);
  return cudaGetLastError();
}

cudaError_t vscale_f32(const float* x, const float* psi, float* y, long long nvox_all, int C,
                       int acc, cudaStream_t st) {
  const long long total = nvox_all * C;
  vscale_kernel<<<blocks(total), 256, 0, st>>>(x, psi, y, C, acc, total);
  return cudaGetLastError();
}

cudaError_t vdot_f32(const float* dy, const float* x, float* dpsi, long long nvox_all, int C,
                     int acc, cudaStream_t st) {
  vdot_kernel<<<(unsigned)ceil_div(nvox_all * 32, 256), 256, 0, st>>>(dy, x, dpsi, C, acc,
                                                                       nvox_all);
  return cudaGetLastError();
}

cudaError_t slice_f32(const float* src, int src_C, int src_off, float* dst, int dst_C,
                      int dst_off, int width, long long nvox_all, int acc, cudaStream_t st) {
  const long long total = nvox_all * width;
  slice_kernel<<<blocks(total), 256, 0, st>>>(src, src_C, src_off, dst, dst_C, dst_off, width,
                                               acc, total);
  return cudaGetLastError();
}

}  // namespace d2ip
