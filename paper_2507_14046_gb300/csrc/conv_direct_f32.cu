// Direct FP32 3D convolution: forward (3x3x3 stride 1 or 2, 1x1x1) and data gradient.
//
// The channel counts of the U-Net are small (8..192) while the grids are large, so a GEMM
// tiling over (voxels x channels) leaves most of the GPU idle.  Here one thread owns one
// output voxel of a 2x8x8 brick and CT output channels; per chunk of CK input channels the
// block stages the brick's input halo and the CT x 27 x CK weights in shared memory, so each
// input value is read from L2 once per brick (not once per tap) and every weight read is a
// shared-memory broadcast.  Accumulation is FP32 in a fixed order (channels, then taps).
//
// The stride-1 data gradient is the same kernel on dy with flipped taps and transposed
// weights (dx[p][ci] = sum_{t,co} W[co][26-t][ci] dy[p + k - 1][co]); the stride-2 data
// gradient gathers, for each input voxel, the taps whose output position is an integer.
#include "common.cuh"

namespace d2ip {
namespace {

constexpr int kBZ = 2, kBY = 8, kBX = 8;
constexpr int kThreads = kBZ * kBY * kBX;

// MODE 0: forward.  MODE 1: stride-1 data gradient (flipped, transposed weights).
template <int K, int S, int CT, int CK, int MODE>
__global__ void __launch_bounds__(kThreads)
direct_conv_kernel(const float* __restrict__ in, const float* __restrict__ W,
                   const float* __restrict__ bias, float* __restrict__ out, Dims3 din,
                   Dims3 dout, int Cin, int Cout, long long in_bs, long long out_bs,
                   long long w_bs, int accumulate) {
  constexpr int T = K * K * K, PAD = (K - 1) / 2;
  constexpr int HZ = (kBZ - 1) * S + K, HY = (kBY - 1) * S + K, HX = (kBX - 1) * S + K;
  constexpr int HV = HZ * HY * HX;
  __shared__ float sx[CK * HV];
  __shared__ float4 sw4[CK * T * (CT / 4)];
  float* sw = reinterpret_cast<float*>(sw4);

  const int b = blockIdx.z;
  in += b * in_bs;
  out += b * out_bs;
  W += b * w_bs;
  if (bias) bias += b * w_bs;
  const int nbx = (dout.x + kBX - 1) / kBX, nby = (dout.y + kBY - 1) / kBY;
  int bid = blockIdx.x;
  const int bx0 = (bid % nbx) * kBX;
  bid /= nbx;
  const int by0 = (bid % nby) * kBY;
  const int bz0 = (bid / nby) * kBZ;
  const int tx = threadIdx.x % kBX, ty = (threadIdx.x / kBX) % kBY, tz = threadIdx.x / (kBX * kBY);
  const int iz0 = bz0 * S - PAD, iy0 = by0 * S - PAD, ix0 = bx0 * S - PAD;
  const int co0 = blockIdx.y * CT;

  float acc[CT];
#pragma unroll
  for (int j = 0; j < CT; ++j) acc[j] = 0.f;

  for (int c0 = 0; c0 < Cin; c0 += CK) {
    __syncthreads();
    for (int e = threadIdx.x; e < CK * HV; e += kThreads) {
      const int c = e % CK, h = e / CK;
      const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
      const int iz = iz0 + hz, iy = iy0 + hy, ix = ix0 + hx;
      float v = 0.f;
      if (c0 + c < Cin && (unsigned)iz < (unsigned)din.z && (unsigned)iy < (unsigned)din.y &&
          (unsigned)ix < (unsigned)din.x)
        v = in[(((long long)iz * din.y + iy) * din.x + ix) * Cin + c0 + c];
      sx[c * HV + h] = v;
    }
    for (int e = threadIdx.x; e < CK * T * CT; e += kThreads) {
      int c, t, j;
      float v = 0.f;
      if (MODE == 0) {  // W[co][t][ci]: consecutive threads read consecutive ci
        c = e % CK;
        const int r = e / CK;
        t = r % T;
        j = r / T;
        if (c0 + c < Cin && co0 + j < Cout) v = W[((long long)(co0 + j) * T + t) * Cin + c0 + c];
      } else {  // W[co = c][T-1-t][ci = j]: consecutive threads read consecutive ci
        j = e % CT;
        const int r = e / CT;
        t = r % T;
        c = r / T;
        if (c0 + c < Cin && co0 + j < Cout)
          v = W[((long long)(c0 + c) * T + (T - 1 - t)) * Cout + co0 + j];
      }
      sw[(c * T + t) * CT + j] = v;
    }
    __syncthreads();
    for (int c = 0; c < CK; ++c) {
      const float* xs = sx + c * HV + (tz * S) * HY * HX + (ty * S) * HX + tx * S;
      const float4* ws = sw4 + c * T * (CT / 4);
#pragma unroll
      for (int kz = 0; kz < K; ++kz)
#pragma unroll
        for (int ky = 0; ky < K; ++ky)
#pragma unroll
          for (int kx = 0; kx < K; ++kx) {
            const float xv = xs[(kz * HY + ky) * HX + kx];
            const int t = (kz * K + ky) * K + kx;
#pragma unroll
            for (int q = 0; q < CT / 4; ++q) {
              const float4 w = ws[t * (CT / 4) + q];
              acc[4 * q + 0] = fmaf(xv, w.x, acc[4 * q + 0]);
              acc[4 * q + 1] = fmaf(xv, w.y, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(xv, w.z, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(xv, w.w, acc[4 * q + 3]);
            }
          }
    }
  }
  const int oz = bz0 + tz, oy = by0 + ty, ox = bx0 + tx;
  if (oz >= dout.z || oy >= dout.y || ox >= dout.x) return;
  const long long o = ((long long)oz * dout.y + oy) * dout.x + ox;
#pragma unroll
  for (int j = 0; j < CT; ++j) {
    const int co = co0 + j;
    if (co < Cout) {
      const float v = acc[j] + (bias ? bias[co] : 0.f);
      float* p = out + o * Cout + co;
      *p = accumulate ? *p + v : v;
    }
  }
}

// Stride-2, 3x3x3 data gradient: dx[p][ci] = sum over taps k with (p + 1 - k) even and
// o = (p + 1 - k)/2 inside the output grid, sum over co of W[co][k][ci] dy[o][co].
constexpr int kS2Chunk = 16;

template <int CT>
__global__ void __launch_bounds__(128)
dgrad_s2_kernel(const float* __restrict__ dy, const float* __restrict__ W,
                float* __restrict__ dx, Dims3 din, Dims3 dout, int Ci, int Co,
                long long dy_bs, long long dx_bs, long long w_bs, int accumulate) {
  __shared__ float sw[kS2Chunk * 27 * CT];
  const int b = blockIdx.z;
  dy += b * dy_bs;
  dx += b * dx_bs;
  W += b * w_bs;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ci0 = blockIdx.y * CT;
  const bool on = p < din.count();
  int ix = 0, iy = 0, iz = 0;
  if (on) {
    ix = (int)(p % din.x);
    const long long r = p / din.x;
    iy = (int)(r % din.y);
    iz = (int)(r / din.y);
  }
  float acc[CT];
#pragma unroll
  for (int j = 0; j < CT; ++j) acc[j] = 0.f;
  for (int c0 = 0; c0 < Co; c0 += kS2Chunk) {
    __syncthreads();
    for (int e = threadIdx.x; e < kS2Chunk * 27 * CT; e += blockDim.x) {
      const int j = e % CT, r = e / CT, t = r % 27, c = r / 27;
      sw[e] = (c0 + c < Co && ci0 + j < Ci) ? W[((long long)(c0 + c) * 27 + t) * Ci + ci0 + j]
                                            : 0.f;
    }
    __syncthreads();
    if (!on) continue;
    for (int kz = 0; kz < 3; ++kz) {
      const int nz = iz + 1 - kz;
      if (nz < 0 || (nz & 1) || (nz >> 1) >= dout.z) continue;
      for (int ky = 0; ky < 3; ++ky) {
        const int ny = iy + 1 - ky;
        if (ny < 0 || (ny & 1) || (ny >> 1) >= dout.y) continue;
        for (int kx = 0; kx < 3; ++kx) {
          const int nx = ix + 1 - kx;
          if (nx < 0 || (nx & 1) || (nx >> 1) >= dout.x) continue;
          const long long o = ((long long)(nz >> 1) * dout.y + (ny >> 1)) * dout.x + (nx >> 1);
          const int t = (kz * 3 + ky) * 3 + kx;
          const float* g = dy + o * Co + c0;
          const int nc = Co - c0 < kS2Chunk ? Co - c0 : kS2Chunk;
          for (int c = 0; c < nc; ++c) {
            const float gv = g[c];
            const float* w = sw + (c * 27 + t) * CT;
#pragma unroll
            for (int j = 0; j < CT; ++j) acc[j] = fmaf(gv, w[j], acc[j]);
          }
        }
      }
    }
  }
  if (!on) return;
#pragma unroll
  for (int j = 0; j < CT; ++j) {
    const int ci = ci0 + j;
    if (ci < Ci) {
      float* q = dx + p * Ci + ci;
      *q = accumulate ? *q + acc[j] : acc[j];
    }
  }
}

// Largest channel tile (16, 8 or 4) that still gives at least two blocks per SM.
int pick_ct(long long blocks_per_tile, int cout) {
  for (int ct : {16, 8}) {
    if (cout >= ct && blocks_per_tile * ceil_div(cout, ct) >= 2 * 152) return ct;
  }
  return 4;
}

long long bricks(Dims3 d) {
  return ceil_div(d.x, kBX) * ceil_div(d.y, kBY) * ceil_div(d.z, kBZ);
}

template <int K, int S, int CK, int MODE>
cudaError_t launch_direct(int ct, const float* in, const float* W, const float* bias, float* out,
                          int B, Dims3 din, Dims3 dout, int Cin, int Cout, long long in_bs,
                          long long out_bs, long long w_bs, int acc, cudaStream_t st) {
  dim3 grid((unsigned)bricks(dout), (unsigned)ceil_div(Cout, ct), B);
  switch (ct) {
    case 16:
      direct_conv_kernel<K, S, 16, CK, MODE><<<grid, kThreads, 0, st>>>(
          in, W, bias, out, din, dout, Cin, Cout, in_bs, out_bs, w_bs, acc);
      break;
    case 8:
      direct_conv_kernel<K, S, 8, CK, MODE><<<grid, kThreads, 0, st>>>(
          in, W, bias, out, din, dout, Cin, Cout, in_bs, out_bs, w_bs, acc);
      break;
    default:
      direct_conv_kernel<K, S, 4, CK, MODE><<<grid, kThreads, 0, st>>>(
          in, W, bias, out, din, dout, Cin, Cout, in_bs, out_bs, w_bs, acc);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t conv3d_fwd_f32(const float* x, const float* W, const float* bias, float* y,
                           int B, Dims3 din, int Ci, int Co, int K, int S, long long x_bs,
                           long long y_bs, long long w_bs, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  const int ct = pick_ct(bricks(dout) * B, Co);
  if (K == 3 && S == 1)
    return launch_direct<3, 1, 8, 0>(ct, x, W, bias, y, B, din, dout, Ci, Co, x_bs, y_bs, w_bs,
                                     0, stream);
  if (K == 3 && S == 2)
    return launch_direct<3, 2, 4, 0>(ct, x, W, bias, y, B, din, dout, Ci, Co, x_bs, y_bs, w_bs,
                                     0, stream);
  if (K == 1 && S == 1)
    return launch_direct<1, 1, 16, 0>(ct, x, W, bias, y, B, din, dout, Ci, Co, x_bs, y_bs,
                                      w_bs, 0, stream);
  return cudaErrorInvalidValue;
}

cudaError_t conv3d_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din,
                             int Ci, int Co, int K, int S, long long dy_bs, long long dx_bs,
                             long long w_bs, int accumulate, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  if (S == 1) {  // convolution of dy (Co channels) into dx (Ci channels)
    const int ct = pick_ct(bricks(din) * B, Ci);
    if (K == 3)
      return launch_direct<3, 1, 8, 1>(ct, dy, W, nullptr, dx, B, dout, din, Co, Ci, dy_bs,
                                       dx_bs, w_bs, accumulate, stream);
    if (K == 1)
      return launch_direct<1, 1, 16, 1>(ct, dy, W, nullptr, dx, B, dout, din, Co, Ci, dy_bs,
                                        dx_bs, w_bs, accumulate, stream);
    return cudaErrorInvalidValue;
  }
  if (K != 3 || S != 2) return cudaErrorInvalidValue;
  const long long blocks = ceil_div(din.count(), 128);
  const int ct = Ci >= 16 && blocks * B * ceil_div(Ci, 16) >= 304 ? 16
                 : Ci >= 8 && blocks * B * ceil_div(Ci, 8) >= 304 ? 8 : 4;
  dim3 grid((unsigned)blocks, (unsigned)ceil_div(Ci, ct), B);
  switch (ct) {
    case 16:
      dgrad_s2_kernel<16><<<grid, 128, 0, stream>>>(dy, W, dx, din, dout, Ci, Co, dy_bs, dx_bs,
                                                     w_bs, accumulate);
      break;
    case 8:
      dgrad_s2_kernel<8><<<grid, 128, 0, stream>>>(dy, W, dx, din, dout, Ci, Co, dy_bs, dx_bs,
                                                    w_bs, accumulate);
      break;
    default:
      dgrad_s2_kernel<4><<<grid, 128, 0, stream>>>(dy, W, dx, din, dout, Ci, Co, dy_bs, dx_bs,
                                                    w_bs, accumulate);
      break;
  }
  return cudaGetLastError();
}

}  // namespace d2ip
