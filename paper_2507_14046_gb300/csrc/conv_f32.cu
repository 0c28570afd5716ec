// FP32 SIMT implicit-GEMM 3D convolution: forward, data gradient, weight gradient.
//
// Convolution of the residual U-Net (3x3x3, stride 1 or 2, zero padding 1, and 1x1x1),
// channels-last activations, weights [Co][K^3][Ci].  Every product is a GEMM whose A
// operand is gathered on the fly from the activation volume:
//   forward : M = output voxels, N = Co, K = taps x Ci
//   dgrad   : M = input voxels,  N = Ci, K = taps x Co (only taps that hit an output voxel)
//   wgrad   : M = Co, N = Ci, K = output voxels of one chunk, one block per (chunk, tap);
//             chunks are summed afterwards in a fixed order (deterministic split-K).
// Tiles are staged in shared memory; each of the 64 threads of a block owns a TM x TN
// register tile of the BM x BN block tile.  Accumulation is FP32 in a fixed order.
#include "common.cuh"

namespace d2ip {
namespace {

constexpr int kThreads = 64;  // 8 x 8 thread grid per block
constexpr int kPadA = 4;      // shared-memory row padding (keeps float4 alignment)

template <int BM, int BN, int BK>
struct Smem {
  float A[BK][BM + kPadA];
  float B[BK][BN + kPadA];
};

template <int BM, int BN, int TM, int TN, int BK>
__device__ __forceinline__ void tile_fma(const Smem<BM, BN, BK>& s, float (&acc)[TM][TN],
                                         int ty, int tx) {
#pragma unroll
  for (int k = 0; k < BK; ++k) {
    float a[TM], b[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = s.A[k][ty * TM + i];
#pragma unroll
    for (int j = 0; j < TN; ++j) b[j] = s.B[k][tx * TN + j];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

// ------------------------------------------------------------------------------------
// forward
// ------------------------------------------------------------------------------------
template <int BN, int BK>
__global__ void __launch_bounds__(kThreads)
conv_fwd_kernel(const float* __restrict__ x, const float* __restrict__ W,
                const float* __restrict__ bias, float* __restrict__ y, Dims3 din, Dims3 dout,
                int Ci, int Co, int K, int S, long long x_bs, long long y_bs, long long w_bs) {
  constexpr int BM = 64, TM = 8, TN = BN / 8;
  __shared__ Smem<BM, BN, BK> s;
  __shared__ int sz[BM], sy[BM], sx[BM];
  const int b = blockIdx.z;
  x += b * x_bs;
  y += b * y_bs;
  W += b * w_bs;
  bias += b * w_bs;
  const long long nout = dout.count();
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int pad = (K - 1) / 2;
  for (int i = threadIdx.x; i < BM; i += kThreads) {
    const long long m = m0 + i;
    if (m < nout) {
      const int ox = (int)(m % dout.x);
      const long long r = m / dout.x;
      const int oy = (int)(r % dout.y);
      const int oz = (int)(r / dout.y);
      sz[i] = oz * S - pad;
      sy[i] = oy * S - pad;
      sx[i] = ox * S - pad;
    } else {
      sz[i] = INT_MIN / 2;
      sy[i] = INT_MIN / 2;
      sx[i] = INT_MIN / 2;
    }
  }
  const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  const int T = K * K * K;
  for (int t = 0; t < T; ++t) {
    const int kz = t / (K * K), ky = (t / K) % K, kx = t % K;
    for (int c0 = 0; c0 < Ci; c0 += BK) {
      __syncthreads();
      for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
        const int i = e / BK, k = e % BK;
        const int iz = sz[i] + kz, iy = sy[i] + ky, ix = sx[i] + kx;
        float v = 0.f;
        if (c0 + k < Ci && (unsigned)iz < (unsigned)din.z && (unsigned)iy < (unsigned)din.y &&
            (unsigned)ix < (unsigned)din.x)
          v = x[(((long long)iz * din.y + iy) * din.x + ix) * Ci + c0 + k];
        s.A[k][i] = v;
      }
      for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
        const int j = e / BK, k = e % BK;
        float v = 0.f;
        if (n0 + j < Co && c0 + k < Ci) v = W[((long long)(n0 + j) * T + t) * Ci + c0 + k];
        s.B[k][j] = v;
      }
      __syncthreads();
      tile_fma<BM, BN, TM, TN, BK>(s, acc, ty, tx);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long m = m0 + ty * TM + i;
    if (m >= nout) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int co = n0 + tx * TN + j;
      if (co < Co) y[m * Co + co] = acc[i][j] + bias[co];
    }
  }
}

// ------------------------------------------------------------------------------------
// data gradient: dx[p, ci] = sum_{t, co} dy[o(p, t), co] W[co][t][ci] over the taps t for
// which p = S*o + k - pad has an integer solution o inside the output grid.
// ------------------------------------------------------------------------------------
template <int BN, int BK>
__global__ void __launch_bounds__(kThreads)
conv_dgrad_kernel(const float* __restrict__ dy, const float* __restrict__ W,
                  float* __restrict__ dx, Dims3 din, Dims3 dout, int Ci, int Co, int K, int S,
                  long long dy_bs, long long dx_bs, long long w_bs, int accumulate) {
  constexpr int BM = 64, TM = 8, TN = BN / 8;
  __shared__ Smem<BM, BN, BK> s;
  __shared__ int sz[BM], sy[BM], sx[BM];
  const int b = blockIdx.z;
  dy += b * dy_bs;
  dx += b * dx_bs;
  W += b * w_bs;
  const long long nin = din.count();
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int pad = (K - 1) / 2;
  for (int i = threadIdx.x; i < BM; i += kThreads) {
    const long long m = m0 + i;
    if (m < nin) {
      const int ix = (int)(m % din.x);
      const long long r = m / din.x;
      const int iy = (int)(r % din.y);
      const int iz = (int)(r / din.y);
      sz[i] = iz + pad;
      sy[i] = iy + pad;
      sx[i] = ix + pad;
    } else {
      sz[i] = INT_MIN / 2;
      sy[i] = INT_MIN / 2;
      sx[i] = INT_MIN / 2;
    }
  }
  const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  const int T = K * K * K;
  for (int t = 0; t < T; ++t) {
    const int kz = t / (K * K), ky = (t / K) % K, kx = t % K;
    for (int c0 = 0; c0 < Co; c0 += BK) {
      __syncthreads();
      for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
        const int i = e / BK, k = e % BK;
        const int nz = sz[i] - kz, ny = sy[i] - ky, nx = sx[i] - kx;  // = S * o
        float v = 0.f;
        if (c0 + k < Co && nz >= 0 && ny >= 0 && nx >= 0 && nz % S == 0 && ny % S == 0 &&
            nx % S == 0) {
          const int oz = nz / S, oy = ny / S, ox = nx / S;
          if (oz < dout.z && oy < dout.y && ox < dout.x)
            v = dy[(((long long)oz * dout.y + oy) * dout.x + ox) * Co + c0 + k];
        }
        s.A[k][i] = v;
      }
      for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
        const int k = e / BN, j = e % BN;
        float v = 0.f;
        if (n0 + j < Ci && c0 + k < Co) v = W[((long long)(c0 + k) * T + t) * Ci + n0 + j];
        s.B[k][j] = v;
      }
      __syncthreads();
      tile_fma<BM, BN, TM, TN, BK>(s, acc, ty, tx);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long m = m0 + ty * TM + i;
    if (m >= nin) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int ci = n0 + tx * TN + j;
      if (ci < Ci) {
        float* p = dx + m * Ci + ci;
        *p = accumulate ? *p + acc[i][j] : acc[i][j];
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// weight gradient, one (chunk of output voxels, tap, Co tile, Ci tile) per block
// ------------------------------------------------------------------------------------
constexpr int kWgradBK = 16;

template <int BM, int BN>
__global__ void __launch_bounds__(kThreads)
conv_wgrad_kernel(const float* __restrict__ x, const float* __restrict__ dy,
                  float* __restrict__ part, Dims3 din, Dims3 dout, int Ci, int Co, int K, int S,
                  long long x_bs, long long dy_bs, int chunk_vox, int nchunks, int co_tiles,
                  int ci_tiles) {
  constexpr int BK = kWgradBK, TM = BM / 8, TN = BN / 8;
  __shared__ Smem<BM, BN, BK> s;
  __shared__ int sz[BK], sy[BK], sx[BK];
  const int tiles = co_tiles * ci_tiles;
  const int b = blockIdx.z / tiles;
  const int tile = blockIdx.z % tiles;
  const int co0 = (tile / ci_tiles) * BM;
  const int ci0 = (tile % ci_tiles) * BN;
  const int chunk = blockIdx.x;
  const int t = blockIdx.y;
  const int T = K * K * K;
  const int kz = t / (K * K), ky = (t / K) % K, kx = t % K;
  const int pad = (K - 1) / 2;
  x += b * x_bs;
  dy += b * dy_bs;
  const long long nout = dout.count();
  const long long v0 = (long long)chunk * chunk_vox;
  const long long v1 = v0 + chunk_vox < nout ? v0 + chunk_vox : nout;
  const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  for (long long vb = v0; vb < v1; vb += BK) {
    __syncthreads();
    if (threadIdx.x < BK) {
      const long long v = vb + threadIdx.x;
      if (v < v1) {
        const int ox = (int)(v % dout.x);
        const long long r = v / dout.x;
        const int oy = (int)(r % dout.y);
        const int oz = (int)(r / dout.y);
        sz[threadIdx.x] = oz * S - pad + kz;
        sy[threadIdx.x] = oy * S - pad + ky;
        sx[threadIdx.x] = ox * S - pad + kx;
      } else {
        sz[threadIdx.x] = -1;
        sy[threadIdx.x] = -1;
        sx[threadIdx.x] = -1;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
      const int k = e / BM, i = e % BM;
      const long long v = vb + k;
      s.A[k][i] = (v < v1 && co0 + i < Co) ? dy[v * Co + co0 + i] : 0.f;
    }
    for (int e = threadIdx.x; e < BN * BK; e += kThreads) {
      const int k = e / BN, j = e % BN;
      const int iz = sz[k], iy = sy[k], ix = sx[k];
      float v = 0.f;
      if (ci0 + j < Ci && (unsigned)iz < (unsigned)din.z && (unsigned)iy < (unsigned)din.y &&
          (unsigned)ix < (unsigned)din.x)
        v = x[(((long long)iz * din.y + iy) * din.x + ix) * Ci + ci0 + j];
      s.B[k][j] = v;
    }
    __syncthreads();
    tile_fma<BM, BN, TM, TN, BK>(s, acc, ty, tx);
  }
  const long long row = (long long)Co * T * Ci + Co;
  float* out = part + ((long long)b * nchunks + chunk) * row;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int co = co0 + ty * TM + i;
    if (co >= Co) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int ci = ci0 + tx * TN + j;
      if (ci < Ci) out[((long long)co * T + t) * Ci + ci] = acc[i][j];
    }
  }
  if (t == 0 && (tile % ci_tiles) == 0) {
    for (int i = threadIdx.x; i < BM; i += kThreads) {
      const int co = co0 + i;
      if (co >= Co) continue;
      float sum = 0.f;
      for (long long v = v0; v < v1; ++v) sum += dy[v * Co + co];
      out[(long long)Co * T * Ci + co] = sum;
    }
  }
}

__global__ void reduce_rows_kernel(const float* __restrict__ part, float* __restrict__ out,
                                   long long R, long long N, long long out_bs, int accumulate) {
  const int b = blockIdx.y;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const float* p = part + (long long)b * R * N + j;
  float sum = 0.f;
  for (long long r = 0; r < R; ++r) sum += p[r * N];
  float* o = out + (long long)b * out_bs + j;
  *o = accumulate ? *o + sum : sum;
}

inline int pick_bn(int n) { return n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }

}  // namespace

cudaError_t conv3d_fwd_f32(const float* x, const float* W, const float* bias, float* y,
                           int B, Dims3 din, int Ci, int Co, int K, int S, long long x_bs,
                           long long y_bs, long long w_bs, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  const int bn = pick_bn(Co);
  dim3 grid((unsigned)ceil_div(dout.count(), 64), (unsigned)ceil_div(Co, bn), B);
  const bool k16 = (Ci % 16) == 0;
#define D2IP_FWD(BN_, BK_) \
  conv_fwd_kernel<BN_, BK_><<<grid, kThreads, 0, stream>>>(x, W, bias, y, din, dout, Ci, Co, \
                                                           K, S, x_bs, y_bs, w_bs)
  switch (bn) {
    case 8: if (k16) D2IP_FWD(8, 16); else D2IP_FWD(8, 8); break;
    case 16: if (k16) D2IP_FWD(16, 16); else D2IP_FWD(16, 8); break;
    case 32: if (k16) D2IP_FWD(32, 16); else D2IP_FWD(32, 8); break;
    default: if (k16) D2IP_FWD(64, 16); else D2IP_FWD(64, 8); break;
  }
#undef D2IP_FWD
  return cudaGetLastError();
}

cudaError_t conv3d_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din,
                             int Ci, int Co, int K, int S, long long dy_bs, long long dx_bs,
                             long long w_bs, int accumulate, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  const int bn = pick_bn(Ci);
  dim3 grid((unsigned)ceil_div(din.count(), 64), (unsigned)ceil_div(Ci, bn), B);
  const bool k16 = (Co % 16) == 0;
#define D2IP_DG(BN_, BK_) \
  conv_dgrad_kernel<BN_, BK_><<<grid, kThreads, 0, stream>>>(dy, W, dx, din, dout, Ci, Co, K, \
                                                             S, dy_bs, dx_bs, w_bs, accumulate)
  switch (bn) {
    case 8: if (k16) D2IP_DG(8, 16); else D2IP_DG(8, 8); break;
    case 16: if (k16) D2IP_DG(16, 16); else D2IP_DG(16, 8); break;
    case 32: if (k16) D2IP_DG(32, 16); else D2IP_DG(32, 8); break;
    default: if (k16) D2IP_DG(64, 16); else D2IP_DG(64, 8); break;
  }
#undef D2IP_DG
  return cudaGetLastError();
}

static long long wgrad_chunk_vox(long long nout) {
  long long c = ceil_div(nout, 64);
  c = ceil_div(c, kWgradBK) * kWgradBK;
  return c < 256 ? 256 : c;
}

long long conv3d_wgrad_chunks(Dims3 din, int K, int S) {
  const long long nout = conv_out_dims(din, K, S).count();
  return ceil_div(nout, wgrad_chunk_vox(nout));
}

cudaError_t conv3d_wgrad_partial_f32(const float* x, const float* dy, float* part, int B,
                                     Dims3 din, int Ci, int Co, int K, int S, long long x_bs,
                                     long long dy_bs, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  const long long nout = dout.count();
  const int cv = (int)wgrad_chunk_vox(nout);
  const int nch = (int)ceil_div(nout, cv);
  const int bm = pick_bn(Co), bn = pick_bn(Ci);
  const int cot = (int)ceil_div(Co, bm), cit = (int)ceil_div(Ci, bn);
  dim3 grid(nch, K * K * K, B * cot * cit);
#define D2IP_WG(BM_, BN_)                                                                 \
  conv_wgrad_kernel<BM_, BN_><<<grid, kThreads, 0, stream>>>(x, dy, part, din, dout, Ci, Co, \
                                                             K, S, x_bs, dy_bs, cv, nch, cot, \
                                                             cit)
#define D2IP_WG_N(BM_)                   \
  switch (bn) {                          \
    case 8: D2IP_WG(BM_, 8); break;      \
    case 16: D2IP_WG(BM_, 16); break;    \
    case 32: D2IP_WG(BM_, 32); break;    \
    default: D2IP_WG(BM_, 64); break;    \
  }
  switch (bm) {
    case 8: D2IP_WG_N(8); break;
    case 16: D2IP_WG_N(16); break;
    case 32: D2IP_WG_N(32); break;
    default: D2IP_WG_N(64); break;
  }
#undef D2IP_WG_N
#undef D2IP_WG
  return cudaGetLastError();
}

cudaError_t reduce_rows_f32(const float* part, float* out, int B, long long R, long long N,
                            long long out_bs, int accumulate, cudaStream_t stream) {
  dim3 grid((unsigned)ceil_div(N, 256), B);
  reduce_rows_kernel<<<grid, 256, 0, stream>>>(part, out, R, N, out_bs, accumulate);
  return cudaGetLastError();
}

}  // namespace d2ip
