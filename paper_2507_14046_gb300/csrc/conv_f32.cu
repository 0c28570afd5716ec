// FP32 SIMT weight gradient of the 3D convolutions (3x3x3 stride 1 or 2, and 1x1x1).
//
// dW[co][t][ci] = sum over output voxels v of dy[v][co] x[S*v + k_t - pad][ci] and
// db[co] = sum_v dy[v][co].  One block takes one brick of BZ x BY x 8 output voxels (and one
// group of taps, one 16-wide Co tile and one 16-wide Ci tile): it stages the brick's dy and
// the matching input halo in shared memory once, then every task (one tap x 4 co x 4 ci)
// accumulates its 4 x 4 register tile over the brick's voxels.  Each brick writes its own
// partial sums; a second kernel adds the bricks' rows in a fixed order (deterministic
// split-K over voxels).  Channels-last activations, weights [Co][K^3][Ci].
#include "common.cuh"

namespace d2ip {
namespace {

constexpr int kWBX = 8;  // output brick = BZ x BY x 8 voxels
constexpr int kWThreads = 128;
constexpr int kWTile = 16;         // Co and Ci tile width

template <int K, int S, int BZ, int BY>
__global__ void __launch_bounds__(kWThreads)
wgrad_brick_kernel(const float* __restrict__ x, const float* __restrict__ dy,
                   float* __restrict__ part, Dims3 din, Dims3 dout, int Ci, int Co,
                   long long x_bs, long long dy_bs, int nbricks, int co_tiles, int ci_tiles,
                   int tgroups) {
  constexpr int T = K * K * K, PAD = (K - 1) / 2;
  constexpr int BV = BZ * BY * kWBX;
  constexpr int HZ = (BZ - 1) * S + K, HY = (BY - 1) * S + K, HX = (kWBX - 1) * S + K;
  constexpr int HV = HZ * HY * HX;
  constexpr int NG = kWTile / 4;
  __shared__ float4 sdy[BV * NG];  // [voxel][co group of 4]
  __shared__ float4 sx[HV * NG];   // [halo voxel][ci group of 4]
  const int b = blockIdx.z;
  int q = blockIdx.y;
  const int tg = q % tgroups;
  q /= tgroups;
  const int cit = q % ci_tiles, cot = q / ci_tiles;
  const int co0 = cot * kWTile, ci0 = cit * kWTile;
  const int tpg = (T + tgroups - 1) / tgroups;
  const int t_lo = tg * tpg, t_hi = t_lo + tpg < T ? t_lo + tpg : T;
  x += b * x_bs;
  dy += b * dy_bs;
  const int nbx = (dout.x + kWBX - 1) / kWBX, nby = (dout.y + BY - 1) / BY;
  int bid = blockIdx.x;
  const int bx0 = (bid % nbx) * kWBX;
  bid /= nbx;
  const int by0 = (bid % nby) * BY;
  const int bz0 = (bid / nby) * BZ;
  const int iz0 = bz0 * S - PAD, iy0 = by0 * S - PAD, ix0 = bx0 * S - PAD;

  float* sdyf = reinterpret_cast<float*>(sdy);
  for (int e = threadIdx.x; e < BV * kWTile; e += kWThreads) {
    const int c = e % kWTile, v = e / kWTile;
    const int vx = v % kWBX, vy = (v / kWBX) % BY, vz = v / (kWBX * BY);
    const int oz = bz0 + vz, oy = by0 + vy, ox = bx0 + vx;
    float val = 0.f;
    if (co0 + c < Co && oz < dout.z && oy < dout.y && ox < dout.x)
      val = dy[(((long long)oz * dout.y + oy) * dout.x + ox) * Co + co0 + c];
    sdyf[e] = val;
  }
  float* sxf = reinterpret_cast<float*>(sx);
  for (int e = threadIdx.x; e < HV * kWTile; e += kWThreads) {
    const int c = e % kWTile, h = e / kWTile;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    const int iz = iz0 + hz, iy = iy0 + hy, ix = ix0 + hx;
    float val = 0.f;
    if (ci0 + c < Ci && (unsigned)iz < (unsigned)din.z && (unsigned)iy < (unsigned)din.y &&
        (unsigned)ix < (unsigned)din.x)
      val = x[(((long long)iz * din.y + iy) * din.x + ix) * Ci + ci0 + c];
    sxf[e] = val;
  }
  __syncthreads();

  const long long row = (long long)Co * T * Ci + Co;
  float* out = part + ((long long)b * nbricks + blockIdx.x) * row;
  const int ntask = (t_hi - t_lo) * NG * NG;
  // 1x1x1 layers have only 16 tasks per block: 8 threads share one task's voxels and their
  // 4 x 4 tiles are added in a fixed order through shared memory.  The split depends on the
  // layer alone, so a problem's sums do not depend on the batch it is fitted in.
  constexpr int lanes = K == 1 ? kWThreads / 16 : 1;
  __shared__ float lane_red[K == 1 ? kWThreads : 1][16];
  for (int base = 0; base < ntask * lanes; base += kWThreads) {  // uniform trip count
    const int slot = base + threadIdx.x;
    const int task = slot / lanes, lane = slot % lanes;
    const bool active = task < ntask;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int gi = task % NG, go = (task / NG) % NG, t = t_lo + task / (NG * NG);
    if (active) {
      const int kz = t / (K * K), ky = (t / K) % K, kx = t % K;
      for (int v = lane; v < BV; v += lanes) {
        const int vx = v % kWBX, vy = (v / kWBX) % BY, vz = v / (kWBX * BY);
        const int h = ((vz * S + kz) * HY + (vy * S + ky)) * HX + (vx * S + kx);
        const float4 g = sdy[v * NG + go];
        const float4 a = sx[h * NG + gi];
        const float gg[4] = {g.x, g.y, g.z, g.w}, aa[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(gg[i], aa[j], acc[i][j]);
      }
    }
    if constexpr (lanes > 1) {
#pragma unroll
      for (int e = 0; e < 16; ++e) lane_red[threadIdx.x][e] = acc[e / 4][e % 4];
      __syncthreads();
      if (active && lane == 0)
        for (int q = 1; q < lanes; ++q)
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[e / 4][e % 4] += lane_red[threadIdx.x + q][e];
      __syncthreads();
    }
    if (active && lane == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int co = co0 + go * 4 + i;
        if (co >= Co) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int ci = ci0 + gi * 4 + j;
          if (ci < Ci) out[((long long)co * T + t) * Ci + ci] = acc[i][j];
        }
      }
    }
  }
  if (tg == 0 && cit == 0) {  // bias partial: sum of dy over the brick
    for (int c = threadIdx.x; c < kWTile; c += kWThreads) {
      if (co0 + c >= Co) continue;
      float sum = 0.f;
      for (int v = 0; v < BV; ++v) sum += sdyf[v * kWTile + c];
      out[(long long)Co * T * Ci + co0 + c] = sum;
    }
  }
}

// out[b][j] (=|+=) sum_r part[b][r][j].  A block covers 32 columns with 8 row groups; each
// thread sums the rows r = g, g + 8, ... of its column, then the 8 group sums are added in a
// fixed order (deterministic).
constexpr int kRedCols = 32, kRedGroups = 8;

__global__ void __launch_bounds__(kRedCols * kRedGroups)
reduce_rows_kernel(const float* __restrict__ part, float* __restrict__ out, long long R,
                   long long N, long long out_bs, int accumulate) {
  __shared__ float red[kRedGroups][kRedCols];
  const int b = blockIdx.y;
  const int col = threadIdx.x % kRedCols, g = threadIdx.x / kRedCols;
  const long long j = (long long)blockIdx.x * kRedCols + col;
  float sum = 0.f;
  if (j < N) {
    const float* p = part + (long long)b * R * N + j;
    for (long long r = g; r < R; r += kRedGroups) sum += p[r * N];
  }
  red[g][col] = sum;
  __syncthreads();
  if (g == 0 && j < N) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kRedGroups; ++q) s += red[q][col];
    float* o = out + (long long)b * out_bs + j;
    *o = accumulate ? *o + s : s;
  }
}

// out[b][j] (=|+=) sum_r part[b][r][j] for few rows and many columns: a thread owns four
// adjacent columns and adds the rows in order (four independent loads in flight).
__global__ void __launch_bounds__(256)
reduce_wide_kernel(const float* __restrict__ part, float* __restrict__ out, long long R,
                   long long N, long long out_bs, int accumulate) {
  const int b = blockIdx.y;
  const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (j >= N) return;
  const float* p = part + (long long)b * R * N + j;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  long long r = 0;
  for (; r + 4 <= R; r += 4) {
    const float4 v0 = *reinterpret_cast<const float4*>(p + r * N);
    const float4 v1 = *reinterpret_cast<const float4*>(p + (r + 1) * N);
    const float4 v2 = *reinterpret_cast<const float4*>(p + (r + 2) * N);
    const float4 v3 = *reinterpret_cast<const float4*>(p + (r + 3) * N);
    s.x += v0.x, s.y += v0.y, s.z += v0.z, s.w += v0.w;
    s.x += v1.x, s.y += v1.y, s.z += v1.z, s.w += v1.w;
    s.x += v2.x, s.y += v2.y, s.z += v2.z, s.w += v2.w;
    s.x += v3.x, s.y += v3.y, s.z += v3.z, s.w += v3.w;
  }
  for (; r < R; ++r) {
    const float4 v = *reinterpret_cast<const float4*>(p + r * N);
    s.x += v.x, s.y += v.y, s.z += v.z, s.w += v.w;
  }
  float4* o = reinterpret_cast<float4*>(out + (long long)b * out_bs + j);
  if (accumulate) {
    const float4 q = *o;
    s.x += q.x, s.y += q.y, s.z += q.z, s.w += q.w;
  }
  *o = s;
}

// Few columns, many rows (LayerNorm partials): 32 row groups per column, combined in order.
constexpr int kNarrowGroups = 32;

__global__ void __launch_bounds__(kRedCols * kNarrowGroups)
reduce_narrow_kernel(const float* __restrict__ part, float* __restrict__ out, long long R,
                     long long N, long long out_bs, int accumulate) {
  __shared__ float red[kNarrowGroups][kRedCols + 1];
  const int b = blockIdx.y;
  const int col = threadIdx.x % kRedCols, g = threadIdx.x / kRedCols;
  const long long j = (long long)blockIdx.x * kRedCols + col;
  float s0 = 0.f, s1 = 0.f;
  if (j < N) {
    const float* p = part + (long long)b * R * N + j;
    long long r = g;
    for (; r + kNarrowGroups < R; r += 2 * kNarrowGroups) {
      s0 += p[r * N];
      s1 += p[(r + kNarrowGroups) * N];
    }
    if (r < R) s0 += p[r * N];
  }
  red[g][col] = s0 + s1;
  __syncthreads();
  if (g == 0 && j < N) {
    float s = 0.f;
#pragma unroll 8
    for (int q = 0; q < kNarrowGroups; ++q) s += red[q][col];
    float* o = out + (long long)b * out_bs + j;
    *o = accumulate ? *o + s : s;
  }
}

// Output brick: 2 x 8 x 8 voxels for stride 1, 1 x 4 x 8 for stride 2 (keeps the stride-2
// halo within static shared memory).
int wgrad_bz(int S) { return S == 1 ? 2 : 1; }
int wgrad_by(int S) { return S == 1 ? 8 : 4; }

template <int K, int S, int BZ, int BY>
void launch_wgrad(dim3 grid, const float* x, const float* dy, float* part, Dims3 din,
                  Dims3 dout, int Ci, int Co, long long x_bs, long long dy_bs, int nb, int cot,
                  int cit, int tg, cudaStream_t st) {
  wgrad_brick_kernel<K, S, BZ, BY><<<grid, kWThreads, 0, st>>>(x, dy, part, din, dout, Ci, Co,
                                                            x_bs, dy_bs, nb, cot, cit, tg);
}

}  // namespace

long long conv3d_wgrad_chunks(Dims3 din, int K, int S) {
  const Dims3 d = conv_out_dims(din, K, S);
  return ceil_div(d.x, kWBX) * ceil_div(d.y, wgrad_by(S)) * ceil_div(d.z, wgrad_bz(S));
}

cudaError_t conv3d_wgrad_partial_f32(const float* x, const float* dy, float* part, int B,
                                     Dims3 din, int Ci, int Co, int K, int S, long long x_bs,
                                     long long dy_bs, cudaStream_t stream) {
  const Dims3 dout = conv_out_dims(din, K, S);
  const int nb = (int)conv3d_wgrad_chunks(din, K, S);
  const int cot = (int)ceil_div(Co, kWTile), cit = (int)ceil_div(Ci, kWTile);
  const int T = K * K * K;
  int tg = 1;  // split the taps over blocks until the grid covers the GPU twice
  while (tg < T && (long long)nb * B * cot * cit * tg < 2 * 152) tg *= 3;
  if (tg > T) tg = T;
  dim3 grid(nb, cot * cit * tg, B);
  if (K == 3 && S == 1)
    launch_wgrad<3, 1, 2, 8>(grid, x, dy, part, din, dout, Ci, Co, x_bs, dy_bs, nb, cot, cit, tg,
                          stream);
  else if (K == 3 && S == 2)
    launch_wgrad<3, 2, 1, 4>(grid, x, dy, part, din, dout, Ci, Co, x_bs, dy_bs, nb, cot, cit, tg,
                          stream);
  else if (K == 1 && S == 1)
    launch_wgrad<1, 1, 2, 8>(grid, x, dy, part, din, dout, Ci, Co, x_bs, dy_bs, nb, cot, cit, tg,
                          stream);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t reduce_rows_f32(const float* part, float* out, int B, long long R, long long N,
                            long long out_bs, int accumulate, cudaStream_t stream) {
  const bool vec = N % 4 == 0 && out_bs % 4 == 0 &&
                   ((reinterpret_cast<uintptr_t>(part) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (vec && N >= 1024 && R <= 64) {  // wide: one thread per 4 columns, rows in order
    dim3 grid((unsigned)ceil_div(N / 4, 256), B);
    reduce_wide_kernel<<<grid, 256, 0, stream>>>(part, out, R, N, out_bs, accumulate);
  } else if (N <= 256) {  // narrow: 32 row groups per column
    dim3 grid((unsigned)ceil_div(N, kRedCols), B);
    reduce_narrow_kernel<<<grid, kRedCols * kNarrowGroups, 0, stream>>>(part, out, R, N, out_bs,
                                                                        accumulate);
  } else {
    dim3 grid((unsigned)ceil_div(N, kRedCols), B);
    reduce_rows_kernel<<<grid, kRedCols * kRedGroups, 0, stream>>>(part, out, R, N, out_bs,
                                                                    accumulate);
  }
  return cudaGetLastError();
}

}  // namespace d2ip
