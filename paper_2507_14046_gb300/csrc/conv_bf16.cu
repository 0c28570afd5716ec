// Implicit-GEMM 3D convolution on the 5th-generation tensor cores (tcgen05), sm_103a.
//
// GEMM view: D[M = output voxels][N = Co] = sum over taps t and input channels c of
// A_t[voxel][c] * W[co][t][c], accumulated in FP32 in tensor memory (TMEM).
//
// * A tile: 128 output voxels = an 8 x 4 x 4 (x, y, z) box.  For tap t and channel chunk c0
//   its im2col rows are exactly one TMA box of the channels-last input volume, shifted by
//   the tap offset (and traversed with element stride 2 for the stride-2 convolutions); the
//   zero padding of the convolution is TMA's out-of-bounds fill, so the halo costs nothing.
//   The box lands in shared memory in the K-major swizzled layout the MMA reads (32/64/128-byte
//   swizzle for 16/32/64-channel chunks).
// * B tile: the [Co][chunk] weights of tap t, one TMA box of the BF16 weight copy.
// * One thread of warp 1 issues tcgen05.mma (M 128, N Co, K 16) and commits each stage
//   back to the producer; one thread of warp 0 issues the TMA loads into a 4-stage ring
//   guarded by mbarriers; after the last MMA all four warps read their 32 TMEM lanes
//   (thread = output voxel, registers = its Co channels) and write FP32 results.
// Every wait on an mbarrier is bounded by a clock budget; on expiry the kernel records an
// error code, lets the in-flight MMAs drain, frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>

#include "conv_bf16.cuh"
#include "tc_prims.cuh"

namespace d2ip {
namespace {

constexpr int kBX = 8, kBY = 4, kBZ = 4;  // output voxel box of one 128-row tile
constexpr int kBM = kBX * kBY * kBZ;
constexpr int kStages = 4;
// Taps of one launch: the input box of tap j starts at origin * s_in + off[j] (x, y, z), its
// weights are tap widx[j] of the weight tensor, and the tile's output voxel q is written at
// q * s_out + r.  A forward convolution is one class of 27 (or 1) taps; the stride-2 data
// gradient is 8 classes, one per output parity, of 1, 2, 4 or 8 taps -- or, packed (pack =
// 8), one CTA per tile whose 8 "taps" are the coarse windows (ox, oy, oz) in {0, 1}^3 and
// whose N holds all 8 classes side by side: class p = px + 2 py + 4 pz takes columns
// [p n0, p n0 + n0) and writes parity r = (px, py, pz); a window's weight block for a class
// that does not read it is zero.
struct TapClass {
  int n;
  int8_t off[27][3];
  uint8_t widx[27];
  int8_t r[3];
};
struct TapPlan {
  int s_in, s_out;
  int pack;  // 0: one class per CTA (blockIdx.y); 8: the packed stride-2 data gradient
  int fold;  // split rows (pack 0): N = 2 n0, output channel c is D[c] + D[n0 + c]
  TapClass cls[8];
};

// 16 accumulator columns of this warp's lanes; with off, plus the 16 columns off further on
// (the two halves of a folded accumulator).
__device__ __forceinline__ void tmem_ld16f(uint32_t taddr, uint32_t (&r)[16], uint32_t off) {
  tmem_ld16(taddr, r);
  if (off) {
    uint32_t r2[16];
    tmem_ld16(taddr + off, r2);
#pragma unroll
    for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r2[j]));
  }
}

template <int CK>
__global__ void __launch_bounds__(128, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
               const __grid_constant__ TapPlan plan, const float* __restrict__ bias,
               float* __restrict__ out, Dims3 dout, int N, int nchunks, int tiles_x,
               int tiles_y, long long out_bs, long long bias_bs, int accumulate,
               int* __restrict__ err) {
  constexpr uint32_t kABytes = kBM * CK * 2;
  const uint32_t b_bytes = (uint32_t)N * CK * 2;
  const uint32_t stage_bytes = kABytes + b_bytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t tmem_base_s;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int b = blockIdx.z;
  const int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * kBX;
  const int y0 = ((tile / tiles_x) % tiles_y) * kBY;
  const int z0 = (tile / (tiles_x * tiles_y)) * kBZ;
  const TapClass& cls = plan.cls[blockIdx.y];
  const int ksteps = cls.n * nchunks;
  const uint32_t tmem_cols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {  // TMA producer
    int k = 0;
    for (; k < ksteps; ++k) {
      const int s = k % kStages, round = k / kStages;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (round - 1) & 1)) {
        atomicOr(err, kErrProducer);
        break;
      }
      const int j = k / nchunks, c = k % nchunks;
      const uint32_t a_dst = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, stage_bytes);
      tma_load_5d(a_dst, &tm_a, c * CK, x0 * plan.s_in + cls.off[j][0],
                  y0 * plan.s_in + cls.off[j][1], z0 * plan.s_in + cls.off[j][2], b, fb);
      tma_load_4d(a_dst + kABytes, &tm_b, c * CK, 0, cls.widx[j], b, fb);
    }
    drain_loads(full_bar, kStages, k, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc(N);
    for (int k = 0; k < ksteps; ++k) {
      const int s = k % kStages;
      if (!mbar_wait(smem_u32(&full_bar[s]), (k / kStages) & 1)) {
        atomicOr(err, kErrMma);
        break;
      }
      tc_fence_after();
      const uint32_t a_addr = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t b_addr = a_addr + kABytes;
#pragma unroll
      for (int kk = 0; kk < CK / 16; ++kk)
        mma_bf16(tmem, smem_desc<CK>(a_addr + kk * 32), smem_desc<CK>(b_addr + kk * 32), idesc,
                 (k > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&done_bar));  // fires once every issued MMA has completed
  }
  __syncwarp();

  const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
  if (!ok && lane == 0) atomicOr(err, kErrEpilogue);
  tc_fence_after();
  if (ok) {
    const int m = warp * 32 + lane;  // TMEM lane = tile row = voxel of the box
    // output channels (columns of one class; folded: half the columns, added to the other)
    const int n0 = plan.pack ? N / plan.pack : plan.fold ? N / 2 : N;
    const int ncol = plan.fold ? n0 : N;
    const float* bb = bias ? bias + (long long)b * bias_bs : nullptr;
    for (int c0 = 0; c0 < ncol; c0 += 16) {
      const int p = c0 / n0, cc = c0 - p * n0;  // packed: class p, its channel cc
      const int rx = plan.pack ? (p & 1) : cls.r[0], ry = plan.pack ? (p >> 1) & 1 : cls.r[1],
                rz = plan.pack ? (p >> 2) & 1 : cls.r[2];
      const int ox = (x0 + m % kBX) * plan.s_out + rx,
                oy = (y0 + (m / kBX) % kBY) * plan.s_out + ry,
                oz = (z0 + m / (kBX * kBY)) * plan.s_out + rz;
      const bool inside = ox < dout.x && oy < dout.y && oz < dout.z;
      const long long vox = ((long long)oz * dout.y + oy) * dout.x + ox;
      float* o = out + (long long)b * out_bs + vox * n0 + cc;
      uint32_t r[16];
      tmem_ld16f(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r,
                 plan.fold ? (uint32_t)n0 : 0u);
      if (inside && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {  // 16-byte stores
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          float4 v = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                 __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
          if (bb) v.x += bb[cc + j], v.y += bb[cc + j + 1], v.z += bb[cc + j + 2],
                  v.w += bb[cc + j + 3];
          float4* d = reinterpret_cast<float4*>(o + j);
          if (accumulate) {
            const float4 a = *d;
            v.x += a.x, v.y += a.y, v.z += a.z, v.w += a.w;
          }
          *d = v;
        }
      } else if (inside) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float v = __uint_as_float(r[j]) + (bb ? bb[cc + j] : 0.f);
          o[j] = accumulate ? o[j] + v : v;
        }
      }
    }
  }
  tc_fence_before();
  // TMEM is freed only once the last commit showed every issued MMA complete; otherwise the
  // error word is set and the columns stay allocated
  const int drained = __syncthreads_and(ok ? 1 : 0);
  if (warp == 1 && drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// 3x3x3 stride-1 convolution with halo boxes.  Tile = 8 x 16 x TZ output voxels (TZ = 1, 2
// or 4 z slices of 128 rows, row m = y * 8 + x).  Per stage (channel chunk, x tap kx) one TMA
// box of 8 x 18 x (TZ + 2) voxels holds the input shifted by kx - 1 in x with a one-voxel
// halo in y and z; tap (ky, kz) of slice zz is the window that starts ((zz + kz) * 18 + ky) * 8
// rows in -- whole swizzle atoms, so each is an ordinary K-major operand.  The stage's B box
// holds the nine taps t = kx + 3 q (TMA element stride 3 along the tap axis of the tap-major
// weights).  Slice zz accumulates in TMEM columns [zz N, zz N + N).  The epilogue moves each
// slice through shared memory (rows padded to N + 4 floats: conflict-free 16-byte writes) and
// stores it with coalesced 16-byte accesses.
// ------------------------------------------------------------------------------------
constexpr int kT3Max = 4;  // pipeline stages (at most)

template <int CK>
__global__ void __launch_bounds__(128, 1)
conv_tc3_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
                const float* __restrict__ bias, float* __restrict__ out, Dims3 dout, int N,
                int nchunks, int tiles_x, int tiles_y, int TZ, long long out_bs,
                long long bias_bs, int accumulate, int nst, int* __restrict__ err) {
  constexpr uint32_t kRowB = CK * 2;
  const uint32_t a_bytes = (uint32_t)(8 * 18 * (TZ + 2)) * kRowB;
  const uint32_t b_tap = (uint32_t)N * CK * 2;
  const uint32_t stage_bytes = a_bytes + 9 * b_tap;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kT3Max], empty_bar[kT3Max], done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ __align__(16) float sbias[256];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int b = blockIdx.z;
  for (int c = threadIdx.x; c < N; c += blockDim.x)
    sbias[c] = bias ? bias[(long long)b * bias_bs + c] : 0.f;
  int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * 8;
  tile /= tiles_x;
  const int y0 = (tile % tiles_y) * 16;
  const int z0 = (tile / tiles_y) * TZ;
  const int ksteps = nchunks * 3;
  const int cols = TZ * N;
  const uint32_t tmem_cols = cols <= 32 ? 32u : cols <= 64 ? 64u : cols <= 128 ? 128u
                                                : cols <= 256 ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int q = 0; q < nst; ++q) {
      mbar_init(smem_u32(&full_bar[q]), 1);
      mbar_init(smem_u32(&empty_bar[q]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {  // TMA producer
    int k = 0;
    for (; k < ksteps; ++k) {
      const int st = k % nst, round = k / nst;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[st]), (round - 1) & 1)) {
        atomicOr(err, kErrProducer);
        break;
      }
      const int c = k / 3, kx = k % 3;
      const uint32_t dst = smem_u32(smem + (size_t)st * stage_bytes);
      const uint32_t fb = smem_u32(&full_bar[st]);
      mbar_expect_tx(fb, stage_bytes);
      tma_load_5d(dst, &tm_a, c * CK, x0 + kx - 1, y0 - 1, z0 - 1, b, fb);
      tma_load_4d(dst + a_bytes, &tm_b, c * CK, 0, kx, b, fb);
    }
    drain_loads(full_bar, nst, k, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc(N);
    for (int k = 0; k < ksteps; ++k) {
      const int st = k % nst;
      if (!mbar_wait(smem_u32(&full_bar[st]), (k / nst) & 1)) {
        atomicOr(err, kErrMma);
        break;
      }
      tc_fence_after();
      // descriptors are linear in the address (start >> 4 in the low field): offset a base
      const uint32_t a_addr = smem_u32(smem + (size_t)st * stage_bytes);
      const uint64_t a0 = smem_desc<CK>(a_addr), b0 = smem_desc<CK>(a_addr + a_bytes);
#pragma unroll 1
      for (int q = 0; q < 9; ++q) {  // tap t = kx + 3 q: kz = q / 3, ky = q % 3
        const uint64_t bq = b0 + ((q * b_tap) >> 4);
        const uint32_t acc = (k > 0 || q > 0) ? 1u : 0u;
#pragma unroll 1
        for (int zz = 0; zz < TZ; ++zz) {
          const uint64_t aq = a0 + ((((zz + q / 3) * 18 + (q % 3)) * 8 * kRowB) >> 4);
#pragma unroll
          for (int kk = 0; kk < CK / 16; ++kk)
            mma_bf16(tmem + (uint32_t)(zz * N), aq + kk * 2, bq + kk * 2, idesc,
                     (acc | kk) ? 1u : 0u);
        }
      }
      mma_commit(smem_u32(&empty_bar[st]));
    }
    mma_commit(smem_u32(&done_bar));
  }
  __syncwarp();

  const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
  if (!ok && lane == 0) atomicOr(err, kErrEpilogue);
  tc_fence_after();
  // every warp reached done_bar: all loads were consumed and all MMAs completed, so the
  // pipeline buffers are free for the output staging
  const int okall = __syncthreads_and(ok ? 1 : 0);
  if (okall) {
    const int m = warp * 32 + lane;
    const int ld = N + 4;  // padded staging row (floats)
    float* stg = reinterpret_cast<float*>(smem);
    const int n4 = N / 4;
    for (int zz = 0; zz < TZ; ++zz) {
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(zz * N + c0), r);
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          float4 v = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                 __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
          const float4 bv = *reinterpret_cast<const float4*>(sbias + c0 + j);
          v.x += bv.x, v.y += bv.y, v.z += bv.z, v.w += bv.w;
          *reinterpret_cast<float4*>(stg + m * ld + c0 + j) = v;
        }
      }
      __syncthreads();
      const int oz = z0 + zz;
      if (oz < dout.z) {
        for (int i = threadIdx.x; i < 128 * n4; i += blockDim.x) {
          const int mv = i / n4, c4 = i % n4;
          const int ox = x0 + mv % 8, oy = y0 + mv / 8;
          if (ox >= dout.x || oy >= dout.y) continue;
          float4 v = *reinterpret_cast<const float4*>(stg + mv * ld + c4 * 4);
          float4* o = reinterpret_cast<float4*>(
              out + (long long)b * out_bs + (((long long)oz * dout.y + oy) * dout.x + ox) * N) + c4;
          if (accumulate) {
            const float4 p = *o;
            v.x += p.x, v.y += p.y, v.z += p.z, v.w += p.w;
          }
          *o = v;
        }
      }
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1 && okall) {  // TMEM is freed only after the last commit showed the MMAs done
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// Persistent, warp-specialised form of the halo-box convolution.  One CTA per SM walks the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... of all problems.  Warp 0 (one thread) keeps
// the TMA ring full across tile boundaries, warp 1 (one thread) issues the MMAs of tile i
// into TMEM accumulator buffer i % 2, and warps 2..5 drain the other buffer (TMEM -> bias ->
// shared-memory staging -> coalesced global stores) while the next tile is multiplied.
// Barriers: full/empty per ring stage (TMA <-> MMA), tfull/tempty per accumulator buffer
// (MMA <-> epilogue).  Every wait is bounded; a wait that runs out records an error bit and
// its role stops, the others then run out too, and before TMEM is freed the MMA thread's
// last commit and the producer's last loads are awaited (bounded).
// ------------------------------------------------------------------------------------
constexpr int kP3Max = 4;


// The persistent halo convolution has kEpiGroups epilogue warpgroups (warps 2..5, 6..9), each
// covering the four TMEM lane quadrants and taking alternate output slices of a tile; group g
// synchronises on named barrier 1 + g.
constexpr int kEpiGroups = 2;
constexpr int kTc3pThreads = 64 + 128 * kEpiGroups;

__device__ __forceinline__ void epi_sync(int grp) {  // the four warps of one epilogue group
  asm volatile("bar.sync %0, 128;" ::"r"(1 + grp) : "memory");
}

// true on every thread of epilogue group grp iff p holds on all 128 of them
__device__ __forceinline__ bool epi_all(bool p, int grp) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred a, q;\n\t"
      "setp.ne.u32 a, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 128, a;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(p ? 1u : 0u), "r"(1 + grp)
      : "memory");
  return r != 0;
}

// Launch arguments of the persistent halo convolution.  mode 0: y = conv(x) + bias.
// mode 1 (forward of a block with a 1x1 projection of the same input): also
// y_p = W_p x + bias_p, from one more MMA per slice on the centre window of the kx = 1 stage.
// mode 2 (data gradient of such a block): dx = conv^T(dz) + W_p^T dz_p, the second term from
// one more stage per channel chunk (the dz_p box of the tile, no halo).
// pack: the three kz taps of one (ky, kx) in one MMA of width 3N.  The layer's weights are
// then stored with ky and kz swapped, so the B box of an x tap holds, for each ky, the kz
// taps 0, 1, 2 as adjacent N-row blocks.  The window of input slice s (= zz + kz) and ky
// feeds output slices s, s - 1, s - 2 through the three column blocks of one MMA written at
// column (TZ + 1 - s) N: slice zz's accumulator sits at (TZ + 1 - zz) N, and blocks that fall
// outside [0, TZ) land in spare columns.  Every MMA accumulates; the epilogue warps zero an
// accumulator buffer before handing it back (and both at the start).  9 TZ MMAs of width N
// per stage become 3 (TZ + 2) of width 3N, at nearly the same issue cost each.
struct P3Args {
  const float* bias;
  float* out;
  const float* bias_p;
  float* out_p;
  int* err;
  Dims3 dout;
  int N, Np, nchunks, tiles_x, tiles_y, tiles_z, B, accumulate, nst, mode, pack;
  int fold;  // N = 2 outputs: output channel c is D[c] + D[N / 2 + c] (split rows, mode 0)
  int split_c;  // > 0: output channels from split_c on go to tm_outp (at channel - split_c)
  uint32_t ring_bytes, stage_bytes;
  uint32_t slice_bytes;  // one epilogue staging slice (128 rows of FP32 outputs, and with the
                         // LayerNorm also xhat and the BF16 copy); per epilogue group, nbuf of
                         // them after the ring, then the groups' bias, gamma and beta copies
  int nbuf;
  long long out_bs, bias_bs, outp_bs, biasp_bs;
  // LayerNorm epilogue (ln = 1, output part 0): y = act(gamma * xhat + beta (+ resid)) with
  // xhat = (z - mean) * rstd over the N channels of each voxel (z = the convolution + bias);
  // y through tm_out, xhat through tm_xh, rstd[b][voxel] directly and, with ybf, a BF16 copy
  // of y in sp channel blocks (stage_bf16x4's layout) through tm_ybf.  z is not stored.
  // LayerNorm backward epilogue (ln = 2, mode 0): the data gradient D (+ resid, a gradient
  // already accumulated for the same tensor) is the gradient of a = act(LN(z) ...), the
  // output of the block before; with dp = D act'(a) (the mask from a >= 0 as stored),
  // dz = rstd (gamma dp - mean(gamma dp) - xhat mean(gamma dp xhat)) over the N channels
  // goes to the BF16 staging through tm_ybf (and, when out is set, as FP32 through tm_out);
  // the sums of dp xhat and dp (the dgamma, dbeta terms) over the voxels of the slices an
  // epilogue group takes from a tile go to row tile * kEpiGroups + group of part[b] (2 N
  // floats; rows_b rows per problem).
  int ln, act, ybf, sp;
  const float* gamma;  // gamma[c], then beta[c] at gamma + N, per problem at gamma_bs
  long long gamma_bs;
  const float* resid;  // [b][voxel][N] at resid_bs, or null
  long long resid_bs;
  float* rstd;         // [b][voxel] at rstd_bs (an input of the backward)
  long long rstd_bs;
  const float* aout;   // backward: a [b][voxel][N] at resid_bs
  const float* xh_in;  // backward: xhat [b][voxel][N] at resid_bs
  float* part;         // backward: [b][rows_b][2 N]
  long long rows_b;
};

// 16-byte chunk index inside a staged row of R bytes (R = 32, 64 or 128) under the TMA
// swizzle of that width: the chunk bits XORed with the row's position in its 8-row (R 128),
// 4-pair (R 64) or 2-quad (R 32) atom.
__device__ __forceinline__ int swz_chunk(int chunk, int m, int R) {
  return chunk ^ ((m * R >> 7) & (R / 16 - 1));
}


// Channels c0..c0+15 of tile row m, values o, into the epilogue's BF16 staging slice: sp
// blocks (hi; or hi, lo, hi) of 128 rows x nc channels, each the swizzled rows of one
// output box (2 nc bytes per row).
__device__ __forceinline__ void stage_slice_bf16(__nv_bfloat16* YB, int m, int nc, int c0,
                                                 const float (&o)[16], int sp) {
#pragma unroll
  for (int j = 0; j < 16; j += 8) {
    __nv_bfloat162 h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = __floats2bfloat162_rn(o[j + 2 * u], o[j + 2 * u + 1]);
      const float2 f = __bfloat1622float2(h[u]);
      l[u] = __floats2bfloat162_rn(o[j + 2 * u] - f.x, o[j + 2 * u + 1] - f.y);
    }
    const int ch = swz_chunk((c0 + j) / 8, m, 2 * nc);
    uint4 uh, ul;
    uh.x = *reinterpret_cast<uint32_t*>(&h[0]), uh.y = *reinterpret_cast<uint32_t*>(&h[1]);
    uh.z = *reinterpret_cast<uint32_t*>(&h[2]), uh.w = *reinterpret_cast<uint32_t*>(&h[3]);
    ul.x = *reinterpret_cast<uint32_t*>(&l[0]), ul.y = *reinterpret_cast<uint32_t*>(&l[1]);
    ul.z = *reinterpret_cast<uint32_t*>(&l[2]), ul.w = *reinterpret_cast<uint32_t*>(&l[3]);
    __nv_bfloat16* yb = YB + m * nc + ch * 8;
    *reinterpret_cast<uint4*>(yb) = uh;  // blocks hi, lo, hi
    if (sp > 1) {
      *reinterpret_cast<uint4*>(yb + 128 * nc) = ul;
      *reinterpret_cast<uint4*>(yb + 256 * nc) = uh;
    }
  }
}

template <int CK, int TZ>
__global__ void __launch_bounds__(kTc3pThreads, 1)
conv_tc3p_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
                 const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_a2,
                 const __grid_constant__ CUtensorMap tm_out,
                 const __grid_constant__ CUtensorMap tm_outp,
                 const __grid_constant__ CUtensorMap tm_xh,
                 const __grid_constant__ CUtensorMap tm_ybf, const __grid_constant__ P3Args g) {
  constexpr uint32_t kRowB = CK * 2;
  constexpr uint32_t a_bytes = (uint32_t)(8 * 18 * (TZ + 2)) * kRowB;
  const int N = g.N, Np = g.mode == 1 ? g.Np : 0;
  const uint32_t b_tap = (uint32_t)N * CK * 2;
  const uint32_t stage_bytes = g.stage_bytes;
  const int spc = g.mode == 2 ? 4 : 3;  // stages per channel chunk
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  // epilogue: two staging slices (each box of w channels stored as the swizzled rows the
  // output tensor map expects), then the bias of the current problem
  float* stg = reinterpret_cast<float*>(smem + g.ring_bytes);
  float* sbias0 = reinterpret_cast<float*>(smem + g.ring_bytes +
                                           (size_t)kEpiGroups * g.nbuf * g.slice_bytes);
  __shared__ __align__(8) uint64_t full_bar[kP3Max], empty_bar[kP3Max], tfull[2], tempty[2],
      done_bar;
  __shared__ uint32_t tmem_base_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int per_b = g.tiles_x * g.tiles_y * g.tiles_z;
  const int total = per_b * g.B;
  const int ntile = blockIdx.x < total ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int ksteps = g.nchunks * spc;
  const int nst = g.nst;
  const bool pack = g.pack != 0;
  // one accumulator buffer: TZ slices of N (+ Np); packed: TZ + 4 blocks of N (+ TZ Np)
  const int acc_cols = pack ? (TZ + 4) * N + TZ * Np : TZ * (N + Np);
  const int pbase = pack ? (TZ + 4) * N : TZ * N;  // projection accumulators
  const int cols = 2 * acc_cols;
  const uint32_t tmem_cols = cols <= 32 ? 32u : cols <= 64 ? 64u : cols <= 128 ? 128u
                                                : cols <= 256 ? 256u : 512u;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nst; ++q) {
      mbar_init(smem_u32(&full_bar[q]), 1);
      mbar_init(smem_u32(&empty_bar[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);
      mbar_init(smem_u32(&tempty[q]), 128 * kEpiGroups);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int k = 0;      // ring position, continuous over tiles
      bool good = true;
      const uint32_t wp_bytes = (uint32_t)Np * CK * 2;
      const uint32_t a2_bytes = (uint32_t)(128 * TZ) * kRowB + b_tap;
      for (int i = 0; i < ntile && good; ++i) {
        int tile = blockIdx.x + i * gridDim.x;
        const int b = tile / per_b;
        tile %= per_b;
        const int x0 = (tile % g.tiles_x) * 8;
        tile /= g.tiles_x;
        const int y0 = (tile % g.tiles_y) * 16;
        const int z0 = (tile / g.tiles_y) * TZ;
        for (int j = 0; j < ksteps; ++j, ++k) {
          const int st = k % nst, round = k / nst;
          if (round > 0 && !mbar_wait(smem_u32(&empty_bar[st]), (round - 1) & 1)) {
            atomicOr(g.err, kErrProducer);
            good = false;
            break;
          }
          const int c = j / spc, kx = j % spc;
          const uint32_t dst = smem_u32(smem + (size_t)st * stage_bytes);
          const uint32_t fb = smem_u32(&full_bar[st]);
          if (kx == 3) {  // mode 2: dz_p box of the tile and W_p^T chunk c
            mbar_expect_tx(fb, a2_bytes);
            tma_load_5d(dst, &tm_a2, c * CK, x0, y0, z0, b, fb);
            tma_load_4d(dst + (uint32_t)(128 * TZ) * kRowB, &tm_p, c * CK, 0, 0, b, fb);
          } else {
            const bool wp = Np > 0 && kx == 1;
            mbar_expect_tx(fb, a_bytes + 9 * b_tap + (wp ? wp_bytes : 0u));
            tma_load_5d(dst, &tm_a, c * CK, x0 + kx - 1, y0 - 1, z0 - 1, b, fb);
            tma_load_4d(dst + a_bytes, &tm_b, c * CK, 0, kx, b, fb);
            if (wp) tma_load_4d(dst + a_bytes + 9 * b_tap, &tm_p, c * CK, 0, 0, b, fb);
          }
        }
      }
      // the last loads issued into each stage have landed before the CTA may exit
      for (int q = 0; q < nst && q < k; ++q) {
        const int last = k - 1 - ((k - 1 - q) % nst + nst) % nst;  // last k with k % nst == q
        if (!mbar_wait(smem_u32(&full_bar[q]), (last / nst) & 1)) atomicOr(g.err, kErrProducer);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = instr_desc(N), idesc_p = instr_desc(Np > 0 ? Np : 16);
      const uint32_t idesc3 = instr_desc(pack ? 3 * N : N);
      int k = 0;
      bool good = true;
      for (int i = 0; i < ntile && good; ++i) {
        const int buf = i & 1;
        // packed: the epilogue zeroed both buffers once at the start (phase 0 of tempty)
        const bool wait_buf = pack || i >= 2;
        const uint32_t par = pack ? (uint32_t)((i >> 1) & 1) : (uint32_t)(((i >> 1) - 1) & 1);
        if (wait_buf && !mbar_wait(smem_u32(&tempty[buf]), par)) {
          atomicOr(g.err, kErrMma);
          break;
        }
        tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(buf * acc_cols);
        for (int j = 0; j < ksteps; ++j, ++k) {
          const int st = k % nst;
          if (!mbar_wait(smem_u32(&full_bar[st]), (k / nst) & 1)) {
            atomicOr(g.err, kErrMma);
            good = false;
            break;
          }
          tc_fence_after();
          const int kx = j % spc;
          const uint32_t a_addr = smem_u32(smem + (size_t)st * stage_bytes);
          const uint64_t a0 = smem_desc<CK>(a_addr);
          const uint32_t alo = (uint32_t)a0, ahi = (uint32_t)(a0 >> 32);
          if (kx == 3) {  // W_p^T dz_p: slice zz is rows [128 zz, 128 zz + 128) of the box
            const uint64_t b0 = smem_desc<CK>(a_addr + (uint32_t)(128 * TZ) * kRowB);
            const uint32_t blo = (uint32_t)b0, bhi = (uint32_t)(b0 >> 32);
#pragma unroll
            for (int zz = 0; zz < TZ; ++zz)
#pragma unroll
              for (int kk = 0; kk < CK / 16; ++kk)
                mma_lh(dbase + (uint32_t)((pack ? TZ + 1 - zz : zz) * N),
                       alo + (uint32_t)(zz * 16 * (8 * kRowB >> 4) + kk * 2), ahi,
                       blo + (uint32_t)(kk * 2), bhi, idesc);
          } else if (pack) {
            const uint64_t b0 = smem_desc<CK>(a_addr + a_bytes);
            const uint32_t blo = (uint32_t)b0, bhi = (uint32_t)(b0 >> 32);
            const uint32_t bt = b_tap >> 4;
            // input slice s, row offset ky: B = the kz taps 0..2 of (ky, kx), rows [3 ky N,
            // 3 ky N + 3 N); D = the three slices s, s - 1, s - 2 at column (TZ + 1 - s) N
#pragma unroll
            for (int sl = 0; sl < TZ + 2; ++sl)
#pragma unroll
              for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk) {
                  constexpr uint32_t kAtom = 8 * kRowB >> 4;
                  const uint32_t ao = (uint32_t)((sl * 18 + ky) * kAtom + kk * 2);
                  const uint32_t bo = (uint32_t)(3 * ky) * bt + (uint32_t)(kk * 2);
                  mma_lh(dbase + (uint32_t)((TZ + 1 - sl) * N), alo + ao, ahi, blo + bo, bhi,
                         idesc3);
                }
            if (Np > 0 && kx == 1) {  // projection: the centre window (ky = kz = 1) per slice
              const uint64_t p0 = smem_desc<CK>(a_addr + a_bytes + 9 * b_tap);
              const uint32_t plo = (uint32_t)p0, phi = (uint32_t)(p0 >> 32);
#pragma unroll
              for (int zz = 0; zz < TZ; ++zz)
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk) {
                  constexpr uint32_t kAtom = 8 * kRowB >> 4;
                  const uint32_t ao = (uint32_t)(((zz + 1) * 18 + 1) * kAtom + kk * 2);
                  mma_lh(dbase + (uint32_t)(pbase + zz * Np), alo + ao, ahi,
                         plo + (uint32_t)(kk * 2), phi, idesc_p);
                }
            }
          } else {
            const uint64_t b0 = smem_desc<CK>(a_addr + a_bytes);
            const uint32_t blo = (uint32_t)b0, bhi = (uint32_t)(b0 >> 32);
            const uint32_t bt = b_tap >> 4;
            const uint32_t first = j >= spc ? 1u : 0u;  // a later chunk accumulates
            // tap t = kx + 3 q (kz = q / 3, ky = q % 3), slice zz, K step kk: all offsets but
            // the weight tap stride are compile-time constants
#pragma unroll
            for (int q = 0; q < 9; ++q)
#pragma unroll
              for (int zz = 0; zz < TZ; ++zz)
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk) {
                  constexpr uint32_t kAtom = 8 * kRowB >> 4;
                  const uint32_t ao = (uint32_t)(((zz + q / 3) * 18 + (q % 3)) * kAtom + kk * 2);
                  const uint32_t bo = (uint32_t)q * bt + (uint32_t)(kk * 2);
                  const uint32_t d = dbase + (uint32_t)(zz * N);
                  if (q == 0 && kk == 0)
                    mma_lh_p(d, alo + ao, ahi, blo + bo, bhi, idesc, (j > 0) ? 1u : 0u);
                  else
                    mma_lh(d, alo + ao, ahi, blo + bo, bhi, idesc);
                }
            if (Np > 0 && kx == 1) {  // projection: the centre window (q = 4) of each slice
              const uint64_t p0 = smem_desc<CK>(a_addr + a_bytes + 9 * b_tap);
              const uint32_t plo = (uint32_t)p0, phi = (uint32_t)(p0 >> 32);
#pragma unroll
              for (int zz = 0; zz < TZ; ++zz)
#pragma unroll
                for (int kk = 0; kk < CK / 16; ++kk) {
                  constexpr uint32_t kAtom = 8 * kRowB >> 4;
                  const uint32_t ao = (uint32_t)(((zz + 1) * 18 + 1) * kAtom + kk * 2);
                  const uint32_t d = dbase + (uint32_t)(TZ * N + zz * Np);
                  if (kk == 0)
                    mma_lh_p(d, alo + ao, ahi, plo, phi, idesc_p, first);
                  else
                    mma_lh(d, alo + ao, ahi, plo + (uint32_t)(kk * 2), phi, idesc_p);
                }
            }
          }
          mma_commit(smem_u32(&empty_bar[st]));
        }
        if (good) mma_commit(smem_u32(&tfull[buf]));
      }
      mma_commit(smem_u32(&done_bar));  // fires once every issued MMA has completed
    }
  } else {  // epilogue warps: group (warp - 2) / 4, TMEM lane quadrant warp % 4
    const int grp = (warp - 2) >> 2;
    const int No = g.fold ? N / 2 : N;          // output channels
    const uint32_t fo = g.fold ? (uint32_t)No : 0u;  // column offset of the second half
    const int quad = warp & 3;
    const int m = quad * 32 + lane;  // tile row = y * 8 + x
    const int tid = (threadIdx.x - 64) & 127;
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    float* sbias = sbias0 + grp * (3 * No + Np);  // this group's bias, gamma, beta
    float* stg_g = stg + (size_t)grp * g.nbuf * (g.slice_bytes / 4);
    // Before a slice's first write into the staging: the group's earlier stores have finished
    // reading it (the wait sits here, not after each store, so it overlaps the TMEM passes).
    auto stage_free = [&]() {
      if (tid == 0) {
        if (g.nbuf > 1)
          bulk_wait_read<1>();
        else
          bulk_wait_read<0>();
      }
      epi_sync(grp);
    };
    if (pack) {  // both accumulator buffers start at zero (each group its half of the columns)
      for (int c = grp * 16; c < cols; c += 16 * kEpiGroups)
        tmem_zero16(tmem + lanes + (uint32_t)c);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[0]));
      mbar_arrive(smem_u32(&tempty[1]));
    }
    // Per output slice: TMEM -> (+ bias) -> shared staging slice, then one thread of the
    // group stores the slice with TMA (a reduce-add when accumulating); out-of-grid rows are
    // clipped by TMA.  Staging rows are the output map's swizzled layout: a box of w channels
    // (w = 32: 128-byte rows and swizzle; w = 16: 64-byte), its 16-byte chunks permuted by
    // swz_chunk -- conflict-free for eight consecutive rows.  Slices s = part * TZ + zz with
    // s % kEpiGroups == grp are this group's; packed accumulators are zeroed slice by slice
    // after they are read (the spare columns are never read).
    int slice = 0, bias_b = -1;
    // LayerNorm backward: this lane's warp sums of the (dgamma, dbeta) terms over the group's
    // slices of the current tile, one per 16-channel chunk (lane l < 16: dgamma of channel
    // 16 k + l; l >= 16: dbeta of channel 16 k + l - 16)
    float lnacc0 = 0.f, lnacc1 = 0.f, lnacc2 = 0.f, lnacc3 = 0.f;
    for (int i = 0; i < ntile; ++i) {
      const int buf = i & 1;
      const bool ok = epi_all(mbar_wait(smem_u32(&tfull[buf]), (i >> 1) & 1), grp);
      if (!ok) {  // uniform over the group's four warps, so none is left at a named barrier
        if (tid == 0) atomicOr(g.err, kErrEpilogue);
        break;
      }
      tc_fence_after();
      int tile = blockIdx.x + i * gridDim.x;
      const int b = tile / per_b;
      tile %= per_b;
      const int tile_b = tile;  // the tile's index within its problem
      const int x0 = (tile % g.tiles_x) * 8;
      tile /= g.tiles_x;
      const int y0 = (tile % g.tiles_y) * 16;
      const int z0 = (tile / g.tiles_y) * TZ;
      if (b != bias_b) {  // this problem's biases (zero when none), then gamma and beta
        epi_sync(grp);
        for (int c = tid; c < No + Np; c += 128) {
          const float* bb = c < No ? g.bias : g.bias_p;
          const long long bs = c < No ? g.bias_bs : g.biasp_bs;
          sbias[c] = bb ? bb[(long long)b * bs + (c < No ? c : c - No)] : 0.f;
        }
        if (g.ln)
          for (int c = tid; c < 2 * No; c += 128)
            sbias[No + Np + c] = g.gamma[(long long)b * g.gamma_bs + c];
        epi_sync(grp);
        bias_b = b;
      }
      const int nparts = Np > 0 ? 2 : 1;
      for (int sidx = grp; sidx < nparts * TZ; sidx += kEpiGroups) {
        const int part = sidx / TZ, zz = sidx % TZ;
        const int nc = part ? Np : No;
        const int w = nc % 32 == 0 ? 32 : 16;  // channels per stored box
        const float* bsm = sbias + (part ? No : 0);
        const CUtensorMap* om = part ? &tm_outp : &tm_out;
        const bool add = !part && g.accumulate;
        const int col0 =
            buf * acc_cols + (part ? pbase + zz * Np : (pack ? TZ + 1 - zz : zz) * N);
        float* S = stg_g + (g.nbuf > 1 ? slice & 1 : 0) * (g.slice_bytes / 4);
        const bool ln = g.ln && !part;
        if (!ln) {
          stage_free();
          for (int c0 = 0; c0 < nc; c0 += 16) {
            uint32_t r[16];
            tmem_ld16f(tmem + lanes + (uint32_t)(col0 + c0), r, fo);
            float* row = S + (c0 / w) * (128 * w) + m * w;  // box c0 / w, row m
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 bv = *reinterpret_cast<const float4*>(bsm + c0 + j);
              const float4 v = make_float4(__uint_as_float(r[j]) + bv.x,
                                           __uint_as_float(r[j + 1]) + bv.y,
                                           __uint_as_float(r[j + 2]) + bv.z,
                                           __uint_as_float(r[j + 3]) + bv.w);
              const int chunk = ((c0 % w) + j) / 4;
              *reinterpret_cast<float4*>(row + swz_chunk(chunk, m, 4 * w) * 4) = v;
            }
          }
        } else if (g.ln == 2) {
          // LayerNorm backward of voxel m (the order of ln_bwd_kernel): dp and xhat into this
          // thread's rows of the slice's two FP32 areas while the sums of gamma dp and gamma
          // dp xhat run and the warp sums of dp xhat and dp accumulate (lnacc); then dz from
          // the thread's own rows
          const float inv_c = 1.0f / (float)nc;
          const int ox = x0 + (m & 7), oy = y0 + (m >> 3), oz = z0 + zz;
          const bool inside = ox < g.dout.x && oy < g.dout.y && oz < g.dout.z;
          const long long vox = ((long long)oz * g.dout.y + oy) * g.dout.x + ox;
          const long long vo = (long long)b * g.resid_bs + vox * nc;
          const float* gam = sbias + No + Np;
          const float rs = inside ? g.rstd[(long long)b * g.rstd_bs + vox] : 0.f;
          float* DP = S;
          float* XH = S + 128 * nc;
          __nv_bfloat16* YB = reinterpret_cast<__nv_bfloat16*>(S + 256 * nc);
          float s1 = 0.f, s2 = 0.f;
          stage_free();
#pragma unroll 1
          for (int c0 = 0; c0 < nc; c0 += 16) {
            uint32_t r[16];
            tmem_ld16f(tmem + lanes + (uint32_t)(col0 + c0), r, fo);
            float d[16], xh[16], a[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              float4 q = make_float4(0.f, 0.f, 0.f, 0.f), av = q, hv = q;
              if (inside) {
                if (g.resid) q = *reinterpret_cast<const float4*>(g.resid + vo + c0 + j);
                av = *reinterpret_cast<const float4*>(g.aout + vo + c0 + j);
                hv = *reinterpret_cast<const float4*>(g.xh_in + vo + c0 + j);
              }
              d[j] = __uint_as_float(r[j]) + q.x, d[j + 1] = __uint_as_float(r[j + 1]) + q.y;
              d[j + 2] = __uint_as_float(r[j + 2]) + q.z, d[j + 3] = __uint_as_float(r[j + 3]) + q.w;
              a[j] = av.x, a[j + 1] = av.y, a[j + 2] = av.z, a[j + 3] = av.w;
              xh[j] = hv.x, xh[j + 1] = hv.y, xh[j + 2] = hv.z, xh[j + 3] = hv.w;
            }
            float v[32];  // dp xhat (dgamma terms) then dp (dbeta terms) of the 16 channels
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              float dp = inside ? d[u] : 0.f;
              if (g.act) dp = a[u] > 0.f ? dp : kLeakySlope * dp;
              const float gd = dp * gam[c0 + u];
              s1 += gd;
              s2 += gd * xh[u];
              d[u] = dp;
              v[u] = dp * xh[u];
              v[16 + u] = dp;
            }
            // reduce-scatter over the warp: afterwards lane l holds the warp's sum of v[l]
#pragma unroll
            for (int k = 16; k >= 1; k >>= 1) {
              const bool up = (lane & k) != 0;
#pragma unroll
              for (int i = 0; i < k; ++i) {
                const float give = up ? v[i] : v[i + k];
                const float keep = up ? v[i + k] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, give, k);
              }
            }
            switch (c0 >> 4) {  // (named registers: the chunk loop is not unrolled)
              case 0: lnacc0 += v[0]; break;
              case 1: lnacc1 += v[0]; break;
              case 2: lnacc2 += v[0]; break;
              default: lnacc3 += v[0]; break;
            }
            float* drow = DP + (c0 / w) * (128 * w) + m * w;
            float* hrow = XH + (c0 / w) * (128 * w) + m * w;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const int ch = swz_chunk(((c0 % w) + j) / 4, m, 4 * w);
              *reinterpret_cast<float4*>(drow + ch * 4) = make_float4(d[j], d[j + 1], d[j + 2], d[j + 3]);
              *reinterpret_cast<float4*>(hrow + ch * 4) =
                  make_float4(xh[j], xh[j + 1], xh[j + 2], xh[j + 3]);
            }
          }
          const float m1 = s1 * inv_c, m2 = s2 * inv_c;
#pragma unroll 1
          for (int c0 = 0; c0 < nc; c0 += 16) {
            float* drow = DP + (c0 / w) * (128 * w) + m * w;
            const float* hrow = XH + (c0 / w) * (128 * w) + m * w;
            float o[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const int ch = swz_chunk(((c0 % w) + j) / 4, m, 4 * w);
              const float4 dd = *reinterpret_cast<const float4*>(drow + ch * 4);
              const float4 xx = *reinterpret_cast<const float4*>(hrow + ch * 4);
              o[j] = rs * (dd.x * gam[c0 + j] - m1 - xx.x * m2);
              o[j + 1] = rs * (dd.y * gam[c0 + j + 1] - m1 - xx.y * m2);
              o[j + 2] = rs * (dd.z * gam[c0 + j + 2] - m1 - xx.z * m2);
              o[j + 3] = rs * (dd.w * gam[c0 + j + 3] - m1 - xx.w * m2);
              *reinterpret_cast<float4*>(drow + ch * 4) =
                  make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);  // FP32 dz, own row
            }
            if (g.ybf) stage_slice_bf16(YB, m, nc, c0, o, g.sp);
          }
        } else {
          // LayerNorm of voxel m over its N channels: three passes over TMEM (mean, the
          // centred second moment, then the outputs), in the order of ln_fwd_kernel
          const float inv_c = 1.0f / (float)nc;
          const int ox = x0 + (m & 7), oy = y0 + (m >> 3), oz = z0 + zz;
          const bool inside = ox < g.dout.x && oy < g.dout.y && oz < g.dout.z;
          const long long vox = ((long long)oz * g.dout.y + oy) * g.dout.x + ox;
          const float* rsd =
              g.resid && inside ? g.resid + (long long)b * g.resid_bs + vox * nc : nullptr;
          float sum = 0.f;
          for (int c0 = 0; c0 < nc; c0 += 16) {
            uint32_t r[16];
            tmem_ld16f(tmem + lanes + (uint32_t)(col0 + c0), r, fo);
#pragma unroll
            for (int j = 0; j < 16; ++j) sum += __uint_as_float(r[j]) + bsm[c0 + j];
          }
          const float mean = sum * inv_c;
          float sq = 0.f;
          for (int c0 = 0; c0 < nc; c0 += 16) {
            uint32_t r[16];
            tmem_ld16f(tmem + lanes + (uint32_t)(col0 + c0), r, fo);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float d = __uint_as_float(r[j]) + bsm[c0 + j] - mean;
              sq += d * d;
            }
          }
          const float rs = 1.0f / sqrtf(sq * inv_c + kLnEps);
          const float* gam = sbias + No + Np;
          stage_free();
          float* XH = S + 128 * nc;                                       // xhat boxes
          __nv_bfloat16* YB = reinterpret_cast<__nv_bfloat16*>(S + 256 * nc);  // BF16 copy
          for (int c0 = 0; c0 < nc; c0 += 16) {
            uint32_t r[16];
            tmem_ld16f(tmem + lanes + (uint32_t)(col0 + c0), r, fo);
            float o[16], xh[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              xh[j] = (__uint_as_float(r[j]) + bsm[c0 + j] - mean) * rs;
              o[j] = fmaf(xh[j], gam[c0 + j], gam[nc + c0 + j]);
            }
            if (rsd) {
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                const float4 q = *reinterpret_cast<const float4*>(rsd + c0 + j);
                o[j] += q.x, o[j + 1] += q.y, o[j + 2] += q.z, o[j + 3] += q.w;
              }
            }
            if (g.act) {
#pragma unroll
              for (int j = 0; j < 16; ++j) o[j] = o[j] > 0.f ? o[j] : kLeakySlope * o[j];
            }
            const int bx = c0 / w;
            float* yrow = S + bx * (128 * w) + m * w;
            float* hrow = XH + bx * (128 * w) + m * w;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const int ch = swz_chunk(((c0 % w) + j) / 4, m, 4 * w);
              *reinterpret_cast<float4*>(yrow + ch * 4) =
                  make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
              *reinterpret_cast<float4*>(hrow + ch * 4) =
                  make_float4(xh[j], xh[j + 1], xh[j + 2], xh[j + 3]);
            }
            if (g.ybf) stage_slice_bf16(YB, m, nc, c0, o, g.sp);
          }
          if (inside) g.rstd[(long long)b * g.rstd_bs + vox] = rs;
        }
        if (pack) {  // zeroed after reading: every MMA of the next tile accumulates
          for (int c0 = 0; c0 < (g.fold ? N : nc); c0 += 16)
            tmem_zero16(tmem + lanes + (uint32_t)(col0 + c0));
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        if (sidx + kEpiGroups >= nparts * TZ) {  // the group's last slice of this buffer
          tc_fence_before();
          mbar_arrive(smem_u32(&tempty[buf]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staging -> TMA
        epi_sync(grp);
        if (tid == 0) {
          if (z0 + zz < g.dout.z) {
            if (!(ln && g.ln == 2) || g.out)  // the backward's FP32 dz only when asked for
              for (int k = 0; k < nc / w; ++k) {
                const bool second = !part && g.split_c > 0 && k * w >= g.split_c;
                tma_store_5d(second ? &tm_outp : om, smem_u32(S + k * (128 * w)),
                             second ? k * w - g.split_c : k * w, x0, y0, z0 + zz, b, add);
              }
            if (ln) {
              if (g.ln == 1)
                for (int k = 0; k < nc / w; ++k)
                  tma_store_5d(&tm_xh, smem_u32(S + 128 * nc + k * (128 * w)), k * w, x0, y0,
                               z0 + zz, b, false);
              if (g.ybf)
                for (int k = 0; k < g.sp; ++k)
                  tma_store_5d(&tm_ybf, smem_u32(S + 256 * nc) + (uint32_t)(k * 128 * nc * 2),
                               k * nc, x0, y0, z0 + zz, b, false);
            }
          }
          bulk_commit();  // (read back before the group next writes this slice: stage_free)
        }
        ++slice;
      }
      if (grp >= nparts * TZ) {  // a group without a slice of this tile still hands it back
        tc_fence_before();
        mbar_arrive(smem_u32(&tempty[buf]));
      }
      if (g.ln == 2) {  // the group's row of this tile: the four warps' sums in order
        float* W = stg_g;
        const int nk = N / 16;
        stage_free();
        const float acc4[4] = {lnacc0, lnacc1, lnacc2, lnacc3};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < nk) W[(quad * 4 + k) * 32 + lane] = acc4[k];
        epi_sync(grp);
        if (tid < 2 * N) {
          const int cc = tid < N ? tid : tid - N;
          const int k = cc / 16, l = (tid < N ? 0 : 16) + cc % 16;
          float acc = 0.f;
          for (int q = 0; q < 4; ++q) acc += W[(q * 4 + k) * 32 + l];
          g.part[((long long)b * g.rows_b + (long long)tile_b * kEpiGroups + grp) *
                     (2 * N) + tid] = acc;
        }
        epi_sync(grp);
        lnacc0 = lnacc1 = lnacc2 = lnacc3 = 0.f;
      }
    }
    if (tid == 0) bulk_wait_all();  // every store has landed before the CTA may exit
  }
  __syncwarp();
  // TMEM is freed only after the MMA thread's last commit showed every issued MMA complete;
  // otherwise the error word is set and the columns stay allocated
  bool fin = true;
  if (warp == 1) {
    fin = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
    if (!fin && lane == 0) atomicOr(g.err, kErrEpilogue);
  }
  tc_fence_before();
  const int drained = __syncthreads_and(fin ? 1 : 0);
  if (warp == 1 && drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// weight gradient on the tensor cores (stride-1 layers)
//
// With u = v + offset(t), dW[co][t][ci] = sum_u dy[u - offset(t)][co] x[u][ci]: the tap
// shift moves to dy, whose out-of-grid values are zero (TMA fill), exactly like x's padding.
// One CTA: M = 128 rows = TG taps x Co (TG = 128 / Co), N = Ci, K = the voxels of a chunk of
// 8 x 4 x 4 tiles.  Per K tile: TG shifted dy boxes and the unshifted x box, both
// channels-last, which the MMA reads as MN-major operands (channels contiguous in 16/32/64-
// channel swizzle atoms, voxels along K in 8-row groups).  The epilogue writes each CTA's
// partial sums; a fixed-order sum over chunks follows.
// ------------------------------------------------------------------------------------
constexpr int kWgMaxStages = 4;

// MN-major descriptor: MN-blocks of CK elements (CK*2 bytes, the swizzle width) at LBO,
// 8-row K groups at SBO = 8 * CK * 2.
template <int CK>
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr, uint32_t lbo) {
  constexpr uint64_t kSwizzle = CK == 16 ? 6 : (CK == 32 ? 4 : 2);
  constexpr uint64_t kSbo = 8ull * CK * 2;
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (kSbo >> 4) << 32;
  d |= 1ull << 46;
  d |= kSwizzle << 61;
  return d;
}

// D FP32, A and B BF16, both MN-major, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc_mn(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

template <int CKA, int CKB>
__global__ void __launch_bounds__(128, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tm_dy, const __grid_constant__ CUtensorMap tm_x,
                float* __restrict__ part, Dims3 d, int Co, int Ci, int K, int tg,
                int tiles_per_chunk, int ntiles, int tiles_x, int tiles_y, int rows_b, int nst,
                int bias_on, int* __restrict__ err) {
  constexpr int KT = kBM;                       // voxels per K tile (8 x 4 x 4 box)
  const int ablocks = Co / CKA;                 // A boxes per tap
  const uint32_t a_box = KT * CKA * 2;          // bytes of one A box
  const uint32_t a_bytes = (uint32_t)kBM * KT * 2;  // the whole 128-row A tile
  const uint32_t b_box = KT * CKB * 2;
  const uint32_t b_bytes = (uint32_t)Ci * KT * 2;         // loaded by TMA
  const uint32_t stage_bytes = a_bytes + b_bytes + b_box;  // + one block of ones
  const int n_mma = Ci + CKB;  // the ones block makes column Ci the bias partial
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kWgMaxStages], empty_bar[kWgMaxStages], done_bar;
  __shared__ uint32_t tmem_base_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int chunk = blockIdx.x, grp = blockIdx.y, b = blockIdx.z;
  const int T = K * K * K, pad = (K - 1) / 2, centre = T / 2;
  const int t0 = grp * tg;
  const int ntap = T - t0 < tg ? T - t0 : tg;
  const int tile0 = chunk * tiles_per_chunk;
  const int tile1 = tile0 + tiles_per_chunk < ntiles ? tile0 + tiles_per_chunk : ntiles;
  const int ksteps = tile1 - tile0;
  const uint32_t tmem_cols = n_mma <= 32 ? 32u : n_mma <= 64 ? 64u : n_mma <= 128 ? 128u : 256u;
  const uint32_t tx_bytes = (uint32_t)ntap * ablocks * a_box + b_bytes;
  // the ones block of every stage (BF16 1.0 = 0x3F80); any swizzle of ones is ones
  for (int s = 0; s < nst; ++s) {
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + (size_t)s * stage_bytes + a_bytes + b_bytes);
    for (int i = threadIdx.x; i < (int)(b_box / 4); i += blockDim.x) ones[i] = 0x3F803F80u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {  // TMA producer
    int k = 0;
    for (; k < ksteps; ++k) {
      const int s = k % nst, round = k / nst;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (round - 1) & 1)) {
        atomicOr(err, kErrProducer);
        break;
      }
      const int tile = tile0 + k;
      const int x0 = (tile % tiles_x) * kBX, y0 = ((tile / tiles_x) % tiles_y) * kBY,
                z0 = (tile / (tiles_x * tiles_y)) * kBZ;
      const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, tx_bytes);
      for (int q = 0; q < ntap; ++q) {
        const int t = t0 + q, kz = t / (K * K), ky = (t / K) % K, kx = t % K;
        for (int a = 0; a < ablocks; ++a)
          tma_load_5d(base + (uint32_t)(q * ablocks + a) * a_box, &tm_dy, a * CKA,
                      x0 - (kx - pad), y0 - (ky - pad), z0 - (kz - pad), b, fb);
      }
      for (int c = 0; c < Ci / CKB; ++c)
        tma_load_5d(base + a_bytes + (uint32_t)c * b_box, &tm_x, c * CKB, x0, y0, z0, b, fb);
    }
    drain_loads(full_bar, nst, k, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc_mn(n_mma);
    for (int k = 0; k < ksteps; ++k) {
      const int s = k % nst;
      if (!mbar_wait(smem_u32(&full_bar[s]), (k / nst) & 1)) {
        atomicOr(err, kErrMma);
        break;
      }
      tc_fence_after();
      const uint32_t a_addr = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t b_addr = a_addr + a_bytes;
#pragma unroll
      for (int kk = 0; kk < KT / 16; ++kk)  // K = 16 voxels = two 8-row groups per MMA
        mma_bf16(tmem, smem_desc_mn<CKA>(a_addr + kk * 2 * 8 * CKA * 2, a_box),
                 smem_desc_mn<CKB>(b_addr + kk * 2 * 8 * CKB * 2, b_box), idesc,
                 (k > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&done_bar));
  }
  __syncwarp();

  const bool drained = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
  const bool ok = drained && ksteps > 0;
  if (!drained && lane == 0) atomicOr(err, kErrEpilogue);
  tc_fence_after();
  const int m = warp * 32 + lane;       // TMEM lane = A row = (tap in group, co)
  const int q = m / Co, co = m % Co;
  const int t = t0 + q;
  const long long row = (long long)Co * T * Ci + Co;
  float* prow = part + ((long long)b * rows_b + chunk) * row;
  float* out = prow + ((long long)co * T + t) * Ci;
  for (int c0 = 0; c0 < Ci; c0 += 16) {
    uint32_t r[16];
    if (ok) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    if (q < ntap) {
#pragma unroll
      for (int j = 0; j < 16; ++j) out[c0 + j] = ok ? __uint_as_float(r[j]) : 0.f;
    }
  }
  {  // column Ci: sum of the row's dy over the chunk; the centre tap's is the bias partial
    uint32_t r[16];
    if (ok) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)Ci, r);
    if (q < ntap && t == centre)
      prow[(long long)Co * T * Ci + co] = ok && bias_on ? __uint_as_float(r[0]) : 0.f;
  }
  tc_fence_before();
  // TMEM is freed only once the last commit showed every issued MMA complete
  const int all_drained = __syncthreads_and(drained ? 1 : 0);
  if (warp == 1 && all_drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// Weight gradient of a 3x3x3 stride-2 layer.  dW[co][t][ci] = sum_v x[2 v + k_t - 1][ci]
// dy[v][co]: M = TG taps x Ci (one M block per tap: the input box of an 8 x 4 x 4 output tile
// traversed with element stride 2, i.e. the forward's own strided map), N = Co (the dy tile),
// K = output voxels.  The group that holds the last taps also gets a block of ones in A, whose
// rows give sum_v dy[v][co] (the bias partial).  A CTA takes one tap group and a chunk of
// tiles; per-chunk partial rows follow the layout [co][t][ci], then the bias.
// ------------------------------------------------------------------------------------
template <int CKA, int CKB>
__global__ void __launch_bounds__(128, 1)
wgrad_s2_tc_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_dy,
                   float* __restrict__ part, Dims3 dout, int Co, int tiles_per_chunk, int ntiles,
                   int tiles_x, int tiles_y, int rows_b, int nst, int bias_on,
                   int* __restrict__ err) {
  constexpr int kTpm = 128 / CKA;               // M blocks (taps) per MMA
  constexpr uint32_t a_box = kBM * CKA * 2;     // one tap's box: 128 voxels x Ci
  constexpr uint32_t a_bytes = kTpm * a_box;    // the whole 128-row A tile
  const uint32_t b_box = kBM * CKB * 2;
  const uint32_t stage_bytes = a_bytes + (uint32_t)(Co / CKB) * b_box;
  const int Ci = CKA;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kWgMaxStages], empty_bar[kWgMaxStages], done_bar;
  __shared__ uint32_t tmem_base_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int chunk = blockIdx.x, grp = blockIdx.y, b = blockIdx.z;
  const int t0 = grp * kTpm;
  const int ntap = 27 - t0 < kTpm ? 27 - t0 : kTpm;  // taps of this group
  const bool ones = ntap < kTpm;                     // block ntap holds ones
  const int tile0 = chunk * tiles_per_chunk;
  const int tile1 = tile0 + tiles_per_chunk < ntiles ? tile0 + tiles_per_chunk : ntiles;
  const int ksteps = tile1 > tile0 ? tile1 - tile0 : 0;
  const uint32_t tmem_cols = Co <= 32 ? 32u : Co <= 64 ? 64u : Co <= 128 ? 128u : 256u;
  if (ones) {  // the ones block of every stage (BF16 1.0); rows past it stay unused
    for (int s = 0; s < nst; ++s) {
      uint32_t* o = reinterpret_cast<uint32_t*>(smem + (size_t)s * stage_bytes + ntap * a_box);
      for (int i = threadIdx.x; i < (int)(a_box / 4); i += blockDim.x) o[i] = 0x3F803F80u;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {  // TMA producer
    const uint32_t tx_bytes = (uint32_t)ntap * a_box + (uint32_t)(Co / CKB) * b_box;
    int k = 0;
    for (; k < ksteps; ++k) {
      const int s = k % nst, round = k / nst;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (round - 1) & 1)) {
        atomicOr(err, kErrProducer);
        break;
      }
      const int tile = tile0 + k;
      const int x0 = (tile % tiles_x) * kBX, y0 = ((tile / tiles_x) % tiles_y) * kBY,
                z0 = (tile / (tiles_x * tiles_y)) * kBZ;
      const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, tx_bytes);
      for (int q = 0; q < ntap; ++q) {
        const int t = t0 + q, kz = t / 9, ky = (t / 3) % 3, kx = t % 3;
        tma_load_5d(base + (uint32_t)q * a_box, &tm_x, 0, 2 * x0 + kx - 1, 2 * y0 + ky - 1,
                    2 * z0 + kz - 1, b, fb);
      }
      for (int c = 0; c < Co / CKB; ++c)
        tma_load_5d(base + a_bytes + (uint32_t)c * b_box, &tm_dy, c * CKB, x0, y0, z0, b, fb);
    }
    drain_loads(full_bar, nst, k, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc_mn(Co);
    for (int k = 0; k < ksteps; ++k) {
      const int s = k % nst;
      if (!mbar_wait(smem_u32(&full_bar[s]), (k / nst) & 1)) {
        atomicOr(err, kErrMma);
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
      const uint64_t a0 = smem_desc_mn<CKA>(base, a_box);
      const uint64_t b0 = smem_desc_mn<CKB>(base + a_bytes, b_box);
      const uint32_t alo = (uint32_t)a0, ahi = (uint32_t)(a0 >> 32);
      const uint32_t blo = (uint32_t)b0, bhi = (uint32_t)(b0 >> 32);
      mma_lh_p(tmem, alo, ahi, blo, bhi, idesc, k > 0 ? 1u : 0u);
#pragma unroll
      for (int kk = 1; kk < kBM / 16; ++kk)  // K = 16 voxels = two 8-row groups per MMA
        mma_lh(tmem, alo + (uint32_t)((kk * 2 * 8 * CKA * 2) >> 4), ahi,
               blo + (uint32_t)((kk * 2 * 8 * CKB * 2) >> 4), bhi, idesc);
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&done_bar));
  }
  __syncwarp();

  const bool drained = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
  const bool ok = drained && ksteps > 0;
  if (!drained && lane == 0) atomicOr(err, kErrEpilogue);
  tc_fence_after();
  const int m = warp * 32 + lane;  // TMEM lane = A row = (tap in group, ci)
  const int q = m / Ci, ci = m % Ci;
  const int t = t0 + q;
  const long long row = (long long)Co * 27 * Ci + Co;
  float* prow = part + ((long long)b * rows_b + chunk) * row;
  for (int c0 = 0; c0 < Co; c0 += 16) {
    uint32_t r[16];
    if (ok) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    if (q < ntap) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        prow[((long long)(c0 + j) * 27 + t) * Ci + ci] = ok ? __uint_as_float(r[j]) : 0.f;
    } else if (ones && q == ntap && ci == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        prow[(long long)Co * 27 * Ci + c0 + j] = ok && bias_on ? __uint_as_float(r[j]) : 0.f;
    }
  }
  tc_fence_before();
  // TMEM is freed only once the last commit showed every issued MMA complete
  const int all_drained = __syncthreads_and(drained ? 1 : 0);
  if (warp == 1 && all_drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// Weight gradient of a 3x3x3 stride-1 layer with halo boxes.  K tile = one column of
// 8 x 1 x TZ input voxels u (rows g * 8 + x, g = z offset).  With dy shifted by the tap,
// dW[co][t][ci] = sum_u dy[u + 1 - k_t][co] x[u][ci]; for one x tap kx the dy values of all
// nine (ky, kz) taps lie in one TMA box of 8 x 3 x (TZ + 2) voxels.  Stored [z][y][x], the
// window of tap (ky, kz) starts p = 8 - 3 kz - ky swizzle atoms (8 rows) into the box and
// steps 3 atoms per z, so an M block of one tap's Co channels is an MN-major operand with
// block stride = 1 atom and 8-row K-group stride = 3 atoms.  One MMA (M = 128) covers
// TPM = 128 / Co consecutive windows; G = ceil(9 / TPM) MMAs per x tap (the last one
// overlaps its predecessor and only its new rows are kept).  B = the unshifted x column
// plus a block of ones, whose column gives sum(dy) per window: the centre tap's is the bias
// partial.  A CTA adds the products of a run of tiles for NKX x taps (all three when the
// accumulators fit in TMEM, else one per grid row) and writes one partial-sum row.
// NKX = 0, the packed form: the x tap moves to the x operand instead, dW[co][t][ci] =
// sum_v dy[v + (0, 1 - ky, 1 - kz)][co] x[v + (kx - 1, 0, 0)][ci], so one unshifted dy box
// serves all 27 taps and B holds the three x-shifted columns side by side plus the ones:
// N = 3 Ci + CKB, the columns of x tap kx at kx * Ci.  Per 16-voxel K step that is G MMAs of
// width N instead of 3 G of width Ci + CKB, at nearly the same issue cost per MMA.
// fold (packed, split precision, a 16 -> 16 layer in one pass): dy and x are read as their
// [hi | lo] 32-channel rows, so M = windows x [co_hi | co_lo] and N = x taps x [ci_hi | ci_lo]
// (+ ones); the template sees Co = Ci = 32 and the epilogue adds the four products of each
// weight (lanes co and co + 16 through a shuffle, columns ci and ci + 16), the whole
// (dy_hi + dy_lo)(x_hi + x_lo).
// NX = 2 (packed, split precision): the hi and lo blocks of x (tm_x, tm_x2) side by side,
// N = 6 Ci + CKB, and the epilogue adds the two products of each tap: dy_hi x_hi + dy_hi x_lo
// in one MMA stream (the pass with dy_lo x_hi is a separate NX = 1 launch).
// ones_sep (the per-x-tap forms whose accumulators of Ci + CKB columns do not fit in tensor
// memory, e.g. 64 -> 64 layers): B is the x column alone (N = Ci, one CKB-wide block per
// channel chunk, no partial swizzle atom) and the centre x tap's CTA adds one MMA of N = 16
// per K step, the M block holding window 4 (tap 13) against a K-major block of ones, into a
// 16-column accumulator of its own (one more for a fused projection's dz_p).
// ------------------------------------------------------------------------------------
constexpr int kWg3MaxStages = 6;


struct Wg3Geom {
  int tz, nkx, tiles_x, tiles_z, ntiles, tiles_per_chunk, nchunks, nst;
  int rows_b;      // partial-sum rows per problem (nchunks times the operand passes)
  int nx;          // x operand sets side by side in N (2: hi and lo of the split precision)
  int bias_on;     // write the ones column's sums (else zeros: a pass that repeats them)
  int fold;        // split precision in one pass (below)
  int ones_sep;    // per-x-tap form: the ones column as separate N = 16 MMAs (below)
  uint32_t a_box, b_box, b_off, ones_off, stage, tmem_cols;
  int proj;        // also the weight gradient of a fused 1x1 projection (its dz_p: p_box)
  uint32_t p_off, p_box;
};

template <int CKA, int CKB, int NKX, int NX = 1>
__global__ void __launch_bounds__(128, 1)
wgrad_tc3_kernel(const __grid_constant__ CUtensorMap tm_dy, const __grid_constant__ CUtensorMap tm_x,
                 const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_x2,
                 float* __restrict__ part,
                 float* __restrict__ part_p, Dims3 d, int Ci, int ci_out,
                 const __grid_constant__ Wg3Geom gm, int* __restrict__ err) {
  constexpr int kTpm = 128 / CKA;                  // taps per MMA
  constexpr int kG = (9 + kTpm - 1) / kTpm;        // MMAs per x tap
  constexpr uint32_t kAtomA = 8 * CKA * 2;         // 8 rows of dy
  constexpr uint32_t kAtomB = 8 * CKB * 2;
  constexpr bool kPack = NKX == 0;                 // the three x taps in N
  constexpr int kNq = kPack ? 1 : NKX;             // dy boxes (accumulator sets) per stage
  static_assert(NX == 1 || kPack, "two x operand sets only in the packed form");
  const int N = (kPack ? 3 * NX * Ci : Ci) + (gm.ones_sep ? 0 : CKB);  // + the ones block
  const int nb = Ci / CKB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kWg3MaxStages], empty_bar[kWg3MaxStages], done_bar;
  __shared__ uint32_t tmem_base_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int chunk = blockIdx.x, kx0 = blockIdx.y * kNq, b = blockIdx.z;
  const int tile0 = chunk * gm.tiles_per_chunk;
  const int tile1 = min(tile0 + gm.tiles_per_chunk, gm.ntiles);
  const int ksteps = max(tile1 - tile0, 0);
  const int nst = gm.nst;
  // the projection's products go with the centre x tap: D_p[co][ci] = sum_u dz_p[u][co] x[u][ci]
  const bool proj = gm.proj && (kPack || (kx0 <= 1 && 1 < kx0 + NKX));
  const uint32_t pcol = (uint32_t)(kNq * kG * N);  // its accumulator
  // ones_sep: the accumulators of the window-4 block's and the projection's ones columns
  constexpr int kGc = 4 / kTpm;                    // the M block holding window 4
  const uint32_t ocol = pcol + (gm.proj ? (uint32_t)N : 0u);
  const int qc = 1 - kx0;                          // the centre x tap's accumulator set
  const bool ones_mma = gm.ones_sep && !kPack && qc >= 0 && qc < kNq;
  for (int s = 0; s < nst; ++s) {
    uint32_t* ones = reinterpret_cast<uint32_t*>(smem + (size_t)s * gm.stage + gm.ones_off);
    for (int i = threadIdx.x; i < (int)(gm.b_box / 4); i += blockDim.x) ones[i] = 0x3F803F80u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"(gm.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {  // TMA producer
    const uint32_t tx_bytes = (uint32_t)kNq * gm.a_box +
                              (uint32_t)(kPack ? 3 * NX * nb : nb) * gm.b_box +
                              (proj ? gm.p_box : 0u);
    int k = 0;
    for (; k < ksteps; ++k) {
      const int s = k % nst, round = k / nst;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (round - 1) & 1)) {
        atomicOr(err, kErrProducer);
        break;
      }
      const int tile = tile0 + k;
      const int x0 = (tile % gm.tiles_x) * 8;
      const int y0 = (tile / gm.tiles_x) % d.y;
      const int z0 = (tile / (gm.tiles_x * d.y)) * gm.tz;
      const uint32_t base = smem_u32(smem + (size_t)s * gm.stage);
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, tx_bytes);
      if (kPack) {  // the unshifted dy box, then x at x offsets -1, 0, +1
        tma_load_5d(base, &tm_dy, 0, x0, y0 - 1, z0 - 1, b, fb);
        for (int xs = 0; xs < NX; ++xs)
          for (int kx = 0; kx < 3; ++kx)
            for (int c = 0; c < nb; ++c)
              tma_load_5d(base + gm.b_off + (uint32_t)((xs * 3 + kx) * nb + c) * gm.b_box,
                          xs ? &tm_x2 : &tm_x, c * CKB, x0 + kx - 1, y0, z0, b, fb);
      } else {
        for (int q = 0; q < NKX; ++q)
          tma_load_5d(base + (uint32_t)q * gm.a_box, &tm_dy, 0, x0 + 1 - (kx0 + q), y0 - 1,
                      z0 - 1, b, fb);
        for (int c = 0; c < nb; ++c)
          tma_load_5d(base + gm.b_off + (uint32_t)c * gm.b_box, &tm_x, c * CKB, x0, y0, z0, b, fb);
      }
      if (proj) tma_load_5d(base + gm.p_off, &tm_p, 0, x0, y0, z0, b, fb);
    }
    drain_loads(full_bar, nst, k, err);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = instr_desc_mn(N);
    const uint32_t idesc_o = instr_desc_major(16, true, false);  // A MN-major, ones K-major
    for (int k = 0; k < ksteps; ++k) {
      const int s = k % nst;
      if (!mbar_wait(smem_u32(&full_bar[s]), (k / nst) & 1)) {
        atomicOr(err, kErrMma);
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + (size_t)s * gm.stage);
      // the ones block read K-major (16 rows of 32 bytes, 32-byte swizzle: ones either way)
      const uint64_t o0 = smem_desc<16>(base + gm.ones_off);
      const uint32_t olo = (uint32_t)o0, ohi = (uint32_t)(o0 >> 32);
      // descriptors are linear in the address (start >> 4 in the low word): offset a base
      const uint64_t a0 = smem_desc_mn2<CKA>(base, kAtomA, 3 * kAtomA);
      const uint64_t b0 = smem_desc_mn2<CKB>(base + gm.b_off, gm.b_box, kAtomB);
      const uint32_t ahi = (uint32_t)(a0 >> 32), bhi = (uint32_t)(b0 >> 32);
      const uint32_t abx = gm.a_box >> 4;
      uint32_t alo = (uint32_t)a0, blo = (uint32_t)b0;
      // dz_p column: every M block reads the same Co rows (block stride 0), K groups adjacent
      const uint64_t p0 = smem_desc_mn2<CKA>(base + gm.p_off, 0, kAtomA);
      uint32_t plo = (uint32_t)p0;
      const uint32_t phi = (uint32_t)(p0 >> 32);
      for (int kk = 0; kk < gm.tz / 2; ++kk) {  // K = 16 voxels = z offsets 2kk, 2kk + 1
#pragma unroll
        for (int q = 0; q < kNq; ++q)
#pragma unroll
          for (int g = 0; g < kG; ++g) {
            constexpr int kLast = 9 - kTpm;
            const int s0 = g * kTpm < kLast ? g * kTpm : kLast;
            const uint32_t ao = (uint32_t)q * abx + (uint32_t)((s0 * kAtomA) >> 4);
            const uint32_t d = tmem + (uint32_t)((q * kG + g) * N);
            if (kk == 0)
              mma_lh_p(d, alo + ao, ahi, blo, bhi, idesc, k > 0 ? 1u : 0u);
            else
              mma_lh(d, alo + ao, ahi, blo, bhi, idesc);
          }
        if (proj) {
          if (kk == 0)
            mma_lh_p(tmem + pcol, plo, phi, blo, bhi, idesc, k > 0 ? 1u : 0u);
          else
            mma_lh(tmem + pcol, plo, phi, blo, bhi, idesc);
        }
        if (ones_mma) {  // sum(dy) of the window-4 block (and of dz_p): B = 16 x 16 ones
          const uint32_t ao = (uint32_t)qc * abx + (uint32_t)((kGc * kTpm * kAtomA) >> 4);
          mma_lh_p(tmem + ocol, alo + ao, ahi, olo, ohi, idesc_o, (k > 0 || kk > 0) ? 1u : 0u);
          if (proj)
            mma_lh_p(tmem + ocol + 16, plo, phi, olo, ohi, idesc_o,
                     (k > 0 || kk > 0) ? 1u : 0u);
        }
        alo += (6 * kAtomA) >> 4;  // next two z offsets: 6 dy atoms, 2 x atoms
        blo += (2 * kAtomB) >> 4;
        plo += (2 * kAtomA) >> 4;
      }
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&done_bar));
  }
  __syncwarp();

  const bool drained = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done_bar), 0));
  const bool ok = drained && ksteps > 0;
  if (!drained && lane == 0) atomicOr(err, kErrEpilogue);
  tc_fence_after();
  const int Co = CKA;
  const int m = warp * 32 + lane;  // TMEM lane = (window in the MMA, co)
  const int pl = m / Co, co = m % Co;
  if (gm.fold) {
    const int Cr = Co / 2;  // the layer's output channels; lanes co, co + Cr: dy_hi, dy_lo
    const int Ch = Ci / 2;  // the layer's input channels; columns c, Ch + c: x_hi, x_lo
    const long long rowf = (long long)Cr * 27 * ci_out + Cr;
    float* prf = part + ((long long)b * gm.rows_b + chunk) * rowf;
    const bool writer = co < Cr;
    for (int q = 0; q < kNq; ++q)
      for (int g = 0; g < kG; ++g) {
        const int s0 = g * kTpm < 9 - kTpm ? g * kTpm : 9 - kTpm;
        const int p = s0 + pl;
        const bool keep = p >= g * kTpm && p < 9;
        const int tq = 8 - p, kz = tq / 3, ky = tq % 3;
        const uint32_t col =
            tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((q * kG + g) * N);
        for (int xi = 0; xi < (kPack ? 3 : 1); ++xi) {
          const int kx = kPack ? xi : kx0 + q;
          const int t = kz * 9 + ky * 3 + kx;
          const uint32_t cx = col + (uint32_t)(kPack ? xi * Ci : 0);
          for (int c0 = 0; c0 < Ch; c0 += 16) {
            uint32_t r[16], r2[16];
            if (ok) {
              tmem_ld16(cx + (uint32_t)c0, r);        // x_hi columns
              tmem_ld16(cx + (uint32_t)(Ch + c0), r2);  // x_lo columns
            }
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              v[j] = ok ? __uint_as_float(r[j]) + __uint_as_float(r2[j]) : 0.f;
              v[j] += __shfl_xor_sync(0xffffffffu, v[j], Cr);  // + the other dy block
            }
            if (keep && writer) {
              float* out = prf + ((long long)co * 27 + t) * ci_out + c0;
#pragma unroll
              for (int j = 0; j < 16; j += 4)
                if (c0 + j < ci_out)
                  *reinterpret_cast<float4*>(out + j) =
                      make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
          }
        }
        uint32_t r[16];
        const bool centre = kPack || kx0 + q == 1;
        if (gm.ones_sep) {  // the ones column lives in its own accumulator (window-4 block)
          if (ok && centre && g == kGc)
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + ocol, r);
        } else if (ok) {
          tmem_ld16(col + (uint32_t)(kPack ? 3 * Ci : Ci), r);  // the ones column
        }
        float v0 = ok ? __uint_as_float(r[0]) : 0.f;
        v0 += __shfl_xor_sync(0xffffffffu, v0, Cr);
        if (keep && writer && tq == 4 && centre)
          prf[(long long)Cr * 27 * ci_out + co] = gm.bias_on ? v0 : 0.f;
      }
    if (proj && warp * 32 < Co) {  // the projection: rows [co_hi | co_lo], centre x columns
      const long long prow_n = (long long)Cr * Ch + Cr;
      float* pp = part_p + ((long long)b * gm.rows_b + chunk) * prow_n;
      const uint32_t col = tmem + ((uint32_t)(warp * 32) << 16) + pcol;
      const uint32_t cx = col + (uint32_t)(kPack ? Ci : 0);
      for (int c0 = 0; c0 < Ch; c0 += 16) {
        uint32_t r[16], r2[16];
        if (ok) {
          tmem_ld16(cx + (uint32_t)c0, r);
          tmem_ld16(cx + (uint32_t)(Ch + c0), r2);
        }
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = ok ? __uint_as_float(r[j]) + __uint_as_float(r2[j]) : 0.f;
          v[j] += __shfl_xor_sync(0xffffffffu, v[j], Cr);
        }
        if (writer)
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(pp + (long long)co * Ch + c0 + j) =
                make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
      uint32_t r[16];
      if (ok)
        tmem_ld16(gm.ones_sep ? tmem + ((uint32_t)(warp * 32) << 16) + ocol + 16
                              : col + (uint32_t)(kPack ? 3 * Ci : Ci), r);
      float v0 = ok ? __uint_as_float(r[0]) : 0.f;
      v0 += __shfl_xor_sync(0xffffffffu, v0, Cr);
      if (writer) pp[(long long)Cr * Ch + co] = gm.bias_on ? v0 : 0.f;
    }
  } else {
  const long long row = (long long)Co * 27 * ci_out + Co;  // the first ci_out channels
  float* prow = part + ((long long)b * gm.rows_b + chunk) * row;
  for (int q = 0; q < kNq; ++q)
    for (int g = 0; g < kG; ++g) {
      const int s0 = g * kTpm < 9 - kTpm ? g * kTpm : 9 - kTpm;
      const int p = s0 + pl;                      // window p <-> tap 3 kz + ky = 8 - p
      const bool keep = p >= g * kTpm && p < 9;   // rows new to this MMA
      const int tq = 8 - p, kz = tq / 3, ky = tq % 3;
      const uint32_t col = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((q * kG + g) * N);
      for (int xi = 0; xi < (kPack ? 3 : 1); ++xi) {  // packed: x tap xi at columns xi * Ci
        const int kx = kPack ? xi : kx0 + q;
        const int t = kz * 9 + ky * 3 + kx;
        float* out = prow + ((long long)co * 27 + t) * ci_out;
        const uint32_t cx = col + (uint32_t)(kPack ? xi * Ci : 0);
        for (int c0 = 0; c0 < Ci; c0 += 16) {
          uint32_t r[16];
          if (ok) tmem_ld16(cx + (uint32_t)c0, r);
          if (NX == 2) {  // + the lo-x products of the same tap
            uint32_t r2[16];
            if (ok) tmem_ld16(cx + (uint32_t)(3 * Ci + c0), r2);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r2[j]));
          }
          if (keep) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              if (c0 + j < ci_out)
                *reinterpret_cast<float4*>(out + c0 + j) =
                  ok ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                   __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
      uint32_t r[16];
      const bool centre = kPack || kx0 + q == 1;
      if (gm.ones_sep) {  // the ones column lives in its own accumulator (window-4 block)
        if (ok && centre && g == kGc) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + ocol, r);
      } else if (ok) {
        tmem_ld16(col + (uint32_t)(kPack ? 3 * NX * Ci : Ci), r);  // the ones column
      }
      if (keep && tq == 4 && centre)  // the centre tap (t = 13): the bias
        prow[(long long)Co * 27 * ci_out + co] = ok && gm.bias_on ? __uint_as_float(r[0]) : 0.f;
    }
  if (proj && warp * 32 < Co) {  // rows co < Co of the projection accumulator
    const long long prow_n = (long long)Co * Ci + Co;
    float* pp = part_p + ((long long)b * gm.rows_b + chunk) * prow_n;
    const uint32_t col = tmem + ((uint32_t)(warp * 32) << 16) + pcol;
    const uint32_t cx = col + (uint32_t)(kPack ? Ci : 0);  // packed: the unshifted x columns
    for (int c0 = 0; c0 < Ci; c0 += 16) {
      uint32_t r[16];
      if (ok) tmem_ld16(cx + (uint32_t)c0, r);
      if (m < Co) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(pp + (long long)m * Ci + c0 + j) =
              ok ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                               __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                 : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    uint32_t r[16];
    if (ok)
      tmem_ld16(gm.ones_sep ? tmem + ((uint32_t)(warp * 32) << 16) + ocol + 16
                            : col + (uint32_t)(kPack ? 3 * Ci : Ci), r);
    if (m < Co) pp[(long long)Co * Ci + m] = ok && gm.bias_on ? __uint_as_float(r[0]) : 0.f;
  }
  }  // not fold
  tc_fence_before();
  // TMEM is freed only once the last commit showed every issued MMA complete
  const int all_drained = __syncthreads_and(drained ? 1 : 0);
  if (warp == 1 && all_drained) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(gm.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------------------------
// staging kernels
// ------------------------------------------------------------------------------------
__global__ void f32_to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                   long long n) {
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i + 3 < n) {
    const float4 v = *reinterpret_cast<const float4*>(x + i);
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), c = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<__nv_bfloat162*>(y + i) = a;
    *reinterpret_cast<__nv_bfloat162*>(y + i + 2) = c;
  } else {
    for (long long j = i; j < n; ++j) y[j] = __float2bfloat16_rn(x[j]);
  }
}

// x [v][C] FP32 -> y [v][sp * C] BF16 staging rows (stage_bf16x4); a thread per 4 channels.
__global__ void f32_to_bf16_rows_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                        long long nvox, int C, int sp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = C / 4;
  if (e >= nvox * g) return;
  const long long v = e / g;
  const int c = (int)(e % g) * 4;
  const float4 val = *reinterpret_cast<const float4*>(x + v * C + c);
  stage_bf16x4(y + v * C * sp, C, c, val, sp);
}

// Stored tap index of tap t of a 27-tap layer whose halo form packs kz into N: ky and kz
// swapped, so the kz taps of one (ky, kx) are adjacent in the B box of x tap kx.
// perm 2 (the packed stride-2 data gradient): the data-gradient row of t = 26 - (forward tap
// f) goes to block 8 w + p, the (window w, class p) pair that reads tap f.  Per axis, tap k
// = 1 is read by parity 0 from window 0, k = 2 by parity 1 from window 0, k = 0 by parity 1
// from window 1.
__device__ __forceinline__ int packed_tap(int t, int perm) {
  if (perm == 2) {
    const int f = 26 - t;
    int w = 0, p = 0;
#pragma unroll
    for (int a = 0, s = 1; a < 3; ++a, s *= 3) {
      const int k = (f / s) % 3;
      w |= (k == 0 ? 1 : 0) << a;
      p |= (k != 1 ? 1 : 0) << a;
    }
    return 8 * w + p;
  }
  return perm ? ((t / 3) % 3) * 9 + (t / 9) * 3 + t % 3 : t;
}

// Forward weights [t][co][ci] and data-gradient weights [T-1-t][ci][co] of one layer (tap
// major), for every problem of the batch.
__global__ void weights_bf16_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wb,
                                    long long Pp, long long wstride, long long w_off,
                                    long long wf_off, long long wd_off, int ci, int ci_real,
                                    int co, int T, int dgrad, int permf, int permd) {
  const int b = blockIdx.y;
  const long long n = (long long)co * T * ci;  // padded input channels
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = (int)(e % ci);
  const long long r = e / ci;
  const int t = (int)(r % T), o = (int)(r / T);
  const float v = c < ci_real ? theta[(long long)b * Pp + w_off + r * ci_real + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);  // W[o][t][c]
  __nv_bfloat16* base = wb + (long long)b * wstride;
  base[wf_off + ((long long)packed_tap(t, permf) * co + o) * ci + c] = h;  // [t][co][ci]
  if (dgrad)  // [26-t][ci][co]
    base[wd_off + ((long long)packed_tap(T - 1 - t, permd) * ci + c) * co + o] = h;
}

// All layers' weights in one launch: a block belongs to the layer whose block range holds
// blockIdx.x (ranges from a prefix table of at most kWMaxLayers layers).
constexpr int kWMaxLayers = 48;
struct WTable {
  int nl;
  int blk0[kWMaxLayers + 1];
  long long w_off[kWMaxLayers], wf_off[kWMaxLayers], wd_off[kWMaxLayers];
  int ci[kWMaxLayers], ci_real[kWMaxLayers], co[kWMaxLayers], T[kWMaxLayers],
      dgrad[kWMaxLayers], permf[kWMaxLayers], permd[kWMaxLayers];
  int hlf[kWMaxLayers], hld[kWMaxLayers];  // split rows doubled in N (TcLayer::hlf / hld)
};

// A block takes one (layer, tap, chunk of 32 output channels): it reads W[o][tap][0..ci) rows
// (coalesced, zero past ci_real) into shared memory, writes the forward rows [tap][o][ci]
// and, through the shared tile, the data-gradient rows [T-1-tap][ci][o] (32 o per row piece).
constexpr int kWOc = 32;

__global__ void __launch_bounds__(256)
weights_all_bf16_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wb,
                        long long Pp, long long wstride, const __grid_constant__ WTable t) {
  __shared__ __nv_bfloat16 tile[kWOc][256 + 2];
  int l = 0;
  while (l + 1 < t.nl && (int)blockIdx.x >= t.blk0[l + 1]) ++l;
  const int b = blockIdx.y;
  const int ci = t.ci[l], cr = t.ci_real[l], co = t.co[l], T = t.T[l];
  const int nch = (co + kWOc - 1) / kWOc;  // (blocks of 32 output channels per tap)
  const int q = blockIdx.x - t.blk0[l];
  const int tap = q / nch, o0 = (q % nch) * kWOc;
  const int no = co - o0 < kWOc ? co - o0 : kWOc;
  const float* src = theta + (long long)b * Pp + t.w_off[l];
  __nv_bfloat16* base = wb + (long long)b * wstride;
  for (int e = threadIdx.x; e < no * ci; e += blockDim.x) {
    const int ol = e / ci, c = e % ci;
    const float v = c < cr ? src[((long long)(o0 + ol) * T + tap) * cr + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    tile[ol][c] = h;
    base[t.wf_off[l] + ((long long)packed_tap(tap, t.permf[l]) * co + o0 + ol) * ci + c] =
        h;  // [t][co][ci]
  }
  if (!t.dgrad[l]) return;
  __syncthreads();
  for (int e = threadIdx.x; e < no * ci; e += blockDim.x) {
    const int ol = e % no, c = e / no;
    base[t.wd_off[l] + ((long long)packed_tap(T - 1 - tap, t.permd[l]) * ci + c) * co + o0 +
         ol] = tile[ol][c];
  }
}

// Split weights of every layer (BF16x3): forward rows [t][co][3 ci] = [hi | hi | lo] over ci
// and data-gradient rows [T-1-t][ci][3 co] = [hi | hi | lo] over co, hi = bf16(w),
// lo = bf16(w - hi).  A block takes one (layer, tap, chunk of 32 output channels), as
// weights_all_bf16_kernel: coalesced reads of W[o][tap][0..ci), forward rows written in
// order, the data-gradient rows through shared-memory tiles of hi and lo.
__global__ void __launch_bounds__(256)
weights_split_bf16_kernel(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wb,
                          long long Pp, long long wstride, const __grid_constant__ WTable t) {
  __shared__ __nv_bfloat16 th[kWOc][256 + 2], tl[kWOc][256 + 2];
  int l = 0;
  while (l + 1 < t.nl && (int)blockIdx.x >= t.blk0[l + 1]) ++l;
  const int b = blockIdx.y;
  const int ci = t.ci[l], cr = t.ci_real[l], co = t.co[l], T = t.T[l];
  const int nch = (co + kWOc - 1) / kWOc;
  const int q = blockIdx.x - t.blk0[l];
  const int tap = q / nch, o0 = (q % nch) * kWOc;
  const int no = co - o0 < kWOc ? co - o0 : kWOc;
  const float* src = theta + (long long)b * Pp + t.w_off[l];
  __nv_bfloat16* base = wb + (long long)b * wstride;
  const bool hf = t.hlf[l] != 0, hd = t.hld[l] != 0;
  const long long frow = t.wf_off[l] + (long long)packed_tap(tap, t.permf[l]) * co * (hf ? 4 : 3) * ci;
  for (int e = threadIdx.x; e < no * ci; e += blockDim.x) {
    const int ol = e / ci, c = e % ci;
    const float v = c < cr ? src[((long long)(o0 + ol) * T + tap) * cr + c] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    th[ol][c] = hi;
    tl[ol][c] = lo;
    if (hf) {  // [t][2 co][2 ci]: rows o: [hi | hi], rows co + o: [lo | lo]
      __nv_bfloat16* f = base + frow + (long long)(o0 + ol) * 2 * ci;
      __nv_bfloat16* g = base + frow + (long long)(co + o0 + ol) * 2 * ci;
      f[c] = hi, f[ci + c] = hi, g[c] = lo, g[ci + c] = lo;
    } else {
      __nv_bfloat16* f = base + frow + (long long)(o0 + ol) * 3 * ci;  // [t][co][3 ci]
      f[c] = hi, f[ci + c] = hi, f[2 * ci + c] = lo;
    }
  }
  if (!t.dgrad[l]) return;
  __syncthreads();
  const long long drow =
      t.wd_off[l] + (long long)packed_tap(T - 1 - tap, t.permd[l]) * ci * (hd ? 4 : 3) * co;
  for (int e = threadIdx.x; e < no * ci; e += blockDim.x) {
    const int ol = e % no, c = e / no;
    if (hd) {  // [26-t][2 ci][2 co]: rows c: [hi | hi], rows ci + c: [lo | lo]
      __nv_bfloat16* d = base + drow + (long long)c * 2 * co + o0 + ol;
      __nv_bfloat16* d2 = base + drow + (long long)(ci + c) * 2 * co + o0 + ol;
      d[0] = th[ol][c], d[co] = th[ol][c], d2[0] = tl[ol][c], d2[co] = tl[ol][c];
    } else {
      __nv_bfloat16* d = base + drow + (long long)c * 3 * co + o0 + ol;  // [26-t][ci][3 co]
      d[0] = th[ol][c], d[co] = th[ol][c], d[2 * co] = tl[ol][c];
    }
  }
}

int chunk_for(int c) { return c % 64 == 0 ? 64 : (c % 32 == 0 ? 32 : 16); }

// Split precision, per-tap forward: reading [hi | lo] rows (K = 2 ci) against weights doubled
// in N (2 co) moves fewer, longer TMA rows than [hi | lo | hi] rows (3 ci) wherever it allows
// a wider channel chunk.
bool bf16_fold_pays(const Bf16Net& bf, int ci, int co) {
  return bf.sp == 3 && 2 * co <= 256 && chunk_for(2 * ci) > chunk_for(3 * ci);
}

int wg3_tz(int Z);
int wg3_tz_fit(const TcLayer& L);
Wg3Geom wg3_geom(const TcLayer& L, int B, bool proj = false);
Wg3Geom wg3_geom_fold(const TcLayer& L, int B, int sp);
TcLayer wg3_fold_view(const TcLayer& L);

CUtensorMapSwizzle swizzle_for(int ck) {
  return ck == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                  : (ck == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

// Channels-last BF16 activations [B][Z][Y][X][row] as a 5-D map over C channels of each
// row (row = 0: row = C; else a C-channel block of a wider staged row, `base` at the block),
// box = one tile's taps.
cudaError_t encode_act(CUtensorMap* m, void* base, int B, Dims3 d, int C, int ck, int S,
                       int row = 0) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.x, (cuuint64_t)d.y, (cuuint64_t)d.z,
                              (cuuint64_t)B};
  const cuuint64_t es = 2, R = (cuuint64_t)(row ? row : C);
  const cuuint64_t strides[4] = {R * es, R * es * d.x, R * es * d.x * d.y,
                                 R * es * d.x * d.y * d.z};
  const cuuint32_t box[5] = {(cuuint32_t)ck, (cuuint32_t)(kBX * S), (cuuint32_t)(kBY * S),
                             (cuuint32_t)(kBZ * S), 1};
  const cuuint32_t estr[5] = {1, (cuuint32_t)S, (cuuint32_t)S, (cuuint32_t)S, 1};
  // a channel block of a wider row: no L2 promotion, which would fetch the other blocks too
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(ck),
                        row && row != C ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                                        : CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tap-major weights [B][T][Cout][Cin] (BF16) as a 4-D map (Cin, Cout, T, B); the box holds
// one channel chunk of `taps` taps spaced `tap_stride` apart (one tap, or the 9 taps sharing
// an x offset).
cudaError_t encode_w(CUtensorMap* m, void* base, int B, long long wstride, int cin, int T,
                     int cout, int ck, int taps, int tap_stride) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)cout, (cuuint64_t)T, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)cin * cout * 2,
                                 (cuuint64_t)wstride * 2};
  const cuuint32_t box[4] = {(cuuint32_t)ck, (cuuint32_t)cout,
                             (cuuint32_t)(taps * tap_stride), 1};
  const cuuint32_t estr[4] = {1, 1, (cuuint32_t)tap_stride, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(ck),
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Channels-last activations [B][Z][Y][X][row] (C channels of each row, as encode_act) with a
// bx x by x bz box of ck channels.
cudaError_t encode_box(CUtensorMap* m, void* base, int B, Dims3 d, int C, int ck, int bx, int by,
                       int bz, int row = 0) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.x, (cuuint64_t)d.y, (cuuint64_t)d.z,
                              (cuuint64_t)B};
  const cuuint64_t es = 2, R = (cuuint64_t)(row ? row : C);
  const cuuint64_t strides[4] = {R * es, R * es * d.x, R * es * d.x * d.y,
                                 R * es * d.x * d.y * d.z};
  const cuuint32_t box[5] = {(cuuint32_t)ck, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(ck),
                        row && row != C ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                                        : CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Channels-last activations with an 8 x 18 x (tz + 2) box: the x-shifted halo of an
// 8 x 16 x tz tile for the (y, z) offsets of every tap.
// (row: the staged row's channel count when the map shows only its first C channels)
cudaError_t encode_act_halo(CUtensorMap* m, void* base, int B, Dims3 d, int C, int ck, int tz,
                            int row = 0) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.x, (cuuint64_t)d.y, (cuuint64_t)d.z,
                              (cuuint64_t)B};
  const cuuint64_t es = 2, R = (cuuint64_t)(row ? row : C);
  const cuuint64_t strides[4] = {R * es, R * es * d.x, R * es * d.x * d.y,
                                 R * es * d.x * d.y * d.z};
  const cuuint32_t box[5] = {(cuuint32_t)ck, 8, 18, (cuuint32_t)(tz + 2), 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(ck),
                        row && row != C ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                                        : CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// FP32 channels-last output [B][Z][Y][X][C] (batch stride bs elements) as a 5-D map whose
// box is one 8 x 16 voxel slice of w channels (w = 32: 128-byte swizzle, 16: 64-byte), the
// store form of the persistent halo convolution's epilogue.
cudaError_t encode_out(CUtensorMap* m, void* base, int B, Dims3 d, int C, int w, long long bs) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.x, (cuuint64_t)d.y, (cuuint64_t)d.z,
                              (cuuint64_t)B};
  const cuuint64_t es = 4;
  const cuuint64_t strides[4] = {C * es, C * es * d.x, C * es * d.x * d.y, (cuuint64_t)bs * es};
  const cuuint32_t box[5] = {(cuuint32_t)w, 8, 16, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        w == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// BF16 channels-last tensor [B][Z][Y][X][C] (batch stride bs elements) as a 5-D map whose
// box is one 8 x 16 voxel slice of w channels (rows of 2 w = 32, 64 or 128 bytes, swizzled
// at that width): the BF16 copy stored by the LayerNorm epilogue.
cudaError_t encode_out_bf16(CUtensorMap* m, void* base, int B, Dims3 d, int C, int w,
                            long long bs) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)d.x, (cuuint64_t)d.y, (cuuint64_t)d.z,
                              (cuuint64_t)B};
  const cuuint64_t es = 2;
  const cuuint64_t strides[4] = {C * es, C * es * d.x, C * es * d.x * d.y, (cuuint64_t)bs * es};
  const cuuint32_t box[5] = {(cuuint32_t)w, 8, 16, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(w),
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Epilogue shared memory of the persistent halo convolution: nbuf staging slices (128 rows
// of max(n, np) FP32 outputs; with a LayerNorm of sp BF16 blocks (ln_sp > 0) also xhat and
// the BF16 copy), the bias, gamma and beta of one problem, and alignment slack.
size_t tc3p_slice(int n, int np, int ln_sp) {
  const size_t plain = (size_t)128 * std::max(n, np) * 4;
  const size_t ln = ln_sp ? (size_t)128 * n * (8 + 2 * ln_sp) : 0;
  return std::max(plain, ln);
}
// (nbuf slices per epilogue group)
size_t tc3p_staging(int n, int np, int ln_sp = 0, int nbuf = 1) {
  return kEpiGroups * (nbuf * tc3p_slice(n, np, ln_sp) + (size_t)(3 * n + np) * 4) + 2048;
}

size_t smem_bytes(int ck, int n) { return (size_t)kStages * (kBM + n) * ck * 2 + 1024; }

size_t tc3_stage(int ck, int n, int tz = 1) {
  return (size_t)8 * 18 * (tz + 2) * ck * 2 + (size_t)9 * n * ck * 2;
}

// Largest channel chunk (64, 32, 16) dividing cin whose halo stage stays within 100 KB.
int tc3_chunk(int cin, int n) {
  for (int ck : {64, 32, 16})
    if (cin % ck == 0 && tc3_stage(ck, n) <= 100 * 1024) return ck;
  return 0;
}

constexpr size_t kTc3SmemMax = 210 * 1024;

// z slices per halo-box tile: the z extent in {1, 2, 4} that loads the fewest halo rows per
// z column (ceil(Z / tz) boxes of tz + 2 planes; ties: the smaller), among those whose stage
// stays within 72 KB and whose accumulators within 256 TMEM columns.
int tc3_tz(int ck, int n, int Z) {
  int best = 1;
  long long best_cost = 3LL * Z;
  for (int tz : {2, 4}) {
    if (tc3_stage(ck, n, tz) > 72 * 1024 || tz * n > 256) continue;
    const long long cost = ceil_div(Z, tz) * (tz + 2);
    if (cost < best_cost) best = tz, best_cost = cost;
  }
  return best;
}


// Halo-box launch geometry.  The persistent kernel is planned first: over z depths tz in
// {4, 2, 1} (accumulators of both TMEM buffers within 512 columns) and channel chunks ck
// dividing cin, with at least two ring stages besides the epilogue staging slice, pick the
// least TMA time per output voxel -- rows loaded per z column (halo box of tz + 2 planes per
// x tap, plus the weight boxes) over the TMA line rate (one 32-byte row per clock for ck = 16,
// 64 bytes for wider chunks).  Otherwise one tile per CTA (np must be 0 then).
struct Tc3Plan {
  int ck = 0, tz = 1, nst = 0;
  size_t stage = 0, staging = 0;
  bool persistent = false;
  bool pack = false;  // kz taps packed into N (P3Args::pack)
};

// One persistent candidate: channel chunk ck, z depth tz, kz packing; persistent = false
// when it does not fit (TMEM columns of both accumulator buffers, a stage of at most 100 KB,
// two ring stages besides the epilogue staging).
Tc3Plan tc3_fixed(int cin, int n, int np, int ck, int tz, bool pack) {
  Tc3Plan p;
  if (cin % ck) return p;
  if (pack ? (3 * n > 256 || tz < 2 || (tz + 4) * n + tz * np > 256) : tz * (n + np) > 256)
    return p;
  const size_t staging = tc3p_staging(n, np);
  const size_t stage = tc3_stage(ck, n, tz) + (size_t)np * ck * 2;
  if (stage > 100 * 1024 || staging + 2 * stage + 1024 > kTc3SmemMax) return p;
  p.ck = ck, p.tz = tz, p.pack = pack, p.stage = stage, p.staging = staging;
  p.nst = (int)std::min<size_t>(kP3Max, (kTc3SmemMax - 1024 - staging) / stage);
  p.persistent = true;
  return p;
}

// Every persistent candidate (the autotuner's search space).
std::vector<Tc3Plan> tc3_candidates(int cin, int n, int np) {
  std::vector<Tc3Plan> out;
  for (bool pack : {true, false})
    for (int tz : {8, 4, 2, 1})
      for (int ck : {64, 32, 16}) {
        const Tc3Plan p = tc3_fixed(cin, n, np, ck, tz, pack);
        if (p.persistent) out.push_back(p);
      }
  return out;
}

// The model's choice: the kz-packed form at the largest z depth that fits (about 2.4x fewer
// MMAs at tz 8, 2x at tz 4), else the plain form; the channel chunk (and the plain form's z
// depth) by TMA time per output voxel -- rows loaded per z column (halo box of tz + 2 planes
// per x tap, plus the weight boxes) over the TMA line rate (one 32-byte row per clock for
// ck = 16, 64 bytes for wider chunks); ties to more ring stages.  Without a persistent
// candidate (np must be 0 then), one tile per CTA.
Tc3Plan tc3_plan(int cin, int n, int np, int Z) {
  Tc3Plan best;
  double best_cost = 1e300;
  for (bool pack : {true, false}) {
    for (int tz : {8, 4, 2, 1}) {
      for (int ck : {64, 32, 16}) {
        const Tc3Plan p = tc3_fixed(cin, n, np, ck, tz, pack);
        if (!p.persistent) continue;
        const double rows = (3.0 * 144 * (tz + 2) + 9.0 * n + np) / std::min(32, ck);
        const double cost = pack ? rows : (double)ceil_div(Z, tz) * rows;
        if (!best.persistent || cost < best_cost * (1 - 1e-9) ||
            (cost <= best_cost * (1 + 1e-9) && p.nst > best.nst))
          best = p, best_cost = cost;
      }
      if (pack && best.persistent) return best;
    }
  }
  if (best.persistent || np) return best;
  best.ck = tc3_chunk(cin, n);
  if (best.ck) best.tz = tc3_tz(best.ck, n, Z);
  return best;
}

// Ring stages of the persistent plan pl when the epilogue also holds a LayerNorm of sp BF16
// blocks (nbuf staging slices); 0 when fewer than two would fit.
int tc3_ln_stages(const Tc3Plan& pl, int n, int np, int sp, int nbuf) {
  const size_t staging = tc3p_staging(n, np, sp, nbuf);
  if (!pl.persistent || staging + 2 * pl.stage + 1024 > kTc3SmemMax) return 0;
  return (int)std::min<size_t>(kP3Max, (kTc3SmemMax - 1024 - staging) / pl.stage);
}

// The persistent form with the layer's choice (ck, tz, pack) when per; else one tile per CTA.
cudaError_t launch_tc3(const CUtensorMap& a, const CUtensorMap& w, int cin, int ck, int tz,
                       bool pack, bool per,
                       const float* bias, float* out, Dims3 dout, int n, int B, long long out_bs,
                       long long bias_bs, int acc, int* err, cudaStream_t st,
                       int mode = 0, const CUtensorMap* wp = nullptr,
                       const CUtensorMap* a2 = nullptr, int np = 0, const float* bias_p = nullptr,
                       float* out_p = nullptr, long long outp_bs = 0,
                       const Bf16Ln* ln = nullptr, int fold = 0, float* out2 = nullptr,
                       int split_c = 0) {
  Tc3Plan pl = per ? tc3_fixed(cin, n, mode == 1 ? np : 0, ck, tz, pack) : Tc3Plan{};
  if (per && !pl.persistent) return cudaErrorInvalidValue;
  if (fold && (!per || mode != 0 || n % 32 || (ln && ln->bwd))) return cudaErrorInvalidValue;
  const int no = fold ? n / 2 : n;  // output channels (n: the MMA width)
  const int wbox = no % 32 == 0 ? 32 : 16;  // channels per stored box (the kernel's choice)
  if (split_c && (!per || mode == 1 || ln || !out2 || split_c % wbox || (no - split_c) <= 0 ||
                  (no - split_c) % wbox))
    return cudaErrorInvalidValue;
  int nbuf = 1;  // staging slices per epilogue group
  if (ln) {  // same tiles and ring, a larger epilogue staging
    const int npm = mode == 1 ? np : 0;
    const int nst = tc3_ln_stages(pl, no, npm, ln->sp, 1);
    if (nst < 2 || no > 64) return cudaErrorInvalidValue;
    pl.nst = nst;
  }
  if (pl.persistent) {
    P3Args g{};
    g.bias = bias, g.out = out, g.bias_p = bias_p, g.out_p = out_p, g.err = err;
    g.dout = dout;
    g.N = n, g.Np = np, g.nchunks = cin / ck;
    g.tiles_x = (int)ceil_div(dout.x, 8), g.tiles_y = (int)ceil_div(dout.y, 16);
    g.tiles_z = (int)ceil_div(dout.z, tz);
    g.B = B, g.accumulate = acc, g.nst = pl.nst, g.mode = mode, g.pack = pl.pack ? 1 : 0;
    g.fold = fold;
    g.split_c = split_c;
    g.stage_bytes = (uint32_t)pl.stage;
    g.ring_bytes = (uint32_t)((pl.nst * pl.stage + 1023) / 1024 * 1024);
    const int npm = mode == 1 ? np : 0;
    const int lsp = ln ? ln->sp : 0;
    g.slice_bytes = (uint32_t)tc3p_slice(no, npm, lsp);
    g.nbuf = nbuf;
    g.out_bs = out_bs, g.bias_bs = bias_bs, g.outp_bs = outp_bs, g.biasp_bs = bias_bs;
    const long long total = (long long)g.tiles_x * g.tiles_y * g.tiles_z * B;
    const int grid = (int)std::min<long long>(total, sm_count());
    // (the staging term's slack covers the kernel's 1024-byte alignment of its base)
    const size_t sm = (size_t)g.ring_bytes + tc3p_staging(no, npm, lsp, nbuf);
    CUtensorMap mo{}, mop, mxh, myb;
    // (the LayerNorm backward stores its FP32 output only when asked to)
    cudaError_t e = cudaSuccess;
    if (split_c) {  // two output tensors of split_c and no - split_c channels
      e = encode_out(&mo, out, B, dout, split_c, wbox, dout.count() * split_c);
      if (e == cudaSuccess)
        e = encode_out(&mop, out2, B, dout, no - split_c, wbox, dout.count() * (no - split_c));
    } else {
      if (out) e = encode_out(&mo, out, B, dout, no, wbox, out_bs);
      if (e == cudaSuccess && mode == 1)
        e = encode_out(&mop, out_p, B, dout, np, np % 32 == 0 ? 32 : 16, outp_bs);
      else
        mop = mo;
    }
    mxh = mo, myb = mo;
    if (ln) {
      g.ln = ln->bwd ? 2 : 1, g.act = ln->act, g.sp = ln->sp, g.ybf = ln->ybf ? 1 : 0;
      g.gamma = ln->gamma, g.gamma_bs = ln->gamma_bs;
      g.resid = ln->resid, g.resid_bs = out_bs;
      g.rstd = ln->rstd, g.rstd_bs = dout.count();
      if (ln->bwd) {
        if (mode != 0 || acc || !ln->aout || !ln->xhat || !ln->part)
          return cudaErrorInvalidValue;
        g.aout = ln->aout, g.xh_in = ln->xhat, g.part = ln->part;
        g.rows_b = (long long)g.tiles_x * g.tiles_y * g.tiles_z * kEpiGroups;
      } else if (e == cudaSuccess) {
        e = encode_out(&mxh, ln->xhat, B, dout, no, no % 32 == 0 ? 32 : 16, out_bs);
      }
      if (e == cudaSuccess && ln->ybf)
        e = encode_out_bf16(&myb, ln->ybf, B, dout, ln->sp * no, no, dout.count() * ln->sp * no);
    }
    if (e != cudaSuccess) return e;
    const CUtensorMap& mp = wp ? *wp : w;
    const CUtensorMap& m2 = a2 ? *a2 : a;
#define D2IP_P3(CK_, TZ_) \
  conv_tc3p_kernel<CK_, TZ_><<<grid, kTc3pThreads, sm, st>>>(a, w, mp, m2, mo, mop, mxh, myb, g)
#define D2IP_P3Z(CK_) \
  if (tz == 8) D2IP_P3(CK_, 8); else if (tz == 4) D2IP_P3(CK_, 4); \
  else if (tz == 2) D2IP_P3(CK_, 2); else D2IP_P3(CK_, 1)
    if (ck == 64) { D2IP_P3Z(64); } else if (ck == 32) { D2IP_P3Z(32); } else { D2IP_P3Z(16); }
#undef D2IP_P3Z
#undef D2IP_P3
    return cudaGetLastError();
  }
  if (mode != 0) return cudaErrorInvalidValue;
  const int tx = (int)ceil_div(dout.x, 8), ty = (int)ceil_div(dout.y, 16);
  dim3 grid((unsigned)(tx * ty * ceil_div(dout.z, tz)), 1, B);
  const size_t stage = tc3_stage(ck, n, tz);
  const int nch = cin / ck;
  const int nst = (int)std::min<size_t>({(size_t)kT3Max, (kTc3SmemMax - 1024) / stage,
                                         (size_t)nch * 3});
  // the epilogue stages one 128 x (N + 4) FP32 slice in the pipeline buffers
  const size_t sm = std::max((size_t)nst * stage, (size_t)128 * (n + 4) * 4) + 1024;
  switch (ck) {
    case 64:
      conv_tc3_kernel<64><<<grid, 128, sm, st>>>(a, w, bias, out, dout, n, nch, tx, ty, tz,
                                                  out_bs, bias_bs, acc, nst, err);
      break;
    case 32:
      conv_tc3_kernel<32><<<grid, 128, sm, st>>>(a, w, bias, out, dout, n, nch, tx, ty, tz,
                                                  out_bs, bias_bs, acc, nst, err);
      break;
    default:
      conv_tc3_kernel<16><<<grid, 128, sm, st>>>(a, w, bias, out, dout, n, nch, tx, ty, tz,
                                                  out_bs, bias_bs, acc, nst, err);
      break;
  }
  return cudaGetLastError();
}

// Forward (and stride-1 data-gradient) taps: offset k - pad, weight tap t, stride S.
TapPlan conv_plan(int K, int S) {
  TapPlan p{};
  p.s_in = S;
  p.s_out = 1;
  TapClass& c = p.cls[0];
  const int pad = (K - 1) / 2;
  c.n = K * K * K;
  for (int t = 0; t < c.n; ++t) {
    c.off[t][0] = (int8_t)(t % K - pad);
    c.off[t][1] = (int8_t)((t / K) % K - pad);
    c.off[t][2] = (int8_t)(t / (K * K) - pad);
    c.widx[t] = (uint8_t)t;
  }
  return p;
}

// Stride-2 3x3x3 data gradient as 8 parity classes on the coarse grid.  Per axis, an even
// input position 2q takes tap k = 1 from dy[q]; an odd one 2q + 1 takes k = 0 from dy[q + 1]
// and k = 2 from dy[q].  The weights are the tap-reversed copy (index 26 - t).
TapPlan dgrad_s2_plan() {
  TapPlan p{};
  p.s_in = 1;
  p.s_out = 2;
  const int ks[2][2] = {{1, -1}, {0, 2}}, ds[2][2] = {{0, 0}, {1, 0}}, nk[2] = {1, 2};
  for (int cl = 0; cl < 8; ++cl) {
    const int rx = cl & 1, ry = (cl >> 1) & 1, rz = (cl >> 2) & 1;
    TapClass& c = p.cls[cl];
    c.r[0] = (int8_t)rx;
    c.r[1] = (int8_t)ry;
    c.r[2] = (int8_t)rz;
    c.n = 0;
    for (int a = 0; a < nk[rz]; ++a)
      for (int bb = 0; bb < nk[ry]; ++bb)
        for (int e = 0; e < nk[rx]; ++e) {
          const int kz = ks[rz][a], ky = ks[ry][bb], kx = ks[rx][e];
          const int t = (kz * 3 + ky) * 3 + kx;
          c.off[c.n][0] = (int8_t)ds[rx][e];
          c.off[c.n][1] = (int8_t)ds[ry][bb];
          c.off[c.n][2] = (int8_t)ds[rz][a];
          c.widx[c.n] = (uint8_t)(26 - t);
          ++c.n;
        }
  }
  return p;
}

// The stride-2 data gradient with its classes packed in N: the 8 windows (ox, oy, oz) in
// {0, 1}^3 of dy, window w's weights at block w of the packed tensor.
TapPlan dgrad_s2_packed_plan() {
  TapPlan p{};
  p.s_in = 1;
  p.s_out = 2;
  p.pack = 8;
  TapClass& c = p.cls[0];
  c.n = 8;
  for (int w = 0; w < 8; ++w) {
    c.off[w][0] = (int8_t)(w & 1);
    c.off[w][1] = (int8_t)((w >> 1) & 1);
    c.off[w][2] = (int8_t)((w >> 2) & 1);
    c.widx[w] = (uint8_t)w;
  }
  return p;
}

// qdims: extent of the tile grid (output voxels for s_out = 1, coarse positions for 2).
cudaError_t launch_tc(const CUtensorMap& a, const CUtensorMap& w, const TapPlan& plan,
                      int nclass, int cin, const float* bias, float* out, Dims3 dout,
                      Dims3 qdims, int n, int B, long long out_bs, long long bias_bs, int acc,
                      int* err, cudaStream_t st) {
  const int ck = chunk_for(cin);
  const int tx = (int)ceil_div(qdims.x, kBX), ty = (int)ceil_div(qdims.y, kBY),
            tz = (int)ceil_div(qdims.z, kBZ);
  dim3 grid((unsigned)(tx * ty * tz), nclass, B);
  const size_t sm = smem_bytes(ck, n);
  const int nch = cin / ck;
  switch (ck) {
    case 64:
      conv_tc_kernel<64><<<grid, 128, sm, st>>>(a, w, plan, bias, out, dout, n, nch, tx, ty,
                                                 out_bs, bias_bs, acc, err);
      break;
    case 32:
      conv_tc_kernel<32><<<grid, 128, sm, st>>>(a, w, plan, bias, out, dout, n, nch, tx, ty,
                                                 out_bs, bias_bs, acc, err);
      break;
    default:
      conv_tc_kernel<16><<<grid, 128, sm, st>>>(a, w, plan, bias, out, dout, n, nch, tx, ty,
                                                 out_bs, bias_bs, acc, err);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

bool bf16_conv_supported(int ci, int co, int k) {
  return ci % 16 == 0 && co % 16 == 0 && co >= 16 && co <= 256 && (k == 3 || k == 1);
}

bool bf16_network_supported(int levels, const int* widths, int) {
  for (int l = 0; l < levels; ++l)
    if (widths[l] % 16 != 0) return false;
  return true;
}

int bf16_add_layer(Bf16Net& bf, int ci, int co, int k, int s, Dims3 din, long long w_off) {
  if (!bf16_conv_supported(ci, co, k)) return -1;
  TcLayer L;
  L.ci = ci;
  L.ci_real = ci;
  L.co = co;
  L.k = k;
  L.s = s;
  L.din = din;
  L.dout = conv_out_dims(din, k, s);
  L.w_off = w_off;
  L.kf = bf.sp * ci;
  L.kd = bf.sp * co;
  L.kf3 = L.kf, L.nf3 = co, L.kd3 = L.kd, L.nd3 = ci;
  L.dgrad = (s == 1 || k == 3) && bf16_conv_supported(co, ci, k);
  if (k == 3 && s == 1) {
    // [hi | lo] rows against doubled weights: the forward of 16-output layers with up to 48
    // inputs (a decoder's first conv; its projection then runs on its own), the data
    // gradient of 16 -> 16 layers
    const bool hl = bf.sp == 3 && ci == 16 && co == 16;
    const bool hlf = bf.sp == 3 && co == 16 && ci % 16 == 0 && ci <= 48;
    Tc3Plan pf = hlf ? tc3_plan(2 * ci, 2 * co, 0, L.dout.z) : Tc3Plan{};
    if (pf.persistent)
      L.hlf = true, L.kf3 = 2 * ci, L.nf3 = 2 * co;
    else
      pf = tc3_plan(L.kf, co, 0, L.dout.z);
    L.ck3f = pf.ck, L.tz3f = pf.tz, L.pack3f = pf.pack, L.per3f = pf.persistent;
    if (L.dgrad) {
      Tc3Plan pd = hl ? tc3_plan(2 * co, 2 * ci, 0, L.din.z) : Tc3Plan{};
      if (pd.persistent)
        L.hld = true, L.kd3 = 2 * co, L.nd3 = 2 * ci;
      else
        pd = tc3_plan(L.kd, ci, 0, L.din.z);
      L.ck3d = pd.ck, L.tz3d = pd.tz, L.pack3d = pd.pack, L.per3d = pd.persistent;
    }
  }
  L.wgrad = s == 1 && co <= 128 && 128 % co == 0 && ci + chunk_for(ci) <= 256;
  if (k == 3 && s == 1) L.wg_tz = wg3_tz_fit(L);
  L.wg3 = L.wgrad && wg3_geom(L, 1).nst > 0;
  if (k == 3 && s == 2 && (ci == 16 || ci == 32 || ci == 64) && co % 16 == 0 && co <= 256)
    L.wgrad = L.wgs2 = true;
  L.s2p = L.dgrad && s == 2 && k == 3 && 8 * ci <= 256;
  // the per-tap forward (stride 2) folded where [hi | lo] rows take a wider channel chunk
  if (k == 3 && s == 2 && bf16_fold_pays(bf, ci, co)) L.hlf = true;
  const long long n = (long long)co * k * k * k * ci * bf.sp;
  const long long n4 = (long long)co * k * k * k * ci * 4;  // the doubled [2 co][2 ci] rows
  const long long n64 = (long long)co * 64 * ci * bf.sp;    // 8 x 8 window-class blocks
  L.wf_off = bf.wstride;
  // (a 1x1 layer keeps room for the doubled rows: a projection run on its own folds)
  bf.wstride += ((L.hlf || (k == 1 && bf.sp == 3) ? n4 : n) + 63) / 64 * 64;
  if (L.dgrad) {
    L.wd_off = bf.wstride;
    bf.wstride += ((L.hld ? n4 : L.s2p ? n64 : n) + 63) / 64 * 64;
  }
  bf.layers.push_back(L);
  return (int)bf.layers.size() - 1;
}

int bf16_add_input_layer(Bf16Net& bf, int ci_real, int co, Dims3 din, long long w_off) {
  if (ci_real < 1 || ci_real > 16 || ci_real % 4 != 0) return -1;
  TcLayer L;
  L.ci = 16;
  L.ci_real = ci_real;
  L.co = co;
  L.k = 3;
  L.s = 1;
  L.din = din;
  L.dout = din;
  L.w_off = w_off;
  L.kf = 16 * bf.sp;
  L.kd = co * bf.sp;
  L.kf3 = L.kf, L.nf3 = co, L.kd3 = L.kd, L.nd3 = 16;
  L.input_layer = true;
  if (bf16_conv_supported(16, co, 3)) {
    Tc3Plan pf = bf.sp == 3 && co == 16 ? tc3_plan(32, 2 * co, 0, din.z) : Tc3Plan{};
    if (pf.persistent)
      L.hlf = true, L.kf3 = 32, L.nf3 = 2 * co;
    else
      pf = tc3_plan(L.kf, co, 0, din.z);
    L.ck3f = pf.ck, L.tz3f = pf.tz, L.pack3f = pf.pack, L.per3f = pf.persistent;
  }
  L.wg_tz = wg3_tz_fit(L);
  L.wgrad = L.wg3 = wg3_geom(L, 1).nst > 0;
  if (!L.ck3f || !L.wg3) return -1;
  L.wf_off = bf.wstride;
  bf.wstride += ((long long)(L.hlf ? 2 * co : co) * 27 * (L.hlf ? 32 : L.kf) + 63) / 64 * 64;
  bf.zcount = din.count() * L.kf;
  bf.layers.push_back(L);
  return (int)bf.layers.size() - 1;
}

static __nv_bfloat16* dy_buf(const Bf16Net& bf, const TcLayer& L) {
  return L.dyslot ? bf.ybf2 : bf.ybf;
}

__nv_bfloat16* bf16_dy_buffer(const Bf16Net& bf, int layer) {
  return dy_buf(bf, bf.layers[layer]);
}

void bf16_layout(Bf16Net& bf, char* base, size_t& used, int B, long long max_act) {
  auto take = [&](size_t bytes) {
    char* p = base ? base + used : nullptr;
    used += (bytes + 1023) / 1024 * 1024;
    return p;
  };
  bf.max_act = max_act;
  const size_t act_bytes = (size_t)B * max_act * 2 * bf.sp;
  bf.err = reinterpret_cast<int*>(take(sizeof(int)));
  bf.xbf = reinterpret_cast<__nv_bfloat16*>(take(act_bytes));
  bf.ybf = reinterpret_cast<__nv_bfloat16*>(take(act_bytes));
  bool two_dy = false;
  for (const TcLayer& L : bf.layers) two_dy |= L.dyslot != 0;
  bf.ybf2 = two_dy ? reinterpret_cast<__nv_bfloat16*>(take(act_bytes)) : nullptr;
  bool any_proj = false;
  for (const TcLayer& L : bf.layers) any_proj |= L.projd || L.projw;
  bf.pbf = any_proj ? reinterpret_cast<__nv_bfloat16*>(take(act_bytes)) : nullptr;
  bf.wbuf = reinterpret_cast<__nv_bfloat16*>(take((size_t)B * bf.wstride * 2));
  bf.zbf = bf.zcount ? reinterpret_cast<__nv_bfloat16*>(take((size_t)B * bf.zcount * 2)) : nullptr;
  for (TcLayer& L : bf.layers) {
    if (L.input_layer)
      L.xin = bf.zbf;
    else if (bf.keep_inputs && L.xin_of >= 0)  // an earlier layer's copy of the same input
      L.xin = bf.layers[L.xin_of].xin;
    else if (bf.keep_inputs)
      L.xin = reinterpret_cast<__nv_bfloat16*>(take((size_t)B * L.din.count() * L.kf * 2));
    else
      L.xin = bf.xbf;
  }
}

// Weight-gradient operand maps of one layer for channel block `blk` (0: hi, 1: lo) of the
// staged dy (ybf, co channels per block) and x (the layer input, ci per block), in the box
// form of the kernel that runs it; a fused projection's dz_p column (pbf) likewise.
cudaError_t encode_wgrad_maps(TcLayer& L, const Bf16Net& bf, int B, int blk) {
  const int sp = bf.sp;
  __nv_bfloat16* y = dy_buf(bf, L) + (size_t)blk * L.co;
  __nv_bfloat16* x = L.xin + (size_t)blk * L.ci;
  const int yrow = sp * L.co, xrow = sp * L.ci;
  cudaError_t e = cudaSuccess;
  if (L.wg3) {
    const int tz = L.wg_tz;
    if (blk == 0 && wg3_geom_fold(L, B, sp).nst > 0) {  // [hi | lo]: the first 2 blocks
      const int tq = wg3_fold_view(L).wg_tz;
      e = encode_box(&L.wgqy, y, B, L.dout, 2 * L.co, 2 * L.co, 8, 3, tq + 2, yrow);
      if (e == cudaSuccess)
        e = encode_box(&L.wgqx, x, B, L.din, 2 * L.ci, chunk_for(2 * L.ci), 8, 1, tq, xrow);
      if (e == cudaSuccess && L.projw)
        e = encode_box(&L.wgqp, bf.pbf, B, L.dout, 2 * L.co, 2 * L.co, 8, 1, tq, yrow);
      if (e != cudaSuccess) return e;
    }
    e = encode_box(&L.wgy[blk], y, B, L.dout, L.co, L.co, 8, 3, tz + 2, yrow);
    if (e == cudaSuccess)
      e = encode_box(&L.wgx[blk], x, B, L.din, L.ci, chunk_for(L.ci), 8, 1, tz, xrow);
    if (e == cudaSuccess && L.projw)
      e = encode_box(&L.wgp[blk], bf.pbf + (size_t)blk * L.co, B, L.dout, L.co, L.co, 8, 1, tz,
                     yrow);
  } else {  // per-tap and stride-2 kernels: dy tile boxes, x tile boxes (strided for s = 2)
    e = encode_act(&L.wgy[blk], y, B, L.dout, L.co, chunk_for(L.co), 1, yrow);
    if (e == cudaSuccess)
      e = encode_act(&L.wgx[blk], x, B, L.din, L.ci, chunk_for(L.ci), L.s, xrow);
  }
  return e;
}

// The halo-box maps of one direction (0 forward, 1 data gradient) of a layer for its current
// channel chunk and z depth (the autotuner re-encodes them per candidate).
cudaError_t encode_halo_maps(TcLayer& L, const Bf16Net& bf, int B, int dir) {
  const int T = L.k * L.k * L.k;
  if (dir == 0) {
    __nv_bfloat16* src = L.input_layer ? bf.zbf : L.xin;
    cudaError_t e = encode_act_halo(&L.act_f3, src, B, L.din, L.kf3, L.ck3f, L.tz3f, L.kf);
    if (e == cudaSuccess)
      e = encode_w(&L.w_f3, bf.wbuf + L.wf_off, B, bf.wstride, L.kf3, T, L.nf3, L.ck3f, 9, 3);
    if (e == cudaSuccess && L.projf) {
      const TcLayer& P = bf.layers[L.proj];
      e = encode_w(&L.pw_f, bf.wbuf + P.wf_off, B, bf.wstride, P.kf, 1, P.co, L.ck3f, 1, 1);
    }
    return e;
  }
  cudaError_t e =
      encode_act_halo(&L.act_d3, dy_buf(bf, L), B, L.dout, L.kd3, L.ck3d, L.tz3d, L.kd);
  if (e == cudaSuccess)
    e = encode_w(&L.w_d3, bf.wbuf + L.wd_off, B, bf.wstride, L.kd3, T, L.nd3, L.ck3d, 9, 3);
  if (e == cudaSuccess && L.projd) {
    const TcLayer& P = bf.layers[L.proj];
    e = encode_w(&L.pw_d, bf.wbuf + P.wd_off, B, bf.wstride, P.kd, 1, P.ci, L.ck3d, 1, 1);
    if (e == cudaSuccess) e = encode_box(&L.pa_d, bf.pbf, B, L.dout, L.kd, L.ck3d, 8, 16, L.tz3d);
  }
  return e;
}

cudaError_t bf16_finalize(Bf16Net& bf, int B) {
  for (TcLayer& L : bf.layers) {
    const int T = L.k * L.k * L.k;
    if (L.input_layer) {  // halo-box forward and weight gradient over zbf only
      cudaError_t e = encode_act_halo(&L.act_f3, bf.zbf, B, L.din, L.kf3, L.ck3f, L.tz3f, L.kf);
      if (e == cudaSuccess)
        e = encode_w(&L.w_f3, bf.wbuf + L.wf_off, B, bf.wstride, L.kf3, T, L.nf3, L.ck3f, 9, 3);
      for (int blk = 0; blk < (bf.sp > 1 ? 2 : 1) && e == cudaSuccess; ++blk)
        e = encode_wgrad_maps(L, bf, B, blk);
      if (e != cudaSuccess) return e;
      continue;
    }
    // per-tap forward; folded (hlf without the halo form): the first 2 ci channels of each
    // staged row against the doubled [2 co][2 ci] weights
    const bool fold = L.hlf && !L.ck3f;
    const int kff = fold ? 2 * L.ci : L.kf;
    cudaError_t e = encode_act(&L.act_f, L.xin, B, L.din, kff, chunk_for(kff), L.s,
                               fold ? L.kf : 0);
    if (e == cudaSuccess)
      e = encode_w(&L.w_f, bf.wbuf + L.wf_off, B, bf.wstride, kff, T, fold ? 2 * L.co : L.co,
                   chunk_for(kff), 1, 1);
    if (e == cudaSuccess && L.dgrad) {
      e = encode_act(&L.act_d, dy_buf(bf, L), B, L.dout, L.kd, chunk_for(L.kd), 1);
      if (e == cudaSuccess && L.s2p)  // [window][class x ci][kd]: one box per window
        e = encode_w(&L.w_d, bf.wbuf + L.wd_off, B, bf.wstride, L.kd, 8, 8 * L.ci,
                     chunk_for(L.kd), 1, 1);
      else if (e == cudaSuccess)
        e = encode_w(&L.w_d, bf.wbuf + L.wd_off, B, bf.wstride, L.kd, T, L.ci, chunk_for(L.kd), 1,
                     1);
    }
    for (int blk = 0; L.wgrad && blk < (bf.sp > 1 ? 2 : 1) && e == cudaSuccess; ++blk)
      e = encode_wgrad_maps(L, bf, B, blk);
    if (e == cudaSuccess && L.ck3f) {
      e = encode_act_halo(&L.act_f3, L.xin, B, L.din, L.kf3, L.ck3f, L.tz3f, L.kf);
      if (e == cudaSuccess)
        e = encode_w(&L.w_f3, bf.wbuf + L.wf_off, B, bf.wstride, L.kf3, T, L.nf3, L.ck3f, 9, 3);
    }
    if (e == cudaSuccess && L.ck3d) {
      e = encode_act_halo(&L.act_d3, dy_buf(bf, L), B, L.dout, L.kd3, L.ck3d, L.tz3d, L.kd);
      if (e == cudaSuccess)
        e = encode_w(&L.w_d3, bf.wbuf + L.wd_off, B, bf.wstride, L.kd3, T, L.nd3, L.ck3d, 9, 3);
    }
    if (e == cudaSuccess && L.projf) {  // W_p [1][co][kf] in chunks of this layer's ck
      const TcLayer& P = bf.layers[L.proj];
      e = encode_w(&L.pw_f, bf.wbuf + P.wf_off, B, bf.wstride, P.kf, 1, P.co, L.ck3f, 1, 1);
    }
    if (e == cudaSuccess && L.projd) {  // W_p^T [1][ci][kd] and the dz_p tile box
      const TcLayer& P = bf.layers[L.proj];
      e = encode_w(&L.pw_d, bf.wbuf + P.wd_off, B, bf.wstride, P.kd, 1, P.ci, L.ck3d, 1, 1);
      if (e == cudaSuccess)
        e = encode_box(&L.pa_d, bf.pbf, B, L.dout, L.kd, L.ck3d, 8, 16, L.tz3d);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t stage_rows(const float* x, __nv_bfloat16* y, long long nvox, int C, int sp,
                              cudaStream_t st);

namespace {

struct WgPlan {
  int tg, groups, tiles_x, tiles_y, ntiles, tiles_per_chunk, chunks, nst;
  size_t smem;
};

WgPlan wgrad_plan(const TcLayer& L, int B) {
  WgPlan p;
  p.tiles_x = (int)ceil_div(L.dout.x, kBX);
  p.tiles_y = (int)ceil_div(L.dout.y, kBY);
  p.ntiles = p.tiles_x * p.tiles_y * (int)ceil_div(L.dout.z, kBZ);
  const int T = L.k * L.k * L.k;
  p.tg = std::min(kBM / L.co, T);
  p.groups = (int)ceil_div(T, p.tg);
  const long long want = std::max(1LL, ceil_div(2 * 152, (long long)p.groups * B));
  const int chunks0 = (int)std::min<long long>(p.ntiles, want);
  p.tiles_per_chunk = (int)ceil_div(p.ntiles, chunks0);
  p.chunks = (int)ceil_div(p.ntiles, p.tiles_per_chunk);
  const size_t stage = (size_t)kBM * kBM * 2 + (size_t)(L.ci + chunk_for(L.ci)) * kBM * 2;
  p.nst = (int)std::min<size_t>(kWgMaxStages, (200 * 1024) / stage);
  p.smem = (size_t)p.nst * stage + 1024;
  return p;
}

constexpr int kWgSmemMax = 210 * 1024;

template <int CKA, int CKB>
cudaError_t wgrad_attr() {
  return cudaFuncSetAttribute(wgrad_tc_kernel<CKA, CKB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmemMax);
}

template <int CKA, int CKB>
void launch_wgrad_tc(dim3 grid, size_t smem, const TcLayer& L, const CUtensorMap& my,
                     const CUtensorMap& mx, float* part, const WgPlan& p, int rows_b,
                     int bias_on, int* err, cudaStream_t st) {
  wgrad_tc_kernel<CKA, CKB><<<grid, 128, smem, st>>>(
      my, mx, part, L.dout, L.co, L.ci, L.k, p.tg, p.tiles_per_chunk, p.ntiles, p.tiles_x,
      p.tiles_y, rows_b, p.nst, bias_on, err);
}


constexpr size_t kWg3SmemMax = 210 * 1024;

// z extent of the halo weight-gradient column: among even tz <= 32, the least padding of Z,
// then the longest column (more MMAs per pipeline stage), whose stage (with room for a fused
// projection) still leaves two stages in shared memory.
int wg3_tz_fit(const TcLayer& L) {
  const int Z = L.dout.z, ckb = chunk_for(L.ci);
  int best = 0;
  long long best_pad = 0;
  for (int tz = 32; tz >= 2; tz -= 2) {
    const size_t a_box = (size_t)8 * 3 * (tz + 2) * L.co * 2, b_box = (size_t)8 * tz * ckb * 2;
    const size_t stage = (3 * a_box + 1023) / 1024 * 1024 + (L.ci / ckb + 2) * b_box +
                         (size_t)8 * tz * L.co * 2 + 2048;
    if (2 * stage + 1024 > kWg3SmemMax) continue;
    const long long pad = ceil_div(Z, tz) * tz;
    if (!best || pad < best_pad) best = tz, best_pad = pad;
  }
  return best ? best : 2;
}

int wg3_tz(int Z) {
  int best = 16;
  long long best_pad = ceil_div(Z, 16) * 16;
  for (int tz = 14; tz >= 2; tz -= 2) {
    const long long pad = ceil_div(Z, tz) * tz;
    if (pad < best_pad) best = tz, best_pad = pad;
  }
  return best;
}

// Geometry of the halo weight gradient in the packed form (pack) or with x taps in separate
// accumulators; nst == 0 when the layer does not fit that form.
Wg3Geom wg3_geom_form(const TcLayer& L, int B, bool proj, bool pack, int nx = 1) {
  Wg3Geom g{};
  if (nx != 1 && (!pack || proj)) return g;
  if (L.k != 3 || L.s != 1 || (L.co != 16 && L.co != 32 && L.co != 64)) return g;
  const int ckb = chunk_for(L.ci);
  const int tpm = 128 / L.co, G = (9 + tpm - 1) / tpm, N = L.ci + ckb;
  if (N > 256) return g;
  auto pow2 = [](int c) {
    int t = 32;
    while (t < c) t *= 2;
    return t;
  };
  const int extra = proj ? 1 : 0;  // the projection's accumulator
  const int Np = 3 * nx * L.ci + ckb;  // packed: the three x taps (of nx x sets) in N
  if (pack) {
    if (Np > 256 || (G + extra) * Np > 512) return g;
    g.nkx = 0;
    g.tmem_cols = (uint32_t)pow2((G + extra) * Np);
  } else if ((G + extra) * N <= 512) {  // per-x-tap accumulators with the ones block in N
    g.nkx = (3 * G + extra) * N <= 512 ? 3 : 1;
    g.tmem_cols = (uint32_t)pow2((g.nkx * G + extra) * N);
  } else {  // accumulators of Ci columns, the ones columns apart (ones_sep): the centre x
            // tap's CTA pays one more MMA per K step, so only where the above does not fit
    const int on = 16 * (1 + extra);
    g.nkx = (3 * G + extra) * L.ci + on <= 512 ? 3 : 1;
    if ((G + extra) * L.ci + on > 512) return g;
    g.ones_sep = 1;
    g.tmem_cols = (uint32_t)pow2((g.nkx * G + extra) * L.ci + on);
  }
  g.proj = extra;
  g.tz = L.wg_tz > 0 ? L.wg_tz : wg3_tz(L.dout.z);
  g.a_box = (uint32_t)(8 * 3 * (g.tz + 2) * L.co * 2);
  g.b_box = (uint32_t)(8 * g.tz * ckb * 2);
  const int a_boxes = g.nkx == 0 ? 1 : g.nkx, x_boxes = (g.nkx == 0 ? 3 * nx : 1) * (L.ci / ckb);
  g.nx = nx;
  g.b_off = (uint32_t)((a_boxes * g.a_box + 1023) / 1024 * 1024);
  g.ones_off = g.b_off + (uint32_t)x_boxes * g.b_box;
  g.p_box = proj ? (uint32_t)(8 * g.tz * L.co * 2) : 0u;
  g.p_off = (g.ones_off + g.b_box + 1023) / 1024 * 1024;
  g.stage = (g.p_off + g.p_box + 1023) / 1024 * 1024;
  const int nst = (int)std::min<size_t>(kWg3MaxStages, (kWg3SmemMax - 1024) / g.stage);
  if (nst < 2) return g;
  g.tiles_x = (int)ceil_div(L.dout.x, 8);
  g.tiles_z = (int)ceil_div(L.dout.z, g.tz);
  g.ntiles = g.tiles_x * L.dout.y * g.tiles_z;
  const size_t smem = (size_t)nst * g.stage + 1024;
  const int cps = std::max(1, std::min((int)(233472 / (smem + 1024)), (int)(512 / g.tmem_cols)));
  const long long slots = (long long)sm_count() * cps;
  const long long want = std::max(1LL, slots / ((g.nkx ? 3 / g.nkx : 1) * (long long)B));
  g.tiles_per_chunk = (int)ceil_div(g.ntiles, std::min<long long>(want, g.ntiles));
  g.nchunks = (int)ceil_div(g.ntiles, g.tiles_per_chunk);
  g.nst = nst;
  return g;
}

// The packed form where it fits (fewer, wider MMAs), else the per-x-tap accumulators.
Wg3Geom wg3_geom(const TcLayer& L, int B, bool proj) {
  const Wg3Geom g = wg3_geom_form(L, B, proj, true);
  return g.nst > 0 ? g : wg3_geom_form(L, B, proj, false);
}

// Split precision: the pass with both x sets (dy_hi against x_hi and x_lo), when it fits;
// its chunking is then shared by the other pass (dy_lo x_hi).
Wg3Geom wg3_geom_dual(const TcLayer& L, int B) {
  if (!L.wg3 || L.projw) return Wg3Geom{};
  return wg3_geom_form(L, B, false, true, 2);
}

// Split precision, a layer with 16 output channels: the halo kernel on [hi | lo] rows of dy
// and x seen as 32 and 2 ci channels, all four products (and a fused projection's) in one
// pass (the kernel's fold); packed when the x taps fit in N, else one x tap per CTA.  The
// column depth is the layer's own when two stages fit, else refitted for the wider rows.
TcLayer wg3_fold_view(const TcLayer& L) {
  TcLayer Q = L;
  Q.co = 2 * L.co, Q.ci = 2 * L.ci;
  Wg3Geom g = wg3_geom(Q, 1, L.projw);
  if (g.nst <= 0) Q.wg_tz = wg3_tz_fit(Q);
  return Q;
}
Wg3Geom wg3_geom_fold(const TcLayer& L, int B, int sp) {
  if (sp != 3 || !L.wg3 || L.co != 16 || L.ci % 16 || L.ci > 48) return Wg3Geom{};
  Wg3Geom g = wg3_geom(wg3_fold_view(L), B, L.projw);
  if (g.nst > 0) g.fold = 1, g.rows_b = g.nchunks, g.bias_on = 1;
  return g;
}

template <int CKA, int CKB>
cudaError_t wg3_attr() {
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc3_kernel<CKA, CKB, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kWg3SmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wgrad_tc3_kernel<CKA, CKB, 3>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWg3SmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wgrad_tc3_kernel<CKA, CKB, 0>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWg3SmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wgrad_tc3_kernel<CKA, CKB, 0, 2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWg3SmemMax);
  return e;
}

template <int CKA, int CKB>
void launch_wg3(const TcLayer& L, const Wg3Geom& g, const CUtensorMap& my, const CUtensorMap& mx,
                const CUtensorMap& mp, float* part, float* part_p, int B, int* err,
                cudaStream_t st, const CUtensorMap* mx2p = nullptr) {
  dim3 grid((unsigned)g.nchunks, (unsigned)(g.nkx ? 3 / g.nkx : 1), (unsigned)B);
  const size_t smem = (size_t)g.nst * g.stage + 1024;
  const CUtensorMap& mx2 = mx2p ? *mx2p : mx;
  if (g.nkx == 0 && g.nx == 2)
    wgrad_tc3_kernel<CKA, CKB, 0, 2><<<grid, 128, smem, st>>>(my, mx, mp, mx2, part, part_p,
                                                              L.dout, L.ci, L.ci_real, g, err);
  else if (g.nkx == 0)
    wgrad_tc3_kernel<CKA, CKB, 0><<<grid, 128, smem, st>>>(my, mx, mp, mx2, part, part_p, L.dout,
                                                           L.ci, L.ci_real, g, err);
  else if (g.nkx == 3)
    wgrad_tc3_kernel<CKA, CKB, 3><<<grid, 128, smem, st>>>(my, mx, mp, mx2, part, part_p, L.dout,
                                                           L.ci, L.ci_real, g, err);
  else
    wgrad_tc3_kernel<CKA, CKB, 1><<<grid, 128, smem, st>>>(my, mx, mp, mx2, part, part_p, L.dout,
                                                           L.ci, L.ci_real, g, err);
}

struct S2Plan {
  int groups, tiles_x, tiles_y, ntiles, tiles_per_chunk, chunks, nst;
  size_t stage, smem;
};

S2Plan wgs2_plan(const TcLayer& L, int B) {
  S2Plan p{};
  const int tpm = 128 / L.ci;
  p.groups = (27 + 1 + tpm - 1) / tpm;  // 27 taps and the ones block
  p.tiles_x = (int)ceil_div(L.dout.x, kBX);
  p.tiles_y = (int)ceil_div(L.dout.y, kBY);
  p.ntiles = p.tiles_x * p.tiles_y * (int)ceil_div(L.dout.z, kBZ);
  const long long want = std::max(1LL, (long long)sm_count() / ((long long)p.groups * B));
  p.tiles_per_chunk = (int)ceil_div(p.ntiles, std::min<long long>(want, p.ntiles));
  p.chunks = (int)ceil_div(p.ntiles, p.tiles_per_chunk);
  p.stage = (size_t)tpm * kBM * L.ci * 2 + (size_t)kBM * L.co * 2;
  p.nst = (int)std::min<size_t>(kWgMaxStages, (200 * 1024) / p.stage);
  p.smem = (size_t)p.nst * p.stage + 1024;
  return p;
}

template <int CKA, int CKB>
cudaError_t wgs2_attr() {
  return cudaFuncSetAttribute(wgrad_s2_tc_kernel<CKA, CKB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmemMax);
}

template <int CKA, int CKB>
void launch_wgs2(const TcLayer& L, const S2Plan& p, const CUtensorMap& mx, const CUtensorMap& my,
                 float* part, int rows_b, int bias_on, int B, int* err, cudaStream_t st) {
  dim3 grid((unsigned)p.chunks, (unsigned)p.groups, (unsigned)B);
  wgrad_s2_tc_kernel<CKA, CKB><<<grid, 128, p.smem, st>>>(mx, my, part, L.dout, L.co,
                                                          p.tiles_per_chunk, p.ntiles, p.tiles_x,
                                                          p.tiles_y, rows_b, p.nst, bias_on, err);
}

}  // namespace

long long bf16_wgrad_chunks(const Bf16Net& bf, int layer, int B) {
  const TcLayer& L = bf.layers[layer];
  if (L.wgs2) return wgs2_plan(L, B).chunks;
  if (L.wg3) {
    if (bf.sp > 1) {
      const Wg3Geom f = wg3_geom_fold(L, B, bf.sp);
      if (f.nst > 0) return f.nchunks;
      const Wg3Geom d = wg3_geom_dual(L, B);
      if (d.nst > 0) return d.nchunks;
    }
    return wg3_geom(L, B, L.projw).nchunks;
  }
  return wgrad_plan(L, B).chunks;
}

int bf16_wgrad_passes(const Bf16Net& bf, int layer) {
  const TcLayer& L = bf.layers[layer];
  if (!L.wgrad || bf.sp == 1 || wg3_geom_fold(L, 1, bf.sp).nst > 0) return 1;
  return wg3_geom_dual(L, 1).nst > 0 ? 2 : 3;
}

// Operand blocks (dy, x) of weight-gradient pass p: (hi, hi), (lo, hi), (hi, lo).  The ones
// column sums dy, so the bias partial is kept in the passes that see dy_hi once and dy_lo
// once (the first two).
constexpr int kPassY[3] = {0, 1, 0}, kPassX[3] = {0, 0, 1}, kPassBias[3] = {1, 1, 0};

cudaError_t bf16_conv_wgrad(Bf16Net& bf, int layer, const float* x, const float* dy,
                            float* part, int B, cudaStream_t stream, const float* dz_p,
                            float* part_p, bool x_staged, bool dy_staged) {
  const TcLayer& L = bf.layers[layer];
  if (!L.wgrad || (dz_p && !L.projw)) return cudaErrorInvalidValue;
  const WgPlan p = wgrad_plan(L, B);
  cudaError_t e = L.input_layer || (x_staged && bf.keep_inputs)
                      ? cudaSuccess
                      : stage_rows(x, L.xin, (long long)B * L.din.count(), L.ci, bf.sp, stream);
  if (e == cudaSuccess && !dy_staged)
    e = stage_rows(dy, dy_buf(bf, L), (long long)B * L.dout.count(), L.co, bf.sp, stream);
  if (e != cudaSuccess) return e;
  const int passes = bf16_wgrad_passes(bf, layer);
  // partial-row length as the kernels write it: the input layer keeps its real channels
  const long long row =
      (long long)L.co * L.k * L.k * L.k * (L.input_layer ? L.ci_real : L.ci) + L.co;
  if (L.wgs2) {
    const S2Plan p2 = wgs2_plan(L, B);
    const int ckb = chunk_for(L.co);
    for (int q = 0; q < passes; ++q) {
      float* pq = part + (long long)q * p2.chunks * row;
      const int rows_b = passes * p2.chunks;
      const CUtensorMap &mx = L.wgx[kPassX[q]], &my = L.wgy[kPassY[q]];
#define D2IP_WS2(A_, B_) launch_wgs2<A_, B_>(L, p2, mx, my, pq, rows_b, kPassBias[q], B, bf.err, stream)
      if (L.ci == 16) {
        if (ckb == 16) D2IP_WS2(16, 16); else if (ckb == 32) D2IP_WS2(16, 32); else D2IP_WS2(16, 64);
      } else if (L.ci == 32) {
        if (ckb == 16) D2IP_WS2(32, 16); else if (ckb == 32) D2IP_WS2(32, 32); else D2IP_WS2(32, 64);
      } else {
        if (ckb == 16) D2IP_WS2(64, 16); else if (ckb == 32) D2IP_WS2(64, 32); else D2IP_WS2(64, 64);
      }
#undef D2IP_WS2
    }
    return cudaGetLastError();
  }
  if (L.wg3 && passes == 1 && bf.sp > 1) {  // the split products in one pass
    const Wg3Geom gf = wg3_geom_fold(L, B, bf.sp);
    if (gf.nst <= 0 || (L.projw && (!dz_p || !part_p))) return cudaErrorInvalidValue;
    if (L.projw && !L.projd)  // the fused projection's dz_p staged (else kept from the dgrad)
      e = stage_rows(dz_p, bf.pbf, (long long)B * L.dout.count(), L.co, bf.sp, stream);
    if (e != cudaSuccess) return e;
    launch_wg3<32, 32>(wg3_fold_view(L), gf, L.wgqy, L.wgqx, L.projw ? L.wgqp : L.wgqy, part,
                       L.projw ? part_p : nullptr, B, bf.err, stream);
    return cudaGetLastError();
  }
  if (L.wg3) {
    Wg3Geom g = wg3_geom(L, B, L.projw);
    if (L.projw) {  // the fused projection needs its dz_p staged (kept from the data gradient)
      if (!dz_p || !part_p) return cudaErrorInvalidValue;
      if (!L.projd)
        e = stage_rows(dz_p, bf.pbf, (long long)B * L.dout.count(), L.co, bf.sp, stream);
      if (e != cudaSuccess) return e;
    }
    const long long prow = (long long)L.co * L.ci + L.co;
    // split precision in two passes: (dy_hi; x_hi and x_lo side by side), then (dy_lo; x_hi)
    // with the same chunking; else three passes (hi, hi), (lo, hi), (hi, lo) or one
    Wg3Geom gd{};
    if (passes == 2) {
      gd = wg3_geom_dual(L, B);
      g.tiles_per_chunk = gd.tiles_per_chunk, g.nchunks = gd.nchunks;
      gd.rows_b = 2 * gd.nchunks;
      gd.bias_on = 1;
    }
    g.rows_b = passes * g.nchunks;
    const int ckb = chunk_for(L.ci);
    for (int q = 0; q < passes; ++q) {
      const bool dual = passes == 2 && q == 0;
      const int py = passes == 2 ? q : kPassY[q], px = passes == 2 ? 0 : kPassX[q];
      g.bias_on = passes == 2 ? 1 : kPassBias[q];
      float* pq = part + (long long)q * g.nchunks * row;
      float* ppq = part_p ? part_p + (long long)q * g.nchunks * prow : nullptr;
      const CUtensorMap &my = L.wgy[py], &mx = L.wgx[px];
      const CUtensorMap& mp = g.proj ? L.wgp[py] : my;
      const Wg3Geom& gq = dual ? gd : g;
#define D2IP_WG3(A_, B_) \
  launch_wg3<A_, B_>(L, gq, my, mx, mp, pq, ppq, B, bf.err, stream, dual ? &L.wgx[1] : nullptr)
      if (L.co == 16) {
        if (ckb == 16) D2IP_WG3(16, 16); else if (ckb == 32) D2IP_WG3(16, 32); else D2IP_WG3(16, 64);
      } else if (L.co == 32) {
        if (ckb == 16) D2IP_WG3(32, 16); else if (ckb == 32) D2IP_WG3(32, 32); else D2IP_WG3(32, 64);
      } else {
        if (ckb == 16) D2IP_WG3(64, 16); else if (ckb == 32) D2IP_WG3(64, 32); else D2IP_WG3(64, 64);
      }
#undef D2IP_WG3
    }
    return cudaGetLastError();
  }
  dim3 grid(p.chunks, p.groups, B);
  const int cka = chunk_for(L.co), ckb = chunk_for(L.ci);
  for (int q = 0; q < passes; ++q) {
    float* pq = part + (long long)q * p.chunks * row;
    const int rows_b = passes * p.chunks;
    const CUtensorMap &my = L.wgy[kPassY[q]], &mx = L.wgx[kPassX[q]];
#define D2IP_WGT(A_, B_) \
  launch_wgrad_tc<A_, B_>(grid, p.smem, L, my, mx, pq, p, rows_b, kPassBias[q], bf.err, stream)
    if (cka == 16) {
      if (ckb == 16) D2IP_WGT(16, 16); else if (ckb == 32) D2IP_WGT(16, 32); else D2IP_WGT(16, 64);
    } else if (cka == 32) {
      if (ckb == 16) D2IP_WGT(32, 16); else if (ckb == 32) D2IP_WGT(32, 32); else D2IP_WGT(32, 64);
    } else {
      if (ckb == 16) D2IP_WGT(64, 16); else if (ckb == 32) D2IP_WGT(64, 32); else D2IP_WGT(64, 64);
    }
#undef D2IP_WGT
  }
  return cudaGetLastError();
}

cudaError_t bf16_prepare_kernels() {
  cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<64>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes(64, 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(32, 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(16, 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_tc3_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTc3SmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_tc3_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTc3SmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_tc3_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTc3SmemMax);
#define D2IP_P3A(CK_, TZ_)                                                          \
  if (e == cudaSuccess)                                                             \
    e = cudaFuncSetAttribute(conv_tc3p_kernel<CK_, TZ_>,                            \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc3SmemMax);
  D2IP_P3A(64, 1) D2IP_P3A(64, 2) D2IP_P3A(64, 4) D2IP_P3A(64, 8) D2IP_P3A(32, 1)
  D2IP_P3A(32, 2) D2IP_P3A(32, 4) D2IP_P3A(32, 8) D2IP_P3A(16, 1) D2IP_P3A(16, 2)
  D2IP_P3A(16, 4) D2IP_P3A(16, 8)
#undef D2IP_P3A
  if (e == cudaSuccess) e = wgrad_attr<16, 16>();
  if (e == cudaSuccess) e = wgrad_attr<16, 32>();
  if (e == cudaSuccess) e = wgrad_attr<16, 64>();
  if (e == cudaSuccess) e = wgrad_attr<32, 16>();
  if (e == cudaSuccess) e = wgrad_attr<32, 32>();
  if (e == cudaSuccess) e = wgrad_attr<32, 64>();
  if (e == cudaSuccess) e = wgrad_attr<64, 16>();
  if (e == cudaSuccess) e = wgrad_attr<64, 32>();
  if (e == cudaSuccess) e = wgrad_attr<64, 64>();
  if (e == cudaSuccess) e = wgs2_attr<16, 16>();
  if (e == cudaSuccess) e = wgs2_attr<16, 32>();
  if (e == cudaSuccess) e = wgs2_attr<16, 64>();
  if (e == cudaSuccess) e = wgs2_attr<32, 16>();
  if (e == cudaSuccess) e = wgs2_attr<32, 32>();
  if (e == cudaSuccess) e = wgs2_attr<32, 64>();
  if (e == cudaSuccess) e = wgs2_attr<64, 16>();
  if (e == cudaSuccess) e = wgs2_attr<64, 32>();
  if (e == cudaSuccess) e = wgs2_attr<64, 64>();
  if (e == cudaSuccess) e = wg3_attr<16, 16>();
  if (e == cudaSuccess) e = wg3_attr<16, 32>();
  if (e == cudaSuccess) e = wg3_attr<16, 64>();
  if (e == cudaSuccess) e = wg3_attr<32, 16>();
  if (e == cudaSuccess) e = wg3_attr<32, 32>();
  if (e == cudaSuccess) e = wg3_attr<32, 64>();
  if (e == cudaSuccess) e = wg3_attr<64, 16>();
  if (e == cudaSuccess) e = wg3_attr<64, 32>();
  if (e == cudaSuccess) e = wg3_attr<64, 64>();
  return e;
}

cudaError_t bf16_prepare_weights(Bf16Net& bf, const float* theta, int B, long long Pp,
                                 cudaStream_t stream) {
  if (bf.sp > 1) {  // split weights: one launch, a block per (layer, tap, 32 output channels)
    if (bf.layers.empty() || bf.layers.size() > (size_t)kWMaxLayers) return cudaErrorInvalidValue;
    for (const TcLayer& L : bf.layers)
      if (L.ci > 256) return cudaErrorInvalidValue;
    WTable t{};
    t.nl = (int)bf.layers.size();
    int blk = 0;
    for (int i = 0; i < t.nl; ++i) {
      const TcLayer& L = bf.layers[i];
      const int T = L.k * L.k * L.k;
      t.blk0[i] = blk;
      blk += T * (int)ceil_div(L.co, kWOc);
      t.w_off[i] = L.w_off, t.wf_off[i] = L.wf_off, t.wd_off[i] = L.wd_off;
      t.ci[i] = L.ci, t.ci_real[i] = L.ci_real, t.co[i] = L.co, t.T[i] = T;
      t.dgrad[i] = L.dgrad ? 1 : 0;
      t.permf[i] = L.pack3f ? 1 : 0, t.permd[i] = L.s2p ? 2 : L.pack3d ? 1 : 0;
      t.hlf[i] = L.hlf ? 1 : 0, t.hld[i] = L.hld ? 1 : 0;
    }
    t.blk0[t.nl] = blk;
    weights_split_bf16_kernel<<<dim3((unsigned)blk, B), 256, 0, stream>>>(theta, bf.wbuf, Pp,
                                                                           bf.wstride, t);
    return cudaGetLastError();
  }
  bool fits = bf.layers.size() <= (size_t)kWMaxLayers && !bf.layers.empty();
  for (const TcLayer& L : bf.layers) fits = fits && L.ci <= 256;
  if (fits) {
    WTable t{};
    t.nl = (int)bf.layers.size();
    int blk = 0;
    for (int i = 0; i < t.nl; ++i) {
      const TcLayer& L = bf.layers[i];
      const int T = L.k * L.k * L.k;
      t.blk0[i] = blk;
      blk += T * (int)ceil_div(L.co, kWOc);
      t.w_off[i] = L.w_off, t.wf_off[i] = L.wf_off, t.wd_off[i] = L.wd_off;
      t.ci[i] = L.ci, t.ci_real[i] = L.ci_real, t.co[i] = L.co, t.T[i] = T;
      t.dgrad[i] = L.dgrad ? 1 : 0;
      t.permf[i] = L.pack3f ? 1 : 0, t.permd[i] = L.s2p ? 2 : L.pack3d ? 1 : 0;
      t.hlf[i] = L.hlf ? 1 : 0, t.hld[i] = L.hld ? 1 : 0;
    }
    t.blk0[t.nl] = blk;
    weights_all_bf16_kernel<<<dim3((unsigned)blk, B), 256, 0, stream>>>(theta, bf.wbuf, Pp,
                                                                         bf.wstride, t);
    return cudaGetLastError();
  }
  for (const TcLayer& L : bf.layers) {
    const int T = L.k * L.k * L.k;
    const long long n = (long long)L.co * T * L.ci;
    dim3 grid((unsigned)ceil_div(n, 256), B);
    weights_bf16_kernel<<<grid, 256, 0, stream>>>(theta, bf.wbuf, Pp, bf.wstride, L.w_off,
                                                  L.wf_off, L.wd_off, L.ci, L.ci_real, L.co, T,
                                                  L.dgrad ? 1 : 0, L.pack3f ? 1 : 0,
                                                  L.s2p ? 2 : L.pack3d ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t stage_rows(const float* x, __nv_bfloat16* y, long long nvox, int C, int sp,
                              cudaStream_t st) {
  if (sp == 1) {
    const long long n = nvox * C;
    f32_to_bf16_kernel<<<(unsigned)ceil_div(ceil_div(n, 4), 256), 256, 0, st>>>(x, y, n);
  } else {
    f32_to_bf16_rows_kernel<<<(unsigned)ceil_div(nvox * (C / 4), 256), 256, 0, st>>>(x, y, nvox,
                                                                                    C, sp);
  }
  return cudaGetLastError();
}

namespace {
// z [v][cr] FP32 -> zp [v][16 sp] BF16, channels cr..15 of each block zero (sp 3: blocks
// [hi | lo | hi]); one thread per (voxel, channel).
__global__ void pad_input_kernel(const float* __restrict__ z, __nv_bfloat16* __restrict__ zp,
                                 long long nvox, int cr, int sp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox * 16) return;
  const long long v = i / 16;
  const int c = (int)(i % 16);
  const float x = c < cr ? z[v * cr + c] : 0.f;
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  __nv_bfloat16* row = zp + v * 16 * sp;
  row[c] = hi;
  if (sp > 1) {
    row[16 + c] = __float2bfloat16_rn(x - __bfloat162float(hi));
    row[32 + c] = hi;
  }
}
}  // namespace

int bf16_fuse_proj(Bf16Net& bf, int la, int lp) {
  TcLayer& A = bf.layers[la];
  TcLayer& P = bf.layers[lp];
  if (A.k != 3 || A.s != 1 || P.k != 1 || P.ci != A.ci || P.co != A.co || A.input_layer)
    return 0;
  A.proj = lp;
  if (A.ck3f) {
    const Tc3Plan pf = A.hlf ? Tc3Plan{} : tc3_plan(A.kf3, A.nf3, P.co, A.dout.z);
    if (pf.persistent)
      A.projf = true, A.ck3f = pf.ck, A.tz3f = pf.tz, A.pack3f = pf.pack, A.per3f = true;
  }
  if (A.ck3d && P.dgrad) A.projd = A.per3d;  // the dz_p stage rides the persistent dgrad
  A.projw = A.wg3 && wg3_geom(A, 1, true).nst > 0;
  if (!A.projf && P.kf == A.kf) {  // its own launch over la's staged input
    P.xin_of = la;
    P.hlf = bf16_fold_pays(bf, P.ci, P.co);
  }
  return (A.projf ? 1 : 0) | (A.projd ? 2 : 0) | (A.projw ? 4 : 0);
}

bool bf16_input_shared(const Bf16Net& bf, int layer) {
  return bf.keep_inputs && bf.layers[layer].xin_of >= 0;
}

cudaError_t bf16_conv_fwd_proj(Bf16Net& bf, int la, const float* x, const float* bias_a,
                               float* y_a, const float* bias_p, float* y_p, int B,
                               long long bias_bs, cudaStream_t stream, bool x_staged) {
  const TcLayer& L = bf.layers[la];
  if (!L.projf) return cudaErrorInvalidValue;
  cudaError_t e = x_staged && bf.keep_inputs
                      ? cudaSuccess
                      : stage_rows(x, L.xin, (long long)B * L.din.count(), L.ci, bf.sp, stream);
  if (e != cudaSuccess) return e;
  return launch_tc3(L.act_f3, L.w_f3, L.kf, L.ck3f, L.tz3f, L.pack3f, L.per3f, bias_a, y_a, L.dout, L.co, B,
                    L.dout.count() * L.co, bias_bs, 0, bf.err, stream, 1, &L.pw_f, nullptr,
                    L.co, bias_p, y_p, L.dout.count() * L.co);
}

cudaError_t bf16_conv_dgrad_proj(Bf16Net& bf, int la, const float* dz_a, const float* dz_p,
                                 float* dx, int B, cudaStream_t stream, bool dza_staged,
                                 bool dzp_staged, float* dx2, int split_c) {
  const TcLayer& L = bf.layers[la];
  if (!L.projd) return cudaErrorInvalidValue;
  const long long nv = (long long)B * L.dout.count();
  cudaError_t e = dza_staged ? cudaSuccess : stage_rows(dz_a, dy_buf(bf, L), nv, L.co, bf.sp, stream);
  if (e == cudaSuccess && !dzp_staged) e = stage_rows(dz_p, bf.pbf, nv, L.co, bf.sp, stream);
  if (e != cudaSuccess) return e;
  return launch_tc3(L.act_d3, L.w_d3, L.kd, L.ck3d, L.tz3d, L.pack3d, L.per3d, nullptr, dx, L.din, L.ci, B,
                    L.din.count() * L.ci, 0, 0, bf.err, stream, 2, &L.pw_d, &L.pa_d, 0, nullptr,
                    nullptr, 0, nullptr, 0, dx2, split_c);
}

namespace {
// Autotuner cache: shape key -> (ck, tz, pack, time of the choice, time of the model's choice)
struct TuneEntry {
  int ck, tz, pack;
  float us, model_us;
};
std::mutex g_tune_mu;
std::map<std::array<long long, 11>, TuneEntry> g_tune;
}  // namespace

cudaError_t bf16_autotune(Bf16Net& bf, int B, float* scratch, const float* bias,
                          cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (size_t li = 0; e == cudaSuccess && li < bf.layers.size(); ++li) {
    TcLayer& L = bf.layers[li];
    for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir) {
      const bool on = dir == 0 ? L.ck3f && L.per3f : L.ck3d && L.per3d;
      if (!on) continue;
      const int cin = dir ? L.kd3 : L.kf3, n = dir ? L.nd3 : L.nf3;
      const int fold = dir ? (L.hld ? 1 : 0) : (L.hlf ? 1 : 0), no = fold ? n / 2 : n;
      const int np = dir == 0 && L.projf ? bf.layers[L.proj].co : 0;
      const int mode = dir == 0 ? (L.projf ? 1 : 0) : (L.projd ? 2 : 0);
      const Dims3 d = dir ? L.din : L.dout;
      int &ck = dir ? L.ck3d : L.ck3f, &tz = dir ? L.tz3d : L.tz3f;
      bool& pack = dir ? L.pack3d : L.pack3f;
      float &tune = dir ? L.tune_d : L.tune_f, &model = dir ? L.model_d : L.model_f;
      const std::array<long long, 11> key{dev, dir, cin, n, np, mode, d.z, d.y, d.x, B, bf.sp};
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
          ck = it->second.ck, tz = it->second.tz, pack = it->second.pack != 0;
          tune = it->second.us, model = it->second.model_us;
          continue;
        }
      }
      const int mck = ck, mtz = tz;
      const bool mpack = pack;
      float best = 1e30f, model_us = -1.f;
      int bck = ck, btz = tz;
      bool bpack = pack;
      auto launch = [&](const Tc3Plan& c) {
        if (dir == 0)
          return launch_tc3(L.act_f3, L.w_f3, cin, c.ck, c.tz, c.pack, true, bias, scratch, d, n,
                            B, d.count() * no, 0, 0, bf.err, st, mode,
                            mode == 1 ? &L.pw_f : nullptr, nullptr, np, bias, scratch,
                            d.count() * np, nullptr, fold);
        return launch_tc3(L.act_d3, L.w_d3, cin, c.ck, c.tz, c.pack, true, nullptr, scratch, d,
                          n, B, d.count() * no, 0, 0, bf.err, st, mode,
                          mode == 2 ? &L.pw_d : nullptr, mode == 2 ? &L.pa_d : nullptr, 0,
                          nullptr, nullptr, 0, nullptr, fold);
      };
      for (const Tc3Plan& c : tc3_candidates(cin, n, np)) {
        ck = c.ck, tz = c.tz, pack = c.pack;
        e = encode_halo_maps(L, bf, B, dir);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch(c);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch(c);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const float us = 1e3f * ms / 5.f;
        if (c.ck == mck && c.tz == mtz && c.pack == mpack) model_us = us;
        if (us < best) best = us, bck = c.ck, btz = c.tz, bpack = c.pack;
      }
      if (e != cudaSuccess) break;
      ck = bck, tz = btz, pack = bpack, tune = best, model = model_us;
      e = encode_halo_maps(L, bf, B, dir);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = TuneEntry{bck, btz, bpack ? 1 : 0, best, model_us};
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

cudaError_t bf16_apply_plan(Bf16Net& bf, int B, const long long* rows, int n_rows) {
  if (n_rows != (int)bf.layers.size()) return cudaErrorInvalidValue;
  for (int i = 0; i < n_rows; ++i) {  // every row must describe layer i as planned here
    const TcLayer& L = bf.layers[i];
    const long long* r = rows + 15LL * i;
    const long long shape[7] = {L.ci_real, L.co, L.k, L.s, L.dout.z, L.dout.y, L.dout.x};
    for (int j = 0; j < 7; ++j)
      if (r[j] != shape[j]) return cudaErrorInvalidValue;
    for (int dir = 0; dir < 2; ++dir) {
      const bool on = dir == 0 ? L.ck3f && L.per3f : L.ck3d && L.per3d;
      const long long* t = r + 7 + 4 * dir;  // persistent, packed, chunk, z depth
      if ((t[0] != 0) != on) return cudaErrorInvalidValue;
      if (!on) continue;
      const int np = dir == 0 && L.projf ? bf.layers[L.proj].co : 0;
      const Tc3Plan p = tc3_fixed(dir ? L.kd3 : L.kf3, dir ? L.nd3 : L.nf3, np, (int)t[2], (int)t[3],
                                  t[1] != 0);
      if (!p.persistent) return cudaErrorInvalidValue;
    }
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_rows && e == cudaSuccess; ++i) {
    TcLayer& L = bf.layers[i];
    const long long* r = rows + 15LL * i;
    for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir) {
      if (!r[7 + 4 * dir]) continue;
      const long long* t = r + 7 + 4 * dir;
      (dir ? L.pack3d : L.pack3f) = t[1] != 0;
      (dir ? L.ck3d : L.ck3f) = (int)t[2];
      (dir ? L.tz3d : L.tz3f) = (int)t[3];
      (dir ? L.tune_d : L.tune_f) = -1.f;
      (dir ? L.model_d : L.model_f) = -1.f;
      e = encode_halo_maps(L, bf, B, dir);
    }
  }
  return e;
}

long long bf16_tune_scratch_floats(const Bf16Net& bf, int B) {
  long long m = 0;
  for (const TcLayer& L : bf.layers)
    m = std::max(m, std::max(L.dout.count() * L.co, L.din.count() * L.ci));
  return m * B;
}

bool bf16_fwd_ln_ok(const Bf16Net& bf, int layer, int np, int sp) {
  const TcLayer& L = bf.layers[layer];
  if (!L.ck3f || !L.per3f || L.co > 64 || (np > 0 && !L.projf)) return false;
  const Tc3Plan pl = tc3_fixed(L.kf3, L.nf3, np, L.ck3f, L.tz3f, L.pack3f);
  return tc3_ln_stages(pl, L.co, np, sp, 1) >= 2;
}

cudaError_t bf16_conv_fwd_ln(Bf16Net& bf, int layer, const float* x, const float* bias, float* y,
                             const Bf16Ln& ln, int B, long long bias_bs, cudaStream_t stream,
                             bool x_staged, const float* bias_p, float* y_p) {
  const TcLayer& L = bf.layers[layer];
  const bool proj = y_p != nullptr;
  if (proj && !L.projf) return cudaErrorInvalidValue;
  cudaError_t e = L.input_layer || (x_staged && bf.keep_inputs)
                      ? cudaSuccess
                      : stage_rows(x, L.xin, (long long)B * L.din.count(), L.ci, bf.sp, stream);
  if (e != cudaSuccess) return e;
  Bf16Ln l = ln;
  l.sp = bf.sp;
  const long long obs = L.dout.count() * L.co;
  return launch_tc3(L.act_f3, L.w_f3, L.kf3, L.ck3f, L.tz3f, L.pack3f, L.per3f, bias, y, L.dout,
                    L.nf3, B, obs, bias_bs, 0, bf.err, stream, proj ? 1 : 0,
                    proj ? &L.pw_f : nullptr, nullptr, proj ? L.co : 0, bias_p, y_p,
                    proj ? obs : 0, &l, L.hlf ? 1 : 0);
}

cudaError_t bf16_stage_input(Bf16Net& bf, int layer, const float* z, int B, cudaStream_t stream) {
  const TcLayer& L = bf.layers[layer];
  if (!L.input_layer || !bf.zbf) return cudaErrorInvalidValue;
  const long long nvox = (long long)B * L.din.count();
  pad_input_kernel<<<(unsigned)ceil_div(nvox * 16, 256), 256, 0, stream>>>(z, bf.zbf, nvox,
                                                                          L.ci_real, bf.sp);
  return cudaGetLastError();
}

__nv_bfloat16* bf16_input_buffer(const Bf16Net& bf, int layer) {
  const TcLayer& L = bf.layers[layer];
  return bf.keep_inputs && !L.input_layer ? L.xin : nullptr;
}

cudaError_t bf16_conv_fwd(Bf16Net& bf, int layer, const float* x, const float* bias, float* y,
                          int B, long long bias_bs, cudaStream_t stream, bool x_staged) {
  const TcLayer& L = bf.layers[layer];
  cudaError_t e = L.input_layer || (x_staged && bf.keep_inputs)
                      ? cudaSuccess
                      : stage_rows(x, L.xin, (long long)B * L.din.count(), L.ci, bf.sp, stream);
  if (e != cudaSuccess) return e;
  if (L.ck3f)
    return launch_tc3(L.act_f3, L.w_f3, L.kf3, L.ck3f, L.tz3f, L.pack3f, L.per3f, bias, y,
                      L.dout, L.nf3, B, L.dout.count() * L.co, bias_bs, 0, bf.err, stream, 0,
                      nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, L.hlf ? 1 : 0);
  TapPlan plan = conv_plan(L.k, L.s);
  plan.fold = L.hlf ? 1 : 0;  // (no halo form here)
  return launch_tc(L.act_f, L.w_f, plan, 1, L.hlf ? 2 * L.ci : L.kf, bias, y, L.dout, L.dout,
                   L.hlf ? 2 * L.co : L.co, B, L.dout.count() * L.co, bias_bs, 0, bf.err,
                   stream);
}

cudaError_t bf16_conv_dgrad(Bf16Net& bf, int layer, const float* dy, float* dx, int B,
                            int accumulate, cudaStream_t stream, bool dy_staged) {
  const TcLayer& L = bf.layers[layer];
  if (!L.dgrad) return cudaErrorInvalidValue;
  cudaError_t e =
      dy_staged ? cudaSuccess
                : stage_rows(dy, dy_buf(bf, L), (long long)B * L.dout.count(), L.co, bf.sp, stream);
  if (e != cudaSuccess) return e;
  if (L.s == 2) {
    const Dims3 q{(L.din.z + 1) / 2, (L.din.y + 1) / 2, (L.din.x + 1) / 2};
    if (L.s2p)
      return launch_tc(L.act_d, L.w_d, dgrad_s2_packed_plan(), 1, L.kd, nullptr, dx, L.din, q,
                       8 * L.ci, B, L.din.count() * L.ci, 0, accumulate, bf.err, stream);
    return launch_tc(L.act_d, L.w_d, dgrad_s2_plan(), 8, L.kd, nullptr, dx, L.din, q, L.ci, B,
                     L.din.count() * L.ci, 0, accumulate, bf.err, stream);
  }
  if (L.ck3d)
    return launch_tc3(L.act_d3, L.w_d3, L.kd3, L.ck3d, L.tz3d, L.pack3d, L.per3d, nullptr, dx,
                      L.din, L.nd3, B, L.din.count() * L.ci, 0, accumulate, bf.err, stream, 0,
                      nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, L.hld ? 1 : 0);
  return launch_tc(L.act_d, L.w_d, conv_plan(L.k, 1), 1, L.kd, nullptr, dx, L.din, L.din, L.ci,
                   B, L.din.count() * L.ci, 0, accumulate, bf.err, stream);
}

bool bf16_dgrad_ln_ok(const Bf16Net& bf, int layer, int sp) {
  const TcLayer& L = bf.layers[layer];
  if (!L.dgrad || L.s != 1 || !L.ck3d || !L.per3d || L.projd || L.ci > 64 || L.hld)
    return false;
  const Tc3Plan pl = tc3_fixed(L.kd3, L.nd3, 0, L.ck3d, L.tz3d, L.pack3d);
  return tc3_ln_stages(pl, L.ci, 0, sp, 1) >= 2;
}

long long bf16_dgrad_ln_rows(const Bf16Net& bf, int layer) {
  const TcLayer& L = bf.layers[layer];
  const int tz = std::max(L.tz3d, 1);
  return ceil_div(L.din.x, 8) * ceil_div(L.din.y, 16) * ceil_div(L.din.z, tz) * kEpiGroups;
}

cudaError_t bf16_conv_dgrad_ln(Bf16Net& bf, int layer, const float* dy, float* dz_out,
                               const Bf16Ln& ln, int B, cudaStream_t stream, bool dy_staged) {
  const TcLayer& L = bf.layers[layer];
  if (!ln.bwd || !bf16_dgrad_ln_ok(bf, layer, bf.sp)) return cudaErrorInvalidValue;
  cudaError_t e =
      dy_staged ? cudaSuccess
                : stage_rows(dy, dy_buf(bf, L), (long long)B * L.dout.count(), L.co, bf.sp, stream);
  if (e != cudaSuccess) return e;
  Bf16Ln l = ln;
  l.sp = bf.sp;
  return launch_tc3(L.act_d3, L.w_d3, L.kd3, L.ck3d, L.tz3d, L.pack3d, L.per3d, nullptr, dz_out,
                    L.din, L.nd3, B, L.din.count() * L.ci, 0, 0, bf.err, stream, 0, nullptr,
                    nullptr, 0, nullptr, nullptr, 0, &l);
}

long long bf16_op_workspace(int B, Dims3 din, int ci, int co, int k, int s) {
  const Dims3 dout = conv_out_dims(din, k, s);
  const long long T = (long long)k * k * k;
  const long long act = std::max(din.count() * ci, dout.count() * co);
  // forward and data-gradient weights (the packed stride-2 form holds 64 blocks, not 27)
  const long long w = (co * T * ci + 63) / 64 * 64 + (co * 64 * ci + 63) / 64 * 64;
  return 1024 + 2 * (((long long)B * act * 2 + 1023) / 1024 * 1024) +
         ((long long)B * w * 2 + 1023) / 1024 * 1024 + 1024;
}

cudaError_t bf16_op_conv(bool dgrad, const float* in, const float* W, const float* bias,
                         float* out, int B, Dims3 din, int ci, int co, int k, int s,
                         long long w_bs, int accumulate, void* workspace, cudaStream_t st) {
  cudaError_t e = bf16_prepare_kernels();  // opt-in shared memory size, once per device
  if (e != cudaSuccess) return e;
  Bf16Net bf;
  const int idx = bf16_add_layer(bf, ci, co, k, s, din, 0);
  if (idx < 0 || (dgrad && !bf.layers[idx].dgrad)) return cudaErrorInvalidValue;
  // per-problem weight blocks are packed at wstride in the workspace copy
  size_t used = 0;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 1023) &
                                       ~(uintptr_t)1023);
  const Dims3 dout = conv_out_dims(din, k, s);
  bf16_layout(bf, base, used, B, std::max(din.count() * ci, dout.count() * co));
  e = bf16_finalize(bf, B);
  if (e == cudaSuccess) e = cudaMemsetAsync(bf.err, 0, sizeof(int), st);
  if (e == cudaSuccess && bf.layers[idx].s2p)  // the packed form's unwritten blocks are zeros
    e = cudaMemsetAsync(bf.wbuf, 0, (size_t)B * bf.wstride * 2, st);
  if (e == cudaSuccess) e = bf16_prepare_weights(bf, W, B, w_bs, st);
  if (e != cudaSuccess) return e;
  return dgrad ? bf16_conv_dgrad(bf, idx, in, out, B, accumulate, st)
               : bf16_conv_fwd(bf, idx, in, bias, out, B, w_bs, st);
}

long long bf16_op_wgrad_workspace(int B, Dims3 din, int ci, int co, int k) {
  Bf16Net bf;
  const int idx = bf16_add_layer(bf, ci, co, k, 1, din, 0);
  if (idx < 0 || !bf.layers[idx].wgrad) return -1;
  const long long rows = bf16_wgrad_chunks(bf, idx, B);
  return bf16_op_workspace(B, din, ci, co, k, 1) +
         (long long)B * rows * ((long long)co * k * k * k * ci + co) * 4 + 1024;
}

cudaError_t bf16_op_wgrad(const float* x, const float* dy, float* dWb, int B, Dims3 din, int ci,
                          int co, int k, long long dw_bs, int accumulate, void* workspace,
                          cudaStream_t st) {
  cudaError_t e = bf16_prepare_kernels();
  if (e != cudaSuccess) return e;
  Bf16Net bf;
  const int idx = bf16_add_layer(bf, ci, co, k, 1, din, 0);
  if (idx < 0 || !bf.layers[idx].wgrad) return cudaErrorInvalidValue;
  size_t used = 0;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 1023) &
                                       ~(uintptr_t)1023);
  bf16_layout(bf, base, used, B, std::max(din.count() * ci, din.count() * co));
  float* part = reinterpret_cast<float*>(base + used);
  e = bf16_finalize(bf, B);
  if (e == cudaSuccess) e = cudaMemsetAsync(bf.err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = bf16_conv_wgrad(bf, idx, x, dy, part, B, st);
  if (e != cudaSuccess) return e;
  const long long row = (long long)co * k * k * k * ci + co;
  return reduce_rows_f32(part, dWb, B, bf16_wgrad_chunks(bf, idx, B), row, dw_bs, accumulate, st);
}

}  // namespace d2ip
