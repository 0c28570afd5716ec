// The sensitivity products J x and J^T r of the data term (Eq. 4) on the tensor cores: one
// warp-specialised kernel for both (warp 0 issues the TMA loads into a 4-stage ring, one thread
// of warp 1 the tcgen05.mma of M 128 x N 16 x K 16, warps 2-5 drain a double-buffered TMEM
// accumulator), the problems of the group in N.
//   J x:    M = 128 measurements i, K = voxels j (split across CTAs into chunks), A = J read
//           MN-major from rows of Jt (two 64 x 64 boxes per 64 voxels), B = the staged x;
//           each (tile, chunk) item writes its partial sums, added in chunk order afterwards.
//   J^T r:  M = 128 voxels j, K = all m measurements, A = Jt K-major (one 128 x 64 box per 64
//           measurements), B = the staged r; the epilogue writes scale * D.
// Every mbarrier wait is bounded; a wait that runs out sets a bit in the error word and the
// role stops, and TMEM is freed only after the MMA thread's last commit completed.
#include <algorithm>

#include "common.cuh"
#include "jprod_tc.cuh"
#include "tc_prims.cuh"

namespace d2ip {
namespace {

constexpr int kJpThreads = 192;
constexpr int kJpStages = 4;
constexpr uint32_t kJpA = 16384;  // A bytes of one operand block per stage: 128 x 64 BF16
constexpr uint32_t kJpB = 2048;   // B bytes: 16 problems x 64 BF16

struct JpArgs {
  int m, n, B;
  int mtiles;      // 128-row tiles of M
  int kblocks;     // 64-wide blocks of K
  int kper;        // K blocks per item
  int items;       // mtiles x K chunks
  int jmul;        // 1: partial sums of J x; 0: J^T r
  float* out;      // jmul: part [chunk][B][m]; else g [b][n] at out_bs
  long long out_bs;
  float scale;
  int* err;
};

template <bool SPLIT>
__global__ void __launch_bounds__(kJpThreads, 1)
jprod_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tal,
                const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap tbl,
                const __grid_constant__ JpArgs g) {
  constexpr int nA = SPLIT ? 2 : 1;
  constexpr uint32_t kStage = nA * (kJpA + kJpB);  // A hi | A lo | B hi | B lo
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kJpStages], empty[kJpStages], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_s;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int b0 = blockIdx.y * 16;
  const int nit = (int)blockIdx.x < g.items ? (g.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kJpStages; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);
      mbar_init(smem_u32(&tempty[q]), 128);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_s)), "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int k = 0;
      bool good = true;
      for (int it = 0; it < nit && good; ++it) {
        const int item = blockIdx.x + it * gridDim.x;
        const int mt = item % g.mtiles, kc = item / g.mtiles;
        const int kb0 = kc * g.kper, kb1 = min(kb0 + g.kper, g.kblocks);
        for (int kb = kb0; kb < kb1; ++kb, ++k) {
          const int s = k % kJpStages, round = k / kJpStages;
          if (round > 0 && !mbar_wait(smem_u32(&empty[s]), (round - 1) & 1)) {
            atomicOr(g.err, kErrProducer);
            good = false;
            break;
          }
          const uint32_t fb = smem_u32(&full[s]);
          const uint32_t dst = smem_u32(smem + (size_t)s * kStage);
          mbar_expect_tx(fb, kStage);
          for (int h = 0; h < nA; ++h) {
            const CUtensorMap* A = h ? &tal : &ta;
            const uint32_t da = dst + (uint32_t)h * kJpA;
            if (g.jmul) {  // J rows i of voxels j: two 64-measurement blocks
              tma_load_2d(da, A, mt * 128, kb * 64, fb);
              tma_load_2d(da + kJpA / 2, A, mt * 128 + 64, kb * 64, fb);
            } else {       // Jt rows j, measurements i
              tma_load_2d(da, A, kb * 64, mt * 128, fb);
            }
            tma_load_2d(dst + nA * kJpA + (uint32_t)h * kJpB, h ? &tbl : &tb, kb * 64, b0, fb);
          }
        }
      }
      drain_loads(full, kJpStages, k, g.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = instr_desc_major(16, g.jmul != 0, false);
      int k = 0;
      bool good = true;
      for (int it = 0; it < nit && good; ++it) {
        const int buf = it & 1;
        if (it >= 2 && !mbar_wait(smem_u32(&tempty[buf]), ((it >> 1) - 1) & 1)) {
          atomicOr(g.err, kErrMma);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 16);
        const int item = blockIdx.x + it * gridDim.x;
        const int kc = item / g.mtiles;
        const int kb0 = kc * g.kper, kb1 = min(kb0 + g.kper, g.kblocks);
        for (int kb = kb0; kb < kb1; ++kb, ++k) {
          const int s = k % kJpStages;
          if (!mbar_wait(smem_u32(&full[s]), (k / kJpStages) & 1)) {
            atomicOr(g.err, kErrMma);
            good = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + (size_t)s * kStage);
          // J x: MN-major A, 64-measurement blocks 8 KB apart, 8-voxel groups 1 KB apart;
          // J^T r: K-major A, 128 rows of 64 measurements
          const uint64_t a0 = g.jmul ? smem_desc_mn2<64>(base, kJpA / 2, 1024) : smem_desc<64>(base);
          const uint64_t a1 = g.jmul ? smem_desc_mn2<64>(base + kJpA, kJpA / 2, 1024)
                                     : smem_desc<64>(base + kJpA);
          const uint64_t b0d = smem_desc<64>(base + nA * kJpA);
          const uint64_t b1d = smem_desc<64>(base + nA * kJpA + kJpB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // K = 16 per MMA
            const uint32_t ao = g.jmul ? (uint32_t)(kk * (2048 >> 4)) : (uint32_t)(kk * 2);
            const uint32_t bo = (uint32_t)(kk * 2);
            const uint32_t acc = (kb > kb0 || kk > 0) ? 1u : 0u;
            mma_lh_p(d, (uint32_t)a0 + ao, (uint32_t)(a0 >> 32), (uint32_t)b0d + bo,
                     (uint32_t)(b0d >> 32), idesc, acc);
            if (SPLIT) {  // + J_lo x_hi + J_hi x_lo
              mma_lh(d, (uint32_t)a1 + ao, (uint32_t)(a1 >> 32), (uint32_t)b0d + bo,
                     (uint32_t)(b0d >> 32), idesc);
              mma_lh(d, (uint32_t)a0 + ao, (uint32_t)(a0 >> 32), (uint32_t)b1d + bo,
                     (uint32_t)(b1d >> 32), idesc);
            }
          }
          mma_commit(smem_u32(&empty[s]));
        }
        if (good) mma_commit(smem_u32(&tfull[buf]));
      }
      mma_commit(smem_u32(&done));  // fires once every issued MMA has completed
    }
  } else {  // epilogue: warps 2..5, TMEM lane quadrant warp % 4
    const int quad = warp & 3;
    for (int it = 0; it < nit; ++it) {
      const int buf = it & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[buf]), (it >> 1) & 1));
      if (!ok) {
        if (lane == 0) atomicOr(g.err, kErrEpilogue);
        break;
      }
      tc_fence_after();
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 16), r);
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[buf]));
      const int item = blockIdx.x + it * gridDim.x;
      const int mt = item % g.mtiles, kc = item / g.mtiles;
      const int row = mt * 128 + quad * 32 + lane;
      if (g.jmul) {
        if (row < g.m)
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (b0 + q < g.B)
              g.out[((long long)kc * g.B + b0 + q) * g.m + row] = __uint_as_float(r[q]);
      } else if (row < g.n) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (b0 + q < g.B) g.out[(long long)(b0 + q) * g.out_bs + row] = g.scale * __uint_as_float(r[q]);
      }
    }
  }
  __syncwarp();
  bool fin = true;
  if (warp == 1) {
    fin = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done), 0));
    if (!fin && lane == 0) atomicOr(g.err, kErrEpilogue);
  }
  tc_fence_before();
  const int drained = __syncthreads_and(fin ? 1 : 0);
  if (warp == 1 && drained) {  // TMEM is freed only once the last commit showed the MMAs done
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u)
                 : "memory");
  }
}

// x [B][n] (batch stride x_bs) -> hi (and lo) BF16 rows [b][n8]; a thread per element.
__global__ void jp_stage_x_kernel(const float* __restrict__ x, long long x_bs, int B, int n, int n8,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)B * n) return;
  const long long b = e / n, j = e % n;
  const float v = x[b * x_bs + j];
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[b * n8 + j] = h;
  if (lo) lo[b * n8 + j] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// r[e] = sum over the chunks (in order) of part[c][e] - dv[e], e = b m + i; and r's BF16
// staging (hi, lo) at the same index.  A thread per element.
__global__ void jp_final_kernel(const float* __restrict__ part, const float* __restrict__ dv,
                                float* __restrict__ r, long long N, int nk,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  float s = 0.f;
  for (int c = 0; c < nk; ++c) s += part[(long long)c * N + e];
  s -= dv[e];
  r[e] = s;
  const __nv_bfloat16 h = __float2bfloat16_rn(s);
  hi[e] = h;
  if (lo) lo[e] = __float2bfloat16_rn(s - __bfloat162float(h));
}

cudaError_t encode_2d(CUtensorMap* m, const void* base, int inner, int rows, long long pitch,
                      int box_inner, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t jp_smem(bool split) { return (size_t)kJpStages * (split ? 2 : 1) * (kJpA + kJpB) + 1024; }

cudaError_t jp_prepare() {
  static int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || done_dev == dev) return e;
  e = cudaFuncSetAttribute(jprod_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)jp_smem(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jprod_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)jp_smem(true));
  if (e == cudaSuccess) done_dev = dev;
  return e;
}

cudaError_t jp_launch(const JprodTc& J, const CUtensorMap* A, const CUtensorMap* Bm, JpArgs a,
                      cudaStream_t st) {
  cudaError_t e = jp_prepare();
  if (e != cudaSuccess) return e;
  const int nb = J.B16 / 16;
  const int grid = (int)std::max<long long>(1, std::min<long long>(a.items, ceil_div(sm_count(), nb)));
  dim3 gd((unsigned)grid, (unsigned)nb);
  if (J.split)
    jprod_tc_kernel<true><<<gd, kJpThreads, jp_smem(true), st>>>(A[0], A[1], Bm[0], Bm[1], a);
  else
    jprod_tc_kernel<false><<<gd, kJpThreads, jp_smem(false), st>>>(A[0], A[0], Bm[0], Bm[0], a);
  return cudaGetLastError();
}

}  // namespace

bool jprod_tc_supported(int m, int n) { return m > 0 && n > 0 && m % 8 == 0; }

int jprod_tc_chunks(int m, int n) {
  const int mtiles = (int)ceil_div(m, 128), kblocks = (int)ceil_div(n, 64);
  const int want = std::max(1, std::min(kblocks, (int)ceil_div(2 * sm_count(), mtiles)));
  const int kper = (int)ceil_div(kblocks, want);
  return (int)ceil_div(kblocks, kper);
}

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

size_t jprod_tc_staging_bytes(int m, int n, int B, bool split) {
  const size_t B16 = (size_t)ceil_div(B, 16) * 16, n8 = (size_t)ceil_div(n, 8) * 8;
  const int parts = split ? 2 : 1;
  return parts * (round256(B16 * n8 * 2) + round256(B16 * (size_t)m * 2));
}

cudaError_t jprod_tc_init(JprodTc& J, const __nv_bfloat16* Jt, const __nv_bfloat16* Jlo,
                          void* staging, int m, int n, int B, cudaStream_t st) {
  if (!jprod_tc_supported(m, n) || B <= 0) return cudaErrorInvalidValue;
  J = JprodTc{};
  J.m = m, J.n = n, J.B = B;
  J.B16 = (int)ceil_div(B, 16) * 16;
  J.n8 = (int)ceil_div(n, 8) * 8;
  J.split = Jlo != nullptr;
  const int mtiles = (int)ceil_div(m, 128), kblocks = (int)ceil_div(n, 64);
  J.nk = jprod_tc_chunks(m, n);
  J.kper = (int)ceil_div(kblocks, J.nk);
  (void)mtiles;
  char* p = static_cast<char*>(staging);
  const int parts = J.split ? 2 : 1;
  for (int h = 0; h < parts; ++h) {
    J.xs[h] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round256((size_t)J.B16 * J.n8 * 2);
    J.rs[h] = reinterpret_cast<__nv_bfloat16*>(p);
    p += round256((size_t)J.B16 * m * 2);
  }
  cudaError_t e = cudaMemsetAsync(staging, 0, jprod_tc_staging_bytes(m, n, B, J.split), st);
  for (int h = 0; h < parts && e == cudaSuccess; ++h) {
    const __nv_bfloat16* src = h ? Jlo : Jt;
    e = encode_2d(&J.jm[h], src, m, n, m, 64, 64);
    if (e == cudaSuccess) e = encode_2d(&J.jt[h], src, m, n, m, 64, 128);
    if (e == cudaSuccess) e = encode_2d(&J.xm[h], J.xs[h], n, J.B16, J.n8, 64, 16);
    if (e == cudaSuccess) e = encode_2d(&J.rm[h], J.rs[h], m, J.B16, m, 64, 16);
  }
  if (!J.split) J.jm[1] = J.jm[0], J.jt[1] = J.jt[0], J.xm[1] = J.xm[0], J.rm[1] = J.rm[0];
  return e;
}

cudaError_t jprod_tc_residual(const JprodTc& J, const float* x, long long x_bs, const float* dv,
                              float* r, float* part, int* err, cudaStream_t st) {
  const long long nx = (long long)J.B * J.n;
  jp_stage_x_kernel<<<(unsigned)ceil_div(nx, 256), 256, 0, st>>>(x, x_bs, J.B, J.n, J.n8, J.xs[0],
                                                                 J.split ? J.xs[1] : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  JpArgs a{};
  a.m = J.m, a.n = J.n, a.B = J.B;
  a.mtiles = (int)ceil_div(J.m, 128);
  a.kblocks = (int)ceil_div(J.n, 64);
  a.kper = J.kper;
  a.items = a.mtiles * J.nk;
  a.jmul = 1, a.out = part, a.out_bs = 0, a.scale = 1.f, a.err = err;
  e = jp_launch(J, J.jm, J.xm, a, st);
  if (e != cudaSuccess) return e;
  const long long N = (long long)J.B * J.m;
  jp_final_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(part, dv, r, N, J.nk, J.rs[0],
                                                              J.split ? J.rs[1] : nullptr);
  return cudaGetLastError();
}

cudaError_t jprod_tc_adjoint(const JprodTc& J, float* g, float scale, long long g_bs, int* err,
                             cudaStream_t st) {
  JpArgs a{};
  a.m = J.m, a.n = J.n, a.B = J.B;
  a.mtiles = (int)ceil_div(J.n, 128);
  a.kblocks = (int)ceil_div(J.m, 64);
  a.kper = a.kblocks;
  a.items = a.mtiles;
  a.jmul = 0, a.out = g, a.out_bs = g_bs, a.scale = scale, a.err = err;
  return jp_launch(J, J.jt, J.rm, a, st);
}

}  // namespace d2ip
