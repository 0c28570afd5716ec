// The sensitivity products of the data term (Eq. 4) on the tensor cores, for a group of B
// problems that share one normalised J (m measurements x n voxels):
//   r[b] = J x[b] - dv[b]        (the residual; x = the network output Delta sigma)
//   g[b] = scale J^T r[b]        (the adjoint, scale = 2 / m)
// as GEMMs with the problems in N (16 per MMA; more problems take more blocks of 16).  J is
// read from its transposed BF16 copy Jt [n][m] (and the BF16 remainder Jlo in the split
// precision): for J x the A operand is J itself, MN-major in Jt's rows; for J^T r it is Jt,
// K-major.  x and r are staged as BF16 (hi, and lo = bf16(v - hi) in the split precision,
// whose products hi hi + lo hi + hi lo accumulate in one FP32 accumulator in tensor memory).
// J x runs split-K over the voxels with fixed-order partial sums, so results are
// deterministic.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace d2ip {

struct JprodTc {
  int m = 0, n = 0, B = 0;
  int B16 = 0;            // problems rounded up to blocks of 16 (staging rows; extra rows zero)
  int n8 = 0;             // staged row length of x (n rounded up to 8: 16-byte TMA rows)
  bool split = false;     // hi + lo operands
  int nk = 0, kper = 0;   // J x: K chunks (of kper 64-voxel blocks) per 128-measurement tile
  __nv_bfloat16* xs[2] = {nullptr, nullptr};  // x staging hi, lo [B16][n8]
  __nv_bfloat16* rs[2] = {nullptr, nullptr};  // r staging hi, lo [B16][m]
  CUtensorMap jm[2];      // Jt (hi, lo) in 64 x 64 boxes: the MN-major A operand of J x
  CUtensorMap jt[2];      // Jt (hi, lo) in 128-row x 64 boxes: the K-major A operand of J^T r
  CUtensorMap xm[2], rm[2];  // the staged x and r in 16-row x 64 boxes (B operands)
};

// Whether the tensor-core form takes this J (m a multiple of 8, so Jt's rows are 16-byte
// aligned for TMA).
bool jprod_tc_supported(int m, int n);
// Bytes of device staging jprod_tc_init carves (x and r, hi and lo when split).
size_t jprod_tc_staging_bytes(int m, int n, int B, bool split);
// Sets J up over Jt (and Jlo when split) and `staging` (jprod_tc_staging_bytes, device,
// 256-byte aligned, zeroed here on `st`).  Jt / Jlo / staging must outlive J.
cudaError_t jprod_tc_init(JprodTc& J, const __nv_bfloat16* Jt, const __nv_bfloat16* Jlo,
                          void* staging, int m, int n, int B, cudaStream_t st);
// Partial sums of J x go to part (J.nk * B * m floats), then r = sum - dv (FP32 [B][m]) and
// r's staging; x [B][n] at batch stride x_bs.  err: the device error word (bounded waits).
cudaError_t jprod_tc_residual(const JprodTc& J, const float* x, long long x_bs, const float* dv,
                              float* r, float* part, int* err, cudaStream_t st);
// g[b] = scale J^T r[b] (g at batch stride g_bs), from r's staging written by the residual.
cudaError_t jprod_tc_adjoint(const JprodTc& J, float* g, float scale, long long g_bs, int* err,
                             cudaStream_t st);
// J x chunks of this setup (the part buffer holds nk * B * m floats).
int jprod_tc_chunks(int m, int n);

}  // namespace d2ip
