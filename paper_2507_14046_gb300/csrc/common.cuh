// Shared definitions for the D²IP CUDA library (device side and launchers).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <climits>
#include <cstdint>

namespace d2ip {

struct Dims3 {
  int z, y, x;
  __host__ __device__ long long count() const { return (long long)z * y * x; }
};

// Output size of a K^3 convolution, stride S, zero padding (K-1)/2: ceil(D/S) for K = 3.
__host__ __device__ inline Dims3 conv_out_dims(Dims3 in, int K, int S) {
  const int p = (K - 1) / 2;
  return Dims3{(in.z + 2 * p - K) / S + 1, (in.y + 2 * p - K) / S + 1,
               (in.x + 2 * p - K) / S + 1};
}

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Store four consecutive channels c..c+3 (c % 4 == 0) of one voxel into its BF16 staging
// row (`row` = the voxel's first staged element, C channels per block).  sp 1: bf16(v).
// sp 3: the split form of the BF16x3 precision, three C-channel blocks [hi | lo | hi] with
// hi = bf16(v) and lo = bf16(v - hi) (v - hi is exact in FP32), so hi + lo holds 16
// significant bits; a convolution whose weights are staged [hi | hi | lo] over the same
// channel blocks then sums x_hi w_hi + x_lo w_hi + x_hi w_lo in one K loop.
__device__ __forceinline__ void stage_bf16x4(__nv_bfloat16* row, int C, int c, float4 v,
                                             int sp) {
  const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
  uint2 hu;
  hu.x = *reinterpret_cast<const uint32_t*>(&h01);
  hu.y = *reinterpret_cast<const uint32_t*>(&h23);
  *reinterpret_cast<uint2*>(row + c) = hu;
  if (sp == 1) return;
  const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
  const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y),
                       l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
  uint2 lu;
  lu.x = *reinterpret_cast<const uint32_t*>(&l01);
  lu.y = *reinterpret_cast<const uint32_t*>(&l23);
  *reinterpret_cast<uint2*>(row + C + c) = lu;
  *reinterpret_cast<uint2*>(row + 2 * C + c) = hu;
}

constexpr float kLeakySlope = 0.2f;
constexpr float kLnEps = 1e-5f;

// ---------------------------------------------------------------------------------
// Launchers (all asynchronous on `stream`, all capturable in a CUDA graph).
// Tensors are channels-last: element (voxel q, channel c) at q*C + c, voxel
// q = (z*Y + y)*X + x.  `*_bs` are batch strides in elements.  Return cudaError_t of
// the launch.
// ---------------------------------------------------------------------------------

// y = conv(x, W) + b.  W is [Co][K^3][Ci] (tap-major, channel fastest).
cudaError_t conv3d_fwd_f32(const float* x, const float* W, const float* bias, float* y,
                           int B, Dims3 din, int Ci, int Co, int K, int S,
                           long long x_bs, long long y_bs, long long w_bs,
                           cudaStream_t stream);
// dx (=|+=) conv^T(dy, W).
cudaError_t conv3d_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din,
                             int Ci, int Co, int K, int S, long long dy_bs, long long dx_bs,
                             long long w_bs, int accumulate, cudaStream_t stream);
// Per-chunk partial weight gradients: part[b][chunk][Co*K^3*Ci + Co] (W part then bias).
long long conv3d_wgrad_chunks(Dims3 din, int K, int S);
cudaError_t conv3d_wgrad_partial_f32(const float* x, const float* dy, float* part, int B,
                                     Dims3 din, int Ci, int Co, int K, int S,
                                     long long x_bs, long long dy_bs, cudaStream_t stream);
// out[b*out_bs + j] (=|+=) sum_r part[(b*R + r)*N + j]
cudaError_t reduce_rows_f32(const float* part, float* out, int B, long long R, long long N,
                            long long out_bs, int accumulate, cudaStream_t stream);

// LayerNorm over channels (+ residual) (+ LeakyReLU).
int layernorm_bwd_blocks(long long nvox, int C);
// ybf (optional): a BF16 copy of y (the next tensor-core convolution's staged input), in sp
// blocks per voxel (stage_bf16x4).
cudaError_t layernorm_act_fwd_f32(const float* z, const float* gamma, const float* resid,
                                  float* y, float* xhat, float* rstd, int B, long long nvox,
                                  int C, int act, long long g_bs, cudaStream_t stream,
                                  __nv_bfloat16* ybf = nullptr, int sp = 1);
// part: [B][blocks][2C] partial (dgamma, dbeta); dzbf, dtbf (optional): BF16 copies of dz, dt
// in sp blocks per voxel.
cudaError_t layernorm_act_bwd_f32(const float* dy, const float* act_out, const float* xhat,
                                  const float* rstd, const float* gamma, float* dz, float* dt,
                                  float* part, int B, long long nvox, int C, long long g_bs,
                                  cudaStream_t stream, __nv_bfloat16* dzbf = nullptr,
                                  __nv_bfloat16* dtbf = nullptr, int sp = 1);

// cat[:, :Cu] = trilinear(low -> dout), cat[:, Cu:] = skip; catbf (optional): a BF16 copy in
// sp blocks per voxel.  cat may be null when catbf is set (only the BF16 copy is written).
cudaError_t upsample_concat_fwd_f32(const float* low, const float* skip, float* cat, int B,
                                    Dims3 dlow, Dims3 dout, int Cu, int Cs,
                                    cudaStream_t stream, __nv_bfloat16* catbf = nullptr,
                                    int sp = 1);
// dlow = adjoint of the upsample applied to dcat[:, :Cu]; dskip = dcat[:, Cu:].
cudaError_t upsample_concat_bwd_f32(const float* dcat, float* dlow, float* dskip, int B,
                                    Dims3 dlow_dims, Dims3 dout, int Cu, int Cs,
                                    cudaStream_t stream);
cudaError_t add_inplace_f32(float* y, const float* x, long long count, cudaStream_t stream);

// Data term.  r[b] = J x[b] - dv[b];  g[b] = scale * J^T r[b];  loss in FP64.
// part: workspace of jmul_chunks(n) * B * m floats (deterministic column-chunk partials).
int jmul_chunks(int n);
cudaError_t jmul_residual_f32(const float* J, const float* x, const float* dv, float* r,
                              float* part, int B, int m, int n, long long x_bs,
                              cudaStream_t stream);
// The same products reading a BF16 copy of J (FP32 accumulation); with Jlo, J is the sum of
// two BF16 copies hi + lo (the split form, 16 significant bits) added in FP32.
cudaError_t jmul_residual_bf16(const __nv_bfloat16* J, const float* x, const float* dv, float* r,
                               float* part, int B, int m, int n, long long x_bs,
                               cudaStream_t stream, const __nv_bfloat16* Jlo = nullptr);
cudaError_t jtmul_bf16(const __nv_bfloat16* J, const float* r, float* g, float scale, int B,
                       int m, int n, long long g_bs, cudaStream_t stream,
                       const __nv_bfloat16* Jlo = nullptr);
cudaError_t convert_bf16(const float* x, __nv_bfloat16* y, long long n, cudaStream_t stream);
// The BF16 forms of the J products take J transposed: Jt[n][m] (BF16), m a multiple of 4;
// Jlo (optional) receives bf16(J - Jt) transposed.
cudaError_t transpose_bf16(const float* J, __nv_bfloat16* Jt, int m, int n, cudaStream_t stream,
                           __nv_bfloat16* Jlo = nullptr);
// Per-device kernel attributes (opt-in shared memory); call once per device before launches.
cudaError_t prepare_pointwise_kernels();
cudaError_t jtmul_f32(const float* J, const float* r, float* g, float scale, int B, int m,
                      int n, long long g_bs, cudaStream_t stream);
// loss[b] = (1/m) sum r^2 (FP64); optional trace ring (slot trace_pos % trace_cap, then
// trace_pos += 1); optional Adam step counter bump; status bit 1 set when a loss is not
// finite.
// reg_part (optional): [B][reg_blocks] regulariser partial sums added to each loss.
cudaError_t residual_loss_f64(const float* r, double* loss, double* trace, int* trace_pos,
                              int trace_cap, int* adam_t, int* status, int B, int m,
                              cudaStream_t stream, const double* reg_part = nullptr,
                              int reg_blocks = 0);
// 4D-TV value (per-block FP64 partials [B][tv4d_blocks]) and gradient added into g; hist holds
// the previous outputs [B][frames][n] (batch stride hist_bs), *nprev_dev of them in use.
int tv4d_blocks(long long n);
cudaError_t set_device_int(int* p, int v, cudaStream_t stream);  // graph-capturable store
cudaError_t tv4d_f32(const float* ds, const float* hist, const int* nprev_dev, float* g,
                     double* part, int B, Dims3 d, long long hist_bs, float lam_s, float lam_t,
                     float eps, cudaStream_t stream);
cudaError_t normalize_columns_f64(float* J, double* colnorm, int m, int n,
                                  cudaStream_t stream);
cudaError_t err_ratio_f64(const float* est, const float* truth, double* out, int B,
                          long long n, cudaStream_t stream);

// Adam over a flat arena; the step count t is read from device memory (after the bump
// done by residual_loss_f64), or taken from `t_host` when t_dev is null.
cudaError_t adam_step_f32(float* theta, const float* g, float* m, float* v, long long count,
                          double lr, double beta1, double beta2, double eps, const int* t_dev,
                          int t_host, cudaStream_t stream);


// 1x1x1 convolution to one output channel (C input channels, weights [C] then bias, per
// problem at w_bs): y = b + w . h, and its backward dh (=|+=) w g with per-block weight
// partials part[b][blk][C + 1] (conv1x1_co1_blocks rows; add them with reduce_rows_f32).
bool conv1x1_co1_supported(int C);
long long conv1x1_co1_blocks(long long nvox);
cudaError_t conv1x1_co1_fwd_f32(const float* h, const float* wb, float* y, int B, long long nvox,
                                int C, long long w_bs, cudaStream_t stream);
cudaError_t conv1x1_co1_bwd_f32(const float* h, const float* g, const float* wb, float* dh,
                                float* part, int B, long long nvox, int C, long long w_bs,
                                int accumulate, cudaStream_t stream);

}  // namespace d2ip
