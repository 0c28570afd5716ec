// The paper-form 3D-FastResUNet variant (Sec. III-D): its kernels (fastres_ops.cu) and the
// node list that runs its forward and backward passes (fastres.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace d2ip {

constexpr int kActLeaky = 0, kActRelu = 1, kActSigmoid = 2;

// ---- kernels (all asynchronous on the stream; [B][voxels][C] tensors) ----------------------
// Pointwise 1x1x1 convolution ci -> co, stride s (1 or 2), weights W[co][ci] then b[co] per
// problem at w_bs.  The weight gradient writes partial rows [B][rows][co*ci + co].
bool pw_supported(int ci, int co);
cudaError_t pw_fwd_f32(const float* x, const float* W, float* y, int B, Dims3 din, int ci,
                       int co, int s, long long w_bs, int acc, cudaStream_t st);
cudaError_t pw_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din, int ci,
                         int co, int s, long long w_bs, int acc, cudaStream_t st);
long long pw_wgrad_rows(Dims3 din, int s);
cudaError_t pw_wgrad_partial_f32(const float* x, const float* dy, float* part, int B, Dims3 din,
                                 int ci, int co, int s, cudaStream_t st);
// Depthwise 3x3x3 convolution of C channels, stride s, dilation d (zero padding d), weights
// W[c][27] then b[c]; weight-gradient partial rows [B][rows][28 C].
cudaError_t dw_fwd_f32(const float* x, const float* W, float* y, int B, Dims3 din, int C, int s,
                       int d, long long w_bs, cudaStream_t st);
cudaError_t dw_dgrad_f32(const float* dy, const float* W, float* dx, int B, Dims3 din, int C,
                         int s, int d, long long w_bs, int acc, cudaStream_t st);
long long dw_wgrad_rows(Dims3 din, int s);
cudaError_t dw_wgrad_partial_f32(const float* x, const float* dy, float* part, int B, Dims3 din,
                                 int C, int s, int d, cudaStream_t st);
// Elementwise activation (kAct*) and its derivative taken from the output.
cudaError_t act_fwd_f32(const float* x, float* y, long long n, int kind, cudaStream_t st);
cudaError_t act_bwd_f32(const float* y, const float* dy, float* dx, long long n, int kind,
                        int acc, cudaStream_t st);
cudaError_t add2_f32(const float* a, const float* b, float* y, long long n, cudaStream_t st);
cudaError_t accum_f32(float* dst, const float* src, long long n, int acc, cudaStream_t st);
// part[B][rows][C] = scale * per-chunk sums over voxels of x (times y when y is given).
long long vox_sum_rows(long long nvox);
cudaError_t vox_sum_partial_f32(const float* x, const float* y, float* part, int B,
                                long long nvox, int C, float scale, cudaStream_t st);
cudaError_t bcast_f32(const float* x, float* y, int B, long long nvox, int C, float scale,
                      int acc, cudaStream_t st);
cudaError_t cscale_f32(const float* x, const float* s, float* y, int B, long long nvox, int C,
                       int acc, cudaStream_t st);
cudaError_t vscale_f32(const float* x, const float* psi, float* y, long long nvox_all, int C,
                       int acc, cudaStream_t st);
cudaError_t vdot_f32(const float* dy, const float* x, float* dpsi, long long nvox_all, int C,
                     int acc, cudaStream_t st);
cudaError_t slice_f32(const float* src, int src_C, int src_off, float* dst, int dst_C,
                      int dst_off, int width, long long nvox_all, int acc, cudaStream_t st);

// ---- the network as a node list ----------------------------------------------------------
struct FrVal {  // one activation [B][voxels of level lvl][C] and its gradient
  int lvl = 0, C = 0;
  bool grad = true;
  float* v = nullptr;
  float* g = nullptr;
};

enum FrKind {
  kFrConv3,   // dense 3x3x3, stride 1 (the stem)
  kFrPw,      // pointwise 1x1x1, stride s
  kFrDw,      // depthwise 3x3x3, stride s, dilation d
  kFrLn,      // LayerNorm (+ residual) + LeakyReLU
  kFrAct,     // elementwise activation
  kFrAdd,     // out = in0 + in1
  kFrPool,    // out[c] = mean over voxels of in0
  kFrBcast,   // out[q][c] = in0[c]
  kFrCscale,  // out[q][c] = in0[q][c] * in1[c]
  kFrVscale,  // out[q][c] = in0[q][c] * in1[q]
  kFrUp,      // trilinear up-sampling of in0 to out's level
  kFrUpcat,   // out = [Up(in0), in1]
  kFrSlice,   // out[:, off : off + C(in0)] = in0
};

struct FrNode {
  int kind = 0, in0 = -1, in1 = -1, out = -1;
  int ci = 0, co = 0, s = 1, d = 1, act = 0, resid = -1, off = 0;
  long long w_off = -1;                      // weights (bias follows) or LN gamma (beta follows)
  float *xh = nullptr, *rs = nullptr;        // LayerNorm caches
  bool acc0 = false, acc1 = false, accr = false;  // backward: add into in0 / in1 / resid grads
};

struct FrRun {
  const float* theta;
  float* grad;
  long long Pp;
  cudaStream_t stream;
  void (*beg)(void*, int, double) = nullptr;  // optional per-launch tracing
  void (*fin)(void*) = nullptr;
  void* user = nullptr;
};

struct FastNet {
  std::vector<Dims3> dims;  // levels 0..L, then the one-voxel level of pooled vectors
  std::vector<FrVal> vals;  // vals[0] = Z
  std::vector<FrNode> nodes;
  int B = 1;
  long long ws_floats = 0, tmp_floats = 0;
  float *ws = nullptr, *tmp = nullptr, *tmp2 = nullptr;

  // Builds the node list and appends the parameter table rows {kind, offset, count, fan_in}.
  void build(Dims3 grid, int L, const std::vector<int>& w, int c_in,
             std::vector<long long>& table, long long& P);
  long long arena_floats(int batch) const;
  // Binds the buffers inside `base` (arena_floats floats); the output is written to dsigma
  // and its gradient read from gds.
  void bind(float* base, int batch, float* zin, float* dsigma, float* gds);
  cudaError_t forward(const FrRun& r) const;
  cudaError_t backward(const FrRun& r) const;
};

// widths multiples of 8 up to 128 (gate inner widths w/2 and ASPP branches pass the 4-channel
// vector paths), c_in 1..256
bool fastres_supported(int L, const int* w, int c_in);

}  // namespace d2ip
