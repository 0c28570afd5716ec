// Tensor-core path of the 3D convolutions: implicit GEMM on tcgen05 (BF16 x BF16 -> FP32 in
// TMEM), operands staged by TMA.
#pragma once

#include <cuda.h>

#include <cstddef>
#include <vector>

#include "common.cuh"

namespace d2ip {

// One convolution served by the tensor cores, with its TMA descriptors.
struct TcLayer {
  CUtensorMap act_f;  // forward input (BF16 staging buffer, this layer's dims and channels)
  CUtensorMap w_f;    // forward weights [B][Co][T][Ci] (BF16)
  CUtensorMap act_d;  // stride-1 data-gradient input (dy staged in BF16)
  CUtensorMap w_d;    // data-gradient weights [B][Ci][T][Co], taps reversed (BF16)
  CUtensorMap act_f3, w_f3, act_d3, w_d3;  // halo-box forms (3x3x3 stride 1)
  // Weight-gradient operands in the box form of the kernel that runs the layer (halo box:
  // dy 8 x 3 x tz+2, x 8 x 1 x tz; stride 2: x strided tile, dy tile; per tap: dy and x
  // tiles) for the hi (index 0) and lo (index 1, split precision only) channel blocks of the
  // staged dy and x, and a fused projection's dz_p column.
  CUtensorMap wgy[2], wgx[2], wgp[2];
  CUtensorMap wgqy, wgqx, wgqp;  // split precision in one pass: dy, x (and a fused
                                 // projection's dz_p) as [hi | lo] rows
  int ci = 0, co = 0, k = 3, s = 1;
  // The halo-form (persistent kernel) view of the forward and data gradient: K channels and
  // MMA width N.  Normally kf, co and kd, ci; with hlf / hld (split precision, a 16 -> 16
  // layer) the kernel reads the first two blocks [hi | lo] of each staged row (K = 2 ci)
  // against weights doubled in N ([w_hi; w_lo] rows, N = 2 co) and its epilogue adds the two
  // column halves: x_hi w_hi + x_lo w_hi + x_hi w_lo + x_lo w_lo.
  int kf3 = 0, nf3 = 0, kd3 = 0, nd3 = 0;
  bool hlf = false, hld = false;
  int kf = 0, kd = 0;             // K channels of the forward and data-gradient operands:
                                  // ci and co times the operand blocks (Bf16Net::sp)
  Dims3 din{}, dout{};
  long long w_off = 0;            // weights of this conv in the FP32 theta arena
  long long wf_off = 0, wd_off = 0;  // offsets in the per-problem BF16 weight block
  bool dgrad = false;             // data gradient on the tensor cores too (stride 1)
  bool wgrad = false;             // weight gradient on the tensor cores too (3x3x3)
  int ck3f = 0, ck3d = 0;         // channel chunk of the halo-box kernel (0: per-tap kernel)
  int tz3f = 1, tz3d = 1;         // z slices per halo-box tile
  bool per3f = false, per3d = false;    // halo forward / data gradient by the persistent kernel
  float tune_f = -1.f, tune_d = -1.f;   // autotuner: time of the chosen tiles (us), or -1
  float model_f = -1.f, model_d = -1.f; // ... of the cost model's tiles
  bool pack3f = false, pack3d = false;  // halo forward / data gradient with the kz taps packed
                                        // into N: that direction's weights are stored with ky
                                        // and kz swapped (tap (kz, ky, kx) at (ky, kz, kx))
  int proj = -1;                  // layer index of a 1x1 projection of the same input, fused
  bool projf = false, projd = false, projw = false;  // ... into forward / dgrad / wgrad
  CUtensorMap pw_f, pw_d, pa_d;   // projection: W_p, W_p^T and the dz_p tile box
  bool wg3 = false;               // weight gradient by the halo-box kernel
  int wg_tz = 0;                  // its column depth (z voxels per K tile)
  bool wgs2 = false;              // stride-2 weight gradient on the tensor cores
  bool s2p = false;               // stride-2 data gradient with its 8 parity classes packed
                                  // in N (one CTA per tile; weights as 8 x 8 window-class
                                  // blocks, 37 of them zero)
  __nv_bfloat16* xin = nullptr;   // BF16 copy of the forward input (kept for the weight gradient)
  int ci_real = 0;                // input channels of the model (ci is padded up to 16)
  bool input_layer = false;       // reads the padded BF16 copy of the network input (zbf)
  int dyslot = 0;                 // BF16 staging buffer of this layer's dy: 0 ybf, 1 ybf2
  int xin_of = -1;                // a projection run on its own: the layer whose kept BF16
                                  // input (the same tensor, the same layout) it reads
};

// Device buffers of the BF16 path (carved from the context arena) and its layers.
struct Bf16Net {
  __nv_bfloat16* xbf = nullptr;   // BF16 staging of one convolution input (or dy)
  __nv_bfloat16* ybf = nullptr;   // BF16 staging of dy for the weight gradient
  __nv_bfloat16* ybf2 = nullptr;  // a second dy staging buffer (layers with dyslot 1), so a
                                  // data gradient can stage the next layer's dy while it reads
  __nv_bfloat16* pbf = nullptr;   // BF16 staging of a fused projection's dy
  __nv_bfloat16* wbuf = nullptr;  // BF16 weights of every tensor-core layer, per problem
  __nv_bfloat16* zbf = nullptr;   // network input, BF16, channels padded to 16 (input layer)
  long long zcount = 0;           // elements per problem of zbf
  long long wstride = 0;          // elements per problem in wbuf
  long long max_act = 0;          // elements per problem of the largest staged input
  int* err = nullptr;             // device error word (bounded waits that ran out)
  bool keep_inputs = false;       // a BF16 input copy per layer (else all share xbf)
  // Operand blocks per staged value: 1 for BF16; 3 for the split BF16x3 precision, where a
  // staged activation or gradient holds [hi | lo | hi] and the weights [hi | hi | lo] (each a
  // block of the channel count), so the forward and data-gradient K loops add up
  // x_hi w_hi + x_lo w_hi + x_hi w_lo, and the weight gradient runs three passes over the
  // (dy, x) block pairs (hi, hi), (lo, hi), (hi, lo).
  int sp = 1;
  std::vector<TcLayer> layers;
};

bool bf16_network_supported(int levels, const int* widths, int c_in);
bool bf16_conv_supported(int ci, int co, int k);
// Register a convolution; returns its index in bf.layers or -1 when it stays on FP32 SIMT.
int bf16_add_layer(Bf16Net& bf, int ci, int co, int k, int s, Dims3 din, long long w_off);
// Register the first convolution, whose input (ci_real <= 16 channels) is fixed per problem:
// it reads a BF16 copy padded to 16 channels, staged once by bf16_stage_input, and has no
// data gradient.  Returns -1 when the halo-box kernels do not fit it.
int bf16_add_input_layer(Bf16Net& bf, int ci_real, int co, Dims3 din, long long w_off);
// z [B][n][ci_real] FP32 -> zbf [B][n][16] BF16 (zero channels ci_real..15).
cudaError_t bf16_stage_input(Bf16Net& bf, int layer, const float* z, int B, cudaStream_t stream);
// Fuse the 1x1 projection lp (same input, same output channels) into the 3x3x3 stride-1
// layer la: its forward and data gradient then run in la's halo-box launches.  Returns
// whether the forward (bit 0), the data gradient (bit 1) and the weight gradient (bit 2)
// were fused.  A forward left unfused (la's folded split form) reads la's kept BF16 input.
int bf16_fuse_proj(Bf16Net& bf, int la, int lp);
// Whether the layer reads another layer's kept BF16 input: once that layer's forward ran,
// this one's input is staged.
bool bf16_input_shared(const Bf16Net& bf, int layer);
// y_a = conv_a(x) + bias_a and y_p = W_p x + bias_p in one launch (layer la with projf).
cudaError_t bf16_conv_fwd_proj(Bf16Net& bf, int la, const float* x, const float* bias_a,
                               float* y_a, const float* bias_p, float* y_p, int B,
                               long long bias_bs, cudaStream_t stream, bool x_staged = false);
// dx = conv_a^T(dz_a) + W_p^T dz_p in one launch (layer la with projd); dz_a is staged into
// bf.ybf and dz_p into bf.pbf unless their producer already wrote them there.
// With dx2 and split_c > 0, dx is stored as two tensors: channels [0, split_c) into dx
// ([B][voxels][split_c]) and the rest into dx2 ([B][voxels][ci - split_c]).
cudaError_t bf16_conv_dgrad_proj(Bf16Net& bf, int la, const float* dz_a, const float* dz_p,
                                 float* dx, int B, cudaStream_t stream, bool dza_staged = false,
                                 bool dzp_staged = false, float* dx2 = nullptr, int split_c = 0);
// Reserve the BF16 buffers in the arena (base == nullptr: size only).
void bf16_layout(Bf16Net& bf, char* base, size_t& used, int B, long long max_act);
// Encode the TMA descriptors once the buffers have addresses.
cudaError_t bf16_finalize(Bf16Net& bf, int B);
// Autotuner of the persistent halo convolutions: for every layer and direction that runs the
// persistent kernel, each candidate tiling (kz packing, z depth, channel chunk) is timed with
// CUDA events on the network's own buffers (2 warm-up + 5 timed launches, outputs to
// scratch, bias_f any B-shared FP32 bias) and the fastest kept, with its time and the cost
// model's choice's time in the layer.  Choices are cached per shape for the process, so every
// context of one shape uses the same tiles (and FP32 summation order).  Synchronous on st;
// call after bf16_finalize, before any capture.
cudaError_t bf16_autotune(Bf16Net& bf, int B, float* scratch, const float* bias_f,
                          cudaStream_t st);
// Sets the persistent halo tilings from rows laid out as d2ip_tile_plan writes them (one
// per layer; the shape columns must match the layer), re-encoding the affected descriptors.
// cudaErrorInvalidValue when a row does not fit the network or names a tiling that cannot run.
cudaError_t bf16_apply_plan(Bf16Net& bf, int B, const long long* rows, int n_rows);
// FP32 elements bf16_autotune's scratch needs.
long long bf16_tune_scratch_floats(const Bf16Net& bf, int B);
cudaError_t bf16_prepare_kernels();
// theta (FP32, [B][Pp]) -> BF16 forward and data-gradient weights of every layer.
cudaError_t bf16_prepare_weights(Bf16Net& bf, const float* theta, int B, long long Pp,
                                 cudaStream_t stream);
// The layer's kept BF16 input copy, when a producer may write it directly (keep_inputs);
// else nullptr.
__nv_bfloat16* bf16_input_buffer(const Bf16Net& bf, int layer);
// y = conv(x) + bias on the tensor cores (x FP32 is staged to BF16 first unless x_staged:
// its producer already wrote bf16_input_buffer).
cudaError_t bf16_conv_fwd(Bf16Net& bf, int layer, const float* x, const float* bias, float* y,
                          int B, long long bias_bs, cudaStream_t stream, bool x_staged = false);
// LayerNorm (+ residual) (+ LeakyReLU) of a convolution's output, fused into the epilogue of
// the persistent halo convolution: y = act(gamma * xhat + beta (+ resid)), xhat = (z - mean)
// rstd over the co channels of each voxel, z = conv(x) + bias (not stored).  xhat and y are
// [B][voxels][co] FP32, rstd [B][voxels]; ybf (or null) receives the BF16 copy of y in sp
// blocks per voxel (stage_bf16x4's layout), the next tensor-core layer's staged input.
struct Bf16Ln {
  const float* gamma;  // gamma[c] then beta[c], per problem at gamma_bs
  long long gamma_bs;
  const float* resid;  // [B][voxels][co] (batch stride voxels * co) or null
  float* xhat;
  float* rstd;
  __nv_bfloat16* ybf;
  int act;             // 1: LeakyReLU
  int sp;              // set by the call: BF16 blocks of ybf (Bf16Net::sp)
  // Backward form (bf16_conv_dgrad_ln): xhat and rstd are the saved inputs, resid (or null)
  // a gradient already accumulated for the data gradient's output, ybf the staging of dz.
  int bwd = 0;
  const float* aout = nullptr;  // the block output a = act(LN(z) ...) [B][voxels][C]
  float* part = nullptr;        // [B][bf16_dgrad_ln_rows][2 C]: dgamma, dbeta partial sums
};
// Whether layer's forward (with a fused projection of np channels when np > 0) runs the
// persistent halo kernel with room for the LayerNorm epilogue (co <= 64).
bool bf16_fwd_ln_ok(const Bf16Net& bf, int layer, int np, int sp);
// y = LN epilogue of conv(x) + bias (and, with y_p, the fused projection y_p = W_p x +
// bias_p, stored without LayerNorm).
cudaError_t bf16_conv_fwd_ln(Bf16Net& bf, int layer, const float* x, const float* bias, float* y,
                             const Bf16Ln& ln, int B, long long bias_bs, cudaStream_t stream,
                             bool x_staged = false, const float* bias_p = nullptr,
                             float* y_p = nullptr);
// dx (=|+=) data gradient on the tensor cores (dy staged into the layer's dy buffer unless
// dy_staged).
cudaError_t bf16_conv_dgrad(Bf16Net& bf, int layer, const float* dy, float* dx, int B,
                            int accumulate, cudaStream_t stream, bool dy_staged = false);
// The BF16 staging buffer that holds this layer's dy (its data and weight gradients read it).
__nv_bfloat16* bf16_dy_buffer(const Bf16Net& bf, int layer);
// Whether the layer's data gradient runs the persistent halo kernel with room for the
// LayerNorm backward epilogue (C = ci <= 64, no fused projection), and the partial-sum rows
// per problem that epilogue writes.
bool bf16_dgrad_ln_ok(const Bf16Net& bf, int layer, int sp);
long long bf16_dgrad_ln_rows(const Bf16Net& bf, int layer);
// The data gradient D of the layer (dy staged unless dy_staged) followed, in its epilogue,
// by the LayerNorm (+ LeakyReLU) backward of the block that produced the layer's input x:
// with d = D (+ ln.resid), dp = d act'(ln.aout), dz = rstd (gamma dp - mean(gamma dp) -
// xhat mean(gamma dp xhat)) per voxel over the C = ci channels; dz goes to ln.ybf (the
// consumer's dy staging, sp blocks) and, when dz_out is set, to dz_out [B][voxels][C] FP32;
// the (dgamma, dbeta) sums of each 8 x 16 voxel slice go to ln.part (fixed order; a row
// reduction gives the gradients).  x's own gradient D + resid is not stored.
cudaError_t bf16_conv_dgrad_ln(Bf16Net& bf, int layer, const float* dy, float* dz_out,
                               const Bf16Ln& ln, int B, cudaStream_t stream,
                               bool dy_staged = false);

// Partial-sum rows (chunks of output voxels) of one pass of a tensor-core weight gradient,
// and the passes (1, or 3 in split precision); a problem's rows are passes x chunks.
long long bf16_wgrad_chunks(const Bf16Net& bf, int layer, int B);
int bf16_wgrad_passes(const Bf16Net& bf, int layer);
// Per-chunk partial sums part[b][pass][chunk][Co*27*Ci + Co] (weights, then bias) of a layer
// with .wgrad set; the caller adds a problem's rows (reduce_rows_f32).
// With dz_p (layer with projw): also the projection's partial sums
// part_p[b][pass][chunk][Co*Ci + Co] (its dz_p is staged here unless the fused data gradient
// did).
// x_staged: the layer's forward has staged x into its kept input copy (keep_inputs) since x
// last changed; dy_staged: its data gradient has just staged this dy (both skip a staging).
cudaError_t bf16_conv_wgrad(Bf16Net& bf, int layer, const float* x, const float* dy,
                            float* part, int B, cudaStream_t stream,
                            const float* dz_p = nullptr, float* part_p = nullptr,
                            bool x_staged = false, bool dy_staged = false);

// Context-free form for the op entry points: one layer, staging buffers, BF16 weights and
// the error word carved from a caller workspace of bf16_op_workspace() bytes.
long long bf16_op_workspace(int B, Dims3 din, int ci, int co, int k, int s);
cudaError_t bf16_op_conv(bool dgrad, const float* in, const float* W, const float* bias,
                         float* out, int B, Dims3 din, int ci, int co, int k, int s,
                         long long w_bs, int accumulate, void* workspace, cudaStream_t st);

long long bf16_op_wgrad_workspace(int B, Dims3 din, int ci, int co, int k);
cudaError_t bf16_op_wgrad(const float* x, const float* dy, float* dWb, int B, Dims3 din, int ci,
                          int co, int k, long long dw_bs, int accumulate, void* workspace,
                          cudaStream_t st);

}  // namespace d2ip
