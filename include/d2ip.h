/*
 * d2ip.h -- C ABI of the GB300 D²IP fitting library (libd2ip.so).
 *
 * The library fits a sequence of 3D conductivity changes to EIT boundary voltages with a
 * deep image prior: each frame's Delta sigma is the output of a residual 3D U-Net phi(theta | Z)
 * fed with a fixed noise volume Z (paper Eq. 2); theta minimises the l2 data term
 * ||J Delta sigma - Delta v||^2 of the linearised model V = J Sigma (Eq. 1, Eq. 4) with Adam;
 * UPWS warm-starts theta on one frame (Eqs. 5-7) and TPP carries it from frame to frame
 * (Eqs. 8-9).  Every step runs in CUDA kernels for sm_103a on one GPU.
 *
 * Conventions (all entry points):
 *  - Return D2IP_OK (0) or a negative d2ip_status; no exception crosses the ABI.  Shapes and
 *    arguments are validated on the host before any launch.  d2ip_last_error(ctx) (or
 *    d2ip_last_error(NULL) for the context-free op calls) gives a message for the calling
 *    context / thread.
 *  - Volumes are channels-last: element (voxel q, channel c) at q*C + c with
 *    q = (z*Y + y)*X + x (x fastest); a batch of B problems is B such volumes back to back.
 *    The vectorised Delta sigma uses the same voxel order (the operator V of Eq. 2).
 *  - Sensitivity matrix J: M x V row-major float32 (V = X*Y*Z voxels, M measurements).
 *  - Flat parameter arena theta, in module order (see d2ip_param_table); a convolution stores
 *    W[co][kz][ky][kx][ci] then b[co]; a LayerNorm stores gamma[c] then beta[c].
 *  - Context calls accept HOST or DEVICE pointers for their arrays unless stated otherwise:
 *    copies use cudaMemcpyDefault, so unified addressing tells them apart (pageable host
 *    memory works; pinned host memory is faster).  Context calls return after their results
 *    are written.
 *  - Context-free op calls (d2ip_conv3d_*, d2ip_layernorm_*, ...) take DEVICE pointers only,
 *    enqueue on `stream` (a cudaStream_t; NULL = legacy default stream) and return at once.
 *  - The caller owns every pointer it passes; the library never frees or keeps them beyond
 *    the call, except the context, which owns its copy of J, Z, theta and its workspace.
 */
#ifndef D2IP_H
#define D2IP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int d2ip_status;
#define D2IP_OK 0
#define D2IP_ERR_BAD_ARG (-1)   /* null pointer, bad enum, bad hyperparameter            */
#define D2IP_ERR_BAD_SHAPE (-2) /* inconsistent sizes (m, n, grid, widths, batch)         */
#define D2IP_ERR_OOM (-3)       /* device allocation failed                               */
#define D2IP_ERR_NONFINITE (-4) /* a loss or residual became NaN/Inf                      */
#define D2IP_ERR_TIMEOUT (-5)   /* a bounded device wait ran out                          */
#define D2IP_ERR_CUDA (-6)      /* a CUDA runtime call failed (message in last_error)     */
#define D2IP_ERR_STATE (-7)     /* call out of order (e.g. fit before d2ip_load_J)        */

#define D2IP_FP32 0 /* convolutions and J products in FP32 (SIMT), FP32 accumulation      */
#define D2IP_BF16 1 /* convolutions on tcgen05 tensor cores and J products from a BF16 copy
                       of J, FP32 accumulation; J column norms and the residual stay FP64    */
#define D2IP_BF16X3 2 /* split BF16: convolutions on tcgen05 tensor cores with every operand
                       v carried as two BF16 numbers hi = bf16(v), lo = bf16(v - hi) (16
                       significant bits); each product sums hi*hi + lo*hi + hi*lo in FP32
                       (three times the MMAs of D2IP_BF16).  J products read J as the same
                       hi + lo pair, added in FP32.  Plain BF16 operands (8 bits) and TF32
                       (11) both carry the Adam trajectory of a 100-step fit away from the
                       FP64 one; 16 bits follow it */

/* parameter-table kinds */
#define D2IP_PARAM_CONV_W 0
#define D2IP_PARAM_CONV_B 1
#define D2IP_PARAM_LN_GAMMA 2
#define D2IP_PARAM_LN_BETA 3

typedef struct d2ip_ctx d2ip_ctx;

/* ---------------------------------------------------------------------------------------
 * Context: one network shape, one grid, one J, B independent problems fitted in lockstep.
 * ------------------------------------------------------------------------------------- */

/* Create a context on CUDA `device`.  `stream` (a cudaStream_t) is the stream all work is
 * issued on; NULL makes the context create its own non-blocking stream (graph capture needs
 * a stream other than the legacy default one).  *out receives the context. */
d2ip_status d2ip_create(d2ip_ctx** out, int device, void* stream);
/* Free the context and all its device memory.  NULL is accepted. */
d2ip_status d2ip_destroy(d2ip_ctx* ctx);

/* Reconstruction grid X x Y x Z (rows, columns, planes of Eq. 1; V = X*Y*Z voxels). */
d2ip_status d2ip_set_grid(d2ip_ctx* ctx, int X, int Y, int Z);

/* Residual 3D U-Net of `levels` levels with channel widths[levels] (each a multiple of 4,
 * at most 128; multiples of 16 for the BF16 precisions), `c_in` input channels of Z,
 * `precision` D2IP_FP32, D2IP_BF16 or D2IP_BF16X3, and `batch`
 * independent problems (each with its own theta, Adam state, Z and measurements; all share
 * the grid and J).  Layout: stem act(LN(conv3(c_in->w0))); per level a ResBlock, preceded
 * for l > 0 by act(LN(conv3 stride 2)); decoder Up(trilinear) + concat(skip) + ResBlock with
 * a 1x1x1 projection; tail conv1(w0->1), linear.  ResBlock: act(LN(conv3(act(LN(conv3 x))))
 * + P x) with the second act after the residual sum.  LN over the channels of each voxel,
 * eps 1e-5; act LeakyReLU(0.2).  (Sec. III-D: residual connections and LayerNorm.) */
d2ip_status d2ip_set_network(d2ip_ctx* ctx, int levels, const int* widths, int c_in,
                             int precision, int batch);

/* The paper-form 3D-FastResUNet of Sec. III-D as a network variant (the section names its
 * parts but gives no sizes; this is one reading of them).  `levels` encoder stages of widths
 * widths[levels] (multiples of 8, 8..128), `c_in` 1..256, precision D2IP_FP32 only (the
 * depthwise and pointwise kernels are FP32 SIMT), `batch` problems as in d2ip_set_network.
 * Layout, in parameter order:
 *   stem act(LN(conv3(c_in -> w0)));
 *   per stage l: SE then ResConv3D(-> w_l, stride 1 for l = 0 else 2), where
 *     SE(C) = x * sigmoid(FC2(relu(FC1(mean over voxels of x)))), FC1: C -> max(C/4, 1);
 *     ResConv3D(ci -> co, s) = act(LN_b(DWSep_b(act(LN_a(DWSep_a(x, s))))) + P x),
 *     DWSep = depthwise 3x3x3 (stride s) then pointwise 1x1x1, P a 1x1x1 convolution with
 *     stride s when ci != co or s != 1, else the identity;
 *   bottleneck: act(LN(DWSep(stride 2))) then ASPP: branches 1x1x1, depthwise dilation 2
 *     and 3 each then 1x1x1, and the global mean through 1x1x1 broadcast back, each of
 *     width max(C/2, 1) with LeakyReLU, concatenated in that order, 1x1x1 back to C,
 *     act(LN);
 *   decoder l = L-1..0: attention gate on the skip e_l, e_l * sigmoid(psi(relu(Wx e_l +
 *     Up(Wg g)))) with max(w_l/2, 1) inner channels, then ResConv3D([Up(g), gated skip] ->
 *     w_l); g is the coarser decoder output (the ASPP output for l = L-1);
 *   tail sigmoid(conv1(w0 -> 1)).
 * Weights: dense W[co][kz][ky][kx][ci] then b[co]; depthwise W[c][kz][ky][kx] then b[c]
 * (kind D2IP_PARAM_CONV_W/B, fan_in 27); LayerNorm gamma then beta.  Every other call
 * (J, input, optimiser, fits, state, tracing) works on it unchanged. */
d2ip_status d2ip_set_network_fastres(d2ip_ctx* ctx, int levels, const int* widths, int c_in,
                                     int precision, int batch);

/* Number of parameters P of one problem's theta. */
d2ip_status d2ip_param_count(d2ip_ctx* ctx, long long* count);
/* Parameter table: row r = {kind, offset, count, fan_in} (kind: D2IP_PARAM_*), written to
 * rows[4*r .. 4*r+3] (host memory) for r < cap; *n_rows receives the number of rows. */
d2ip_status d2ip_param_table(d2ip_ctx* ctx, long long* rows, int cap, int* n_rows);
/* The same table without a context or a device: the plan of network `net` (0 the residual
 * U-Net of d2ip_set_network, 1 the FastResUNet variant of d2ip_set_network_fastres) on an
 * X x Y x Z grid, for host code that lays out or initialises theta before any GPU call.
 * rows as above (host memory); *count (may be NULL) receives P.  Shapes are checked as in
 * the two set-network calls (D2IP_ERR_BAD_ARG / D2IP_ERR_BAD_SHAPE). */
d2ip_status d2ip_plan_param_table(int net, int X, int Y, int Z, int levels, const int* widths,
                                  int c_in, long long* rows, int cap, int* n_rows,
                                  long long* count);

/* Copy J (m x n, n = X*Y*Z) into the context.  normalize_cols != 0 scales every column to
 * unit l2 norm with the norm accumulated in FP64 (Eq. 1, "normalized" sensitivity); a zero
 * column is left as is.  J may be host or device memory.  m <= 6400; with the BF16 precisions
 * also m a multiple of 4 and at most 1024 (D2IP_ERR_BAD_SHAPE otherwise). */
d2ip_status d2ip_load_J(d2ip_ctx* ctx, const float* J, int m, int n, int normalize_cols);
/* The FP64 column norms used by the last d2ip_load_J (n values; host or device memory). */
d2ip_status d2ip_get_colnorms(d2ip_ctx* ctx, double* out);

/* Fixed network input Z ([batch][n][c_in], Eq. 2) and initial weights theta0 ([batch][P],
 * UPWS starts from them, Sec. III-B).  Resets the Adam state. */
d2ip_status d2ip_set_input(d2ip_ctx* ctx, const float* Z, const float* theta0);

/* Adam hyperparameters (Sec. III-A; defaults lr 1e-3, 0.9, 0.999, 1e-8).  Given in double:
 * (1 - beta) is formed in double before rounding to the float the kernels use. */
d2ip_status d2ip_set_optim(d2ip_ctx* ctx, double lr, double beta1, double beta2, double eps);
/* 4D-TV regulariser of Sec. III-E added to the data term (Eq. 13): lambda_tv * (lambda_s *
 * R_spatial + lambda_t * R_temporal); the paper uses 0.002, 1 and 0.1 (Sec. IV-D).  R_spatial
 * = (1/V) sum_voxels sqrt(dx^2 + dy^2 + dz^2 + eps) with forward differences (0 past the far
 * face); R_temporal = (1/sum a) sum_j a_j sum_voxels sqrt((s - s_j)^2 + eps) over the earlier
 * frames j of the sequence, a_j = exp(-(i - j)).  lambda_tv = 0 (the default) turns it off.
 * d2ip_fit_sequence/batched keep the earlier outputs on the device; d2ip_fit_frame and
 * d2ip_run_steps see no earlier frame (spatial term only).  The loss trace includes it;
 * residual_out stays the data term alone. */
d2ip_status d2ip_set_regularizer(d2ip_ctx* ctx, double lambda_tv, double lambda_s,
                                 double lambda_t, double eps);
/* Zero the Adam moments and step count (done at the start of every fitted frame). */
d2ip_status d2ip_reset_optimizer(d2ip_ctx* ctx);
/* reset_moments_per_frame != 0 (the default): d2ip_fit_frame and every frame of
 * d2ip_fit_sequence/batched start with a fresh Adam state, the paper's reading of Eqs. 7-8
 * (only the weights theta carry from UPWS to frame 1 and from frame to frame).  0: the Adam
 * moments and step count carry on too -- a sequence is then one Adam run whose target
 * measurements change at each frame (its state is reset once, at the start of UPWS, or of
 * frame 0 when there is no UPWS phase); d2ip_fit_frame then continues the current state. */
d2ip_status d2ip_set_frame_reset(d2ip_ctx* ctx, int reset_moments_per_frame);

/* n_steps DIP iterations (forward phi, r = J phi - dv, loss = |r|^2/m in FP64, gradient
 * (2/m) J^T r back through phi, Adam) on measurements dV ([batch][m]) WITHOUT resetting the
 * Adam state.  loss_trace ([n_steps][batch], host, FP64) receives the loss at each iterate
 * before its update, or pass NULL. */
d2ip_status d2ip_run_steps(d2ip_ctx* ctx, const float* dV, int n_steps, double* loss_trace);
/* Delta sigma = phi(theta | Z) at the current theta ([batch][n]). */
d2ip_status d2ip_forward(d2ip_ctx* ctx, float* dsigma_out);
/* dL/dtheta of the last iteration ([batch][P]). */
d2ip_status d2ip_get_grad(d2ip_ctx* ctx, float* grad_out);

/* One frame (Eqs. 4 and 6): reset Adam, n_steps iterations on dV ([batch][m]), then
 * dsigma_out ([batch][n]) = phi at the last iterate and residual_out ([batch], FP64, host or
 * device) = |J dsigma - dV|^2 / m.  loss_trace as in d2ip_run_steps (or NULL). */
d2ip_status d2ip_fit_frame(d2ip_ctx* ctx, const float* dV, int n_steps, float* dsigma_out,
                           double* residual_out, double* loss_trace);

/* A time sequence (Secs. III-B, III-C): UPWS = upws_steps iterations on dV0 ([batch][m];
 * NULL = frame 0 of V) from the current theta; then frame 0 with first_steps and each later
 * frame with later_steps iterations, each frame starting from the previous frame's weights
 * with a fresh Adam state.  V is [batch][T][m]; Sigma_out [batch][T][n] receives each frame's
 * phi at its last iterate; residual_out [batch][T] (FP64) its data residual. */
d2ip_status d2ip_fit_sequence(d2ip_ctx* ctx, const float* V, int T, const float* dV0,
                              int upws_steps, int first_steps, int later_steps,
                              float* Sigma_out, double* residual_out);

/* Batched form: `count` contexts (for example one per grid and measurement-count group of a
 * set of independent sequences, each context holding its group's problems as its batch) fit
 * their sequences concurrently, every context on its own stream, with the schedule of
 * d2ip_fit_sequence.  V[i], dV0[i] (dV0 may be NULL, or entries NULL), Sigma_out[i] and
 * residual_out[i] are context i's arrays exactly as in d2ip_fit_sequence.  Returns after
 * all contexts finished; the first failing context's status is returned. */
d2ip_status d2ip_fit_batched(d2ip_ctx* const* ctxs, int count, const float* const* V, int T,
                             const float* const* dV0, int upws_steps, int first_steps,
                             int later_steps, float* const* Sigma_out,
                             double* const* residual_out);

/* Checkpoint: theta, Adam m and v ([batch][P] each) and the Adam step count.  Any pointer
 * may be NULL to skip that part. */
d2ip_status d2ip_get_state(d2ip_ctx* ctx, float* theta, float* adam_m, float* adam_v,
                           int* adam_t);
d2ip_status d2ip_set_state(d2ip_ctx* ctx, const float* theta, const float* adam_m,
                           const float* adam_v, int adam_t);

/* ERR = |est - truth| / |truth| per problem in FP64 (Sec. V-A); est, truth [batch][n]. */
d2ip_status d2ip_err_ratio(d2ip_ctx* ctx, const float* est, const float* truth, double* out);

/* Autotuning of the tensor-core tilings (BF16 precisions; on by default): when the context's
 * workspace is built (the first d2ip_load_J / d2ip_set_input / d2ip_set_state after
 * d2ip_set_network), every persistent halo convolution of the network -- forward and data
 * gradient of each 3x3x3 stride-1 layer -- is timed with CUDA events for every candidate
 * tiling (kz taps packed into one MMA or not, output z depth 1..8, channel chunk 16/32/64)
 * on the context's own buffers, and the fastest is kept.  Choices are cached for the process
 * per shape, so contexts of one shape share them (and their FP32 summation order); on = 0
 * keeps the cost model's tilings.  Takes effect when the workspace is next built.  The
 * tuning runs synchronously on the context's stream, before any graph is captured. */
d2ip_status d2ip_set_autotune(d2ip_ctx* ctx, int on);
/* The tilings in use, one row per tensor-core layer in module order (host arrays, rows of 15:
 * ci, co, k, stride, out dims z, y, x, then forward {persistent, kz-packed, channel chunk,
 * z depth} and data gradient {persistent, kz-packed, channel chunk, z depth}); us (may be
 * NULL) receives 4 per row: the forward's tuned and cost-model times (us per launch), then the
 * data gradient's (-1 where not timed).  *n_rows receives the number of layers (0 in FP32).
 * D2IP_ERR_STATE before the workspace exists. */
d2ip_status d2ip_tile_plan(d2ip_ctx* ctx, long long* rows, int cap, int* n_rows, double* us);
/* LayerNorm (+ LeakyReLU) backward in the epilogue of the data gradient that produces its
 * input gradient (BF16 precisions; off by default): conv b's data gradient then also runs
 * LayerNorm a's backward, and conv a's (adding the residual gradient already in dx) the
 * backward of the unit before the block, writing the BF16 dy staging of the next layer and
 * per-tile (dgamma, dbeta) partial sums instead of the FP32 gradients in between.  Applies
 * where that data gradient runs the persistent halo kernel with room for the epilogue.
 * Measured on the batched 48x48x24 group it moves about as much time into the data
 * gradients as it removes from the standalone LayerNorm backward (whose loads run near
 * HBM speed), hence opt-in.  Takes effect at the next graph capture. */
d2ip_status d2ip_set_ln_backward_fusion(d2ip_ctx* ctx, int on);
/* Restores tilings saved from d2ip_tile_plan (e.g. by an earlier process on this GPU), so a
 * context of the same network, grid and batch skips the timing sweep: rows (host, n_rows x 15,
 * copied) are applied when the workspace is next built, in place of the autotuner.  Call
 * after d2ip_set_network and before the workspace exists (D2IP_ERR_STATE afterwards).  When
 * the workspace is built, a row whose shape columns or persistent flags do not match the
 * layer, or whose tiling cannot run, fails that call with D2IP_ERR_BAD_ARG.  n_rows = 0
 * clears a stored plan.  BF16 precisions only (rows are ignored in FP32). */
d2ip_status d2ip_set_tile_plan(d2ip_ctx* ctx, const long long* rows, int n_rows);

/* Kernel classes reported by d2ip_profile_iterations, in this order. */
#define D2IP_KCLASS_CONV_FWD 0   /* work: FLOPs (2 * out voxels * K^3 * ci * co)        */
#define D2IP_KCLASS_CONV_DGRAD 1 /* work: FLOPs (same count as the forward)             */
#define D2IP_KCLASS_CONV_WGRAD 2 /* work: FLOPs (same count; includes the chunk sum)    */
#define D2IP_KCLASS_LN_FWD 3     /* work: bytes read + written                          */
#define D2IP_KCLASS_LN_BWD 4     /* work: bytes (includes the dgamma/dbeta sum)          */
#define D2IP_KCLASS_UP_FWD 5     /* work: bytes                                          */
#define D2IP_KCLASS_UP_BWD 6     /* work: bytes                                          */
#define D2IP_KCLASS_JMUL 7       /* work: bytes of J + vectors                          */
#define D2IP_KCLASS_LOSS 8       /* work: bytes                                          */
#define D2IP_KCLASS_JTMUL 9      /* work: bytes of J + vectors                          */
#define D2IP_KCLASS_ADAM 10      /* work: bytes (7 x 4 per parameter)                   */
#define D2IP_KCLASS_MISC 11      /* residual adds; work: bytes                          */
#define D2IP_KCLASS_COUNT 12

/* Tracing: run n_iters DIP iterations eagerly (no graph) on dV ([batch][m]) with a CUDA-event
 * pair around every kernel launch, and accumulate per kernel class (D2IP_KCLASS_*) the
 * device time in ms, the algorithmic work and the number of launches (host arrays of
 * D2IP_KCLASS_COUNT entries).  The iterations update theta like d2ip_run_steps. */
d2ip_status d2ip_profile_iterations(d2ip_ctx* ctx, const float* dV, int n_iters, double* ms,
                                    double* work, long long* launches);

/* Kernel launches of one training iteration (the captured step graph: forward, data term,
 * backward, Adam) and of one evaluation (forward and data term), counted as the kernel
 * nodes of the CUDA graphs the context replays (captured here if not yet). */
d2ip_status d2ip_graph_kernels(d2ip_ctx* ctx, long long* step_kernels, long long* eval_kernels);

/* Wait for the context's stream; report asynchronous CUDA errors. */
d2ip_status d2ip_sync(d2ip_ctx* ctx);
/* Message of the last failure of `ctx` (NULL: of the calling thread's op calls). */
const char* d2ip_last_error(d2ip_ctx* ctx);

/* ---------------------------------------------------------------------------------------
 * Context-free ops (DEVICE pointers, asynchronous on `stream`).  Volume dims are (dz, dy,
 * dx) of the op's input; a K^3 conv (K = 3 or 1) with stride S and zero padding (K-1)/2 has
 * output dims (d + 2*((K-1)/2) - K)/S + 1 per axis.  Weights W are [co][K^3][ci] followed
 * by bias [co] in a per-problem block; `w_batch_stride` is the distance between problems'
 * blocks (0 = shared).
 * ------------------------------------------------------------------------------------- */

/* y = conv(x, W) + b  (implicit GEMM; FP32). */
d2ip_status d2ip_conv3d_forward(const float* x, const float* W, const float* b, float* y,
                                int batch, int dz, int dy, int dx, int ci, int co, int ksize,
                                int stride, long long w_batch_stride, void* stream);
/* dx (=, or += when accumulate) transposed conv of dy with W: the input gradient. */
d2ip_status d2ip_conv3d_dgrad(const float* dy, const float* W, float* dx, int batch, int dz,
                              int dy_, int dx_, int ci, int co, int ksize, int stride,
                              long long w_batch_stride, int accumulate, void* stream);
/* Tensor-core forms (tcgen05, sm_103a) of the two calls above: x (or dy) and W are rounded
 * to BF16 (round to nearest even), products accumulate in FP32 in tensor memory; the
 * bias is added in FP32.  Needs ci and co multiples of 16, co <= 256 (ci <= 256 too for the
 * data gradient; its stride-2 form runs as 8 output-parity classes of 1 to 8 taps on the
 * coarse grid).  x (or dy) and y (or dx) must be 16-byte aligned (D2IP_ERR_BAD_ARG
 * otherwise).  `workspace` (device, d2ip_conv3d_tc_workspace bytes) receives the
 * BF16 staging copies; the int at its first 1024-byte aligned address is an error word,
 * non-zero after the call when a pipeline wait of the kernel gave up (about 1 s). */
long long d2ip_conv3d_tc_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                   int ksize, int stride);
d2ip_status d2ip_conv3d_forward_tc(const float* x, const float* W, const float* b, float* y,
                                   int batch, int dz, int dy, int dx, int ci, int co, int ksize,
                                   int stride, long long w_batch_stride, void* workspace,
                                   long long workspace_bytes, void* stream);
d2ip_status d2ip_conv3d_dgrad_tc(const float* dy, const float* W, float* dx, int batch, int dz,
                                 int dy_, int dx_, int ci, int co, int ksize, int stride,
                                 long long w_batch_stride, int accumulate, void* workspace,
                                 long long workspace_bytes, void* stream);

/* Tensor-core weight gradient of a stride-1 convolution (3x3x3 or 1x1x1; tcgen05, x and dy
 * rounded to BF16, FP32 accumulation, the bias gradient from the same MMAs): result as
 * d2ip_conv3d_wgrad.  Needs ci and co multiples of 16, co dividing 128, ci + min(64, ci) <= 256.
 * Workspace: d2ip_conv3d_wgrad_tc_workspace bytes (device); the int at its first 1024-byte
 * aligned address is the error word. */
long long d2ip_conv3d_wgrad_tc_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                         int ksize);
d2ip_status d2ip_conv3d_wgrad_tc(const float* x, const float* dy, float* dWb, int batch,
                                 int dz, int dy_, int dx_, int ci, int co, int ksize,
                                 long long dw_batch_stride, int accumulate, void* workspace,
                                 long long workspace_bytes, void* stream);

/* Workspace bytes needed by d2ip_conv3d_wgrad for these sizes. */
long long d2ip_conv3d_wgrad_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                      int ksize, int stride);
/* dWb[batch][co*K^3*ci + co] (=, or +=) weight and bias gradients of conv(x) against dy
 * (deterministic: per-chunk partial sums in `workspace`, then a fixed-order sum). */
d2ip_status d2ip_conv3d_wgrad(const float* x, const float* dy, float* dWb, int batch, int dz,
                              int dy_, int dx_, int ci, int co, int ksize, int stride,
                              long long dw_batch_stride, int accumulate, void* workspace,
                              long long workspace_bytes, void* stream);

/* The weight gradient above, for callers that cannot allocate device memory while they
 * need it: a bedside monitoring loop that runs with a fixed device footprint and must not
 * block or fail on the allocator mid-sequence, or a host application whose device memory is
 * all owned by another allocator (a framework's caching pool), so it has no workspace to
 * hand over.  This entry point allocates nothing (no cudaMalloc, cudaFree or allocating
 * library call): its partial sums live in a 16 MiB static __device__ array that is part of
 * the library on every GPU that loads it, until the process exits.  The paper has no
 * counterpart; it is an interface convenience.
 * Same arguments and result as d2ip_conv3d_wgrad without the workspace.  Sizes whose
 * d2ip_conv3d_wgrad_workspace exceeds 16 MiB are rejected with D2IP_ERR_BAD_SHAPE.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it; make that first call before any stream capture.
 * All calls share the one array, and it keeps the last call's partial sums (each call
 * writes every partial it reads, so nothing needs clearing): calls that overlap on the GPU
 * (different streams, or different host threads) race and must not be issued. */
d2ip_status d2ip_conv3d_wgrad_noalloc(const float* x, const float* dy, float* dWb, int batch,
                                      int dz, int dy_, int dx_, int ci, int co, int ksize,
                                      int stride, long long dw_batch_stride, int accumulate,
                                      void* stream);

/* y = act(gamma * xhat + beta (+ resid)), xhat = (z - mean)/sqrt(var + 1e-5) over the c
 * channels of each voxel; saves xhat ([batch][nvox][c]) and rstd ([batch][nvox]) for the
 * backward.  gamma_beta = [gamma[c], beta[c]] per problem.  act: 0 none, 1 LeakyReLU(0.2).
 * c must be a multiple of 4, at most 128. */
d2ip_status d2ip_layernorm_act_forward(const float* z, const float* gamma_beta,
                                       const float* resid, float* y, float* xhat, float* rstd,
                                       int batch, long long nvox, int c, int act,
                                       long long gb_batch_stride, void* stream);
long long d2ip_layernorm_workspace(int batch, long long nvox, int c);
/* Backward of the above given dy = dL/dy: dpre = dy * act'(act_out) (act_out NULL: no act),
 * dt = dpre (optional, the residual-branch gradient), dz = LN backward of dpre, and
 * dgamma_beta[batch][2c] (=, or +=) sum over voxels of (dpre * xhat, dpre). */
d2ip_status d2ip_layernorm_act_backward(const float* dy, const float* act_out,
                                        const float* xhat, const float* rstd,
                                        const float* gamma_beta, float* dz, float* dt,
                                        float* dgamma_beta, int batch, long long nvox, int c,
                                        long long gb_batch_stride, int accumulate,
                                        void* workspace, long long workspace_bytes,
                                        void* stream);

/* cat[:, :cu] = trilinear(low (lz,ly,lx) -> (oz,oy,ox)), half-pixel centres, source index
 * clamped at 0 (PyTorch align_corners=False with an explicit size); cat[:, cu:] = skip.
 * cu and cs are multiples of 4 (cs may be 0). */
d2ip_status d2ip_upsample_concat_forward(const float* low, const float* skip, float* cat,
                                         int batch, int lz, int ly, int lx, int oz, int oy,
                                         int ox, int cu, int cs, void* stream);
/* Adjoint: dlow = upsample^T(dcat[:, :cu]) (a gather, deterministic); dskip = dcat[:, cu:]
 * (dskip may be NULL). */
d2ip_status d2ip_upsample_concat_backward(const float* dcat, float* dlow, float* dskip,
                                          int batch, int lz, int ly, int lx, int oz, int oy,
                                          int ox, int cu, int cs, void* stream);

/* Data term of Eq. 4: r[b] = J x[b] - dv[b] (FP32, x [batch][n]) and, when loss is not NULL,
 * loss[b] = |r[b]|^2 / m accumulated in FP64 (device memory).  The products are summed in
 * fixed-order column chunks held in `workspace` (d2ip_sensitivity_workspace bytes). */
long long d2ip_sensitivity_workspace(int batch, int m, int n);
d2ip_status d2ip_sensitivity_residual(const float* J, const float* x, const float* dv,
                                      float* r, double* loss, int batch, int m, int n,
                                      void* workspace, long long workspace_bytes,
                                      void* stream);
/* g[b] = scale * J^T r[b]  (scale = 2/m gives the gradient of the mean-square data term). */
d2ip_status d2ip_sensitivity_adjoint(const float* J, const float* r, float* g, float scale,
                                     int batch, int m, int n, void* stream);
/* The two products above on the tensor cores (tcgen05, the form the BF16 precisions use in a
 * context): J is rounded to BF16 (split != 0: carried as hi + lo, hi = bf16(J), lo =
 * bf16(J - hi)), and so are x and r, the products accumulate in FP32 with the problems as the
 * MMA's N: r = J x - dv (FP32, summed over fixed voxel chunks, so deterministic) and, when g is
 * not NULL, g = scale J^T r.  J [m][n] FP32, x and g [batch][n], dv and r [batch][m], all
 * device memory.  m a multiple of 8 and at most 1024 (D2IP_ERR_BAD_SHAPE otherwise).
 * workspace: d2ip_sensitivity_tc_workspace bytes (device; holds the transposed BF16 J, the
 * staged x and r and the partial sums); its int at the first 256-byte aligned address is the
 * error word, non-zero after the call when a pipeline wait of the kernel gave up. */
long long d2ip_sensitivity_tc_workspace(int batch, int m, int n, int split);
d2ip_status d2ip_sensitivity_products_tc(const float* J, const float* x, const float* dv,
                                         float* r, float* g, float scale, int batch, int m,
                                         int n, int split, void* workspace,
                                         long long workspace_bytes, void* stream);
/* The 4D-TV regulariser alone: grad[b] += its gradient at dsigma[b] ([batch][n]) given
 * n_previous earlier outputs previous[b][j][n]; value_host[b] (host, may be NULL) receives
 * its value (a synchronising copy).  Workspace: d2ip_tv4d_workspace bytes (device). */
long long d2ip_tv4d_workspace(int batch, int dz, int dy, int dx);
d2ip_status d2ip_tv4d(const float* dsigma, const float* previous, int n_previous, float* grad,
                      double* value_host, int batch, int dz, int dy, int dx, double lambda_tv,
                      double lambda_s, double lambda_t, double eps, void* workspace,
                      long long workspace_bytes, void* stream);
/* In place: J[:, j] /= |J[:, j]|_2 with the norm in FP64; colnorm[j] receives it. */
d2ip_status d2ip_normalize_columns(float* J, double* colnorm, int m, int n, void* stream);
/* One Adam step (bias-corrected, step number t >= 1) over `count` parameters. */
d2ip_status d2ip_adam_update(float* theta, const float* g, float* m, float* v,
                             long long count, double lr, double beta1, double beta2,
                             double eps, int t, void* stream);

/* Self-test of the bounded-wait error path on `device`: a one-thread kernel waits on a
 * device flag for at most spin_limit polls (1..2^26, about 64 ns apart), as the tensor-core
 * kernels wait on their pipeline barriers.  set_flag = 0 leaves the flag unset, so the wait
 * runs out; the kernel then writes code 2 to its status word instead of hanging or trapping,
 * and the call returns D2IP_ERR_TIMEOUT.  set_flag = 1 sets the flag first and the call
 * returns D2IP_OK.  *status_out receives the status word (0 or 2).  Synchronous; leaves
 * the device usable. */
d2ip_status d2ip_wait_selftest(int device, long long spin_limit, int set_flag, int* status_out);

#ifdef __cplusplus
}
#endif

#endif /* D2IP_H */
