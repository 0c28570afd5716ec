// Runtime of the D²IP fitting library: the network plan (module order, parameter arena,
// activation and gradient buffers), the launch sequences of one DIP iteration, CUDA-graph
// capture and replay, the UPWS/TPP sequence driver and the C-ABI entry points.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/d2ip.h"
#include "common.cuh"
#include "conv_bf16.cuh"
#include "jprod_tc.cuh"
#include "fastres.cuh"

using namespace d2ip;

namespace {

thread_local std::string g_op_error;

constexpr int kTraceCap = 4096;  // device loss-trace ring (iterations)
constexpr long long kAlign = 64;  // floats (256 bytes)

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

struct ConvL {
  int ci = 0, co = 0, k = 3, s = 1;
  Dims3 din{}, dout{};
  long long w_off = 0;  // bias follows at w_off + co*k^3*ci
  int tc = -1;          // index of its tensor-core layer (BF16 precision), -1: FP32 SIMT
  long long wcount() const { return (long long)co * k * k * k * ci; }
};

struct LnL {
  int c = 0;
  long long g_off = 0;  // beta follows at g_off + c
};

struct Unit {  // act(LN(conv(x))): the stem and the stride-2 down convolutions
  ConvL conv;
  LnL ln;
  int lvl_in = 0, lvl_out = 0;
  const float* x = nullptr;
  float *xh = nullptr, *rs = nullptr, *a = nullptr;
};

struct Res {  // act(LN_b(conv_b(act(LN_a(conv_a(x))))) + P(x))
  ConvL a, b, p;
  LnL lna, lnb;
  bool proj = false;
  bool fuse_f = false, fuse_d = false, fuse_w = false;  // projection fused into conv a (BF16)
  int lvl = 0;
  const float* x = nullptr;
  float *xh_a = nullptr, *rs_a = nullptr, *h1 = nullptr, *xh_b = nullptr, *rs_b = nullptr,
        *out = nullptr;
};

struct LevelBufs {
  float *g1 = nullptr, *g2 = nullptr, *tz = nullptr, *tt = nullptr, *th = nullptr,
        *de = nullptr, *cat = nullptr;
};

}  // namespace

struct d2ip_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // configuration
  int X = 0, Y = 0, Z = 0;
  int L = 0, c_in = 0, precision = D2IP_FP32, B = 1;
  int arch = 0;  // 0: residual U-Net; 1: paper-form 3D-FastResUNet variant (node list fr)
  std::vector<int> w;
  bool net_ready = false;
  int m = 0;
  bool j_ready = false, input_ready = false;
  double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
  bool frame_reset = true;  // fresh Adam state at every fitted frame (else carried)
  bool autotune = true;     // time the tensor-core tilings when the arena is built
  std::vector<long long> tile_rows;  // tilings to apply instead (d2ip_set_tile_plan)
  bool ln_bwd_fused = false;  // LayerNorm backward in data-gradient epilogues (opt-in)
  // 4D-TV regulariser (off when lam_tv == 0)
  double lam_tv = 0.0, lam_s = 1.0, lam_t = 0.1, tv_eps = 1e-8;

  // plan
  std::vector<Dims3> dims;
  std::vector<long long> table;  // rows of {kind, offset, count, fan_in}
  long long P = 0, Pp = 0;       // parameters, padded per-problem stride
  Unit stem;
  std::vector<Unit> down;        // index l (l >= 1)
  std::vector<Res> enc, dec;     // enc[l], dec[l] (l <= L-2)
  ConvL tail;
  std::vector<LevelBufs> lb;
  long long ws_floats = 0;

  // device memory
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  float *zin = nullptr, *dsigma = nullptr, *r = nullptr, *gds = nullptr, *dv = nullptr;
  float *ztmp = nullptr, *ptmp = nullptr, *ws = nullptr, *stage = nullptr;
  double *loss = nullptr, *resid = nullptr, *trace = nullptr, *seq_resid = nullptr;
  int *trace_pos = nullptr, *adam_t = nullptr, *status = nullptr, *nprev = nullptr;
  double* reg_part = nullptr;  // [B][tv4d_blocks] regulariser partial sums
  float* hist = nullptr;       // previous frames' outputs [B][hist_cap][n]
  int hist_cap = 0;
  float* J = nullptr;
  __nv_bfloat16* Jbf = nullptr;  // BF16 copy of the normalised J, transposed [n][m] (BF16)
  __nv_bfloat16* Jlo = nullptr;  // its low part bf16(J - Jbf) (split precision)
  JprodTc jp;                    // the J products on the tensor cores (when jp_stage is set)
  void* jp_stage = nullptr;      // their BF16 staging of x and r
  float* jpart = nullptr;  // column-chunk partial sums of J x
  double* colnorm = nullptr;
  size_t j_bytes = 0;
  int seq_T_cap = 0;
  Bf16Net bf;  // tensor-core path: BF16 staging buffers, weights, TMA descriptors
  FastNet fr;  // the FastResUNet variant's nodes and buffers (arch 1)

  // graphs
  cudaGraphExec_t g_step = nullptr, g_eval = nullptr;
  long long step_kernels = 0, eval_kernels = 0;  // kernel nodes of the captured graphs

  long long n() const { return (long long)X * Y * Z; }
};

namespace {

d2ip_status fail(d2ip_ctx* c, d2ip_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_op_error = msg;
  return st;
}

d2ip_status cuda_fail(d2ip_ctx* c, cudaError_t e, const char* what) {
  return fail(c, D2IP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                         \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);               \
  } while (0)

void drop_graphs(d2ip_ctx* c) {
  if (c->g_step) cudaGraphExecDestroy(c->g_step);
  if (c->g_eval) cudaGraphExecDestroy(c->g_eval);
  c->g_step = c->g_eval = nullptr;
}

void free_arena(d2ip_ctx* c) {
  drop_graphs(c);
  if (c->arena) cudaFree(c->arena);
  c->arena = nullptr;
  c->arena_bytes = 0;
}

// ------------------------------------------------------------------------------------
// plan construction (module order = parameter order)
// ------------------------------------------------------------------------------------
struct Builder {
  d2ip_ctx* c;
  long long off = 0;
  ConvL conv(int ci, int co, int k, int s, int lvl_in, bool input = false) {
    ConvL L;
    L.ci = ci;
    L.co = co;
    L.k = k;
    L.s = s;
    L.din = c->dims[lvl_in];
    L.dout = conv_out_dims(L.din, k, s);
    L.w_off = off;
    if (c->precision != D2IP_FP32)
      L.tc = input && ci < 16 ? bf16_add_input_layer(c->bf, ci, co, L.din, off)
                              : bf16_add_layer(c->bf, ci, co, k, s, L.din, off);
    const long long fan = (long long)ci * k * k * k;
    c->table.insert(c->table.end(), {D2IP_PARAM_CONV_W, off, L.wcount(), fan});
    off += L.wcount();
    c->table.insert(c->table.end(), {D2IP_PARAM_CONV_B, off, (long long)co, fan});
    off += co;
    return L;
  }
  LnL ln(int ch) {
    LnL L;
    L.c = ch;
    L.g_off = off;
    c->table.insert(c->table.end(), {D2IP_PARAM_LN_GAMMA, off, (long long)ch, (long long)ch});
    off += ch;
    c->table.insert(c->table.end(), {D2IP_PARAM_LN_BETA, off, (long long)ch, (long long)ch});
    off += ch;
    return L;
  }
  Res res(int ci, int co, int lvl) {
    Res R;
    R.lvl = lvl;
    R.a = conv(ci, co, 3, 1, lvl);
    // conv a's dy has a staging buffer of its own: conv b's data gradient writes it (the
    // LayerNorm backward in its epilogue) while reading conv b's dy from the other one
    if (R.a.tc >= 0) c->bf.layers[R.a.tc].dyslot = 1;
    R.lna = ln(co);
    R.b = conv(co, co, 3, 1, lvl);
    R.lnb = ln(co);
    R.proj = ci != co;
    if (R.proj) R.p = conv(ci, co, 1, 1, lvl);
    if (R.proj && R.a.tc >= 0 && R.p.tc >= 0) {
      const int f = bf16_fuse_proj(c->bf, R.a.tc, R.p.tc);
      R.fuse_f = (f & 1) != 0;
      R.fuse_d = (f & 2) != 0;
      R.fuse_w = (f & 4) != 0;
    }
    return R;
  }
};

void build_plan(d2ip_ctx* c) {
  if (c->arch == 1) {
    c->bf = Bf16Net{};
    c->stem = Unit{};
    c->down.clear();
    c->enc.clear();
    c->dec.clear();
    c->fr.build(Dims3{c->Z, c->Y, c->X}, c->L, c->w, c->c_in, c->table, c->P);
    c->dims.assign(c->fr.dims.begin(), c->fr.dims.end() - 1);
    c->Pp = round_up(c->P, kAlign);
    return;
  }
  c->dims.assign(c->L, Dims3{});
  c->dims[0] = Dims3{c->Z, c->Y, c->X};
  for (int l = 1; l < c->L; ++l) c->dims[l] = conv_out_dims(c->dims[l - 1], 3, 2);
  c->table.clear();
  c->bf = Bf16Net{};
  c->bf.keep_inputs = true;  // layer inputs stay staged in BF16 from forward to backward
  c->bf.sp = c->precision == D2IP_BF16X3 ? 3 : 1;
  Builder b{c};
  const auto& w = c->w;
  c->stem.conv = b.conv(c->c_in, w[0], 3, 1, 0, /*input=*/true);
  c->stem.ln = b.ln(w[0]);
  c->stem.lvl_in = c->stem.lvl_out = 0;
  c->enc.assign(c->L, Res{});
  c->down.assign(c->L, Unit{});
  c->dec.assign(c->L > 1 ? c->L - 1 : 0, Res{});
  c->enc[0] = b.res(w[0], w[0], 0);
  for (int l = 1; l < c->L; ++l) {
    c->down[l].conv = b.conv(w[l - 1], w[l], 3, 2, l - 1);
    c->down[l].ln = b.ln(w[l]);
    c->down[l].lvl_in = l - 1;
    c->down[l].lvl_out = l;
    c->enc[l] = b.res(w[l], w[l], l);
  }
  for (int l = c->L - 2; l >= 0; --l) c->dec[l] = b.res(w[l + 1] + w[l], w[l], l);
  c->tail = b.conv(w[0], 1, 1, 1, 0);
  c->P = b.off;
  c->Pp = round_up(c->P, kAlign);
}

// ------------------------------------------------------------------------------------
// buffers
// ------------------------------------------------------------------------------------
struct Carve {
  char* base;
  size_t used = 0;
  bool dry;
  template <class T>
  T* take(long long count) {
    const size_t bytes = (size_t)round_up(count * (long long)sizeof(T), 256);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// Weight gradients of 3x3x3 layers use the tensor cores; 1x1x1 ones stay on the SIMT kernel,
// which is faster there (only Co of the 128 MMA rows would carry work while the A tile still
// takes 32 KB of shared memory per stage, leaving one CTA per SM).
bool tc_wgrad(const d2ip_ctx* c, const ConvL& L) {
  return L.tc >= 0 && L.k == 3 && c->bf.layers[L.tc].wgrad;
}

// Whether every reader of a residual block's input takes its BF16 staged copy: conv a and
// its projection on the tensor cores (the projection fused, or reading conv a's kept copy),
// both weight gradients there too, and the residual taken from the projection.
bool bf16_only_input(const d2ip_ctx* c, const Res& R) {
  if (c->precision == D2IP_FP32 || !c->bf.keep_inputs || R.a.tc < 0 || !R.proj || R.p.tc < 0)
    return false;
  const bool p_fwd = R.fuse_f || bf16_input_shared(c->bf, R.p.tc);
  return p_fwd && tc_wgrad(c, R.a) && (R.fuse_w || tc_wgrad(c, R.p));
}

// The last layer (1x1x1 to one channel) has its own memory-bound kernels.
bool co1_layer(const ConvL& L) {
  return L.k == 1 && L.s == 1 && L.co == 1 && conv1x1_co1_supported(L.ci);
}

// Partial-sum rows per problem of a layer's weight gradient (chunks x operand passes).
long long wgrad_rows(const d2ip_ctx* c, const ConvL& L) {
  if (co1_layer(L)) return conv1x1_co1_blocks(L.din.count());
  if (tc_wgrad(c, L))
    return bf16_wgrad_chunks(c->bf, L.tc, c->B) * bf16_wgrad_passes(c->bf, L.tc);
  return conv3d_wgrad_chunks(L.din, L.k, L.s);
}

long long conv_ws_floats(const d2ip_ctx* c, const ConvL& L) {
  return (long long)c->B * wgrad_rows(c, L) * (L.wcount() + L.co);
}
long long ln_ws_floats(const d2ip_ctx* c, const LnL& L, int lvl) {
  return (long long)c->B * layernorm_bwd_blocks(c->dims[lvl].count(), L.c) * 2 * L.c;
}

void layout_buffers(d2ip_ctx* c, Carve& cv) {
  const int B = c->B;
  const auto& w = c->w;
  const auto nv = [&](int l) { return c->dims[l].count(); };
  c->theta = cv.take<float>(B * c->Pp);
  c->grad = cv.take<float>(B * c->Pp);
  c->am = cv.take<float>(B * c->Pp);
  c->av = cv.take<float>(B * c->Pp);
  c->zin = cv.take<float>(B * nv(0) * c->c_in);
  c->dsigma = cv.take<float>(B * nv(0));
  c->gds = cv.take<float>(B * nv(0));
  c->stage = cv.take<float>(B * nv(0));
  if (c->arch == 1) {
    float* frm = cv.take<float>(c->fr.arena_floats(B));
    if (!cv.dry) c->fr.bind(frm, B, c->zin, c->dsigma, c->gds);
    c->ws = nullptr;
    c->ws_floats = 0;
  } else {
    long long maxz = 0;
    for (int l = 0; l < c->L; ++l) maxz = std::max(maxz, nv(l) * w[l]);
    c->ztmp = cv.take<float>(B * maxz);
    c->ptmp = cv.take<float>(B * maxz);
    auto unit_bufs = [&](Unit& u) {
      const long long n = nv(u.lvl_out);
      u.xh = cv.take<float>(B * n * u.ln.c);
      u.rs = cv.take<float>(B * n);
      u.a = cv.take<float>(B * n * u.ln.c);
    };
    auto res_bufs = [&](Res& R) {
      const long long n = nv(R.lvl);
      const int co = R.lna.c;
      R.xh_a = cv.take<float>(B * n * co);
      R.rs_a = cv.take<float>(B * n);
      R.h1 = cv.take<float>(B * n * co);
      R.xh_b = cv.take<float>(B * n * co);
      R.rs_b = cv.take<float>(B * n);
      R.out = cv.take<float>(B * n * co);
    };
    unit_bufs(c->stem);
    for (int l = 0; l < c->L; ++l) {
      if (l > 0) unit_bufs(c->down[l]);
      res_bufs(c->enc[l]);
    }
    for (int l = 0; l + 1 < c->L; ++l) res_bufs(c->dec[l]);
    c->lb.assign(c->L, LevelBufs{});
    for (int l = 0; l < c->L; ++l) {
      const long long cmax = w[l] + (l + 1 < c->L ? w[l + 1] : 0);
      LevelBufs& L = c->lb[l];
      L.g1 = cv.take<float>(B * nv(l) * cmax);
      L.g2 = cv.take<float>(B * nv(l) * cmax);
      L.tz = cv.take<float>(B * nv(l) * w[l]);
      L.tt = cv.take<float>(B * nv(l) * w[l]);
      L.th = cv.take<float>(B * nv(l) * w[l]);
      L.de = cv.take<float>(B * nv(l) * w[l]);
      if (l + 1 < c->L) L.cat = cv.take<float>(B * nv(l) * cmax);
    }
    // wiring of block inputs
    c->stem.x = c->zin;
    c->enc[0].x = c->stem.a;
    for (int l = 1; l < c->L; ++l) {
      c->down[l].x = c->enc[l - 1].out;
      c->enc[l].x = c->down[l].a;
    }
    for (int l = 0; l + 1 < c->L; ++l) c->dec[l].x = c->lb[l].cat;
    // workspace: the largest split-K / LayerNorm partial buffer of any layer
    long long ws = conv_ws_floats(c, c->stem.conv);
    ws = std::max(ws, ln_ws_floats(c, c->stem.ln, 0));
    auto res_ws = [&](const Res& R) {
      ws = std::max(ws, conv_ws_floats(c, R.a));
      if (R.fuse_w)
        ws = std::max(ws, conv_ws_floats(c, R.a) +
                              (long long)c->B * wgrad_rows(c, R.a) * (R.p.wcount() + R.p.co));
      ws = std::max(ws, conv_ws_floats(c, R.b));
      if (R.proj) ws = std::max(ws, conv_ws_floats(c, R.p));
      ws = std::max(ws, ln_ws_floats(c, R.lna, R.lvl));
      ws = std::max(ws, ln_ws_floats(c, R.lnb, R.lvl));
    };
    for (int l = 0; l < c->L; ++l) {
      res_ws(c->enc[l]);
      if (l > 0) {
        ws = std::max(ws, conv_ws_floats(c, c->down[l].conv));
        ws = std::max(ws, ln_ws_floats(c, c->down[l].ln, l));
      }
    }
    for (int l = 0; l + 1 < c->L; ++l) res_ws(c->dec[l]);
    // the LayerNorm backward fused into a data gradient: (dgamma, dbeta) rows per slice
    for (const TcLayer& T : c->bf.layers)
      if (T.dgrad && T.s == 1)
        ws = std::max(ws, (long long)B * ceil_div(T.din.x, 8) * ceil_div(T.din.y, 16) *
                              (T.din.z + 7) * 2 * T.ci);
    ws = std::max(ws, conv_ws_floats(c, c->tail));
    c->ws_floats = ws;
    c->ws = cv.take<float>(ws);
  }
  c->loss = cv.take<double>(B);
  c->resid = cv.take<double>(B);
  c->trace = cv.take<double>((long long)kTraceCap * B);
  c->trace_pos = cv.take<int>(1);
  c->adam_t = cv.take<int>(1);
  c->status = cv.take<int>(1);
  c->nprev = cv.take<int>(1);
  c->reg_part = cv.take<double>((long long)B * tv4d_blocks(nv(0)));
  if (c->precision != D2IP_FP32) {
    long long max_act = 0;
    for (int l = 0; l < c->L; ++l)
      max_act = std::max(max_act, nv(l) * (w[l] + (l + 1 < c->L ? w[l + 1] : 0)));
    bf16_layout(c->bf, cv.dry ? nullptr : cv.base, cv.used, B, max_act);
  }
}

d2ip_status ensure_arena(d2ip_ctx* c) {
  if (c->arena) return D2IP_OK;
  Carve dry{nullptr, 0, true};
  layout_buffers(c, dry);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, dry.used);
  if (e != cudaSuccess) return fail(c, D2IP_ERR_OOM, "device allocation of the workspace failed");
  c->arena = p;
  c->arena_bytes = dry.used;
  Carve real{static_cast<char*>(p), 0, false};
  layout_buffers(c, real);
  CK(cudaMemsetAsync(p, 0, dry.used, c->stream));
  if (c->precision != D2IP_FP32) {
    CK(bf16_finalize(c->bf, c->B));
    if (!c->tile_rows.empty()) {  // a saved plan replaces the sweep
      const cudaError_t e = bf16_apply_plan(c->bf, c->B, c->tile_rows.data(),
                                            (int)(c->tile_rows.size() / 15));
      if (e == cudaErrorInvalidValue)
        return fail(c, D2IP_ERR_BAD_ARG, "the stored tile plan does not fit this network");
      if (e != cudaSuccess) return cuda_fail(c, e, "applying the stored tile plan");
      CK(bf16_finalize(c->bf, c->B));
    } else if (c->autotune) {  // on the arena's own (zeroed) buffers, outputs to a scratch buffer
      float* scratch = nullptr;
      const size_t bytes = sizeof(float) * (size_t)bf16_tune_scratch_floats(c->bf, c->B);
      if (cudaMalloc(&scratch, bytes) != cudaSuccess)
        return fail(c, D2IP_ERR_OOM, "device allocation of the autotuner scratch failed");
      cudaError_t e = bf16_autotune(c->bf, c->B, scratch, c->theta, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      cudaFree(scratch);
      if (e != cudaSuccess) return cuda_fail(c, e, "autotuning the tensor-core tilings");
      CK(bf16_finalize(c->bf, c->B));
      int tc = 0;
      CK(cudaMemcpy(&tc, c->bf.err, sizeof(int), cudaMemcpyDeviceToHost));
      if (tc) return fail(c, D2IP_ERR_TIMEOUT, "a tensor-core kernel timed out while autotuning");
    }
  }
  return D2IP_OK;
}

// ------------------------------------------------------------------------------------
// launch sequences
// ------------------------------------------------------------------------------------
// Optional per-launch CUDA-event tracing (d2ip_profile_iterations).
struct Tracer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cls;
  std::vector<double> work;
  size_t used = 0;
  cudaError_t begin(int k, double w, cudaStream_t s) {
    if (used + 2 > pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        pool.push_back(e);
      }
    }
    cls.push_back(k);
    work.push_back(w);
    return cudaEventRecord(pool[used++], s);
  }
  cudaError_t end(cudaStream_t s) { return cudaEventRecord(pool[used++], s); }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    cls.clear();
    work.clear();
    used = 0;
  }
};

struct Launcher {
  d2ip_ctx* c;
  Tracer* tr = nullptr;
  cudaError_t e = cudaSuccess;
  // BF16 staging done by producers (BF16 precision): layers whose kept input copy the
  // producing kernel wrote this pass, the layer whose dy sits in the dy staging buffer, and
  // the block whose projection dy sits in the projection staging buffer.
  std::vector<const ConvL*> staged_x;
  const ConvL* dy_owner[2] = {nullptr, nullptr};  // the layer whose dy each staging slot holds
  const void* pbf_owner = nullptr;
  __nv_bfloat16* bf_in(const ConvL* L) {
    return L && L->tc >= 0 && c->precision != D2IP_FP32 ? bf16_input_buffer(c->bf, L->tc)
                                                        : nullptr;
  }
  bool take_staged(const ConvL& L) {
    auto it = std::find(staged_x.begin(), staged_x.end(), &L);
    if (it == staged_x.end()) return false;
    staged_x.erase(it);
    return true;
  }
  bool tc_dy_consumer(const ConvL* L) {
    return L && L->tc >= 0 && c->precision != D2IP_FP32 &&
           (c->bf.layers[L->tc].dgrad || c->bf.layers[L->tc].wgrad);
  }
  int dy_slot(const ConvL& L) const { return L.tc >= 0 ? c->bf.layers[L.tc].dyslot : 0; }
  bool dy_staged(const ConvL& L) const { return dy_owner[dy_slot(L)] == &L; }
  void own_dy(const ConvL& L) { dy_owner[dy_slot(L)] = &L; }
  void ok(cudaError_t x) {
    if (e == cudaSuccess) e = x;
  }
  // bracket one kernel launch of class k with algorithmic work w (FLOPs or bytes)
  void beg(int k, double w) {
    if (tr) ok(tr->begin(k, w, c->stream));
  }
  void fin() {
    if (tr) ok(tr->end(c->stream));
  }
  float* W(const ConvL& L) { return c->theta + L.w_off; }
  float* G(long long off) { return c->grad + off; }
  double conv_flops(const ConvL& L) const {
    return 2.0 * c->B * (double)L.dout.count() * L.k * L.k * L.k * L.ci * L.co;
  }

  // staged: x already sits in the layer's BF16 input (another layer's kept copy of it)
  void conv_fwd(const ConvL& L, const float* x, float* y, bool staged = false) {
    beg(D2IP_KCLASS_CONV_FWD, conv_flops(L));
    if (L.tc >= 0) {
      ok(bf16_conv_fwd(c->bf, L.tc, x, W(L) + L.wcount(), y, c->B, c->Pp, c->stream,
                       take_staged(L) || staged));
    } else {
      ok(conv3d_fwd_f32(x, W(L), W(L) + L.wcount(), y, c->B, L.din, L.ci, L.co, L.k, L.s,
                        L.din.count() * L.ci, L.dout.count() * L.co, c->Pp, c->stream));
    }
    fin();
  }
  void conv_dgrad(const ConvL& L, const float* dy, float* dx, int acc) {
    beg(D2IP_KCLASS_CONV_DGRAD, conv_flops(L));
    if (L.tc >= 0 && c->bf.layers[L.tc].dgrad) {
      ok(bf16_conv_dgrad(c->bf, L.tc, dy, dx, c->B, acc, c->stream, dy_staged(L)));
      own_dy(L);  // dy now sits in the staging buffer
    } else
      ok(conv3d_dgrad_f32(dy, W(L), dx, c->B, L.din, L.ci, L.co, L.k, L.s,
                          L.dout.count() * L.co, L.din.count() * L.ci, c->Pp, acc, c->stream));
    fin();
  }
  // x: the forward of this iteration staged it; dy: staged when this layer owns the buffer
  void conv_wgrad(const ConvL& L, const float* x, const float* dy) {
    beg(D2IP_KCLASS_CONV_WGRAD, conv_flops(L));
    if (tc_wgrad(c, L))
      ok(bf16_conv_wgrad(c->bf, L.tc, x, dy, c->ws, c->B, c->stream, nullptr, nullptr, true,
                         dy_staged(L)));
    else
      ok(conv3d_wgrad_partial_f32(x, dy, c->ws, c->B, L.din, L.ci, L.co, L.k, L.s,
                                  L.din.count() * L.ci, L.dout.count() * L.co, c->stream));
    ok(reduce_rows_f32(c->ws, G(L.w_off), c->B, wgrad_rows(c, L), L.wcount() + L.co, c->Pp, 0,
                       c->stream));
    fin();
  }
  // consumer: the tensor-core convolution that reads y next (its BF16 input is written here)
  void ln_fwd(const LnL& L, int lvl, const float* z, const float* resid, float* y, float* xh,
              float* rs, const ConvL* consumer = nullptr) {
    const double nv = (double)c->dims[lvl].count() * c->B;
    beg(D2IP_KCLASS_LN_FWD, 4.0 * nv * (L.c * (resid ? 4 : 3) + 1));
    __nv_bfloat16* ybf = bf_in(consumer);
    ok(layernorm_act_fwd_f32(z, c->theta + L.g_off, resid, y, xh, rs, c->B,
                             c->dims[lvl].count(), L.c, 1, c->Pp, c->stream, ybf, c->bf.sp));
    if (ybf) staged_x.push_back(consumer);
    fin();
  }
  // dz_consumer: the convolution whose output gradient dz is (dz also goes to the dy staging
  // buffer); dt_owner: the block whose fused projection reads dt (dt also goes to its buffer)
  void ln_bwd(const LnL& L, int lvl, const float* dy, const float* aout, const float* xh,
              const float* rs, float* dz, float* dt, const ConvL* dz_consumer = nullptr,
              const void* dt_owner = nullptr) {
    const long long nv = c->dims[lvl].count();
    beg(D2IP_KCLASS_LN_BWD, 4.0 * c->B * nv * (L.c * (dt ? 5 : 4) + 1));
    __nv_bfloat16* dzbf =
        tc_dy_consumer(dz_consumer) ? bf16_dy_buffer(c->bf, dz_consumer->tc) : nullptr;
    __nv_bfloat16* dtbf = dt && dt_owner && c->bf.pbf ? c->bf.pbf : nullptr;
    // dz in FP32 only when the consumer reads it so: a data gradient off the tensor cores (a
    // layer that needs one) or a weight gradient off them
    const bool fp32_dz = !dzbf ||
                         (!c->bf.layers[dz_consumer->tc].dgrad &&
                          !c->bf.layers[dz_consumer->tc].input_layer) ||
                         !tc_wgrad(c, *dz_consumer);
    ok(layernorm_act_bwd_f32(dy, aout, xh, rs, c->theta + L.g_off, fp32_dz ? dz : nullptr, dt,
                             c->ws, c->B, nv, L.c, c->Pp, c->stream, dzbf, dtbf, c->bf.sp));
    if (dzbf) own_dy(*dz_consumer);
    if (dtbf) pbf_owner = dt_owner;
    ok(reduce_rows_f32(c->ws, G(L.g_off), c->B, layernorm_bwd_blocks(nv, L.c), 2 * L.c, c->Pp,
                       0, c->stream));
    fin();
  }

  // act(LN(conv(x)) (+ resid)) with the LayerNorm in the epilogue of the persistent halo
  // convolution (z never stored), when the layer runs that kernel; with proj (a decoder
  // block's conv a) the fused 1x1 projection's output goes to ptmp.  False: not fused.
  bool conv_ln_fused(const ConvL& L, const LnL& ln, const float* x, const float* resid,
                     float* y, float* xh, float* rs, const ConvL* consumer, const Res* proj) {
    if (L.tc < 0 || c->precision == D2IP_FP32 ||
        !bf16_fwd_ln_ok(c->bf, L.tc, proj ? proj->p.co : 0, c->bf.sp))
      return false;
    beg(D2IP_KCLASS_CONV_FWD, conv_flops(L) + (proj ? conv_flops(proj->p) : 0.0));
    __nv_bfloat16* ybf = bf_in(consumer);
    Bf16Ln l{};
    l.gamma = c->theta + ln.g_off, l.gamma_bs = c->Pp;
    l.resid = resid, l.xhat = xh, l.rstd = rs, l.ybf = ybf, l.act = 1;
    ok(bf16_conv_fwd_ln(c->bf, L.tc, x, W(L) + L.wcount(), y, l, c->B, c->Pp, c->stream,
                        take_staged(L), proj ? W(proj->p) + proj->p.wcount() : nullptr,
                        proj ? c->ptmp : nullptr));
    if (ybf) staged_x.push_back(consumer);
    fin();
    return true;
  }
  // next: the convolution that reads the unit's (block's) output
  void unit_fwd(Unit& u, const ConvL* next) {
    if (conv_ln_fused(u.conv, u.ln, u.x, nullptr, u.a, u.xh, u.rs, next, nullptr)) return;
    conv_fwd(u.conv, u.x, c->ztmp);
    ln_fwd(u.ln, u.lvl_out, c->ztmp, nullptr, u.a, u.xh, u.rs, next);
  }
  void res_fwd(Res& R, const ConvL* next) {
    if (!conv_ln_fused(R.a, R.lna, R.x, nullptr, R.h1, R.xh_a, R.rs_a, &R.b,
                       R.fuse_f ? &R : nullptr)) {
      if (R.fuse_f) {  // conv a and the projection in one launch
        beg(D2IP_KCLASS_CONV_FWD, conv_flops(R.a) + conv_flops(R.p));
        ok(bf16_conv_fwd_proj(c->bf, R.a.tc, R.x, W(R.a) + R.a.wcount(), c->ztmp,
                              W(R.p) + R.p.wcount(), c->ptmp, c->B, c->Pp, c->stream,
                              take_staged(R.a)));
        fin();
      } else {
        conv_fwd(R.a, R.x, c->ztmp);
      }
      ln_fwd(R.lna, R.lvl, c->ztmp, nullptr, R.h1, R.xh_a, R.rs_a, &R.b);
    }
    if (R.proj && !R.fuse_f)  // reading conv a's kept input where it shares it (staged now)
      conv_fwd(R.p, R.x, c->ptmp, R.p.tc >= 0 && bf16_input_shared(c->bf, R.p.tc));
    const float* resid = R.proj ? c->ptmp : R.x;
    if (conv_ln_fused(R.b, R.lnb, R.h1, resid, R.out, R.xh_b, R.rs_b, next, nullptr)) return;
    conv_fwd(R.b, R.h1, c->ztmp);
    ln_fwd(R.lnb, R.lvl, c->ztmp, resid, R.out, R.xh_b, R.rs_b, next);
  }
  static void tr_beg(void* u, int k, double w) { static_cast<Launcher*>(u)->beg(k, w); }
  static void tr_fin(void* u) { static_cast<Launcher*>(u)->fin(); }
  FrRun fr_run() {
    FrRun r{c->theta, c->grad, c->Pp, c->stream};
    if (tr) {
      r.beg = tr_beg;
      r.fin = tr_fin;
      r.user = this;
    }
    return r;
  }
  void forward() {
    if (c->arch == 1) {
      ok(c->fr.forward(fr_run()));
      return;
    }
    if (c->precision != D2IP_FP32)
      ok(bf16_prepare_weights(c->bf, c->theta, c->B, c->Pp, c->stream));
    staged_x.clear();
    unit_fwd(c->stem, &c->enc[0].a);
    res_fwd(c->enc[0], c->L > 1 ? &c->down[1].conv : nullptr);
    for (int l = 1; l < c->L; ++l) {
      unit_fwd(c->down[l], &c->enc[l].a);
      res_fwd(c->enc[l], l + 1 < c->L ? &c->down[l + 1].conv : nullptr);
    }
    const float* cur = c->enc[c->L - 1].out;
    for (int l = c->L - 2; l >= 0; --l) {
      __nv_bfloat16* catbf = bf_in(&c->dec[l].a);
      // the FP32 concatenation only where a consumer reads it (not the tensor-core block
      // whose layers all take the BF16 copy)
      const bool cat32 = !catbf || !bf16_only_input(c, c->dec[l]);
      const double fine = (double)c->dims[l].count() * (c->w[l] + c->w[l + 1]);
      const double bytes = c->B * (4.0 * ((double)c->dims[l + 1].count() * c->w[l + 1] +
                                          (double)c->dims[l].count() * c->w[l]) +
                                   (cat32 ? 4.0 * fine : 0.0) +
                                   (catbf ? 2.0 * c->bf.sp * fine : 0.0));
      beg(D2IP_KCLASS_UP_FWD, bytes);
      ok(upsample_concat_fwd_f32(cur, c->enc[l].out, cat32 ? c->lb[l].cat : nullptr, c->B,
                                 c->dims[l + 1], c->dims[l], c->w[l + 1], c->w[l], c->stream,
                                 catbf, c->bf.sp));
      if (catbf) staged_x.push_back(&c->dec[l].a);
      fin();
      res_fwd(c->dec[l], nullptr);
      cur = c->dec[l].out;
    }
    if (co1_layer(c->tail)) {
      beg(D2IP_KCLASS_CONV_FWD, conv_flops(c->tail));
      ok(conv1x1_co1_fwd_f32(cur, W(c->tail), c->dsigma, c->B, c->tail.din.count(), c->tail.ci,
                             c->Pp, c->stream));
      fin();
    } else {
      conv_fwd(c->tail, cur, c->dsigma);
    }
  }
  void data_term(bool training) {
    const long long n = c->n();
    const bool jb16 = c->precision != D2IP_FP32;  // transposed BF16 J (hi, + lo when split)
    const double jb = (c->precision == D2IP_BF16 ? 2.0 : 4.0) * c->m * (double)n,
                 vb = 4.0 * c->B * ((double)n + 2.0 * c->m);
    beg(D2IP_KCLASS_JMUL, jb + vb);
    if (jb16 && c->jp_stage)
      ok(jprod_tc_residual(c->jp, c->dsigma, n, c->dv, c->r, c->jpart, c->bf.err, c->stream));
    else if (jb16)
      ok(jmul_residual_bf16(c->Jbf, c->dsigma, c->dv, c->r, c->jpart, c->B, c->m, (int)n, n,
                            c->stream, c->Jlo));
    else
      ok(jmul_residual_f32(c->J, c->dsigma, c->dv, c->r, c->jpart, c->B, c->m, (int)n, n,
                           c->stream));
    fin();
    if (training) {
      beg(D2IP_KCLASS_JTMUL, jb + vb);
      if (jb16 && c->jp_stage)
        ok(jprod_tc_adjoint(c->jp, c->gds, 2.0f / (float)c->m, n, c->bf.err, c->stream));
      else if (jb16)
        ok(jtmul_bf16(c->Jbf, c->r, c->gds, 2.0f / (float)c->m, c->B, c->m, (int)n, n,
                      c->stream, c->Jlo));
      else
        ok(jtmul_f32(c->J, c->r, c->gds, 2.0f / (float)c->m, c->B, c->m, (int)n, n, c->stream));
      fin();
    }
    const bool reg = training && c->lam_tv != 0.0;
    if (reg) {  // 4D-TV (Sec. III-E): value into the loss, gradient into dL/d dsigma
      beg(D2IP_KCLASS_MISC, 4.0 * c->B * (double)n * 8);
      ok(tv4d_f32(c->dsigma, c->hist, c->nprev, c->gds, c->reg_part, c->B, c->dims[0],
                  (long long)c->hist_cap * n, (float)(c->lam_tv * c->lam_s / (double)n),
                  (float)(c->lam_tv * c->lam_t), (float)c->tv_eps, c->stream));
      fin();
    }
    beg(D2IP_KCLASS_LOSS, 4.0 * c->B * c->m);
    if (training) {
      ok(residual_loss_f64(c->r, c->loss, c->trace, c->trace_pos, kTraceCap, c->adam_t,
                           c->status, c->B, c->m, c->stream, reg ? c->reg_part : nullptr,
                           reg ? tv4d_blocks(n) : 0));
    } else {
      ok(residual_loss_f64(c->r, c->resid, nullptr, nullptr, 0, nullptr, c->status, c->B, c->m,
                           c->stream));
    }
    fin();
  }
  // The data gradient of L (dy: its output gradient) with the LayerNorm (+ LeakyReLU)
  // backward of the block whose output (aout, saved xh, rs) is L's input, in the epilogue of
  // the persistent halo kernel: dz of that block goes to consumer's dy staging, (dgamma,
  // dbeta) to the gradient; resid: a gradient already accumulated for L's input.  False
  // (nothing launched) where the fused form does not apply.
  bool dgrad_ln(const ConvL& L, const float* dy, const LnL& ln, const float* resid,
                const float* aout, const float* xh, const float* rs, const ConvL* consumer) {
    if (!c->ln_bwd_fused || L.tc < 0 || c->precision == D2IP_FP32 ||
        !c->bf.layers[L.tc].dgrad ||
        ln.c != L.ci || !tc_dy_consumer(consumer) || dy_slot(L) == dy_slot(*consumer) ||
        !bf16_dgrad_ln_ok(c->bf, L.tc, c->bf.sp))
      return false;
    const long long rows = bf16_dgrad_ln_rows(c->bf, L.tc);
    if ((long long)c->B * rows * 2 * ln.c > c->ws_floats) return false;
    beg(D2IP_KCLASS_CONV_DGRAD, conv_flops(L));
    Bf16Ln l{};
    l.gamma = c->theta + ln.g_off, l.gamma_bs = c->Pp;
    l.resid = resid, l.xhat = const_cast<float*>(xh), l.rstd = const_cast<float*>(rs);
    l.ybf = bf16_dy_buffer(c->bf, consumer->tc), l.act = 1;
    l.bwd = 1, l.aout = aout, l.part = c->ws;
    ok(bf16_conv_dgrad_ln(c->bf, L.tc, dy, nullptr, l, c->B, c->stream, dy_staged(L)));
    own_dy(L);
    own_dy(*consumer);
    ok(reduce_rows_f32(c->ws, G(ln.g_off), c->B, rows, 2 * ln.c, c->Pp, 0, c->stream));
    fin();
    return true;
  }
  // dout: gradient of R.out; writes dx (gradient of R.x).  Without a projection the residual
  // gradient dt goes straight into dx and conv a's data gradient adds onto it; then, when
  // next (the unit whose output is R.x) can take it, next's LayerNorm backward runs in that
  // data gradient's epilogue instead (dx is not stored) and true is returned.
  // dskip / split (a decoder block): with the fused projection's data gradient, its input
  // gradient is stored split, the first `split` channels (the up-sampled part) into dx and the
  // rest (the skip part) into dskip; *split_done reports it.
  bool res_bwd(Res& R, const float* dout, float* dx, Unit* next = nullptr, float* dskip = nullptr,
               int split = 0, bool* split_done = nullptr) {
    LevelBufs& T = c->lb[R.lvl];
    ln_bwd(R.lnb, R.lvl, dout, R.out, R.xh_b, R.rs_b, T.tz, R.proj ? T.tt : dx, &R.b,
           R.fuse_d || R.fuse_w ? &R : nullptr);
    if (dgrad_ln(R.b, T.tz, R.lna, nullptr, R.h1, R.xh_a, R.rs_a, &R.a)) {
      conv_wgrad(R.b, R.h1, T.tz);
    } else {
      conv_dgrad(R.b, T.tz, T.th, 0);
      conv_wgrad(R.b, R.h1, T.tz);
      ln_bwd(R.lna, R.lvl, T.th, R.h1, R.xh_a, R.rs_a, T.tz, nullptr, &R.a);
    }
    bool next_done = false;
    if (R.fuse_d) {  // dx = conv_a^T(dz_a) + W_p^T dz_p in one launch
      beg(D2IP_KCLASS_CONV_DGRAD, conv_flops(R.a) + conv_flops(R.p));
      const bool sp = dskip && split > 0;
      ok(bf16_conv_dgrad_proj(c->bf, R.a.tc, T.tz, T.tt, dx, c->B, c->stream,
                              dy_staged(R.a), pbf_owner == &R, sp ? dskip : nullptr,
                              sp ? split : 0));
      if (split_done) *split_done = sp;
      own_dy(R.a);
      pbf_owner = &R;
      fin();
    } else if (next && !R.proj &&
               dgrad_ln(R.a, T.tz, next->ln, dx, next->a, next->xh, next->rs, &next->conv)) {
      next_done = true;
    } else {
      conv_dgrad(R.a, T.tz, dx, R.proj ? 0 : 1);
    }
    if (R.fuse_w) {  // weight gradients of conv a and the projection in one launch
      const long long rows = wgrad_rows(c, R.a);
      float* part_p = c->ws + (long long)c->B * rows * (R.a.wcount() + R.a.co);
      beg(D2IP_KCLASS_CONV_WGRAD, conv_flops(R.a) + conv_flops(R.p));
      ok(bf16_conv_wgrad(c->bf, R.a.tc, R.x, T.tz, c->ws, c->B, c->stream, T.tt, part_p, true,
                         dy_staged(R.a)));
      ok(reduce_rows_f32(c->ws, G(R.a.w_off), c->B, rows, R.a.wcount() + R.a.co, c->Pp, 0,
                         c->stream));
      ok(reduce_rows_f32(part_p, G(R.p.w_off), c->B, rows, R.p.wcount() + R.p.co, c->Pp, 0,
                         c->stream));
      fin();
    } else {
      conv_wgrad(R.a, R.x, T.tz);
    }
    if (R.proj) {
      if (!R.fuse_d) conv_dgrad(R.p, T.tt, dx, 1);
      if (!R.fuse_w) conv_wgrad(R.p, R.x, T.tt);
    }
    return next_done;
  }
  // ln_done: the unit's LayerNorm backward already ran (dz staged for u.conv)
  void unit_bwd(Unit& u, const float* da, float* dx, int acc, bool dgrad, bool ln_done = false) {
    float* tz = c->lb[u.lvl_out].tz;
    if (!ln_done) ln_bwd(u.ln, u.lvl_out, da, u.a, u.xh, u.rs, tz, nullptr, &u.conv);
    if (dgrad) conv_dgrad(u.conv, tz, dx, acc);
    conv_wgrad(u.conv, u.x, tz);
  }
  void backward() {
    if (c->arch == 1) {
      ok(c->fr.backward(fr_run()));
      return;
    }
    dy_owner[0] = dy_owner[1] = nullptr;
    pbf_owner = nullptr;
    const int L = c->L;
    const float* tail_in = L > 1 ? c->dec[0].out : c->enc[0].out;
    if (co1_layer(c->tail)) {  // data and weight gradients of the last layer in one pass
      const ConvL& T = c->tail;
      beg(D2IP_KCLASS_CONV_WGRAD, 2.0 * conv_flops(T));
      ok(conv1x1_co1_bwd_f32(tail_in, c->gds, W(T), c->lb[0].g1, c->ws, c->B, T.din.count(), T.ci,
                             c->Pp, 0, c->stream));
      ok(reduce_rows_f32(c->ws, G(T.w_off), c->B, wgrad_rows(c, T), T.wcount() + T.co, c->Pp, 0,
                         c->stream));
      fin();
    } else {
      conv_dgrad(c->tail, c->gds, c->lb[0].g1, 0);
      conv_wgrad(c->tail, tail_in, c->gds);
    }
    for (int l = 0; l + 1 < L; ++l) {
      bool split = false;  // the skip part already in de, g2 holds the up-sampled part only
      res_bwd(c->dec[l], c->lb[l].g1, c->lb[l].g2, nullptr, c->lb[l].de, c->w[l + 1], &split);
      const double bytes = 4.0 * c->B *
                           ((double)c->dims[l + 1].count() * c->w[l + 1] +
                            2.0 * c->dims[l].count() * c->w[l] +
                            (double)c->dims[l].count() * c->w[l + 1]);
      beg(D2IP_KCLASS_UP_BWD, bytes);
      ok(upsample_concat_bwd_f32(c->lb[l].g2, c->lb[l + 1].g1, split ? nullptr : c->lb[l].de,
                                 c->B, c->dims[l + 1], c->dims[l], c->w[l + 1],
                                 split ? 0 : c->w[l], c->stream));
      fin();
    }
    for (int l = L - 1; l >= 1; --l) {
      const float* dout = l == L - 1 ? c->lb[l].g1 : c->lb[l].de;
      const bool done = res_bwd(c->enc[l], dout, c->lb[l].g2, &c->down[l]);
      unit_bwd(c->down[l], c->lb[l].g2, c->lb[l - 1].de, 1, true, done);
    }
    const float* d0 = L == 1 ? c->lb[0].g1 : c->lb[0].de;
    const bool done0 = res_bwd(c->enc[0], d0, c->lb[0].g2, &c->stem);
    unit_bwd(c->stem, c->lb[0].g2, nullptr, 0, false, done0);
  }
  void adam() {
    beg(D2IP_KCLASS_ADAM, 28.0 * c->B * c->P);
    ok(adam_step_f32(c->theta, c->grad, c->am, c->av, (long long)c->B * c->Pp, c->lr,
                     c->beta1, c->beta2, c->eps, c->adam_t, 0, c->stream));
    fin();
  }
};

d2ip_status capture(d2ip_ctx* c, bool step, cudaGraphExec_t* out) {
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  Launcher Lr{c};
  Lr.forward();
  Lr.data_term(step);
  if (step) {
    Lr.backward();
    Lr.adam();
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (Lr.e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, Lr.e, "kernel launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  size_t nn = 0;
  e = cudaGraphGetNodes(g, nullptr, &nn);
  long long nk = 0;
  if (e == cudaSuccess && nn) {
    std::vector<cudaGraphNode_t> nodes(nn);
    e = cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(c, e, "cudaGraphGetNodes");
  }
  (step ? c->step_kernels : c->eval_kernels) = nk;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return D2IP_OK;
}

d2ip_status ready(d2ip_ctx* c) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->net_ready || !c->X) return fail(c, D2IP_ERR_STATE, "grid and network not set");
  if (!c->j_ready) return fail(c, D2IP_ERR_STATE, "J not loaded");
  if (!c->input_ready) return fail(c, D2IP_ERR_STATE, "input Z and theta0 not set");
  CK(cudaSetDevice(c->device));
  if (!c->g_step) {
    d2ip_status s = capture(c, true, &c->g_step);
    if (s) return s;
  }
  if (!c->g_eval) {
    d2ip_status s = capture(c, false, &c->g_eval);
    if (s) return s;
  }
  return D2IP_OK;
}

d2ip_status check_status(d2ip_ctx* c) {
  int st = 0, tc = 0;
  CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (c->precision != D2IP_FP32 && c->bf.err)
    CK(cudaMemcpyAsync(&tc, c->bf.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (tc) {
    CK(cudaMemsetAsync(c->bf.err, 0, sizeof(int), c->stream));
    return fail(c, D2IP_ERR_TIMEOUT,
                "a tensor-core convolution gave up waiting on its pipeline (code " +
                    std::to_string(tc) + ")");
  }
  if (st & 1) {
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    return fail(c, D2IP_ERR_NONFINITE, "a loss or residual became NaN or Inf");
  }
  return D2IP_OK;
}

// copy rows: dst[b*dpitch ..] <- src[b*spitch ..], `width` floats, B rows (host or device)
cudaError_t copy_rows(void* dst, long long dpitch, const void* src, long long spitch,
                      long long width, int rows, size_t elem, cudaStream_t s) {
  return cudaMemcpy2DAsync(dst, dpitch * elem, src, spitch * elem, width * elem, rows,
                           cudaMemcpyDefault, s);
}

d2ip_status reset_optimizer(d2ip_ctx* c) {
  CK(cudaMemsetAsync(c->am, 0, sizeof(float) * c->B * c->Pp, c->stream));
  CK(cudaMemsetAsync(c->av, 0, sizeof(float) * c->B * c->Pp, c->stream));
  CK(cudaMemsetAsync(c->adam_t, 0, sizeof(int), c->stream));
  return D2IP_OK;
}

d2ip_status run_steps(d2ip_ctx* c, int n_steps, double* loss_trace) {
  int done = 0;
  while (done < n_steps) {
    const int chunk = std::min(kTraceCap, n_steps - done);
    CK(cudaMemsetAsync(c->trace_pos, 0, sizeof(int), c->stream));
    for (int i = 0; i < chunk; ++i) CK(cudaGraphLaunch(c->g_step, c->stream));
    if (loss_trace)
      CK(cudaMemcpyAsync(loss_trace + (long long)done * c->B, c->trace,
                         sizeof(double) * chunk * c->B, cudaMemcpyDefault, c->stream));
    done += chunk;
  }
  return D2IP_OK;
}

d2ip_status stage_dv(d2ip_ctx* c, const float* dV, long long spitch) {
  CK(copy_rows(c->dv, c->m, dV, spitch, c->m, c->B, sizeof(float), c->stream));
  return D2IP_OK;
}

}  // namespace

namespace {

// One context's sequence as a list of operations, issued a few graph launches at a time.
struct SeqOp {
  enum Kind { kStage, kReset, kSteps, kEval, kResiduals, kPrev, kSave } kind;
  int arg;                 // frame index (kStage: -1 = the UPWS frame), step count
};

struct SeqJob {
  d2ip_ctx* c = nullptr;
  const float* V = nullptr;
  const float* dV0 = nullptr;
  float* Sigma = nullptr;
  double* resid = nullptr;
  int T = 0;
  std::vector<SeqOp> ops;
  size_t pc = 0;
  int done_steps = 0;      // of the current kSteps op
};

SeqJob make_sequence_job(d2ip_ctx* c, const float* V, int T, const float* dV0, int upws,
                         int first, int later, float* Sigma, double* resid) {
  SeqJob j;
  j.c = c;
  j.V = V;
  j.T = T;
  j.dV0 = dV0;
  j.Sigma = Sigma;
  j.resid = resid;
  const bool reg = c->lam_tv != 0.0;
  if (reg) j.ops.push_back({SeqOp::kPrev, 0});
  // (with the carried-state option the Adam state restarts once, at the sequence's start)
  if (upws > 0) {  // UPWS (Eqs. 5-7): N_0 steps on one frame from the initial weights
    j.ops.push_back({SeqOp::kStage, -1});
    j.ops.push_back({SeqOp::kReset, 0});
    j.ops.push_back({SeqOp::kSteps, upws});
  }
  for (int i = 0; i < T; ++i) {  // TPP (Eqs. 8-9): theta carries over, Adam restarts
    j.ops.push_back({SeqOp::kStage, i});
    if (c->frame_reset || (i == 0 && upws == 0)) j.ops.push_back({SeqOp::kReset, 0});
    j.ops.push_back({SeqOp::kSteps, i == 0 ? first : later});
    j.ops.push_back({SeqOp::kEval, i});
    if (reg) {  // the temporal term of frame i + 1 sees frames 0..i
      j.ops.push_back({SeqOp::kSave, i});
      j.ops.push_back({SeqOp::kPrev, i + 1});
    }
  }
  j.ops.push_back({SeqOp::kResiduals, 0});
  return j;
}

// Issue the job's next operations, at most `budget` step graphs.
d2ip_status issue(SeqJob& j, int budget) {
  d2ip_ctx* c = j.c;
  const long long m = c->m, n = c->n();
  while (j.pc < j.ops.size()) {
    const SeqOp& op = j.ops[j.pc];
    switch (op.kind) {
      case SeqOp::kStage: {
        d2ip_status s = op.arg < 0 ? (j.dV0 ? stage_dv(c, j.dV0, m)
                                            : stage_dv(c, j.V, (long long)j.T * m))
                                   : stage_dv(c, j.V + (long long)op.arg * m, (long long)j.T * m);
        if (s) return s;
        break;
      }
      case SeqOp::kReset: {
        d2ip_status s = reset_optimizer(c);
        if (s) return s;
        break;
      }
      case SeqOp::kSteps:
        while (j.done_steps < op.arg && budget > 0) {
          CK(cudaGraphLaunch(c->g_step, c->stream));
          ++j.done_steps;
          --budget;
        }
        if (j.done_steps < op.arg) return D2IP_OK;
        j.done_steps = 0;
        break;
      case SeqOp::kEval:
        CK(cudaGraphLaunch(c->g_eval, c->stream));
        if (j.Sigma)
          CK(copy_rows(j.Sigma + (long long)op.arg * n, (long long)j.T * n, c->dsigma, n, n,
                       c->B, sizeof(float), c->stream));
        CK(cudaMemcpy2DAsync(c->seq_resid + op.arg, sizeof(double) * j.T, c->resid,
                             sizeof(double), sizeof(double), c->B, cudaMemcpyDeviceToDevice,
                             c->stream));
        break;
      case SeqOp::kPrev:
        CK(set_device_int(c->nprev, op.arg, c->stream));
        break;
      case SeqOp::kSave:
        CK(copy_rows(c->hist + (long long)op.arg * n, (long long)c->hist_cap * n, c->dsigma, n,
                     n, c->B, sizeof(float), c->stream));
        break;
      case SeqOp::kResiduals:
        if (j.resid)
          CK(cudaMemcpyAsync(j.resid, c->seq_resid, sizeof(double) * j.T * c->B,
                             cudaMemcpyDefault, c->stream));
        break;
    }
    ++j.pc;
  }
  return D2IP_OK;
}

}  // namespace

namespace d2ip {
// Message for d2ip_last_error(NULL) from op entry points defined in other files.
void record_op_error(const std::string& msg) { g_op_error = msg; }
}  // namespace d2ip

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

d2ip_status d2ip_create(d2ip_ctx** out, int device, void* stream) {
  if (!out) return fail(nullptr, D2IP_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, D2IP_ERR_CUDA, "no CUDA device available");
  if (device < 0 || device >= ndev) return fail(nullptr, D2IP_ERR_BAD_ARG, "bad device index");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(nullptr, D2IP_ERR_CUDA, cudaGetErrorString(e));
  d2ip_ctx* c = new d2ip_ctx();
  c->device = device;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, D2IP_ERR_CUDA, cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  e = prepare_pointwise_kernels();
  if (e == cudaSuccess) e = bf16_prepare_kernels();
  if (e != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return fail(nullptr, D2IP_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = c;
  return D2IP_OK;
}

d2ip_status d2ip_destroy(d2ip_ctx* c) {
  if (!c) return D2IP_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_arena(c);
  if (c->J) cudaFree(c->J);
  if (c->colnorm) cudaFree(c->colnorm);
  if (c->r) cudaFree(c->r);
  if (c->dv) cudaFree(c->dv);
  if (c->jpart) cudaFree(c->jpart);
  if (c->Jbf) cudaFree(c->Jbf);
  if (c->Jlo) cudaFree(c->Jlo);
  if (c->jp_stage) cudaFree(c->jp_stage);
  if (c->seq_resid) cudaFree(c->seq_resid);
  if (c->hist) cudaFree(c->hist);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return D2IP_OK;
}

d2ip_status d2ip_set_grid(d2ip_ctx* c, int X, int Y, int Z) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (X <= 0 || Y <= 0 || Z <= 0 || (long long)X * Y * Z > (1LL << 30))
    return fail(c, D2IP_ERR_BAD_SHAPE, "grid dimensions must be positive (at most 2^30 voxels)");
  cudaSetDevice(c->device);
  free_arena(c);
  c->X = X;
  c->Y = Y;
  c->Z = Z;
  c->j_ready = c->input_ready = false;
  if (c->net_ready) build_plan(c);
  return D2IP_OK;
}

d2ip_status d2ip_set_network(d2ip_ctx* c, int levels, const int* widths, int c_in,
                             int precision, int batch) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->X) return fail(c, D2IP_ERR_STATE, "call d2ip_set_grid first");
  if (levels < 1 || levels > 8 || !widths)
    return fail(c, D2IP_ERR_BAD_ARG, "levels must be 1..8 with a widths array");
  for (int l = 0; l < levels; ++l)
    if (widths[l] <= 0 || widths[l] % 4 != 0 || widths[l] > 128)
      return fail(c, D2IP_ERR_BAD_SHAPE, "each width must be a positive multiple of 4, <= 128");
  if (c_in <= 0 || c_in > 256) return fail(c, D2IP_ERR_BAD_SHAPE, "c_in must be 1..256");
  if (precision != D2IP_FP32 && precision != D2IP_BF16 && precision != D2IP_BF16X3)
    return fail(c, D2IP_ERR_BAD_ARG, "precision must be D2IP_FP32, D2IP_BF16 or D2IP_BF16X3");
  if (precision != D2IP_FP32 && !bf16_network_supported(levels, widths, c_in))
    return fail(c, D2IP_ERR_BAD_SHAPE, "BF16 paths need widths that are multiples of 16");
  if (batch < 1 || batch > 4096) return fail(c, D2IP_ERR_BAD_ARG, "batch must be 1..4096");
  cudaSetDevice(c->device);
  free_arena(c);
  c->L = levels;
  c->w.assign(widths, widths + levels);
  c->c_in = c_in;
  c->precision = precision;
  c->B = batch;
  c->arch = 0;
  c->net_ready = true;
  c->j_ready = c->input_ready = false;
  build_plan(c);
  return D2IP_OK;
}

d2ip_status d2ip_set_network_fastres(d2ip_ctx* c, int levels, const int* widths, int c_in,
                                     int precision, int batch) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->X) return fail(c, D2IP_ERR_STATE, "call d2ip_set_grid first");
  if (levels < 1 || levels > 6 || !widths)
    return fail(c, D2IP_ERR_BAD_ARG, "levels must be 1..6 with a widths array");
  if (!fastres_supported(levels, widths, c_in))
    return fail(c, D2IP_ERR_BAD_SHAPE,
                "each width must be a multiple of 8 in 8..128 and c_in 1..256");
  if (precision != D2IP_FP32)
    return fail(c, D2IP_ERR_BAD_ARG, "the FastResUNet variant runs in D2IP_FP32");
  if (batch < 1 || batch > 4096) return fail(c, D2IP_ERR_BAD_ARG, "batch must be 1..4096");
  cudaSetDevice(c->device);
  free_arena(c);
  c->L = levels;
  c->w.assign(widths, widths + levels);
  c->c_in = c_in;
  c->precision = precision;
  c->B = batch;
  c->arch = 1;
  c->net_ready = true;
  c->j_ready = c->input_ready = false;
  build_plan(c);
  return D2IP_OK;
}

d2ip_status d2ip_param_count(d2ip_ctx* c, long long* count) {
  if (!c || !count) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->net_ready) return fail(c, D2IP_ERR_STATE, "network not set");
  *count = c->P;
  return D2IP_OK;
}

d2ip_status d2ip_param_table(d2ip_ctx* c, long long* rows, int cap, int* n_rows) {
  if (!c || !n_rows) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->net_ready) return fail(c, D2IP_ERR_STATE, "network not set");
  const int n = (int)(c->table.size() / 4);
  *n_rows = n;
  if (rows)
    for (int i = 0; i < std::min(n, cap) * 4; ++i) rows[i] = c->table[i];
  return D2IP_OK;
}

d2ip_status d2ip_plan_param_table(int net, int X, int Y, int Z, int levels, const int* widths,
                                  int c_in, long long* rows, int cap, int* n_rows,
                                  long long* count) {
  if (!n_rows || !widths || (net != 0 && net != 1))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "null argument or unknown network");
  if (X <= 0 || Y <= 0 || Z <= 0 || (long long)X * Y * Z > (1LL << 30))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "grid dimensions must be positive");
  if (net == 0) {
    if (levels < 1 || levels > 8 || c_in <= 0 || c_in > 256)
      return fail(nullptr, D2IP_ERR_BAD_ARG, "levels must be 1..8 and c_in 1..256");
    for (int l = 0; l < levels; ++l)
      if (widths[l] <= 0 || widths[l] % 4 != 0 || widths[l] > 128)
        return fail(nullptr, D2IP_ERR_BAD_SHAPE,
                    "each width must be a positive multiple of 4, <= 128");
  } else if (levels < 1 || levels > 6 || !fastres_supported(levels, widths, c_in)) {
    return fail(nullptr, D2IP_ERR_BAD_SHAPE,
                "levels 1..6, each width a multiple of 8 in 8..128, c_in 1..256");
  }
  d2ip_ctx t;  // host-side plan only: nothing here touches a device
  t.X = X, t.Y = Y, t.Z = Z;
  t.L = levels;
  t.w.assign(widths, widths + levels);
  t.c_in = c_in;
  t.precision = D2IP_FP32;
  t.arch = net;
  build_plan(&t);
  const int n = (int)(t.table.size() / 4);
  *n_rows = n;
  if (rows)
    for (int i = 0; i < std::min(n, cap) * 4; ++i) rows[i] = t.table[i];
  if (count) *count = t.P;
  return D2IP_OK;
}

d2ip_status d2ip_load_J(d2ip_ctx* c, const float* J, int m, int n, int normalize_cols) {
  if (!c || !J) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->net_ready) return fail(c, D2IP_ERR_STATE, "set grid and network first");
  if (m <= 0 || (long long)n != c->n())
    return fail(c, D2IP_ERR_BAD_SHAPE, "J must be m x (X*Y*Z)");
  if ((size_t)8 * m * sizeof(float) > 200 * 1024)
    return fail(c, D2IP_ERR_BAD_SHAPE, "m too large for the adjoint kernel (max 6400)");
  if (c->precision != D2IP_FP32 && (m % 4 != 0 || m > 1024))
    return fail(c, D2IP_ERR_BAD_SHAPE, "the BF16 paths need m a multiple of 4, at most 1024");
  CK(cudaSetDevice(c->device));
  d2ip_status s = ensure_arena(c);
  if (s) return s;
  const size_t bytes = (size_t)m * n * sizeof(float);
  if (bytes != c->j_bytes || m != c->m) {
    drop_graphs(c);
    if (c->J) cudaFree(c->J);
    if (c->colnorm) cudaFree(c->colnorm);
    if (c->r) cudaFree(c->r);
    if (c->dv) cudaFree(c->dv);
    if (c->jpart) cudaFree(c->jpart);
    if (c->Jbf) cudaFree(c->Jbf);
    if (c->Jlo) cudaFree(c->Jlo);
    c->Jbf = c->Jlo = nullptr;
    if (c->jp_stage) cudaFree(c->jp_stage);
    c->jp_stage = nullptr;
    c->J = nullptr;
    c->colnorm = nullptr;
    c->r = c->dv = c->jpart = nullptr;
    c->j_bytes = 0;
    if (cudaMalloc(&c->J, bytes) != cudaSuccess ||
        cudaMalloc(&c->colnorm, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&c->r, sizeof(float) * m * c->B) != cudaSuccess ||
        cudaMalloc(&c->dv, sizeof(float) * m * c->B) != cudaSuccess ||
        cudaMalloc(&c->jpart, sizeof(float) * jmul_chunks(n) * (size_t)m * c->B) != cudaSuccess ||
        (c->precision != D2IP_FP32 &&
         cudaMalloc(&c->Jbf, sizeof(__nv_bfloat16) * (size_t)m * n) != cudaSuccess) ||
        (c->precision == D2IP_BF16X3 &&
         cudaMalloc(&c->Jlo, sizeof(__nv_bfloat16) * (size_t)m * n) != cudaSuccess))
      return fail(c, D2IP_ERR_OOM, "device allocation of J failed");
    c->j_bytes = bytes;
    c->m = m;
  }
  CK(cudaMemcpyAsync(c->J, J, bytes, cudaMemcpyDefault, c->stream));
  if (normalize_cols) {
    CK(normalize_columns_f64(c->J, c->colnorm, m, n, c->stream));
  } else {
    CK(cudaMemsetAsync(c->colnorm, 0, sizeof(double) * n, c->stream));
  }
  if (c->precision != D2IP_FP32) {
    CK(transpose_bf16(c->J, c->Jbf, m, (int)n, c->stream, c->Jlo));
    if (jprod_tc_supported(m, (int)n)) {  // J x and J^T r on the tensor cores
      if (!c->jp_stage &&
          cudaMalloc(&c->jp_stage, jprod_tc_staging_bytes(m, (int)n, c->B, c->Jlo != nullptr)) !=
              cudaSuccess) {
        c->jp_stage = nullptr;
        return fail(c, D2IP_ERR_OOM, "device allocation of the J-product staging failed");
      }
      CK(jprod_tc_init(c->jp, c->Jbf, c->Jlo, c->jp_stage, m, (int)n, c->B, c->stream));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  c->j_ready = true;
  return D2IP_OK;
}

d2ip_status d2ip_get_colnorms(d2ip_ctx* c, double* out) {
  if (!c || !out) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->j_ready) return fail(c, D2IP_ERR_STATE, "J not loaded");
  CK(cudaSetDevice(c->device));
  CK(cudaMemcpyAsync(out, c->colnorm, sizeof(double) * c->n(), cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_set_input(d2ip_ctx* c, const float* Zin, const float* theta0) {
  if (!c || !Zin || !theta0) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->net_ready) return fail(c, D2IP_ERR_STATE, "set grid and network first");
  CK(cudaSetDevice(c->device));
  d2ip_status s = ensure_arena(c);
  if (s) return s;
  CK(cudaMemcpyAsync(c->zin, Zin, sizeof(float) * c->B * c->n() * c->c_in, cudaMemcpyDefault,
                     c->stream));
  if (c->stem.conv.tc >= 0 && c->bf.layers[c->stem.conv.tc].input_layer)
    CK(bf16_stage_input(c->bf, c->stem.conv.tc, c->zin, c->B, c->stream));
  CK(copy_rows(c->theta, c->Pp, theta0, c->P, c->P, c->B, sizeof(float), c->stream));
  s = reset_optimizer(c);
  if (s) return s;
  CK(cudaStreamSynchronize(c->stream));
  c->input_ready = true;
  return D2IP_OK;
}

d2ip_status d2ip_set_optim(d2ip_ctx* c, double lr, double beta1, double beta2, double eps) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
      !(eps > 0.0))
    return fail(c, D2IP_ERR_BAD_ARG, "need lr > 0, 0 <= beta < 1, eps > 0");
  if (lr != c->lr || beta1 != c->beta1 || beta2 != c->beta2 || eps != c->eps) drop_graphs(c);
  c->lr = lr;
  c->beta1 = beta1;
  c->beta2 = beta2;
  c->eps = eps;
  return D2IP_OK;
}

d2ip_status d2ip_set_regularizer(d2ip_ctx* c, double lambda_tv, double lambda_s,
                                 double lambda_t, double eps) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!(lambda_tv >= 0.0) || !(lambda_s >= 0.0) || !(lambda_t >= 0.0) || !(eps > 0.0))
    return fail(c, D2IP_ERR_BAD_ARG, "need lambdas >= 0 and eps > 0");
  drop_graphs(c);
  c->lam_tv = lambda_tv;
  c->lam_s = lambda_s;
  c->lam_t = lambda_t;
  c->tv_eps = eps;
  return D2IP_OK;
}

d2ip_status d2ip_set_autotune(d2ip_ctx* c, int on) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  c->autotune = on != 0;
  return D2IP_OK;
}

d2ip_status d2ip_tile_plan(d2ip_ctx* c, long long* rows, int cap, int* n_rows, double* us) {
  if (!c || !n_rows) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->arena) return fail(c, D2IP_ERR_STATE, "network workspace not built yet");
  const auto& ls = c->bf.layers;
  const int n = c->precision == D2IP_FP32 ? 0 : (int)ls.size();
  *n_rows = n;
  for (int i = 0; i < n && i < cap; ++i) {
    const TcLayer& L = ls[i];
    const long long r[15] = {L.ci_real, L.co, L.k, L.s, L.dout.z, L.dout.y, L.dout.x,
                             L.per3f, L.pack3f, L.ck3f, L.tz3f,
                             L.per3d, L.pack3d, L.ck3d, L.tz3d};
    if (rows)
      for (int j = 0; j < 15; ++j) rows[15LL * i + j] = r[j];
    if (us) {
      us[4LL * i] = L.tune_f, us[4LL * i + 1] = L.model_f;
      us[4LL * i + 2] = L.tune_d, us[4LL * i + 3] = L.model_d;
    }
  }
  return D2IP_OK;
}

d2ip_status d2ip_set_tile_plan(d2ip_ctx* c, const long long* rows, int n_rows) {
  if (!c || n_rows < 0 || (n_rows > 0 && !rows)) return fail(c, D2IP_ERR_BAD_ARG, "bad argument");
  if (c->arena) return fail(c, D2IP_ERR_STATE, "the workspace already exists");
  c->tile_rows.assign(rows, rows + 15LL * n_rows);
  return D2IP_OK;
}

d2ip_status d2ip_set_ln_backward_fusion(d2ip_ctx* c, int on) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  c->ln_bwd_fused = on != 0;
  drop_graphs(c);  // captured graphs hold the old launch sequence
  return D2IP_OK;
}

d2ip_status d2ip_set_frame_reset(d2ip_ctx* c, int reset_moments_per_frame) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  c->frame_reset = reset_moments_per_frame != 0;
  return D2IP_OK;
}

d2ip_status d2ip_reset_optimizer(d2ip_ctx* c) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->arena) return fail(c, D2IP_ERR_STATE, "network not set up");
  CK(cudaSetDevice(c->device));
  d2ip_status s = reset_optimizer(c);
  if (s) return s;
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_run_steps(d2ip_ctx* c, const float* dV, int n_steps, double* loss_trace) {
  d2ip_status s = ready(c);
  if (s) return s;
  if (!dV || n_steps < 0) return fail(c, D2IP_ERR_BAD_ARG, "bad dV or n_steps");
  s = stage_dv(c, dV, c->m);
  if (s) return s;
  s = run_steps(c, n_steps, loss_trace);
  if (s) return s;
  return check_status(c);
}

d2ip_status d2ip_forward(d2ip_ctx* c, float* dsigma_out) {
  if (!c || !dsigma_out) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  d2ip_status s = ready(c);
  if (s) return s;
  Launcher Lr{c};
  Lr.forward();
  if (Lr.e != cudaSuccess) return cuda_fail(c, Lr.e, "forward launch");
  CK(cudaMemcpyAsync(dsigma_out, c->dsigma, sizeof(float) * c->B * c->n(), cudaMemcpyDefault,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_get_grad(d2ip_ctx* c, float* grad_out) {
  if (!c || !grad_out) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->arena) return fail(c, D2IP_ERR_STATE, "network not set up");
  CK(cudaSetDevice(c->device));
  CK(copy_rows(grad_out, c->P, c->grad, c->Pp, c->P, c->B, sizeof(float), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_fit_frame(d2ip_ctx* c, const float* dV, int n_steps, float* dsigma_out,
                           double* residual_out, double* loss_trace) {
  d2ip_status s = ready(c);
  if (s) return s;
  if (!dV || n_steps < 0) return fail(c, D2IP_ERR_BAD_ARG, "bad dV or n_steps");
  s = stage_dv(c, dV, c->m);
  if (s) return s;
  if (c->frame_reset) {
    s = reset_optimizer(c);
    if (s) return s;
  }
  if (c->lam_tv != 0.0) CK(set_device_int(c->nprev, 0, c->stream));  // no earlier frames
  s = run_steps(c, n_steps, loss_trace);
  if (s) return s;
  CK(cudaGraphLaunch(c->g_eval, c->stream));
  if (dsigma_out)
    CK(cudaMemcpyAsync(dsigma_out, c->dsigma, sizeof(float) * c->B * c->n(), cudaMemcpyDefault,
                       c->stream));
  if (residual_out)
    CK(cudaMemcpyAsync(residual_out, c->resid, sizeof(double) * c->B, cudaMemcpyDefault,
                       c->stream));
  return check_status(c);
}

d2ip_status d2ip_fit_sequence(d2ip_ctx* c, const float* V, int T, const float* dV0,
                              int upws_steps, int first_steps, int later_steps,
                              float* Sigma_out, double* residual_out) {
  d2ip_ctx* one[1] = {c};
  const float* Vs[1] = {V};
  const float* d0[1] = {dV0};
  float* So[1] = {Sigma_out};
  double* Ro[1] = {residual_out};
  return d2ip_fit_batched(one, 1, Vs, T, d0, upws_steps, first_steps, later_steps, So, Ro);
}

d2ip_status d2ip_fit_batched(d2ip_ctx* const* ctxs, int count, const float* const* V, int T,
                             const float* const* dV0, int upws_steps, int first_steps,
                             int later_steps, float* const* Sigma_out,
                             double* const* residual_out) {
  if (!ctxs || count < 1 || !V) return fail(nullptr, D2IP_ERR_BAD_ARG, "bad context list");
  if (T < 1 || upws_steps < 0 || first_steps < 0 || later_steps < 0)
    return fail(ctxs[0], D2IP_ERR_BAD_ARG, "bad T or step counts");
  std::vector<SeqJob> jobs(count);
  for (int i = 0; i < count; ++i) {
    d2ip_ctx* c = ctxs[i];
    d2ip_status s = ready(c);
    if (s) return s;
    if (!V[i]) return fail(c, D2IP_ERR_BAD_ARG, "null V");
    if (T > c->seq_T_cap) {
      if (c->seq_resid) cudaFree(c->seq_resid);
      c->seq_resid = nullptr;
      if (cudaMalloc(&c->seq_resid, sizeof(double) * T * c->B) != cudaSuccess)
        return fail(c, D2IP_ERR_OOM, "residual buffer allocation failed");
      c->seq_T_cap = T;
    }
    if (c->lam_tv != 0.0 && T > c->hist_cap) {
      if (c->hist) cudaFree(c->hist);
      c->hist = nullptr;
      c->hist_cap = 0;
      drop_graphs(c);  // the step graph holds the history's address and stride
      if (cudaMalloc(&c->hist, sizeof(float) * (size_t)T * c->B * c->n()) != cudaSuccess)
        return fail(c, D2IP_ERR_OOM, "frame history allocation failed");
      c->hist_cap = T;
      s = ready(c);
      if (s) return s;
    }
    jobs[i] = make_sequence_job(c, V[i], T, dV0 ? dV0[i] : nullptr, upws_steps, first_steps,
                                later_steps, Sigma_out ? Sigma_out[i] : nullptr,
                                residual_out ? residual_out[i] : nullptr);
  }
  // issue a few graph launches per context in turn, so every context's stream keeps work
  bool left = true;
  while (left) {
    left = false;
    for (SeqJob& j : jobs) {
      d2ip_status s = issue(j, 8);
      if (s) return s;
      left = left || j.pc < j.ops.size();
    }
  }
  d2ip_status first_err = D2IP_OK;
  for (SeqJob& j : jobs) {
    d2ip_status s = check_status(j.c);
    if (s && !first_err) first_err = s;
  }
  return first_err;
}

d2ip_status d2ip_get_state(d2ip_ctx* c, float* theta, float* adam_m, float* adam_v,
                           int* adam_t) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->arena) return fail(c, D2IP_ERR_STATE, "network not set up");
  CK(cudaSetDevice(c->device));
  if (theta) CK(copy_rows(theta, c->P, c->theta, c->Pp, c->P, c->B, sizeof(float), c->stream));
  if (adam_m) CK(copy_rows(adam_m, c->P, c->am, c->Pp, c->P, c->B, sizeof(float), c->stream));
  if (adam_v) CK(copy_rows(adam_v, c->P, c->av, c->Pp, c->P, c->B, sizeof(float), c->stream));
  int t = 0;
  CK(cudaMemcpyAsync(&t, c->adam_t, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (adam_t) *adam_t = t;
  return D2IP_OK;
}

d2ip_status d2ip_set_state(d2ip_ctx* c, const float* theta, const float* adam_m,
                           const float* adam_v, int adam_t) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  if (!c->net_ready) return fail(c, D2IP_ERR_STATE, "network not set");
  if (adam_t < 0) return fail(c, D2IP_ERR_BAD_ARG, "adam_t must be >= 0");
  CK(cudaSetDevice(c->device));
  d2ip_status s = ensure_arena(c);
  if (s) return s;
  if (theta) CK(copy_rows(c->theta, c->Pp, theta, c->P, c->P, c->B, sizeof(float), c->stream));
  if (adam_m) CK(copy_rows(c->am, c->Pp, adam_m, c->P, c->P, c->B, sizeof(float), c->stream));
  if (adam_v) CK(copy_rows(c->av, c->Pp, adam_v, c->P, c->P, c->B, sizeof(float), c->stream));
  CK(cudaMemcpyAsync(c->adam_t, &adam_t, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_err_ratio(d2ip_ctx* c, const float* est, const float* truth, double* out) {
  if (!c || !est || !truth || !out) return fail(c, D2IP_ERR_BAD_ARG, "null argument");
  if (!c->arena) return fail(c, D2IP_ERR_STATE, "network not set up");
  CK(cudaSetDevice(c->device));
  const long long n = c->n();
  CK(cudaMemcpyAsync(c->stage, truth, sizeof(float) * c->B * n, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(c->gds, est, sizeof(float) * c->B * n, cudaMemcpyDefault, c->stream));
  CK(err_ratio_f64(c->gds, c->stage, c->resid, c->B, n, c->stream));
  CK(cudaMemcpyAsync(out, c->resid, sizeof(double) * c->B, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return D2IP_OK;
}

d2ip_status d2ip_profile_iterations(d2ip_ctx* c, const float* dV, int n_iters, double* ms,
                                    double* work, long long* launches) {
  d2ip_status s = ready(c);
  if (s) return s;
  if (!dV || n_iters < 1 || !ms || !work || !launches)
    return fail(c, D2IP_ERR_BAD_ARG, "bad dV, n_iters or output arrays");
  s = stage_dv(c, dV, c->m);
  if (s) return s;
  CK(cudaMemsetAsync(c->trace_pos, 0, sizeof(int), c->stream));
  Tracer tr;
  Launcher Lr{c, &tr};
  for (int it = 0; it < n_iters && Lr.e == cudaSuccess; ++it) {
    Lr.forward();
    Lr.data_term(true);
    Lr.backward();
    Lr.adam();
  }
  cudaError_t e = Lr.e;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  for (int k = 0; k < D2IP_KCLASS_COUNT; ++k) {
    ms[k] = 0.0;
    work[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; e == cudaSuccess && i < tr.cls.size(); ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, tr.pool[2 * i], tr.pool[2 * i + 1]);
    ms[tr.cls[i]] += t;
    work[tr.cls[i]] += tr.work[i];
    launches[tr.cls[i]] += 1;
  }
  tr.release();
  if (e != cudaSuccess) return cuda_fail(c, e, "profiled iterations");
  return check_status(c);
}

d2ip_status d2ip_graph_kernels(d2ip_ctx* c, long long* step_kernels, long long* eval_kernels) {
  d2ip_status s = ready(c);
  if (s) return s;
  if (!step_kernels || !eval_kernels) return fail(c, D2IP_ERR_BAD_ARG, "null output");
  *step_kernels = c->step_kernels;
  *eval_kernels = c->eval_kernels;
  return D2IP_OK;
}

d2ip_status d2ip_sync(d2ip_ctx* c) {
  if (!c) return fail(nullptr, D2IP_ERR_BAD_ARG, "null context");
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return D2IP_OK;
}

const char* d2ip_last_error(d2ip_ctx* c) { return c ? c->err.c_str() : g_op_error.c_str(); }

// ---------------------------------------------------------------------------------------
// context-free ops
// ---------------------------------------------------------------------------------------
#define OPCK(call)                                                              \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) return cuda_fail(nullptr, e_, #call);                \
  } while (0)

static bool bad_conv(int batch, int dz, int dy, int dx, int ci, int co, int k, int s) {
  return batch < 1 || dz < 1 || dy < 1 || dx < 1 || ci < 1 || co < 1 || (k != 1 && k != 3) ||
         (s != 1 && s != 2);
}

d2ip_status d2ip_conv3d_forward(const float* x, const float* W, const float* b, float* y,
                                int batch, int dz, int dy, int dx, int ci, int co, int ksize,
                                int stride, long long w_bs, void* stream) {
  if (!x || !W || !b || !y) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad convolution shape");
  const Dims3 din{dz, dy, dx};
  const Dims3 dout = conv_out_dims(din, ksize, stride);
  OPCK(conv3d_fwd_f32(x, W, b, y, batch, din, ci, co, ksize, stride, din.count() * ci,
                      dout.count() * co, w_bs, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_conv3d_dgrad(const float* dyp, const float* W, float* dxp, int batch, int dz,
                              int dy, int dx, int ci, int co, int ksize, int stride,
                              long long w_bs, int accumulate, void* stream) {
  if (!dyp || !W || !dxp) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad convolution shape");
  const Dims3 din{dz, dy, dx};
  const Dims3 dout = conv_out_dims(din, ksize, stride);
  OPCK(conv3d_dgrad_f32(dyp, W, dxp, batch, din, ci, co, ksize, stride, dout.count() * co,
                        din.count() * ci, w_bs, accumulate, (cudaStream_t)stream));
  return D2IP_OK;
}

long long d2ip_conv3d_tc_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                   int ksize, int stride) {
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride) || !bf16_conv_supported(ci, co, ksize))
    return -1;
  return bf16_op_workspace(batch, Dims3{dz, dy, dx}, ci, co, ksize, stride);
}

static d2ip_status tc_op(bool dgrad, const float* in, const float* W, const float* b,
                         float* out, int batch, int dz, int dy, int dx, int ci, int co,
                         int ksize, int stride, long long w_bs, int accumulate, void* ws,
                         long long ws_bytes, void* stream) {
  if (!in || !W || !out || !ws) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride) || !bf16_conv_supported(ci, co, ksize) ||
      (dgrad && !bf16_conv_supported(co, ci, ksize)))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE,
                "tensor-core convolution needs ci, co multiples of 16 (both <= 256 for the data "
                "gradient, co <= 256 for the forward)");
  if (ws_bytes < d2ip_conv3d_tc_workspace(batch, dz, dy, dx, ci, co, ksize, stride))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)
    return fail(nullptr, D2IP_ERR_BAD_ARG, "input and output must be 16-byte aligned");
  const long long blk = (long long)co * ksize * ksize * ksize * ci + co;
  OPCK(bf16_op_conv(dgrad, in, W, b, out, batch, Dims3{dz, dy, dx}, ci, co, ksize, stride,
                    w_bs ? w_bs : blk, accumulate, ws, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_conv3d_forward_tc(const float* x, const float* W, const float* b, float* y,
                                   int batch, int dz, int dy, int dx, int ci, int co, int ksize,
                                   int stride, long long w_bs, void* ws, long long ws_bytes,
                                   void* stream) {
  if (!b) return fail(nullptr, D2IP_ERR_BAD_ARG, "null bias");
  return tc_op(false, x, W, b, y, batch, dz, dy, dx, ci, co, ksize, stride, w_bs, 0, ws,
               ws_bytes, stream);
}

d2ip_status d2ip_conv3d_dgrad_tc(const float* dyp, const float* W, float* dxp, int batch,
                                 int dz, int dy, int dx, int ci, int co, int ksize, int stride,
                                 long long w_bs, int accumulate, void* ws, long long ws_bytes,
                                 void* stream) {
  return tc_op(true, dyp, W, nullptr, dxp, batch, dz, dy, dx, ci, co, ksize, stride, w_bs,
               accumulate, ws, ws_bytes, stream);
}

long long d2ip_conv3d_wgrad_tc_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                         int ksize) {
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, 1) || !bf16_conv_supported(ci, co, ksize))
    return -1;
  return bf16_op_wgrad_workspace(batch, Dims3{dz, dy, dx}, ci, co, ksize);
}

d2ip_status d2ip_conv3d_wgrad_tc(const float* x, const float* dyp, float* dWb, int batch, int dz,
                                 int dy, int dx, int ci, int co, int ksize, long long dw_bs,
                                 int accumulate, void* ws, long long ws_bytes, void* stream) {
  if (!x || !dyp || !dWb || !ws) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  const long long need = d2ip_conv3d_wgrad_tc_workspace(batch, dz, dy, dx, ci, co, ksize);
  if (need < 0)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE,
                "tensor-core weight gradient: stride 1, ci and co multiples of 16, co dividing "
                "128, ci + min(64, ci) <= 256");
  if (ws_bytes < need) return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  const long long row = (long long)co * ksize * ksize * ksize * ci + co;
  OPCK(bf16_op_wgrad(x, dyp, dWb, batch, Dims3{dz, dy, dx}, ci, co, ksize, dw_bs ? dw_bs : row,
                     accumulate, ws, (cudaStream_t)stream));
  return D2IP_OK;
}

long long d2ip_conv3d_wgrad_workspace(int batch, int dz, int dy, int dx, int ci, int co,
                                      int ksize, int stride) {
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride)) return -1;
  const Dims3 din{dz, dy, dx};
  return (long long)sizeof(float) * batch * conv3d_wgrad_chunks(din, ksize, stride) *
         ((long long)co * ksize * ksize * ksize * ci + co);
}

d2ip_status d2ip_conv3d_wgrad(const float* x, const float* dyp, float* dWb, int batch, int dz,
                              int dy, int dx, int ci, int co, int ksize, int stride,
                              long long dw_bs, int accumulate, void* workspace,
                              long long ws_bytes, void* stream) {
  if (!x || !dyp || !dWb || !workspace) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (bad_conv(batch, dz, dy, dx, ci, co, ksize, stride))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad convolution shape");
  if (ws_bytes < d2ip_conv3d_wgrad_workspace(batch, dz, dy, dx, ci, co, ksize, stride))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  const Dims3 din{dz, dy, dx};
  const Dims3 dout = conv_out_dims(din, ksize, stride);
  float* part = static_cast<float*>(workspace);
  OPCK(conv3d_wgrad_partial_f32(x, dyp, part, batch, din, ci, co, ksize, stride,
                                din.count() * ci, dout.count() * co, (cudaStream_t)stream));
  const long long row = (long long)co * ksize * ksize * ksize * ci + co;
  OPCK(reduce_rows_f32(part, dWb, batch, conv3d_wgrad_chunks(din, ksize, stride), row,
                       dw_bs ? dw_bs : row, accumulate, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_layernorm_act_forward(const float* z, const float* gb, const float* resid,
                                       float* y, float* xhat, float* rstd, int batch,
                                       long long nvox, int c, int act, long long gb_bs,
                                       void* stream) {
  if (!z || !gb || !y || !xhat || !rstd) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || nvox < 1 || c < 4 || c % 4 || c > 128 || (act != 0 && act != 1))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad LayerNorm shape (c multiple of 4, <= 128)");
  OPCK(layernorm_act_fwd_f32(z, gb, resid, y, xhat, rstd, batch, nvox, c, act, gb_bs,
                             (cudaStream_t)stream));
  return D2IP_OK;
}

long long d2ip_layernorm_workspace(int batch, long long nvox, int c) {
  if (batch < 1 || nvox < 1 || c < 4 || c % 4 || c > 128) return -1;
  return (long long)sizeof(float) * batch * layernorm_bwd_blocks(nvox, c) * 2 * c;
}

d2ip_status d2ip_layernorm_act_backward(const float* dy, const float* act_out,
                                        const float* xhat, const float* rstd, const float* gb,
                                        float* dz, float* dt, float* dgb, int batch,
                                        long long nvox, int c, long long gb_bs, int accumulate,
                                        void* workspace, long long ws_bytes, void* stream) {
  if (!dy || !xhat || !rstd || !gb || !dz || !dgb || !workspace)
    return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || nvox < 1 || c < 4 || c % 4 || c > 128)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad LayerNorm shape (c multiple of 4, <= 128)");
  if (ws_bytes < d2ip_layernorm_workspace(batch, nvox, c))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  float* part = static_cast<float*>(workspace);
  OPCK(layernorm_act_bwd_f32(dy, act_out, xhat, rstd, gb, dz, dt, part, batch, nvox, c, gb_bs,
                             (cudaStream_t)stream));
  OPCK(reduce_rows_f32(part, dgb, batch, layernorm_bwd_blocks(nvox, c), 2 * c, 2 * c,
                       accumulate, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_upsample_concat_forward(const float* low, const float* skip, float* cat,
                                         int batch, int lz, int ly, int lx, int oz, int oy,
                                         int ox, int cu, int cs, void* stream) {
  if (!low || !cat || (cs > 0 && !skip)) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || lz < 1 || ly < 1 || lx < 1 || oz < 1 || oy < 1 || ox < 1 || cu < 4 || cs < 0 ||
      cu % 4 || cs % 4)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad upsample shape (cu, cs multiples of 4)");
  OPCK(upsample_concat_fwd_f32(low, skip, cat, batch, Dims3{lz, ly, lx}, Dims3{oz, oy, ox}, cu,
                               cs, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_upsample_concat_backward(const float* dcat, float* dlow, float* dskip,
                                          int batch, int lz, int ly, int lx, int oz, int oy,
                                          int ox, int cu, int cs, void* stream) {
  if (!dcat || !dlow) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || lz < 1 || ly < 1 || lx < 1 || oz < 1 || oy < 1 || ox < 1 || cu < 4 || cs < 0 ||
      cu % 4 || cs % 4)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad upsample shape (cu, cs multiples of 4)");
  // the gather visits at most 8 outputs per input and axis: needs out/in <= about 3
  if (oz > 3 * lz || oy > 3 * ly || ox > 3 * lx)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "upsample factor above 3 not supported");
  OPCK(upsample_concat_bwd_f32(dcat, dlow, dskip, batch, Dims3{lz, ly, lx}, Dims3{oz, oy, ox},
                               cu, cs, (cudaStream_t)stream));
  return D2IP_OK;
}

long long d2ip_sensitivity_workspace(int batch, int m, int n) {
  if (batch < 1 || m < 1 || n < 1) return -1;
  return (long long)sizeof(float) * jmul_chunks(n) * m * batch;
}

d2ip_status d2ip_sensitivity_residual(const float* J, const float* x, const float* dv,
                                      float* r, double* loss, int batch, int m, int n,
                                      void* workspace, long long workspace_bytes,
                                      void* stream) {
  if (!J || !x || !dv || !r || !workspace) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || m < 1 || n < 1) return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad J shape");
  if (workspace_bytes < d2ip_sensitivity_workspace(batch, m, n))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  OPCK(jmul_residual_f32(J, x, dv, r, static_cast<float*>(workspace), batch, m, n, n,
                         (cudaStream_t)stream));
  if (loss)
    OPCK(residual_loss_f64(r, loss, nullptr, nullptr, 0, nullptr, nullptr, batch, m,
                           (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_sensitivity_adjoint(const float* J, const float* r, float* g, float scale,
                                     int batch, int m, int n, void* stream) {
  if (!J || !r || !g) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || m < 1 || n < 1 || m > 6400)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad J shape (m <= 6400)");
  OPCK(prepare_pointwise_kernels());
  OPCK(jtmul_f32(J, r, g, scale, batch, m, n, n, (cudaStream_t)stream));
  return D2IP_OK;
}

static size_t ws_round(size_t b) { return (b + 255) / 256 * 256; }

long long d2ip_sensitivity_tc_workspace(int batch, int m, int n, int split) {
  if (batch < 1 || n < 1 || !jprod_tc_supported(m, n) || m > 1024) return -1;
  const size_t jt = ws_round((size_t)m * n * 2);
  return (long long)(256 + 256 + (split ? 2 : 1) * jt +
                     ws_round(jprod_tc_staging_bytes(m, n, batch, split != 0)) +
                     ws_round(sizeof(float) * jprod_tc_chunks(m, n) * (size_t)batch * m));
}

d2ip_status d2ip_sensitivity_products_tc(const float* J, const float* x, const float* dv,
                                         float* r, float* g, float scale, int batch, int m,
                                         int n, int split, void* workspace,
                                         long long workspace_bytes, void* stream) {
  if (!J || !x || !dv || !r || !workspace) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  const long long need = d2ip_sensitivity_tc_workspace(batch, m, n, split);
  if (need < 0)
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad shape (m a multiple of 8, at most 1024)");
  if (workspace_bytes < need) return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~(uintptr_t)255);
  int* err = reinterpret_cast<int*>(p);
  p += 256;
  const size_t jt = ws_round((size_t)m * n * 2);
  __nv_bfloat16* Jt = reinterpret_cast<__nv_bfloat16*>(p);
  p += jt;
  __nv_bfloat16* Jlo = nullptr;
  if (split) {
    Jlo = reinterpret_cast<__nv_bfloat16*>(p);
    p += jt;
  }
  void* stage = p;
  p += ws_round(jprod_tc_staging_bytes(m, n, batch, split != 0));
  float* part = reinterpret_cast<float*>(p);
  OPCK(prepare_pointwise_kernels());
  OPCK(cudaMemsetAsync(err, 0, sizeof(int), st));
  OPCK(transpose_bf16(J, Jt, m, n, st, Jlo));
  JprodTc jp;
  OPCK(jprod_tc_init(jp, Jt, Jlo, stage, m, n, batch, st));
  OPCK(jprod_tc_residual(jp, x, n, dv, r, part, err, st));
  if (g) OPCK(jprod_tc_adjoint(jp, g, scale, n, err, st));
  return D2IP_OK;
}

long long d2ip_tv4d_workspace(int batch, int dz, int dy, int dx) {
  if (batch < 1 || dz < 1 || dy < 1 || dx < 1) return -1;
  return 256 + (long long)sizeof(double) * batch * tv4d_blocks((long long)dz * dy * dx);
}

d2ip_status d2ip_tv4d(const float* dsigma, const float* previous, int n_previous, float* grad,
                      double* value_host, int batch, int dz, int dy, int dx, double lambda_tv,
                      double lambda_s, double lambda_t, double eps, void* workspace,
                      long long workspace_bytes, void* stream) {
  if (!dsigma || !grad || !workspace || (n_previous > 0 && !previous))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (batch < 1 || dz < 1 || dy < 1 || dx < 1 || n_previous < 0 || !(eps > 0.0))
    return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad 4D-TV arguments");
  if (workspace_bytes < d2ip_tv4d_workspace(batch, dz, dy, dx))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "workspace too small");
  const Dims3 d{dz, dy, dx};
  const long long n = d.count();
  int* np = static_cast<int*>(workspace);
  double* part = reinterpret_cast<double*>(static_cast<char*>(workspace) + 256);
  const cudaStream_t st = (cudaStream_t)stream;
  OPCK(set_device_int(np, n_previous, st));
  OPCK(tv4d_f32(dsigma, previous, np, grad, part, batch, d, (long long)n_previous * n,
                (float)(lambda_tv * lambda_s / (double)n), (float)(lambda_tv * lambda_t),
                (float)eps, st));
  if (value_host) {
    const int nb = tv4d_blocks(n);
    std::vector<double> h((size_t)batch * nb);
    OPCK(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    OPCK(cudaStreamSynchronize(st));
    for (int b = 0; b < batch; ++b) {
      double v = 0.0;
      for (int k = 0; k < nb; ++k) v += h[(size_t)b * nb + k];
      value_host[b] = v;
    }
  }
  return D2IP_OK;
}

d2ip_status d2ip_normalize_columns(float* J, double* colnorm, int m, int n, void* stream) {
  if (!J || !colnorm) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (m < 1 || n < 1) return fail(nullptr, D2IP_ERR_BAD_SHAPE, "bad J shape");
  OPCK(normalize_columns_f64(J, colnorm, m, n, (cudaStream_t)stream));
  return D2IP_OK;
}

d2ip_status d2ip_adam_update(float* theta, const float* g, float* m, float* v, long long count,
                             double lr, double beta1, double beta2, double eps, int t,
                             void* stream) {
  if (!theta || !g || !m || !v) return fail(nullptr, D2IP_ERR_BAD_ARG, "null pointer");
  if (count < 1 || t < 1 || !(lr > 0.0) || !(eps > 0.0))
    return fail(nullptr, D2IP_ERR_BAD_ARG, "bad Adam arguments");
  OPCK(adam_step_f32(theta, g, m, v, count, lr, beta1, beta2, eps, nullptr, t,
                     (cudaStream_t)stream));
  return D2IP_OK;
}

}  // extern "C"
