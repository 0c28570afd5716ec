// Allocation-free variant of the convolution weight gradient.
//
// d2ip_conv3d_wgrad needs a caller-provided workspace for its per-chunk partial sums.  Some
// callers cannot allocate device memory at the point where they need the gradient (see the
// declaration in d2ip.h).  This variant keeps that workspace in a fixed-size array that is
// part of the library image on every GPU, so the call allocates nothing.
#include <mutex>
#include <string>

#include "../../include/d2ip.h"
#include "common.cuh"

namespace d2ip {
void record_op_error(const std::string& msg);
}

namespace {

// 16 MiB of partial-sum scratch.  Every GPU that loads the library keeps it until exit.
constexpr long long kNoAllocScratchBytes = 16LL << 20;
__device__ __align__(256) float g_wgrad_scratch[kNoAllocScratchBytes / sizeof(float)];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name
// is only a host-side stand-in, so the real address is looked up once per device (with that
// device current) and cached.
cudaError_t scratch_on_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_wgrad_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" d2ip_status d2ip_conv3d_wgrad_noalloc(const float* x, const float* dy, float* dWb,
                                                 int batch, int dz, int dy_, int dx_, int ci,
                                                 int co, int ksize, int stride,
                                                 long long dw_batch_stride, int accumulate,
                                                 void* stream) {
  using namespace d2ip;
  if (!x || !dy || !dWb) {
    record_op_error("null pointer");
    return D2IP_ERR_BAD_ARG;
  }
  const long long need =
      d2ip_conv3d_wgrad_workspace(batch, dz, dy_, dx_, ci, co, ksize, stride);
  if (need < 0) {
    record_op_error("bad convolution shape");
    return D2IP_ERR_BAD_SHAPE;
  }
  if (need > kNoAllocScratchBytes) {
    record_op_error("d2ip_conv3d_wgrad_noalloc: these sizes need " + std::to_string(need) +
                    " bytes of scratch, the static scratch holds " +
                    std::to_string(kNoAllocScratchBytes) +
                    " bytes; use d2ip_conv3d_wgrad with a caller workspace");
    return D2IP_ERR_BAD_SHAPE;
  }
  float* part = nullptr;
  cudaError_t e = scratch_on_current_device(&part);
  if (e != cudaSuccess) {
    record_op_error(std::string("scratch address lookup: ") + cudaGetErrorString(e));
    return D2IP_ERR_CUDA;
  }
  const Dims3 din{dz, dy_, dx_};
  const Dims3 dout = conv_out_dims(din, ksize, stride);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every partial the sum below reads is written first by this launch, so the scratch
  // needs no clearing between calls.
  e = conv3d_wgrad_partial_f32(x, dy, part, batch, din, ci, co, ksize, stride,
                               din.count() * ci, dout.count() * co, s);
  if (e == cudaSuccess) {
    const long long row = (long long)co * ksize * ksize * ksize * ci + co;
    e = reduce_rows_f32(part, dWb, batch, conv3d_wgrad_chunks(din, ksize, stride), row,
                        dw_batch_stride ? dw_batch_stride : row, accumulate, s);
  }
  if (e != cudaSuccess) {
    record_op_error(std::string("d2ip_conv3d_wgrad_noalloc launch: ") + cudaGetErrorString(e));
    return D2IP_ERR_CUDA;
  }
  return D2IP_OK;
}
