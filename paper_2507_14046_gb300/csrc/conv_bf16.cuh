// Tensor-core (tcgen05, BF16 x BF16 -> FP32) path of the convolutions and J products.
#pragma once

#include <cstddef>

#include "common.cuh"

namespace d2ip {

// Device buffers of the BF16 path, carved from the context arena.
struct Bf16Net {
  __nv_bfloat16* wbf = nullptr;   // BF16 copy of theta (per problem, padded stride)
  __nv_bfloat16* xbf = nullptr;   // BF16 staging of a conv input
  __nv_bfloat16* Jbf = nullptr;   // BF16 copy of J
  long long Pp = 0;
};

bool bf16_network_supported(int levels, const int* widths, int c_in);
bool bf16_conv_supported(int ci, int co, int k);
// Reserve the BF16 buffers in the arena (base == nullptr: size only).
void bf16_layout(Bf16Net& bf, char* base, size_t& used, int B, long long Pp, long long max_act,
                 long long zin_count);
cudaError_t bf16_prepare_kernels();
cudaError_t bf16_prepare_weights(Bf16Net& bf, const float* theta, int B, long long Pp,
                                 cudaStream_t stream);
cudaError_t bf16_set_J(Bf16Net& bf, const float* J, int m, int n, cudaStream_t stream);
cudaError_t bf16_conv_fwd(Bf16Net& bf, const float* theta, long long w_off, const float* x,
                          float* y, int B, Dims3 din, int Ci, int Co, int K, int S,
                          long long x_bs, long long y_bs, long long w_bs, cudaStream_t stream);

}  // namespace d2ip
