// Tensor-core path (tcgen05).  Not enabled yet: every query reports "unsupported", so the
// runtime rejects D2IP_BF16 at d2ip_set_network.
#include "conv_bf16.cuh"

namespace d2ip {

bool bf16_network_supported(int, const int*, int) { return false; }
bool bf16_conv_supported(int, int, int) { return false; }
void bf16_layout(Bf16Net&, char*, size_t&, int, long long, long long, long long) {}
cudaError_t bf16_prepare_kernels() { return cudaSuccess; }
cudaError_t bf16_prepare_weights(Bf16Net&, const float*, int, long long, cudaStream_t) {
  return cudaSuccess;
}
cudaError_t bf16_set_J(Bf16Net&, const float*, int, int, cudaStream_t) { return cudaSuccess; }
cudaError_t bf16_conv_fwd(Bf16Net&, const float*, long long, const float*, float*, int, Dims3,
                          int, int, int, int, long long, long long, long long, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace d2ip
