// Self-test of the bounded-wait error path: a one-thread kernel waits on a device flag with an
// iteration limit, the way the tensor-core kernels wait on their pipeline barriers; when the
// limit runs out it records an error code in a status word instead of hanging or trapping, and
// the host turns that code into D2IP_ERR_TIMEOUT.  The context stays usable afterwards.
#include <cuda_runtime.h>

#include "../../include/d2ip.h"

namespace {

__global__ void wait_flag_kernel(const volatile int* flag, long long limit, int* status) {
  for (long long i = 0; i < limit; ++i) {
    if (*flag != 0) {
      *status = 0;
      return;
    }
    __nanosleep(64);
  }
  *status = 2;  // gave up
}

}  // namespace

extern "C" d2ip_status d2ip_wait_selftest(int device, long long spin_limit, int set_flag,
                                          int* status_out) {
  if (spin_limit < 1 || spin_limit > (1LL << 26) || !status_out) return D2IP_ERR_BAD_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return D2IP_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return D2IP_ERR_CUDA;
  int* buf = nullptr;  // [0] the flag, [1] the status word
  if (cudaMalloc(&buf, 2 * sizeof(int)) != cudaSuccess) return D2IP_ERR_OOM;
  const int init[2] = {set_flag ? 1 : 0, -1};
  int st = -1;
  cudaError_t e = cudaMemcpy(buf, init, sizeof(init), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    wait_flag_kernel<<<1, 1>>>(buf, spin_limit, buf + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&st, buf + 1, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return D2IP_ERR_CUDA;
  *status_out = st;
  return st == 0 ? D2IP_OK : (st == 2 ? D2IP_ERR_TIMEOUT : D2IP_ERR_CUDA);
}
