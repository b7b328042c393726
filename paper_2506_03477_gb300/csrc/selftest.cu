// Self-test of the bounded device-side wait that every pipeline barrier of the tensor-core kernel
// uses (mbar_wait_bounded): one thread waits on an mbarrier phase that nothing completes, gives up
// after the limit, and records DEV_TIMEOUT, which the host returns as QSGW_ERR_TIMEOUT. The wait
// ends by the %globaltimer limit, so the kernel cannot hang, and the device stays usable.
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace qsgw {

__global__ void wait_timeout_selftest_kernel(unsigned long long limit_ns, int* d_err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one expected arrival that never comes: phase 0 never completes
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns)) atomicCAS(d_err, DEV_OK, DEV_TIMEOUT);
}

}  // namespace qsgw

using namespace qsgw;

extern "C" qsgw_status qsgw_selftest_wait_timeout(double limit_seconds, void* cuda_stream) {
  if (!(limit_seconds >= 1e-3 && limit_seconds <= 2.0)) return QSGW_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return QSGW_ERR_NOMEM;
  int h_err = -1;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)(limit_seconds * 1e9), d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) return QSGW_ERR_CUDA;
  return h_err == DEV_TIMEOUT ? QSGW_ERR_TIMEOUT : QSGW_OK;
}
