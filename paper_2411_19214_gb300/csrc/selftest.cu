// selftest.cu -- the failure path of the device-side waits, exercised without
// a fault: one CTA waits, with the same bounded mbarrier wait every pipeline
// role of the tensor-core kernels uses, on a barrier that nothing signals; the
// wait gives up after its limit, the kernel records the timeout in the error
// word (the same code path a stalled pipeline takes) and returns, and the
// context stays usable.
#include "tu_internal.cuh"

namespace {

__global__ void k_wait_selftest(uint64_t limit_ns, int* __restrict__ err, unsigned long long* __restrict__ waited) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tu::mbar_init(&bar, 1);
    abort_flag = 0;
    tu::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = tu::global_timer_ns();
    const bool ok = tu::mbar_wait(&bar, 0, &abort_flag, limit_ns);  // nothing arrives on phase 0
    *waited = tu::global_timer_ns() - t0;
    if (!ok) atomicCAS(err, tu::kErrNone, tu::kErrTimeout);
  }
}

}  // namespace

extern "C" tu_status tu_selftest_wait_timeout(double limit_seconds, double* waited_seconds) {
  if (!(limit_seconds > 0.0) || limit_seconds > 5.0) return TU_ERR_INVALID_ARG;
  int* err = nullptr;
  unsigned long long* waited = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return TU_ERR_OOM;
  if (cudaMalloc(&waited, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(err);
    return TU_ERR_OOM;
  }
  int h_err = 0;
  unsigned long long h_waited = 0;
  cudaError_t e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>((uint64_t)(limit_seconds * 1e9), err, waited);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h_waited, waited, sizeof(h_waited), cudaMemcpyDeviceToHost);
  cudaFree(err);
  cudaFree(waited);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TU_ERR_CUDA;
  }
  if (waited_seconds != nullptr) *waited_seconds = (double)h_waited * 1e-9;
  return h_err == tu::kErrTimeout ? TU_ERR_TIMEOUT : TU_OK;
}
