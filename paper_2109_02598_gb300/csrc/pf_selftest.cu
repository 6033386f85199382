// Self-test of the bounded-wait path used by the TMA kernels: one CTA waits, with a short
// clock budget, on an mbarrier phase that nothing will complete.  The wait gives up, the
// kernel records the timeout in an error word and returns; the host reads the word.  No
// copy is in flight and nothing waits without bound, so the GPU context stays usable.
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_tma.cuh"

namespace pf {
namespace {

__global__ void wait_timeout_kernel(long long budget, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival that never comes
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, budget);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(flag, 1);
}

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" int pf_selftest_wait_timeout(int64_t budget_cycles, void* stream) {
  if (budget_cycles < 1 || budget_cycles > 4000000000LL)
    return invalid("budget_cycles must be in [1, 4e9]");
  cudaStream_t s = (cudaStream_t)stream;
  int* d_flag = nullptr;
  int flag = 0;
  PF_CUDA_TRY(cudaMalloc(&d_flag, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 64, 0, s>>>((long long)budget_cycles, d_flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_flag);
  if (e != cudaSuccess) return cuda_fail(e, "pf_selftest_wait_timeout");
  if (flag) {
    set_error("bounded wait ran out after %lld cycles (expected in this self-test)",
              (long long)budget_cycles);
    return PF_ERR_TIMEOUT;
  }
  return PF_OK;
}
