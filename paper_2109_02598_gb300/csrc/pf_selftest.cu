// Self-test of the bounded waits used by the kernels: one CTA waits, with a short clock
// budget, on an mbarrier phase that nothing will complete (the TMA kernels' wait), then on
// tagged words that nothing writes (the band kernel's wait for its neighbours' edge rows).
// Each wait gives up, the kernel records the timeouts in an error word and returns; the host
// reads the word. No copy is in flight and nothing waits without bound, so the GPU context
// stays usable.
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_sync.cuh"
#include "pf_tma.cuh"

namespace pf {
namespace {

// flag[0]: the mbarrier wait gave up; flag[1]: the tagged-word wait gave up; words: four
// tagged words that stay 0 (tag 0; the wait expects tag 1).
__global__ void wait_timeout_kernel(long long budget, int* flag,
                                    const unsigned long long* words) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival that never comes
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0u, budget);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(flag, 1);
  float v[4];
  if (threadIdx.x == 0 && !ll_wait<4>(words, 1u, budget, v)) atomicExch(flag + 1, 1);
}

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" int pf_selftest_wait_timeout(int64_t budget_cycles, void* stream) {
  if (budget_cycles < 1 || budget_cycles > 4000000000LL)
    return invalid("budget_cycles must be in [1, 4e9]");
  cudaStream_t s = (cudaStream_t)stream;
  int* d_flag = nullptr;
  int flag[2] = {0, 0};
  // two error words, then four tagged words (32-byte aligned)
  PF_CUDA_TRY(cudaMalloc(&d_flag, 64));
  const unsigned long long* words = reinterpret_cast<const unsigned long long*>(d_flag) + 4;
  cudaError_t e = cudaMemsetAsync(d_flag, 0, 64, s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 64, 0, s>>>((long long)budget_cycles, d_flag, words);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag, d_flag, sizeof(flag), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_flag);
  if (e != cudaSuccess) return cuda_fail(e, "pf_selftest_wait_timeout");
  if (flag[0] && flag[1]) {
    set_error("bounded wait ran out after %lld cycles (expected in this self-test)",
              (long long)budget_cycles);
    return PF_ERR_TIMEOUT;
  }
  if (flag[0] || flag[1]) {
    set_error("only the %s wait ran out", flag[0] ? "mbarrier" : "tagged-word");
    return PF_ERR_CUDA;
  }
  return PF_OK;
}
