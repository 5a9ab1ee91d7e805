// Self-test of the library's bounded device waits.
//
// Every spin-wait in the kernels (the grid barrier of the persistent kernels, the
// mbarrier waits on TMA copies) is bounded: when the awaited arrival never comes it
// gives up after its limit, records kStTimeout in the status word and lets the
// kernel return, so a broken launch turns into ABFT_E_TIMEOUT on the host and the
// CUDA context stays usable.  abft_selftest_wait makes one of those waits run out
// on purpose, without any fault:
//   case 0: a grid barrier that the last CTA of the launch never reaches (it returns
//           at once, like a block that died); the other CTAs wait, one of them times
//           out, the rest see the timeout bit while polling and leave;
//   case 1: an mbarrier that expects 16 bytes of transaction no copy will deliver.
// The control block is a file-scope device variable (no allocation); concurrent
// calls race on it and must be serialised.
#include <cstring>
#include <mutex>

#include "device_common.cuh"

namespace abft {
namespace {

struct SelftestState {
  DevCtrl ctrl;
  unsigned long long count;
};

static __device__ SelftestState g_selftest;

__global__ void k_selftest_barrier(SelftestState* st, unsigned long long limit_ns) {
  if (blockIdx.x == gridDim.x - 1) return;  // this CTA never arrives
  grid_barrier(&st->count, &st->ctrl, limit_ns);
}

__global__ void k_selftest_mbar(SelftestState* st, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 16);  // the arrival happens, the 16 bytes never do
    mbar_wait(&bar, 0, &st->ctrl, limit_ns);
  }
}

std::mutex g_lock;

}  // namespace
}  // namespace abft

using namespace abft;

extern "C" ABFT_API abft_status abft_selftest_wait(int32_t which, int64_t limit_us, void* stream,
                                                   double* elapsed_ms) {
  if ((which != 0 && which != 1) || limit_us < 1000 || limit_us > 10 * 1000 * 1000 || !elapsed_ms)
    return ABFT_E_INVAL;
  std::lock_guard<std::mutex> hold(g_lock);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SelftestState* st = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void**>(&st), g_selftest) != cudaSuccess) return ABFT_E_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ABFT_E_CUDA;
  abft_status r = ABFT_E_CUDA;
  SelftestState h;
  float ms = 0.f;
  const unsigned long long limit_ns = (unsigned long long)limit_us * 1000ull;
  do {
    if (cudaMemsetAsync(st, 0, sizeof(SelftestState), s) != cudaSuccess) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) break;
    if (which == 0)
      k_selftest_barrier<<<4, 32, 0, s>>>(st, limit_ns);
    else
      k_selftest_mbar<<<1, 32, 0, s>>>(st, limit_ns);
    if (cudaGetLastError() != cudaSuccess) break;
    if (cudaEventRecord(e1, s) != cudaSuccess) break;
    if (cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) break;
    *elapsed_ms = ms;
    r = (h.ctrl.status & kStTimeout) ? ABFT_E_TIMEOUT : ABFT_OK;
  } while (0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}
