// Measurement probe: sustained L2 copy bandwidth of this GPU.
//
// Grids small enough to stay in the 129 MB L2 (the 512x512x8 workload moves 24 MB
// per sweep) are not bound by HBM; their roofline is the rate at which the SMs can
// stream data through L2.  A copy by torch or cudaMemcpy of such a buffer is too
// short to measure that rate (one launch of a few microseconds is mostly launch
// latency), so this probe copies src -> dst `passes` times inside one persistent
// launch of 2 CTAs per SM, 16-byte loads and stores that bypass L1 (.cg), and
// times the launch with CUDA events.  Bytes moved = 2 * bytes * passes.
#include "abft_internal.h"

namespace abft {
namespace {

__global__ void __launch_bounds__(512) k_l2_copy(const float4* __restrict__ src, float4* __restrict__ dst,
                                                 size_t n, int passes) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float4 v;
      asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "l"(src + i));
      asm volatile("st.global.cg.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + i), "f"(v.x), "f"(v.y), "f"(v.z),
                   "f"(v.w)
                   : "memory");
    }
  }
}

}  // namespace
}  // namespace abft

using namespace abft;

extern "C" ABFT_API abft_status abft_probe_l2_copy(const void* src, void* dst, size_t bytes, int32_t passes,
                                                   void* stream, double* elapsed_ms) {
  if (!src || !dst || !elapsed_ms || bytes == 0 || bytes % 16 != 0 || passes < 1 || passes > 100000)
    return ABFT_E_INVAL;
  if (((uintptr_t)src & 15) != 0 || ((uintptr_t)dst & 15) != 0) return ABFT_E_INVAL;
  const char* s0 = static_cast<const char*>(src);
  const char* d0 = static_cast<const char*>(dst);
  if (s0 < d0 + bytes && d0 < s0 + bytes) return ABFT_E_INVAL;  // overlapping buffers
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ABFT_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ABFT_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return ABFT_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ABFT_E_CUDA;
  }
  const size_t n = bytes / 16;
  // one warm-up pass brings both buffers into L2, then the timed launch
  k_l2_copy<<<2 * sms, 512, 0, st>>>(static_cast<const float4*>(src), static_cast<float4*>(dst), n, 1);
  cudaEventRecord(e0, st);
  k_l2_copy<<<2 * sms, 512, 0, st>>>(static_cast<const float4*>(src), static_cast<float4*>(dst), n, passes);
  cudaEventRecord(e1, st);
  abft_status r = ABFT_OK;
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    r = ABFT_E_CUDA;
  *elapsed_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}
