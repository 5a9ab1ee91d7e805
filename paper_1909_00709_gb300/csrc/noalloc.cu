// One protected sweep with its checksums, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool, a plugin whose host forbids device allocations after
// start-up, or a process that must not allocate while a CUDA graph is being
// captured.  abft_sweep_checksums_static gives them the fused sweep and the
// per-plane checksums of its result without a context or a workspace: the caller
// passes the input grid, the constant term, the output grid and the two checksum
// vectors, and the per-tile partial sums the sweep needs live in a fixed
// file-scope device array of kScratchBytes (8 MiB) that every GPU loading this
// library keeps until the process exits.
//
// Rules of use:
//   - The first call on a device looks up the array's device address (once per
//     device, with that device current).  Make that first call before any stream
//     capture begins.
//   - All calls share the one array.  Calls whose work overlaps on the GPU (two
//     streams, or two host threads) race on it; serialise them.
//   - Grids whose partials exceed the array are refused with ABFT_E_INVAL.
//   - Nothing here allocates: no cudaMalloc, cudaFree, pinned or managed memory.
//   - The sweep applies the clamped boundary rule (Fig. 2) and forms FP32 tile
//     partials that are reduced across tiles in FP64 (the ABFT_ACC_FP32 variant);
//     callers that need periodic or empty faces, or TwoSum/FP64 accumulation, use a
//     context.
#include <cstring>
#include <mutex>

#include "abft_internal.h"

namespace abft {
namespace {

constexpr size_t kScratchBytes = 8u << 20;
constexpr int kMaxDevices = 64;
constexpr int kStaticTy = 16;
constexpr size_t kCtrlBytes = 1024;  // DevCtrl + DevGridCtrl, kept at the front of the array

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices];  // device address of g_scratch, per device (null until set up)

constexpr size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Once per device, with that device current: the device address of g_scratch.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> hold(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace abft

using namespace abft;

extern "C" ABFT_API abft_status abft_sweep_checksums_static(const float* u_in, const float* C, float* u_out,
                                                            double* a_out, double* b_out, int32_t nx,
                                                            int32_t ny, int32_t nz, int64_t pitch,
                                                            const abft_coeffs* coeffs, void* stream) {
  if (!u_in || !C || !u_out || !a_out || !b_out || !coeffs) return ABFT_E_INVAL;
  if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || pitch < nx || pitch % 4 != 0 || pitch > (1 << 22))
    return ABFT_E_INVAL;
  if (u_in == u_out) return ABFT_E_INVAL;
  for (const void* p : {(const void*)u_in, (const void*)C, (const void*)u_out})
    if (((uintptr_t)p & 15) != 0) return ABFT_E_INVAL;
  if (((uintptr_t)a_out & 7) != 0 || ((uintptr_t)b_out & 7) != 0) return ABFT_E_INVAL;

  const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kStaticTy - 1) / kStaticTy;
  const size_t pa = round_up((size_t)nty * nz * ntx * kTX * sizeof(float), 256);
  const size_t pb = round_up((size_t)ntx * nz * round_up(ny, 4) * sizeof(float), 256);
  if (kCtrlBytes + pa + pb > kScratchBytes) return ABFT_E_INVAL;  // grid too large for the array

  void* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return ABFT_E_CUDA;
  unsigned char* s = static_cast<unsigned char*>(base);
  // the grid control block sits at round_up(sizeof(DevCtrl), 16), as placed below
  static_assert(round_up(sizeof(DevCtrl), 16) + sizeof(DevGridCtrl) <= kCtrlBytes, "control block must fit");

  GridDev g;
  memset(&g, 0, sizeof g);
  g.nx = nx; g.ny = ny; g.nz = nz; g.px = (int)pitch;
  g.ntx = ntx; g.nty = nty; g.ty = kStaticTy;
  g.pa_stride = ntx * kTX;
  g.pb_stride = (int)round_up(ny, 4);
  g.acc = ABFT_ACC_FP32;
  g.gid = 0;
  g.eps = 1e-5;
  g.k = Coef{coeffs->cc, coeffs->cw, coeffs->ce, coeffs->cn, coeffs->cs, coeffs->cb, coeffs->ct};
  g.u[0] = const_cast<float*>(u_in);
  g.u[1] = u_out;
  g.u[2] = u_out;
  g.C = const_cast<float*>(C);
  g.A[0] = a_out;
  g.B[0] = b_out;
  g.PA = s + kCtrlBytes;
  g.PB = s + kCtrlBytes + pa;
  DevCtrl* ctrl = reinterpret_cast<DevCtrl*>(s);
  g.gc = reinterpret_cast<DevGridCtrl*>(s + round_up(sizeof(DevCtrl), 16));

  CUtensorMap tm_u[3], tm_c;
  char err[128];
  if (make_tensor_maps(g, kStaticTy, tm_u, &tm_c, err, sizeof err) != cudaSuccess) return ABFT_E_CUDA;

  Launch L;
  L.s = static_cast<cudaStream_t>(stream);
  L.ctrl = ctrl;
  L.events = nullptr;
  L.sched.flips = nullptr;
  L.sched.off = nullptr;
  // the control block (tickets, step counter, injection off) must start at zero on every call
  if (cudaMemsetAsync(s, 0, kCtrlBytes, L.s) != cudaSuccess) return ABFT_E_CUDA;
  if (launch_sweep(L, g, tm_u[0], tm_c, 0, 1, true) != cudaSuccess) return ABFT_E_CUDA;
  if (launch_reduce_partials(L, g, 0) != cudaSuccess) return ABFT_E_CUDA;
  return ABFT_OK;
}
