// Kernels of the check (Theorem 1, Sec. 3.4, Sec. 3.5), the offline chain of Fig. 10,
// and the plain checksum and source-term kernels used at set-up.
//
// Predictions, comparisons and corrections run in FP64; the per-tile partial sums
// of the sweep are reduced across tiles in a fixed order.
#include <algorithm>

#include "check_dev.cuh"

namespace abft {

constexpr int kCheckThreads = 256;

// ------------------------------------------------------------ online check

// One sweep's check (Sec. 3): reduce the partials into a^{t+1}, b^{t+1}; interpolate
// from a^t, b^t (Theorem 1); compare (Sec. 3.4).  Failing entries go to the per-plane
// lists that k_resolve then works through.
template <int ACC>
__global__ void __launch_bounds__(kCheckThreads)
    k_check_online(const GridDev g, int in, int out, DevCtrl* ctrl, abft_event* ev) {
  (void)ctrl;
  (void)ev;
  const int n = g.nz * (g.nx + g.ny), first = g.vec == 1 ? g.nz * g.nx : 0;
  const int nw = kCheckThreads / 32;
  check_warps<ACC>(g, in, out, blockIdx.x * nw + (int)(threadIdx.x >> 5), gridDim.x * nw, first, n);
}

// The same check with the partials brought in by TMA: warp w of a block takes rounds
// of 32 entries, one box of all tiles' partials per round in its own shared-memory
// buffer (grids with at most 256 tiles along x and along y).
template <int ACC>
__global__ void __launch_bounds__(256)
    k_check_box(const GridDev g, const __grid_constant__ PartialMaps pm, int in, int out, DevCtrl* ctrl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int box = (check_box_bytes(g.nty, g.ntx, ACC) + 127) / 128 * 128;
  unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base) + warp;  // at most 8 warps: 64 bytes of the 128-byte head
  unsigned char* buf = base + 128 + (size_t)warp * box;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    prefetch_tensormap(&pm.m[0]);
    prefetch_tensormap(&pm.m[2]);
  }
  __syncwarp();
  unsigned phase = 0;
  const InterpW iw(g.k);
  const int rounds = check_rounds_of(g);
  for (int r = blockIdx.x * nw + warp; r < rounds; r += gridDim.x * nw)
    check_box_round<ACC>(g, iw, pm.m, in, out, 0, r, buf, bar, phase, ctrl, nullptr);
}

// Location and correction (Sec. 3.5) after the online check of the sweep just done,
// one block per plane with failing entries (planes are independent): a single
// intersection by Eq. (8), other patterns by recomputing lines from u[in].
__global__ void __launch_bounds__(kCheckThreads)
    k_resolve(const GridDev g, int in, int out, DevCtrl* ctrl, abft_event* ev, long long step) {
  __shared__ ResolveSmem sm;
  __shared__ int s_hit;
  if (threadIdx.x == 0) sm.nfix = 0;
  for (int z = blockIdx.x; z < g.nz; z += gridDim.x) {
    if (threadIdx.x == 0) s_hit = (__ldcg(&g.fcnt[2 * z]) | __ldcg(&g.fcnt[2 * z + 1])) != 0;
    __syncthreads();
    const bool hit = s_hit != 0;
    __syncthreads();  // every thread has read s_hit before thread 0 rewrites it
    if (hit) {
      resolve_plane(sm, g, g.u[in], g.u[out], g.A[out], g.B[out], g.AP[0], g.BP[0], step, ctrl, ev,
                    &g.gc->unresolved, z, g.vec == 1);
      // u[out] changed: a next sweep already started is stale in every tile whose
      // stencil read a changed point (with periodic boundaries a fix on a face also
      // reaches the opposite face: every tile row or column, or every plane)
      if (threadIdx.x == 0) {
        const int ntiles = g.ntx * g.nty;
        int* hi1 = g.tdirty;            // highest marked plane + 1
        int* lorev = g.tdirty + ntiles;  // nz - lowest marked plane
        const bool every = sm.nfix > kFixCap;  // the list overflowed: the whole plane
        for (int k = 0; k < (every ? 1 : sm.nfix); ++k) {
          const int4 f = every ? make_int4(kFixPlane, z, -1, -1) : sm.fix[k];  // (kind, z, y, x)
          const bool wrap = g.bc == ABFT_BC_PERIODIC;
          const bool all_y = f.x == kFixPlane || f.x == kFixCol || (wrap && (f.z == 0 || f.z == g.ny - 1));
          const bool all_x = f.x == kFixPlane || f.x == kFixRow || (wrap && (f.w == 0 || f.w == g.nx - 1));
          const bool all_z = wrap && (f.y == 0 || f.y == g.nz - 1);
          const int y0 = all_y ? 0 : max(f.z - 1, 0) / g.ty, y1 = all_y ? g.nty - 1 : min(f.z + 1, g.ny - 1) / g.ty;
          const int x0 = all_x ? 0 : max(f.w - 1, 0) / kTX, x1 = all_x ? g.ntx - 1 : min(f.w + 1, g.nx - 1) / kTX;
          for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) {
              atomicMax(&hi1[ty * g.ntx + tx], all_z ? g.nz : f.y + 1);
              atomicMax(&lorev[ty * g.ntx + tx], all_z ? g.nz : g.nz - f.y);
            }
        }
        sm.nfix = 0;
        atomicExch(&g.gc->redo, 1u);
      }
      __syncthreads();
    }
  }
  // the plane list of the one-vector check was consumed by k_demand_sums (an earlier
  // launch); the next check starts a new one
  if (g.vec == 1 && blockIdx.x == 0 && threadIdx.x == 0) g.gc->nbz = 0;
}

// One-vector checks (Sec. 3.2): the on-demand column sums before the location step, as
// a launch of its own (per-launch paths; the persistent kernel runs demand_sums itself).
__global__ void __launch_bounds__(256) k_demand_sums(const GridDev g, int in, int out) {
  demand_sums(g, g.u[in], g.u[out], g.A[out], g.AP[1], blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------ offline pieces

template <int ACC>
__global__ void __launch_bounds__(kCheckThreads) k_reduce_partials(const GridDev g, int out) {
  const int na = g.nz * g.nx, nb = g.nz * g.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / g.nx, x = i - z * g.nx;
      g.A[out][i] = reduce_a<ACC>(g, z, x);
    } else {
      const int j = i - na;
      const int z = j / g.ny, y = j - z * g.ny;
      g.B[out][j] = reduce_b<ACC>(g, z, y);
    }
  }
}

// one link of the chain of Fig. 10: Eq. (6)/(7) (boundary terms vanish)
__global__ void __launch_bounds__(kCheckThreads)
    k_chain(const GridDev g, const double* a_in, const double* b_in, double* a_out, double* b_out) {
  const int na = g.nz * g.nx, nb = g.nz * g.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / g.nx, x = i - z * g.nx;
      a_out[i] = predict_a(g, a_in, nullptr, z, x);
    } else {
      const int j = i - na;
      const int z = j / g.ny, y = j - z * g.ny;
      b_out[j] = predict_b(g, b_in, nullptr, z, y);
    }
  }
}

// Compare interpolated (ap, bp) with recomputed (a, b); failing entries go to the
// per-plane lists and are counted in the grid's verdict.
__global__ void __launch_bounds__(kCheckThreads)
    k_compare(const GridDev g, const double* ap, const double* bp, const double* a, const double* b) {
  const int na = g.nz * g.nx, nb = g.nz * g.ny;
  unsigned long long nf = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += gridDim.x * blockDim.x) {
    if (i < na) {
      note_resid(g, ap[i], a[i]);
      if (fails(ap[i], a[i], g.eps)) {
        const int z = i / g.nx;
        append_fail(g, z, 0, i - z * g.nx);
        ++nf;
      }
    } else {
      const int j = i - na;
      note_resid(g, bp[j], b[j]);
      if (fails(bp[j], b[j], g.eps)) {
        const int z = j / g.ny;
        append_fail(g, z, 1, j - z * g.ny);
        ++nf;
      }
    }
  }
  nf = (unsigned long long)warp_sum((double)nf);
  if ((threadIdx.x & 31) == 0 && nf) atomicAdd(&g.gc->verdict, nf);
}

__global__ void k_clear_fails(const GridDev g) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * g.nz; i += gridDim.x * blockDim.x) g.fcnt[i] = 0;
}

// correct the current state from the fail lists (abft_correct at zero distance)
__global__ void __launch_bounds__(kCheckThreads)
    k_correct_planes(const GridDev g, int cur, const double* ap, const double* bp, DevCtrl* ctrl,
                     abft_event* ev) {
  resolve_planes(g, nullptr, g.u[cur], g.A[cur], g.B[cur], ap, bp, g.gc->step - 1, ctrl, ev, &g.gc->unresolved);
}

// ------------------------------------------------------------ set-up kernels

// HotSpot-like constant term of Eq. (1): C holds P on entry, sdc*P + c_amb*t_amb on exit
__global__ void k_source_term(const GridDev g, float sdc, float amb) {
  const size_t n = (size_t)g.nz * g.ny * g.px;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.px);
    g.C[i] = x < g.nx ? __fmaf_rn(sdc, g.C[i], amb) : 0.f;
  }
}

// Eq. (2): a[z][x] = sum over y, one thread per column, sequential in y (FP64)
__global__ void k_checksum_a(const GridDev g, const float* u, double* A) {
  const int z = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const float* p = u + (size_t)z * g.ny * g.px + x;
  double s = 0.0;
  for (int y = 0; y < g.ny; ++y) s += (double)p[(size_t)y * g.px];
  A[(size_t)z * g.nx + x] = s;
}

// Eq. (3): b[z][y] = sum over x, one warp per row (FP64, fixed order)
__global__ void k_checksum_b(const GridDev g, const float* u, double* B) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= g.nz * g.ny) return;
  const int z = warp / g.ny, y = warp - z * g.ny;
  const float* p = u + ((size_t)z * g.ny + y) * g.px;
  double s = 0.0;
  for (int x = lane; x < g.nx; x += 32) s += (double)p[x];
  s = warp_sum(s);
  if (lane == 0) B[warp] = s;
}

// ------------------------------------------------------------------ launchers

static int check_blocks(const GridDev& g, int lanes = 1) {
  const long long n = (long long)g.nz * (g.nx + g.ny) * lanes;
  long long b = (n + kCheckThreads - 1) / kCheckThreads;
  if (b > 65535) b = 65535;
  return (int)(b < 1 ? 1 : b);
}

// multiprocessors of the current device (cached per device)
static int sm_count() {
  static int cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}

int check_box_warps(int box_bytes) {
  const int nw = 65536 / (box_bytes + 128);
  return nw < 1 ? 1 : (nw > 8 ? 8 : nw);
}

bool check_box_usable(const GridDev& g) { return g.nty <= 256 && g.ntx <= 256; }

int check_box_bytes_host(int nty, int ntx, int acc) { return check_box_bytes(nty, ntx, acc); }

cudaError_t launch_check_online(const Launch& L, const GridDev& g, const PartialMaps& pm, int in, int out,
                                int max_warps) {
  if (check_box_usable(g)) {
    const int box = (check_box_bytes(g.nty, g.ntx, g.acc) + 127) / 128 * 128;
    const int nw = std::min(check_box_warps(box), std::max(max_warps, 1));
    const int smem = 256 + nw * box;
    const long long rounds = check_rounds_host(g);
    const int blocks = (int)std::min<long long>((rounds + nw - 1) / nw, (nw == 1 ? 8LL : 4LL) * sm_count());
    cudaError_t e = cudaSuccess;
    switch (g.acc) {
      case ABFT_ACC_TWOSUM:
        e = cudaFuncSetAttribute(k_check_box<ABFT_ACC_TWOSUM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_check_box<ABFT_ACC_TWOSUM><<<blocks, nw * 32, smem, L.s>>>(g, pm, in, out, L.ctrl);
        break;
      case ABFT_ACC_FP64:
        e = cudaFuncSetAttribute(k_check_box<ABFT_ACC_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_check_box<ABFT_ACC_FP64><<<blocks, nw * 32, smem, L.s>>>(g, pm, in, out, L.ctrl);
        break;
      default:
        e = cudaFuncSetAttribute(k_check_box<ABFT_ACC_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_check_box<ABFT_ACC_FP32><<<blocks, nw * 32, smem, L.s>>>(g, pm, in, out, L.ctrl);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  // 32 entries per warp, up to one wave of 8 blocks per SM; further entries by striding
  const long long entries = (long long)g.nz * (g.nx + g.ny) - check_entries_first(g);
  const int blocks = (int)std::min<long long>((entries + kCheckThreads - 1) / kCheckThreads, 8LL * sm_count());
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: k_check_online<ABFT_ACC_TWOSUM><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
    case ABFT_ACC_FP64: k_check_online<ABFT_ACC_FP64><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
    default: k_check_online<ABFT_ACC_FP32><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_resolve(const Launch& L, const GridDev& g, int in, int out, long long step) {
  if (g.vec == 1) {
    k_demand_sums<<<2 * sm_count(), 256, 0, L.s>>>(g, in, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_resolve<<<std::min(g.nz, 1024), kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events, step);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const Launch& L, const GridDev& g, int out) {
  const int blocks = check_blocks(g);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: k_reduce_partials<ABFT_ACC_TWOSUM><<<blocks, kCheckThreads, 0, L.s>>>(g, out); break;
    case ABFT_ACC_FP64: k_reduce_partials<ABFT_ACC_FP64><<<blocks, kCheckThreads, 0, L.s>>>(g, out); break;
    default: k_reduce_partials<ABFT_ACC_FP32><<<blocks, kCheckThreads, 0, L.s>>>(g, out); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_chain(const Launch& L, const GridDev& g, const double* a_in, const double* b_in,
                         double* a_out, double* b_out) {
  k_chain<<<check_blocks(g), kCheckThreads, 0, L.s>>>(g, a_in, b_in, a_out, b_out);
  return cudaGetLastError();
}

cudaError_t launch_compare(const Launch& L, const GridDev& g, const double* ap, const double* bp,
                           const double* a, const double* b) {
  k_clear_fails<<<1, 256, 0, L.s>>>(g);
  k_compare<<<check_blocks(g), kCheckThreads, 0, L.s>>>(g, ap, bp, a, b);
  return cudaGetLastError();
}

cudaError_t launch_correct_planes(const Launch& L, const GridDev& g, int cur, const double* ap,
                                  const double* bp) {
  k_correct_planes<<<1, kCheckThreads, 0, L.s>>>(g, cur, ap, bp, L.ctrl, L.events);
  return cudaGetLastError();
}

cudaError_t launch_source_term(const Launch& L, const GridDev& g, const abft_coeffs& co) {
  const float amb = co.c_amb * co.t_amb;
  k_source_term<<<4 * 152, 256, 0, L.s>>>(g, co.sdc, amb);
  return cudaGetLastError();
}

cudaError_t launch_checksums(const Launch& L, const GridDev& g, const float* u, double* A, double* B) {
  dim3 ga((g.nx + 127) / 128, g.nz);
  k_checksum_a<<<ga, 128, 0, L.s>>>(g, u, A);
  const long long warps = (long long)g.nz * g.ny;
  k_checksum_b<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, L.s>>>(g, u, B);
  return cudaGetLastError();
}

}  // namespace abft
