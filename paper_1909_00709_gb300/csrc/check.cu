// Checksum interpolation (Theorem 1), detection (Sec. 3.4), location and correction
// (Sec. 3.5, Eq. 8 / Fig. 9), the offline chain of Fig. 10, and the plain checksum
// and source-term kernels used at set-up.
//
// Predictions, comparisons and corrections run in FP64; the per-tile partial sums
// of the sweep are reduced across tiles here, in a fixed order.
#include "device_common.cuh"

namespace abft {

constexpr int kCheckThreads = 256;

template <int ACC>
__device__ __forceinline__ double load_partial(const void* p, size_t i) {
  if (ACC == ABFT_ACC_FP32) return (double)static_cast<const float*>(p)[i];
  if (ACC == ABFT_ACC_TWOSUM) {
    const float2 q = static_cast<const float2*>(p)[i];
    return (double)q.x + (double)q.y;
  }
  return static_cast<const double*>(p)[i];
}

// a[z][x] of the last protected sweep: the tiles' partials summed in tile order
template <int ACC>
__device__ __forceinline__ double reduce_a(const GridDev& g, int z, int x) {
  double s = 0.0;
  for (int t = 0; t < g.nty; ++t) s += load_partial<ACC>(g.PA, ((size_t)t * g.nz + z) * g.pa_stride + x);
  return s;
}

template <int ACC>
__device__ __forceinline__ double reduce_b(const GridDev& g, int z, int y) {
  double s = 0.0;
  for (int t = 0; t < g.ntx; ++t) s += load_partial<ACC>(g.PB, ((size_t)t * g.nz + z) * g.ny + y);
  return s;
}

// Theorem 1 for the clamped 7-point set, one entry of a (Eq. 4): shifts along x and z
// are clamped index shifts of the vector; the two y-shifts add a to itself plus the
// boundary term (cn - cs) * (u[z][0][x] - u[z][ny-1][x]), zero when cn == cs.
__device__ __forceinline__ double predict_a(const GridDev& g, const double* A, const float* u, int z, int x) {
  const int nx = g.nx;
  const int xm = x > 0 ? x - 1 : 0, xp = x < nx - 1 ? x + 1 : nx - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double p = g.cx[(size_t)z * nx + x] + ((double)k.cc + (double)k.cn + (double)k.cs) * A[(size_t)z * nx + x] +
             (double)k.cw * A[(size_t)z * nx + xm] + (double)k.ce * A[(size_t)z * nx + xp] +
             (double)k.cb * A[(size_t)zm * nx + x] + (double)k.ct * A[(size_t)zp * nx + x];
  if (u != nullptr && k.cn != k.cs) {
    const size_t pl = (size_t)z * g.ny * g.px;
    p += ((double)k.cn - (double)k.cs) * ((double)u[pl + x] - (double)u[pl + (size_t)(g.ny - 1) * g.px + x]);
  }
  return p;
}

// Eq. (5): the same along y for the column checksum b
__device__ __forceinline__ double predict_b(const GridDev& g, const double* B, const float* u, int z, int y) {
  const int ny = g.ny;
  const int ym = y > 0 ? y - 1 : 0, yp = y < ny - 1 ? y + 1 : ny - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double p = g.cy[(size_t)z * ny + y] + ((double)k.cc + (double)k.cw + (double)k.ce) * B[(size_t)z * ny + y] +
             (double)k.cn * B[(size_t)z * ny + ym] + (double)k.cs * B[(size_t)z * ny + yp] +
             (double)k.cb * B[(size_t)zm * ny + y] + (double)k.ct * B[(size_t)zp * ny + y];
  if (u != nullptr && k.cw != k.ce) {
    const size_t row = ((size_t)z * g.ny + y) * g.px;
    p += ((double)k.cw - (double)k.ce) * ((double)u[row] - (double)u[row + g.nx - 1]);
  }
  return p;
}

// Sec. 3.4: flag unless |pred - comp| <= eps |comp| (NaN and Inf are flagged)
__device__ __forceinline__ bool fails(double pred, double comp, double eps) {
  return !(fabs(pred - comp) <= eps * fabs(comp));
}

__device__ __forceinline__ void append_fail(const GridDev& g, int z, int which, int idx) {
  const int k = atomicAdd(&g.fcnt[2 * z + which], 1);
  if (k < kFCap) g.fidx[(size_t)(2 * z + which) * kFCap + k] = idx;
}

// ------------------------------------------------ plane resolution (one block)

struct ResolveSmem {
  int fa[kFCap], fb[kFCap];
  int na, nb;
  double red[32];
  unsigned char flag[1024];
};

// Eq. (8) / Fig. 9 at (ex, ey) of plane z, using the interpolated vectors ap, bp.
// Both estimates are formed as "interpolated checksum minus the other points of
// the line", the same value as a' - (a - u) without cancelling against u.
__device__ void correct_point(const GridDev& g, int z, int ex, int ey, float* u, double* A, double* B,
                              const double* ap, const double* bp, long long step, DevCtrl* ctrl,
                              abft_event* ev, ResolveSmem& sm) {
  const size_t pl = (size_t)z * g.ny * g.px;
  double sa = 0.0, sb = 0.0;
  for (int y = threadIdx.x; y < g.ny; y += blockDim.x)
    if (y != ey) sa += (double)u[pl + (size_t)y * g.px + ex];
  sa = block_sum(sa, sm.red);
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x)
    if (x != ex) sb += (double)u[pl + (size_t)ey * g.px + x];
  sb = block_sum(sb, sm.red);
  if (threadIdx.x == 0) {
    const size_t c = pl + (size_t)ey * g.px + ex;
    const float bad = u[c];
    const double va = __ldcg(&ap[(size_t)z * g.nx + ex]) - sa;
    const double vb = __ldcg(&bp[(size_t)z * g.ny + ey]) - sb;
    const float f = (float)((va + vb) * 0.5);
    u[c] = f;
    A[(size_t)z * g.nx + ex] = sa + (double)f;
    B[(size_t)z * g.ny + ey] = sb + (double)f;
    log_event(ctrl, ev, step, g.gid, z, ey, ex, ABFT_EV_CORRECTED, bad, f);
  }
  __syncthreads();
}

// Recompute rows fb / columns fa of plane z from the intact previous state uin
// (whole plane when `all`), then sum the plane's checksums again.
__device__ void recompute_lines(const GridDev& g, int z, const float* uin, float* u, double* A, double* B,
                                bool all, long long step, DevCtrl* ctrl, abft_event* ev, ResolveSmem& sm) {
  const size_t pl = (size_t)z * g.ny * g.px;
  if (all) {
    for (int i = threadIdx.x; i < g.nx * g.ny; i += blockDim.x) {
      const int y = i / g.nx, x = i - y * g.nx;
      u[pl + (size_t)y * g.px + x] = point_update(g, uin, z, y, x);
    }
  } else {
    for (int k = 0; k < sm.nb; ++k)
      for (int x = threadIdx.x; x < g.nx; x += blockDim.x)
        u[pl + (size_t)sm.fb[k] * g.px + x] = point_update(g, uin, z, sm.fb[k], x);
    __syncthreads();
    for (int k = 0; k < sm.na; ++k)
      for (int y = threadIdx.x; y < g.ny; y += blockDim.x)
        u[pl + (size_t)y * g.px + sm.fa[k]] = point_update(g, uin, z, y, sm.fa[k]);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    double s = 0.0;
    for (int y = 0; y < g.ny; ++y) s += (double)u[pl + (size_t)y * g.px + x];
    A[(size_t)z * g.nx + x] = s;
  }
  for (int y = threadIdx.x; y < g.ny; y += blockDim.x) {
    double s = 0.0;
    for (int x = 0; x < g.nx; ++x) s += (double)u[pl + (size_t)y * g.px + x];
    B[(size_t)z * g.ny + y] = s;
  }
  if (threadIdx.x == 0) {
    if (all) {
      log_event(ctrl, ev, step, g.gid, z, -1, -1, ABFT_EV_RECOMPUTED, 0.f, 0.f);
    } else {
      for (int k = 0; k < sm.nb; ++k) log_event(ctrl, ev, step, g.gid, z, sm.fb[k], -1, ABFT_EV_RECOMPUTED, 0.f, 0.f);
      for (int k = 0; k < sm.na; ++k) log_event(ctrl, ev, step, g.gid, z, -1, sm.fa[k], ABFT_EV_RECOMPUTED, 0.f, 0.f);
    }
  }
  __syncthreads();
}

static __device__ void sort_small(int* v, int n) {
  for (int i = 1; i < n; ++i) {
    const int t = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
    v[j + 1] = t;
  }
}

// Location (Sec. 3.4/3.5) for every plane with failing entries; run by one block.
// uin == nullptr means no previous state is available: only single intersections
// can then be corrected, other patterns are counted in ctrl->verdict.
__device__ void resolve_planes(const GridDev& g, const float* uin, float* u, double* A, double* B,
                               const double* ap, const double* bp, long long step, DevCtrl* ctrl,
                               abft_event* ev, unsigned long long* unresolved) {
  __shared__ ResolveSmem sm;
  for (int zb = 0; zb < g.nz; zb += 1024) {
    const int zn = min(1024, g.nz - zb);
    for (int j = threadIdx.x; j < zn; j += blockDim.x)
      sm.flag[j] = (__ldcg(&g.fcnt[2 * (zb + j)]) | __ldcg(&g.fcnt[2 * (zb + j) + 1])) != 0;
    __syncthreads();
    for (int j = 0; j < zn; ++j) {
      if (!sm.flag[j]) continue;
      const int z = zb + j;
      if (threadIdx.x == 0) {
        const int ca = __ldcg(&g.fcnt[2 * z]), cb = __ldcg(&g.fcnt[2 * z + 1]);
        sm.na = ca;
        sm.nb = cb;
        for (int k = 0; k < min(ca, kFCap); ++k) sm.fa[k] = __ldcg(&g.fidx[(size_t)(2 * z) * kFCap + k]);
        for (int k = 0; k < min(cb, kFCap); ++k) sm.fb[k] = __ldcg(&g.fidx[(size_t)(2 * z + 1) * kFCap + k]);
        sort_small(sm.fa, min(ca, kFCap));
        sort_small(sm.fb, min(cb, kFCap));
        g.fcnt[2 * z] = 0;
        g.fcnt[2 * z + 1] = 0;
      }
      __syncthreads();
      const bool overflow = sm.na > kFCap || sm.nb > kFCap;
      if (sm.na == 1 && sm.nb == 1) {
        correct_point(g, z, sm.fa[0], sm.fb[0], u, A, B, ap, bp, step, ctrl, ev, sm);
      } else if (uin != nullptr) {
        if (overflow && threadIdx.x == 0) set_status(ctrl, kStFailOverflow);
        recompute_lines(g, z, uin, u, A, B, overflow, step, ctrl, ev, sm);
      } else if (threadIdx.x == 0) {
        atomicAdd(unresolved, 1ull);
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ online check

// One sweep's check (Sec. 3): reduce the partials into a^{t+1}, b^{t+1}; interpolate
// from a^t, b^t (Theorem 1); compare (Sec. 3.4); the last block to finish locates
// and corrects (Sec. 3.5) in place in u[out].
template <int ACC>
__global__ void __launch_bounds__(kCheckThreads)
    k_check_online(const GridDev g, int in, int out, DevCtrl* ctrl, abft_event* ev) {
  const int na = g.nz * g.nx, nb = g.nz * g.ny;
  const double* Ain = g.A[in];
  const double* Bin = g.B[in];
  double* Aout = g.A[out];
  double* Bout = g.B[out];
  const float* uin = g.u[in];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / g.nx, x = i - z * g.nx;
      const double s = reduce_a<ACC>(g, z, x);
      Aout[i] = s;
      const double p = predict_a(g, Ain, uin, z, x);
      g.AP[0][i] = p;
      if (fails(p, s, g.eps)) append_fail(g, z, 0, x);
    } else {
      const int j = i - na;
      const int z = j / g.ny, y = j - z * g.ny;
      const double s = reduce_b<ACC>(g, z, y);
      Bout[j] = s;
      const double p = predict_b(g, Bin, uin, z, y);
      g.BP[0][j] = p;
      if (fails(p, s, g.eps)) append_fail(g, z, 1, y);
    }
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&g.gc->done_check, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  resolve_planes(g, uin, g.u[out], Aout, Bout, g.AP[0], g.BP[0], g.gc->step - 1, ctrl, ev, &g.gc->unresolved);
  if (threadIdx.x == 0) g.gc->done_check = 0;
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
      if (fails(ap[i], a[i], g.eps)) {
        const int z = i / g.nx;
        append_fail(g, z, 0, i - z * g.nx);
        ++nf;
      }
    } else {
      const int j = i - na;
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

static int check_blocks(const GridDev& g) {
  const long long n = (long long)g.nz * (g.nx + g.ny);
  long long b = (n + kCheckThreads - 1) / kCheckThreads;
  if (b > 4 * 152) b = 4 * 152;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_check_online(const Launch& L, const GridDev& g, int in, int out) {
  const int blocks = check_blocks(g);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: k_check_online<ABFT_ACC_TWOSUM><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
    case ABFT_ACC_FP64: k_check_online<ABFT_ACC_FP64><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
    default: k_check_online<ABFT_ACC_FP32><<<blocks, kCheckThreads, 0, L.s>>>(g, in, out, L.ctrl, L.events); break;
  }
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
