// Device side of the check: cross-tile reduction of the sweep's partial checksums,
// the interpolation of Theorem 1, the relative test of Sec. 3.4, and location and
// correction (Sec. 3.5, Eq. 8 / Fig. 9) by one block.  Shared by the per-sweep
// check kernel and the persistent kernel.
#pragma once

#include "device_common.cuh"

namespace abft {


template <int ACC>
__device__ __forceinline__ double load_partial(const void* p, size_t i) {
  if (ACC == ABFT_ACC_FP32) return (double)__ldcg(static_cast<const float*>(p) + i);
  if (ACC == ABFT_ACC_TWOSUM) {
    const float2 q = __ldcg(static_cast<const float2*>(p) + i);
    return (double)q.x + (double)q.y;
  }
  return __ldcg(static_cast<const double*>(p) + i);
}

// Sum of n partials p[i0 + k*stride], k = 0..n-1, in order; loads are issued in
// batches of 8 so that their latencies overlap.
template <int ACC>
__device__ __forceinline__ double sum_partials(const void* p, size_t i0, size_t stride, int n) {
  double s = 0.0;
  int k = 0;
  for (; k + 8 <= n; k += 8) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = load_partial<ACC>(p, i0 + (size_t)(k + j) * stride);
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
  }
  for (; k < n; ++k) s += load_partial<ACC>(p, i0 + (size_t)k * stride);
  return s;
}

// a[z][x] of the last protected sweep: the tiles' partials summed in tile order
template <int ACC>
__device__ __forceinline__ double reduce_a(const GridDev& g, int z, int x, int pbuf = 0) {
  return sum_partials<ACC>(pbuf ? g.PA2 : g.PA, (size_t)z * g.pa_stride + x, (size_t)g.nz * g.pa_stride, g.nty);
}

template <int ACC>
__device__ __forceinline__ double reduce_b(const GridDev& g, int z, int y, int pbuf = 0) {
  return sum_partials<ACC>(pbuf ? g.PB2 : g.PB, (size_t)z * g.ny + y, (size_t)g.nz * g.ny, g.ntx);
}

// Theorem 1 for the clamped 7-point set, one entry of a (Eq. 4): shifts along x and z
// are clamped index shifts of the vector; the two y-shifts add a to itself plus the
// boundary term (cn - cs) * (u[z][0][x] - u[z][ny-1][x]), zero when cn == cs.
__device__ __forceinline__ double predict_a(const GridDev& g, const double* A, const float* u, int z, int x) {
  const int nx = g.nx;
  const int xm = x > 0 ? x - 1 : 0, xp = x < nx - 1 ? x + 1 : nx - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double p = g.cx[(size_t)z * nx + x] + ((double)k.cc + (double)k.cn + (double)k.cs) * __ldcg(A + (size_t)z * nx + x) +
             (double)k.cw * __ldcg(A + (size_t)z * nx + xm) + (double)k.ce * __ldcg(A + (size_t)z * nx + xp) +
             (double)k.cb * __ldcg(A + (size_t)zm * nx + x) + (double)k.ct * __ldcg(A + (size_t)zp * nx + x);
  if (u != nullptr && k.cn != k.cs) {
    const size_t pl = (size_t)z * g.ny * g.px;
    p += ((double)k.cn - (double)k.cs) *
         ((double)__ldcg(u + pl + x) - (double)__ldcg(u + pl + (size_t)(g.ny - 1) * g.px + x));
  }
  return p;
}

// Eq. (5): the same along y for the column checksum b
__device__ __forceinline__ double predict_b(const GridDev& g, const double* B, const float* u, int z, int y) {
  const int ny = g.ny;
  const int ym = y > 0 ? y - 1 : 0, yp = y < ny - 1 ? y + 1 : ny - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double p = g.cy[(size_t)z * ny + y] + ((double)k.cc + (double)k.cw + (double)k.ce) * __ldcg(B + (size_t)z * ny + y) +
             (double)k.cn * __ldcg(B + (size_t)z * ny + ym) + (double)k.cs * __ldcg(B + (size_t)z * ny + yp) +
             (double)k.cb * __ldcg(B + (size_t)zm * ny + y) + (double)k.ct * __ldcg(B + (size_t)zp * ny + y);
  if (u != nullptr && k.cw != k.ce) {
    const size_t row = ((size_t)z * g.ny + y) * g.px;
    p += ((double)k.cw - (double)k.ce) * ((double)__ldcg(u + row) - (double)__ldcg(u + row + g.nx - 1));
  }
  return p;
}

// Sec. 3.4: flag unless |pred - comp| <= eps |comp| (NaN and Inf are flagged)
__device__ __forceinline__ bool fails(double pred, double comp, double eps) {
  return !(fabs(pred - comp) <= eps * fabs(comp));
}

__device__ __forceinline__ void append_fail(const GridDev& g, int z, int which, int idx,
                                            unsigned* any = nullptr) {
  const int k = atomicAdd(&g.fcnt[2 * z + which], 1);
  if (k < kFCap) g.fidx[(size_t)(2 * z + which) * kFCap + k] = idx;
  if (any) atomicAdd(any, 1u);
}

// ------------------------------------------------ plane resolution (one block)

// what a resolution changed in one plane: a point (z, y, x), a row (z, y), a column
// (z, x) or the whole plane z; consumed by the persistent kernel's fix-up
enum FixKind { kFixPoint = 0, kFixRow = 1, kFixCol = 2, kFixPlane = 3 };
constexpr int kFixCap = 64;

struct ResolveSmem {
  int fa[kFCap], fb[kFCap];
  int na, nb;
  double red[32];
  unsigned char flag[1024];
  int4 fix[kFixCap];  // (kind, z, y, x)
  int nfix;
};

__device__ __forceinline__ void add_fix(ResolveSmem& sm, int kind, int z, int y, int x) {
  if (sm.nfix < kFixCap) sm.fix[sm.nfix] = make_int4(kind, z, y, x);
  ++sm.nfix;
}

// Eq. (8) / Fig. 9 at (ex, ey) of plane z, using the interpolated vectors ap, bp.
// Both estimates are formed as "interpolated checksum minus the other points of
// the line", the same value as a' - (a - u) without cancelling against u.
static __device__ void correct_point(const GridDev& g, int z, int ex, int ey, float* u, double* A, double* B,
                              const double* ap, const double* bp, long long step, DevCtrl* ctrl,
                              abft_event* ev, ResolveSmem& sm) {
  const size_t pl = (size_t)z * g.ny * g.px;
  double sa = 0.0, sb = 0.0;
  for (int y = threadIdx.x; y < g.ny; y += blockDim.x)
    if (y != ey) sa += (double)__ldcg(u + pl + (size_t)y * g.px + ex);
  sa = block_sum(sa, sm.red);
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x)
    if (x != ex) sb += (double)__ldcg(u + pl + (size_t)ey * g.px + x);
  sb = block_sum(sb, sm.red);
  if (threadIdx.x == 0) {
    const size_t c = pl + (size_t)ey * g.px + ex;
    const float bad = __ldcg(u + c);
    const double va = __ldcg(&ap[(size_t)z * g.nx + ex]) - sa;
    const double vb = __ldcg(&bp[(size_t)z * g.ny + ey]) - sb;
    const float f = (float)((va + vb) * 0.5);
    u[c] = f;
    A[(size_t)z * g.nx + ex] = sa + (double)f;
    B[(size_t)z * g.ny + ey] = sb + (double)f;
    log_event(ctrl, ev, step, g.gid, z, ey, ex, ABFT_EV_CORRECTED, bad, f);
    add_fix(sm, kFixPoint, z, ey, ex);
  }
  __syncthreads();
}

// Recompute rows fb / columns fa of plane z from the intact previous state uin
// (whole plane when `all`), then sum the plane's checksums again.
static __device__ void recompute_lines(const GridDev& g, int z, const float* uin, float* u, double* A, double* B,
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
    for (int y = 0; y < g.ny; ++y) s += (double)__ldcg(u + pl + (size_t)y * g.px + x);
    A[(size_t)z * g.nx + x] = s;
  }
  for (int y = threadIdx.x; y < g.ny; y += blockDim.x) {
    double s = 0.0;
    for (int x = 0; x < g.nx; ++x) s += (double)__ldcg(u + pl + (size_t)y * g.px + x);
    B[(size_t)z * g.ny + y] = s;
  }
  if (threadIdx.x == 0) {
    if (all) {
      log_event(ctrl, ev, step, g.gid, z, -1, -1, ABFT_EV_RECOMPUTED, 0.f, 0.f);
      add_fix(sm, kFixPlane, z, -1, -1);
    } else {
      for (int k = 0; k < sm.nb; ++k) {
        log_event(ctrl, ev, step, g.gid, z, sm.fb[k], -1, ABFT_EV_RECOMPUTED, 0.f, 0.f);
        add_fix(sm, kFixRow, z, sm.fb[k], -1);
      }
      for (int k = 0; k < sm.na; ++k) {
        log_event(ctrl, ev, step, g.gid, z, -1, sm.fa[k], ABFT_EV_RECOMPUTED, 0.f, 0.f);
        add_fix(sm, kFixCol, z, -1, sm.fa[k]);
      }
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
static __device__ void resolve_planes_into(ResolveSmem& sm, const GridDev& g, const float* uin, float* u, double* A,
                                           double* B, const double* ap, const double* bp, long long step,
                                           DevCtrl* ctrl, abft_event* ev, unsigned long long* unresolved) {
  if (threadIdx.x == 0) sm.nfix = 0;
  __syncthreads();
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

static __device__ void resolve_planes(const GridDev& g, const float* uin, float* u, double* A, double* B,
                                      const double* ap, const double* bp, long long step, DevCtrl* ctrl,
                                      abft_event* ev, unsigned long long* unresolved) {
  __shared__ ResolveSmem sm;
  resolve_planes_into(sm, g, uin, u, A, B, ap, bp, step, ctrl, ev, unresolved);
}

// One entry of the online check (Sec. 3): i < nz*nx addresses a[z][x], the rest b[z][y].
// Reduces the partials into a^{t+1} / b^{t+1}, interpolates from a^t / b^t (Theorem 1),
// stores the interpolation and appends the entry to its plane's list if it fails.
template <int ACC>
__device__ __forceinline__ void check_entry(const GridDev& g, int in, int out, int i, unsigned* any = nullptr,
                                            int pbuf = 0) {
  const int na = g.nz * g.nx;
  if (i < na) {
    const int z = i / g.nx, x = i - z * g.nx;
    const double s = reduce_a<ACC>(g, z, x, pbuf);
    g.A[out][i] = s;
    const double p = predict_a(g, g.A[in], g.u[in], z, x);
    g.AP[0][i] = p;
    if (fails(p, s, g.eps)) append_fail(g, z, 0, x, any);
  } else {
    const int j = i - na;
    const int z = j / g.ny, y = j - z * g.ny;
    const double s = reduce_b<ACC>(g, z, y, pbuf);
    g.B[out][j] = s;
    const double p = predict_b(g, g.B[in], g.u[in], z, y);
    g.BP[0][j] = p;
    if (fails(p, s, g.eps)) append_fail(g, z, 1, y, any);
  }
}

}  // namespace abft
