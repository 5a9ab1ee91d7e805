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

// The canonical cross-tile sum of n partials p[i0 + k*stride]: eight interleaved
// lanes j accumulate p_k over k = j, j+8, j+16, ... (ascending), then the lanes are
// combined in order 0..7.  FP32 and TwoSum partials are accumulated as compensated
// FP32 pairs (hi, lo) with TwoSum (error about n u^2, below FP64 rounding of the
// total here, and at FP32 speed: GB300's FP64 rate is a small fraction of its FP32
// rate); the pair is widened once, hi + lo in FP64.  The FP64 variant sums in FP64.
// Every path (one thread per entry, or eight cooperating warps) evaluates exactly
// this, so results agree bit for bit.
constexpr int kLanes = 8;

template <int ACC>
struct PartialType { using T = float; };
template <>
struct PartialType<ABFT_ACC_TWOSUM> { using T = float2; };
template <>
struct PartialType<ABFT_ACC_FP64> { using T = double; };

template <int ACC>
__device__ __forceinline__ typename PartialType<ACC>::T load_raw(const void* p, size_t i) {
  return __ldcg(static_cast<const typename PartialType<ACC>::T*>(p) + i);
}

// running sum of one lane: (hi, lo) FP32 pair, or d for the FP64 variant
struct LaneSum {
  float hi = 0.f, lo = 0.f;
  double d = 0.0;
  __device__ __forceinline__ void add(float v) { acc2(hi, lo, v); }
  __device__ __forceinline__ void add(float2 v) {
    acc2(hi, lo, v.x);
    lo += v.y;
  }
  __device__ __forceinline__ void add(double v) { d = __dadd_rn(d, v); }
  // lane combination: (this) += other, in the same arithmetic
  template <int ACC>
  __device__ __forceinline__ void merge(const LaneSum& o) {
    if (ACC == ABFT_ACC_FP64) {
      d = __dadd_rn(d, o.d);
    } else {
      acc2(hi, lo, o.hi);
      lo += o.lo;
    }
  }
  template <int ACC>
  __device__ __forceinline__ double total() const {
    return ACC == ABFT_ACC_FP64 ? d : __dadd_rn((double)hi, (double)lo);
  }
};

template <int ACC>
__device__ __forceinline__ LaneSum lane_sum(const void* p, size_t i0, size_t stride, int n, int j) {
  LaneSum t;
  for (int k = j; k < n; k += kLanes) t.add(load_raw<ACC>(p, i0 + (size_t)k * stride));
  return t;
}

template <int ACC>
__device__ __forceinline__ double sum_partials(const void* p, size_t i0, size_t stride, int n) {
  LaneSum s = lane_sum<ACC>(p, i0, stride, n, 0);
#pragma unroll
  for (int j = 1; j < kLanes; ++j) s.merge<ACC>(lane_sum<ACC>(p, i0, stride, n, j));
  return s.total<ACC>();
}

// a[z][x] of the last protected sweep: the tiles' partials summed in the canonical order
template <int ACC>
__device__ __forceinline__ double reduce_a(const GridDev& g, int z, int x, int pbuf = 0) {
  return sum_partials<ACC>(pbuf ? g.PA2 : g.PA, (size_t)z * g.pa_stride + x, (size_t)g.nz * g.pa_stride, g.nty);
}

template <int ACC>
__device__ __forceinline__ double reduce_b(const GridDev& g, int z, int y, int pbuf = 0) {
  return sum_partials<ACC>(pbuf ? g.PB2 : g.PB, (size_t)z * g.pb_stride + y, (size_t)g.nz * g.pb_stride, g.ntx);
}

// Theorem 1 for the clamped 7-point set (Eq. 4 for a, Eq. 5 for b): shifts along the
// surviving in-plane axis and along z are clamped index shifts of the vector; the two
// shifts along the collapsed axis add the entry to itself plus the boundary term
// (w_- - w_+) * (u at the first minus u at the last index), zero for equal weights.
// Evaluated with explicit FP64 roundings in a fixed order: c the checksum of C, v0 the
// entry, v1/v2 its clamped neighbours along the surviving in-plane axis, v3/v4 along z,
// w0 the summed weight of the centre and the collapsed-axis pair.
__device__ __forceinline__ double interp(double c, double v0, double v1, double v2, double v3, double v4,
                                         double w0, double w1, double w2, double w3, double w4, double edge) {
  double p = __fma_rn(w0, v0, c);
  p = __fma_rn(w1, v1, p);
  p = __fma_rn(w2, v2, p);
  p = __fma_rn(w3, v3, p);
  p = __fma_rn(w4, v4, p);
  return __dadd_rn(p, edge);
}

__device__ __forceinline__ double weight_sum3(float a, float b, float c) {
  return __dadd_rn(__dadd_rn((double)a, (double)b), (double)c);
}

__device__ __forceinline__ double edge_term(float wm, float wp, float first, float last) {
  return __dmul_rn(__dadd_rn((double)wm, -(double)wp), __dadd_rn((double)first, -(double)last));
}

__device__ __forceinline__ double predict_a(const GridDev& g, const double* A, const float* u, int z, int x) {
  const int nx = g.nx;
  const int xm = x > 0 ? x - 1 : 0, xp = x < nx - 1 ? x + 1 : nx - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double edge = 0.0;
  if (u != nullptr && k.cn != k.cs) {
    const size_t pl = (size_t)z * g.ny * g.px;
    edge = edge_term(k.cn, k.cs, __ldcg(u + pl + x), __ldcg(u + pl + (size_t)(g.ny - 1) * g.px + x));
  }
  return interp(g.cx[(size_t)z * nx + x], __ldcg(A + (size_t)z * nx + x), __ldcg(A + (size_t)z * nx + xm),
                __ldcg(A + (size_t)z * nx + xp), __ldcg(A + (size_t)zm * nx + x), __ldcg(A + (size_t)zp * nx + x),
                weight_sum3(k.cc, k.cn, k.cs), k.cw, k.ce, k.cb, k.ct, edge);
}

__device__ __forceinline__ double predict_b(const GridDev& g, const double* B, const float* u, int z, int y) {
  const int ny = g.ny;
  const int ym = y > 0 ? y - 1 : 0, yp = y < ny - 1 ? y + 1 : ny - 1;
  const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
  const Coef& k = g.k;
  double edge = 0.0;
  if (u != nullptr && k.cw != k.ce) {
    const size_t row = ((size_t)z * g.ny + y) * g.px;
    edge = edge_term(k.cw, k.ce, __ldcg(u + row), __ldcg(u + row + g.nx - 1));
  }
  return interp(g.cy[(size_t)z * ny + y], __ldcg(B + (size_t)z * ny + y), __ldcg(B + (size_t)z * ny + ym),
                __ldcg(B + (size_t)z * ny + yp), __ldcg(B + (size_t)zm * ny + y), __ldcg(B + (size_t)zp * ny + y),
                weight_sum3(k.cc, k.cw, k.ce), k.cn, k.cs, k.cb, k.ct, edge);
}

// Sec. 3.4: flag unless |pred - comp| <= eps |comp| (NaN and Inf are flagged)
__device__ __forceinline__ bool fails(double pred, double comp, double eps) {
  return !(fabs(pred - comp) <= eps * fabs(comp));
}

// the running maximum of |pred - comp| / |comp| over passing entries (a non-negative
// double's bits order like its value, so an integer maximum suffices)
__device__ __forceinline__ void note_resid(const GridDev& g, double pred, double comp) {
  if (!g.track) return;
  const double rel = fabs(pred - comp) / fabs(comp);
  if (rel <= g.eps) atomicMax(&g.gc->max_resid, (unsigned long long)__double_as_longlong(rel));
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
    note_resid(g, p, s);
  } else {
    const int j = i - na;
    const int z = j / g.ny, y = j - z * g.ny;
    const double s = reduce_b<ACC>(g, z, y, pbuf);
    g.B[out][j] = s;
    const double p = predict_b(g, g.B[in], g.u[in], z, y);
    g.BP[0][j] = p;
    if (fails(p, s, g.eps)) append_fail(g, z, 1, y, any);
    note_resid(g, p, s);
  }
}

// ------------------------------------------------------------ block check rounds
// One round of the online check (Sec. 3) by a block of 8 warps: 32 consecutive
// entries, entry e = base + lane.  Warp w is lane w of the canonical sum: it loads the
// partials k = w, w+8, ... of its lane's entry (coalesced across the warp) and one
// interpolation input (w = 0..4 the entry and its neighbours, 5 the constant-term
// checksum, 6/7 the boundary-term values).  finish() meets the eight warp sums in
// shared memory and warp 0 adds them in order, interpolates and tests.  load()
// before a sweep and finish() after it hide the load latency.  The arithmetic is that
// of sum_partials and predict_a/b, so results are bit-identical to check_entry.
struct CheckShared {
  float th[kLanes][32], tl[kLanes][32];
  double td[kLanes][32];
  double p[kLanes][32];
};

template <int ACC>
struct CheckRound {
  static constexpr int PF = 8;  // prefetched partials per warp lane (more are loaded in finish)
  typename PartialType<ACC>::T pv[PF];
  double pin;
  int e;  // this thread's entry, -1 if beyond the range

  // where entry e's partials live
  __device__ __forceinline__ static void partials_of(const GridDev& g, int e, int pbuf, const void** P, size_t* i0,
                                                     size_t* stride, int* n) {
    const int na = g.nz * g.nx;
    if (e < na) {
      const int z = e / g.nx, x = e - z * g.nx;
      *P = pbuf ? g.PA2 : g.PA;
      *i0 = (size_t)z * g.pa_stride + x;
      *stride = (size_t)g.nz * g.pa_stride;
      *n = g.nty;
    } else {
      const int b = e - na;
      const int z = b / g.ny, y = b - z * g.ny;
      *P = pbuf ? g.PB2 : g.PB;
      *i0 = (size_t)z * g.pb_stride + y;
      *stride = (size_t)g.nz * g.pb_stride;
      *n = g.ntx;
    }
  }

  __device__ __forceinline__ void load(const GridDev& g, int in, int pbuf, int base, int end) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    e = base + lane < end ? base + lane : -1;
    pin = 0.0;
    if (e < 0) return;
    const int na = g.nz * g.nx;
    if (e < na) {
      const int z = e / g.nx, x = e - z * g.nx;
      const int xm = x > 0 ? x - 1 : 0, xp = x < g.nx - 1 ? x + 1 : g.nx - 1;
      const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
      const double* A = g.A[in];
      const size_t pl = (size_t)z * g.ny * g.px;
      switch (w) {
        case 0: pin = __ldcg(A + (size_t)z * g.nx + x); break;
        case 1: pin = __ldcg(A + (size_t)z * g.nx + xm); break;
        case 2: pin = __ldcg(A + (size_t)z * g.nx + xp); break;
        case 3: pin = __ldcg(A + (size_t)zm * g.nx + x); break;
        case 4: pin = __ldcg(A + (size_t)zp * g.nx + x); break;
        case 5: pin = g.cx[(size_t)z * g.nx + x]; break;
        case 6: if (g.k.cn != g.k.cs) pin = (double)__ldcg(g.u[in] + pl + x); break;
        default: if (g.k.cn != g.k.cs) pin = (double)__ldcg(g.u[in] + pl + (size_t)(g.ny - 1) * g.px + x); break;
      }
    } else {
      const int b = e - na;
      const int z = b / g.ny, y = b - z * g.ny;
      const int ym = y > 0 ? y - 1 : 0, yp = y < g.ny - 1 ? y + 1 : g.ny - 1;
      const int zm = z > 0 ? z - 1 : 0, zp = z < g.nz - 1 ? z + 1 : g.nz - 1;
      const double* B = g.B[in];
      const size_t row = ((size_t)z * g.ny + y) * g.px;
      switch (w) {
        case 0: pin = __ldcg(B + (size_t)z * g.ny + y); break;
        case 1: pin = __ldcg(B + (size_t)z * g.ny + ym); break;
        case 2: pin = __ldcg(B + (size_t)z * g.ny + yp); break;
        case 3: pin = __ldcg(B + (size_t)zm * g.ny + y); break;
        case 4: pin = __ldcg(B + (size_t)zp * g.ny + y); break;
        case 5: pin = g.cy[(size_t)z * g.ny + y]; break;
        case 6: if (g.k.cw != g.k.ce) pin = (double)__ldcg(g.u[in] + row); break;
        default: if (g.k.cw != g.k.ce) pin = (double)__ldcg(g.u[in] + row + g.nx - 1); break;
      }
    }
    const void* P;
    size_t i0, stride;
    int n;
    partials_of(g, e, pbuf, &P, &i0, &stride, &n);
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int k = w + kLanes * q;
      if (k < n) pv[q] = load_raw<ACC>(P, i0 + (size_t)k * stride);
    }
  }

  // every thread of the block must call this
  __device__ __forceinline__ void finish(const GridDev& g, int out, int pbuf, unsigned* any, CheckShared& sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    LaneSum t;
    if (e >= 0) {
      const void* P;
      size_t i0, stride;
      int n;
      partials_of(g, e, pbuf, &P, &i0, &stride, &n);
#pragma unroll
      for (int q = 0; q < PF; ++q)
        if (w + kLanes * q < n) t.add(pv[q]);
      for (int k = w + kLanes * PF; k < n; k += kLanes) t.add(load_raw<ACC>(P, i0 + (size_t)k * stride));
    }
    sh.th[w][lane] = t.hi;
    sh.tl[w][lane] = t.lo;
    sh.td[w][lane] = t.d;
    sh.p[w][lane] = pin;
    __syncthreads();
    if (w == 0 && e >= 0) {
      LaneSum acc;
      acc.hi = sh.th[0][lane];
      acc.lo = sh.tl[0][lane];
      acc.d = sh.td[0][lane];
#pragma unroll
      for (int q = 1; q < kLanes; ++q) {
        LaneSum o;
        o.hi = sh.th[q][lane];
        o.lo = sh.tl[q][lane];
        o.d = sh.td[q][lane];
        acc.merge<ACC>(o);
      }
      const double s = acc.total<ACC>();
      const double* v = &sh.p[0][lane];
      const int st = 32;  // stride between the lanes' inputs in sh.p
      const Coef& k = g.k;
      const int na = g.nz * g.nx;
      if (e < na) {
        const int z = e / g.nx, x = e - z * g.nx;
        const double edge = k.cn != k.cs ? edge_term(k.cn, k.cs, (float)v[6 * st], (float)v[7 * st]) : 0.0;
        const double p = interp(v[5 * st], v[0], v[st], v[2 * st], v[3 * st], v[4 * st], weight_sum3(k.cc, k.cn, k.cs),
                                k.cw, k.ce, k.cb, k.ct, edge);
        g.A[out][e] = s;
        g.AP[0][e] = p;
        if (fails(p, s, g.eps)) append_fail(g, z, 0, x, any);
        note_resid(g, p, s);
      } else {
        const int b = e - na;
        const int z = b / g.ny, y = b - z * g.ny;
        const double edge = k.cw != k.ce ? edge_term(k.cw, k.ce, (float)v[6 * st], (float)v[7 * st]) : 0.0;
        const double p = interp(v[5 * st], v[0], v[st], v[2 * st], v[3 * st], v[4 * st], weight_sum3(k.cc, k.cw, k.ce),
                                k.cn, k.cs, k.cb, k.ct, edge);
        g.B[out][b] = s;
        g.BP[0][b] = p;
        if (fails(p, s, g.eps)) append_fail(g, z, 1, y, any);
        note_resid(g, p, s);
      }
    }
    __syncthreads();
  }
};

// Rounds base0, base0 + stride, ... (below n) of the online check by one block; the
// loads of the next round are issued before the current round is finished, so one
// round's memory latency hides behind the other's reduction.
template <int ACC>
__device__ __forceinline__ void check_rounds(const GridDev& g, int in, int out, int base0, int stride, int n,
                                             CheckShared& sh) {
  CheckRound<ACC> ca, cb;
  int b = base0;
  if (b >= n) return;
  ca.load(g, in, 0, b, n);
  for (;;) {
    const int b1 = b + stride;
    if (b1 < n) cb.load(g, in, 0, b1, n);
    ca.finish(g, out, 0, nullptr, sh);
    if (b1 >= n) return;
    const int b2 = b1 + stride;
    if (b2 < n) ca.load(g, in, 0, b2, n);
    cb.finish(g, out, 0, nullptr, sh);
    if (b2 >= n) return;
    b = b2;
  }
}

}  // namespace abft
