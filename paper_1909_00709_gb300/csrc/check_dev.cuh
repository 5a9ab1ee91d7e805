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
// Every path (one thread per entry, or a warp per 32 entries: the per-sweep check
// kernels and the persistent kernel's check warp) evaluates exactly this, so results
// agree bit for bit.
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

// Theorem 1 for the 7-point set (Eq. 4 for a, Eq. 5 for b): shifts along the surviving
// in-plane axis and along z are shifts of the vector under the boundary rule (clamped
// index, wrapped index, or zero outside); the two shifts along the collapsed axis add
// the entry to itself plus the boundary term alpha/beta (edge_of).
// Evaluated with explicit FP64 roundings in a fixed order: c the checksum of C, v0 the
// entry, v1/v2 its neighbours along the surviving in-plane axis, v3/v4 along z, w0 the
// summed weight of the centre and the collapsed-axis pair.
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

// The boundary term along the collapsed axis for its weights wm (shift -1) and wp
// (shift +1), from u at the first and last index of that axis.  The shifted sums are
// the checksum plus (ghost before the first index - last) for wm and (ghost after the
// last index - first) for wp:
//   clamped (ghosts first, last): (wm - wp)(first - last)
//   periodic (ghosts last, first): 0
//   empty (ghosts 0): -(wm last + wp first), both products exact in FP64
__device__ __forceinline__ bool edge_needed(int bc, float wm, float wp) {
  return bc == ABFT_BC_CLAMP ? wm != wp : (bc == ABFT_BC_ZERO && (wm != 0.f || wp != 0.f));
}
__device__ __forceinline__ double edge_of(int bc, float wm, float wp, float first, float last) {
  if (bc == ABFT_BC_CLAMP) return edge_term(wm, wp, first, last);
  if (bc == ABFT_BC_PERIODIC) return 0.0;
  return __dadd_rn(-__dmul_rn((double)wm, (double)last), -__dmul_rn((double)wp, (double)first));
}

// entry (z, i) of a vector with `len` entries per plane; zero outside (index -1)
__device__ __forceinline__ double ld_entry(const double* V, int z, int i, int len) {
  return (z < 0 || i < 0) ? 0.0 : __ldcg(V + (size_t)z * len + i);
}

__device__ __forceinline__ double predict_a(const GridDev& g, const double* A, const float* u, int z, int x) {
  const int nx = g.nx;
  const int xm = nb_index(x, -1, nx, g.bc), xp = nb_index(x, 1, nx, g.bc);
  const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
  const Coef& k = g.k;
  double edge = 0.0;
  if (u != nullptr && edge_needed(g.bc, k.cn, k.cs)) {
    const size_t pl = (size_t)z * g.ny * g.px;
    edge = edge_of(g.bc, k.cn, k.cs, __ldcg(u + pl + x), __ldcg(u + pl + (size_t)(g.ny - 1) * g.px + x));
  }
  return interp(g.cx[(size_t)z * nx + x], __ldcg(A + (size_t)z * nx + x), ld_entry(A, z, xm, nx),
                ld_entry(A, z, xp, nx), ld_entry(A, zm, x, nx), ld_entry(A, zp, x, nx),
                weight_sum3(k.cc, k.cn, k.cs), k.cw, k.ce, k.cb, k.ct, edge);
}

__device__ __forceinline__ double predict_b(const GridDev& g, const double* B, const float* u, int z, int y) {
  const int ny = g.ny;
  const int ym = nb_index(y, -1, ny, g.bc), yp = nb_index(y, 1, ny, g.bc);
  const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
  const Coef& k = g.k;
  double edge = 0.0;
  if (u != nullptr && edge_needed(g.bc, k.cw, k.ce)) {
    const size_t row = ((size_t)z * g.ny + y) * g.px;
    edge = edge_of(g.bc, k.cw, k.ce, __ldcg(u + row), __ldcg(u + row + g.nx - 1));
  }
  return interp(g.cy[(size_t)z * ny + y], __ldcg(B + (size_t)z * ny + y), ld_entry(B, z, ym, ny),
                ld_entry(B, z, yp, ny), ld_entry(B, zm, y, ny), ld_entry(B, zp, y, ny),
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
  if (g.vec == 1 && which == 1 && k == 0) {  // one-vector checks: list the plane once
    const unsigned j = atomicAdd(&g.gc->nbz, 1u);
    if (j < (unsigned)kBzCap) g.gc->bz[j] = z;
  }
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

// The point update a recomputation uses: Eq. (1) with the 7-point set of the sweep
// kernels (point_update).  The general-stencil path passes its own (any set S).
struct SevenPointUpdate {
  __device__ __forceinline__ static float at(const GridDev& g, const float* u, int z, int y, int x) {
    return point_update(g, u, z, y, x);
  }
};

// Recompute rows fb / columns fa of plane z from the intact previous state uin
// (whole plane when `all`), then sum the plane's checksums again.
template <class PU = SevenPointUpdate>
static __device__ void recompute_lines(const GridDev& g, int z, const float* uin, float* u, double* A, double* B,
                                bool all, long long step, DevCtrl* ctrl, abft_event* ev, ResolveSmem& sm) {
  const size_t pl = (size_t)z * g.ny * g.px;
  if (all) {
    for (int i = threadIdx.x; i < g.nx * g.ny; i += blockDim.x) {
      const int y = i / g.nx, x = i - y * g.nx;
      u[pl + (size_t)y * g.px + x] = PU::at(g, uin, z, y, x);
    }
  } else {
    for (int k = 0; k < sm.nb; ++k)
      for (int x = threadIdx.x; x < g.nx; x += blockDim.x)
        u[pl + (size_t)sm.fb[k] * g.px + x] = PU::at(g, uin, z, sm.fb[k], x);
    __syncthreads();
    for (int k = 0; k < sm.na; ++k)
      for (int y = threadIdx.x; y < g.ny; y += blockDim.x)
        u[pl + (size_t)y * g.px + sm.fa[k]] = PU::at(g, uin, z, y, sm.fa[k]);
  }
  __syncthreads();
  // the plane's checksums again in compensated FP32 (TwoSum pairs widened once, as the
  // check sums its partials; GB300's FP64 rate would make a million FP64 additions per
  // plane the slowest step) and a fixed order: a[x] by one thread per column with eight
  // interleaved pairs (rows y = j mod 8, merged in order), b[y] by one warp per row
  // (lane pairs over x = lane mod 32, merged by the butterfly)
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    LaneSum L[8];
    int y = 0;
    for (; y + 8 <= g.ny; y += 8)
#pragma unroll
      for (int j = 0; j < 8; ++j) L[j].add(__ldcg(u + pl + (size_t)(y + j) * g.px + x));
    for (int j = 0; y + j < g.ny; ++j) L[j].add(__ldcg(u + pl + (size_t)(y + j) * g.px + x));
#pragma unroll
    for (int j = 1; j < 8; ++j) L[0].merge<ABFT_ACC_TWOSUM>(L[j]);
    A[(size_t)z * g.nx + x] = L[0].total<ABFT_ACC_TWOSUM>();
  }
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int y = threadIdx.x >> 5; y < g.ny; y += nw) {
    LaneSum t;
    for (int x = lane; x < g.nx; x += 32) t.add(__ldcg(u + pl + (size_t)y * g.px + x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      LaneSum q;
      q.hi = __shfl_xor_sync(0xffffffffu, t.hi, o);
      q.lo = __shfl_xor_sync(0xffffffffu, t.lo, o);
      t.merge<ABFT_ACC_TWOSUM>(q);
    }
    if (lane == 0) B[(size_t)z * g.ny + y] = t.total<ABFT_ACC_TWOSUM>();
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

// Location (Sec. 3.4/3.5) of plane z, whose entries failed, by one block: its lists
// are read (and cleared), a single intersection is corrected by Eq. (8), other
// patterns recompute the failing lines from uin (R5).  uin == nullptr means no
// previous state is available: only single intersections can then be corrected,
// other patterns are counted in *unresolved.  Planes are independent, so blocks may
// resolve different planes at the same time.
// One-vector checks (Sec. 3.2): plane z's b entries failed, its a entries were not
// tested.  a^t of the planes Theorem 1 reads (z and its z neighbours under the boundary
// rule) is summed from the previous state uin into the scratch vector at, a^{t+1}[z]
// from u into A, the interpolation of a^{t+1}[z] goes to ap, and the failing a entries
// are listed -- what the two-vector check would have found.  Column sums in the order
// recompute_lines uses (compensated FP32, eight interleaved row lanes).
static __device__ void column_sums(const GridDev& g, const float* u, int z, double* out) {
  const size_t pl = (size_t)z * g.ny * g.px;
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    LaneSum L[8];
    int y = 0;
    for (; y + 8 <= g.ny; y += 8)
#pragma unroll
      for (int j = 0; j < 8; ++j) L[j].add(__ldcg(u + pl + (size_t)(y + j) * g.px + x));
    for (int j = 0; y + j < g.ny; ++j) L[j].add(__ldcg(u + pl + (size_t)(y + j) * g.px + x));
#pragma unroll
    for (int j = 1; j < 8; ++j) L[0].merge<ABFT_ACC_TWOSUM>(L[j]);
    out[(size_t)z * g.nx + x] = L[0].total<ABFT_ACC_TWOSUM>();
  }
}

// For every plane z whose b entries failed (listed by the check), the column sums
// a^{t+1}[z] of uout (into Aout) and a^t of the planes Theorem 1 reads, z and its z
// neighbours, of uin (into the scratch at).  Work item (plane, k, 32 columns), items
// b0, b0 + stride, ... for this block: eight warps of 32 threads, thread (j, column) sums
// the rows y = j mod 8 (compensated FP32), merged in order -- the arithmetic of
// column_sums, spread over many blocks so that large planes are summed at bandwidth.
// With no failure the block leaves after one load; past the list's capacity every plane
// is visited and its failure count consulted.  Threads beyond the first 256 only join
// the block barriers.
static __device__ void demand_sums(const GridDev& g, const float* uin, const float* uout, double* Aout, double* at,
                                   int b0, int stride) {
  __shared__ __align__(16) unsigned char raw[8 * 32 * sizeof(LaneSum)];
  LaneSum(*L)[32] = reinterpret_cast<LaneSum(*)[32]>(raw);
  const unsigned nb = __ldcg(&g.gc->nbz);
  if (nb == 0) return;
  const bool listed = nb <= (unsigned)kBzCap;
  const int nxb = (g.nx + 31) / 32;
  const long long items = (long long)(listed ? (int)nb : g.nz) * 4 * nxb;
  const int col = threadIdx.x & 31, j = threadIdx.x >> 5;
  for (long long it = b0; it < items; it += stride) {
    const int p = (int)(it / (4 * nxb)), rem = (int)(it % (4 * nxb));
    const int k = rem / nxb, xb = rem % nxb;
    const int z = listed ? __ldcg(&g.gc->bz[p]) : p;
    if (!listed && __ldcg(&g.fcnt[2 * z + 1]) == 0) continue;  // uniform over the block
    const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
    int pz = z;
    if (k == 1) {
      if (zm < 0 || zm == z) continue;
      pz = zm;
    } else if (k == 3) {
      if (zp < 0 || zp == z || zp == zm) continue;
      pz = zp;
    }
    const float* u = k == 0 ? uout : uin;
    double* dst = k == 0 ? Aout : at;
    const int x = xb * 32 + col;
    if (j < 8) {
      LaneSum t;
      if (x < g.nx) {
        const float* q = u + (size_t)pz * g.ny * g.px + x;
        for (int y = j; y < g.ny; y += 8) t.add(__ldcg(q + (size_t)y * g.px));
      }
      L[j][col] = t;
    }
    __syncthreads();
    if (j == 0 && x < g.nx) {
      LaneSum s = L[0][col];
#pragma unroll
      for (int q = 1; q < 8; ++q) s.merge<ABFT_ACC_TWOSUM>(L[q][col]);
      dst[(size_t)pz * g.nx + x] = s.total<ABFT_ACC_TWOSUM>();
    }
    __syncthreads();  // L is reused by the next item
  }
}

static __device__ void demand_a(const GridDev& g, const float* uin, const float* u, double* A, double* ap,
                                double* at, int z, bool summed) {
  if (!summed) {  // otherwise k_demand_sums formed them, in the same order
    const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
    column_sums(g, uin, z, at);
    if (zm >= 0 && zm != z) column_sums(g, uin, zm, at);
    if (zp >= 0 && zp != z && zp != zm) column_sums(g, uin, zp, at);
    column_sums(g, u, z, A);
    __threadfence_block();
    __syncthreads();
  }
  for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
    const double p = predict_a(g, at, uin, z, x);
    const double s = A[(size_t)z * g.nx + x];
    ap[(size_t)z * g.nx + x] = p;
    if (fails(p, s, g.eps)) append_fail(g, z, 0, x);
    note_resid(g, p, s);
  }
  __threadfence_block();
  __syncthreads();
}

template <class PU = SevenPointUpdate>
static __device__ void resolve_plane(ResolveSmem& sm, const GridDev& g, const float* uin, float* u, double* A,
                                     double* B, const double* ap, const double* bp, long long step, DevCtrl* ctrl,
                                     abft_event* ev, unsigned long long* unresolved, int z, bool a_summed = false) {
  if (g.vec == 1 && uin != nullptr) {
    __shared__ int s_nb;
    if (threadIdx.x == 0) s_nb = __ldcg(&g.fcnt[2 * z + 1]);
    __syncthreads();
    const bool b_failed = s_nb != 0;
    __syncthreads();
    if (b_failed) demand_a(g, uin, u, A, const_cast<double*>(ap), g.AP[1], z, a_summed);
  }
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
    recompute_lines<PU>(g, z, uin, u, A, B, overflow, step, ctrl, ev, sm);
  } else if (threadIdx.x == 0) {
    atomicAdd(unresolved, 1ull);
  }
  __syncthreads();
}

// Location for every plane with failing entries, by one block (the fix list `sm.fix`
// collects what was changed, for the persistent kernel's repair).
static __device__ void resolve_planes_into(ResolveSmem& sm, const GridDev& g, const float* uin, float* u, double* A,
                                           double* B, const double* ap, const double* bp, long long step,
                                           DevCtrl* ctrl, abft_event* ev, unsigned long long* unresolved,
                                           bool a_summed = false) {
  if (threadIdx.x == 0) sm.nfix = 0;
  __syncthreads();
  for (int zb = 0; zb < g.nz; zb += 1024) {
    const int zn = min(1024, g.nz - zb);
    for (int j = threadIdx.x; j < zn; j += blockDim.x)
      sm.flag[j] = (__ldcg(&g.fcnt[2 * (zb + j)]) | __ldcg(&g.fcnt[2 * (zb + j) + 1])) != 0;
    __syncthreads();
    for (int j = 0; j < zn; ++j)
      if (sm.flag[j]) resolve_plane(sm, g, uin, u, A, B, ap, bp, step, ctrl, ev, unresolved, zb + j, a_summed);
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

// ------------------------------------------------------------ warp check
// The interpolation weights of Theorem 1 in FP64, converted once per thread (the
// float-to-double conversions are exact, so this equals converting per entry).
struct InterpW {
  double a0, b0, cw, ce, cn, cs, cb, ct;
  __device__ __forceinline__ explicit InterpW(const Coef& k)
      : a0(weight_sum3(k.cc, k.cn, k.cs)), b0(weight_sum3(k.cc, k.cw, k.ce)), cw(k.cw), ce(k.ce), cn(k.cn),
        cs(k.cs), cb(k.cb), ct(k.ct) {}
};

// One entry of the online check (Sec. 3), e < nz*nx addressing a[z][x] and the rest
// b[z][y]: the entry's tile partials summed in the canonical order (lanes j = k mod 8,
// combined in order), the interpolation from a^t / b^t (Theorem 1), the test of Sec.
// 3.4, the entry appended to its plane's list if it fails.  The partial loads are
// issued eight at a time; across a warp (32 consecutive entries) every load is
// coalesced.  Arithmetic identical to check_entry and to the boxed rounds below (the
// persistent kernel's check warp).
template <int ACC>
__device__ __forceinline__ void check_lane(const GridDev& g, const InterpW& w, int in, int out, int e) {
  const int na = g.nz * g.nx;
  const Coef& k = g.k;
  double c, v0, v1, v2, v3, v4, edge = 0.0;
  const void* P;
  size_t i0, stride;
  int np, z, idx, which;
  if (e < na) {
    z = e / g.nx;
    idx = e - z * g.nx;
    which = 0;
    const int x = idx, nx = g.nx;
    const int xm = nb_index(x, -1, nx, g.bc), xp = nb_index(x, 1, nx, g.bc);
    const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
    const double* A = g.A[in];
    c = g.cx[(size_t)z * nx + x];
    v0 = __ldcg(A + (size_t)z * nx + x);
    v1 = ld_entry(A, z, xm, nx);
    v2 = ld_entry(A, z, xp, nx);
    v3 = ld_entry(A, zm, x, nx);
    v4 = ld_entry(A, zp, x, nx);
    if (edge_needed(g.bc, k.cn, k.cs)) {
      const size_t pl = (size_t)z * g.ny * g.px;
      edge = edge_of(g.bc, k.cn, k.cs, __ldcg(g.u[in] + pl + x),
                     __ldcg(g.u[in] + pl + (size_t)(g.ny - 1) * g.px + x));
    }
    P = g.PA;
    i0 = (size_t)z * g.pa_stride + x;
    stride = (size_t)g.nz * g.pa_stride;
    np = g.nty;
  } else {
    const int b = e - na;
    z = b / g.ny;
    idx = b - z * g.ny;
    which = 1;
    const int y = idx, ny = g.ny;
    const int ym = nb_index(y, -1, ny, g.bc), yp = nb_index(y, 1, ny, g.bc);
    const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
    const double* B = g.B[in];
    c = g.cy[(size_t)z * ny + y];
    v0 = __ldcg(B + (size_t)z * ny + y);
    v1 = ld_entry(B, z, ym, ny);
    v2 = ld_entry(B, z, yp, ny);
    v3 = ld_entry(B, zm, y, ny);
    v4 = ld_entry(B, zp, y, ny);
    if (edge_needed(g.bc, k.cw, k.ce)) {
      const size_t row = ((size_t)z * g.ny + y) * g.px;
      edge = edge_of(g.bc, k.cw, k.ce, __ldcg(g.u[in] + row), __ldcg(g.u[in] + row + g.nx - 1));
    }
    P = g.PB;
    i0 = (size_t)z * g.pb_stride + y;
    stride = (size_t)g.nz * g.pb_stride;
    np = g.ntx;
  }
  using T = typename PartialType<ACC>::T;
  LaneSum L[kLanes];
  int q = 0;
  // partials fetched kDeep lane steps at a time, so that many loads are in flight (an a
  // entry sums one partial per tile row); each lane sum still takes its partials in
  // ascending order
  constexpr int kDeep = sizeof(T) == 4 ? 4 : 2;
  for (; q + kDeep * kLanes <= np; q += kDeep * kLanes) {
    T v[kDeep * kLanes];
#pragma unroll
    for (int j = 0; j < kDeep * kLanes; ++j) v[j] = load_raw<ACC>(P, i0 + (size_t)(q + j) * stride);
#pragma unroll
    for (int j = 0; j < kDeep * kLanes; ++j) L[j % kLanes].add(v[j]);
  }
  for (; q + kLanes <= np; q += kLanes) {
    T v[kLanes];
#pragma unroll
    for (int j = 0; j < kLanes; ++j) v[j] = load_raw<ACC>(P, i0 + (size_t)(q + j) * stride);
#pragma unroll
    for (int j = 0; j < kLanes; ++j) L[j].add(v[j]);
  }
#pragma unroll
  for (int j = 0; j < kLanes; ++j)
    if (q + j < np) L[j].add(load_raw<ACC>(P, i0 + (size_t)(q + j) * stride));
  LaneSum t = L[0];
#pragma unroll
  for (int j = 1; j < kLanes; ++j) t.merge<ACC>(L[j]);
  const double s = t.total<ACC>();
  double p;
  if (which == 0) {
    p = interp(c, v0, v1, v2, v3, v4, w.a0, w.cw, w.ce, w.cb, w.ct, edge);
    g.A[out][e] = s;
    g.AP[0][e] = p;
  } else {
    p = interp(c, v0, v1, v2, v3, v4, w.b0, w.cn, w.cs, w.cb, w.ct, edge);
    g.B[out][e - na] = s;
    g.BP[0][e - na] = p;
  }
  if (fails(p, s, g.eps)) append_fail(g, z, which, idx);
  note_resid(g, p, s);
}

// Entries of warps wbase, wbase + wstride, ... (32 consecutive entries each, below n)
// checked by the calling warp; no block-wide synchronisation.
template <int ACC>
__device__ __forceinline__ void check_warps(const GridDev& g, int in, int out, int wbase, int wstride, int first,
                                            int n) {
  const InterpW w(g.k);
  const int lane = threadIdx.x & 31;
  for (int base = first + wbase * 32; base < n; base += wstride * 32)
    if (base + lane < n) check_lane<ACC>(g, w, in, out, base + lane);
}

// ------------------------------------------------------------ box check rounds
// A round is 32 consecutive entries of one plane (a[z][32 xb ...] or b[z][32 yb ...]);
// one TMA box brings all tiles' partials of the round into shared memory (its own
// mbarrier) while each lane loads its entry's interpolation inputs.  The lane then
// sums its entry's partials in the canonical order and tests as check_lane does, so
// the results are bit-identical to the other paths.  One warp, no block barrier:
// used by the persistent kernel's check warp and by the box check kernels.
// tm_p: the maps of PA, PA2, PB, PB2 (boxes of 32 entries by all tiles of a plane;
// only for grids with at most 256 tiles along x and along y).
__host__ __device__ inline int check_box_bytes(int nty, int ntx, int acc) {
  const int per = acc == ABFT_ACC_TWOSUM ? 2 : 1, esz = acc == ABFT_ACC_FP64 ? 8 : 4;
  return kCheckBox * per * esz * (nty > ntx ? nty : ntx);
}

// rounds of one check: the a rounds (nz * ceil(nx/32)) then the b rounds; with one
// checksum vector (Sec. 3.2) only the b rounds
__device__ __forceinline__ int check_rounds_of(const GridDev& g) {
  return g.nz * ((g.vec == 1 ? 0 : (g.nx + kCheckBox - 1) / kCheckBox) + (g.ny + kCheckBox - 1) / kCheckBox);
}

// One round of the boxed online check: 32 consecutive entries of a[z][.] or b[z][.]
// whose tile partials arrive as one TMA box ([n partials][32 entries]).  The steps are
// separate steps (placement of the copy, the input loads, the lane sums and the
// finish), run in this order by one warp in check_box_round.
struct CheckRound {
  bool is_a;
  int z, c, len, n;  // plane, first entry, entries per plane, partials per entry
};

__device__ __forceinline__ CheckRound check_round_at(const GridDev& g, int round) {
  CheckRound r;
  const int nxb = (g.nx + kCheckBox - 1) / kCheckBox;
  const int ra = g.nz * nxb;
  if (g.vec == 1) round += ra;  // b rounds only
  r.is_a = round < ra;
  if (r.is_a) {
    r.z = round / nxb;
    r.c = (round - r.z * nxb) * kCheckBox;
    r.len = g.nx;
    r.n = g.nty;
  } else {
    const int nyb = (g.ny + kCheckBox - 1) / kCheckBox;
    const int q = round - ra;
    r.z = q / nyb;
    r.c = (q - r.z * nyb) * kCheckBox;
    r.len = g.ny;
    r.n = g.ntx;
  }
  return r;
}

// one thread: start the TMA copy of the round's partial box (buffer pbuf) into buf
template <int ACC>
__device__ __forceinline__ void check_round_issue(const CheckRound& r, const CUtensorMap* tm_p, int pbuf,
                                                  unsigned char* buf, uint64_t* cbar) {
  constexpr int per = ACC == ABFT_ACC_TWOSUM ? 2 : 1;
  fence_proxy_async();  // earlier reads of buf come before this TMA write
  mbar_expect_tx(cbar, kCheckBox * per * (ACC == ABFT_ACC_FP64 ? 8 : 4) * r.n);
  tma_load_3d(buf, r.is_a ? &tm_p[pbuf] : &tm_p[2 + pbuf], r.c * per, r.z, 0, cbar);
}

// Theorem 1's inputs of the lane's entry (entry c + lane; zeros past the plane's end)
struct CheckIn {
  double v0, v1, v2, v3, v4, cc;
  float ef, el;
};

__device__ __forceinline__ CheckIn check_round_inputs(const GridDev& g, const CheckRound& r, int in, int lane) {
  CheckIn q{0, 0, 0, 0, 0, 0, 0.f, 0.f};
  const int idx = r.c + lane, len = r.len, z = r.z;
  if (idx >= len) return q;
  const int im = nb_index(idx, -1, len, g.bc), ip = nb_index(idx, 1, len, g.bc);
  const int zm = nb_index(z, -1, g.nz, g.bc), zp = nb_index(z, 1, g.nz, g.bc);
  const double* V = r.is_a ? g.A[in] : g.B[in];
  q.v0 = __ldcg(V + (size_t)z * len + idx);
  q.v1 = ld_entry(V, z, im, len);
  q.v2 = ld_entry(V, z, ip, len);
  q.v3 = ld_entry(V, zm, idx, len);
  q.v4 = ld_entry(V, zp, idx, len);
  q.cc = (r.is_a ? g.cx : g.cy)[(size_t)z * len + idx];
  const Coef& k = g.k;
  if (r.is_a ? edge_needed(g.bc, k.cn, k.cs) : edge_needed(g.bc, k.cw, k.ce)) {
    const float* u = g.u[in];
    if (r.is_a) {
      const size_t pl = (size_t)z * g.ny * g.px;
      q.ef = __ldcg(u + pl + idx);
      q.el = __ldcg(u + pl + (size_t)(g.ny - 1) * g.px + idx);
    } else {
      const size_t row = ((size_t)z * g.ny + idx) * g.px;
      q.ef = __ldcg(u + row);
      q.el = __ldcg(u + row + g.nx - 1);
    }
  }
  return q;
}

// the eight lane sums of the lane's entry from the box: lane sum j takes partials
// k = j, j + 8, ... in ascending order; the eight are advanced together (eight
// independent shared-memory loads per step), which keeps one warp's round short
template <int ACC>
__device__ __forceinline__ void check_round_lanes(const CheckRound& r, const unsigned char* buf, int lane,
                                                  LaneSum (&t)[kLanes]) {
  using T = typename PartialType<ACC>::T;
  const T* part = reinterpret_cast<const T*>(buf);
  if (r.c + lane >= r.len) return;
  const int n = r.n;
  int q = 0;
  for (; q + kLanes <= n; q += kLanes) {
#pragma unroll
    for (int j = 0; j < kLanes; ++j) t[j].add(part[(q + j) * kCheckBox + lane]);
  }
#pragma unroll
  for (int j = 0; j < kLanes; ++j)
    if (q + j < n) t[j].add(part[(q + j) * kCheckBox + lane]);
}

// the lane sums merged in order 0..7, Theorem 1, the Sec. 3.4 test; results stored
// (checksum into A/B[out], prediction into AP/BP[0]) and a failing entry listed
template <int ACC>
__device__ __forceinline__ void check_round_finish(const GridDev& g, const InterpW& w, const CheckRound& r,
                                                   const CheckIn& q, LaneSum (&t)[kLanes], int out, int lane,
                                                   unsigned* any) {
  const int idx = r.c + lane;
  if (idx >= r.len) return;
#pragma unroll
  for (int j = 1; j < kLanes; ++j) t[0].merge<ACC>(t[j]);
  const double s = t[0].total<ACC>();
  const Coef& k = g.k;
  double p;
  const size_t e = (size_t)r.z * r.len + idx;
  if (r.is_a) {
    const double edge = edge_needed(g.bc, k.cn, k.cs) ? edge_of(g.bc, k.cn, k.cs, q.ef, q.el) : 0.0;
    p = interp(q.cc, q.v0, q.v1, q.v2, q.v3, q.v4, w.a0, w.cw, w.ce, w.cb, w.ct, edge);
    g.A[out][e] = s;
    g.AP[0][e] = p;
  } else {
    const double edge = edge_needed(g.bc, k.cw, k.ce) ? edge_of(g.bc, k.cw, k.ce, q.ef, q.el) : 0.0;
    p = interp(q.cc, q.v0, q.v1, q.v2, q.v3, q.v4, w.b0, w.cn, w.cs, w.cb, w.ct, edge);
    g.B[out][e] = s;
    g.BP[0][e] = p;
  }
  if (fails(p, s, g.eps)) append_fail(g, r.z, r.is_a ? 0 : 1, idx, any);
  note_resid(g, p, s);
}

// one warp runs a whole round: box copy and interpolation inputs in flight together,
// then the eight lane sums, then the finish
template <int ACC>
__device__ __forceinline__ void check_box_round(const GridDev& g, const InterpW& w, const CUtensorMap* tm_p, int in,
                                                int out, int pbuf, int round, unsigned char* buf, uint64_t* cbar,
                                                unsigned& phase, DevCtrl* ctrl, unsigned* any) {
  const int lane = threadIdx.x & 31;
  const CheckRound r = check_round_at(g, round);
  if (lane == 0) check_round_issue<ACC>(r, tm_p, pbuf, buf, cbar);
  const CheckIn q = check_round_inputs(g, r, in, lane);
  mbar_wait(cbar, phase, ctrl);
  phase ^= 1u;
  LaneSum t[kLanes];
  check_round_lanes<ACC>(r, buf, lane, t);
  __syncwarp();  // every lane has read buf before lane 0 may start the next copy into it
  check_round_finish<ACC>(g, w, r, q, t, out, lane, any);
}

}  // namespace abft
