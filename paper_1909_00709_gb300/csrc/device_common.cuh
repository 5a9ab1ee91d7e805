// Device helpers: the Eq. (1) point update, reductions, mbarrier and TMA wrappers.
#pragma once

#include "abft_internal.h"

namespace abft {

// Eq. (1) for the 7-point HotSpot3D set: C + cc*c + cw*w + ce*e + cn*n + cs*s + cb*b + ct*t.
// One fixed chain of fused multiply-adds, used by the sweep and by every recomputation,
// so that a recomputed point is bit-identical to the swept one.
__device__ __forceinline__ float hs_update(const Coef& k, float c, float w, float e, float n,
                                           float s, float b, float t, float C) {
  float v = __fmaf_rn(k.cc, c, C);
  v = __fmaf_rn(k.cw, w, v);
  v = __fmaf_rn(k.ce, e, v);
  v = __fmaf_rn(k.cn, n, v);
  v = __fmaf_rn(k.cs, s, v);
  v = __fmaf_rn(k.cb, b, v);
  v = __fmaf_rn(k.ct, t, v);
  return v;
}

// Eq. (1) at one point read straight from global memory.  A neighbour outside the grid
// follows the boundary rule: the centre (clamped, Fig. 2), the point on the opposite
// face (periodic) or zero (empty boundaries, Sec. 3.3).
__device__ __forceinline__ float point_update(const GridDev& g, const float* __restrict__ u,
                                              int z, int y, int x) {
  const size_t plane = (size_t)g.ny * g.px;
  const float* p = u + (size_t)z * plane + (size_t)y * g.px + x;
  const float c = __ldcg(p);
  // outside: clamped -> c, periodic -> the wrapped point at offset `wrap`, empty -> 0
  auto edge = [&](ptrdiff_t wrap) -> float {
    return g.bc == ABFT_BC_CLAMP ? c : (g.bc == ABFT_BC_PERIODIC ? __ldcg(p + wrap) : 0.f);
  };
  const float w = x > 0 ? __ldcg(p - 1) : edge(g.nx - 1);
  const float e = x < g.nx - 1 ? __ldcg(p + 1) : edge(-(ptrdiff_t)(g.nx - 1));
  const float n = y > 0 ? __ldcg(p - g.px) : edge((ptrdiff_t)(g.ny - 1) * g.px);
  const float s = y < g.ny - 1 ? __ldcg(p + g.px) : edge(-(ptrdiff_t)(g.ny - 1) * g.px);
  const float b = z > 0 ? __ldcg(p - (ptrdiff_t)plane) : edge((ptrdiff_t)(g.nz - 1) * (ptrdiff_t)plane);
  const float t = z < g.nz - 1 ? __ldcg(p + plane) : edge(-(ptrdiff_t)(g.nz - 1) * (ptrdiff_t)plane);
  const float C = g.C[(size_t)z * plane + (size_t)y * g.px + x];
  return hs_update(g.k, c, w, e, n, s, b, t, C);
}

// Index of entry i + d (d = -1 or +1) of a length-n vector or axis under the boundary
// rule: clamped to i, wrapped, or -1 for "outside, reads zero".
__device__ __forceinline__ int nb_index(int i, int d, int n, int bc) {
  const int j = i + d;
  if (j >= 0 && j < n) return j;
  return bc == ABFT_BC_CLAMP ? i : (bc == ABFT_BC_PERIODIC ? (j < 0 ? n - 1 : 0) : -1);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// compensated accumulation of v into (hi, lo)
__device__ __forceinline__ void acc2(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  hi = s;
  lo += e;
}

__device__ __forceinline__ void warp_sum2(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h, s, e);
    hi = s;
    lo = lo + l + e;
  }
}

// block-wide FP64 sum (deterministic; every thread gets the result); `red` holds 32 doubles
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

__device__ __forceinline__ void set_status(DevCtrl* c, unsigned bits) { atomicOr(&c->status, bits); }

__device__ __forceinline__ void log_event(DevCtrl* c, abft_event* ev, long long step, int grid, int z,
                                          int y, int x, int kind, float before, float after) {
  const unsigned long long i = atomicAdd(&c->ev_count, 1ull);
  if (i < (unsigned long long)c->ev_cap) {
    abft_event e;
    e.step = step; e.grid = grid; e.z = z; e.y = y; e.x = x; e.kind = kind;
    e.before = before; e.after = after;
    ev[i] = e;
  } else {
    set_status(c, kStEventOverflow);
  }
}

// ---------------------------------------------------------------- mbarrier / TMA

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order this thread's generic-proxy global writes before later async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch on a monotonic arrival counter (zeroed
// before the launch): arrival a waits until the count reaches the next multiple of
// the grid size.  One release fetch-add and acquire polls.  The wait is bounded in
// time; on timeout, or when another CTA has already timed out, the status word
// records it and the barrier returns false, so a broken launch winds down instead
// of hanging.  All threads of every block must call it.
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, DevCtrl* ctrl,
                                             unsigned long long limit_ns = kBarrierTimeoutNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long n = gridDim.x * gridDim.y * gridDim.z;
    unsigned long long a;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;" : "=l"(a) : "l"(count) : "memory");
    const unsigned long long target = (a / n + 1) * n;
    unsigned long long seen;
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; ++spins) {
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(count) : "memory");
      if (seen >= target) break;
      if ((spins & 1023u) == 1023u) {
        const unsigned long long t = globaltimer_ns();
        if (t0 == 0) t0 = t;
        if (t - t0 > limit_ns || (ld_acquire_u32(&ctrl->status) & kStTimeout)) {
          set_status(ctrl, kStTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid barrier whose arrivals carry a payload (the online kernel's count of failing
// entries, a shared-memory word that thread 0 takes and clears after the block has
// synchronised), so that leaving the barrier also tells every CTA the total without a
// second round trip.  Instance k (counted identically by every CTA) uses
// counters[k % 3]: each arrival adds 1 + (payload << 32), and a CTA leaves when the
// low half reaches the grid size; the high half is then the total.  Block 0, on leaving
// instance k, clears the counter of instance k + 2 (last used by instance k - 1, which
// every CTA has left, and not used again before block 0 arrives at instance k + 1).
// Time-bounded like grid_barrier; returns false on timeout.
static __device__ __forceinline__ bool grid_barrier_sum(unsigned long long* counters, unsigned k, unsigned* payload,
                                                     DevCtrl* ctrl, unsigned* total) {
  __shared__ int s_ok;
  __shared__ unsigned s_tot;
  __syncthreads();  // every thread's contribution to *payload is in
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned tot = 0;
    const unsigned n = gridDim.x * gridDim.y * gridDim.z;
    unsigned long long* c = counters + (k % 3u);
    const unsigned long long add = 1ull | ((unsigned long long)(payload ? *payload : 0u) << 32);
    if (payload) *payload = 0u;  // taken; cleared before the block moves on
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(c), "l"(add) : "memory");
    unsigned long long seen;
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; ++spins) {
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(c) : "memory");
      if ((unsigned)(seen & 0xffffffffull) >= n) {
        tot = (unsigned)(seen >> 32);
        break;
      }
      if ((spins & 1023u) == 1023u) {
        const unsigned long long t = globaltimer_ns();
        if (t0 == 0) t0 = t;
        if (t - t0 > kBarrierTimeoutNs || (ld_acquire_u32(&ctrl->status) & kStTimeout)) {
          set_status(ctrl, kStTimeout);
          ok = 0;
          break;
        }
      }
    }
    if (ok && blockIdx.x == 0) counters[(k + 2u) % 3u] = 0ull;
    s_ok = ok;
    s_tot = tot;
  }
  __syncthreads();
  *total = s_tot;
  return s_ok != 0;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Wait for phase `parity` of the barrier to complete; gives up after `limit_ns` of
// global time (or kSpinLimit polls, whichever comes first) and reports it through the
// status word instead of hanging.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, DevCtrl* ctrl,
                                          unsigned long long limit_ns = kWaitTimeoutNs) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255u) == 255u) {
      const unsigned long long t = globaltimer_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) break;
    }
  }
  set_status(ctrl, kStTimeout);
  return false;
}

// 3D tiled TMA load of one box into shared memory, completion on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

}  // namespace abft
