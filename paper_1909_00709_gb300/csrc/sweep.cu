// The stencil sweep of Eq. (1) on sm_103a, with the per-plane checksums of Eq. (2)/(3)
// fused into its epilogue (Sec. 3.2) and the flip-injection hook of Sec. 5.1.
//
// One CTA owns a 128 x TY column of the grid and streams it along z.  Plane tiles
// (with a one-cell y halo and a 4-cell, 16-byte aligned x halo) and the matching
// tiles of the constant term C are staged into a ring of S shared-memory stages by
// TMA, signalled through one mbarrier per stage.  Every thread computes one float4
// of each of its rows; all seven neighbours come from shared memory, the x
// neighbours across float4 boundaries by warp shuffles.  Clamped boundaries (Fig. 2)
// are selects on the grid edges, since TMA fills out-of-range cells with zeros.
//
// The checksum epilogue sums exactly the stored values (after injection):
//   b[z][y] partial: the row's 128 values, warp-shuffle reduction;
//   a[z][x] partial: the tile's TY values per column, registers then one
//                    cross-warp pass through shared memory.
// Partials are written per tile and reduced across tiles in a fixed order by the
// check kernel, so results are bitwise repeatable.
#include <cstdio>

#include "device_common.cuh"

namespace abft {

template <int TY>
struct SweepCfg {
  static constexpr int NW = 8;                        // warps per CTA
  static constexpr int S = TY <= 8 ? 6 : (TY <= 16 ? 5 : 4);  // ring depth (>= 4)
  static constexpr int RPW = TY / NW;                 // rows per warp
  static constexpr int UBOX = (TY + 2) * kUW * 4;     // bytes of a staged u box
  static constexpr int UBOX_AL = (UBOX + 127) / 128 * 128;
  static constexpr int CBOX = TY * kTX * 4;
  static constexpr int STAGE = UBOX_AL + CBOX;        // multiple of 128
  static constexpr int RED = 2 * NW * 32 * 32;        // cross-warp reduction buffer (bytes)
  static constexpr int FLIPS = kLocalFlips * 16 + 16;
  static constexpr int SMEM = 128 + 128 + S * STAGE + RED + FLIPS;  // + slack to align the base
  static_assert(TY % NW == 0, "TY must be a multiple of the warp count");
  static_assert(S >= 4, "the ring must hold z-1, z, z+1 and one load in flight");
};

// ------------------------------------------------------------ accumulators

template <int ACC>
struct AccA;  // per-thread column partial over this thread's rows (4 columns)

template <>
struct AccA<ABFT_ACC_FP32> {
  float v[4];
  __device__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.f; }
  __device__ void add(const float (&m)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] += m[i];
  }
  __device__ void put(unsigned char* red, int slot) const {
    reinterpret_cast<float4*>(red)[slot] = make_float4(v[0], v[1], v[2], v[3]);
  }
  __device__ void take_add(const unsigned char* red, int slot) {
    const float4 q = reinterpret_cast<const float4*>(red)[slot];
    v[0] += q.x; v[1] += q.y; v[2] += q.z; v[3] += q.w;
  }
  __device__ void store(void* PA, size_t idx) const {
    *reinterpret_cast<float4*>(static_cast<float*>(PA) + idx) = make_float4(v[0], v[1], v[2], v[3]);
  }
  // row partial: sum of the 4 values, then across the warp
  __device__ static void row_store(const float (&m)[4], void* PB, size_t idx, bool write) {
    float r = ((m[0] + m[1]) + m[2]) + m[3];
    r = warp_sum(r);
    if (write) static_cast<float*>(PB)[idx] = r;
  }
};

template <>
struct AccA<ABFT_ACC_TWOSUM> {
  float h[4], l[4];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = l[i] = 0.f;
  }
  __device__ void add(const float (&m)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) acc2(h[i], l[i], m[i]);
  }
  __device__ void put(unsigned char* red, int slot) const {
    float4* p = reinterpret_cast<float4*>(red) + 2 * slot;
    p[0] = make_float4(h[0], h[1], h[2], h[3]);
    p[1] = make_float4(l[0], l[1], l[2], l[3]);
  }
  __device__ void take_add(const unsigned char* red, int slot) {
    const float4* p = reinterpret_cast<const float4*>(red) + 2 * slot;
    const float4 qh = p[0], ql = p[1];
    const float hh[4] = {qh.x, qh.y, qh.z, qh.w}, ll[4] = {ql.x, ql.y, ql.z, ql.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc2(h[i], l[i], hh[i]);
      l[i] += ll[i];
    }
  }
  __device__ void store(void* PA, size_t idx) const {
    float4* p = reinterpret_cast<float4*>(static_cast<float2*>(PA) + idx);
    p[0] = make_float4(h[0], l[0], h[1], l[1]);
    p[1] = make_float4(h[2], l[2], h[3], l[3]);
  }
  __device__ static void row_store(const float (&m)[4], void* PB, size_t idx, bool write) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc2(hi, lo, m[i]);
    warp_sum2(hi, lo);
    if (write) static_cast<float2*>(PB)[idx] = make_float2(hi, lo);
  }
};

template <>
struct AccA<ABFT_ACC_FP64> {
  double v[4];
  __device__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.0; }
  __device__ void add(const float (&m)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] += (double)m[i];
  }
  __device__ void put(unsigned char* red, int slot) const {
    double2* p = reinterpret_cast<double2*>(red) + 2 * slot;
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
  }
  __device__ void take_add(const unsigned char* red, int slot) {
    const double2* p = reinterpret_cast<const double2*>(red) + 2 * slot;
    const double2 a = p[0], b = p[1];
    v[0] += a.x; v[1] += a.y; v[2] += b.x; v[3] += b.y;
  }
  __device__ void store(void* PA, size_t idx) const {
    double2* p = reinterpret_cast<double2*>(static_cast<double*>(PA) + idx);
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
  }
  __device__ static void row_store(const float (&m)[4], void* PB, size_t idx, bool write) {
    double r = (((double)m[0] + (double)m[1]) + (double)m[2]) + (double)m[3];
    r = warp_sum(r);
    if (write) static_cast<double*>(PB)[idx] = r;
  }
};

// ------------------------------------------------------------------ kernel

template <int TY, bool PROT, int ACC>
__global__ void __launch_bounds__(SweepCfg<TY>::NW * 32)
    k_sweep(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_c,
            const GridDev g, float* __restrict__ uout, DevCtrl* __restrict__ ctrl, const DevSched sched) {
  using Cfg = SweepCfg<TY>;
  constexpr int S = Cfg::S, NW = Cfg::NW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned in the shared window
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  unsigned char* stages = smem + 128;
  unsigned char* red = stages + S * Cfg::STAGE;
  int4* lflips = reinterpret_cast<int4*>(red + Cfg::RED);
  int* nlf = reinterpret_cast<int*>(lflips + kLocalFlips);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int txi = blockIdx.x % g.ntx, tyi = blockIdx.x / g.ntx;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz;

  auto stage_u = [&](int s) { return reinterpret_cast<float*>(stages + s * Cfg::STAGE); };
  auto stage_c = [&](int s) { return reinterpret_cast<float*>(stages + s * Cfg::STAGE + Cfg::UBOX_AL); };
  auto issue = [&](int p) {  // TMA loads of plane p into stage p % S (thread 0 only)
    const int s = p % S;
    mbar_expect_tx(&bar[s], Cfg::UBOX + Cfg::CBOX);
    tma_load_3d(stage_u(s), &tm_u, x0 - kHaloX, y0 - 1, p, &bar[s]);
    tma_load_3d(stage_c(s), &tm_c, x0, y0, p, &bar[s]);
  };

  if (tid == 0) {
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_c);
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
    *nlf = 0;
  }
  __syncthreads();
  if (tid == 0) {
    const int np = nz < S ? nz : S;
    for (int p = 0; p < np; ++p) issue(p);
  }

  // flips of this sweep that land in this tile (Sec. 5.1: after the update, before the store)
  const long long step = g.gc->step;
  if (ctrl->inject_enabled) {
    const long long i = step - ctrl->sched_t0;
    if (i >= 0 && i < ctrl->sched_n) {
      const int b = sched.off[i], e = sched.off[i + 1];
      for (int k = b + tid; k < e; k += blockDim.x) {
        const DevFlip f = sched.flips[k];
        if (f.grid == g.gid && f.target == 0 && f.x >= x0 && f.x < x0 + kTX && f.x < g.nx &&
            f.y >= y0 && f.y < y0 + TY && f.y < g.ny && f.z >= 0 && f.z < nz && f.x >= 0 && f.y >= 0) {
          const int j = atomicAdd(nlf, 1);
          if (j < kLocalFlips) lflips[j] = make_int4(f.x, f.y, f.z, f.bit & 31);
          else set_status(ctrl, kStFlipOverflow);
        }
      }
    }
  }
  __syncthreads();
  const int nflip = min(*nlf, kLocalFlips);
  const int gx0 = x0 + 4 * lane;
  const int last = g.nx - 1 - gx0;  // element holding x = nx-1, if 0..3

  for (int z = 0; z < nz; ++z) {
    if (z == 0) mbar_wait(&bar[0], 0, ctrl);
    if (z + 1 < nz) mbar_wait(&bar[(z + 1) % S], ((z + 1) / S) & 1, ctrl);
    const float* Uc = stage_u(z % S);
    const float* Ub = z > 0 ? stage_u((z - 1) % S) : Uc;
    const float* Ut = z + 1 < nz ? stage_u((z + 1) % S) : Uc;
    const float* Cs = stage_c(z % S);
    AccA<ACC> acc;
    if (PROT) acc.zero();
#pragma unroll
    for (int rr = 0; rr < Cfg::RPW; ++rr) {
      const int r = warp + rr * NW;
      const int y = y0 + r;
      const int o = (r + 1) * kUW + kHaloX + 4 * lane;
      const float4 c = *reinterpret_cast<const float4*>(Uc + o);
      float4 n = *reinterpret_cast<const float4*>(Uc + o - kUW);
      float4 s = *reinterpret_cast<const float4*>(Uc + o + kUW);
      const float4 b = *reinterpret_cast<const float4*>(Ub + o);
      const float4 t = *reinterpret_cast<const float4*>(Ut + o);
      const float4 cs = *reinterpret_cast<const float4*>(Cs + r * kTX + 4 * lane);
      float wl = __shfl_up_sync(0xffffffffu, c.w, 1);
      float er = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (lane == 0) wl = Uc[o - 1];
      if (lane == 31) er = Uc[o + 4];
      if (y == 0) n = c;
      if (y == g.ny - 1) s = c;
      const float w0 = gx0 == 0 ? c.x : wl;
      float e0 = c.y, e1 = c.z, e2 = c.w, e3 = er;
      if (last == 0) e0 = c.x;
      if (last == 1) e1 = c.y;
      if (last == 2) e2 = c.z;
      if (last == 3) e3 = c.w;
      float v[4];
      v[0] = hs_update(g.k, c.x, w0, e0, n.x, s.x, b.x, t.x, cs.x);
      v[1] = hs_update(g.k, c.y, c.x, e1, n.y, s.y, b.y, t.y, cs.y);
      v[2] = hs_update(g.k, c.z, c.y, e2, n.z, s.z, b.z, t.z, cs.z);
      v[3] = hs_update(g.k, c.w, c.z, e3, n.w, s.w, b.w, t.w, cs.w);
      if (nflip > 0) {
        for (int f = 0; f < nflip; ++f) {
          const int4 q = lflips[f];
          if (q.z == z && q.y == y) {
            const int d = q.x - gx0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (d == i) v[i] = __int_as_float(__float_as_int(v[i]) ^ (1 << q.w));
          }
        }
      }
      const bool yv = y < g.ny;
      float* dst = uout + ((size_t)z * g.ny + y) * g.px + gx0;
      if (yv) {
        if (last >= 3) {
          *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (i <= last) dst[i] = v[i];
        }
      }
      if (PROT) {
        float m[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) m[i] = (yv && i <= last) ? v[i] : 0.f;
        AccA<ACC>::row_store(m, g.PB, ((size_t)txi * nz + z) * g.ny + y, yv && lane == 0);
        acc.add(m);
      }
    }
    if (PROT) acc.put(red + (z & 1) * (Cfg::RED / 2), warp * 32 + lane);
    __syncthreads();
    if (tid == 0 && z >= 1 && z - 1 + S < nz) {
      fence_proxy_async();
      issue(z - 1 + S);
    }
    if (PROT && warp == 0) {
      AccA<ACC> tot;
      tot.zero();
      const unsigned char* rb = red + (z & 1) * (Cfg::RED / 2);
      for (int w = 0; w < NW; ++w) tot.take_add(rb, w * 32 + lane);
      tot.store(g.PA, ((size_t)tyi * nz + z) * g.pa_stride + gx0);
    }
  }

  // the last CTA commits the sweep: the step counter drives injection and event stamps
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == gridDim.x - 1) {
      g.gc->done_sweep = 0;
      g.gc->step = step + 1;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------ host side

int sweep_smem_bytes(int ty, bool) {
  switch (ty) {
    case 8: return SweepCfg<8>::SMEM;
    case 16: return SweepCfg<16>::SMEM;
    default: return SweepCfg<32>::SMEM;
  }
}

template <int TY, bool PROT, int ACC>
static cudaError_t launch_t(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                            const CUtensorMap& tm_c, int out) {
  auto kern = k_sweep<TY, PROT, ACC>;
  static bool attr_set = false;  // per instantiation; all devices share the setting's value
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SweepCfg<TY>::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int blocks = g.ntx * g.nty;
  kern<<<blocks, SweepCfg<TY>::NW * 32, SweepCfg<TY>::SMEM, L.s>>>(tm_in, tm_c, g, g.u[out], L.ctrl,
                                                                    L.sched);
  return cudaGetLastError();
}

template <int TY>
static cudaError_t launch_ty(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                             const CUtensorMap& tm_c, int out, bool prot) {
  if (!prot) return launch_t<TY, false, ABFT_ACC_FP32>(L, g, tm_in, tm_c, out);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: return launch_t<TY, true, ABFT_ACC_TWOSUM>(L, g, tm_in, tm_c, out);
    case ABFT_ACC_FP64: return launch_t<TY, true, ABFT_ACC_FP64>(L, g, tm_in, tm_c, out);
    default: return launch_t<TY, true, ABFT_ACC_FP32>(L, g, tm_in, tm_c, out);
  }
}

cudaError_t launch_sweep(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                         const CUtensorMap& tm_c, int in, int out, bool prot) {
  (void)in;
  switch (g.ty) {
    case 8: return launch_ty<8>(L, g, tm_in, tm_c, out, prot);
    case 16: return launch_ty<16>(L, g, tm_in, tm_c, out, prot);
    case 32: return launch_ty<32>(L, g, tm_in, tm_c, out, prot);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace abft
