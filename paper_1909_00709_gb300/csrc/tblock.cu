// Temporal blocking: K sweeps of Eq. (1) in one pass over the grid.
//
// A plain sweep moves 12 bytes per point-update (read u and C, write u'), so it is
// bound by HBM at about 557 GLUP/s.  Here a CTA owns a 128 x TY column of the output
// and streams z as the single-sweep kernel does, but it stages the input planes with
// a K-row halo in y (and the 4-column halo in x, enough for K <= 4) and advances
// them K sweeps in shared memory: at iteration i it computes level 1 of plane i-1,
// level 2 of plane i-2, ..., level K of plane i-K, each level from the three planes
// of the level below.  Level tau is computed on the output region widened by K-tau
// cells in x and y (the cells a later level still reads), so neighbouring CTAs
// recompute a thin halo instead of exchanging it; only level K is written to global
// memory.  Per K point-updates the grid is read and written once: 12/K bytes each.
//
// Every level uses the point update of the single-sweep kernel (hs_update, the same
// clamps at the grid's faces) and applies the flips scheduled for its sweep to every
// point it computes, halo included, so the result is bit-identical to K single
// sweeps.
//
// Protected passes (online checks with temporal blocking, PVEC = 1 or 2) also write the
// partial checksums of every level over the CTA's own 128 x TY region: the b partial of
// each row (the lane sums of four values and the warp butterfly of the single-sweep
// epilogue, so the b checksums equal a single sweep's bit for bit) and, with PVEC = 2,
// the a partial of each column (its TY values in row order).  A check of all K levels
// then runs after the pass (k_check_tb_level); a level that fails sends the pass back to
// single sweeps from its input (the pass never overwrites it).
#include <algorithm>

#include "check_dev.cuh"
#include "sweep_tile.cuh"

namespace abft {

constexpr int kTbFlips = 64;  // flips of the K sweeps that land in one CTA's region

template <int TY, int K>
struct TbCfg {
  static constexpr int NW = 8;
  static constexpr int R = TY + 2 * K;             // staged rows
  static constexpr int PBYTES = R * kUW * 4;       // one staged plane (136 columns)
  static constexpr int PB_AL = (PBYTES + 127) / 128 * 128;
  static constexpr int S = K <= 2 ? K + 3 : K + 2;  // input stages, u and C of one plane each
  static constexpr int STAGE = 2 * PB_AL;
  static constexpr int LVL = (K - 1) * 3 * PB_AL;  // levels 1..K-1, three planes each
  static constexpr int FLIPS = kTbFlips * 16 + 16;
  static constexpr int SMEM = 128 + 128 + S * STAGE + LVL + FLIPS;
  static constexpr int MIN_BLOCKS = K <= 2 ? 2 : 1;
  static_assert(K >= 2 && K <= kHaloX, "the x halo of the staged box covers K <= 4");
  static_assert(S <= 16, "mbarriers fit the 128-byte head");
  static_assert(TY % NW == 0, "rows per warp");
};

// Eq. (1) on the float4 of columns x .. x+3 (global x of element 0) of row y, from the
// staged planes (centre c, rows above/below, planes below/above) with the grid's
// clamped faces; the same expressions as the single-sweep tile.
__device__ __forceinline__ void tb_update4(const Coef& k, float4 c, float4 n, float4 s, float4 b, float4 t, float wl,
                                           float er, float4 cs, int gx, int nx, float (&v)[4]) {
  const int last = nx - 1 - gx;
  const float w0 = gx == 0 ? c.x : wl;
  float e0 = c.y, e1 = c.z, e2 = c.w, e3 = er;
  if (last == 0) e0 = c.x;
  if (last == 1) e1 = c.y;
  if (last == 2) e2 = c.z;
  if (last == 3) e3 = c.w;
  // gx is a multiple of 4: only element 0 can sit on the x = 0 face
  v[0] = hs_update(k, c.x, w0, e0, n.x, s.x, b.x, t.x, cs.x);
  v[1] = hs_update(k, c.y, c.x, e1, n.y, s.y, b.y, t.y, cs.y);
  v[2] = hs_update(k, c.z, c.y, e2, n.z, s.z, b.z, t.z, cs.z);
  v[3] = hs_update(k, c.w, c.z, e3, n.w, s.w, b.w, t.w, cs.w);
}

template <int TY, int K, int PVEC>
__global__ void __launch_bounds__(256, TbCfg<TY, K>::MIN_BLOCKS)
    k_sweep_tb(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_c, const GridDev g,
               float* __restrict__ uout, DevCtrl* __restrict__ ctrl, DevSched sched, TbLevels lp) {
  using Cfg = TbCfg<TY, K>;
  static_assert(TY == Cfg::NW, "protected passes reduce one owned row per warp");
  __shared__ float colk[PVEC == 2 ? Cfg::NW * kTX : 1];  // level K values of the owned rows (a partials)
  constexpr int S = Cfg::S, R = Cfg::R, NW = Cfg::NW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sb = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb);
  unsigned char* stages = sb + 128;
  unsigned char* lvl = stages + S * Cfg::STAGE;
  int4* lflips = reinterpret_cast<int4*>(lvl + Cfg::LVL);
  int* nlf = reinterpret_cast<int*>(lflips + kTbFlips);
  auto su = [&](int p) { return reinterpret_cast<float*>(stages + (p % S) * Cfg::STAGE); };
  auto sc = [&](int p) { return reinterpret_cast<float*>(stages + (p % S) * Cfg::STAGE + Cfg::PB_AL); };
  auto lv = [&](int tau, int p) { return reinterpret_cast<float*>(lvl + ((tau - 1) * 3 + p % 3) * Cfg::PB_AL); };

  sched.load(ctrl);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long step = g.gc->step;  // the first of the K sweeps
  const int nty = (g.ny + TY - 1) / TY;
  const int txi = blockIdx.x % g.ntx, tyi = blockIdx.x / g.ntx;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz, ny = g.ny, nx = g.nx;
  auto issue = [&](int p) {  // u and C of plane p, rows y0-K .. y0+TY+K-1 (thread 0)
    mbar_expect_tx(&bar[p % S], 2 * Cfg::PBYTES);
    tma_load_3d(su(p), &tm_u, x0 - kHaloX, y0 - K, p, &bar[p % S]);
    tma_load_3d(sc(p), &tm_c, x0 - kHaloX, y0 - K, p, &bar[p % S]);
  };
  if (tid == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&bar[k], 1);
    fence_barrier_init();
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_c);
    fence_proxy_async_global();
    for (int p = 0; p < S && p < nz; ++p) issue(p);
    *nlf = 0;
  }
  __syncthreads();
  // flips of the K sweeps inside the widened region (Sec. 5.1), with their level
  if (sched.enabled) {
    for (int tau = 1; tau <= K; ++tau) {
      const long long i = step + tau - 1 - sched.t0;
      if (i < 0 || i >= sched.n) continue;
      for (int k = sched.off[i] + tid; k < sched.off[i + 1]; k += blockDim.x) {
        const DevFlip f = sched.flips[k];
        if (f.grid == g.gid && f.target == 0 && f.x >= x0 - K && f.x < x0 + kTX + K && f.x >= 0 && f.x < nx &&
            f.y >= y0 - K && f.y < y0 + TY + K && f.y >= 0 && f.y < ny && f.z >= 0 && f.z < nz) {
          const int j = atomicAdd(nlf, 1);
          if (j < kTbFlips) lflips[j] = make_int4(f.x, f.y, f.z, (tau << 5) | (f.bit & 31));
          else set_status(ctrl, kStFlipOverflow);
        }
      }
    }
  }
  __syncthreads();
  const int nflip = min(*nlf, kTbFlips);
  auto flip4 = [&](float (&v)[4], int tau, int z, int y, int gx) {
    for (int f = 0; f < nflip; ++f) {
      const int4 q = lflips[f];
      if ((q.w >> 5) == tau && q.z == z && q.y == y) {
        const int d = q.x - gx;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (d == e) v[e] = __int_as_float(__float_as_int(v[e]) ^ (1 << (q.w & 31)));
      }
    }
  };

  for (int i = 0; i < nz + K; ++i) {
    if (i < nz) mbar_wait(&bar[i % S], (unsigned)(i / S) & 1u, ctrl);
#pragma unroll
    for (int tau = 1; tau <= K; ++tau) {
      const int p = i - tau;
      if (p >= 0 && p < nz) {
        const int pb = p > 0 ? p - 1 : p, pt = p + 1 < nz ? p + 1 : p;
        const float* Pc = tau == 1 ? su(p) : lv(tau - 1, p);
        const float* Pb = tau == 1 ? su(pb) : lv(tau - 1, pb);
        const float* Pt = tau == 1 ? su(pt) : lv(tau - 1, pt);
        const float* Cp = sc(p);
        if (tau < K) {
          // level tau on rows tau .. R-tau-1 and all 34 column groups of the box
          float* dst = lv(tau, p);
          const int nitems = (R - 2 * tau) * (kUW / 4);
          for (int it = tid; it < nitems; it += blockDim.x) {
            const int r = tau + it / (kUW / 4), q = it % (kUW / 4);
            const int o = r * kUW + 4 * q;
            const int gy = y0 - K + r, gx = x0 - kHaloX + 4 * q;
            const float4 c = *reinterpret_cast<const float4*>(Pc + o);
            float4 n = *reinterpret_cast<const float4*>(Pc + o - kUW);
            float4 s = *reinterpret_cast<const float4*>(Pc + o + kUW);
            const float4 b = *reinterpret_cast<const float4*>(Pb + o);
            const float4 t = *reinterpret_cast<const float4*>(Pt + o);
            const float4 cs = *reinterpret_cast<const float4*>(Cp + o);
            const float wl = q > 0 ? Pc[o - 1] : c.x;
            const float er = q < kUW / 4 - 1 ? Pc[o + 4] : c.w;
            if (gy == 0) n = c;
            if (gy == ny - 1) s = c;
            float v[4];
            tb_update4(g.k, c, n, s, b, t, wl, er, cs, gx, nx, v);
            if (nflip > 0) flip4(v, tau, p, gy, gx);
            *reinterpret_cast<float4*>(dst + o) = make_float4(v[0], v[1], v[2], v[3]);
          }
        } else {
          // level K: the 128 x TY output, one row per warp at a time, stored to u_out
#pragma unroll
          for (int rr = 0; rr < TY / NW; ++rr) {
            const int r = K + warp + rr * NW;
            const int gy = y0 - K + r, gx = x0 + 4 * lane;
            const int o = r * kUW + kHaloX + 4 * lane;
            const float4 c = *reinterpret_cast<const float4*>(Pc + o);
            float4 n = *reinterpret_cast<const float4*>(Pc + o - kUW);
            float4 s = *reinterpret_cast<const float4*>(Pc + o + kUW);
            const float4 b = *reinterpret_cast<const float4*>(Pb + o);
            const float4 t = *reinterpret_cast<const float4*>(Pt + o);
            const float4 cs = *reinterpret_cast<const float4*>(Cp + o);
            float wl = __shfl_up_sync(0xffffffffu, c.w, 1);
            float er = __shfl_down_sync(0xffffffffu, c.x, 1);
            if (lane == 0) wl = Pc[o - 1];
            if (lane == 31) er = Pc[o + 4];
            if (gy == 0) n = c;
            if (gy == ny - 1) s = c;
            float v[4];
            tb_update4(g.k, c, n, s, b, t, wl, er, cs, gx, nx, v);
            if (nflip > 0) flip4(v, K, p, gy, gx);
            if (PVEC) {  // level K's partials: the row's b partial now, the columns after the barrier
              float m[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) m[e] = (gy < ny && gx + e < nx) ? v[e] : 0.f;
              const float rsum = warp_sum(((m[0] + m[1]) + m[2]) + m[3]);
              if (lane == 0 && gy < ny) static_cast<float*>(lp.PB[K - 1])[((size_t)txi * nz + p) * g.pb_stride + gy] = rsum;
              if (PVEC == 2)
#pragma unroll
                for (int e = 0; e < 4; ++e) colk[warp * kTX + 4 * lane + e] = m[e];
            }
            if (gy < ny && gx < nx) {
              float* out = uout + ((size_t)p * ny + gy) * g.px + gx;
              const int last = nx - 1 - gx;
              if (last >= 3) {
                *reinterpret_cast<float4*>(out) = make_float4(v[0], v[1], v[2], v[3]);
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (e <= last) out[e] = v[e];
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if (PVEC) {  // partials of the owned region at every level computed in this iteration
#pragma unroll
      for (int tau = 1; tau < K; ++tau) {
        const int p = i - tau;
        if (p < 0 || p >= nz) continue;
        const float* L = lv(tau, p);
        const int gy = y0 + warp, gx = x0 + 4 * lane;  // owned row `warp`, columns of this lane
        const float4 c = *reinterpret_cast<const float4*>(L + (K + warp) * kUW + kHaloX + 4 * lane);
        const float m[4] = {(gy < ny && gx < nx) ? c.x : 0.f, (gy < ny && gx + 1 < nx) ? c.y : 0.f,
                            (gy < ny && gx + 2 < nx) ? c.z : 0.f, (gy < ny && gx + 3 < nx) ? c.w : 0.f};
        const float rsum = warp_sum(((m[0] + m[1]) + m[2]) + m[3]);
        if (lane == 0 && gy < ny) static_cast<float*>(lp.PB[tau - 1])[((size_t)txi * nz + p) * g.pb_stride + gy] = rsum;
        if (PVEC == 2 && tid < kTX && x0 + tid < nx) {
          float a = 0.f;
          for (int rr = 0; rr < TY && y0 + rr < ny; ++rr) a += L[(K + rr) * kUW + kHaloX + tid];
          static_cast<float*>(lp.PA[tau - 1])[((size_t)tyi * nz + p) * g.pa_stride + x0 + tid] = a;
        }
      }
      const int pk = i - K;
      if (PVEC == 2 && pk >= 0 && pk < nz && tid < kTX && x0 + tid < nx) {
        float a = 0.f;
        for (int rr = 0; rr < TY && y0 + rr < ny; ++rr) a += colk[rr * kTX + tid];
        static_cast<float*>(lp.PA[K - 1])[((size_t)tyi * nz + pk) * g.pa_stride + x0 + tid] = a;
      }
    }
    // plane i-K's stage (its C was read by level K just now) takes plane i-K+S
    if (tid == 0 && i - K >= 0 && i - K + S < nz) {
      fence_proxy_async();
      issue(i - K + S);
    }
  }
  fence_proxy_async_global();  // this thread's stores, before any later TMA read of them
  if (tid == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == (unsigned)(g.ntx * nty) - 1) {  // the last CTA commits the K sweeps
      g.gc->done_sweep = 0;
      g.gc->step = step + K;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------------ host side

constexpr int kTbTY = kTbRows;

template <int K, int PVEC>
static cudaError_t tb_launch(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                             float* uout, const TbLevels& lp) {
  auto kern = k_sweep_tb<kTbTY, K, PVEC>;
  const int smem = TbCfg<kTbTY, K>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int blocks = g.ntx * ((g.ny + kTbTY - 1) / kTbTY);
  kern<<<blocks, 256, smem, L.s>>>(tm_in, tm_c, g, uout, L.ctrl, L.sched, lp);
  return cudaGetLastError();
}

cudaError_t launch_sweep_tb(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                            int out, int k) {
  const TbLevels none{};
  switch (k) {
    case 2: return tb_launch<2, 0>(L, g, tm_in, tm_c, g.u[out], none);
    case 3: return tb_launch<3, 0>(L, g, tm_in, tm_c, g.u[out], none);
    case 4: return tb_launch<4, 0>(L, g, tm_in, tm_c, g.u[out], none);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep_tb_prot(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                                 int out, int k, const TbLevels& lp) {
  const bool two = g.vec == 2;
  switch (k) {
    case 2: return two ? tb_launch<2, 2>(L, g, tm_in, tm_c, g.u[out], lp) : tb_launch<2, 1>(L, g, tm_in, tm_c, g.u[out], lp);
    case 3: return two ? tb_launch<3, 2>(L, g, tm_in, tm_c, g.u[out], lp) : tb_launch<3, 1>(L, g, tm_in, tm_c, g.u[out], lp);
    case 4: return two ? tb_launch<4, 2>(L, g, tm_in, tm_c, g.u[out], lp) : tb_launch<4, 1>(L, g, tm_in, tm_c, g.u[out], lp);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------ level checks

// The check of level tau of a protected pass (Sec. 3, one level after the other): the
// level's partials (gt.PA/gt.PB, tiles of kTbRows rows) reduced in the canonical
// order into (a_out, b_out), Theorem 1 from the level before (a_prev, b_prev; the
// boundary terms vanish for the grids temporal blocking serves), the Sec. 3.4 test;
// failing entries are only counted (gt.gc->verdict): a failing pass is recomputed.
__global__ void __launch_bounds__(256)
    k_check_tb_level(const GridDev gt, const double* a_prev, const double* b_prev, double* a_out, double* b_out) {
  const int na = gt.vec == 2 ? gt.nz * gt.nx : 0, n = na + gt.nz * gt.ny;
  unsigned long long nf = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / gt.nx, x = i - z * gt.nx;
      const double s = reduce_a<ABFT_ACC_FP32>(gt, z, x);
      a_out[i] = s;
      const double p = predict_a(gt, a_prev, nullptr, z, x);
      if (fails(p, s, gt.eps)) ++nf;
      note_resid(gt, p, s);
    } else {
      const int j = i - na;
      const int z = j / gt.ny, y = j - z * gt.ny;
      const double s = reduce_b<ABFT_ACC_FP32>(gt, z, y);
      b_out[j] = s;
      const double p = predict_b(gt, b_prev, nullptr, z, y);
      if (fails(p, s, gt.eps)) ++nf;
      note_resid(gt, p, s);
    }
  }
  if (nf) atomicAdd(&gt.gc->verdict, nf);
}

cudaError_t launch_check_tb_level(const Launch& L, const GridDev& gt, const double* a_prev, const double* b_prev,
                                  double* a_out, double* b_out) {
  const long long n = (long long)gt.nz * ((gt.vec == 2 ? gt.nx : 0) + gt.ny);
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8 * 152));
  k_check_tb_level<<<blocks, 256, 0, L.s>>>(gt, a_prev, b_prev, a_out, b_out);
  return cudaGetLastError();
}

}  // namespace abft
