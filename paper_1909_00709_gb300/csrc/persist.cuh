// Persistent cooperative kernels: many sweeps of one grid in one launch (kernels and
// their launch helpers, included by persist.cu, persist_bc.cu and persist_zero.cu).
//
// Every CTA stays resident for the whole run and owns a fixed set of 128 x TY tiles;
// sweeps are separated by a grid barrier instead of a kernel boundary.
//
// Unprotected (k_persist_plain): sweep, barrier, repeat.
//
// Online (k_persist_online), with the check one sweep behind the sweep:
//   iteration k (sweep index s = step0 + k), buffers rotate u^{s-1}, u^s, u^{s+1}:
//     a. start the TMA loads of the first tile of sweep s;
//     b. check u^s: every thread takes a slice of the checksum entries (cross-tile
//        reduction of the partials sweep s-1 wrote, Theorem 1 from a^{s-1}, b^{s-1},
//        the Sec. 3.4 test), overlapping the load latency;
//     c. sweep u^s -> u^{s+1} (partials into the other partial buffer);
//     d. grid barrier;
//     e. only if some entry of u^s failed: block 0 locates and corrects u^s
//        (Sec. 3.5, lines recomputed from u^{s-1}) and then repairs u^{s+1}: every
//        point whose stencil read a repaired point is recomputed from the repaired
//        u^s (with the same arithmetic as the sweep, flips of sweep s+1 re-applied)
//        and the partials of the touched tile rows and columns are recomputed with
//        the sweep epilogue's exact arithmetic; a second barrier publishes it.
//   A final check of the last output ends the launch.  The result (grid, events,
//   checksums) is bit-identical to checking after every sweep, with one barrier
//   per sweep in the fault-free case instead of three.
// Barrier waits are bounded: on timeout the status word is set and the launch winds
// down instead of hanging.
#pragma once

#include <algorithm>
#include <cstring>

#include "check_dev.cuh"
#include "sweep_tile.cuh"

namespace abft {

struct PersistArgs {
  CUtensorMap tm_u[3];
  CUtensorMap tm_c;
  CUtensorMap tm_p[4];  // partial buffers for the check warp: PA, PA2, PB, PB2
  GridDev g;
  long long step0;   // sweep index of the first sweep of this launch
  int n_steps;
  int first_in;      // buffer of the first sweep's input (offline: the checkpoint)
  int p, q;          // then outputs alternate p, q, p, ... (sweep k >= 1 reads the previous output)
  int delta;         // offline detection period
};

template <class Tiles>
__global__ void __launch_bounds__(256, 2)
    k_persist_plain(const __grid_constant__ PersistArgs a, DevCtrl* __restrict__ ctrl, abft_event* __restrict__ ev,
                    DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const GridDev& g = a.g;
  sched.load(ctrl);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) prefetch_tensormap(&a.tm_u[k]);
    prefetch_tensormap(&a.tm_c);
  }
  __syncthreads();
  const int ntiles = g.ntx * g.nty;
  const bool resident_c = (int)gridDim.x >= ntiles;  // one tile per CTA: C stays in shared memory
  bool ok = true;
  for (int k = 0; k < a.n_steps && ok; ++k) {
    const int in = k == 0 ? a.first_in : ((k & 1) ? a.p : a.q);
    const int out = (k & 1) ? a.q : a.p;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      tiles.issue(&a.tm_u[in], &a.tm_c, g, tile % g.ntx, tile / g.ntx, a.step0 + k, ctrl, sched,
                  !resident_c || k == 0);
      tiles.template run<false, ABFT_ACC_FP32>(&a.tm_u[in], &a.tm_c, g, g.u[in], g.u[out], tile % g.ntx,
                                               tile / g.ntx, ctrl, 0);
    }
    ok = grid_barrier(&g.gc->bar, ctrl);
  }
  if (ok && blockIdx.x == 0 && threadIdx.x == 0) g.gc->step = a.step0 + a.n_steps;
}

// Box (z, y, x ranges) of u^{s+1} points whose stencil read something that the fix
// f = (kind, z, y, x) of u^s changed.  With periodic boundaries a fix on a face also
// reaches the opposite face: the box then spans that axis.
__device__ __forceinline__ void fix_box(const GridDev& g, int4 f, int lo[3], int hi[3]) {
  const int zz = f.y, yy = f.z, xx = f.w;
  const bool wrap = g.bc == ABFT_BC_PERIODIC;
  lo[0] = max(zz - 1, 0); hi[0] = min(zz + 1, g.nz - 1);
  if (wrap && (zz == 0 || zz == g.nz - 1)) { lo[0] = 0; hi[0] = g.nz - 1; }
  if (f.x == kFixPlane || f.x == kFixCol || (wrap && (yy == 0 || yy == g.ny - 1))) { lo[1] = 0; hi[1] = g.ny - 1; }
  else { lo[1] = max(yy - 1, 0); hi[1] = min(yy + 1, g.ny - 1); }
  if (f.x == kFixPlane || f.x == kFixRow || (wrap && (xx == 0 || xx == g.nx - 1))) { lo[2] = 0; hi[2] = g.nx - 1; }
  else { lo[2] = max(xx - 1, 0); hi[2] = min(xx + 1, g.nx - 1); }
}

// points of u^{s+1} that repair_next would recompute for the fixes in `sm` (every
// plane when the fix list overflowed)
__device__ __forceinline__ long long repair_volume(const GridDev& g, const ResolveSmem& sm) {
  if (sm.nfix > kFixCap) return (long long)g.nz * g.ny * g.nx;
  long long v = 0;
  for (int i = 0; i < sm.nfix; ++i) {
    int lo[3], hi[3];
    fix_box(g, sm.fix[i], lo, hi);
    v += (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  }
  return v;
}

// Block 0: after the fixes `sm.fix` of u^s, recompute the affected points of u^{s+1}
// (the output of sweep `sweep_s`, whose flips are re-applied) and the partials
// (buffer PA/PB) of every tile row and column that holds one.
template <class Tiles, int TY, int ACC>
__device__ void repair_next(const GridDev& g, const float* u_s, float* u_n, void* PA, void* PB, const ResolveSmem& sm,
                            long long sweep_s, DevCtrl* ctrl, const DevSched& sched) {
  const int nfix = sm.nfix;
  const bool overflow = nfix > kFixCap;
  const int nitems = overflow ? g.nz : nfix;
  auto item = [&](int i) -> int4 {  // on overflow: every plane
    return overflow ? make_int4(kFixPlane, i, -1, -1) : sm.fix[i];
  };
  for (int i = 0; i < nitems; ++i) {
    int lo[3], hi[3];
    fix_box(g, item(i), lo, hi);
    const int ny = hi[1] - lo[1] + 1, nx = hi[2] - lo[2] + 1;
    const long long vol = (long long)(hi[0] - lo[0] + 1) * ny * nx;
    for (long long t = threadIdx.x; t < vol; t += blockDim.x) {
      const int z = lo[0] + (int)(t / ((long long)ny * nx));
      const int r = (int)(t % ((long long)ny * nx));
      const int y = lo[1] + r / nx, x = lo[2] + r % nx;
      const float v = reapply_flips(point_update(g, u_s, z, y, x), g, ctrl, sched, sweep_s, z, y, x);
      u_n[((size_t)z * g.ny + y) * g.px + x] = v;
    }
  }
  __threadfence();
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int i = 0; i < nitems; ++i) {
    int lo[3], hi[3];
    fix_box(g, item(i), lo, hi);
    const int tx0 = lo[2] / kTX, tx1 = hi[2] / kTX;
    const int ty0 = lo[1] / TY, ty1 = hi[1] / TY;
    // row partials: one warp per (z, y, tile-x)
    const int nrows = (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (tx1 - tx0 + 1);
    for (int t = warp; t < nrows; t += nwarps) {
      const int ntx = tx1 - tx0 + 1, nyy = hi[1] - lo[1] + 1;
      const int z = lo[0] + t / (nyy * ntx);
      const int r = t % (nyy * ntx);
      recompute_pb<ACC>(g, u_n, PB, tx0 + r % ntx, z, lo[1] + r / ntx);
    }
    // column partials: one thread per (z, x, tile-y); none with one checksum vector
    if (g.vec == 1) continue;
    const int xa = lo[2], xb = hi[2];
    const int ncols = (hi[0] - lo[0] + 1) * (xb - xa + 1) * (ty1 - ty0 + 1);
    for (int t = threadIdx.x; t < ncols; t += blockDim.x) {
      const int nxx = xb - xa + 1, nty = ty1 - ty0 + 1;
      const int z = lo[0] + t / (nxx * nty);
      const int r = t % (nxx * nty);
      Tiles::template recompute_col<ACC>(g, u_n, PA, ty0 + r / nxx, z, xa + r % nxx);
    }
  }
  __threadfence();
  fence_proxy_async_global();  // u^{s+1} is read by TMA in the next sweep
  __syncthreads();
}

// Eight sweep warps and one check warp.  Two such CTAs per SM hold 18 warps, five on
// some of the SM's four register-file quarters (16,384 registers each), which caps a
// thread at 96 registers; a 112-register cap left one CTA per SM (measured 3.4x slower).
constexpr int kOnlineThreads = kSweepThreads + 32;

template <class Tiles, int TY, int ACC, int VEC = 2>
__global__ void __launch_bounds__(kOnlineThreads, 2)
    k_persist_online(const __grid_constant__ PersistArgs a, DevCtrl* __restrict__ ctrl, abft_event* __restrict__ ev,
                     DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ResolveSmem rs;
  const GridDev& g = a.g;
  sched.load(ctrl);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) prefetch_tensormap(&a.tm_u[k]);
    prefetch_tensormap(&a.tm_c);
  }
  __syncthreads();
  unsigned long long* bars = g.gc->bars;
  unsigned nbar = 0;  // barrier instances passed (identical in every CTA)
  __shared__ unsigned s_fails, s_redo;
  if (threadIdx.x == 0) s_fails = s_redo = 0;
  const int ntiles = g.ntx * g.nty;
  const bool resident_c = (int)gridDim.x >= ntiles;
  const bool sweeper = threadIdx.x < kSweepThreads;
  // the check warp's rounds and its shared-memory box (after the tiles' shared memory)
  const int rounds = check_rounds_of(g);
  const int r0 = (int)((long long)rounds * blockIdx.x / gridDim.x);
  const int r1 = (int)((long long)rounds * (blockIdx.x + 1) / gridDim.x);
  unsigned char* craw = smem_raw + Tiles::smem_bytes(g.nz);  // past the tiles' region
  unsigned char* cbase = craw + ((128 - (smem_u32(craw) & 127)) & 127);
  uint64_t* cbar = reinterpret_cast<uint64_t*>(cbase);
  unsigned char* cbuf = cbase + 128;
  unsigned cphase = 0;
  if (threadIdx.x == kSweepThreads) {
    mbar_init(cbar, 1);
    fence_barrier_init();
    for (int k = 0; k < 4; ++k) prefetch_tensormap(&a.tm_p[k]);
  }
  __syncthreads();
  bool ok = true;
  for (int k = 0; k <= a.n_steps && ok; ++k) {
    const long long s = a.step0 + k;
    const int cur = (a.first_in + k) % 3, nxt = (a.first_in + k + 1) % 3, prv = (a.first_in + k + 2) % 3;
    const int pb_cur = (int)(s & 1), pb_nxt = (int)((s + 1) & 1);
    const bool sweep = k < a.n_steps, check = k > 0;
    if (sweeper) {
      // sweep warps: u^s -> u^{s+1}, partials into the other partial buffer
      if (sweep)
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
          tiles.issue(&a.tm_u[cur], &a.tm_c, g, tile % g.ntx, tile / g.ntx, s, ctrl, sched, !resident_c || k == 0);
          tiles.template run<true, ACC, VEC>(&a.tm_u[cur], &a.tm_c, g, g.u[cur], g.u[nxt], tile % g.ntx, tile / g.ntx,
                                        ctrl, pb_nxt);
        }
    } else if (check) {
      // check warp, concurrently: u^s against the interpolation from a^{s-1}, b^{s-1}
      const InterpW iw(g.k);
      for (int r = r0; r < r1; ++r)
        check_box_round<ACC>(g, iw, a.tm_p, prv, cur, pb_cur, r, cbuf, cbar, cphase, ctrl, &s_fails);
    }
    // the barrier carries this CTA's failing-entry count and returns the total
    unsigned total = 0;
    ok = grid_barrier_sum(bars, nbar++, &s_fails, ctrl, &total);
    if (!ok || !check) continue;
    // rare: locate, correct, repair the speculative sweep
    if (total != 0) {
      // one-vector checks: every CTA sums a share of the columns the location needs (the
      // other kernels leave it to the location step's block)
      constexpr bool summed = VEC == 1;
      if (summed) {
        demand_sums(g, g.u[prv], g.u[cur], g.A[cur], g.AP[1], blockIdx.x, gridDim.x);
        unsigned none = 0;
        ok = grid_barrier_sum(bars, nbar++, nullptr, ctrl, &none);
        if (!ok) continue;
      }
      if (blockIdx.x == 0) {
        // u^s is the output of sweep s - 1; u^{s+1} that of sweep s
        resolve_planes_into(rs, g, g.u[prv], g.u[cur], g.A[cur], g.B[cur], g.AP[0], g.BP[0], s - 1, ctrl, ev,
                            &g.gc->unresolved, summed);
        if (summed && threadIdx.x == 0) g.gc->nbz = 0;  // the plane list is consumed
        __syncthreads();
        // a targeted repair by this block only while it is smaller than a few tiles'
        // work; beyond that every CTA recomputes its tiles of the speculative sweep
        const bool redo = sweep && repair_volume(g, rs) > 4LL * TY * kTX * g.nz;
        if (sweep && !redo)
          repair_next<Tiles, TY, ACC>(g, g.u[cur], g.u[nxt], pb_nxt ? g.PA2 : g.PA, pb_nxt ? g.PB2 : g.PB, rs, s,
                                      ctrl, sched);
        if (threadIdx.x == 0) s_redo = redo ? 1u : 0u;
        fence_proxy_async_global();
      }
      unsigned redo_all = 0;  // block 0's decision, carried by the barrier
      ok = grid_barrier_sum(bars, nbar++, blockIdx.x == 0 ? &s_redo : nullptr, ctrl, &redo_all);
      if (ok && sweep && redo_all != 0) {
        if (sweeper)
          for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            tiles.issue(&a.tm_u[cur], &a.tm_c, g, tile % g.ntx, tile / g.ntx, s, ctrl, sched, !resident_c);
            tiles.template run<true, ACC, VEC>(&a.tm_u[cur], &a.tm_c, g, g.u[cur], g.u[nxt], tile % g.ntx,
                                          tile / g.ntx, ctrl, pb_nxt);
          }
        unsigned none = 0;
        ok = grid_barrier_sum(bars, nbar++, nullptr, ctrl, &none);
      }
    }
  }
  if (ok && blockIdx.x == 0 && threadIdx.x == 0) g.gc->step = a.step0 + a.n_steps;
}

// extra dynamic shared memory of the online kernel's check warp: alignment slack,
// mbarrier line, one box
static int check_smem(const GridDev& g, int acc) { return 256 + check_box_bytes(g.nty, g.ntx, acc); }

// ---------------------------------------------------------------- offline
// Windows of d = delta sweeps (the last may be shorter) from a checkpoint ck (Sec. 4):
//   sweeps ck -> W0 -> W1 -> W0 ... (the last one protected, writing partials), while the
//   spare warp advances the chain of Fig. 10 one link per sweep: P^0 = a(ck),
//   P^{k+1} = Theorem 1 applied to P^k (boundary terms vanish), into AP[(k+1) & 1];
//   after the window every thread reduces a slice of the partials into a(F) and compares
//   with P^d; on a mismatch the window is recomputed from ck without injection (the same
//   buffers, so the roles stay fixed) and compared again.  Then F becomes the checkpoint.
// One grid barrier per sweep plus one per window (a payload barrier that returns the
// comparison's count of failing entries to every CTA).
__device__ __forceinline__ void window_buffers(int ck, int& w0, int& w1) {
  w0 = (ck + 1) % 3;
  w1 = (ck + 2) % 3;
}

template <class Tiles, int TY, int ACC>
__global__ void __launch_bounds__(kOnlineThreads, 2)
    k_persist_offline(const __grid_constant__ PersistArgs a, DevCtrl* __restrict__ ctrl,
                      abft_event* __restrict__ ev, DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const GridDev& g = a.g;
  sched.load(ctrl);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) prefetch_tensormap(&a.tm_u[k]);
    prefetch_tensormap(&a.tm_c);
  }
  __syncthreads();
  unsigned long long* bar = &g.gc->bar;
  unsigned long long* bars = g.gc->bars;  // payload barrier of the window comparisons
  unsigned nbar = 0;
  __shared__ unsigned s_fails;
  if (threadIdx.x == 0) s_fails = 0;
  const int ntiles = g.ntx * g.nty;
  const bool resident_c = (int)gridDim.x >= ntiles;
  const bool sweeper = threadIdx.x < kSweepThreads;
  const int na = g.nz * g.nx, n_entries = g.nz * (g.nx + g.ny);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gsize = (long long)gridDim.x * blockDim.x;
  const int c0 = (int)((long long)n_entries * blockIdx.x / gridDim.x);  // chain slice of this CTA
  const int c1 = (int)((long long)n_entries * (blockIdx.x + 1) / gridDim.x);
  int ck = a.first_in;
  bool ok = true, first_load = true;
  long long t = a.step0;
  const long long t_end = a.step0 + a.n_steps;
  while (t < t_end && ok) {
    const int d = (int)min((long long)a.delta, t_end - t);
    int w[2];
    window_buffers(ck, w[0], w[1]);
    const int fin = w[(d - 1) & 1];
    for (int attempt = 0; attempt < 2 && ok; ++attempt) {
      DevSched sw = sched;
      if (attempt) sw.enabled = 0;  // a recomputed window is fault-free
      for (int k = 0; k < d && ok; ++k) {
        const int in = k == 0 ? ck : w[(k - 1) & 1], out = w[k & 1];
        const long long s = t + k;
        if (sweeper) {
          for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            tiles.issue(&a.tm_u[in], &a.tm_c, g, tile % g.ntx, tile / g.ntx, s, ctrl, sw, !resident_c || first_load);
            if (k == d - 1)
              tiles.template run<true, ACC>(&a.tm_u[in], &a.tm_c, g, g.u[in], g.u[out], tile % g.ntx,
                                            tile / g.ntx, ctrl, 0);
            else
              tiles.template run<false, ACC>(&a.tm_u[in], &a.tm_c, g, g.u[in], g.u[out], tile % g.ntx,
                                             tile / g.ntx, ctrl, 0);
          }
        } else if (attempt == 0) {
          // one link of the chain, this CTA's slice, concurrently with the sweep
          const double* pa = k == 0 ? g.A[ck] : g.AP[k & 1];
          const double* pb = k == 0 ? g.B[ck] : g.BP[k & 1];
          double* qa = g.AP[(k + 1) & 1];
          double* qb = g.BP[(k + 1) & 1];
          for (int e = c0 + (int)(threadIdx.x & 31); e < c1; e += 32) {
            if (e < na) {
              const int z = e / g.nx, x = e - z * g.nx;
              qa[e] = predict_a(g, pa, nullptr, z, x);
            } else {
              const int b = e - na, z = b / g.ny, y = b - z * g.ny;
              qb[b] = predict_b(g, pb, nullptr, z, y);
            }
          }
        }
        first_load = false;
        ok = grid_barrier(bar, ctrl);
      }
      if (!ok) break;
      // compare the recomputed checksums of the window's result with the chain; the
      // count of failing entries rides on the next barrier's arrivals
      const double* pa = g.AP[d & 1];
      const double* pb = g.BP[d & 1];
      unsigned nf = 0;
      for (long long i = gtid; i < n_entries; i += gsize) {
        if (i < na) {
          const int z = (int)i / g.nx, x = (int)i - z * g.nx;
          const double sum = reduce_a<ACC>(g, z, x, 0);
          g.A[fin][i] = sum;
          nf += fails(__ldcg(pa + i), sum, g.eps) ? 1u : 0u;
          note_resid(g, __ldcg(pa + i), sum);
        } else {
          const int b = (int)(i - na), z = b / g.ny, y = b - z * g.ny;
          const double sum = reduce_b<ACC>(g, z, y, 0);
          g.B[fin][b] = sum;
          nf += fails(__ldcg(pb + b), sum, g.eps) ? 1u : 0u;
          note_resid(g, __ldcg(pb + b), sum);
        }
      }
      if (nf) atomicAdd(&s_fails, nf);
      unsigned bad = 0;
      ok = grid_barrier_sum(bars, nbar++, &s_fails, ctrl, &bad);
      if (!ok) break;
      if (bad == 0) break;
      if (attempt == 1) {  // the fault-free recomputation must verify
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctrl, kStUncorrectable);
        ok = false;
        break;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {  // Sec. 4.2: restore the checkpoint and recompute
        log_event(ctrl, ev, t, g.gid, -1, -1, -1, ABFT_EV_ROLLBACK, (float)bad, (float)d);
        atomicAdd(&g.gc->rollbacks, 1u);
      }
    }
    ck = fin;
    t += d;
  }
  if (ok && blockIdx.x == 0 && threadIdx.x == 0) g.gc->step = t_end;
}

template <class Tiles, int TY, int ACC>
static cudaError_t launch_offline_t(const Launch& L, const PersistArgs& a, int* blocks_out) {
  auto kern = k_persist_offline<Tiles, TY, ACC>;
  const int smem = Tiles::smem_bytes(a.g.nz);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOnlineThreads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ntiles = a.g.ntx * a.g.nty;
  int blocks = std::min(per_sm * sms, ntiles);
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  const int rounds = (ntiles + blocks - 1) / blocks;
  blocks = (ntiles + rounds - 1) / rounds;
  *blocks_out = blocks;
  DevCtrl* ctrl = L.ctrl;
  abft_event* ev = L.events;
  DevSched sched = L.sched;
  void* args[] = {(void*)&a, (void*)&ctrl, (void*)&ev, (void*)&sched};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kOnlineThreads), args, smem, L.s);
}

template <class Tiles, int TY>
static cudaError_t launch_offline_ty(const Launch& L, const PersistArgs& a, int* blocks) {
  switch (a.g.acc) {
    case ABFT_ACC_TWOSUM: return launch_offline_t<Tiles, TY, ABFT_ACC_TWOSUM>(L, a, blocks);
    case ABFT_ACC_FP64: return launch_offline_t<Tiles, TY, ABFT_ACC_FP64>(L, a, blocks);
    default: return launch_offline_t<Tiles, TY, ABFT_ACC_FP32>(L, a, blocks);
  }
}

template <class Tiles, int TY, bool PROT, int ACC, int VEC = 2>
static cudaError_t launch_persist_t(const Launch& L, const PersistArgs& a, int* blocks_out) {
  auto kern = PROT ? k_persist_online<Tiles, TY, ACC, VEC> : k_persist_plain<Tiles>;
  const int smem = Tiles::smem_bytes(a.g.nz) + (PROT ? check_smem(a.g, ACC) : 0);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int threads = PROT ? kOnlineThreads : 256;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ntiles = a.g.ntx * a.g.nty;
  int blocks = per_sm * sms;
  if (blocks > ntiles) blocks = ntiles;
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  // every CTA should own the same number of tiles: trim to the largest grid that does
  const int rounds = (ntiles + blocks - 1) / blocks;
  blocks = (ntiles + rounds - 1) / rounds;
  *blocks_out = blocks;
  DevCtrl* ctrl = L.ctrl;
  abft_event* ev = L.events;
  DevSched sched = L.sched;
  void* args[] = {(void*)&a, (void*)&ctrl, (void*)&ev, (void*)&sched};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(threads), args, smem, L.s);
}

template <class Tiles, int TY>
static cudaError_t launch_persist_ty(const Launch& L, const PersistArgs& a, bool prot, int* blocks) {
  if (!prot) return launch_persist_t<Tiles, TY, false, ABFT_ACC_FP32>(L, a, blocks);
  switch (a.g.acc) {
    case ABFT_ACC_TWOSUM: return launch_persist_t<Tiles, TY, true, ABFT_ACC_TWOSUM>(L, a, blocks);
    case ABFT_ACC_FP64: return launch_persist_t<Tiles, TY, true, ABFT_ACC_FP64>(L, a, blocks);
    default:
      return a.g.vec == 1 ? launch_persist_t<Tiles, TY, true, ABFT_ACC_FP32, 1>(L, a, blocks)
                          : launch_persist_t<Tiles, TY, true, ABFT_ACC_FP32>(L, a, blocks);
  }
}

// Whether the persistent kernel suits this grid: every CTA owns a single tile (the
// case it is built for), or, for unprotected sweeps, at least two CTAs fit on an SM and
// each CTA streams several tiles per sweep (measured faster than one launch per sweep
// at 1024x1024x256; the online kernel with several tiles per CTA was slower).
template <class Tiles, int TY>
static bool fits_t(const GridDev& g, bool prot) {
  if (prot && (g.nty > 256 || g.ntx > 256)) return false;  // one TMA box per check round
  const void* kern = prot ? (const void*)k_persist_online<Tiles, TY, ABFT_ACC_FP32> : (const void*)k_persist_plain<Tiles>;
  const int smem = Tiles::smem_bytes(g.nz) + (prot ? check_smem(g, g.acc) : 0);
  if (smem > 227 * 1024) return false;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, prot ? kOnlineThreads : 256, smem) != cudaSuccess)
    return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  return (long long)g.ntx * g.nty <= (long long)per_sm * sms || (!prot && per_sm >= 2);
}

template <class Tiles, int TY>
static bool offline_fits_t(const GridDev& g) {
  const void* kern = (const void*)k_persist_offline<Tiles, TY, ABFT_ACC_FP32>;
  const int smem = Tiles::smem_bytes(g.nz);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return false;
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOnlineThreads, smem) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  return (long long)g.ntx * g.nty <= (long long)per_sm * sms;
}

template <int BC>
static bool persistent_fits_cl(const GridDev& g, bool prot) {
  if (g.shallow)
    return g.ty == 7   ? fits_t<ShallowTiles<7, BC>, 7>(g, prot)
           : g.ty == 8 ? fits_t<ShallowTiles<8, BC>, 8>(g, prot)
                       : fits_t<ShallowTiles<16, BC>, 16>(g, prot);
  switch (g.ty) {
    case 8: return fits_t<StreamTiles<8, BC>, 8>(g, prot);
    case 16: return fits_t<StreamTiles<16, BC>, 16>(g, prot);
    default: return fits_t<StreamTiles<32, BC>, 32>(g, prot);
  }
}

template <int BC>
static cudaError_t launch_persistent_cl(const Launch& L, const PersistArgs& a, bool prot, int* blocks) {
  const GridDev& g = a.g;
  if (g.shallow) {
    switch (g.ty) {
      case 7: return launch_persist_ty<ShallowTiles<7, BC>, 7>(L, a, prot, blocks);
      case 8: return launch_persist_ty<ShallowTiles<8, BC>, 8>(L, a, prot, blocks);
      case 16: return launch_persist_ty<ShallowTiles<16, BC>, 16>(L, a, prot, blocks);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.ty) {
    case 8: return launch_persist_ty<StreamTiles<8, BC>, 8>(L, a, prot, blocks);
    case 16: return launch_persist_ty<StreamTiles<16, BC>, 16>(L, a, prot, blocks);
    case 32: return launch_persist_ty<StreamTiles<32, BC>, 32>(L, a, prot, blocks);
    default: return cudaErrorInvalidValue;
  }
}

template <int BC>
static cudaError_t launch_offline_cl(const Launch& L, const PersistArgs& a, int* blocks) {
  const GridDev& g = a.g;
  if (g.shallow) {
    switch (g.ty) {
      case 7: return launch_offline_ty<ShallowTiles<7, BC>, 7>(L, a, blocks);
      case 8: return launch_offline_ty<ShallowTiles<8, BC>, 8>(L, a, blocks);
      case 16: return launch_offline_ty<ShallowTiles<16, BC>, 16>(L, a, blocks);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.ty) {
    case 8: return launch_offline_ty<StreamTiles<8, BC>, 8>(L, a, blocks);
    case 16: return launch_offline_ty<StreamTiles<16, BC>, 16>(L, a, blocks);
    case 32: return launch_offline_ty<StreamTiles<32, BC>, 32>(L, a, blocks);
    default: return cudaErrorInvalidValue;
  }
}

template <int BC>
static bool offline_fits_cl(const GridDev& g) {
  if (g.shallow)
    return g.ty == 7   ? offline_fits_t<ShallowTiles<7, BC>, 7>(g)
           : g.ty == 8 ? offline_fits_t<ShallowTiles<8, BC>, 8>(g)
                       : offline_fits_t<ShallowTiles<16, BC>, 16>(g);
  switch (g.ty) {
    case 8: return offline_fits_t<StreamTiles<8, BC>, 8>(g);
    case 16: return offline_fits_t<StreamTiles<16, BC>, 16>(g);
    default: return offline_fits_t<StreamTiles<32, BC>, 32>(g);
  }
}

// The same launches for grids with a periodic (persist_bc.cu) or an empty boundary
// (persist_zero.cu), each rule's kernels compiled in a translation unit of its own.
bool persistent_fits_periodic(const GridDev& g, bool prot);
cudaError_t launch_persistent_periodic(const Launch& L, const PersistArgs& a, bool prot, int* blocks);
cudaError_t launch_offline_periodic(const Launch& L, const PersistArgs& a, int* blocks);
bool persistent_offline_fits_periodic(const GridDev& g);
bool persistent_fits_zero(const GridDev& g, bool prot);
cudaError_t launch_persistent_zero(const Launch& L, const PersistArgs& a, bool prot, int* blocks);
cudaError_t launch_offline_zero(const Launch& L, const PersistArgs& a, int* blocks);
bool persistent_offline_fits_zero(const GridDev& g);

}  // namespace abft
