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
// check kernel, so results are bitwise repeatable.  The tile body is sweep_tile()
// in sweep_tile.cuh, shared with the persistent kernel.
#include "sweep_tile.cuh"

namespace abft {

// One sweep of one grid: one CTA per tile.  The last CTA to finish commits the sweep
// by advancing the grid's step counter (it drives injection and event stamps).
template <class Tiles, bool PROT, int ACC, int VEC = 2>
__global__ void __launch_bounds__(256, 2)
    k_sweep(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_c,
            const GridDev g, const float* __restrict__ uin, float* __restrict__ uout, DevCtrl* __restrict__ ctrl,
            DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  sched.load(ctrl);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_c);
  }
  __syncthreads();
  const long long step = g.gc->step;
  const int txi = blockIdx.x % g.ntx, tyi = blockIdx.x / g.ntx;
  tiles.issue(&tm_u, &tm_c, g, txi, tyi, step, ctrl, sched, true);
  tiles.template run<PROT, ACC, VEC>(&tm_u, &tm_c, g, uin, uout, txi, tyi, ctrl, 0);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == gridDim.x - 1) {
      g.gc->done_sweep = 0;
      g.gc->step = step + 1;
      __threadfence();
    }
  }
}

// The conditional repair of the sweep just committed, after a late correction of its
// input (the overlapped online path, where the sweep started before the previous
// check had finished): every CTA leaves at once unless the location step flagged a
// correction.  A tile it marked recomputes, from the corrected input, what the
// correction reached: for a few planes (the marked range widened by one plane on each
// side) the points one by one with the sweep's arithmetic and flips, then those planes'
// partial checksums with the epilogue's exact arithmetic; for more planes the whole
// tile, streamed as the sweep streams it.  The last CTA clears the flag.
constexpr int kRedoPlanes = 8;  // above this many planes a tile is streamed again

template <class Tiles, int TY, int ACC, int VEC = 2>
__global__ void __launch_bounds__(256, 2)
    k_redo_tiles(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_c, const GridDev g,
                 const float* __restrict__ uin, float* __restrict__ uout, DevCtrl* __restrict__ ctrl, DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int4 lf[kLocalFlips];
  __shared__ int nlf;
  if (__ldcg(&g.gc->redo) == 0) return;  // uniform: the flag only changes after every CTA
  const int t = blockIdx.x, ntiles = gridDim.x;
  int* hi1 = g.tdirty;            // highest marked plane + 1 (0: clean)
  int* lorev = g.tdirty + ntiles;  // nz - lowest marked plane
  const int h = __ldcg(hi1 + t);
  if (h != 0) {
    sched.load(ctrl);
    const long long step = g.gc->step - 1;  // the committed sweep
    const int zl = max(g.nz - __ldcg(lorev + t) - 1, 0), zh = min(h, g.nz - 1);
    const int txi = t % g.ntx, tyi = t / g.ntx;
    const int x0 = txi * kTX, y0 = tyi * TY;
    const int npl = zh - zl + 1;
    if (npl > kRedoPlanes) {
      Tiles tiles;
      tiles.setup(smem_raw, g.nz);
      if (threadIdx.x == 0) {
        prefetch_tensormap(&tm_u);
        prefetch_tensormap(&tm_c);
      }
      __syncthreads();
      tiles.issue(&tm_u, &tm_c, g, txi, tyi, step, ctrl, sched, true);
      tiles.template run<true, ACC, VEC>(&tm_u, &tm_c, g, uin, uout, txi, tyi, ctrl, 0);
    } else {
      const int ncol = min(kTX, g.nx - x0), nrow = min(TY, g.ny - y0);
      // this sweep's flips inside the tile, gathered once
      if (threadIdx.x == 0) nlf = 0;
      __syncthreads();
      if (sched.enabled) {
        const long long i = step - sched.t0;
        if (i >= 0 && i < sched.n)
          for (int k = sched.off[i] + threadIdx.x; k < sched.off[i + 1]; k += blockDim.x) {
            const DevFlip f = sched.flips[k];
            if (f.grid == g.gid && f.target == 0 && f.x >= x0 && f.x < x0 + ncol && f.y >= y0 && f.y < y0 + nrow &&
                f.z >= zl && f.z <= zh) {
              const int j = atomicAdd(&nlf, 1);
              if (j < kLocalFlips) lf[j] = make_int4(f.x, f.y, f.z, f.bit & 31);
              else set_status(ctrl, kStFlipOverflow);
            }
          }
      }
      __syncthreads();
      const int nf = min(nlf, kLocalFlips);
      for (int i = threadIdx.x; i < npl * nrow * ncol; i += blockDim.x) {
        const int z = zl + i / (nrow * ncol), r = i % (nrow * ncol);
        const int y = y0 + r / ncol, x = x0 + r % ncol;
        float v = point_update(g, uin, z, y, x);
        for (int k = 0; k < nf; ++k)
          if (lf[k].x == x && lf[k].y == y && lf[k].z == z) v = __int_as_float(__float_as_int(v) ^ (1 << lf[k].w));
        uout[((size_t)z * g.ny + y) * g.px + x] = v;
      }
      __syncthreads();
      if (VEC == 2)
        for (int i = threadIdx.x; i < npl * kTX; i += blockDim.x)
          Tiles::template recompute_col<ACC>(g, uout, g.PA, tyi, zl + i / kTX, x0 + i % kTX);
      for (int w = threadIdx.x >> 5; w < npl * nrow; w += blockDim.x >> 5)
        recompute_pb<ACC>(g, uout, g.PB, txi, zl + w / nrow, y0 + w % nrow);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      hi1[t] = 0;
      lorev[t] = 0;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == gridDim.x - 1) {
      g.gc->done_sweep = 0;
      g.gc->redo = 0;
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

template <class Tiles, bool PROT, int ACC, int VEC = 2>
static cudaError_t launch_t(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                            int in, int out) {
  auto kern = k_sweep<Tiles, PROT, ACC, VEC>;
  const int smem = Tiles::smem_bytes(g.nz);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<g.ntx * g.nty, 256, smem, L.s>>>(tm_in, tm_c, g, g.u[in], g.u[out], L.ctrl, L.sched);
  return cudaGetLastError();
}

template <class Tiles>
static cudaError_t launch_tiles(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                                int in, int out, bool prot) {
  if (!prot) return launch_t<Tiles, false, ABFT_ACC_FP32>(L, g, tm_in, tm_c, in, out);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: return launch_t<Tiles, true, ABFT_ACC_TWOSUM>(L, g, tm_in, tm_c, in, out);
    case ABFT_ACC_FP64: return launch_t<Tiles, true, ABFT_ACC_FP64>(L, g, tm_in, tm_c, in, out);
    default:
      return g.vec == 1 ? launch_t<Tiles, true, ABFT_ACC_FP32, 1>(L, g, tm_in, tm_c, in, out)
                        : launch_t<Tiles, true, ABFT_ACC_FP32>(L, g, tm_in, tm_c, in, out);
  }
}

template <int BC>
static cudaError_t launch_sweep_bc(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                                   const CUtensorMap& tm_c, int in, int out, bool prot) {
  if (g.shallow) {
    switch (g.ty) {
      case 7: return launch_tiles<ShallowTiles<7, BC>>(L, g, tm_in, tm_c, in, out, prot);
      case 8: return launch_tiles<ShallowTiles<8, BC>>(L, g, tm_in, tm_c, in, out, prot);
      case 16: return launch_tiles<ShallowTiles<16, BC>>(L, g, tm_in, tm_c, in, out, prot);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.ty) {
    case 8: return launch_tiles<StreamTiles<8, BC>>(L, g, tm_in, tm_c, in, out, prot);
    case 16: return launch_tiles<StreamTiles<16, BC>>(L, g, tm_in, tm_c, in, out, prot);
    case 32: return launch_tiles<StreamTiles<32, BC>>(L, g, tm_in, tm_c, in, out, prot);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c, int in,
                         int out, bool prot) {
  switch (g.bc) {
    case ABFT_BC_PERIODIC: return launch_sweep_bc<ABFT_BC_PERIODIC>(L, g, tm_in, tm_c, in, out, prot);
    case ABFT_BC_ZERO: return launch_sweep_bc<ABFT_BC_ZERO>(L, g, tm_in, tm_c, in, out, prot);
    default: return launch_sweep_bc<ABFT_BC_CLAMP>(L, g, tm_in, tm_c, in, out, prot);
  }
}

template <class Tiles, int TY>
static cudaError_t redo_t(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c, int in,
                          int out) {
  const int blocks = g.ntx * g.nty, smem = Tiles::smem_bytes(g.nz);
  auto kern = g.acc == ABFT_ACC_TWOSUM ? k_redo_tiles<Tiles, TY, ABFT_ACC_TWOSUM>
              : g.acc == ABFT_ACC_FP64 ? k_redo_tiles<Tiles, TY, ABFT_ACC_FP64>
              : g.vec == 1             ? k_redo_tiles<Tiles, TY, ABFT_ACC_FP32, 1>
                                       : k_redo_tiles<Tiles, TY, ABFT_ACC_FP32>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, 256, smem, L.s>>>(tm_in, tm_c, g, g.u[in], g.u[out], L.ctrl, L.sched);
  return cudaGetLastError();
}

template <int BC>
static cudaError_t launch_redo_bc(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                                  const CUtensorMap& tm_c, int in, int out) {
  if (g.shallow) {
    switch (g.ty) {
      case 7: return redo_t<ShallowTiles<7, BC>, 7>(L, g, tm_in, tm_c, in, out);
      case 8: return redo_t<ShallowTiles<8, BC>, 8>(L, g, tm_in, tm_c, in, out);
      case 16: return redo_t<ShallowTiles<16, BC>, 16>(L, g, tm_in, tm_c, in, out);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.ty) {
    case 8: return redo_t<StreamTiles<8, BC>, 8>(L, g, tm_in, tm_c, in, out);
    case 16: return redo_t<StreamTiles<16, BC>, 16>(L, g, tm_in, tm_c, in, out);
    case 32: return redo_t<StreamTiles<32, BC>, 32>(L, g, tm_in, tm_c, in, out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_redo_tiles(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                              int in, int out) {
  switch (g.bc) {
    case ABFT_BC_PERIODIC: return launch_redo_bc<ABFT_BC_PERIODIC>(L, g, tm_in, tm_c, in, out);
    case ABFT_BC_ZERO: return launch_redo_bc<ABFT_BC_ZERO>(L, g, tm_in, tm_c, in, out);
    default: return launch_redo_bc<ABFT_BC_CLAMP>(L, g, tm_in, tm_c, in, out);
  }
}

}  // namespace abft
