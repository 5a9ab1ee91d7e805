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
// REDO: the conditional recomputation of the sweep just committed (used when the
// next sweep was started before the previous check had finished): every CTA leaves at
// once unless the location step flagged a correction; then only the tiles it marked
// are recomputed (for the committed sweep index), and the last CTA clears the flag
// instead of advancing the step.
template <class Tiles, bool PROT, int ACC, bool REDO>
__global__ void __launch_bounds__(256, 2)
    k_sweep(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_c,
            const GridDev g, float* __restrict__ uout, DevCtrl* __restrict__ ctrl, DevSched sched) {
  constexpr bool redo = REDO;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (redo && __ldcg(&g.gc->redo) == 0) return;  // uniform: the flag only changes after every CTA
  if (redo && __ldcg(&g.tdirty[blockIdx.x]) == 0) {  // this tile needs no recomputation
    if (threadIdx.x == 0) {
      const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
      if (ticket == gridDim.x - 1) {
        g.gc->done_sweep = 0;
        g.gc->redo = 0;
        __threadfence();
      }
    }
    return;
  }
  sched.load(ctrl);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_c);
  }
  __syncthreads();
  const long long step = g.gc->step - (redo ? 1 : 0);
  const int txi = blockIdx.x % g.ntx, tyi = blockIdx.x / g.ntx;
  tiles.issue(&tm_u, &tm_c, g, txi, tyi, step, ctrl, sched, true);
  tiles.template run<PROT, ACC>(&tm_u, &tm_c, g, uout, txi, tyi, ctrl, 0);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (redo) g.tdirty[blockIdx.x] = 0;
    if (ticket == gridDim.x - 1) {
      g.gc->done_sweep = 0;
      if (redo) g.gc->redo = 0;
      else g.gc->step = step + 1;
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

template <class Tiles, bool PROT, int ACC>
static cudaError_t launch_t(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                            int out, int redo) {
  auto kern = redo ? k_sweep<Tiles, PROT, ACC, true> : k_sweep<Tiles, PROT, ACC, false>;
  const int smem = Tiles::smem_bytes(g.nz);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<g.ntx * g.nty, 256, smem, L.s>>>(tm_in, tm_c, g, g.u[out], L.ctrl, L.sched);
  return cudaGetLastError();
}

template <class Tiles>
static cudaError_t launch_tiles(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                                int out, bool prot, int redo) {
  if (!prot) return launch_t<Tiles, false, ABFT_ACC_FP32>(L, g, tm_in, tm_c, out, redo);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: return launch_t<Tiles, true, ABFT_ACC_TWOSUM>(L, g, tm_in, tm_c, out, redo);
    case ABFT_ACC_FP64: return launch_t<Tiles, true, ABFT_ACC_FP64>(L, g, tm_in, tm_c, out, redo);
    default: return launch_t<Tiles, true, ABFT_ACC_FP32>(L, g, tm_in, tm_c, out, redo);
  }
}

cudaError_t launch_sweep(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c, int in,
                         int out, bool prot, int redo) {
  (void)in;
  if (g.shallow) {
    switch (g.ty) {
      case 8: return launch_tiles<ShallowTiles<8>>(L, g, tm_in, tm_c, out, prot, redo);
      case 16: return launch_tiles<ShallowTiles<16>>(L, g, tm_in, tm_c, out, prot, redo);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (g.ty) {
    case 8: return launch_tiles<StreamTiles<8>>(L, g, tm_in, tm_c, out, prot, redo);
    case 16: return launch_tiles<StreamTiles<16>>(L, g, tm_in, tm_c, out, prot, redo);
    case 32: return launch_tiles<StreamTiles<32>>(L, g, tm_in, tm_c, out, prot, redo);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace abft
