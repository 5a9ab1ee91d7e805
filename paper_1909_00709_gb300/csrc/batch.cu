// Many independent grids of uneven sizes advanced together: one sweep launch per
// tile class (streaming or whole-column tiles, rows per tile) and one check launch
// per sweep cover every grid of the context.
//
// A grid alone rarely fills 152 SMs: a 544 x 544 x 34 grid has 170 tiles for 304
// CTA slots, so launching grids one after another leaves half the GPU idle and
// pays a launch per grid and kernel.  Here a launch's blocks are the tiles of all
// its grids (grid i owning blocks off[i] .. off[i+1]-1, found by binary search), so
// the GPU stays full to the last tile and a sweep of the whole batch costs two or
// three launches.  Work order puts the deepest grids first (their tiles run
// longest) to shorten the tail.
//
// Grid descriptors and tensor maps live in device memory.  Buffer roles are derived
// from each grid's own sweep counter (BatchRole), so a captured CUDA graph of T
// sweeps replays correctly at any later sweep without re-recording.  Tile bodies,
// partial-sum layouts and the check arithmetic are those of the per-grid kernels:
// results are bitwise identical to advancing the grids one by one.
#include "check_dev.cuh"
#include "sweep_tile.cuh"

namespace abft {

__device__ __forceinline__ int batch_slot(const int* __restrict__ off, int n, int b) {
  int lo = 0, hi = n;  // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void batch_roles(const BatchRole& r, long long s, int* in, int* out) {
  const long long k = s - r.s0;
  if (r.mode) {
    const int i = (int)(((r.first + k) % 3 + 3) % 3);  // in 0..2 whatever k is
    *in = i;
    *out = i == 2 ? 0 : i + 1;
  } else if (k == 0) {
    *in = r.first;
    *out = r.a;
  } else {
    *in = (k & 1) ? r.a : r.b;
    *out = (k & 1) ? r.b : r.a;
  }
}

template <class T>
__device__ __forceinline__ T pick3(T v0, T v1, T v2, int i) {
  return i == 0 ? v0 : (i == 1 ? v1 : v2);
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* tm) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tm))
               : "memory");
}

template <class Tiles, bool PROT, int ACC>
__global__ void __launch_bounds__(256, 2) k_sweep_batch(const BatchArgs a, DevCtrl* __restrict__ ctrl, DevSched sched) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  sched.load(ctrl);
  const int slot = batch_slot(a.off, a.n, blockIdx.x);
  const int gi = __ldg(a.grids + slot);
  const int t = blockIdx.x - __ldg(a.off + slot);
  const GridDev g = a.g[gi];
  const long long step = g.gc->step;
  int in, out;
  batch_roles(a.roles[gi], step, &in, &out);
  const CUtensorMap* tm_u = a.tm + kBatchMaps * gi + in;
  const CUtensorMap* tm_c = a.tm + kBatchMaps * gi + 3;
  float* uout = pick3(g.u[0], g.u[1], g.u[2], out);
  const float* uin = pick3(g.u[0], g.u[1], g.u[2], in);
  Tiles tiles;
  tiles.setup(smem_raw, g.nz);
  if (threadIdx.x == 0) {
    tensormap_acquire(tm_u);
    tensormap_acquire(tm_c);
    prefetch_tensormap(tm_u);
    prefetch_tensormap(tm_c);
  }
  __syncthreads();
  const int txi = t % g.ntx, tyi = t / g.ntx;
  tiles.issue(tm_u, tm_c, g, txi, tyi, step, ctrl, sched, true);
  tiles.template run<PROT, ACC>(tm_u, tm_c, g, uin, uout, txi, tyi, ctrl, 0);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == (unsigned)(g.ntx * g.nty) - 1) {  // this grid's last tile commits its sweep
      g.gc->done_sweep = 0;
      g.gc->step = step + 1;
      __threadfence();
    }
  }
}

// The online check of the sweep just done (Sec. 3) for every grid of the batch:
// each block's warps take 32-entry rounds of one grid (BOX: one TMA box of all tiles'
// partials per round and warp; otherwise plain coalesced loads); that grid's last
// block to finish locates and corrects (Sec. 3.5).
template <int ACC, bool BOX>
__global__ void __launch_bounds__(256, 2)
    k_check_batch(const BatchArgs a, int box, DevCtrl* __restrict__ ctrl, abft_event* __restrict__ ev) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int slot = batch_slot(a.off, a.n, blockIdx.x);
  const int gi = __ldg(a.grids + slot);
  const int b0 = __ldg(a.off + slot);
  const int lb = blockIdx.x - b0, nb = __ldg(a.off + slot + 1) - b0;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the grid's descriptor, its buffer roles normalised to slots 0 (the state the sweep
  // read) and 1 (its result) so that every index into its arrays is a constant; kept
  // in shared memory, where the location step can take its address
  __shared__ GridDev sg;
  __shared__ long long s_step;
  if (threadIdx.x == 0) {
    GridDev d = a.g[gi];
    const long long s = __ldcg(&d.gc->step) - 1;
    int in, out;
    batch_roles(a.roles[gi], s, &in, &out);
    float* ui = pick3(d.u[0], d.u[1], d.u[2], in);
    float* uo = pick3(d.u[0], d.u[1], d.u[2], out);
    double* ai = pick3(d.A[0], d.A[1], d.A[2], in);
    double* ao = pick3(d.A[0], d.A[1], d.A[2], out);
    double* bi = pick3(d.B[0], d.B[1], d.B[2], in);
    double* bo = pick3(d.B[0], d.B[1], d.B[2], out);
    d.u[0] = ui; d.u[1] = uo;
    d.A[0] = ai; d.A[1] = ao;
    d.B[0] = bi; d.B[1] = bo;
    sg = d;
    s_step = s;
  }
  __syncthreads();
  const GridDev& g = sg;
  const long long s = s_step;
  if (BOX) {
    const CUtensorMap* tm_p = a.tm + kBatchMaps * gi + 4;
    unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base) + warp;  // at most 8 warps
    unsigned char* buf = base + 128 + (size_t)warp * box;
    if (lane == 0) {
      tensormap_acquire(tm_p);
      tensormap_acquire(tm_p + 2);
      prefetch_tensormap(tm_p);
      prefetch_tensormap(tm_p + 2);
      mbar_init(bar, 1);
      fence_barrier_init();
    }
    __syncwarp();
    unsigned phase = 0;
    const InterpW iw(g.k);
    const int rounds = check_rounds_of(g);
    for (int r = lb * nw + warp; r < rounds; r += nb * nw)
      check_box_round<ACC>(g, iw, tm_p, 0, 1, 0, r, buf, bar, phase, ctrl, nullptr);
  } else {
    check_warps<ACC>(g, 0, 1, lb * nw + warp, nb * nw, g.vec == 1 ? g.nz * g.nx : 0, g.nz * (g.nx + g.ny));
  }
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&g.gc->done_check, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  resolve_planes(g, g.u[0], g.u[1], g.A[1], g.B[1], g.AP[0], g.BP[0], s, ctrl, ev, &g.gc->unresolved);
  if (threadIdx.x == 0) g.gc->done_check = 0;
}

// ------------------------------------------------------------------ host side

int batch_sweep_smem(int shallow, int ty, int nz) {
  if (shallow)
    return ty == 16 ? ShallowTiles<16>::smem_bytes(nz)
                    : (ty == 7 ? ShallowTiles<7>::smem_bytes(nz) : ShallowTiles<8>::smem_bytes(nz));
  switch (ty) {
    case 8: return StreamTiles<8>::smem_bytes(nz);
    case 32: return StreamTiles<32>::smem_bytes(nz);
    default: return StreamTiles<16>::smem_bytes(nz);
  }
}

template <class Tiles, bool PROT, int ACC>
static cudaError_t prep_t(int smem) {
  return cudaFuncSetAttribute(k_sweep_batch<Tiles, PROT, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class Tiles, bool PROT, int ACC>
static cudaError_t launch_t(const Launch& L, const BatchArgs& a, int blocks, int smem) {
  k_sweep_batch<Tiles, PROT, ACC><<<blocks, 256, smem, L.s>>>(a, L.ctrl, L.sched);
  return cudaGetLastError();
}

// dispatch on the tile class, protection and accumulation; `prep` only sets the
// shared-memory attribute (kept out of stream capture)
template <class Tiles>
static cudaError_t dispatch_acc(bool prep, const Launch* L, const BatchArgs* a, int blocks, int smem, bool prot,
                                int acc) {
  if (!prot) return prep ? prep_t<Tiles, false, 0>(smem) : launch_t<Tiles, false, 0>(*L, *a, blocks, smem);
  switch (acc) {
    case ABFT_ACC_TWOSUM:
      return prep ? prep_t<Tiles, true, ABFT_ACC_TWOSUM>(smem) : launch_t<Tiles, true, ABFT_ACC_TWOSUM>(*L, *a, blocks, smem);
    case ABFT_ACC_FP64:
      return prep ? prep_t<Tiles, true, ABFT_ACC_FP64>(smem) : launch_t<Tiles, true, ABFT_ACC_FP64>(*L, *a, blocks, smem);
    default:
      return prep ? prep_t<Tiles, true, ABFT_ACC_FP32>(smem) : launch_t<Tiles, true, ABFT_ACC_FP32>(*L, *a, blocks, smem);
  }
}

template <int BC>
static cudaError_t dispatch_bc(bool prep, const Launch* L, const BatchArgs* a, int blocks, int smem, int shallow, int ty,
                               bool prot, int acc) {
  if (shallow) {
    if (ty == 16) return dispatch_acc<ShallowTiles<16, BC>>(prep, L, a, blocks, smem, prot, acc);
    if (ty == 8) return dispatch_acc<ShallowTiles<8, BC>>(prep, L, a, blocks, smem, prot, acc);
    if (ty == 7) return dispatch_acc<ShallowTiles<7, BC>>(prep, L, a, blocks, smem, prot, acc);
    return cudaErrorInvalidValue;
  }
  switch (ty) {
    case 8: return dispatch_acc<StreamTiles<8, BC>>(prep, L, a, blocks, smem, prot, acc);
    case 16: return dispatch_acc<StreamTiles<16, BC>>(prep, L, a, blocks, smem, prot, acc);
    case 32: return dispatch_acc<StreamTiles<32, BC>>(prep, L, a, blocks, smem, prot, acc);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch(bool prep, const Launch* L, const BatchArgs* a, int blocks, int smem, int shallow, int ty,
                            bool prot, int acc, int bc) {
  switch (bc) {
    case ABFT_BC_PERIODIC: return dispatch_bc<ABFT_BC_PERIODIC>(prep, L, a, blocks, smem, shallow, ty, prot, acc);
    case ABFT_BC_ZERO: return dispatch_bc<ABFT_BC_ZERO>(prep, L, a, blocks, smem, shallow, ty, prot, acc);
    default: return dispatch_bc<ABFT_BC_CLAMP>(prep, L, a, blocks, smem, shallow, ty, prot, acc);
  }
}

cudaError_t batch_prepare(int shallow, int ty, bool prot, int acc, int bc, int smem) {
  return dispatch(true, nullptr, nullptr, 0, smem, shallow, ty, prot, acc, bc);
}

cudaError_t launch_sweep_batch(const Launch& L, const BatchArgs& a, int blocks, int smem, int shallow, int ty,
                               bool prot, int acc, int bc) {
  if (blocks <= 0) return cudaSuccess;
  return dispatch(false, &L, &a, blocks, smem, shallow, ty, prot, acc, bc);
}

template <int ACC>
static cudaError_t check_batch_t(const Launch& L, const BatchArgs& a, int blocks, int box, int nw, int smem) {
  if (box > 0)
    k_check_batch<ACC, true><<<blocks, nw * 32, smem, L.s>>>(a, box, L.ctrl, L.events);
  else
    k_check_batch<ACC, false><<<blocks, 256, 0, L.s>>>(a, 0, L.ctrl, L.events);
  return cudaGetLastError();
}

cudaError_t batch_check_prepare(int acc, int smem) {
  switch (acc) {
    case ABFT_ACC_TWOSUM:
      return cudaFuncSetAttribute(k_check_batch<ABFT_ACC_TWOSUM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case ABFT_ACC_FP64:
      return cudaFuncSetAttribute(k_check_batch<ABFT_ACC_FP64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    default:
      return cudaFuncSetAttribute(k_check_batch<ABFT_ACC_FP32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
}

cudaError_t launch_check_batch(const Launch& L, const BatchArgs& a, int blocks, int acc, int box, int nw, int smem) {
  if (blocks <= 0) return cudaSuccess;
  switch (acc) {
    case ABFT_ACC_TWOSUM: return check_batch_t<ABFT_ACC_TWOSUM>(L, a, blocks, box, nw, smem);
    case ABFT_ACC_FP64: return check_batch_t<ABFT_ACC_FP64>(L, a, blocks, box, nw, smem);
    default: return check_batch_t<ABFT_ACC_FP32>(L, a, blocks, box, nw, smem);
  }
}

}  // namespace abft
