// General stencil sets: Eq. (1) with any set S of offsets within -2..2 (Sec. 3.1; e.g.
// a 13-point star or the 27-point box), every boundary rule of Sec. 3.3 (clamped,
// periodic, empty, constant), and the ABFT of the paper on top: fused per-tile partial
// checksums (Eq. 2, 3), the online check with Theorem 1's boundary terms evaluated
// literally from the previous state, location and correction (Eq. 8, lines recomputed
// otherwise), and the links of an offline chain (Fig. 10) whose boundary terms come from
// each step's own state where they do not vanish.
//
// The sweep: one CTA per 128 x 8 tile (one row per warp) streams z.  Staged planes (8 + 2r
// rows, 136 columns: a 4-column, 16-byte aligned x halo that covers r <= 2) and the
// tile's plane of C rotate through a ring of 2r + 3 shared-memory slots, filled by
// cp.async two planes ahead of their use: interior 16-byte chunks directly, cells outside
// the grid by 4-byte copies of the cell the boundary rule maps them to (clamped or
// wrapped index) or by stores of its fixed value (zero, the constant).  Every point
// sums its set in the set's order (one FMA chain) and adds C, the same arithmetic as
// gen_update, which the location step uses to recompute lines.  The partial checksums
// have the layout of the 7-point tiles (b: the row's 128 values by a warp butterfly;
// a: the tile's TY values per column, registers then one pass over the eight warps),
// so the cross-tile reductions of check_dev.cuh apply unchanged.
#include <algorithm>

#include "check_dev.cuh"
#include "sweep_tile.cuh"

namespace abft {

constexpr int kGenThreads = 256;
constexpr int kGenW = kTX + 2 * kHaloX;  // staged columns
constexpr int kGenChunks = kGenW / 4;    // 16-byte chunks per staged row

// ------------------------------------------------------------ the boundary rule

// map one coordinate onto 0..n-1; false when the cell lies outside with a fixed value
__device__ __forceinline__ bool gen_map(int& i, int n, int bc) {
  if (i >= 0 && i < n) return true;
  if (bc == ABFT_BC_CLAMP) {
    i = i < 0 ? 0 : n - 1;
    return true;
  }
  if (bc == ABFT_BC_PERIODIC) {
    i %= n;
    if (i < 0) i += n;
    return true;
  }
  return false;
}

__device__ __forceinline__ float gen_outside(const GridDev& g) { return g.bc == ABFT_BC_CONST ? g.bval : 0.f; }

// u at any coordinate, cells outside the grid included (each axis mapped on its own)
__device__ __forceinline__ float gen_ghost(const GridDev& g, const float* u, int z, int y, int x) {
  if (!gen_map(z, g.nz, g.bc) || !gen_map(y, g.ny, g.bc) || !gen_map(x, g.nx, g.bc)) return gen_outside(g);
  return __ldcg(u + ((size_t)z * g.ny + y) * g.px + x);
}

// Eq. (1) at one point: the set's terms in order as one FMA chain, then + C
__device__ __forceinline__ float gen_update(const GridDev& g, const float* u, int z, int y, int x) {
  const GenSten& s = *g.gs;
  float acc = 0.f;
  for (int k = 0; k < s.npts; ++k) acc = __fmaf_rn(s.w[k], gen_ghost(g, u, z + s.dz[k], y + s.dy[k], x + s.dx[k]), acc);
  return __fadd_rn(__ldcg(g.C + ((size_t)z * g.ny + y) * g.px + x), acc);
}

struct GenUpdate {
  __device__ __forceinline__ static float at(const GridDev& g, const float* u, int z, int y, int x) {
    return gen_update(g, u, z, y, x);
  }
};

// ------------------------------------------------------------ Theorem 1, any set

// entry (z, i) of a vector with nline entries per plane; outside the grid the rule is
// applied to the vector: a clamped or wrapped index, or a line of ncoll outside cells
__device__ __forceinline__ double gen_vec_at(const GridDev& g, const double* V, int nline, int ncoll, int z, int i) {
  if (!gen_map(z, g.nz, g.bc) || !gen_map(i, nline, g.bc)) return (double)ncoll * (double)gen_outside(g);
  return __ldcg(V + (size_t)z * nline + i);
}

// alpha of Theorem 1 for column x of plane z shifted by j along y: the cells shifted in
// from beyond the boundary minus the cells shifted out (read from u; zero without u)
__device__ __forceinline__ double gen_alpha(const GridDev& g, const float* u, int z, int x, int j) {
  double t = 0.0;
  if (j == 0 || u == nullptr) return t;
  if (j < 0) {
    for (int y = j; y <= -1; ++y) t = __dadd_rn(t, (double)gen_ghost(g, u, z, y, x));
    for (int y = g.ny + j; y <= g.ny - 1; ++y) t = __dadd_rn(t, -(double)gen_ghost(g, u, z, y, x));
  } else {
    for (int y = g.ny; y <= g.ny + j - 1; ++y) t = __dadd_rn(t, (double)gen_ghost(g, u, z, y, x));
    for (int y = 0; y <= j - 1; ++y) t = __dadd_rn(t, -(double)gen_ghost(g, u, z, y, x));
  }
  return t;
}

// beta: the same along x for row y of plane z
__device__ __forceinline__ double gen_beta(const GridDev& g, const float* u, int z, int y, int i) {
  double t = 0.0;
  if (i == 0 || u == nullptr) return t;
  if (i < 0) {
    for (int x = i; x <= -1; ++x) t = __dadd_rn(t, (double)gen_ghost(g, u, z, y, x));
    for (int x = g.nx + i; x <= g.nx - 1; ++x) t = __dadd_rn(t, -(double)gen_ghost(g, u, z, y, x));
  } else {
    for (int x = g.nx; x <= g.nx + i - 1; ++x) t = __dadd_rn(t, (double)gen_ghost(g, u, z, y, x));
    for (int x = 0; x <= i - 1; ++x) t = __dadd_rn(t, -(double)gen_ghost(g, u, z, y, x));
  }
  return t;
}

// Eq. (4): a'[z][x] = c_x + sum over S of w (a[z+k][x+i] + alpha), in the set's order
__device__ __forceinline__ double gen_predict_a(const GridDev& g, const double* A, const float* u, int z, int x) {
  const GenSten& s = *g.gs;
  double acc = 0.0;
  for (int k = 0; k < s.npts; ++k) {
    const int zz = z + s.dz[k], xx = x + s.dx[k];
    const double v = __dadd_rn(gen_vec_at(g, A, g.nx, g.ny, zz, xx), gen_alpha(g, u, zz, xx, s.dy[k]));
    acc = __dadd_rn(acc, __dmul_rn((double)s.w[k], v));
  }
  return __dadd_rn(__ldcg(g.cx + (size_t)z * g.nx + x), acc);
}

// Eq. (5) for b'[z][y]
__device__ __forceinline__ double gen_predict_b(const GridDev& g, const double* B, const float* u, int z, int y) {
  const GenSten& s = *g.gs;
  double acc = 0.0;
  for (int k = 0; k < s.npts; ++k) {
    const int zz = z + s.dz[k], yy = y + s.dy[k];
    const double v = __dadd_rn(gen_vec_at(g, B, g.ny, g.nx, zz, yy), gen_beta(g, u, zz, yy, s.dx[k]));
    acc = __dadd_rn(acc, __dmul_rn((double)s.w[k], v));
  }
  return __dadd_rn(__ldcg(g.cy + (size_t)z * g.ny + y), acc);
}

// ------------------------------------------------------------ the sweep

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_ahead() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// one value added to a column partial, in the accumulation's arithmetic
template <int ACC>
__device__ __forceinline__ void col_add(typename RowPart<ACC>::T& t, float v);
template <>
__device__ __forceinline__ void col_add<ABFT_ACC_FP32>(float& t, float v) { t += v; }
template <>
__device__ __forceinline__ void col_add<ABFT_ACC_TWOSUM>(float2& t, float v) { acc2(t.x, t.y, v); }
template <>
__device__ __forceinline__ void col_add<ABFT_ACC_FP64>(double& t, float v) { t += (double)v; }

template <int ACC>
__device__ __forceinline__ typename RowPart<ACC>::T col_zero() {
  return typename RowPart<ACC>::T{};
}

// Tiles of the general sweep: 128 x kGenTY (one row per warp).  A ring slot holds one
// staged plane of u (kGenTY + 2r rows by 136 columns) and the tile's plane of C
// (kGenTY rows by 128 columns); planes arrive kGenAhead iterations before they are
// needed, so the copies of two planes are in flight while the CTA computes.
constexpr int kGenAhead = 2;

__host__ __device__ constexpr int gen_slot_floats(int r) { return (kGenTY + 2 * r) * kGenW + kGenTY * kTX; }

template <int ACC, bool PROT>
__global__ void __launch_bounds__(kGenThreads, 2)
    k_sweep_gen(const GridDev g, const float* __restrict__ uin, float* __restrict__ uout, int r,
                DevCtrl* __restrict__ ctrl, DevSched sched) {
  using RP = RowPart<ACC>;
  using T = typename RP::T;
  extern __shared__ __align__(16) float ring[];
  __shared__ int s_off[kGenMaxPts];   // in-plane offset of each point: dy * kGenW + dx
  __shared__ int s_koff[kGenMaxPts];  // this plane's slot base plus s_off
  __shared__ float s_w[kGenMaxPts];
  __shared__ int4 lf[kLocalFlips];
  __shared__ int nlf;
  const int R = kGenTY + 2 * r, S = 2 * r + 1 + kGenAhead, PS = gen_slot_floats(r);
  T* colp = reinterpret_cast<T*>(ring + (size_t)S * PS);  // [8 warps][128 columns] of one plane
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const GenSten* gs = g.gs;
  const int npts = gs->npts;
  if (tid < npts) {
    s_off[tid] = gs->dy[tid] * kGenW + gs->dx[tid];
    s_w[tid] = gs->w[tid];
  }
  if (tid == 0) nlf = 0;
  sched.load(ctrl);
  const long long step = g.gc->step;
  const int txi = blockIdx.x % g.ntx, tyi = blockIdx.x / g.ntx;
  const int x0 = txi * kTX, y0 = tyi * kGenTY;
  __syncthreads();
  // this sweep's flips in the tile's output region (Sec. 5.1)
  if (sched.enabled) {
    const long long i = step - sched.t0;
    if (i >= 0 && i < sched.n)
      for (int k = sched.off[i] + tid; k < sched.off[i + 1]; k += kGenThreads) {
        const DevFlip f = sched.flips[k];
        if (f.grid == g.gid && f.target == 0 && f.x >= x0 && f.x < x0 + kTX && f.x < g.nx && f.y >= y0 &&
            f.y < y0 + kGenTY && f.y < g.ny && f.z >= 0 && f.z < g.nz) {
          const int j = atomicAdd(&nlf, 1);
          if (j < kLocalFlips) lf[j] = make_int4(f.x, f.y, f.z, f.bit & 31);
          else set_status(ctrl, kStFlipOverflow);
        }
      }
  }
  // plane p (possibly outside 0..nz-1) of u and, inside the grid, of C into its slot:
  // 16-byte copies where a chunk lies inside the grid, 4-byte copies of the cell the
  // rule maps an outside cell to (clamped, periodic), stores of the fixed value otherwise
  auto load_plane = [&](int p) {
    if (p <= g.nz - 1 + r) {
      float* dst = ring + (size_t)((p + r) % S) * PS;
      for (int c = tid; c < R * kGenChunks; c += kGenThreads) {
        const int row = c / kGenChunks, q = c - row * kGenChunks;
        const int gy = y0 - r + row, gx = x0 - kHaloX + 4 * q;
        float* d = dst + row * kGenW + 4 * q;
        if (p >= 0 && p < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx + 3 < g.nx) {
          cp_async16(d, uin + ((size_t)p * g.ny + gy) * g.px + gx);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            int zz = p, yy = gy, xx = gx + e;
            if (gen_map(zz, g.nz, g.bc) && gen_map(yy, g.ny, g.bc) && gen_map(xx, g.nx, g.bc))
              cp_async4(d + e, uin + ((size_t)zz * g.ny + yy) * g.px + xx);
            else
              d[e] = gen_outside(g);
          }
        }
      }
      if (p >= 0 && p < g.nz) {  // C of the tile's own points, one 16-byte chunk per thread
        float* dc = dst + R * kGenW;
        for (int c = tid; c < kGenTY * (kTX / 4); c += kGenThreads) {
          const int row = c / (kTX / 4), q = c - row * (kTX / 4);
          const int gy = y0 + row, gx = x0 + 4 * q;
          if (gy < g.ny && gx < g.nx) cp_async16(dc + row * kTX + 4 * q, g.C + ((size_t)p * g.ny + gy) * g.px + gx);
        }
      }
    }
    cp_async_commit();  // one group per plane, empty past the last one
  };
  for (int p = -r; p <= r + kGenAhead - 1; ++p) load_plane(p);
  __syncthreads();
  const int nf = min(nlf, kLocalFlips);
  T ca[4];
  const int row = warp, gy = y0 + row;
  for (int z = 0; z < g.nz; ++z) {
    if (tid < npts) s_koff[tid] = ((z + gs->dz[tid] + r) % S) * PS + s_off[tid];
    load_plane(z + r + kGenAhead);
    cp_async_wait_ahead();  // every plane up to z + r has landed
    __syncthreads();
    if (PROT && z > 0 && tid < kTX && x0 + tid < g.nx) {  // column partials of plane z-1
      T t = colp[tid];
#pragma unroll
      for (int w = 1; w < 8; ++w) t = RP::comb(t, colp[w * kTX + tid]);
      RP::store(g.PA, ((size_t)tyi * g.nz + (z - 1)) * g.pa_stride + x0 + tid, t);
    }
    const float* rb = ring + (row + r) * kGenW + lane + kHaloX;  // column lane + 32 j of this row
    float acc[4] = {0.f, 0.f, 0.f, 0.f};  // four independent FMA chains, one per column
    for (int k = 0; k < npts; ++k) {
      const float w = s_w[k];
      const float* q = rb + s_koff[k];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = __fmaf_rn(w, q[32 * j], acc[j]);
    }
    const float* cs = ring + (size_t)((z + r) % S) * PS + R * kGenW + row * kTX + lane;
    float* Urow = uout + ((size_t)z * g.ny + gy) * g.px;
    float m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gx = x0 + lane + 32 * j;
      float v = 0.f;
      if (gy < g.ny && gx < g.nx) {
        v = __fadd_rn(cs[32 * j], acc[j]);
        for (int f = 0; f < nf; ++f)
          if (lf[f].x == gx && lf[f].y == gy && lf[f].z == z) v = __int_as_float(__float_as_int(v) ^ (1 << lf[f].w));
        Urow[gx] = v;
      }
      m[j] = v;
      if (PROT) {
        ca[j] = col_zero<ACC>();
        col_add<ACC>(ca[j], v);
      }
    }
    if (PROT) {
      T t = RP::of(m);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = RP::comb(t, RP::shfl(t, o));
      if (lane == 0 && gy < g.ny) RP::store(g.PB, ((size_t)txi * g.nz + z) * g.pb_stride + gy, t);
    }
    __syncthreads();  // the slot of plane z - r and the column scratch are free again
    if (PROT) {
#pragma unroll
      for (int j = 0; j < 4; ++j) colp[warp * kTX + lane + 32 * j] = ca[j];
    }
  }
  cp_async_wait_0();
  __syncthreads();
  if (PROT && tid < kTX && x0 + tid < g.nx) {  // column partials of the last plane
    T t = colp[tid];
#pragma unroll
    for (int w = 1; w < 8; ++w) t = RP::comb(t, colp[w * kTX + tid]);
    RP::store(g.PA, ((size_t)tyi * g.nz + (g.nz - 1)) * g.pa_stride + x0 + tid, t);
  }
  if (tid == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&g.gc->done_sweep, 1u);
    if (ticket == gridDim.x - 1) {  // the last CTA commits the sweep
      g.gc->done_sweep = 0;
      g.gc->step = step + 1;
      __threadfence();
    }
  }
}

// ------------------------------------------------------------ check, location, chain

// One sweep's online check: reduce the partials into a^{t+1}, b^{t+1} (canonical
// order), interpolate from a^t, b^t and the boundary terms of u^t, compare.
template <int ACC>
__global__ void __launch_bounds__(256) k_check_gen(const GridDev g, int in, int out) {
  const int na = g.nz * g.nx, n = na + g.nz * g.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / g.nx, x = i - z * g.nx;
      const double s = reduce_a<ACC>(g, z, x);
      g.A[out][i] = s;
      const double p = gen_predict_a(g, g.A[in], g.u[in], z, x);
      g.AP[0][i] = p;
      if (fails(p, s, g.eps)) append_fail(g, z, 0, x);
      note_resid(g, p, s);
    } else {
      const int j = i - na;
      const int z = j / g.ny, y = j - z * g.ny;
      const double s = reduce_b<ACC>(g, z, y);
      g.B[out][j] = s;
      const double p = gen_predict_b(g, g.B[in], g.u[in], z, y);
      g.BP[0][j] = p;
      if (fails(p, s, g.eps)) append_fail(g, z, 1, y);
      note_resid(g, p, s);
    }
  }
}

// Location and correction, one block per plane with failing entries: Eq. (8) at a
// single intersection, otherwise the flagged lines recomputed from u[in] with the set S.
__global__ void __launch_bounds__(256)
    k_resolve_gen(const GridDev g, int in, int out, DevCtrl* ctrl, abft_event* ev, long long step) {
  __shared__ ResolveSmem sm;
  __shared__ int s_hit;
  for (int z = blockIdx.x; z < g.nz; z += gridDim.x) {
    if (threadIdx.x == 0) {
      s_hit = (__ldcg(&g.fcnt[2 * z]) | __ldcg(&g.fcnt[2 * z + 1])) != 0;
      sm.nfix = 0;
    }
    __syncthreads();
    const bool hit = s_hit != 0;
    __syncthreads();
    if (hit)
      resolve_plane<GenUpdate>(sm, g, g.u[in], g.u[out], g.A[out], g.B[out], g.AP[0], g.BP[0], step, ctrl, ev,
                               &g.gc->unresolved, z);
  }
}

// One link of a chain of Theorem 1 (Fig. 10): predictions from predictions, with the
// boundary terms of the state u the step starts from (u == nullptr: terms vanish).
__global__ void __launch_bounds__(256)
    k_chain_gen(const GridDev g, const double* a_in, const double* b_in, const float* u, double* a_out,
                double* b_out) {
  const int na = g.nz * g.nx, n = na + g.nz * g.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < na) {
      const int z = i / g.nx, x = i - z * g.nx;
      a_out[i] = gen_predict_a(g, a_in, u, z, x);
    } else {
      const int j = i - na;
      const int z = j / g.ny, y = j - z * g.ny;
      b_out[j] = gen_predict_b(g, b_in, u, z, y);
    }
  }
}

// ------------------------------------------------------------ launchers

int gen_sweep_smem(const GridDev& g, int r) {
  const int S = 2 * r + 1 + kGenAhead;
  return S * gen_slot_floats(r) * (int)sizeof(float) + 8 * kTX * (g.acc == ABFT_ACC_FP32 ? 4 : 8);
}

template <int ACC, bool PROT>
static cudaError_t sweep_gen_as(const Launch& L, const GridDev& g, int r, int in, int out) {
  const int smem = gen_sweep_smem(g, r);
  cudaError_t e = cudaFuncSetAttribute(k_sweep_gen<ACC, PROT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_sweep_gen<ACC, PROT><<<g.ntx * g.nty, kGenThreads, smem, L.s>>>(g, g.u[in], g.u[out], r, L.ctrl, L.sched);
  return cudaGetLastError();
}

cudaError_t launch_sweep_gen(const Launch& L, const GridDev& g, int r, int in, int out, bool prot) {
  if (r < 0 || r > kGenRadius || g.ty != kGenTY) return cudaErrorInvalidValue;
  if (!prot) return sweep_gen_as<ABFT_ACC_FP32, false>(L, g, r, in, out);
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: return sweep_gen_as<ABFT_ACC_TWOSUM, true>(L, g, r, in, out);
    case ABFT_ACC_FP64: return sweep_gen_as<ABFT_ACC_FP64, true>(L, g, r, in, out);
    default: return sweep_gen_as<ABFT_ACC_FP32, true>(L, g, r, in, out);
  }
}

static int gen_blocks(const GridDev& g) {
  const long long n = (long long)g.nz * (g.nx + g.ny);
  long long b = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(b, 8 * 152));
}

cudaError_t launch_check_gen(const Launch& L, const GridDev& g, int in, int out) {
  switch (g.acc) {
    case ABFT_ACC_TWOSUM: k_check_gen<ABFT_ACC_TWOSUM><<<gen_blocks(g), 256, 0, L.s>>>(g, in, out); break;
    case ABFT_ACC_FP64: k_check_gen<ABFT_ACC_FP64><<<gen_blocks(g), 256, 0, L.s>>>(g, in, out); break;
    default: k_check_gen<ABFT_ACC_FP32><<<gen_blocks(g), 256, 0, L.s>>>(g, in, out); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_resolve_gen(const Launch& L, const GridDev& g, int in, int out, long long step) {
  k_resolve_gen<<<std::min(g.nz, 1024), 256, 0, L.s>>>(g, in, out, L.ctrl, L.events, step);
  return cudaGetLastError();
}

cudaError_t launch_chain_gen(const Launch& L, const GridDev& g, const double* a_in, const double* b_in,
                             const float* u, double* a_out, double* b_out) {
  k_chain_gen<<<gen_blocks(g), 256, 0, L.s>>>(g, a_in, b_in, u, a_out, b_out);
  return cudaGetLastError();
}

}  // namespace abft
