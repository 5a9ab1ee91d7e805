// One tile of the stencil sweep of Eq. (1) with the per-plane checksums of Eq. (2)/(3)
// fused into its epilogue (Sec. 3.2) and the flip-injection hook of Sec. 5.1.
//
// A CTA owns a 128 x TY column of the grid and streams it along z.  Plane tiles
// (with a one-cell y halo and a 4-cell, 16-byte aligned x halo) and the matching
// tiles of the constant term C are staged into a ring of S shared-memory stages by
// TMA, one mbarrier per stage.  Every thread computes one float4 of each of its
// rows; all seven neighbours come from shared memory, the x neighbours across
// float4 boundaries by warp shuffles.  Clamped boundaries (Fig. 2) are selects on
// the grid edges, since TMA fills out-of-range cells with zeros.
//
// The checksum epilogue sums exactly the stored values (after injection):
//   b[z][y] partial: the row's 128 values, warp-shuffle reduction;
//   a[z][x] partial: the tile's TY values per column, in registers per warp, then
//                    one pass over shared memory by 128 threads (one per column).
// Partials are written per tile and reduced across tiles in a fixed order by the
// check, so results are bitwise repeatable.
#pragma once

#include "device_common.cuh"

namespace abft {

// The tile code runs on the first kSweepThreads threads of a block and synchronises
// them with named barrier 1, so that other warps of the block (the persistent online
// kernel's check warp) can run independently.
constexpr int kSweepThreads = 256;
__device__ __forceinline__ void tile_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kSweepThreads) : "memory"); }

// row pitch (floats) of the FP32 epilogue's lane partials: 36 keeps the 16-byte
// loads of eight consecutive rows on distinct banks
constexpr int kRowPitch = 36;

template <int TY>
struct SweepCfg {
  static constexpr int NW = 8;                        // warps per CTA
  static constexpr int S = TY <= 8 ? 6 : (TY <= 16 ? 5 : 4);  // ring depth (>= 4)
  static constexpr int RPW = TY / NW;                 // rows per warp
  static constexpr int UBOX = (TY + 2) * kUW * 4;     // bytes of a staged u box
  static constexpr int UBOX_AL = (UBOX + 127) / 128 * 128;
  static constexpr int CBOX = TY * kTX * 4;
  static constexpr int STAGE = UBOX_AL + CBOX;        // multiple of 128
  // one z-parity of the reduction buffer: column partials [NW][kTX] (8-byte sums), or
  // for FP32 column partials [NW][kTX] then row lane partials [TY][kRowPitch]
  static constexpr int RED_HALF_A = NW * kTX * 8, RED_HALF_B = NW * kTX * 4 + TY * kRowPitch * 4;
  static constexpr int RED_HALF = ((RED_HALF_A > RED_HALF_B ? RED_HALF_A : RED_HALF_B) + 127) / 128 * 128;
  static constexpr int RED = 2 * RED_HALF;
  static constexpr int FLIPS = kLocalFlips * 16 + 16;
  static constexpr int SMEM = 128 + 128 + S * STAGE + RED + FLIPS;  // + slack to align the base
  static_assert(TY % NW == 0, "TY must be a multiple of the warp count");
  static_assert(S >= 4, "the ring must hold z-1, z, z+1 and one load in flight");
};

// ------------------------------------------------------------ accumulators
// Per-thread column partials over this thread's rows (4 columns), their exchange
// through shared memory (layout [warp][column]) and the row partial of one row.

template <int ACC>
struct AccA;

template <>
struct AccA<ABFT_ACC_FP32> {
  float v[4];
  __device__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.f; }
  __device__ void add(const float (&m)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] += m[i];
  }
  __device__ void put(unsigned char* red, int warp, int lane) const {
    reinterpret_cast<float4*>(red)[warp * 32 + lane] = make_float4(v[0], v[1], v[2], v[3]);
  }
  __device__ void store4(void* PA, size_t idx) const {  // this lane's 4 columns, directly
    *reinterpret_cast<float4*>(static_cast<float*>(PA) + idx) = make_float4(v[0], v[1], v[2], v[3]);
  }
  // column c summed over the NW warp partials, written as partial PA[idx]
  template <int NW>
  __device__ static void column_store(const unsigned char* red, int c, void* PA, size_t idx) {
    const float* r = reinterpret_cast<const float*>(red);
    float s = r[c];
#pragma unroll
    for (int w = 1; w < NW; ++w) s += r[w * kTX + c];
    static_cast<float*>(PA)[idx] = s;
  }
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
  __device__ void put(unsigned char* red, int warp, int lane) const {
    float4* p = reinterpret_cast<float4*>(red);
    p[warp * 32 + lane] = make_float4(h[0], h[1], h[2], h[3]);
    p[8 * 32 + warp * 32 + lane] = make_float4(l[0], l[1], l[2], l[3]);  // lo half after 8 warps
  }
  __device__ void store4(void* PA, size_t idx) const {
    float4* p = reinterpret_cast<float4*>(static_cast<float2*>(PA) + idx);
    p[0] = make_float4(h[0], l[0], h[1], l[1]);
    p[1] = make_float4(h[2], l[2], h[3], l[3]);
  }
  template <int NW>
  __device__ static void column_store(const unsigned char* red, int c, void* PA, size_t idx) {
    const float* r = reinterpret_cast<const float*>(red);
    float hi = r[c], lo = r[8 * kTX + c];
#pragma unroll
    for (int w = 1; w < NW; ++w) {
      acc2(hi, lo, r[w * kTX + c]);
      lo += r[8 * kTX + w * kTX + c];
    }
    static_cast<float2*>(PA)[idx] = make_float2(hi, lo);
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
  __device__ void put(unsigned char* red, int warp, int lane) const {
    double2* p = reinterpret_cast<double2*>(red) + (warp * 32 + lane) * 2;
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
  }
  __device__ void store4(void* PA, size_t idx) const {
    double2* p = reinterpret_cast<double2*>(static_cast<double*>(PA) + idx);
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
  }
  template <int NW>
  __device__ static void column_store(const unsigned char* red, int c, void* PA, size_t idx) {
    const double* r = reinterpret_cast<const double*>(red);
    double s = r[c];
#pragma unroll
    for (int w = 1; w < NW; ++w) s += r[w * kTX + c];
    static_cast<double*>(PA)[idx] = s;
  }
  __device__ static void row_store(const float (&m)[4], void* PB, size_t idx, bool write) {
    double r = (((double)m[0] + (double)m[1]) + (double)m[2]) + (double)m[3];
    r = warp_sum(r);
    if (write) static_cast<double*>(PB)[idx] = r;
  }
};

// --------------------------------------------- multi-row reduction of row partials
// R rows (R = 2, 4, 8 or 16) held by every lane of a warp, one lane-partial per row, are
// reduced to R row totals with log2(R) halving exchanges (offsets 16, 8, ...) and
// butterfly exchanges for the remaining offsets.  Every stage pairs lanes l and l^o,
// the same pairs, in the same stage order, as the per-row butterfly of row_store, and
// each stage's addition is commutative, so every row total is bit-identical to
// row_store's.  Lane l ends holding row (l >> (5 - log2 R)).
template <int ACC>
struct RowPart;
template <>
struct RowPart<ABFT_ACC_FP32> {
  using T = float;
  __device__ static T of(const float (&m)[4]) { return ((m[0] + m[1]) + m[2]) + m[3]; }
  __device__ static T comb(T a, T b) { return a + b; }
  __device__ static T shfl(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  __device__ static void store(void* PB, size_t i, T v) { static_cast<float*>(PB)[i] = v; }
};
template <>
struct RowPart<ABFT_ACC_TWOSUM> {
  using T = float2;
  __device__ static T of(const float (&m)[4]) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc2(hi, lo, m[i]);
    return make_float2(hi, lo);
  }
  __device__ static T comb(T a, T b) {  // as warp_sum2: two_sum(a.hi, b.hi), lo = a.lo + b.lo + e
    float s, e;
    two_sum(a.x, b.x, s, e);
    return make_float2(s, a.y + b.y + e);
  }
  __device__ static T shfl(T v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
  }
  __device__ static void store(void* PB, size_t i, T v) { static_cast<float2*>(PB)[i] = v; }
};
template <>
struct RowPart<ABFT_ACC_FP64> {
  using T = double;
  __device__ static T of(const float (&m)[4]) { return (((double)m[0] + (double)m[1]) + (double)m[2]) + (double)m[3]; }
  __device__ static T comb(T a, T b) { return a + b; }
  __device__ static T shfl(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  __device__ static void store(void* PB, size_t i, T v) { static_cast<double*>(PB)[i] = v; }
};

template <int ACC, int R>
__device__ __forceinline__ typename RowPart<ACC>::T reduce_rows(typename RowPart<ACC>::T (&v)[R], int lane) {
  using RP = RowPart<ACC>;
  static_assert(R == 2 || R == 4 || R == 8 || R == 16, "row count");
  constexpr int L = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));  // halving stages
  int cnt = R;
#pragma unroll
  for (int st = 0; st < L; ++st) {
    const int o = 16 >> st;
    const bool up = (lane & o) != 0;  // keeps the upper half of its current rows
    cnt >>= 1;
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      if (i < cnt) {
        const typename RP::T send = up ? v[i] : v[i + cnt];
        const typename RP::T keep = up ? v[i + cnt] : v[i];
        v[i] = RP::comb(keep, RP::shfl(send, o));
      }
    }
  }
  typename RP::T t = v[0];
#pragma unroll
  for (int o = 16 >> L; o > 0; o >>= 1) t = RP::comb(t, RP::shfl(t, o));
  return t;
}

// shared-memory layout of the sweep
template <int TY>
struct SweepSmem {
  uint64_t* bar;
  unsigned char* stages;
  unsigned char* red;
  int4* lflips;
  int* nlf;
  __device__ static SweepSmem carve(unsigned char* raw) {
    using Cfg = SweepCfg<TY>;
    SweepSmem m;
    unsigned char* s = raw + ((128 - (smem_u32(raw) & 127)) & 127);  // TMA needs 128-byte alignment
    m.bar = reinterpret_cast<uint64_t*>(s);
    m.stages = s + 128;
    m.red = m.stages + Cfg::S * Cfg::STAGE;
    m.lflips = reinterpret_cast<int4*>(m.red + Cfg::RED);
    m.nlf = reinterpret_cast<int*>(m.lflips + kLocalFlips);
    return m;
  }
  __device__ float* stage_u(int s) const { return reinterpret_cast<float*>(stages + s * SweepCfg<TY>::STAGE); }
  __device__ float* stage_c(int s) const {
    return reinterpret_cast<float*>(stages + s * SweepCfg<TY>::STAGE + SweepCfg<TY>::UBOX_AL);
  }
  // thread 0 only, once per CTA
  __device__ void init_barriers() const {
    for (int s = 0; s < SweepCfg<TY>::S; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
};

// One tile (txi, tyi) of one sweep, u_in -> uout, in two halves: sweep_tile_issue()
// starts the TMA loads and gathers the tile's flips, sweep_tile_run() streams the
// planes.  Work that does not touch the ring (the persistent kernel's check) may run
// between the two.  `seq` counts the plane loads this CTA has issued so far
// (identical in every thread); the k-th load uses stage k % S with mbarrier phase
// parity (k / S) & 1.  `pbuf` selects the partial-checksum buffers (PA/PB or
// PA2/PB2).  Every thread must call both halves; the ring is idle before and after.
template <int TY>
__device__ __forceinline__ void sweep_tile_issue(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g,
                                                 int txi, int tyi, long long step, DevCtrl* __restrict__ ctrl,
                                                 const DevSched& sched, const SweepSmem<TY>& sm, unsigned seq) {
  using Cfg = SweepCfg<TY>;
  constexpr int S = Cfg::S;
  const int tid = threadIdx.x;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz;
  if (tid == 0) {
    fence_proxy_async_global();  // grid data written by the generic proxy before TMA reads it
    const int np = nz < S ? nz : S;
    for (int p = 0; p < np; ++p) {
      const int s = (int)((seq + p) % S);
      mbar_expect_tx(&sm.bar[s], Cfg::UBOX + Cfg::CBOX);
      tma_load_3d(sm.stage_u(s), tm_u, x0 - kHaloX, y0 - 1, p, &sm.bar[s]);
      tma_load_3d(sm.stage_c(s), tm_c, x0, y0, p, &sm.bar[s]);
    }
    *sm.nlf = 0;
  }
  tile_sync();
  // flips of this sweep that land in this tile (Sec. 5.1: after the update, before the store)
  if (sched.enabled) {
    const long long i = step - sched.t0;
    if (i >= 0 && i < sched.n) {
      const int b = sched.off[i], e = sched.off[i + 1];
      for (int k = b + tid; k < e; k += kSweepThreads) {
        const DevFlip f = sched.flips[k];
        if (f.grid == g.gid && f.target == 0 && f.x >= x0 && f.x < x0 + kTX && f.x < g.nx && f.y >= y0 &&
            f.y < y0 + TY && f.y < g.ny && f.z >= 0 && f.z < nz && f.x >= 0 && f.y >= 0) {
          const int j = atomicAdd(sm.nlf, 1);
          if (j < kLocalFlips) sm.lflips[j] = make_int4(f.x, f.y, f.z, f.bit & 31);
          else set_status(ctrl, kStFlipOverflow);
        }
      }
    }
  }
  tile_sync();
}

// Neighbours of a thread's four points (x = gx0 .. gx0 + 3 of row y, plane z) that
// lie outside the grid, by the boundary rule.  On entry they hold what the staged tile
// has there: TMA fills out-of-range cells with zeros, and at a z face the caller passes
// the centre plane (or, for whole-column tiles, the opposite face when it is staged).
//   clamped (Fig. 2): the centre value;
//   empty (zero): the in-plane zero fill is already right, the z faces become zero;
//   periodic: the opposite face, read from the input grid in global memory (through
//   L2: it was written by other CTAs in this launch or the previous one).
// Periodic boundaries: the opposite faces' values one row needs -- the wrapped x
// neighbours of its first and last points and, on a y face, the row on the other face
// -- loaded by wrap_row ahead of the row's computation (streaming tiles: one plane
// ahead) so that the latency of these global loads is hidden; `pre` says they were.
struct WrapRow {
  float xw, xe;  // u at x = nx - 1 (for the point x = 0) and at x = 0 (for x = nx - 1)
  float4 yf;     // the row on the other y face (rows y = 0 and y = ny - 1)
};

__device__ __forceinline__ WrapRow wrap_row(const GridDev& g, const float* __restrict__ uin, int z, int y, int gx0,
                                            int last) {
  WrapRow w{0.f, 0.f, make_float4(0.f, 0.f, 0.f, 0.f)};
  if (y >= g.ny || last < 0) return w;
  const float* row = uin + ((size_t)z * g.ny + y) * g.px;
  if (gx0 == 0) w.xw = __ldcg(row + g.nx - 1);
  if (last <= 3) w.xe = __ldcg(row);
  if (y == 0) w.yf = __ldcg(reinterpret_cast<const float4*>(row + (size_t)(g.ny - 1) * g.px + gx0));
  else if (y == g.ny - 1) w.yf = __ldcg(reinterpret_cast<const float4*>(row - (size_t)(g.ny - 1) * g.px + gx0));
  return w;
}

// BC: the rule (abft_boundary), fixed at compile time.
template <bool Z_STAGED, int BC>
__device__ __forceinline__ void boundary_cells(const GridDev& g, const float* __restrict__ uin, int z, int y, int gx0,
                                               int last, const float4& c, float4& n, float4& s, float4& b, float4& t,
                                               float& w0, float& e0, float& e1, float& e2, float& e3,
                                               const WrapRow* pre = nullptr) {
  if (BC == ABFT_BC_CLAMP) {
    if (y == 0) n = c;
    if (y == g.ny - 1) s = c;
    if (gx0 == 0) w0 = c.x;
    if (last == 0) e0 = c.x;
    if (last == 1) e1 = c.y;
    if (last == 2) e2 = c.z;
    if (last == 3) e3 = c.w;
    return;
  }
  if (BC == ABFT_BC_ZERO) {
    if (z == 0) b = make_float4(0.f, 0.f, 0.f, 0.f);
    if (z == g.nz - 1) t = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  if (y >= g.ny || last < 0) return;  // no grid point among the four (gx0 < nx keeps the loads in the row)
  const size_t plane = (size_t)g.ny * g.px;
  const float* row = uin + (size_t)z * plane + (size_t)y * g.px;
  const WrapRow w = pre != nullptr ? *pre : wrap_row(g, uin, z, y, gx0, last);
  if (y == 0) n = w.yf;
  if (y == g.ny - 1) s = w.yf;  // for ny = 1 both wrap to the row itself
  if (gx0 == 0) w0 = w.xw;
  if (last == 0) e0 = w.xe;
  if (last == 1) e1 = w.xe;
  if (last == 2) e2 = w.xe;
  if (last == 3) e3 = w.xe;
  if (!Z_STAGED) {
    if (z == 0) b = __ldcg(reinterpret_cast<const float4*>(row + (size_t)(g.nz - 1) * plane + gx0));
    if (z == g.nz - 1) t = __ldcg(reinterpret_cast<const float4*>(row - (size_t)(g.nz - 1) * plane + gx0));
  }
}

// VEC: checksum vectors of the epilogue (2: a and b partials; 1: b partials only, for
// the one-vector online check of Sec. 3.2)
template <int TY, bool PROT, int ACC, int BC, int VEC = 2>
__device__ __forceinline__ void sweep_tile_run(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g,
                                               const float* __restrict__ uin, float* __restrict__ uout, int txi, int tyi,
                                               DevCtrl* __restrict__ ctrl, const SweepSmem<TY>& sm, unsigned& seq,
                                               int pbuf) {
  using Cfg = SweepCfg<TY>;
  constexpr int S = Cfg::S, NW = Cfg::NW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz;
  const unsigned base = seq;
  void* PA = pbuf ? g.PA2 : g.PA;
  void* PB = pbuf ? g.PB2 : g.PB;
  auto issue = [&](int p) {  // TMA loads of plane p of this tile (thread 0 only)
    const int s = (int)((base + p) % S);
    mbar_expect_tx(&sm.bar[s], Cfg::UBOX + Cfg::CBOX);
    tma_load_3d(sm.stage_u(s), tm_u, x0 - kHaloX, y0 - 1, p, &sm.bar[s]);
    tma_load_3d(sm.stage_c(s), tm_c, x0, y0, p, &sm.bar[s]);
  };
  auto wait = [&](int p) {
    const unsigned k = base + (unsigned)p;
    mbar_wait(&sm.bar[k % S], (k / S) & 1u, ctrl);
  };
  const int nflip = min(*sm.nlf, kLocalFlips);
  const int gx0 = x0 + 4 * lane;
  const int last = g.nx - 1 - gx0;  // element holding x = nx-1, if 0..3
  const bool full = x0 + kTX <= g.nx && y0 + TY <= g.ny;  // no ragged edge in this tile
  // FP32 partials: lane partials through shared memory, reduced by one warp per plane
  constexpr bool SMEM_EPI = ACC == ABFT_ACC_FP32;
  constexpr bool PA_ON = PROT && VEC == 2;  // column partials (the a vector)
  static_assert(NW * kTX * 4 + TY * kRowPitch * 4 <= Cfg::RED_HALF, "FP32 epilogue buffer");
  // periodic: the wrapped face values of this warp's rows, for this plane and the next
  constexpr bool WRAP = BC == ABFT_BC_PERIODIC;
  WrapRow wcur[WRAP ? Cfg::RPW : 1], wnxt[WRAP ? Cfg::RPW : 1];
  if (WRAP)
#pragma unroll
    for (int rr = 0; rr < Cfg::RPW; ++rr) wcur[rr] = wrap_row(g, uin, 0, y0 + warp + rr * NW, gx0, last);

  for (int z = 0; z < nz; ++z) {
    if (WRAP && z + 1 < nz)
#pragma unroll
      for (int rr = 0; rr < Cfg::RPW; ++rr) wnxt[rr] = wrap_row(g, uin, z + 1, y0 + warp + rr * NW, gx0, last);
    if (z == 0) wait(0);
    if (z + 1 < nz) wait(z + 1);
    const float* Uc = sm.stage_u((int)((base + z) % S));
    const float* Ub = z > 0 ? sm.stage_u((int)((base + z - 1) % S)) : Uc;
    const float* Ut = z + 1 < nz ? sm.stage_u((int)((base + z + 1) % S)) : Uc;
    const float* Cs = sm.stage_c((int)((base + z) % S));
    unsigned char* red = sm.red + (z & 1) * Cfg::RED_HALF;
    float* rowp = reinterpret_cast<float*>(red + NW * kTX * 4);  // FP32 epilogue: [TY][kRowPitch] lane partials
    AccA<ACC> acc;
    if (PA_ON) acc.zero();
    typename RowPart<ACC>::T rp[Cfg::RPW > 1 ? Cfg::RPW : 2];
#pragma unroll
    for (int rr = 0; rr < Cfg::RPW; ++rr) {
      const int r = warp + rr * NW;
      const int y = y0 + r;
      const int o = (r + 1) * kUW + kHaloX + 4 * lane;
      const float4 c = *reinterpret_cast<const float4*>(Uc + o);
      float4 n = *reinterpret_cast<const float4*>(Uc + o - kUW);
      float4 s = *reinterpret_cast<const float4*>(Uc + o + kUW);
      float4 b = *reinterpret_cast<const float4*>(Ub + o);
      float4 t = *reinterpret_cast<const float4*>(Ut + o);
      const float4 cs = *reinterpret_cast<const float4*>(Cs + r * kTX + 4 * lane);
      float wl = __shfl_up_sync(0xffffffffu, c.w, 1);
      float er = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (lane == 0) wl = Uc[o - 1];
      if (lane == 31) er = Uc[o + 4];
      float w0 = wl;
      float e0 = c.y, e1 = c.z, e2 = c.w, e3 = er;
      boundary_cells<false, BC>(g, uin, z, y, gx0, last, c, n, s, b, t, w0, e0, e1, e2, e3,
                                WRAP ? &wcur[WRAP ? rr : 0] : nullptr);
      float v[4];
      v[0] = hs_update(g.k, c.x, w0, e0, n.x, s.x, b.x, t.x, cs.x);
      v[1] = hs_update(g.k, c.y, c.x, e1, n.y, s.y, b.y, t.y, cs.y);
      v[2] = hs_update(g.k, c.z, c.y, e2, n.z, s.z, b.z, t.z, cs.z);
      v[3] = hs_update(g.k, c.w, c.z, e3, n.w, s.w, b.w, t.w, cs.w);
      if (nflip > 0) {
        for (int f = 0; f < nflip; ++f) {
          const int4 q = sm.lflips[f];
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
        for (int i = 0; i < 4; ++i) m[i] = full ? v[i] : ((yv && i <= last) ? v[i] : 0.f);
        if (SMEM_EPI) rowp[r * kRowPitch + lane] = ((m[0] + m[1]) + m[2]) + m[3];  // RowPart<FP32>::of
        else if (Cfg::RPW == 1) AccA<ACC>::row_store(m, PB, ((size_t)txi * nz + z) * g.pb_stride + y, yv && lane == 0);
        else rp[rr] = RowPart<ACC>::of(m);
        if (PA_ON) acc.add(m);
      }
    }
    if (PROT && !SMEM_EPI && Cfg::RPW > 1) {  // this warp's rows reduced together; lane (rr << SH) holds row rr
      constexpr int SH = Cfg::RPW == 2 ? 4 : (Cfg::RPW == 4 ? 3 : 2);
      const typename RowPart<ACC>::T tot = reduce_rows<ACC, (Cfg::RPW > 1 ? Cfg::RPW : 2)>(rp, lane);
      const int y = y0 + warp + (lane >> SH) * NW;
      if ((lane & ((1 << SH) - 1)) == 0 && y < g.ny)
        RowPart<ACC>::store(PB, ((size_t)txi * nz + z) * g.pb_stride + y, tot);
    }
    if (PA_ON) acc.put(sm.red + (z & 1) * Cfg::RED_HALF, warp, lane);
    tile_sync();
    if (tid == 0 && z >= 1 && z - 1 + S < nz) {
      fence_proxy_async();
      issue(z - 1 + S);
    }
    if (PROT && SMEM_EPI) {
      // two warps per plane (rotating with z) reduce the plane's partials: one sums four
      // columns per lane over the eight warps in order, the other row `lane` over its 32
      // lane partials by the butterfly's own pairing (the same sums as row_store)
      if (PA_ON && warp == (z & (NW - 1))) {
        const float* r = reinterpret_cast<const float*>(red);
        float4 c = reinterpret_cast<const float4*>(r)[lane];
#pragma unroll
        for (int w = 1; w < NW; ++w) {
          const float4 q = reinterpret_cast<const float4*>(r + w * kTX)[lane];
          c.x += q.x; c.y += q.y; c.z += q.z; c.w += q.w;
        }
        *reinterpret_cast<float4*>(static_cast<float*>(PA) + ((size_t)tyi * nz + z) * g.pa_stride + x0 + 4 * lane) = c;
      }
      if (warp == ((z + NW / 2) & (NW - 1))) {
        if (lane < TY && y0 + lane < g.ny) {
          float t[32];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float4 q = reinterpret_cast<const float4*>(rowp + lane * kRowPitch)[k];
            t[4 * k] = q.x; t[4 * k + 1] = q.y; t[4 * k + 2] = q.z; t[4 * k + 3] = q.w;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int l = 0; l < o; ++l) t[l] = t[l] + t[l + o];
          static_cast<float*>(PB)[((size_t)txi * nz + z) * g.pb_stride + y0 + lane] = t[0];
        }
      }
    } else if (PA_ON && tid < kTX) {
      AccA<ACC>::template column_store<NW>(sm.red + (z & 1) * Cfg::RED_HALF, tid, PA,
                                           ((size_t)tyi * nz + z) * g.pa_stride + x0 + tid);
    }
    if (WRAP)
#pragma unroll
      for (int rr = 0; rr < Cfg::RPW; ++rr) wcur[rr] = wnxt[rr];
  }
  seq = base + (unsigned)nz;
  fence_proxy_async_global();  // this thread's grid stores, before any later TMA read of them
  tile_sync();             // the ring and the reduction buffer are idle again
}

// flips of sweep `step` at point (z, y, x), applied to v exactly as the sweep does
static __device__ __forceinline__ float reapply_flips(float v, const GridDev& g, DevCtrl* ctrl, const DevSched& sched,
                                               long long step, int z, int y, int x) {
  (void)ctrl;
  if (!sched.enabled) return v;
  const long long i = step - sched.t0;
  if (i < 0 || i >= sched.n) return v;
  for (int k = sched.off[i]; k < sched.off[i + 1]; ++k) {
    const DevFlip f = sched.flips[k];
    if (f.grid == g.gid && f.target == 0 && f.z == z && f.y == y && f.x == x)
      v = __int_as_float(__float_as_int(v) ^ (1 << (f.bit & 31)));
  }
  return v;
}

// ------------------------------------------------- partials, recomputed exactly
// The same arithmetic, in the same order, as the sweep epilogue above, for one
// column (a-partial) or one row (b-partial, one full warp) of one tile.  Used when
// a repaired grid must yield the partials the sweep would have produced.

template <int TY, int ACC>
__device__ void recompute_pa(const GridDev& g, const float* __restrict__ u, void* PA, int tyi, int z, int x) {
  constexpr int NW = SweepCfg<TY>::NW, RPW = SweepCfg<TY>::RPW;
  const int y0 = tyi * TY;
  auto val = [&](int r) -> float {
    const int y = y0 + r;
    return (y < g.ny && x < g.nx) ? __ldcg(u + ((size_t)z * g.ny + y) * g.px + x) : 0.f;
  };
  const size_t idx = ((size_t)tyi * g.nz + z) * g.pa_stride + x;
  if (ACC == ABFT_ACC_FP32) {
    float s = 0.f;
    for (int w = 0; w < NW; ++w) {
      float a = 0.f;
      for (int rr = 0; rr < RPW; ++rr) a += val(w + rr * NW);
      s = w == 0 ? a : s + a;
    }
    static_cast<float*>(PA)[idx] = s;
  } else if (ACC == ABFT_ACC_TWOSUM) {
    float hi = 0.f, lo = 0.f;
    for (int w = 0; w < NW; ++w) {
      float h = 0.f, l = 0.f;
      for (int rr = 0; rr < RPW; ++rr) acc2(h, l, val(w + rr * NW));
      if (w == 0) {
        hi = h;
        lo = l;
      } else {
        acc2(hi, lo, h);
        lo += l;
      }
    }
    static_cast<float2*>(PA)[idx] = make_float2(hi, lo);
  } else {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) {
      double a = 0.0;
      for (int rr = 0; rr < RPW; ++rr) a += (double)val(w + rr * NW);
      s = w == 0 ? a : s + a;
    }
    static_cast<double*>(PA)[idx] = s;
  }
}

// one full warp: the b-partial of row y of tile txi in plane z
template <int ACC>
__device__ void recompute_pb(const GridDev& g, const float* __restrict__ u, void* PB, int txi, int z, int y) {
  const int lane = threadIdx.x & 31;
  const int gx0 = txi * kTX + 4 * lane;
  float m[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    m[i] = (y < g.ny && gx0 + i < g.nx) ? __ldcg(u + ((size_t)z * g.ny + y) * g.px + gx0 + i) : 0.f;
  AccA<ACC>::row_store(m, PB, ((size_t)txi * g.nz + z) * g.pb_stride + y, lane == 0);
}

// ======================================================= shallow grids (nz <= kShallowMaxZ)
// The whole column of a tile (all nz planes) is staged at once by one TMA box for u
// (y halo of one row, x halo of 4) and one for C, signalled by one mbarrier.  Warp w
// computes planes w, w + 8, ...; within a plane it walks the TY rows, so the a-partial
// of each of its columns stays in registers (summed over rows in order) and no
// cross-warp exchange or per-plane barrier is needed.  A persistent CTA that owns a
// single tile keeps C resident and reloads only u.

template <int TY>
struct ShallowCfg {
  static constexpr int NW = 8;
  static constexpr int UROW = kUW * 4;                            // bytes of one staged u row
  static constexpr int CROW = kTX * 4;
  static constexpr int FLIPS = kLocalFlips * 16 + 16;
  __host__ __device__ static int ubox(int nz) { return nz * (TY + 2) * UROW; }
  __host__ __device__ static int ubox_al(int nz) { return (ubox(nz) + 127) / 128 * 128; }
  __host__ __device__ static int cbox(int nz) { return nz * TY * CROW; }
  __host__ __device__ static int smem(int nz) { return 128 + 128 + ubox_al(nz) + cbox(nz) + FLIPS; }
};

template <int TY>
struct ShallowSmem {
  uint64_t* bar;
  float* u;
  float* c;
  int4* lflips;
  int* nlf;
  __device__ static ShallowSmem carve(unsigned char* raw, int nz) {
    ShallowSmem m;
    unsigned char* s = raw + ((128 - (smem_u32(raw) & 127)) & 127);
    m.bar = reinterpret_cast<uint64_t*>(s);
    m.u = reinterpret_cast<float*>(s + 128);
    m.c = reinterpret_cast<float*>(s + 128 + ShallowCfg<TY>::ubox_al(nz));
    m.lflips = reinterpret_cast<int4*>(s + 128 + ShallowCfg<TY>::ubox_al(nz) + ShallowCfg<TY>::cbox(nz));
    m.nlf = reinterpret_cast<int*>(m.lflips + kLocalFlips);
    return m;
  }
  __device__ void init_barriers() const {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
};

// One shallow tile of one sweep, in two halves like the streaming tile: the issue half
// starts the TMA loads (C too when load_c; otherwise C is already resident) and
// gathers the flips; the run half waits for the loads (mbarrier phase parity `phase`,
// toggled) and computes.  Every thread must call both.
template <int TY>
__device__ __forceinline__ void shallow_tile_issue(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g,
                                                   int txi, int tyi, long long step, DevCtrl* __restrict__ ctrl,
                                                   const DevSched& sched, const ShallowSmem<TY>& sm, bool load_c) {
  using Cfg = ShallowCfg<TY>;
  const int tid = threadIdx.x;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz;
  if (tid == 0) {
    fence_proxy_async_global();
    mbar_expect_tx(sm.bar, Cfg::ubox(nz) + (load_c ? Cfg::cbox(nz) : 0));
    tma_load_3d(sm.u, tm_u, x0 - kHaloX, y0 - 1, 0, sm.bar);
    if (load_c) tma_load_3d(sm.c, tm_c, x0, y0, 0, sm.bar);
    *sm.nlf = 0;
  }
  tile_sync();
  if (sched.enabled) {
    const long long i = step - sched.t0;
    if (i >= 0 && i < sched.n) {
      const int b = sched.off[i], e = sched.off[i + 1];
      for (int k = b + tid; k < e; k += kSweepThreads) {
        const DevFlip f = sched.flips[k];
        if (f.grid == g.gid && f.target == 0 && f.x >= x0 && f.x < x0 + kTX && f.x < g.nx && f.y >= y0 &&
            f.y < y0 + TY && f.y < g.ny && f.z >= 0 && f.z < nz && f.x >= 0 && f.y >= 0) {
          const int j = atomicAdd(sm.nlf, 1);
          if (j < kLocalFlips) sm.lflips[j] = make_int4(f.x, f.y, f.z, f.bit & 31);
          else set_status(ctrl, kStFlipOverflow);
        }
      }
    }
  }
  tile_sync();
}

// Periodic boundaries on whole-column tiles: the wrapped values of the rows of plane z
// that this lane needs -- u at x = nx - 1 for a row's first point (W[r]), at x = 0 for
// its last (W[TY + r]), and on a y face the row on the other face (W + WrapCols<TY>::X:
// for y = 0; W + X + kTX: for y = ny - 1) -- copied from global memory to the plane's
// slice W of a shared buffer.  Called before the wait for the tile's copy, so that these
// loads run while it is in flight; a lane later reads only what it wrote.
template <int TY>
struct WrapCols {
  static constexpr int X = (2 * TY + 3) / 4 * 4;  // the row copies start 16-byte aligned
  static constexpr int PLANE = X + 2 * kTX;       // floats per plane (a multiple of 4)
};

template <int TY>
__device__ __forceinline__ void wrap_fetch(const GridDev& g, const float* __restrict__ uin, int z, int y0, int gx0,
                                           int last, int lane, float* W) {
  if (last < 0) return;  // no grid point among the lane's four
  float xw[TY], xe[TY];
  float4 yn = make_float4(0.f, 0.f, 0.f, 0.f), ys = yn;
  const float* base = uin + (size_t)z * g.ny * g.px;
#pragma unroll
  for (int r = 0; r < TY; ++r) {
    const int y = y0 + r;
    xw[r] = xe[r] = 0.f;
    if (y >= g.ny) continue;
    const float* row = base + (size_t)y * g.px;
    if (gx0 == 0) xw[r] = __ldcg(row + g.nx - 1);
    if (last <= 3) xe[r] = __ldcg(row);
    if (y == 0) yn = __ldcg(reinterpret_cast<const float4*>(base + (size_t)(g.ny - 1) * g.px + gx0));
    else if (y == g.ny - 1) ys = __ldcg(reinterpret_cast<const float4*>(base + gx0));
  }
#pragma unroll
  for (int r = 0; r < TY; ++r) {
    if (gx0 == 0) W[r] = xw[r];
    if (last <= 3) W[TY + r] = xe[r];
  }
  constexpr int X = WrapCols<TY>::X;
  if (y0 == 0) *reinterpret_cast<float4*>(W + X + 4 * lane) = yn;
  if (y0 + TY >= g.ny) *reinterpret_cast<float4*>(W + X + kTX + 4 * lane) = ys;
}

template <int TY, bool PROT, int ACC, int BC, int VEC = 2>
__device__ __forceinline__ void shallow_tile_run(const GridDev& g, const float* __restrict__ uin,
                                                 float* __restrict__ uout, int txi, int tyi,
                                                 DevCtrl* __restrict__ ctrl, const ShallowSmem<TY>& sm,
                                                 unsigned& phase, int pbuf) {
  constexpr int NW = ShallowCfg<TY>::NW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = txi * kTX, y0 = tyi * TY;
  const int nz = g.nz;
  const int gx0 = x0 + 4 * lane;
  const int last = g.nx - 1 - gx0;
  // periodic: this warp's planes' wrapped values, fetched while the tile's copy is in flight
  constexpr bool WRAP = BC == ABFT_BC_PERIODIC;
  constexpr int WPL = WrapCols<TY>::PLANE;  // floats of wrapped values per plane
  __shared__ __align__(16) float wbuf[WRAP ? kShallowMaxZ * WPL : 4];
  if (WRAP)
    for (int z = warp; z < nz; z += NW) wrap_fetch<TY>(g, uin, z, y0, gx0, last, lane, wbuf + z * WPL);
  mbar_wait(sm.bar, phase, ctrl);
  phase ^= 1u;
  if (WRAP) __syncwarp();
  const int nflip = min(*sm.nlf, kLocalFlips);
  void* PA = pbuf ? g.PA2 : g.PA;
  void* PB = pbuf ? g.PB2 : g.PB;
  const bool full = x0 + kTX <= g.nx && y0 + TY <= g.ny;  // no ragged edge in this tile
  constexpr int PLANE = (TY + 2) * kUW;
  constexpr bool PA_ON = PROT && VEC == 2;  // column partials (the a vector)
  for (int z = warp; z < nz; z += NW) {
    const float* Uz = sm.u + z * PLANE;
    // at a z face: the centre plane, or for periodic boundaries the staged opposite face
    const float* Ub = z > 0 ? Uz - PLANE : (WRAP ? Uz + (nz - 1) * PLANE : Uz);
    const float* Ut = z + 1 < nz ? Uz + PLANE : (WRAP ? sm.u : Uz);
    const float* W = wbuf + (WRAP ? z * WPL : 0);
    const float* Cz = sm.c + z * TY * kTX;
    AccA<ACC> acc;
    if (PA_ON) acc.zero();
    // row partials, padded with empty rows to a power of two for reduce_rows
    constexpr int RP = TY <= 8 ? 8 : 16;
    typename RowPart<ACC>::T rp[RP];
#pragma unroll
    for (int r = TY; r < RP; ++r) rp[r] = typename RowPart<ACC>::T{};
#pragma unroll
    for (int r = 0; r < TY; ++r) {
      const int y = y0 + r;
      const int o = (r + 1) * kUW + kHaloX + 4 * lane;
      const float4 c = *reinterpret_cast<const float4*>(Uz + o);
      float4 n = *reinterpret_cast<const float4*>(Uz + o - kUW);
      float4 s = *reinterpret_cast<const float4*>(Uz + o + kUW);
      float4 b = *reinterpret_cast<const float4*>(Ub + o);
      float4 t = *reinterpret_cast<const float4*>(Ut + o);
      const float4 cs = *reinterpret_cast<const float4*>(Cz + r * kTX + 4 * lane);
      float wl = __shfl_up_sync(0xffffffffu, c.w, 1);
      float er = __shfl_down_sync(0xffffffffu, c.x, 1);
      if (lane == 0) wl = Uz[o - 1];
      if (lane == 31) er = Uz[o + 4];
      float w0 = wl;
      float e0 = c.y, e1 = c.z, e2 = c.w, e3 = er;
      WrapRow pre{0.f, 0.f, make_float4(0.f, 0.f, 0.f, 0.f)};
      if (WRAP && y < g.ny && last >= 0) {
        pre.xw = W[r];
        pre.xe = W[TY + r];
        if (y == 0) pre.yf = *reinterpret_cast<const float4*>(W + WrapCols<TY>::X + 4 * lane);
        else if (y == g.ny - 1) pre.yf = *reinterpret_cast<const float4*>(W + WrapCols<TY>::X + kTX + 4 * lane);
      }
      boundary_cells<true, BC>(g, uin, z, y, gx0, last, c, n, s, b, t, w0, e0, e1, e2, e3, WRAP ? &pre : nullptr);
      float v[4];
      v[0] = hs_update(g.k, c.x, w0, e0, n.x, s.x, b.x, t.x, cs.x);
      v[1] = hs_update(g.k, c.y, c.x, e1, n.y, s.y, b.y, t.y, cs.y);
      v[2] = hs_update(g.k, c.z, c.y, e2, n.z, s.z, b.z, t.z, cs.z);
      v[3] = hs_update(g.k, c.w, c.z, e3, n.w, s.w, b.w, t.w, cs.w);
      if (nflip > 0) {
        for (int f = 0; f < nflip; ++f) {
          const int4 q = sm.lflips[f];
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
        for (int i = 0; i < 4; ++i) m[i] = full ? v[i] : ((yv && i <= last) ? v[i] : 0.f);
        rp[r] = RowPart<ACC>::of(m);
        if (PA_ON) acc.add(m);
      }
    }
    if (PROT) {
      if (PA_ON) acc.store4(PA, ((size_t)tyi * nz + z) * g.pa_stride + gx0);
      const typename RowPart<ACC>::T tot = reduce_rows<ACC, RP>(rp, lane);
      constexpr int SH = RP == 8 ? 2 : 1;  // lane l holds row l >> SH
      const int r = lane >> SH, y = y0 + r;
      if ((lane & ((1 << SH) - 1)) == 0 && r < TY && y < g.ny)
        RowPart<ACC>::store(PB, ((size_t)txi * nz + z) * g.pb_stride + y, tot);
    }
  }
  fence_proxy_async_global();
  tile_sync();
}

// a-partial of column x of shallow tile tyi in plane z, in the shallow tile's order
template <int TY, int ACC>
__device__ void recompute_pa_shallow(const GridDev& g, const float* __restrict__ u, void* PA, int tyi, int z, int x) {
  const int y0 = tyi * TY;
  auto val = [&](int r) -> float {
    const int y = y0 + r;
    return (y < g.ny && x < g.nx) ? __ldcg(u + ((size_t)z * g.ny + y) * g.px + x) : 0.f;
  };
  const size_t idx = ((size_t)tyi * g.nz + z) * g.pa_stride + x;
  if (ACC == ABFT_ACC_FP32) {
    float a = 0.f;
    for (int r = 0; r < TY; ++r) a += val(r);
    static_cast<float*>(PA)[idx] = a;
  } else if (ACC == ABFT_ACC_TWOSUM) {
    float h = 0.f, l = 0.f;
    for (int r = 0; r < TY; ++r) acc2(h, l, val(r));
    static_cast<float2*>(PA)[idx] = make_float2(h, l);
  } else {
    double a = 0.0;
    for (int r = 0; r < TY; ++r) a += (double)val(r);
    static_cast<double*>(PA)[idx] = a;
  }
}

// ---------------------------------------------------------------- tile policies
// The persistent and per-launch kernels are written once against these.

// BC: the boundary rule the tiles are compiled for (abft_boundary; clamped by default).
// The host picks the policy by the grid's rule, so each kernel carries the code of its
// rule only.
template <int TY, int BC = ABFT_BC_CLAMP>
struct StreamTiles {
  static constexpr int NW = SweepCfg<TY>::NW;
  SweepSmem<TY> sm;
  unsigned seq;
  __host__ __device__ static int smem_bytes(int) { return SweepCfg<TY>::SMEM; }
  __device__ __forceinline__ void setup(unsigned char* raw, int) {
    sm = SweepSmem<TY>::carve(raw);
    seq = 0;
    if (threadIdx.x == 0) sm.init_barriers();
  }
  __device__ __forceinline__ void issue(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g, int txi, int tyi,
                        long long step, DevCtrl* ctrl, const DevSched& sched, bool) {
    sweep_tile_issue<TY>(tm_u, tm_c, g, txi, tyi, step, ctrl, sched, sm, seq);
  }
  template <bool PROT, int ACC, int VEC = 2>
  __device__ __forceinline__ void run(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g,
                                      const float* uin, float* uout, int txi, int tyi, DevCtrl* ctrl, int pbuf) {
    sweep_tile_run<TY, PROT, ACC, BC, VEC>(tm_u, tm_c, g, uin, uout, txi, tyi, ctrl, sm, seq, pbuf);
  }
  template <int ACC>
  __device__ static void recompute_col(const GridDev& g, const float* u, void* PA, int tyi, int z, int x) {
    recompute_pa<TY, ACC>(g, u, PA, tyi, z, x);
  }
};

template <int TY, int BC = ABFT_BC_CLAMP>
struct ShallowTiles {
  static constexpr int NW = ShallowCfg<TY>::NW;
  ShallowSmem<TY> sm;
  unsigned phase;
  __host__ __device__ static int smem_bytes(int nz) { return ShallowCfg<TY>::smem(nz); }
  __device__ __forceinline__ void setup(unsigned char* raw, int nz) {
    sm = ShallowSmem<TY>::carve(raw, nz);
    phase = 0;
    if (threadIdx.x == 0) sm.init_barriers();
  }
  __device__ __forceinline__ void issue(const CUtensorMap* tm_u, const CUtensorMap* tm_c, const GridDev& g, int txi, int tyi,
                        long long step, DevCtrl* ctrl, const DevSched& sched, bool load_c) {
    shallow_tile_issue<TY>(tm_u, tm_c, g, txi, tyi, step, ctrl, sched, sm, load_c);
  }
  template <bool PROT, int ACC, int VEC = 2>
  __device__ __forceinline__ void run(const CUtensorMap*, const CUtensorMap*, const GridDev& g, const float* uin,
                                      float* uout, int txi, int tyi, DevCtrl* ctrl, int pbuf) {
    shallow_tile_run<TY, PROT, ACC, BC, VEC>(g, uin, uout, txi, tyi, ctrl, sm, phase, pbuf);
  }
  template <int ACC>
  __device__ static void recompute_col(const GridDev& g, const float* u, void* PA, int tyi, int z, int x) {
    recompute_pa_shallow<TY, ACC>(g, u, PA, tyi, z, x);
  }
};

}  // namespace abft
