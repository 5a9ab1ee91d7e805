// Host side of the C ABI declared in include/abft.h: context and workspace layout,
// seeded flip schedules, and the drivers of the online (Sec. 3) and offline
// (Sec. 4) modes.  No device memory is allocated here: everything lives in the
// caller's workspace.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "abft_internal.h"

using namespace abft;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// bump allocator over the caller's workspace
struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = align_up(off, 256);
    const size_t at = off;
    off += align_up(bytes ? bytes : 1, 256);
    return at;
  }
};

struct GridPlan {
  size_t u[3], C, cx, cy, A[3], B[3], AP[3], BP[3], PA, PB, PA2, PB2, fcnt, fidx, tdirty, gs;
  size_t tbpa[4], tbpb[4];  // per-level partials of protected temporally blocked passes
};

// per-launch control words of a grid: fails[3], redo, nbz, bar, bars[3] (zeroed before
// every persistent launch)
constexpr size_t kLaunchCtrlBytes = offsetof(DevGridCtrl, verdict) - offsetof(DevGridCtrl, fails);
static_assert(offsetof(DevGridCtrl, redo) == offsetof(DevGridCtrl, fails) + 3 * sizeof(unsigned) &&
                  offsetof(DevGridCtrl, nbz) == offsetof(DevGridCtrl, redo) + sizeof(unsigned) &&
                  offsetof(DevGridCtrl, bar) == offsetof(DevGridCtrl, nbz) + 2 * sizeof(unsigned) &&
                  offsetof(DevGridCtrl, bars) == offsetof(DevGridCtrl, bar) + sizeof(unsigned long long) &&
                  offsetof(DevGridCtrl, verdict) == offsetof(DevGridCtrl, bars) + 3 * sizeof(unsigned long long),
              "per-launch control words must be contiguous");

struct Plan {
  std::vector<GridPlan> g;
  size_t ctrl, gctrl, events, flips, off, total;
  size_t bgrid, btmap, broles, bints;  // batched launches: descriptors, tensor maps, roles, work lists
  int64_t sched_cap;
};

bool is_shallow(const abft_options& o, const abft_grid& G) { return o.shallow && G.nz <= kShallowMaxZ; }

// contexts that sweep with the general kernels (general.cu): a general set or constant
// boundaries
bool general_opts(const abft_options& o) { return o.stencils != nullptr || o.boundary == ABFT_BC_CONST; }

// rows per tile: streaming tiles default to 16, whole-column tiles to 8 (16 allowed; 7 by
// default where it balances a single grid's tiles over the SMs); the general kernels'
// tiles have kGenTY rows
int pick_ty(const abft_options& o, const abft_grid& G, int n_grids) {
  if (general_opts(o)) return kGenTY;
  if (is_shallow(o, G)) {
    if (o.tile_y == 16 && G.nz <= 8) return 16;
    return o.tile_y == 0 && n_grids == 1 ? abft::balanced_shallow_rows(G) : 8;
  }
  return o.tile_y == 8 || o.tile_y == 16 || o.tile_y == 32 ? o.tile_y : 16;
}

size_t partial_elem(int acc) { return acc == ABFT_ACC_FP32 ? 4 : 8; }

bool valid_grid(const abft_grid& g) {
  return g.nx >= 1 && g.ny >= 1 && g.nz >= 1 && g.nx <= (1 << 20) && g.ny <= (1 << 20) && g.nz <= 65535 &&
         (int64_t)g.nx * g.ny * g.nz <= (int64_t)1 << 34;
}

bool valid_options(const abft_options& o) {
  return o.eps > 0 && std::isfinite(o.eps) && o.delta >= 1 && o.acc >= 0 && o.acc <= 2 &&
         o.event_capacity >= 1 && o.graph_steps >= 0 && o.max_flips_per_step >= 0 &&
         o.max_flips_per_step <= 511 && (o.tile_y == 0 || o.tile_y == 8 || o.tile_y == 16 || o.tile_y == 32) &&
         (o.persistent == 0 || o.persistent == 1) && (o.shallow == 0 || o.shallow == 1) &&
         (o.track_residual == 0 || o.track_residual == 1) && (o.batch == 0 || o.batch == 1) &&
         o.depth >= 1 && o.depth <= 4 && (o.overlap == 0 || o.overlap == 1) && o.boundary >= ABFT_BC_CLAMP &&
         o.boundary <= ABFT_BC_CONST && (o.vectors == 1 || o.vectors == 2) && std::isfinite(o.boundary_value);
}

bool make_plan(const abft_grid* grids, int n, const abft_options& o, Plan* P) {
  if (!grids || n < 1 || !valid_options(o)) return false;
  Bump b;
  P->g.resize(n);
  for (int i = 0; i < n; ++i) {
    const abft_grid& G = grids[i];
    if (!valid_grid(G)) return false;
    const int ty = pick_ty(o, G, n);
    const size_t px = align_up(G.nx, 32);
    const size_t vol = px * G.ny * G.nz * sizeof(float);
    const size_t na = (size_t)G.nz * G.nx * 8, nb = (size_t)G.nz * G.ny * 8;
    const size_t ntx = (G.nx + kTX - 1) / kTX, nty = (G.ny + ty - 1) / ty;
    GridPlan& p = P->g[i];
    for (int k = 0; k < 3; ++k) p.u[k] = b.take(vol);
    p.C = b.take(vol);
    p.cx = b.take(na);
    p.cy = b.take(nb);
    for (int k = 0; k < 3; ++k) { p.A[k] = b.take(na); p.B[k] = b.take(nb); }
    for (int k = 0; k < 3; ++k) { p.AP[k] = b.take(na); p.BP[k] = b.take(nb); }
    p.PA = b.take(nty * G.nz * ntx * kTX * partial_elem(o.acc));
    p.PB = b.take(ntx * G.nz * align_up(G.ny, 4) * partial_elem(o.acc));
    p.PA2 = b.take(nty * G.nz * ntx * kTX * partial_elem(o.acc));
    p.PB2 = b.take(ntx * G.nz * align_up(G.ny, 4) * partial_elem(o.acc));
    p.fcnt = b.take((size_t)2 * G.nz * sizeof(int));
    p.fidx = b.take((size_t)2 * G.nz * kFCap * sizeof(int));
    p.tdirty = b.take(2 * ntx * nty * sizeof(int));
    p.gs = b.take(sizeof(GenSten));
    // online checks with temporal blocking: FP32 partials of every level, tiles of
    // kTbRows rows (a partials only with two checksum vectors)
    const size_t nty8 = (G.ny + kTbRows - 1) / kTbRows;
    for (int k = 0; k < 4; ++k) {
      const bool lvl = o.depth >= 2 && k < o.depth;
      p.tbpa[k] = b.take(lvl && o.vectors == 2 ? nty8 * G.nz * ntx * kTX * 4 : 0);
      p.tbpb[k] = b.take(lvl ? ntx * G.nz * align_up(G.ny, 4) * 4 : 0);
    }
  }
  P->ctrl = b.take(sizeof(DevCtrl));
  P->gctrl = b.take(sizeof(DevGridCtrl) * n);
  P->events = b.take(sizeof(abft_event) * (size_t)o.event_capacity);
  P->sched_cap = std::max<int64_t>(1 << 16, (int64_t)o.max_flips_per_step * n * 64);
  P->flips = b.take(sizeof(DevFlip) * P->sched_cap);
  P->off = b.take(sizeof(int) * (kSchedSteps + 1));
  P->bgrid = b.take(sizeof(GridDev) * n);
  P->btmap = b.take(sizeof(CUtensorMap) * kBatchMaps * n);
  P->broles = b.take(sizeof(BatchRole) * n);
  P->bints = b.take(sizeof(int) * (4 * (size_t)n + 16));
  P->total = align_up(b.off, 256);
  return true;
}

// SplitMix64 (Steele, Lea & Flood 2014): output k of the stream seeded with `seed`
struct SplitMix64 {
  uint64_t seed;
  uint64_t at(uint64_t k) const {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (k + 1);
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

// Seeded flips of one (grid, sweep): counter block (t*n_grids + grid)*1024; draw 0 sets
// the count floor(rate) + Bernoulli(frac(rate)), draws 1+2i / 2+2i the point and the bit.
void seeded_flips(uint64_t seed, double rate, uint32_t mask, int grid, int n_grids, const abft_grid& G,
                  int64_t t, std::vector<abft_flip>* out) {
  if (rate <= 0.0 || mask == 0) return;
  const SplitMix64 r{seed};
  const uint64_t base = ((uint64_t)t * (uint64_t)n_grids + (uint64_t)grid) << 10;
  const double whole = std::floor(rate);
  const uint64_t threshold = (uint64_t)((rate - whole) * 9007199254740992.0);
  int64_t count = (int64_t)whole + ((r.at(base) >> 11) < threshold ? 1 : 0);
  count = std::min<int64_t>(count, 511);
  int bits[32], nbits = 0;
  for (int b = 0; b < 32; ++b)
    if (mask & (1u << b)) bits[nbits++] = b;
  const uint64_t npts = (uint64_t)G.nx * G.ny * G.nz;
  for (int64_t i = 0; i < count; ++i) {
    const uint64_t p = (uint64_t)(((unsigned __int128)r.at(base + 1 + 2 * i) * npts) >> 64);
    const uint64_t j = ((r.at(base + 2 + 2 * i) >> 32) * (uint64_t)nbits) >> 32;
    abft_flip f;
    f.step = t;
    f.grid = grid;
    f.x = (int32_t)(p % (uint64_t)G.nx);
    f.y = (int32_t)((p / (uint64_t)G.nx) % (uint64_t)G.ny);
    f.z = (int32_t)(p / ((uint64_t)G.nx * G.ny));
    f.bit = bits[j];
    f.target = 0;
    out->push_back(f);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

namespace abft {

// SMs of the current device (GB300's count where none can be asked, so that layouts
// computed without a GPU are the same)
int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, n = 0;
    sms = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0
              ? n
              : 152;
  }
  return sms;
}

// Whole-column tiles of a grid swept alone: 8 rows, or 7 where that puts fewer rows on
// the busiest SM.  A sweep ends when its slowest SM does, and two tiles share an SM once
// there are more tiles than SMs: 512 rows in columns of 128 make 256 tiles of 8 rows, two
// on 104 of 152 SMs, or 296 tiles of 7 rows, two on 144 SMs and each an eighth smaller.
// Kept to at most two tiles per SM (the persistent kernels hold one tile per CTA).
int balanced_shallow_rows(const abft_grid& G) {
  const int64_t sms = device_sms(), ntx = (G.nx + kTX - 1) / kTX;
  auto rows_on_busiest = [&](int ty) -> int64_t {
    const int64_t tiles = ntx * ((G.ny + ty - 1) / ty);
    return tiles > 2 * sms ? INT64_MAX : ty * ((tiles + sms - 1) / sms);
  };
  return rows_on_busiest(7) < rows_on_busiest(8) ? 7 : 8;
}

cudaError_t make_tensor_maps(const GridDev& g, int ty, CUtensorMap tm_u[3], CUtensorMap* tm_c, char* err,
                             size_t errlen) {
  auto enc = encode_fn();
  if (!enc) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
    return cudaErrorNotSupported;
  }
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.px * g.ny * 4};
  cuuint32_t ebox[3] = {1, 1, 1};
  // streaming tiles stage one plane per box, whole-column tiles all nz planes
  const cuuint32_t depth = g.shallow ? (cuuint32_t)g.nz : 1u;
  cuuint32_t ubox[3] = {(cuuint32_t)kUW, (cuuint32_t)(ty + 2), depth};
  cuuint32_t cbox[3] = {(cuuint32_t)kTX, (cuuint32_t)ty, depth};
  for (int k = 0; k < 4; ++k) {
    CUtensorMap* m = k < 3 ? &tm_u[k] : tm_c;
    void* base = k < 3 ? (void*)g.u[k] : (void*)g.C;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, k < 3 ? ubox : cbox, ebox,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)r);
      return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

cudaError_t make_tb_maps(const GridDev& g, int k, CUtensorMap tm_u[3], CUtensorMap* tm_c, char* err, size_t errlen) {
  auto enc = encode_fn();
  if (!enc) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
    return cudaErrorNotSupported;
  }
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.px * g.ny * 4};
  cuuint32_t ebox[3] = {1, 1, 1};
  cuuint32_t box[3] = {(cuuint32_t)kUW, (cuuint32_t)(kTbRows + 2 * k), 1u};  // u and C alike
  for (int i = 0; i < 4; ++i) {
    CUtensorMap* m = i < 3 ? &tm_u[i] : tm_c;
    void* base = i < 3 ? (void*)g.u[i] : (void*)g.C;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, ebox,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      snprintf(err, errlen, "cuTensorMapEncodeTiled (temporal blocking) failed (%d)", (int)r);
      return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

cudaError_t make_partial_maps(const GridDev& g, CUtensorMap tm[4], char* err, size_t errlen) {
  auto enc = encode_fn();
  if (!enc) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
    return cudaErrorNotSupported;
  }
  // TwoSum partials are (hi, lo) float pairs: twice the FP32 elements per entry
  const int per = g.acc == ABFT_ACC_TWOSUM ? 2 : 1;
  const CUtensorMapDataType dt = g.acc == ABFT_ACC_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const size_t esz = g.acc == ABFT_ACC_FP64 ? 8 : 4;
  for (int k = 0; k < 4; ++k) {
    const bool is_a = k < 2;
    const size_t row = (size_t)(is_a ? g.pa_stride : g.pb_stride) * per;  // elements per (tile, plane) row
    const int nt = is_a ? g.nty : g.ntx;
    if (nt > 256) {  // box limit; the persistent kernel is not used for such grids
      memset(&tm[k], 0, sizeof tm[k]);
      continue;
    }
    cuuint64_t dims[3] = {(cuuint64_t)row, (cuuint64_t)g.nz, (cuuint64_t)nt};
    cuuint64_t strides[2] = {(cuuint64_t)(row * esz), (cuuint64_t)(row * esz * g.nz)};
    cuuint32_t box[3] = {(cuuint32_t)(kCheckBox * per), 1, (cuuint32_t)nt};
    cuuint32_t ebox[3] = {1, 1, 1};
    void* base = k == 0 ? g.PA : k == 1 ? g.PA2 : k == 2 ? g.PB : g.PB2;
    CUresult r = enc(&tm[k], dt, 3, base, dims, strides, box, ebox, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      snprintf(err, errlen, "cuTensorMapEncodeTiled (partials) failed (%d)", (int)r);
      return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

}  // namespace abft

struct abft_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  abft_options opt{};
  int n = 0;
  std::vector<abft_grid> grids;
  std::vector<abft_coeffs> co;
  std::vector<GridDev> g;
  std::vector<CUtensorMap> tm_u, tm_c, tm_p;
  std::vector<CUtensorMap> tm_tb;  // temporal blocking (depth >= 2): u[0..2], C per grid
  std::vector<int> cur, ref;
  std::vector<int64_t> ref_step;
  // general stencil sets (general.cu): every grid's set as a GenSten (the 7-point set
  // too, for per-step chains); `general`: the context sweeps with the general kernels
  bool general = false;
  std::vector<GenSten> gen;
  std::vector<char> vanish;    // Theorem 1's boundary terms vanish for the grid's set and rule
  // online checks with temporal blocking: per-level partials, and the verdict of each
  // pass copied to pinned memory behind an event (two in flight)
  std::vector<TbLevels> tbl;
  unsigned long long* h_tbflag = nullptr;
  cudaEvent_t tb_ev[2] = {nullptr, nullptr};
  std::vector<char> ck_valid;  // A/B[cur] are the current state's checksums: 0 no, 1 both, 2 only B
  std::vector<char> ref_ck;    // the same for A/B[ref], the verified state
  int64_t step = 0;
  DevCtrl* ctrl = nullptr;
  DevGridCtrl* gctrl = nullptr;
  abft_event* events = nullptr;
  DevFlip* d_flips = nullptr;
  int* d_off = nullptr;
  int64_t sched_cap = 0;
  // injection
  int inj_kind = 0;  // 0 none, 1 seeded, 2 list
  uint64_t seed = 0;
  double rate = 0;
  uint32_t mask = 0;
  std::vector<abft_flip> list;
  int64_t sched_t0 = 0, sched_n = 0;  // what the device currently holds
  bool sched_live = false;
  // pinned host staging
  DevFlip* h_flips = nullptr;
  int* h_off = nullptr;
  DevCtrl* h_ctrl = nullptr;
  DevGridCtrl* h_gctrl = nullptr;
  abft_event* h_ev = nullptr;
  // verify state
  bool verified = false;
  std::vector<int64_t> v_dist;
  std::vector<unsigned long long> v_fail;
  // timing hook
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  // batched launches (contexts with several grids)
  struct BClass {
    int shallow, ty, smem, blocks, n, grids_at, off_at;
    int box, nw;  // check launch: box bytes (0: no TMA boxes), warps per block
  };
  std::vector<BClass> bcls;      // sweep launches, one per tile class
  BClass bchk{};                 // the check launch
  GridDev* d_bgrid = nullptr;
  CUtensorMap* d_btmap = nullptr;
  BatchRole* d_roles = nullptr;
  int* d_bints = nullptr;
  std::vector<int> h_bints;
  std::vector<CUtensorMap> h_btmap;
  BatchRole* h_roles = nullptr;  // pinned
  cudaEvent_t roles_ev = nullptr;
  bool roles_pending = false;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream = nullptr;  // concurrent tile classes (and their captured branch)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [unprotected, online]: graph_steps sweeps each
  // counters
  int64_t launches = 0, rollbacks = 0, flips_scheduled = 0, tb_redo = 0;
  unsigned status_seen = 0;
  std::string err;
};

namespace {

abft_status fail(abft_ctx* c, abft_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, ABFT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

Launch launcher(abft_ctx* ctx) {
  Launch L;
  L.s = ctx->stream;
  L.ctrl = ctx->ctrl;
  L.events = ctx->events;
  L.sched.flips = ctx->d_flips;
  L.sched.off = ctx->d_off;
  return L;
}

// every kernel launch goes through here: counted, and bracketed by events when timing
template <class F>
cudaError_t run(abft_ctx* ctx, int kind, F&& f) {
  if (ctx->timing) {
    if (ctx->ev_used + 2 > ctx->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ctx->ev_pool.push_back(e);
      }
    }
    cudaEventRecord(ctx->ev_pool[ctx->ev_used], ctx->stream);
    const cudaError_t r = f();
    cudaEventRecord(ctx->ev_pool[ctx->ev_used + 1], ctx->stream);
    ctx->ev_kind.push_back(kind);
    ctx->ev_used += 2;
    ++ctx->launches;
    return r;
  }
  ++ctx->launches;
  return f();
}

int other_than(int a, int b) {
  for (int k = 0; k < 3; ++k)
    if (k != a && k != b) return k;
  return -1;
}

// Theorem 1 without the grid (the chain of Fig. 10) needs vanishing boundary terms:
// always for periodic boundaries, for clamped ones when opposite in-plane weights are
// equal, never for empty ones (their terms hold the edge rows themselves)
bool offline_capable(const abft_coeffs& c, int bc) {
  return bc == ABFT_BC_PERIODIC || (bc == ABFT_BC_CLAMP && c.cn == c.cs && c.cw == c.ce);
}

// the chain of a grid's offline windows: Eq. (6)/(7) up front (7-point kernels, terms
// vanish), or one link per sweep with the terms of the sweep's input state
bool simple_chain(const abft_ctx* ctx, int gi) {
  return !ctx->general && offline_capable(ctx->co[gi], ctx->opt.boundary);
}

// the set S of grid gi: the caller's general set, or the 7-point set of its coefficients
// (Eq. 1's order: centre, x-1, x+1, y-1, y+1, z-1, z+1); false for an invalid set
bool build_gen(const abft_options& o, const abft_coeffs& c, int gi, GenSten* s) {
  memset(s, 0, sizeof *s);
  if (o.stencils) {
    const abft_stencil& st = o.stencils[gi];
    if (st.npts < 1 || st.npts > kGenMaxPts) return false;
    s->npts = st.npts;
    for (int k = 0; k < st.npts; ++k) {
      const abft_point& p = st.pts[k];
      if (std::abs(p.dx) > kGenRadius || std::abs(p.dy) > kGenRadius || std::abs(p.dz) > kGenRadius ||
          !std::isfinite(p.w))
        return false;
      s->dx[k] = p.dx; s->dy[k] = p.dy; s->dz[k] = p.dz; s->w[k] = p.w;
      s->r = std::max({s->r, std::abs(p.dx), std::abs(p.dy), std::abs(p.dz)});
    }
    return true;
  }
  const int off[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  const float w[7] = {c.cc, c.cw, c.ce, c.cn, c.cs, c.cb, c.ct};
  s->npts = 7;
  s->r = 1;
  for (int k = 0; k < 7; ++k) {
    s->dx[k] = off[k][0]; s->dy[k] = off[k][1]; s->dz[k] = off[k][2]; s->w[k] = w[k];
  }
  return true;
}

// Theorem 1's alpha, beta vanish: periodic boundaries; clamped ones when every point has
// an equal-weight partner mirrored in x and one mirrored in y and no in-plane offset
// exceeds one (offsets of two leave 2u_0 - u_{n-2} - u_{n-1}); never for empty or
// constant boundaries
bool gen_vanish(const GenSten& s, int bc) {
  if (bc == ABFT_BC_PERIODIC) return true;
  if (bc != ABFT_BC_CLAMP) return false;
  for (int k = 0; k < s.npts; ++k) {
    if (std::abs(s.dx[k]) > 1 || std::abs(s.dy[k]) > 1) return false;
    bool mx = false, my = false;
    for (int m = 0; m < s.npts; ++m) {
      if (s.dz[m] != s.dz[k] || s.w[m] != s.w[k]) continue;
      if (s.dx[m] == -s.dx[k] && s.dy[m] == s.dy[k]) mx = true;
      if (s.dx[m] == s.dx[k] && s.dy[m] == -s.dy[k]) my = true;
    }
    if (!mx || !my) return false;
  }
  return true;
}

// upload the flips of sweeps [t0, t0 + n) (n <= kSchedSteps); returns the number of
// sweeps actually covered (less than n when the capacity runs out)
abft_status upload_schedule(abft_ctx* ctx, int64_t t0, int64_t n, int64_t* covered) {
  *covered = n;
  if (ctx->inj_kind == 0) {
    if (ctx->sched_live) {
      ctx->h_ctrl->sched_n = 0;
      CK(cudaMemcpyAsync(&ctx->ctrl->sched_n, &ctx->h_ctrl->sched_n, sizeof(int), cudaMemcpyHostToDevice,
                         ctx->stream));
      ctx->sched_live = false;
    }
    return ABFT_OK;
  }
  CK(cudaStreamSynchronize(ctx->stream));  // staging buffers are about to be rewritten
  std::vector<abft_flip> fl;
  int64_t total = 0;
  int64_t t = t0;
  ctx->h_off[0] = 0;
  for (; t < t0 + n; ++t) {
    fl.clear();
    if (ctx->inj_kind == 1) {
      for (int gi = 0; gi < ctx->n; ++gi)
        seeded_flips(ctx->seed, ctx->rate, ctx->mask, gi, ctx->n, ctx->grids[gi], t, &fl);
    } else {
      auto lo = std::lower_bound(ctx->list.begin(), ctx->list.end(), t,
                                 [](const abft_flip& f, int64_t s) { return f.step < s; });
      for (auto it = lo; it != ctx->list.end() && it->step == t; ++it) fl.push_back(*it);
    }
    if (total + (int64_t)fl.size() > ctx->sched_cap) break;
    for (const abft_flip& f : fl) {
      DevFlip& d = ctx->h_flips[total++];
      d.step = f.step; d.grid = f.grid; d.z = f.z; d.y = f.y; d.x = f.x; d.bit = f.bit; d.target = f.target;
    }
    ctx->h_off[t - t0 + 1] = (int)total;
  }
  if (t == t0 && n > 0) return fail(ctx, ABFT_E_INVAL, "flips of one sweep exceed the schedule capacity");
  *covered = t - t0;
  ctx->flips_scheduled += total;
  if (total) CK(cudaMemcpyAsync(ctx->d_flips, ctx->h_flips, sizeof(DevFlip) * total, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_off, ctx->h_off, sizeof(int) * (*covered + 1), cudaMemcpyHostToDevice, ctx->stream));
  ctx->h_ctrl->sched_t0 = t0;
  ctx->h_ctrl->sched_n = (int)*covered;
  CK(cudaMemcpyAsync(&ctx->ctrl->sched_t0, &ctx->h_ctrl->sched_t0, sizeof(long long) + sizeof(int),
                     cudaMemcpyHostToDevice, ctx->stream));
  ctx->sched_live = true;
  return ABFT_OK;
}

abft_status set_inject_enabled(abft_ctx* ctx, int on) {
  ctx->h_ctrl->inject_enabled = on;
  CK(cudaMemcpyAsync(&ctx->ctrl->inject_enabled, &ctx->h_ctrl->inject_enabled, sizeof(int),
                     cudaMemcpyHostToDevice, ctx->stream));
  return ABFT_OK;
}

abft_status read_ctrl(abft_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_ctrl, ctx->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_gctrl, ctx->gctrl, sizeof(DevGridCtrl) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return ABFT_OK;
}

// what an online sweep leaves valid: both vectors, or only B with one-vector checks
char online_ck(const GridDev& g) { return g.vec == 1 ? 2 : 1; }

// make A[cur], B[cur] the checksums of the current state (trusted, Theorem 2's premise);
// need_a = false: B alone suffices (one-vector online checks)
abft_status ensure_checksums(abft_ctx* ctx, int gi, bool need_a = true) {
  if (ctx->ck_valid[gi] == 1 || (!need_a && ctx->ck_valid[gi] == 2)) return ABFT_OK;
  const GridDev& g = ctx->g[gi];
  const int c = ctx->cur[gi];
  const Launch L = launcher(ctx);
  CK(run(ctx, kKOther, [&] { return launch_checksums(L, g, g.u[c], g.A[c], g.B[c]); }));
  ctx->ck_valid[gi] = 1;
  if (ctx->ref[gi] == c) ctx->ref_ck[gi] = 1;
  return ABFT_OK;
}

// `n` sweeps of every grid, one persistent cooperative launch per grid
abft_status persistent_all(abft_ctx* ctx, int64_t n, int mode) {
  const Launch L = launcher(ctx);
  const bool prot = mode == ABFT_MODE_ONLINE;
  for (int gi = 0; gi < ctx->n; ++gi) {
    if (prot) {
      abft_status s = ensure_checksums(ctx, gi, ctx->g[gi].vec != 1);
      if (s) return s;
    }
    const GridDev& g = ctx->g[gi];
    const int c = ctx->cur[gi];
    int p, q;
    if (prot) {
      p = (c + 1) % 3;
      q = c;
    } else if (c == ctx->ref[gi]) {
      p = other_than(c, -1);
      q = other_than(c, p);
    } else {
      p = other_than(c, ctx->ref[gi]);
      q = c;
    }
    // zero the per-sweep fail counters, redo flag and barrier counters (contiguous)
    CK(cudaMemsetAsync(&ctx->gctrl[gi].fails[0], 0, kLaunchCtrlBytes, ctx->stream));
    int blocks = 0;
    CK(run(ctx, prot ? kKPersistProt : kKPersistPlain, [&] {
      return launch_persistent(L, g, &ctx->tm_u[3 * gi], ctx->tm_c[gi], &ctx->tm_p[4 * gi], ctx->step, (int)n, c, p, q,
                               prot, &blocks);
    }));
    ctx->cur[gi] = prot ? (int)((c + n) % 3) : (((n - 1) & 1) ? q : p);
    if (prot) {
      ctx->ref[gi] = ctx->cur[gi];
      ctx->ref_step[gi] = ctx->step + n;
      ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(g);
    } else {
      ctx->ck_valid[gi] = 0;
    }
  }
  ctx->step += n;
  return ABFT_OK;
}

// `n` sweeps of every grid in offline windows, one persistent launch per grid
abft_status persistent_offline_all(abft_ctx* ctx, int64_t n) {
  const Launch L = launcher(ctx);
  const int delta = std::max(ctx->opt.delta, 1);
  for (int gi = 0; gi < ctx->n; ++gi) {
    abft_status s = ensure_checksums(ctx, gi);
    if (s) return s;
    const GridDev& g = ctx->g[gi];
    CK(cudaMemsetAsync(&ctx->gctrl[gi].fails[0], 0, kLaunchCtrlBytes, ctx->stream));
    int blocks = 0;
    const int ck = ctx->cur[gi];
    CK(run(ctx, kKPersistProt, [&] {
      return launch_persistent_offline(L, g, &ctx->tm_u[3 * gi], ctx->tm_c[gi], ctx->step, (int)n, delta, ck, &blocks);
    }));
    // the buffer roles follow the window lengths only (a recomputed window reuses its buffers)
    int c = ck;
    for (int64_t t = 0; t < n; t += delta) {
      const int64_t d = std::min<int64_t>(delta, n - t);
      const int w0 = (c + 1) % 3, w1 = (c + 2) % 3;
      c = ((d - 1) & 1) ? w1 : w0;
    }
    ctx->cur[gi] = c;
    ctx->ref[gi] = c;
    ctx->ref_step[gi] = ctx->step + n;
    ctx->ck_valid[gi] = ctx->ref_ck[gi] = 1;
  }
  ctx->step += n;
  return ABFT_OK;
}

// one sweep of every grid; protected sweeps write partial checksums
abft_status sweep_all(abft_ctx* ctx, int mode) {
  const Launch L = launcher(ctx);
  for (int gi = 0; gi < ctx->n; ++gi) {
    const GridDev& g = ctx->g[gi];
    const int in = ctx->cur[gi];
    if (ctx->general) {  // any set S, any boundary rule (general.cu)
      const int r = ctx->gen[gi].r;
      if (mode == ABFT_MODE_ONLINE) {
        const int out = (in + 1) % 3;
        CK(run(ctx, kKSweepProt, [&] { return launch_sweep_gen(L, g, r, in, out, true); }));
        CK(run(ctx, kKCheckOnline, [&] { return launch_check_gen(L, g, in, out); }));
        CK(run(ctx, kKOther, [&] { return launch_resolve_gen(L, g, in, out, ctx->step); }));
        ctx->cur[gi] = out;
        ctx->ref[gi] = out;
        ctx->ref_step[gi] = ctx->step + 1;
        ctx->ck_valid[gi] = ctx->ref_ck[gi] = 1;
      } else {
        const int out = other_than(in, ctx->ref[gi]);
        CK(run(ctx, kKSweepPlain, [&] { return launch_sweep_gen(L, g, r, in, out, false); }));
        ctx->cur[gi] = out;
        ctx->ck_valid[gi] = 0;
      }
      continue;
    }
    if (mode == ABFT_MODE_ONLINE) {
      const int out = (in + 1) % 3;  // the verified state moves with every sweep
      CK(run(ctx, kKSweepProt, [&] { return launch_sweep(L, g, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out, true); }));
      const PartialMaps* pm = reinterpret_cast<const PartialMaps*>(&ctx->tm_p[4 * gi]);
      CK(run(ctx, kKCheckOnline, [&] { return launch_check_online(L, g, *pm, in, out); }));
      CK(run(ctx, kKOther, [&] { return launch_resolve(L, g, in, out, ctx->step); }));
      ctx->cur[gi] = out;
      ctx->ref[gi] = out;
      ctx->ref_step[gi] = ctx->step + 1;
      ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(g);
    } else {
      const int out = other_than(in, ctx->ref[gi]);
      CK(run(ctx, kKSweepPlain, [&] { return launch_sweep(L, g, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out, false); }));
      ctx->cur[gi] = out;
      ctx->ck_valid[gi] = 0;
    }
  }
  ++ctx->step;
  return ABFT_OK;
}

// `n` online sweeps of a single grid with the check of each sweep overlapping the next
// sweep.  Sweep s+1 starts as soon as sweep s is done; the check and location of sweep
// s run beside it on a side stream (one-warp box-check blocks fit next to the sweep's
// CTAs) and write their fixes into u^{s+1} directly; a conditional recomputation of
// sweep s+1 then runs only if a fix was made (its CTAs leave at once otherwise).
// Partial checksums alternate between two buffers by sweep parity, so the sweep never
// overwrites the partials its predecessor's check is reading.  Results equal the
// sequential order bit for bit.
abft_status online_overlap(abft_ctx* ctx, int64_t n) {
  const int gi = 0;
  const GridDev& g = ctx->g[gi];
  Launch A = launcher(ctx);
  cudaError_t e = cudaSuccess;
  if (!ctx->side_stream) e = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->fork_ev) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->join_ev) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail(ctx, ABFT_E_CUDA, "overlap set-up: %s", cudaGetErrorString(e));
  Launch B = A;
  B.s = ctx->side_stream;
  CK(cudaMemsetAsync(&ctx->gctrl[gi].redo, 0, sizeof(unsigned), A.s));
  for (int64_t k = 0; k < n; ++k) {
    const int64_t s = ctx->step;
    const int in = ctx->cur[gi], out = (in + 1) % 3;
    // this sweep's partial buffers (parity of s)
    GridDev gs = g;
    PartialMaps pm = *reinterpret_cast<const PartialMaps*>(&ctx->tm_p[4 * gi]);
    if (s & 1) {
      gs.PA = g.PA2;
      gs.PB = g.PB2;
      std::swap(pm.m[0], pm.m[1]);
      std::swap(pm.m[2], pm.m[3]);
    }
    CK(run(ctx, kKSweepProt, [&] { return launch_sweep(A, gs, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out, true); }));
    if (k > 0) {  // the previous sweep's check may have fixed u^s: recompute this sweep if so
      CK(cudaStreamWaitEvent(A.s, ctx->join_ev, 0));
      CK(run(ctx, kKOther,
             [&] { return launch_redo_tiles(A, gs, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out); }));
    }
    CK(cudaEventRecord(ctx->fork_ev, A.s));
    CK(cudaStreamWaitEvent(B.s, ctx->fork_ev, 0));
    CK(run(ctx, kKCheckOnline, [&] { return launch_check_online(B, gs, pm, in, out, 1); }));
    CK(run(ctx, kKOther, [&] { return launch_resolve(B, gs, in, out, s); }));
    CK(cudaEventRecord(ctx->join_ev, B.s));
    ctx->cur[gi] = out;
    ctx->ref[gi] = out;
    ctx->ref_step[gi] = s + 1;
    ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(g);
    ++ctx->step;
  }
  CK(cudaStreamWaitEvent(A.s, ctx->join_ev, 0));  // the last check and its fixes
  return ABFT_OK;
}

// Work lists of the batched launches: grids grouped by tile class, deepest first;
// the check launch gives each grid blocks of 32-entry rounds (eight per warp with TMA
// boxes; otherwise kBatchMinRounds to kBatchRounds per block, by the batch's size).
void build_batch_tables(abft_ctx* ctx) {
  const int n = ctx->n;
  ctx->h_btmap.resize((size_t)kBatchMaps * n);
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) ctx->h_btmap[kBatchMaps * i + k] = ctx->tm_u[3 * i + k];
    ctx->h_btmap[kBatchMaps * i + 3] = ctx->tm_c[i];
    for (int k = 0; k < 4; ++k) ctx->h_btmap[kBatchMaps * i + 4 + k] = ctx->tm_p[4 * i + k];
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const GridDev &x = ctx->g[a], &y = ctx->g[b];
    if (x.nz != y.nz) return x.nz > y.nz;
    return x.ntx * x.nty > y.ntx * y.nty;
  });
  std::vector<int> grids, offs;
  ctx->bcls.clear();
  std::vector<std::pair<int, int>> classes;  // (shallow, ty) in first-seen order
  for (int i : order) {
    const std::pair<int, int> c(ctx->g[i].shallow, ctx->g[i].ty);
    if (std::find(classes.begin(), classes.end(), c) == classes.end()) classes.push_back(c);
  }
  std::vector<std::pair<size_t, size_t>> at;
  std::vector<std::vector<int>> off_lists;
  for (const auto& c : classes) {
    abft_ctx::BClass b{};
    b.shallow = c.first;
    b.ty = c.second;
    b.grids_at = (int)grids.size();
    std::vector<int> off{0};
    for (int i : order) {
      const GridDev& g = ctx->g[i];
      if (g.shallow != c.first || g.ty != c.second) continue;
      grids.push_back(i);
      off.push_back(off.back() + g.ntx * g.nty);
      b.smem = std::max(b.smem, batch_sweep_smem(g.shallow, g.ty, g.nz));
    }
    b.n = (int)off.size() - 1;
    b.blocks = off.back();
    off_lists.push_back(off);
    ctx->bcls.push_back(b);
  }
  abft_ctx::BClass& k = ctx->bchk;
  k = abft_ctx::BClass{};
  k.grids_at = (int)grids.size();
  // the check reads the partials with plain coalesced loads: measured on the uneven
  // 256-grid batch, per-warp TMA boxes (one descriptor per grid, fetched from global
  // memory) were slower; the single-grid check uses boxes
  bool box = false;
  int box_bytes = 0;
  for (int i = 0; i < n; ++i) {
    box = box && check_box_usable(ctx->g[i]);  // (kept for a future per-shape choice)
    box_bytes = std::max(box_bytes, (check_box_bytes_host(ctx->g[i].nty, ctx->g[i].ntx, ctx->opt.acc) + 127) / 128 * 128);
  }
  k.box = box ? box_bytes : 0;
  k.nw = box ? check_box_warps(box_bytes) : 8;
  k.smem = box ? 256 + k.nw * box_bytes : 0;
  auto rounds_of = [&](const GridDev& g) -> int64_t {
    return box ? check_rounds_host(g) : ((int64_t)g.nz * (g.nx + g.ny) - check_entries_first(g) + 31) / 32;
  };
  // 32-entry rounds per block: with plain loads, as many as keep about four waves of two
  // blocks per SM (a block's set-up is spread over its rounds), between kBatchMinRounds
  // and kBatchRounds
  int per_block = 8 * k.nw;
  if (!box) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev) != cudaSuccess || sms < 1) sms = 1;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) total += rounds_of(ctx->g[i]);
    per_block = (int)std::min<int64_t>(kBatchRounds, std::max<int64_t>(kBatchMinRounds, total / (8LL * sms)));
  }
  std::vector<int> koff{0};
  for (int i = 0; i < n; ++i) {
    grids.push_back(i);
    koff.push_back(koff.back() + (int)((rounds_of(ctx->g[i]) + per_block - 1) / per_block));
  }
  k.n = n;
  k.blocks = koff.back();
  off_lists.push_back(koff);
  ctx->h_bints = grids;
  for (size_t c = 0; c < off_lists.size(); ++c) {
    abft_ctx::BClass& b = c < ctx->bcls.size() ? ctx->bcls[c] : ctx->bchk;
    b.off_at = (int)ctx->h_bints.size();
    ctx->h_bints.insert(ctx->h_bints.end(), off_lists[c].begin(), off_lists[c].end());
  }
}

BatchArgs batch_args(const abft_ctx* ctx, const abft_ctx::BClass& b) {
  BatchArgs a;
  a.g = ctx->d_bgrid;
  a.tm = ctx->d_btmap;
  a.roles = ctx->d_roles;
  a.grids = ctx->d_bints + b.grids_at;
  a.off = ctx->d_bints + b.off_at;
  a.n = b.n;
  return a;
}

int batch_kernels_per_sweep(const abft_ctx* ctx, bool prot) {
  int k = 0;
  for (const auto& b : ctx->bcls) k += b.blocks > 0;
  return k + (prot && ctx->bchk.blocks > 0 ? 1 : 0);
}

// one sweep of every grid: the class sweeps, then the check; `counted` routes the
// launches through run() (counting and timing), otherwise they are being captured
cudaError_t batch_sweep(abft_ctx* ctx, const Launch& L, bool prot, bool counted) {
  const int acc = ctx->opt.acc;
  // tile classes after the first run on a side stream, concurrently (their grids are
  // disjoint); the check waits for all of them.  Sequential while kernels are timed.
  const bool fork = ctx->bcls.size() > 1 && !ctx->timing;
  if (fork) {
    cudaError_t e = cudaSuccess;
    if (!ctx->side_stream) e = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->fork_ev) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->join_ev) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->fork_ev, L.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side_stream, ctx->fork_ev, 0);
    if (e != cudaSuccess) return e;
  }
  for (size_t c = 0; c < ctx->bcls.size(); ++c) {
    const auto& b = ctx->bcls[c];
    const BatchArgs a = batch_args(ctx, b);
    Launch Lc = L;
    if (fork && c > 0) Lc.s = ctx->side_stream;
    auto f = [&] {
      return launch_sweep_batch(Lc, a, b.blocks, b.smem, b.shallow, b.ty, prot, acc, ctx->opt.boundary);
    };
    const cudaError_t e = counted ? run(ctx, prot ? kKSweepProt : kKSweepPlain, f) : f();
    if (e != cudaSuccess) return e;
  }
  if (fork) {
    cudaError_t e = cudaEventRecord(ctx->join_ev, ctx->side_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.s, ctx->join_ev, 0);
    if (e != cudaSuccess) return e;
  }
  if (!prot) return cudaSuccess;
  const BatchArgs a = batch_args(ctx, ctx->bchk);
  auto f = [&] { return launch_check_batch(L, a, ctx->bchk.blocks, acc, ctx->bchk.box, ctx->bchk.nw, ctx->bchk.smem); };
  return counted ? run(ctx, kKCheckOnline, f) : f();
}

// a CUDA graph of graph_steps batched sweeps, captured on a private stream
abft_status batch_graph(abft_ctx* ctx, bool prot, cudaGraphExec_t* out) {
  if (ctx->graph[prot]) {
    *out = ctx->graph[prot];
    return ABFT_OK;
  }
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  Launch L = launcher(ctx);
  L.s = ctx->cap_stream;
  CK(cudaStreamBeginCapture(L.s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < ctx->opt.graph_steps && e == cudaSuccess; ++t) e = batch_sweep(ctx, L, prot, false);
  cudaGraph_t gr = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(L.s, &gr);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph[prot], gr, 0);
  if (gr) cudaGraphDestroy(gr);
  if (e != cudaSuccess) return fail(ctx, ABFT_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
  *out = ctx->graph[prot];
  return ABFT_OK;
}

// `n` sweeps of every grid with batched launches (graphs of graph_steps sweeps where
// they fit, single sweeps for the rest)
abft_status batch_all(abft_ctx* ctx, int64_t n, int mode) {
  const bool prot = mode == ABFT_MODE_ONLINE;
  if (prot)
    for (int gi = 0; gi < ctx->n; ++gi) {
      abft_status s = ensure_checksums(ctx, gi, ctx->g[gi].vec != 1);
      if (s) return s;
    }
  for (const auto& b : ctx->bcls) CK(batch_prepare(b.shallow, b.ty, prot, ctx->opt.acc, ctx->opt.boundary, b.smem));
  if (prot && ctx->bchk.box) CK(batch_check_prepare(ctx->opt.acc, ctx->bchk.smem));
  if (ctx->roles_pending) CK(cudaEventSynchronize(ctx->roles_ev));  // the previous upload has been read
  for (int gi = 0; gi < ctx->n; ++gi) {
    BatchRole& r = ctx->h_roles[gi];
    const int c = ctx->cur[gi], ref = ctx->ref[gi];
    r.s0 = ctx->step;
    r.first = c;
    r.mode = prot ? 1 : 0;
    r.a = other_than(c, ref);
    r.b = c == ref ? other_than(ref, r.a) : c;
  }
  CK(cudaMemcpyAsync(ctx->d_roles, ctx->h_roles, sizeof(BatchRole) * ctx->n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaEventRecord(ctx->roles_ev, ctx->stream));
  ctx->roles_pending = true;
  const Launch L = launcher(ctx);
  int64_t k = 0;
  const int T = ctx->opt.graph_steps;
  if (T > 0 && !ctx->timing && n >= T) {
    cudaGraphExec_t ex = nullptr;
    abft_status s = batch_graph(ctx, prot, &ex);
    if (s) return s;
    for (; n - k >= T; k += T) {
      CK(cudaGraphLaunch(ex, ctx->stream));
      ctx->launches += (int64_t)T * batch_kernels_per_sweep(ctx, prot);
    }
  }
  for (; k < n; ++k) CK(batch_sweep(ctx, L, prot, true));
  for (int gi = 0; gi < ctx->n; ++gi) {
    const BatchRole& r = ctx->h_roles[gi];
    if (prot) {
      ctx->cur[gi] = (int)((r.first + n) % 3);
      ctx->ref[gi] = ctx->cur[gi];
      ctx->ref_step[gi] = ctx->step + n;
      ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(ctx->g[gi]);
    } else {
      ctx->cur[gi] = ((n - 1) & 1) ? r.b : r.a;
      ctx->ck_valid[gi] = 0;
    }
  }
  ctx->step += n;
  return ABFT_OK;
}

// `depth` unprotected sweeps of every grid, one temporally blocked pass per grid
abft_status tb_all(abft_ctx* ctx) {
  const Launch L = launcher(ctx);
  const int k = ctx->opt.depth;
  for (int gi = 0; gi < ctx->n; ++gi) {
    const GridDev& g = ctx->g[gi];
    const int in = ctx->cur[gi], out = other_than(in, ctx->ref[gi]);
    CK(run(ctx, kKSweepPlain,
           [&] { return launch_sweep_tb(L, g, ctx->tm_tb[4 * gi + in], ctx->tm_tb[4 * gi + 3], out, k); }));
    ctx->cur[gi] = out;
    ctx->ck_valid[gi] = 0;
  }
  ctx->step += k;
  return ABFT_OK;
}

// Online checks with temporal blocking (a single clamped grid whose boundary terms vanish,
// FP32 checksums): passes of k = depth sweeps, each one blocked launch that also writes
// every level's partial checksums, then one check launch per level (Theorem 1 from the
// level before, the Sec. 3.4 test).  The verdict of a pass is read on the host one pass
// later, while the next pass runs: a pass writes the third buffer, so the input of the
// previous one is still intact.  A pass with a failing entry is discarded (and the one
// launched after it) and its k sweeps are recomputed as single sweeps with the online
// check of every sweep, which locates and corrects what failed and logs the events
// exactly as the single-sweep online mode does.
abft_status set_grid_step(abft_ctx* ctx, int gi, int64_t step);

bool online_tb_ok(const abft_ctx* ctx) {
  return ctx->n == 1 && ctx->opt.depth >= 2 && !ctx->general && ctx->opt.boundary == ABFT_BC_CLAMP &&
         simple_chain(ctx, 0) && ctx->opt.acc == ABFT_ACC_FP32;
}

abft_status online_tb(abft_ctx* ctx, int64_t n) {
  const int gi = 0, k = ctx->opt.depth;
  const GridDev& g = ctx->g[gi];
  const Launch L = launcher(ctx);
  GridDev gt = g;  // the level checks' view: partials of kTbRows-row tiles
  gt.ty = kTbRows;
  gt.nty = (g.ny + kTbRows - 1) / kTbRows;
  const int64_t t_end = ctx->step + n;
  struct Pass {
    int64_t t0 = -1;
    int in = 0, slot = 0;
  } prev;
  int slot = 0;
  abft_status s = ABFT_OK;
  for (;;) {
    Pass cur;
    const bool launch = ctx->step + k <= t_end;
    if (launch) {
      s = ensure_checksums(ctx, gi, g.vec != 1);
      if (s) return s;
      const int in = ctx->cur[gi], out = (in + 1) % 3;
      cur.t0 = ctx->step;
      cur.in = in;
      cur.slot = slot;
      CK(cudaMemsetAsync(&ctx->gctrl[gi].verdict, 0, sizeof(unsigned long long), ctx->stream));
      CK(run(ctx, kKSweepProt, [&] {
        return launch_sweep_tb_prot(L, g, ctx->tm_tb[4 * gi + in], ctx->tm_tb[4 * gi + 3], out, k, ctx->tbl[gi]);
      }));
      for (int tau = 1; tau <= k; ++tau) {
        gt.PA = ctx->tbl[gi].PA[tau - 1];
        gt.PB = ctx->tbl[gi].PB[tau - 1];
        const double* a_prev = tau == 1 ? g.A[in] : g.AP[tau - 2];
        const double* b_prev = tau == 1 ? g.B[in] : g.BP[tau - 2];
        double* a_out = tau == k ? g.A[out] : g.AP[tau - 1];
        double* b_out = tau == k ? g.B[out] : g.BP[tau - 1];
        CK(run(ctx, kKCheckOnline, [&] { return launch_check_tb_level(L, gt, a_prev, b_prev, a_out, b_out); }));
      }
      CK(cudaMemcpyAsync(&ctx->h_tbflag[slot], &ctx->gctrl[gi].verdict, sizeof(unsigned long long),
                         cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaEventRecord(ctx->tb_ev[slot], ctx->stream));
      ctx->cur[gi] = out;
      ctx->ref[gi] = out;
      ctx->ref_step[gi] = ctx->step + k;
      ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(g);
      ctx->step += k;
      slot ^= 1;
    }
    if (prev.t0 >= 0) {
      CK(cudaEventSynchronize(ctx->tb_ev[prev.slot]));
      if (ctx->h_tbflag[prev.slot] != 0) {  // recompute the failed pass sweep by sweep
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->cur[gi] = ctx->ref[gi] = prev.in;
        ctx->step = ctx->ref_step[gi] = prev.t0;
        ctx->ck_valid[gi] = ctx->ref_ck[gi] = online_ck(g);
        s = set_grid_step(ctx, gi, prev.t0);
        if (s) return s;
        ++ctx->tb_redo;
        for (int j = 0; j < k; ++j) {
          s = sweep_all(ctx, ABFT_MODE_ONLINE);
          if (s) return s;
        }
        prev.t0 = -1;
        continue;
      }
    }
    if (!launch) break;
    prev = cur;
  }
  while (ctx->step < t_end) {  // a remainder shorter than a pass
    s = sweep_all(ctx, ABFT_MODE_ONLINE);
    if (s) return s;
  }
  return ABFT_OK;
}

abft_status status_from_device(abft_ctx* ctx) {
  const unsigned st = ctx->h_ctrl->status;
  ctx->status_seen |= st;
  if (st & kStTimeout) return fail(ctx, ABFT_E_TIMEOUT, "a device-side wait timed out");
  if (st & kStFlipOverflow) return fail(ctx, ABFT_E_INVAL, "more than %d flips in one tile and sweep", kLocalFlips);
  if (st & kStUncorrectable)
    return fail(ctx, ABFT_E_UNCORRECTABLE, "an offline window still mismatched after its recomputation");
  if (st & kStEventOverflow) return fail(ctx, ABFT_E_TRUNCATED, "event log overflow (capacity %d)", ctx->opt.event_capacity);
  return ABFT_OK;
}

// host-side event append (rollbacks): stream-ordered copies from pinned staging
abft_status host_event(abft_ctx* ctx, int64_t step, int grid, int kind, float before, float after) {
  abft_status s = read_ctrl(ctx);
  if (s) return s;
  const unsigned long long i = ctx->h_ctrl->ev_count;
  if (i < (unsigned long long)ctx->opt.event_capacity) {
    abft_event* e = ctx->h_ev;
    memset(e, 0, sizeof *e);
    e->step = step; e->grid = grid; e->z = -1; e->y = -1; e->x = -1; e->kind = kind;
    e->before = before; e->after = after;
    CK(cudaMemcpyAsync(ctx->events + i, e, sizeof *e, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    ctx->h_ctrl->status |= kStEventOverflow;
    CK(cudaMemcpyAsync(&ctx->ctrl->status, &ctx->h_ctrl->status, sizeof(unsigned), cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  ctx->h_ctrl->ev_count = i + 1;
  CK(cudaMemcpyAsync(&ctx->ctrl->ev_count, &ctx->h_ctrl->ev_count, sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return ABFT_OK;
}

abft_status set_grid_step(abft_ctx* ctx, int gi, int64_t step) {
  ctx->h_gctrl[gi].step = step;
  CK(cudaMemcpyAsync(&ctx->gctrl[gi].step, &ctx->h_gctrl[gi].step, sizeof(long long), cudaMemcpyHostToDevice,
                     ctx->stream));
  return ABFT_OK;
}

abft_status clear_verdicts(abft_ctx* ctx) {
  for (int gi = 0; gi < ctx->n; ++gi)
    CK(cudaMemsetAsync(&ctx->gctrl[gi].verdict, 0, 2 * sizeof(unsigned long long), ctx->stream));
  return ABFT_OK;
}

// chain Theorem 1 d times from (a0, b0); returns the index of the AP/BP slot holding the result
abft_status chain(abft_ctx* ctx, int gi, const double* a0, const double* b0, int64_t d, int* slot,
                  cudaStream_t on = nullptr) {
  const GridDev& g = ctx->g[gi];
  Launch L = launcher(ctx);
  if (on) L.s = on;
  const double* a = a0;
  const double* b = b0;
  int s = 0;
  for (int64_t k = 0; k < d; ++k) {
    s = (int)(k & 1);
    CK(run(ctx, kKChain, [&] { return launch_chain(L, g, a, b, g.AP[s], g.BP[s]); }));
    a = g.AP[s];
    b = g.BP[s];
  }
  *slot = s;
  return ABFT_OK;
}

// one offline window of d sweeps (Sec. 4): checkpoint, sweep, chain, compare, roll back
abft_status offline_window(abft_ctx* ctx, int64_t d) {
  const Launch L = launcher(ctx);
  const int64_t t_start = ctx->step;
  for (int gi = 0; gi < ctx->n; ++gi) {
    abft_status s = ensure_checksums(ctx, gi);
    if (s) return s;
    ctx->ref[gi] = ctx->cur[gi];  // the checkpoint is the retained buffer itself
    ctx->ref_step[gi] = t_start;
  }
  abft_status s = clear_verdicts(ctx);
  if (s) return s;
  // The chains of Fig. 10 that need no grid (Eq. 6/7) depend only on the checkpoint's
  // checksums: they run on a side stream beside the window's sweeps and join before the
  // comparison (not while kernels are being timed one by one).
  bool side = !ctx->timing, forked = false, joined = false;
  if (side) {
    cudaError_t e = cudaSuccess;
    if (!ctx->side_stream) e = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->fork_ev) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->join_ev) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(ctx, ABFT_E_CUDA, "offline set-up: %s", cudaGetErrorString(e));
  }
  auto run_window = [&](const std::vector<int>& which) -> abft_status {
    bool all_simple = true;  // per-step chains need every intermediate state
    for (int gi : which) all_simple = all_simple && simple_chain(ctx, gi);
    const int depth = all_simple ? ctx->opt.depth : 1;
    for (int64_t k = 0; k < d; ++k) {
      if (depth >= 2 && d - 1 - k >= depth) {  // unprotected sweeps of the window, temporally blocked
        for (int gi : which) {
          const GridDev& g = ctx->g[gi];
          const int in = ctx->cur[gi], out = other_than(in, ctx->ref[gi]);
          CK(run(ctx, kKSweepPlain, [&] {
            return launch_sweep_tb(L, g, ctx->tm_tb[4 * gi + in], ctx->tm_tb[4 * gi + 3], out, depth);
          }));
          ctx->cur[gi] = out;
        }
        k += depth - 1;
        continue;
      }
      for (int gi : which) {
        GridDev g = ctx->g[gi];
        g.vec = 2;  // a window's last sweep forms both vectors whatever the online option
        const int in = ctx->cur[gi], out = other_than(in, ctx->ref[gi]);
        const bool last = k == d - 1;
        if (!simple_chain(ctx, gi)) {  // link k of the chain, with the terms of this sweep's input
          const double* a_in = k == 0 ? g.A[ctx->ref[gi]] : g.AP[(k - 1) & 1];
          const double* b_in = k == 0 ? g.B[ctx->ref[gi]] : g.BP[(k - 1) & 1];
          CK(run(ctx, kKChain,
                 [&] { return launch_chain_gen(L, g, a_in, b_in, g.u[in], g.AP[k & 1], g.BP[k & 1]); }));
        }
        if (ctx->general) {
          const int r = ctx->gen[gi].r;
          CK(run(ctx, last ? kKSweepProt : kKSweepPlain, [&] { return launch_sweep_gen(L, g, r, in, out, last); }));
        } else {
          CK(run(ctx, last ? kKSweepProt : kKSweepPlain,
                 [&] { return launch_sweep(L, g, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out, last); }));
        }
        ctx->cur[gi] = out;
      }
    }
    if (side && !joined) {  // the chains ran beside the window's sweeps
      CK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
      joined = true;
    }
    for (int gi : which) {
      GridDev g = ctx->g[gi];
      g.vec = 2;
      const int c = ctx->cur[gi];
      CK(run(ctx, kKCheckOffline, [&] { return launch_reduce_partials(L, g, c); }));
      const int slot = (int)((d - 1) & 1);
      CK(run(ctx, kKCheckOffline, [&] { return launch_compare(L, g, g.AP[slot], g.BP[slot], g.A[c], g.B[c]); }));
    }
    return ABFT_OK;
  };
  std::vector<int> all(ctx->n);
  for (int gi = 0; gi < ctx->n; ++gi) {
    all[gi] = gi;
    if (!simple_chain(ctx, gi)) continue;  // chained sweep by sweep inside the window
    if (side && !forked) {
      CK(cudaEventRecord(ctx->fork_ev, ctx->stream));
      CK(cudaStreamWaitEvent(ctx->side_stream, ctx->fork_ev, 0));
      forked = true;
    }
    int slot;
    s = chain(ctx, gi, ctx->g[gi].A[ctx->ref[gi]], ctx->g[gi].B[ctx->ref[gi]], d, &slot,
              side ? ctx->side_stream : nullptr);
    if (s) return s;
  }
  if (forked) CK(cudaEventRecord(ctx->join_ev, ctx->side_stream));
  else side = false;
  s = run_window(all);
  if (s) return s;
  s = read_ctrl(ctx);
  if (s) return s;
  std::vector<int> bad;
  for (int gi = 0; gi < ctx->n; ++gi)
    if (ctx->h_gctrl[gi].verdict) bad.push_back(gi);
  if (!bad.empty()) {  // Sec. 4.2: restore the checkpoint and recompute, without injection
    for (int gi : bad) {
      s = host_event(ctx, t_start, gi, ABFT_EV_ROLLBACK, (float)ctx->h_gctrl[gi].verdict, (float)d);
      if (s) return s;
      s = set_grid_step(ctx, gi, t_start);
      if (s) return s;
      ctx->cur[gi] = ctx->ref[gi];
      ++ctx->rollbacks;
    }
    s = clear_verdicts(ctx);
    if (s) return s;
    s = set_inject_enabled(ctx, 0);
    if (s) return s;
    s = run_window(bad);
    if (s) return s;
    s = set_inject_enabled(ctx, 1);
    if (s) return s;
    s = read_ctrl(ctx);
    if (s) return s;
    for (int gi : bad)
      if (ctx->h_gctrl[gi].verdict)
        return fail(ctx, ABFT_E_UNCORRECTABLE, "grid %d: recomputed window from step %lld still mismatches", gi,
                    (long long)t_start);
  }
  ctx->step = t_start + d;
  for (int gi = 0; gi < ctx->n; ++gi) {
    ctx->ref[gi] = ctx->cur[gi];
    ctx->ref_step[gi] = ctx->step;
    ctx->ck_valid[gi] = ctx->ref_ck[gi] = 1;
  }
  return ABFT_OK;
}

}  // namespace

// ======================================================================= C ABI

extern "C" {

void abft_default_options(abft_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->eps = 1e-5;
  o->delta = 16;
  o->acc = ABFT_ACC_FP32;
  o->event_capacity = 4096;
  o->graph_steps = 50;
  o->batch = 1;
  o->depth = 1;
  o->overlap = 1;
  o->tile_y = 0;
  o->max_flips_per_step = 64;
  o->persistent = 1;
  o->shallow = 1;
  o->boundary = ABFT_BC_CLAMP;
  o->vectors = 2;
  o->stream = nullptr;
}

size_t abft_workspace_bytes(const abft_grid* grids, int32_t n_grids, const abft_options* opt) {
  if (!opt) return 0;
  Plan P;
  if (!make_plan(grids, n_grids, *opt, &P)) return 0;
  return P.total;
}

const char* abft_status_string(abft_status s) {
  switch (s) {
    case ABFT_OK: return "ok";
    case ABFT_E_INVAL: return "invalid argument";
    case ABFT_E_CUDA: return "CUDA error";
    case ABFT_E_NOMEM: return "workspace too small";
    case ABFT_E_STATE: return "invalid state";
    case ABFT_E_TIMEOUT: return "device wait timed out";
    case ABFT_E_UNCORRECTABLE: return "uncorrectable mismatch";
    case ABFT_E_TRUNCATED: return "event log truncated";
  }
  return "unknown status";
}

const char* abft_last_error(const abft_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t abft_schedule(uint64_t seed, double rate, uint32_t bitmask, int32_t grid, int32_t n_grids, int32_t nx,
                      int32_t ny, int32_t nz, int64_t t_begin, int64_t t_end, abft_flip* out, int64_t cap) {
  const abft_grid G{nx, ny, nz};
  if (!valid_grid(G) || n_grids < 1 || grid < 0 || grid >= n_grids || t_begin < 0 || t_end < t_begin ||
      !(rate >= 0) || !std::isfinite(rate) || cap < 0 || (cap > 0 && !out))
    return -1;
  std::vector<abft_flip> fl;
  int64_t n = 0;
  for (int64_t t = t_begin; t < t_end; ++t) {
    fl.clear();
    seeded_flips(seed, rate, bitmask, grid, n_grids, G, t, &fl);
    for (const abft_flip& f : fl) {
      if (n < cap) out[n] = f;
      ++n;
    }
  }
  return n;
}

void abft_destroy(abft_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (cudaGraphExec_t& x : ctx->graph)
    if (x) cudaGraphExecDestroy(x);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->roles_ev) cudaEventDestroy(ctx->roles_ev);
  if (ctx->h_roles) cudaFreeHost(ctx->h_roles);
  if (ctx->h_flips) cudaFreeHost(ctx->h_flips);
  if (ctx->h_off) cudaFreeHost(ctx->h_off);
  if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
  if (ctx->h_gctrl) cudaFreeHost(ctx->h_gctrl);
  if (ctx->h_ev) cudaFreeHost(ctx->h_ev);
  if (ctx->h_tbflag) cudaFreeHost(ctx->h_tbflag);
  for (cudaEvent_t e : ctx->tb_ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

abft_status abft_init(abft_ctx** out, const abft_grid* grids, int32_t n_grids, const float* const* temp,
                      const float* const* power, const abft_coeffs* coeffs, const abft_options* opt,
                      void* workspace, size_t workspace_bytes) {
  if (!out) return ABFT_E_INVAL;
  *out = nullptr;
  if (!grids || n_grids < 1 || !temp || !power || !coeffs || !opt || !workspace) return ABFT_E_INVAL;
  if (((uintptr_t)workspace & 255) != 0) return ABFT_E_INVAL;
  Plan P;
  if (!make_plan(grids, n_grids, *opt, &P)) return ABFT_E_INVAL;
  if (workspace_bytes < P.total) return ABFT_E_NOMEM;
  for (int i = 0; i < n_grids; ++i)
    if (!temp[i] || !power[i]) return ABFT_E_INVAL;

  abft_ctx* ctx = new (std::nothrow) abft_ctx;
  if (!ctx) return ABFT_E_NOMEM;
  abft_status st = ABFT_OK;
  auto bail = [&](abft_status s) {
    abft_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->dev) != cudaSuccess) return bail(ABFT_E_CUDA);
  ctx->opt = *opt;
  // temporal blocking recomputes halo cells level by level, which the clamped rule
  // allows locally; other boundaries sweep one level at a time
  if (opt->boundary != ABFT_BC_CLAMP) ctx->opt.depth = 1;
  // general sets and constant boundaries run the general kernels: one launch per sweep,
  // check and location, both checksum vectors
  ctx->general = general_opts(*opt);
  ctx->opt.stencils = nullptr;  // not kept past this call
  if (ctx->general) {
    ctx->opt.depth = 1;
    ctx->opt.persistent = 0;
    ctx->opt.batch = 0;
    ctx->opt.overlap = 0;
    ctx->opt.vectors = 2;
  }
  ctx->gen.resize(n_grids);
  ctx->vanish.resize(n_grids);
  for (int i = 0; i < n_grids; ++i) {
    if (!build_gen(*opt, coeffs[i], i, &ctx->gen[i])) {
      fail(ctx, ABFT_E_INVAL, "grid %d: a stencil set needs 1..%d points with offsets within -%d..%d", i,
           kGenMaxPts, kGenRadius, kGenRadius);
      return bail(ABFT_E_INVAL);
    }
    ctx->vanish[i] = gen_vanish(ctx->gen[i], opt->boundary);
  }
  ctx->stream = (cudaStream_t)opt->stream;
  ctx->n = n_grids;
  ctx->grids.assign(grids, grids + n_grids);
  ctx->co.assign(coeffs, coeffs + n_grids);
  char* ws = (char*)workspace;
  ctx->g.resize(n_grids);
  ctx->ctrl = (DevCtrl*)(ws + P.ctrl);
  ctx->gctrl = (DevGridCtrl*)(ws + P.gctrl);
  ctx->events = (abft_event*)(ws + P.events);
  ctx->d_flips = (DevFlip*)(ws + P.flips);
  ctx->d_off = (int*)(ws + P.off);
  ctx->d_bgrid = (GridDev*)(ws + P.bgrid);
  ctx->d_btmap = (CUtensorMap*)(ws + P.btmap);
  ctx->d_roles = (BatchRole*)(ws + P.broles);
  ctx->d_bints = (int*)(ws + P.bints);
  ctx->sched_cap = P.sched_cap;
  if (cudaMallocHost(&ctx->h_flips, sizeof(DevFlip) * P.sched_cap) != cudaSuccess ||
      cudaMallocHost(&ctx->h_off, sizeof(int) * (kSchedSteps + 1)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_ctrl, sizeof(DevCtrl)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_gctrl, sizeof(DevGridCtrl) * n_grids) != cudaSuccess ||
      cudaMallocHost(&ctx->h_ev, sizeof(abft_event)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_roles, sizeof(BatchRole) * n_grids) != cudaSuccess)
    return bail(ABFT_E_NOMEM);
  if (cudaEventCreateWithFlags(&ctx->roles_ev, cudaEventDisableTiming) != cudaSuccess) return bail(ABFT_E_CUDA);
  if (cudaMallocHost(&ctx->h_tbflag, 2 * sizeof(unsigned long long)) != cudaSuccess) return bail(ABFT_E_NOMEM);
  for (cudaEvent_t& e : ctx->tb_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(ABFT_E_CUDA);
  memset(ctx->h_ctrl, 0, sizeof(DevCtrl));
  memset(ctx->h_gctrl, 0, sizeof(DevGridCtrl) * n_grids);
  for (int i = 0; i < n_grids; ++i) {
    const abft_grid& G = grids[i];
    const GridPlan& p = P.g[i];
    GridDev& g = ctx->g[i];
    memset(&g, 0, sizeof g);
    g.nx = G.nx; g.ny = G.ny; g.nz = G.nz;
    g.px = (int)align_up(G.nx, 32);
    g.ty = pick_ty(*opt, G, n_grids);
    g.shallow = is_shallow(*opt, G) ? 1 : 0;
    g.track = opt->track_residual;
    g.ntx = (G.nx + kTX - 1) / kTX;
    g.nty = (G.ny + g.ty - 1) / g.ty;
    g.pa_stride = g.ntx * kTX;
    g.pb_stride = (int)align_up(G.ny, 4);
    g.acc = opt->acc;
    g.gid = i;
    g.bc = opt->boundary;
    g.vec = ctx->opt.vectors;
    g.bval = opt->boundary_value;
    g.gs = (const GenSten*)(ws + p.gs);
    g.eps = opt->eps;
    const abft_coeffs& c = coeffs[i];
    g.k = Coef{c.cc, c.cw, c.ce, c.cn, c.cs, c.cb, c.ct};
    for (int k = 0; k < 3; ++k) {
      g.u[k] = (float*)(ws + p.u[k]);
      g.A[k] = (double*)(ws + p.A[k]);
      g.B[k] = (double*)(ws + p.B[k]);
      g.AP[k] = (double*)(ws + p.AP[k]);
      g.BP[k] = (double*)(ws + p.BP[k]);
    }
    g.C = (float*)(ws + p.C);
    g.cx = (double*)(ws + p.cx);
    g.cy = (double*)(ws + p.cy);
    g.PA = ws + p.PA;
    g.PB = ws + p.PB;
    g.PA2 = ws + p.PA2;
    g.PB2 = ws + p.PB2;
    g.fcnt = (int*)(ws + p.fcnt);
    g.fidx = (int*)(ws + p.fidx);
    g.tdirty = (int*)(ws + p.tdirty);
    g.gc = ctx->gctrl + i;
    TbLevels lvl{};
    for (int k = 0; k < 4; ++k) {
      lvl.PA[k] = ws + p.tbpa[k];
      lvl.PB[k] = ws + p.tbpb[k];
    }
    ctx->tbl.push_back(lvl);
  }
  ctx->tm_u.resize(3 * n_grids);
  ctx->tm_c.resize(n_grids);
  ctx->tm_p.resize(4 * n_grids);
  ctx->tm_tb.resize(4 * n_grids);
  ctx->cur.assign(n_grids, 0);
  ctx->ref.assign(n_grids, 0);
  ctx->ref_step.assign(n_grids, 0);
  ctx->ck_valid.assign(n_grids, 1);
  ctx->ref_ck.assign(n_grids, 1);
  cudaStream_t s = ctx->stream;
#define CKI(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      st = fail(ctx, ABFT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                    \
      fprintf(stderr, "abft_init: %s\n", ctx->err.c_str());                                    \
      return bail(st);                                                                         \
    }                                                                                          \
  } while (0)
  CKI(cudaMemsetAsync(workspace, 0, P.total, s));
  const Launch L = launcher(ctx);
  for (int i = 0; i < n_grids; ++i) {
    GridDev& g = ctx->g[i];
    const size_t rows = (size_t)g.ny * g.nz;
    CKI(cudaMemcpy2DAsync(g.u[0], g.px * 4, temp[i], (size_t)g.nx * 4, (size_t)g.nx * 4, rows, cudaMemcpyDefault, s));
    CKI(cudaMemcpy2DAsync(g.C, g.px * 4, power[i], (size_t)g.nx * 4, (size_t)g.nx * 4, rows, cudaMemcpyDefault, s));
    CKI(cudaMemcpyAsync((void*)g.gs, &ctx->gen[i], sizeof(GenSten), cudaMemcpyHostToDevice, s));
    CKI(run(ctx, kKOther, [&] { return launch_source_term(L, g, coeffs[i]); }));
    CKI(run(ctx, kKOther, [&] { return launch_checksums(L, g, g.C, g.cx, g.cy); }));
    CKI(run(ctx, kKOther, [&] { return launch_checksums(L, g, g.u[0], g.A[0], g.B[0]); }));
    char e[256];
    if (make_tensor_maps(g, g.ty, &ctx->tm_u[3 * i], &ctx->tm_c[i], e, sizeof e) != cudaSuccess ||
        make_partial_maps(g, &ctx->tm_p[4 * i], e, sizeof e) != cudaSuccess ||
        (ctx->opt.depth >= 2 &&
         make_tb_maps(g, ctx->opt.depth, &ctx->tm_tb[4 * i], &ctx->tm_tb[4 * i + 3], e, sizeof e) != cudaSuccess)) {
      st = fail(ctx, ABFT_E_CUDA, "%s", e);
      return bail(st);
    }
  }
  build_batch_tables(ctx);
  CKI(cudaMemcpyAsync(ctx->d_bgrid, ctx->g.data(), sizeof(GridDev) * n_grids, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_btmap, ctx->h_btmap.data(), sizeof(CUtensorMap) * ctx->h_btmap.size(),
                      cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_bints, ctx->h_bints.data(), sizeof(int) * ctx->h_bints.size(), cudaMemcpyHostToDevice, s));
  ctx->h_ctrl->ev_cap = opt->event_capacity;
  ctx->h_ctrl->inject_enabled = 1;
  CKI(cudaMemcpyAsync(ctx->ctrl, ctx->h_ctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, s));
  CKI(cudaStreamSynchronize(s));
#undef CKI
  *out = ctx;
  return ABFT_OK;
}

abft_status abft_inject(abft_ctx* ctx, uint64_t seed, double rate, uint32_t bitmask) {
  if (!ctx) return ABFT_E_INVAL;
  if (!(rate >= 0) || !std::isfinite(rate)) return fail(ctx, ABFT_E_INVAL, "rate must be finite and >= 0");
  if (rate > ctx->opt.max_flips_per_step) return fail(ctx, ABFT_E_INVAL, "rate above max_flips_per_step");
  ctx->inj_kind = (rate > 0 && bitmask) ? 1 : 0;
  ctx->seed = seed;
  ctx->rate = rate;
  ctx->mask = bitmask;
  ctx->list.clear();
  return ABFT_OK;
}

abft_status abft_inject_list(abft_ctx* ctx, const abft_flip* flips, int64_t n) {
  if (!ctx || n < 0 || (n > 0 && !flips)) return ABFT_E_INVAL;
  std::vector<abft_flip> v(flips, flips + n);
  for (const abft_flip& f : v) {
    if (f.grid < 0 || f.grid >= ctx->n || f.step < 0 || f.bit < 0 || f.bit > 31 || f.target != 0)
      return fail(ctx, ABFT_E_INVAL, "invalid flip entry");
    const abft_grid& G = ctx->grids[f.grid];
    if (f.x < 0 || f.x >= G.nx || f.y < 0 || f.y >= G.ny || f.z < 0 || f.z >= G.nz)
      return fail(ctx, ABFT_E_INVAL, "flip outside grid %d", f.grid);
  }
  std::stable_sort(v.begin(), v.end(), [](const abft_flip& a, const abft_flip& b) {
    return a.step < b.step || (a.step == b.step && a.grid < b.grid);
  });
  ctx->list.swap(v);
  ctx->inj_kind = ctx->list.empty() ? 0 : 2;
  return ABFT_OK;
}

abft_status abft_step(abft_ctx* ctx, int64_t n, int32_t mode) {
  if (!ctx) return ABFT_E_INVAL;
  if (n < 0 || mode < 0 || mode > 2) return fail(ctx, ABFT_E_INVAL, "bad step count or mode");
  if (ctx->status_seen & kStTimeout) return fail(ctx, ABFT_E_TIMEOUT, "context poisoned by an earlier timeout");
  ctx->verified = false;
  const int64_t t_end = ctx->step + n;
  abft_status s = ABFT_OK;
  while (ctx->step < t_end) {
    int64_t want = std::min<int64_t>(t_end - ctx->step, kSchedSteps);
    bool persist_off = false;
    if (mode == ABFT_MODE_OFFLINE) {
      const int64_t delta = std::max<int64_t>(ctx->opt.delta, 1);
      persist_off = ctx->opt.persistent != 0;
      for (int gi = 0; gi < ctx->n && persist_off; ++gi)
        persist_off = persistent_offline_fits(ctx->g[gi]) && simple_chain(ctx, gi);
      if (persist_off) {
        if (want > delta && want < t_end - ctx->step) want -= want % delta;  // whole windows per launch
      } else {
        want = std::min<int64_t>(want, delta);
      }
    }
    int64_t covered = 0;
    s = upload_schedule(ctx, ctx->step, want, &covered);
    if (s) return s;
    if (mode == ABFT_MODE_OFFLINE) {
      if (persist_off) {
        const int64_t delta = std::max<int64_t>(ctx->opt.delta, 1);
        if (covered > delta && covered < t_end - ctx->step) covered -= covered % delta;
        s = persistent_offline_all(ctx, covered);
      } else {
        s = offline_window(ctx, covered);
      }
      if (s) return s;
      continue;
    }
    if (ctx->opt.batch && ctx->n > 1 && covered > 0) {
      s = batch_all(ctx, covered, mode);
      if (s) return s;
      continue;
    }
    bool persist = ctx->opt.persistent && covered > 0;
    for (int gi = 0; gi < ctx->n && persist; ++gi) persist = persistent_fits(ctx->g[gi], mode == ABFT_MODE_ONLINE);
    if (persist) {
      s = persistent_all(ctx, covered, mode);
      if (s) return s;
      continue;
    }
    for (int64_t k = 0; k < covered; ++k) {
      if (mode == ABFT_MODE_NONE && ctx->opt.depth >= 2 && covered - k >= ctx->opt.depth) {
        s = tb_all(ctx);
        if (s) return s;
        k += ctx->opt.depth - 1;
        continue;
      }
      if (mode == ABFT_MODE_ONLINE)
        for (int gi = 0; gi < ctx->n; ++gi) {
          s = ensure_checksums(ctx, gi, ctx->g[gi].vec != 1);
          if (s) return s;
        }
      if (mode == ABFT_MODE_ONLINE && online_tb_ok(ctx) && covered - k >= ctx->opt.depth) {
        s = online_tb(ctx, covered - k);
        if (s) return s;
        break;
      }
      if (mode == ABFT_MODE_ONLINE && ctx->n == 1 && ctx->opt.overlap && !ctx->timing) {
        s = online_overlap(ctx, covered - k);
        if (s) return s;
        break;
      }
      s = sweep_all(ctx, mode);
      if (s) return s;
    }
  }
  s = read_ctrl(ctx);
  if (s) return s;
  return status_from_device(ctx);
}

abft_status abft_verify(abft_ctx* ctx, int64_t* n_mismatch) {
  if (!ctx || !n_mismatch) return ABFT_E_INVAL;
  const Launch L = launcher(ctx);
  abft_status s = clear_verdicts(ctx);
  if (s) return s;
  ctx->v_dist.assign(ctx->n, 0);
  for (int gi = 0; gi < ctx->n; ++gi) {
    GridDev g = ctx->g[gi];
    g.vec = 2;  // verification compares both vectors whatever the online option
    const int c = ctx->cur[gi], r = ctx->ref[gi];
    const int64_t d = ctx->step - ctx->ref_step[gi];
    ctx->v_dist[gi] = d;
    const bool simple = simple_chain(ctx, gi);
    if (d > 1 && !simple && !ctx->vanish[gi])
      return fail(ctx, ABFT_E_INVAL,
                  "verification %lld sweeps past the verified state needs vanishing boundary terms (grid %d)",
                  (long long)d, gi);
    if (ctx->ref_ck[gi] != 1) {  // one-vector checks left a of the verified state unsummed
      CK(run(ctx, kKOther, [&] { return launch_checksums(L, g, g.u[r], g.A[r], g.B[r]); }));
      ctx->ref_ck[gi] = 1;
      if (r == c) ctx->ck_valid[gi] = 1;
    }
    CK(run(ctx, kKOther, [&] { return launch_checksums(L, g, g.u[c], g.AP[2], g.BP[2]); }));
    const double* pa = g.A[r];
    const double* pb = g.B[r];
    if (d > 0 && simple) {
      int slot;
      s = chain(ctx, gi, g.A[r], g.B[r], d, &slot);
      if (s) return s;
      pa = g.AP[slot];
      pb = g.BP[slot];
    } else if (d > 0) {  // one sweep: the terms of the verified state; more: the terms vanish
      for (int64_t k = 0; k < d; ++k) {
        const double* a_in = k == 0 ? g.A[r] : g.AP[(k - 1) & 1];
        const double* b_in = k == 0 ? g.B[r] : g.BP[(k - 1) & 1];
        const float* us = d == 1 ? g.u[r] : nullptr;
        CK(run(ctx, kKChain, [&] { return launch_chain_gen(L, g, a_in, b_in, us, g.AP[k & 1], g.BP[k & 1]); }));
      }
      pa = g.AP[(d - 1) & 1];
      pb = g.BP[(d - 1) & 1];
    }
    CK(run(ctx, kKCheckOffline, [&] { return launch_compare(L, g, pa, pb, g.AP[2], g.BP[2]); }));
  }
  s = read_ctrl(ctx);
  if (s) return s;
  int64_t tot = 0;
  ctx->v_fail.assign(ctx->n, 0);
  for (int gi = 0; gi < ctx->n; ++gi) {
    ctx->v_fail[gi] = ctx->h_gctrl[gi].verdict;
    tot += (int64_t)ctx->h_gctrl[gi].verdict;
  }
  ctx->verified = true;
  *n_mismatch = tot;
  return status_from_device(ctx);
}

abft_status abft_correct(abft_ctx* ctx, int64_t* n_fixed) {
  if (!ctx || !n_fixed) return ABFT_E_INVAL;
  if (!ctx->verified) return fail(ctx, ABFT_E_STATE, "abft_correct needs a preceding abft_verify");
  const Launch L = launcher(ctx);
  *n_fixed = 0;
  abft_status s = ABFT_OK;
  for (int gi = 0; gi < ctx->n; ++gi) {
    if (!ctx->v_fail[gi]) continue;
    const GridDev& g = ctx->g[gi];
    const int64_t d = ctx->v_dist[gi];
    if (d == 0) {  // Eq. (8) against the stored checksums of this very state
      const int c = ctx->cur[gi];
      CK(cudaMemsetAsync(&ctx->gctrl[gi].unresolved, 0, sizeof(unsigned long long), ctx->stream));
      CK(run(ctx, kKOther, [&] { return launch_correct_planes(L, g, c, g.A[c], g.B[c]); }));
      s = read_ctrl(ctx);
      if (s) return s;
      if (ctx->h_gctrl[gi].unresolved)
        return fail(ctx, ABFT_E_UNCORRECTABLE, "grid %d: mismatch pattern cannot be located", gi);
      *n_fixed += (int64_t)ctx->v_fail[gi] / 2;
    } else {  // Sec. 4.2: roll back to the verified state and recompute d sweeps
      CK(cudaStreamSynchronize(ctx->stream));
      s = set_grid_step(ctx, gi, ctx->ref_step[gi]);
      if (s) return s;
      s = host_event(ctx, ctx->ref_step[gi], gi, ABFT_EV_ROLLBACK, (float)ctx->v_fail[gi], (float)d);
      if (s) return s;
      s = set_inject_enabled(ctx, 0);
      if (s) return s;
      ctx->cur[gi] = ctx->ref[gi];
      for (int64_t k = 0; k < d; ++k) {
        const int in = ctx->cur[gi], out = other_than(in, ctx->ref[gi]);
        if (ctx->general) {
          const int rr = ctx->gen[gi].r;
          CK(run(ctx, kKSweepPlain, [&] { return launch_sweep_gen(L, g, rr, in, out, false); }));
        } else {
          CK(run(ctx, kKSweepPlain,
                 [&] { return launch_sweep(L, g, ctx->tm_u[3 * gi + in], ctx->tm_c[gi], in, out, false); }));
        }
        ctx->cur[gi] = out;
      }
      s = set_inject_enabled(ctx, 1);
      if (s) return s;
      ++ctx->rollbacks;
      *n_fixed += d;
    }
    ctx->ck_valid[gi] = 0;
  }
  ctx->verified = false;
  s = read_ctrl(ctx);
  if (s) return s;
  return status_from_device(ctx);
}

abft_status abft_events(abft_ctx* ctx, abft_event* buf, int64_t cap, int64_t* n_out) {
  if (!ctx || !n_out || cap < 0 || (cap > 0 && !buf)) return ABFT_E_INVAL;
  abft_status s = read_ctrl(ctx);
  if (s) return s;
  const int64_t n = (int64_t)ctx->h_ctrl->ev_count;
  const int64_t kept = std::min<int64_t>(n, ctx->opt.event_capacity);
  const int64_t m = std::min<int64_t>(kept, cap);
  if (m > 0) CK(cudaMemcpy(buf, ctx->events, sizeof(abft_event) * m, cudaMemcpyDeviceToHost));
  *n_out = n;
  return n > ctx->opt.event_capacity ? fail(ctx, ABFT_E_TRUNCATED, "event log overflow") : ABFT_OK;
}

abft_status abft_read(abft_ctx* ctx, int32_t grid, float* dst) {
  if (!ctx || !dst || grid < 0 || grid >= ctx->n) return ABFT_E_INVAL;
  const GridDev& g = ctx->g[grid];
  CK(cudaMemcpy2DAsync(dst, (size_t)g.nx * 4, g.u[ctx->cur[grid]], (size_t)g.px * 4, (size_t)g.nx * 4,
                       (size_t)g.ny * g.nz, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return ABFT_OK;
}

abft_status abft_read_checksums(abft_ctx* ctx, int32_t grid, double* a, double* b) {
  if (!ctx || !a || !b || grid < 0 || grid >= ctx->n) return ABFT_E_INVAL;
  abft_status s = ensure_checksums(ctx, grid);
  if (s) return s;
  const GridDev& g = ctx->g[grid];
  const int c = ctx->cur[grid];
  CK(cudaMemcpyAsync(a, g.A[c], sizeof(double) * g.nz * g.nx, cudaMemcpyDefault, ctx->stream));
  CK(cudaMemcpyAsync(b, g.B[c], sizeof(double) * g.nz * g.ny, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return ABFT_OK;
}

abft_status abft_current(abft_ctx* ctx, int32_t grid, float** dev_ptr, int64_t* pitch) {
  if (!ctx || !dev_ptr || !pitch || grid < 0 || grid >= ctx->n) return ABFT_E_INVAL;
  *dev_ptr = ctx->g[grid].u[ctx->cur[grid]];
  *pitch = ctx->g[grid].px;
  return ABFT_OK;
}

abft_status abft_get_counters(const abft_ctx* ctx, abft_counters* out) {
  if (!ctx || !out) return ABFT_E_INVAL;
  out->steps_done = ctx->step;
  out->kernel_launches = ctx->launches;
  out->events = (int64_t)ctx->h_ctrl->ev_count;
  int64_t dev_rollbacks = 0;
  for (int gi = 0; gi < ctx->n; ++gi) dev_rollbacks += ctx->h_gctrl[gi].rollbacks;
  out->rollbacks = ctx->rollbacks + dev_rollbacks;
  out->flips_scheduled = ctx->flips_scheduled;
  double mr = 0.0;
  for (int gi = 0; gi < ctx->n; ++gi) {
    double v;
    memcpy(&v, &ctx->h_gctrl[gi].max_resid, sizeof v);
    mr = std::max(mr, v);
  }
  out->max_residual = mr;
  out->passes_recomputed = ctx->tb_redo;
  return ABFT_OK;
}

abft_status abft_time_kernels(abft_ctx* ctx, int64_t n, int32_t mode, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return ABFT_E_INVAL;
  for (int k = 0; k < ABFT_KERNEL_KINDS; ++k) { ms[k] = 0; launches[k] = 0; }
  ctx->timing = true;
  ctx->ev_used = 0;
  ctx->ev_kind.clear();
  abft_status s = abft_step(ctx, n, mode);
  ctx->timing = false;
  if (s != ABFT_OK && s != ABFT_E_TRUNCATED) return s;
  CK(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < ctx->ev_kind.size(); ++i) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]));
    ms[ctx->ev_kind[i]] += t;
    launches[ctx->ev_kind[i]] += 1;
  }
  return s;
}

}  // extern "C"
