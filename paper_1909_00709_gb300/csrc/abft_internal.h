// Internal declarations shared by the library's translation units (host + device).
// Not part of the public ABI; see include/abft.h for that.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "abft.h"

namespace abft {

constexpr int kTX = 128;          // sweep tile width: one warp, one float4 per lane
constexpr int kHaloX = 4;         // x halo of a TMA tile (16-byte aligned start)
constexpr int kUW = kTX + 2 * kHaloX;  // width of the staged u tile
constexpr int kFCap = 64;         // failing entries kept per plane and vector
constexpr int kLocalFlips = 32;   // flips a tile can apply in one sweep
constexpr int kSchedSteps = 4096; // sweeps covered by one uploaded schedule chunk
constexpr int kShallowMaxZ = 16;  // grids this shallow are swept with whole-column tiles
// rows of the whole-column tiles of a grid swept alone with the default tile height (7 or 8)
int balanced_shallow_rows(const abft_grid& G);
constexpr unsigned kSpinLimit = 1u << 26;  // bound of every device-side mbarrier wait loop
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000 * 1000 * 1000;  // grid barrier wait bound
constexpr unsigned long long kWaitTimeoutNs = 4ull * 1000 * 1000 * 1000;     // mbarrier wait bound

// sticky device status bits
enum : unsigned {
  kStTimeout = 1u,        // a TMA/mbarrier wait gave up
  kStFlipOverflow = 2u,   // more flips in one tile and sweep than kLocalFlips
  kStEventOverflow = 4u,  // event log full
  kStFailOverflow = 8u,   // more failing entries in a plane than kFCap (plane recomputed)
  kStUncorrectable = 16u  // an offline window still mismatched after its recomputation
};

// kernel kinds for launch accounting and abft_time_kernels
enum KernelKind { kKSweepPlain = 0, kKSweepProt = 1, kKCheckOnline = 2, kKCheckOffline = 3,
                  kKChain = 4, kKOther = 5, kKPersistPlain = 6, kKPersistProt = 7 };

struct Coef {
  float cc, cw, ce, cn, cs, cb, ct;
};

// A general stencil set S of Eq. (1) (Sec. 3.1), offsets within -2..2 on every axis,
// in the order the update sums them; device copy per grid (the general path).
constexpr int kGenMaxPts = 32;  // ABFT_MAX_POINTS
constexpr int kGenRadius = 2;
constexpr int kGenTY = 8;       // rows per tile of the general sweep (its partial checksums' tiles)
struct GenSten {
  int npts;
  int r;  // largest |offset| over the set (1 or 2; 0 for a centre-only set)
  int dx[kGenMaxPts], dy[kGenMaxPts], dz[kGenMaxPts];
  float w[kGenMaxPts];
};

// device-resident control block of a context
struct DevCtrl {
  unsigned int status;
  int inject_enabled;
  long long sched_t0;       // sweep index of schedule offset 0
  int sched_n;              // sweeps covered by the uploaded schedule
  int ev_cap;
  unsigned long long ev_count;
  unsigned long long verdict;  // failing entries found by the last offline/verify check
};

// per-grid device counters
struct DevGridCtrl {
  long long step;           // sweeps committed on this grid
  unsigned int done_sweep;  // last-block tickets
  unsigned int done_check;
  unsigned int done_aux;
  unsigned int rollbacks;   // offline windows the persistent kernel recomputed
  unsigned int fails[3];    // failing entries found by the persistent kernel, by sweep index mod 3
  unsigned int redo;         // 1: a correction was made after the next sweep had started (per-launch overlap)
  unsigned int nbz;          // one-vector checks: planes whose b failed this sweep (list bz)
  unsigned int pad;          // keeps bar 8-byte aligned right after
  unsigned long long bar;   // grid barrier of the persistent kernel: arrivals since launch
  unsigned long long bars[3];  // payload barrier (online kernel): per instance mod 3, arrivals | payload << 32
  unsigned long long verdict;  // failing entries of the last offline/verify comparison
  unsigned long long unresolved;  // planes a zero-distance correction could not fix
  unsigned long long max_resid;   // bits of the largest |a'-a|/|a| of a passing entry (when tracked)
  int bz[64];                     // the first of those planes (kBzCap)
};
constexpr int kBzCap = 64;

// everything a kernel needs to know about one grid (passed by value)
struct GridDev {
  int nx, ny, nz, px;       // px: row pitch in elements (multiple of 32)
  int ntx, nty, ty;         // sweep tiles along x and y, rows per tile
  int pa_stride;            // row stride of the a-partials (ntx * kTX)
  int pb_stride;            // row stride of the b-partials (ny rounded up to a multiple of 4)
  int acc;                  // abft_acc
  int shallow;              // 1: whole-column tiles (all nz planes staged at once)
  int track;                // 1: keep the running maximum of the passing residuals
  int gid;
  int bc;                   // abft_boundary: what a neighbour outside the grid reads
  int vec;                  // checksum vectors the online check tests every sweep (2: a and b; 1: b)
  float bval;               // ABFT_BC_CONST: the value of every cell outside the grid
  Coef k;
  const GenSten* gs;        // the grid's stencil set as a general set (device memory)
  double eps;
  float* u[3];              // state buffers
  float* C;                 // constant term, same pitch
  double* cx; double* cy;   // checksums of C (Theorem 1's c_x, c_y)
  double* A[3]; double* B[3];  // checksums of the state held in u[i]
  double* AP[3]; double* BP[3];  // interpolated vectors (prediction, chain ping-pong, fresh sums)
  void* PA; void* PB;       // per-tile partial checksums of the last protected sweep
  void* PA2; void* PB2;     // second set: the persistent kernel alternates by sweep parity
  int* fcnt;                // [nz][2] failing-entry counts (a, b)
  int* fidx;                // [nz][2][kFCap] failing indices
  int* tdirty;              // [2][nty*ntx] per tile: highest marked plane + 1, nz - lowest marked plane
                            // (0 = clean): planes whose sweep must be repaired after a late correction
  DevGridCtrl* gc;
};

// device flip entry (same layout as abft_flip)
struct DevFlip { long long step; int grid, z, y, x, bit, target; };

struct DevSched {
  const DevFlip* flips;
  const int* off;           // off[i]..off[i+1]: flips of sweep sched_t0 + i (all grids)
  // copies of the control block's injection fields, constant during a launch
  int enabled;
  int n;
  long long t0;
  // read them once, at the start of a kernel
  __device__ __forceinline__ void load(const DevCtrl* c) {
    enabled = c->inject_enabled;
    t0 = c->sched_t0;
    n = c->sched_n;
  }
};

// host-side launchers (defined in sweep.cu / check.cu); all enqueue on `s`
struct Launch {
  cudaStream_t s;
  DevCtrl* ctrl;
  abft_event* events;
  DevSched sched;
};

cudaError_t make_tensor_maps(const GridDev& g, int ty, CUtensorMap tm_u[3], CUtensorMap* tm_c,
                             char* err, size_t errlen);
// tensor maps of the partial buffers as seen by the persistent kernel's check warp:
// [0] PA, [1] PA2, [2] PB, [3] PB2; boxes of 32 entries by all tiles of one plane
cudaError_t make_partial_maps(const GridDev& g, CUtensorMap tm[4], char* err, size_t errlen);
constexpr int kCheckBox = 32;  // entries per check-warp round
int sweep_smem_bytes(int ty, bool prot);
cudaError_t launch_sweep(const Launch& L, const GridDev& g, const CUtensorMap& tm_in,
                         const CUtensorMap& tm_c, int in, int out, bool prot);
// repair the sweep in -> out just committed where a late correction of u[in] reached
// (tiles and planes marked by k_resolve; nothing unless the grid's redo flag is set)
cudaError_t launch_redo_tiles(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                              int in, int out);
cudaError_t launch_source_term(const Launch& L, const GridDev& g, const abft_coeffs& co);
cudaError_t launch_checksums(const Launch& L, const GridDev& g, const float* u, double* A, double* B);
// the tensor maps of a grid's partial buffers PA, PA2, PB, PB2 (make_partial_maps)
struct PartialMaps {
  CUtensorMap m[4];
};
// max_warps caps the box check's warps per block (1 lets it run beside a sweep's CTAs)
cudaError_t launch_check_online(const Launch& L, const GridDev& g, const PartialMaps& pm, int in, int out,
                                int max_warps = 8);
// the box check needs at most 256 tiles along x and along y
bool check_box_usable(const GridDev& g);
int check_box_bytes_host(int nty, int ntx, int acc);
// 32-entry rounds of one online check (only the b entries with one vector)
inline long long check_rounds_host(const GridDev& g) {
  return (long long)g.nz * ((g.vec == 1 ? 0 : (g.nx + kCheckBox - 1) / kCheckBox) + (g.ny + kCheckBox - 1) / kCheckBox);
}
// entries [first, nz (nx + ny)) of one online check: a[z][x] first, then b[z][y]
inline long long check_entries_first(const GridDev& g) { return g.vec == 1 ? (long long)g.nz * g.nx : 0; }
int check_box_warps(int box_bytes);
// location and correction after launch_check_online, one block per plane
// `step`: the sweep whose output is checked (event stamps); a resolved plane sets the
// grid's redo flag
cudaError_t launch_resolve(const Launch& L, const GridDev& g, int in, int out, long long step);
cudaError_t launch_reduce_partials(const Launch& L, const GridDev& g, int out);
cudaError_t launch_chain(const Launch& L, const GridDev& g, const double* a_in, const double* b_in,
                         double* a_out, double* b_out);
cudaError_t launch_compare(const Launch& L, const GridDev& g, const double* ap, const double* bp,
                           const double* a, const double* b);
cudaError_t launch_persistent(const Launch& L, const GridDev& g, const CUtensorMap tm_u[3], const CUtensorMap& tm_c,
                              const CUtensorMap tm_p[4], long long step0, int n_steps, int first_in, int p, int q,
                              bool prot, int* blocks);
// offline windows of `delta` sweeps from checkpoint buffer `ck` (Sec. 4), in one launch
cudaError_t launch_persistent_offline(const Launch& L, const GridDev& g, const CUtensorMap tm_u[3],
                                      const CUtensorMap& tm_c, long long step0, int n_steps, int delta, int ck,
                                      int* blocks);
bool persistent_offline_fits(const GridDev& g);
bool persistent_fits(const GridDev& g, bool prot);
cudaError_t launch_correct_planes(const Launch& L, const GridDev& g, int cur, const double* ap,
                                  const double* bp);

// ------------------------------------------------------------ general stencil sets
// Eq. (1) with any set S of radius <= 2 and every boundary rule (general.cu): the sweep
// with fused partial checksums (same partial layout as the 7-point tiles, so the
// reductions of check.cu apply), the online check (Theorem 1 with literal boundary
// terms), location and correction, and one link of an offline chain with per-step
// boundary terms (u: the state the step starts from; nullptr when the terms vanish).
int gen_sweep_smem(const GridDev& g, int r);
cudaError_t launch_sweep_gen(const Launch& L, const GridDev& g, int r, int in, int out, bool prot);
cudaError_t launch_check_gen(const Launch& L, const GridDev& g, int in, int out);
cudaError_t launch_resolve_gen(const Launch& L, const GridDev& g, int in, int out, long long step);
cudaError_t launch_chain_gen(const Launch& L, const GridDev& g, const double* a_in, const double* b_in,
                             const float* u, double* a_out, double* b_out);

// ------------------------------------------------------------ temporal blocking
// k (2..4) unprotected sweeps in one pass; maps with boxes of 136 columns by 8 + 2k rows
constexpr int kTbRows = 8;
cudaError_t make_tb_maps(const GridDev& g, int k, CUtensorMap tm_u[3], CUtensorMap* tm_c, char* err, size_t errlen);
cudaError_t launch_sweep_tb(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                            int out, int k);
// Online checks with temporal blocking: a protected pass of k sweeps writes the FP32
// partial checksums of every level tau (1..k) into PA[tau-1] (a, with two vectors) and
// PB[tau-1] (b), tiles of kTbRows rows; then one check launch per level.
struct TbLevels {
  void* PA[4];
  void* PB[4];
};
cudaError_t launch_sweep_tb_prot(const Launch& L, const GridDev& g, const CUtensorMap& tm_in, const CUtensorMap& tm_c,
                                 int out, int k, const TbLevels& lp);
// gt: the grid with PA/PB of the level and nty/ty of kTbRows-row tiles; failing entries
// are added to gt.gc->verdict
cudaError_t launch_check_tb_level(const Launch& L, const GridDev& gt, const double* a_prev, const double* b_prev,
                                  double* a_out, double* b_out);

// ------------------------------------------------------------ batched grids
// Buffer roles of sweep s of one grid in a batched run that started at sweep s0.
// mode 1 (protected): in = (first + s - s0) mod 3, out = in + 1 mod 3.
// mode 0 (unprotected): sweep s0 reads `first` and writes `a`; later sweeps go
// a -> b at odd offsets and b -> a at even ones.
struct BatchRole {
  long long s0;
  int first, a, b, mode;
};

// one batched launch: the blocks of `n` grids, grid grids[i] owning blocks
// off[i] .. off[i+1]-1 (all arrays in device memory)
constexpr int kBatchMaps = 8;  // tensor maps per grid: u[0], u[1], u[2], C, PA, PA2, PB, PB2
struct BatchArgs {
  const GridDev* g;          // [n_grids]
  const CUtensorMap* tm;     // [n_grids][kBatchMaps]
  const BatchRole* roles;    // [n_grids]
  const int* grids;
  const int* off;            // [n + 1]
  int n;
};
constexpr int kBatchRounds = 128;    // most 32-entry check rounds per block of the batched check (16 per warp)
constexpr int kBatchMinRounds = 16;  // fewest (2 per warp)
int batch_sweep_smem(int shallow, int ty, int nz);
// bc: the grids' abft_boundary (one rule per context)
cudaError_t batch_prepare(int shallow, int ty, bool prot, int acc, int bc, int smem);
cudaError_t launch_sweep_batch(const Launch& L, const BatchArgs& a, int blocks, int smem, int shallow, int ty,
                               bool prot, int acc, int bc);
// box > 0: the partials come in TMA boxes of `box` bytes, nw warps per block, `smem`
// bytes of dynamic shared memory; box == 0: plain loads, 8 warps per block
cudaError_t launch_check_batch(const Launch& L, const BatchArgs& a, int blocks, int acc, int box, int nw, int smem);
cudaError_t batch_check_prepare(int acc, int smem);

}  // namespace abft
