/*
 * abft.h - C ABI of the GB300 (sm_103a) library for algorithm-based fault tolerance
 * of 3D stencil sweeps, after Cavelan & Ciorba, "Algorithm-Based Fault Tolerance for
 * Parallel Stencil Computations" (arXiv 1909.00709).
 *
 * What the library computes, per grid of nx*ny*nz FP32 points u[z][y][x]:
 *   - the sweep of Eq. (1) with the 7-point HotSpot3D set S (centre, x-1, x+1, y-1,
 *     y+1, z-1, z+1) and the constant term C = sdc*P + c_amb*t_amb, with clamped
 *     boundaries (an out-of-range neighbour is the centre, Fig. 2), or periodic or
 *     empty (zero) ones (Sec. 3.3, "Dealing with Boundary Conditions"); or, through
 *     option `stencils`, Eq. (1) with any set S of offsets within -2..2 (Sec. 3.1:
 *     a 13-point star, the 27-point box, asymmetric weights), and with constant
 *     boundaries (every cell outside the grid holds one value);
 *   - per-plane row and column checksums a[z][x] = sum_y u, b[z][y] = sum_x u
 *     (Eq. 2, 3), fused into the sweep (both every sweep, or, as Sec. 3.2 recommends,
 *     b every sweep and a only in planes where b failed: option `vectors`);
 *   - the interpolated checksums of Theorem 1 (Eq. 4, 5; boundary terms alpha, beta
 *     in closed form for each boundary rule; zero for the periodic one, which gives
 *     the simple form of Eq. 6, 7), the relative test of Sec. 3.4, location
 *     at the intersection of the failing row and column, and the correction of
 *     Eq. (8) / Fig. 9, every sweep (online mode, Sec. 3);
 *   - the offline mode of Sec. 4: a checkpoint every Delta sweeps, Theorem 1 chained
 *     Delta times (Fig. 10), one comparison per window and rollback on a mismatch;
 *     where the boundary terms alpha, beta do not vanish, each link of the chain takes
 *     them from the state its sweep starts from (Theorem 1 defines them from u^t).
 *
 * Conventions for every call:
 *   - Every function returns an abft_status and never throws or aborts.  On failure
 *     abft_last_error(ctx) holds a one-line message.
 *   - Device memory is owned by the caller.  abft_init borrows one device workspace
 *     of at least abft_workspace_bytes() bytes for the lifetime of the context; the
 *     library itself never calls cudaMalloc.  Host-side state (schedules, graphs,
 *     the context) is owned by the library and freed by abft_destroy.
 *   - All device work is enqueued on opt->stream (a cudaStream_t; NULL = the
 *     legacy default stream).  Calls that return device results to the host
 *     (abft_step, abft_verify, abft_correct, abft_events, abft_read) synchronise that
 *     stream before returning.
 *   - Arrays are row-major with x fastest: index (z*ny + y)*nx + x.
 *   - Not thread-safe: one host thread per context at a time.
 */
#ifndef ABFT_H
#define ABFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ABFT_API __attribute__((visibility("default")))
#else
#define ABFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct abft_ctx abft_ctx; /* opaque, library-owned */

typedef enum {
  ABFT_OK = 0,
  ABFT_E_INVAL = 1,         /* an argument is out of range or inconsistent */
  ABFT_E_CUDA = 2,          /* a CUDA runtime call failed */
  ABFT_E_NOMEM = 3,         /* workspace smaller than abft_workspace_bytes(), or host allocation failed */
  ABFT_E_STATE = 4,         /* the call is not valid in the context's current state */
  ABFT_E_TIMEOUT = 5,       /* a bounded device-side wait gave up; the context is poisoned */
  ABFT_E_UNCORRECTABLE = 6, /* a mismatch survived correction (offline: the recomputed window failed too) */
  ABFT_E_TRUNCATED = 7      /* more events than event_capacity; the first ones were kept */
} abft_status;

typedef enum {
  ABFT_MODE_NONE = 0,    /* unprotected sweeps (the paper's No-ABFT baseline) */
  ABFT_MODE_ONLINE = 1,  /* detect and correct after every sweep (Sec. 3) */
  ABFT_MODE_OFFLINE = 2  /* detect every Delta sweeps, roll back on a mismatch (Sec. 4) */
} abft_mode;

typedef enum {
  ABFT_ACC_FP32 = 0,     /* FP32 tile sums, FP64 across tiles */
  ABFT_ACC_TWOSUM = 1,   /* compensated (TwoSum) FP32 tile sums, FP64 across tiles */
  ABFT_ACC_FP64 = 2      /* FP64 accumulation from the first add */
} abft_acc;

/* Boundary rule of Eq. (1) for a neighbour outside the grid, on every axis (Sec. 3.3,
   "Dealing with Boundary Conditions"). */
typedef enum {
  ABFT_BC_CLAMP = 0,     /* the centre point (Fig. 2) */
  ABFT_BC_PERIODIC = 1,  /* the point on the opposite face; alpha = beta = 0 in Theorem 1 */
  ABFT_BC_ZERO = 2,      /* zero ("empty" boundaries) */
  ABFT_BC_CONST = 3      /* the constant abft_options.boundary_value (a fixed temperature, say) */
} abft_boundary;

/* One point (i, j, k) of a stencil set S with its weight (Sec. 3.1's {i, j, w}, with a z
   offset k for 3D): Eq. (1) adds w * u[z+dz][y+dy][x+dx].  Offsets within -2..2. */
typedef struct { int32_t dx, dy, dz; float w; } abft_point;

#define ABFT_MAX_POINTS 32
/* A stencil set S of 1..ABFT_MAX_POINTS points, summed in this order. */
typedef struct { int32_t npts; abft_point pts[ABFT_MAX_POINTS]; } abft_stencil;

typedef enum {
  ABFT_EV_CORRECTED = 1,  /* Eq. (8) applied at (z, y, x); before/after hold the values */
  ABFT_EV_RECOMPUTED = 2, /* a flagged line recomputed from u^t: row y (x = -1) or column x (y = -1) */
  ABFT_EV_ROLLBACK = 3    /* offline window starting at `step` restored and recomputed */
} abft_event_kind;

/* one grid; the library pads rows to a pitch that is a multiple of 32 elements */
typedef struct { int32_t nx, ny, nz; } abft_grid;

/* Stencil weights of Eq. (1) (cw/ce: x-1/x+1, cn/cs: y-1/y+1, cb/ct: z-1/z+1) and
   the source-term constants C = sdc*P + c_amb*t_amb. */
typedef struct { float cc, cw, ce, cn, cs, cb, ct, sdc, c_amb, t_amb; } abft_coeffs;

typedef struct {
  double eps;               /* detection threshold of Sec. 3.4 (paper: 1e-5) */
  int32_t delta;            /* offline detection period (paper: 16) */
  int32_t acc;              /* abft_acc */
  int32_t event_capacity;   /* events kept on the device (>= 1) */
  int32_t graph_steps;      /* sweeps per captured CUDA graph; 0 disables graphs */
  int32_t tile_y;           /* rows per sweep tile (8, 16 or 32); 0 = library default: 16 for
                               streaming tiles, 8 for whole-column tiles, or 7 in a context of
                               one grid where 7-row tiles put fewer rows on the busiest SM (a
                               sweep ends when its slowest SM does); the tuner may return 0 */
  int32_t max_flips_per_step; /* schedule capacity per step and grid (<= 511) */
  int32_t persistent;       /* 1: run online/unprotected sweeps in one persistent cooperative
                               launch per grid and schedule chunk where the grid's tiles fit one per
                               CTA (unprotected: also several per CTA when two CTAs fit per SM);
                               0: one launch per kernel */
  int32_t shallow;          /* 1: grids with nz <= 16 use whole-column tiles (all planes staged
                               at once); 0: always stream the planes */
  int32_t track_residual;   /* 1: keep the largest relative residual |a'-a|/|a| of the entries
                               that pass (abft_counters.max_residual); costs one atomic per entry */
  int32_t depth;            /* temporal blocking: unprotected sweeps (mode NONE, and the sweeps of
                               an offline window before its last) advance `depth` (1..4) sweeps per
                               pass over the grid where a grid is swept launch by launch; 1 = off.
                               Online checks of a single grid launched sweep by sweep (FP32
                               checksums, boundary terms that vanish) also run in passes: each pass
                               writes every level's partial checksums, every level is checked
                               (Theorem 1 from the level before, Sec. 3.4), and a pass with a
                               failing entry is recomputed sweep by sweep with the online check of
                               every sweep, which locates, corrects and logs as single sweeps do.
                               Used with the clamped boundary only (others sweep one at a time). */
  int32_t overlap;          /* 1: a single grid checked online launch by launch (too large for the
                               persistent kernel) runs each sweep's check beside the next sweep and
                               recomputes that sweep only when the check corrected something */
  int32_t batch;            /* 1: a context with several grids advances them all with one sweep
                               launch per tile class and one check launch per sweep (CUDA graphs
                               of graph_steps sweeps); 0: grid by grid. Offline steps always go
                               grid by grid. */
  int32_t boundary;         /* abft_boundary of every grid of the context */
  int32_t vectors;          /* online checks: 2 = test both checksum vectors every sweep; 1 = test
                               b (sums along x) every sweep and compute a, from the grid, only in
                               planes where b failed, to locate (Sec. 3.2: one vector detects, the
                               second is needed only after a detection).  1 finds the same faults
                               where b's threshold is not above a's (nx <= ny) and skips the a
                               partials and a checks; offline and unprotected steps ignore it */
  void* stream;             /* cudaStream_t used for all device work */
  const abft_stencil* stencils; /* NULL: each grid's 7-point set from its abft_coeffs; else one set
                               per grid (read by abft_init only, then not kept).  Grids with a
                               general set, and contexts with ABFT_BC_CONST, run the general
                               kernels: one launch per sweep, check and location, both checksum
                               vectors every sweep (persistent, batch, depth, overlap and vectors
                               do not apply) */
  float boundary_value;     /* ABFT_BC_CONST: the value of every cell outside the grid */
} abft_options;

/* an event recorded on the device */
typedef struct {
  int64_t step;                 /* sweep index whose output was checked (window start for rollbacks) */
  int32_t grid, z, y, x, kind;  /* abft_event_kind; -1 marks "whole line/window" */
  float before, after;          /* Eq. (8) values; rollback: flagged entries / window length */
} abft_event;

/* a scheduled bit flip: XOR bit `bit` (0..31) of the FP32 result of point (z, y, x)
   of grid `grid` at sweep `step`, after the update and before it is stored (Sec. 5.1);
   target 0 = grid point (others reserved) */
typedef struct { int64_t step; int32_t grid, z, y, x, bit, target; } abft_flip;

typedef struct {
  int64_t steps_done;       /* sweeps committed so far */
  int64_t kernel_launches;  /* kernels this context launched (graph nodes counted) */
  int64_t events;           /* events recorded (may exceed event_capacity) */
  int64_t rollbacks;        /* offline windows recomputed */
  int64_t flips_scheduled;  /* flips handed to the device */
  double max_residual;      /* largest passing |a'-a|/|a| so far (0 unless track_residual) */
  int64_t passes_recomputed; /* online passes of temporal blocking (depth >= 2) whose check failed
                               and that were recomputed sweep by sweep */
} abft_counters;

/* Fill defaults: eps 1e-5, delta 16 (Table 1), acc FP32, 4096 events, graphs of 50
   sweeps, default tile, 64 flips per step, persistent launches, whole-column tiles for
   shallow grids, no residual tracking, depth 1, overlapped checks, batched launches,
   clamped boundaries, both checksum vectors, NULL stream, no general sets, boundary
   value 0. */
ABFT_API void abft_default_options(abft_options* opt);

/* Bytes of device workspace abft_init needs for these grids and options
   (0 if the arguments are invalid). */
ABFT_API size_t abft_workspace_bytes(const abft_grid* grids, int32_t n_grids, const abft_options* opt);

/* Create a context for n_grids independent grids (Sec. 3.1's state u and constant
   term C, Table 1's eps and Delta).  temp[g] and power[g] point to nx*ny*nz FP32
   values each, in host or device memory (copied, not kept).  coeffs[g] holds grid
   g's weights and source constants.  The initial checksums a^0, b^0 and the
   constant-term checksums c_x, c_y of Theorem 1 are computed here.  workspace is
   device memory, 256-byte aligned, borrowed until abft_destroy.
   Errors: ABFT_E_INVAL (bad sizes, NULL pointers, misaligned workspace, offline-
   incapable weights are allowed but later OFFLINE steps fail), ABFT_E_NOMEM,
   ABFT_E_CUDA. */
ABFT_API abft_status abft_init(abft_ctx** out, const abft_grid* grids, int32_t n_grids,
                      const float* const* temp, const float* const* power,
                      const abft_coeffs* coeffs, const abft_options* opt,
                      void* workspace, size_t workspace_bytes);

/* Advance every grid by n sweeps in the given mode (abft_mode).  ONLINE checks and
   corrects after each sweep (Sec. 3.2-3.5).  OFFLINE runs windows of Delta sweeps
   (the last one may be shorter), compares once per window and recomputes a
   window from its checkpoint on a mismatch (Sec. 4).  Where the boundary terms do
   not vanish (empty or constant boundaries, clamped ones with cn != cs or cw != ce,
   general sets with offsets of two), the chain of each window takes them from every
   sweep's input state, so such windows run one sweep per launch.
   Synchronises the stream at the end.  Errors: ABFT_E_INVAL, ABFT_E_CUDA,
   ABFT_E_TIMEOUT, ABFT_E_UNCORRECTABLE, ABFT_E_TRUNCATED (events dropped; the
   sweeps still completed). */
ABFT_API abft_status abft_step(abft_ctx* ctx, int64_t n, int32_t mode);

/* Theorem 2 on demand: recompute the checksums of the current state and compare
   them with the interpolated ones (chained over the sweeps made since the last
   verified state, Sec. 4.1).  *n_mismatch receives the number of failing entries.
   More than one sweep past the verified state needs vanishing boundary terms (the
   intermediate states are gone): ABFT_E_INVAL otherwise. */
ABFT_API abft_status abft_verify(abft_ctx* ctx, int64_t* n_mismatch);

/* Correct what the last abft_verify found: Eq. (8) at single row/column
   intersections when the state is one sweep or less past the verified one,
   otherwise roll back to the verified state and recompute (Sec. 4.2).
   *n_fixed receives the number of corrected points or recomputed sweeps. */
ABFT_API abft_status abft_correct(abft_ctx* ctx, int64_t* n_fixed);

/* Seeded random bit flips from the next sweep on (Sec. 5.1's injection): `rate` is the
   expected number of flips per sweep and grid (floor(rate) plus one with
   probability frac(rate)), points uniform over the grid, bits uniform over the set
   bits of `bitmask`, drawn by SplitMix64 (see abft_schedule).  rate 0 disables. */
ABFT_API abft_status abft_inject(abft_ctx* ctx, uint64_t seed, double rate, uint32_t bitmask);

/* An explicit flip list (replaces any seeded schedule); entries are copied. */
ABFT_API abft_status abft_inject_list(abft_ctx* ctx, const abft_flip* flips, int64_t n);

/* The seeded schedule of one grid for sweeps [t_begin, t_end): the flips abft_inject
   would apply.  Pure host function, no context needed.  Returns the number of
   flips (entries beyond cap are not written), or -1 on invalid arguments. */
ABFT_API int64_t abft_schedule(uint64_t seed, double rate, uint32_t bitmask, int32_t grid,
                      int32_t n_grids, int32_t nx, int32_t ny, int32_t nz,
                      int64_t t_begin, int64_t t_end, abft_flip* out, int64_t cap);

/* Copy up to cap recorded events to host memory; *n_out = number recorded (may
   exceed cap).  Returns ABFT_E_TRUNCATED when the device log overflowed. */
ABFT_API abft_status abft_events(abft_ctx* ctx, abft_event* buf, int64_t cap, int64_t* n_out);

/* Copy grid g's current state (nx*ny*nz FP32, unpadded) to dst (host or device). */
ABFT_API abft_status abft_read(abft_ctx* ctx, int32_t grid, float* dst);

/* Copy grid g's checksum vectors of the current state, a (nz*nx) and b (nz*ny), FP64,
   to host or device memory (Eq. 2, 3; computed first if the last sweeps were
   unprotected). */
ABFT_API abft_status abft_read_checksums(abft_ctx* ctx, int32_t grid, double* a, double* b);

/* Device pointer and row pitch (elements) of grid g's current state, valid until
   the next abft_step/abft_correct. */
ABFT_API abft_status abft_current(abft_ctx* ctx, int32_t grid, float** dev_ptr, int64_t* pitch);

ABFT_API abft_status abft_get_counters(const abft_ctx* ctx, abft_counters* out);

/* Measurement hook: run n sweeps of `mode`, bracketing every kernel launch with CUDA
   events on the context stream, and report per kernel kind the summed milliseconds
   and launch counts (arrays of length ABFT_KERNEL_KINDS, in the order sweep-plain,
   sweep-protected, check-online, check-offline, chain, other, persistent-plain,
   persistent-protected). */
#define ABFT_KERNEL_KINDS 8
ABFT_API abft_status abft_time_kernels(abft_ctx* ctx, int64_t n, int32_t mode, double* ms, int64_t* launches);

/* Measurement probe (no counterpart in the paper): the sustained L2 copy bandwidth that
   bounds grids small enough to stay in L2.  Copies `bytes` (a multiple of 16) from src
   to dst (device buffers, 16-byte aligned, not overlapping, both caller-owned) `passes`
   (1..100000) times inside one launch of two CTAs per SM with 16-byte L2-only loads and
   stores, after one untimed warm-up pass; *elapsed_ms receives the timed launch's CUDA-
   event duration on `stream` (synchronised before return).  Bytes moved =
   2 * bytes * passes.  Choose 2 * bytes well below the L2 size (e.g. 2 x 8 MiB).
   Errors: ABFT_E_INVAL (arguments), ABFT_E_CUDA. */
ABFT_API abft_status abft_probe_l2_copy(const void* src, void* dst, size_t bytes, int32_t passes, void* stream,
                                        double* elapsed_ms);

ABFT_API const char* abft_last_error(const abft_ctx* ctx);
ABFT_API const char* abft_status_string(abft_status s);

/* Autotuner: time short fault-free runs of every distinct launch configuration for
   these grids and `mode` (rows per tile 8/16/32, whole-column tiles on/off,
   persistent launches on/off, batched launches on/off for several grids) and return
   the fastest. Every candidate runs through abft_init/abft_step/abft_destroy on the
   caller's device `workspace` (at least abft_tune_workspace_bytes, which is 0 for
   invalid arguments) and the caller's inputs (same meaning as for abft_init), on
   base->stream; `sweeps` (1..100000) are timed after 2 warm-up sweeps. *best receives
   *base with tile_y, shallow, persistent and batch set to the winner's;
   *best_us_per_sweep its time. Results are cached per (shapes, mode, acc, delta,
   sweeps, track_residual, boundary, vectors) for the process: a repeated call returns
   at once.
   Errors: ABFT_E_INVAL (arguments), ABFT_E_NOMEM (no candidate fits the workspace),
   or the first failing call's status. */
ABFT_API size_t abft_tune_workspace_bytes(const abft_grid* grids, int32_t n_grids, const abft_options* base);
ABFT_API abft_status abft_tune(const abft_grid* grids, int32_t n_grids, const float* const* temp,
                               const float* const* power, const abft_coeffs* coeffs, const abft_options* base,
                               int32_t mode, int32_t sweeps, void* workspace, size_t workspace_bytes,
                               abft_options* best, double* best_us_per_sweep);

/* Self-test of failure detection without a fault: make one bounded device wait run out
   on purpose and report how it ended.
     which 0: a grid barrier (the one the persistent kernels use) that the last CTA of a
              4-CTA launch never reaches;
     which 1: an mbarrier wait (the one every TMA copy uses) for 16 bytes of transaction
              that no copy delivers.
   limit_us (1 ms .. 10 s) bounds the wait. Returns ABFT_E_TIMEOUT when the kernel gave
   up, set its timeout status and returned (the expected outcome), ABFT_OK if the wait
   ended some other way, ABFT_E_INVAL for bad arguments, ABFT_E_CUDA on a runtime
   error. *elapsed_ms receives the kernel's duration (CUDA events on `stream`). Uses a
   file-scope device control block: serialise calls; allocates nothing. */
ABFT_API abft_status abft_selftest_wait(int32_t which, int64_t limit_us, void* stream, double* elapsed_ms);

/* One protected sweep (Eq. 1 with the fused checksum epilogue) and the per-plane
   checksums a[z][x], b[z][y] of its result, for callers that cannot allocate
   device memory: code living inside another framework's memory pool, plug-ins
   whose host forbids device allocations once running, or code that must not
   allocate while a stream is being captured.  The paper has no counterpart; this
   is a packaging of the library's own sweep.
   The caller owns every buffer: u_in, C (constant term) and u_out are device FP32
   grids with rows of `pitch` elements (pitch >= nx, a multiple of 4; pointers
   16-byte aligned; u_out != u_in); a_out (nz*nx) and b_out (nz*ny) are device FP64.
   The sweep uses the clamped boundary rule (Fig. 2) with the weights of *coeffs, and
   the checksums are FP32 tile partials summed across tiles in FP64 (ABFT_ACC_FP32);
   periodic or empty faces and the TwoSum/FP64 accumulations need a context.
   No context, workspace or allocation: the per-tile partial sums live in one fixed
   8 MiB device array inside the library, held by every GPU that loads it until
   the process exits.  Grids whose partials do not fit are refused.  The first call
   on a device looks up that array's address (once per device, with the device
   current): make it before any stream capture.  All calls share the array, so
   calls that overlap on the GPU race; serialise them.  Work is enqueued on
   `stream` (cudaStream_t) and the call returns without synchronising.
   Errors: ABFT_E_INVAL (NULL or misaligned pointers, bad sizes, grid too large for
   the array), ABFT_E_CUDA. */
ABFT_API abft_status abft_sweep_checksums_static(const float* u_in, const float* C, float* u_out,
                                                 double* a_out, double* b_out, int32_t nx, int32_t ny,
                                                 int32_t nz, int64_t pitch, const abft_coeffs* coeffs,
                                                 void* stream);

/* Release host state and graphs; the workspace is the caller's to free. */
ABFT_API void abft_destroy(abft_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ABFT_H */
