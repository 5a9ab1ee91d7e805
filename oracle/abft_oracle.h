/*
 * FP64 CPU oracle for ABFT-protected stencil sweeps, after Cavelan & Ciorba,
 * "Algorithm-Based Fault Tolerance for Parallel Stencil Computations" (arXiv 1909.00709).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or constant
 * with the CUDA library.
 *
 * Grid layout: u[(z*ny + y)*nx + x], x fastest, no padding, double precision.
 * Checksum layout: a[z*nx + x] (row checksum, Eq. 2, sum over y),
 *                  b[z*ny + y] (column checksum, Eq. 3, sum over x).
 */
#ifndef ABFT_ORACLE_H
#define ABFT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CLAMP = 0, ORC_PERIODIC = 1, ORC_ZERO = 2, ORC_CONST = 3 };
enum { ORC_MODE_NONE = 0, ORC_MODE_ONLINE = 1, ORC_MODE_OFFLINE = 2 };
enum { ORC_EV_CORRECTED = 1, ORC_EV_RECOMPUTED = 2, ORC_EV_ROLLBACK = 3 };
enum { ORC_TARGET_GRID = 0, ORC_TARGET_A = 1, ORC_TARGET_B = 2 };

/* one stencil point {i, j, w} of Sec. 3.1, extended by a z offset k for 3D */
typedef struct { int32_t dx, dy, dz; double w; } orc_point;

typedef struct {
  int32_t nx, ny, nz;
  int32_t npts;
  const orc_point* pts;
  int32_t boundary; /* ORC_CLAMP (Fig. 2), ORC_PERIODIC, ORC_ZERO, ORC_CONST */
  double bvalue;    /* ORC_CONST: the value every cell outside the grid holds */
} orc_stencil;

/* a bit-flip: at step `step`, XOR bit `bit` of the FP32 image of the target value */
typedef struct { int64_t step; int32_t grid, z, y, x, bit, target; } orc_flip;

typedef struct { int64_t step; int32_t z, y, x, kind; double before, after; } orc_event;

typedef struct {
  double eps;          /* detection threshold (Sec. 3.4) */
  int32_t delta;       /* offline detection period (Sec. 4.1) */
  int32_t literal_eq8; /* 1: evaluate Eq. (8) as a' - (a - u); 0: as a' - sum of the others */
  double band_lo, band_hi; /* guard band on |a'-a| / (eps |a|) that is logged as marginal */
  int32_t vectors;     /* online: 2 = test a and b every sweep; 1 = test b every sweep and a only
                          in planes where b failed (Sec. 3.2: one vector detects, the second
                          locates and is needed only after a detection) */
} orc_opts;

typedef struct {
  orc_event* ev; int64_t ev_cap; int64_t n_ev;
  int64_t* marg_step; int32_t* marg_z; int64_t marg_cap; int64_t n_marg;
  double max_resid;    /* largest |a'-a|/|a| over every compared entry */
  int64_t n_rollbacks;
  int64_t n_flips_applied;
} orc_out;

/* OpenMP threads for the z loops of the sweep, checksums and interpolation (1 when the
   library was built without OpenMP); results do not depend on the count */
void orc_set_threads(int32_t n);
int32_t orc_max_threads(void);

/* HotSpot-like constant term of Eq. (1): C = sdc*P + c_amb*t_amb */
void orc_source_term(int64_t n, const float* power, float sdc, float c_amb, float t_amb, double* C);

/* Eq. (1) over the whole grid */
void orc_sweep(const orc_stencil* s, const double* C, const double* u, double* out);

/* Eq. (2) and Eq. (3), per plane */
void orc_checksums(int32_t nx, int32_t ny, int32_t nz, const double* u, double* a, double* b);

/* Theorem 1 (Eq. 4, 5) with the boundary terms alpha, beta evaluated literally from u^t */
void orc_interpolate(const orc_stencil* s, const double* cx, const double* cy,
                     const double* a, const double* b, const double* u,
                     double* ap, double* bp);

/* Theorem 1 (Eq. 4, 5) for a chain of predictions: a, b are predicted vectors (not sums of
   u); every vector entry outside the grid is the rule applied to the vector (clamped or
   wrapped index, 0 for empty boundaries, n*K for constant ones with n the collapsed
   axis' length), and alpha, beta are evaluated literally from the state u the step
   starts from (per-step boundary terms) */
void orc_interpolate_chain(const orc_stencil* s, const double* cx, const double* cy,
                           const double* a, const double* b, const double* u,
                           double* ap, double* bp);

/* Eq. (6), (7): Theorem 1 with alpha = beta = 0 (the boundary rule applied to the vectors) */
void orc_interpolate_simple(const orc_stencil* s, const double* cx, const double* cy,
                            const double* a, const double* b, double* ap, double* bp);

/* Sec. 3.4 relative test on n entries; writes failing indices, returns their count */
int64_t orc_detect(int64_t n, const double* pred, const double* comp, double eps, int32_t* fail);

/* whole run: `nsteps` sweeps from step t0 in the given mode; u is updated in place */
int orc_run(const orc_stencil* s, const double* C, double* u, int64_t t0, int64_t nsteps,
            int32_t mode, const orc_flip* flips, int64_t nflips, const orc_opts* o, orc_out* r);

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) output number `counter` (0-based) of the
   stream seeded with `seed` */
uint64_t orc_splitmix64(uint64_t seed, uint64_t counter);

/* seeded flip schedule of one grid for steps [t_begin, t_end); returns count (<= cap) */
int64_t orc_schedule(uint64_t seed, double rate, uint32_t bitmask, int32_t grid, int32_t n_grids,
                     int32_t nx, int32_t ny, int32_t nz, int64_t t_begin, int64_t t_end,
                     orc_flip* out, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
