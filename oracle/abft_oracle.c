/*
 * FP64 CPU oracle for ABFT-protected stencil sweeps, after Cavelan & Ciorba,
 * "Algorithm-Based Fault Tolerance for Parallel Stencil Computations" (arXiv 1909.00709).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  Plain and slow on purpose: every function
 * follows one passage of the paper (cited beside it) in the paper's order and
 * notation, in double precision, with no blocking, fusion or reordering.
 *
 * Readings taken where the paper is silent or garbled (each also listed in the
 * design notes):
 *  R1  3D: checksums are per plane (a[z][x], b[z][y]); the z-neighbours of Eq. (1)
 *      enter Theorem 1 as the adjacent planes' checksums (Sec. 3, "apply the 2D
 *      scheme on every layer"; each layer owns its checksums, Sec. 5.1).
 *  R2  Sum limits "0..n_y" of Eq. (2), (3) and of alpha/beta are read as 0..n_y-1
 *      (n_y points); alpha uses u at column x+i as in the proof of Theorem 1.
 *  R3  Detection flags an entry unless |a' - a| <= eps |a| (Sec. 3.4's |a'/a - 1| > eps,
 *      written without the division so that NaN/Inf count as mismatches).
 *  R4  Eq. (8) is evaluated as a' - (sum of the other points of the line), the same
 *      value as a' - (a - u) without the cancellation against a corrupted u; the two
 *      estimates are averaged as in Fig. 9.  `literal_eq8` selects the printed form.
 *  R5  Location: exactly one failing a-entry and one failing b-entry in a plane
 *      -> Eq. (8) at their intersection.  Any other non-empty pattern (one vector
 *      only, as in Fig. 4b, or several entries in both) -> the flagged rows and
 *      columns are recomputed from the intact previous state u^t by Eq. (1) and the
 *      plane's checksums are summed again.
 *  R6  A flip is applied after the point is updated and before it is stored and
 *      summed (Sec. 5.1); the oracle adds the FP32 perturbation
 *      delta = f32(flip(f32(u))) - f32(u) to its FP64 value.
 *  R7  Offline: checkpoint every Delta steps, chain Eq. (6)/(7) Delta times from the
 *      checkpoint's checksums, compare once at the window end, and on a mismatch
 *      restore the checkpoint and recompute the window without injection
 *      (Sec. 4.1, 4.2, Fig. 10).  Where alpha, beta do not vanish (empty or constant
 *      boundaries, clamped ones with unequal opposite weights or offsets beyond one)
 *      each link of the chain is Theorem 1 with the terms alpha, beta of the state the
 *      step starts from, taken from the window's own intermediate states (per-step
 *      boundary terms; Theorem 1 defines them from u^t).
 *  R13 Boundary rules (Sec. 3.3): clamped (Fig. 2: an outside neighbour reads the
 *      nearest in-range point, per axis), periodic (the point on the opposite face),
 *      empty (zero) and constant (every outside cell holds the value bvalue).
 */
#include "abft_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads: the sweep, checksum and interpolation loops below split their outer z loop
   (the sweep: its z and y loops) over OpenMP threads (one `parallel for`, nothing else).  Every output entry is still
   computed by one thread in the same order, so results do not depend on the count. */
void orc_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int32_t orc_max_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ helpers */

static int64_t lin(const orc_stencil* s, int64_t z, int64_t y, int64_t x) {
  return (z * s->ny + y) * (int64_t)s->nx + x;
}

/* Map a coordinate onto [0, n) under the boundary rule.  Returns 0 when the
   ghost cell is an empty (zero) boundary cell. */
static int map_axis(int64_t* i, int64_t n, int32_t boundary) {
  if (*i >= 0 && *i < n) return 1;
  if (boundary == ORC_CLAMP) { /* Fig. 2: a neighbour outside the grid reads the nearest
                                  in-range point on that axis */
    *i = *i < 0 ? 0 : n - 1;
    return 1;
  }
  if (boundary == ORC_PERIODIC) {
    *i = ((*i % n) + n) % n;
    return 1;
  }
  return 0; /* ORC_ZERO and ORC_CONST: an outside cell holds a fixed value, Sec. 3.3 */
}

/* the fixed value of a cell outside the grid (empty: 0, constant: bvalue) */
static double outside(const orc_stencil* s) { return s->boundary == ORC_CONST ? s->bvalue : 0.0; }

/* value of u at any coordinate, ghost cells included */
static double ghost(const orc_stencil* s, const double* u, int64_t z, int64_t y, int64_t x) {
  if (!map_axis(&z, s->nz, s->boundary)) return outside(s);
  if (!map_axis(&y, s->ny, s->boundary)) return outside(s);
  if (!map_axis(&x, s->nx, s->boundary)) return outside(s);
  return u[lin(s, z, y, x)];
}

static int stencil_radius(const orc_stencil* s) {
  int r = 0;
  for (int k = 0; k < s->npts; k++) {
    int m = abs(s->pts[k].dx);
    if (abs(s->pts[k].dy) > m) m = abs(s->pts[k].dy);
    if (abs(s->pts[k].dz) > m) m = abs(s->pts[k].dz);
    if (m > r) r = m;
  }
  return r;
}

/* Eq. (1) at one point: C + sum over S of w * u(x+i, y+j, z+k) */
static double update_point(const orc_stencil* s, const double* C, const double* u,
                           int64_t z, int64_t y, int64_t x) {
  double acc = 0.0;
  for (int k = 0; k < s->npts; k++) {
    const orc_point* p = &s->pts[k];
    acc += p->w * ghost(s, u, z + p->dz, y + p->dy, x + p->dx);
  }
  return C[lin(s, z, y, x)] + acc;
}

/* --------------------------------------------------------- Eq. (1): sweep */

void orc_source_term(int64_t n, const float* power, float sdc, float c_amb, float t_amb, double* C) {
  for (int64_t i = 0; i < n; i++) C[i] = (double)sdc * (double)power[i] + (double)c_amb * (double)t_amb;
}

void orc_sweep(const orc_stencil* s, const double* C, const double* u, double* out) {
  const int r = stencil_radius(s);
  int64_t* off = malloc(sizeof(int64_t) * (s->npts > 0 ? s->npts : 1));
  for (int k = 0; k < s->npts; k++) off[k] = lin(s, s->pts[k].dz, s->pts[k].dy, s->pts[k].dx);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t z = 0; z < s->nz; z++)
    for (int64_t y = 0; y < s->ny; y++)
      for (int64_t x = 0; x < s->nx; x++) {
        const int64_t c = lin(s, z, y, x);
        const int interior = z >= r && z < s->nz - r && y >= r && y < s->ny - r &&
                             x >= r && x < s->nx - r;
        if (interior) { /* same sum as update_point, without the no-op boundary mapping */
          double acc = 0.0;
          for (int k = 0; k < s->npts; k++) acc += s->pts[k].w * u[c + off[k]];
          out[c] = C[c] + acc;
        } else {
          out[c] = update_point(s, C, u, z, y, x);
        }
      }
  free(off);
}

/* ------------------------------------------------ Eq. (2), (3): checksums */

void orc_checksums(int32_t nx, int32_t ny, int32_t nz, const double* u, double* a, double* b) {
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < nz; z++) {
    for (int64_t x = 0; x < nx; x++) {
      double t = 0.0;
      for (int64_t y = 0; y < ny; y++) t += u[(z * ny + y) * nx + x];
      a[z * nx + x] = t;
    }
    for (int64_t y = 0; y < ny; y++) {
      double t = 0.0;
      for (int64_t x = 0; x < nx; x++) t += u[(z * ny + y) * nx + x];
      b[z * ny + y] = t;
    }
  }
}

/* ------------------------------------------------ Theorem 1: interpolation */

/* a_x of a possibly ghost column: the stored entry in range, else the sum of the
   ghost column's cells */
static double a_at(const orc_stencil* s, const double* a, const double* u, int64_t z, int64_t x) {
  if (z >= 0 && z < s->nz && x >= 0 && x < s->nx) return a[z * s->nx + x];
  double t = 0.0;
  for (int64_t y = 0; y < s->ny; y++) t += ghost(s, u, z, y, x);
  return t;
}

static double b_at(const orc_stencil* s, const double* b, const double* u, int64_t z, int64_t y) {
  if (z >= 0 && z < s->nz && y >= 0 && y < s->ny) return b[z * s->ny + y];
  double t = 0.0;
  for (int64_t x = 0; x < s->nx; x++) t += ghost(s, u, z, y, x);
  return t;
}

/* alpha_{x,j}: cells shifted into the column from beyond the boundary minus the
   cells shifted out of it (Theorem 1) */
static double alpha(const orc_stencil* s, const double* u, int64_t z, int64_t x, int j) {
  double t = 0.0;
  if (j < 0) {
    for (int64_t y = j; y <= -1; y++) t += ghost(s, u, z, y, x);
    for (int64_t y = s->ny + j; y <= s->ny - 1; y++) t -= ghost(s, u, z, y, x);
  } else if (j > 0) {
    for (int64_t y = s->ny; y <= s->ny + j - 1; y++) t += ghost(s, u, z, y, x);
    for (int64_t y = 0; y <= j - 1; y++) t -= ghost(s, u, z, y, x);
  }
  return t;
}

/* beta_{i,y}: same along x for the column checksum */
static double beta(const orc_stencil* s, const double* u, int64_t z, int64_t y, int i) {
  double t = 0.0;
  if (i < 0) {
    for (int64_t x = i; x <= -1; x++) t += ghost(s, u, z, y, x);
    for (int64_t x = s->nx + i; x <= s->nx - 1; x++) t -= ghost(s, u, z, y, x);
  } else if (i > 0) {
    for (int64_t x = s->nx; x <= s->nx + i - 1; x++) t += ghost(s, u, z, y, x);
    for (int64_t x = 0; x <= i - 1; x++) t -= ghost(s, u, z, y, x);
  }
  return t;
}

void orc_interpolate(const orc_stencil* s, const double* cx, const double* cy,
                     const double* a, const double* b, const double* u,
                     double* ap, double* bp) {
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < s->nz; z++) {
    for (int64_t x = 0; x < s->nx; x++) { /* Eq. (4) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * (a_at(s, a, u, z + p->dz, x + p->dx) + alpha(s, u, z + p->dz, x + p->dx, p->dy));
      }
      ap[z * s->nx + x] = cx[z * s->nx + x] + acc;
    }
    for (int64_t y = 0; y < s->ny; y++) { /* Eq. (5) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * (b_at(s, b, u, z + p->dz, y + p->dy) + beta(s, u, z + p->dz, y + p->dy, p->dx));
      }
      bp[z * s->ny + y] = cy[z * s->ny + y] + acc;
    }
  }
}

/* entry of a predicted vector v (n_line entries per plane; the collapsed axis has
   n_coll cells) at a possibly outside (z, i): the boundary rule applied to the vector */
static double chain_at(const orc_stencil* s, const double* v, int64_t n_line, int64_t n_coll, int64_t z,
                       int64_t i) {
  if (!map_axis(&z, s->nz, s->boundary) || !map_axis(&i, n_line, s->boundary))
    return (double)n_coll * outside(s); /* a line of outside cells */
  return v[z * n_line + i];
}

void orc_interpolate_chain(const orc_stencil* s, const double* cx, const double* cy,
                           const double* a, const double* b, const double* u,
                           double* ap, double* bp) {
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < s->nz; z++) {
    for (int64_t x = 0; x < s->nx; x++) { /* Eq. (4) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * (chain_at(s, a, s->nx, s->ny, z + p->dz, x + p->dx) +
                       alpha(s, u, z + p->dz, x + p->dx, p->dy));
      }
      ap[z * s->nx + x] = cx[z * s->nx + x] + acc;
    }
    for (int64_t y = 0; y < s->ny; y++) { /* Eq. (5) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * (chain_at(s, b, s->ny, s->nx, z + p->dz, y + p->dy) +
                       beta(s, u, z + p->dz, y + p->dy, p->dx));
      }
      bp[z * s->ny + y] = cy[z * s->ny + y] + acc;
    }
  }
}

/* vector entry under the boundary rule applied to the 1D vector (Fig. 3's w/e lines) */
static double vec_at(const double* v, int64_t n_line, int64_t nz, int32_t boundary, int64_t z, int64_t i) {
  if (!map_axis(&z, nz, boundary)) return 0.0;
  if (!map_axis(&i, n_line, boundary)) return 0.0;
  return v[z * n_line + i];
}

void orc_interpolate_simple(const orc_stencil* s, const double* cx, const double* cy,
                            const double* a, const double* b, double* ap, double* bp) {
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < s->nz; z++) {
    for (int64_t x = 0; x < s->nx; x++) { /* Eq. (6) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * vec_at(a, s->nx, s->nz, s->boundary, z + p->dz, x + p->dx);
      }
      ap[z * s->nx + x] = cx[z * s->nx + x] + acc;
    }
    for (int64_t y = 0; y < s->ny; y++) { /* Eq. (7) */
      double acc = 0.0;
      for (int k = 0; k < s->npts; k++) {
        const orc_point* p = &s->pts[k];
        acc += p->w * vec_at(b, s->ny, s->nz, s->boundary, z + p->dz, y + p->dy);
      }
      bp[z * s->ny + y] = cy[z * s->ny + y] + acc;
    }
  }
}

/* ------------------------------------------------------ Sec. 3.4: detection */

static int entry_fails(double pred, double comp, double eps) {
  return !(fabs(pred - comp) <= eps * fabs(comp));
}

int64_t orc_detect(int64_t n, const double* pred, const double* comp, double eps, int32_t* fail) {
  int64_t count = 0;
  for (int64_t i = 0; i < n; i++)
    if (entry_fails(pred[i], comp[i], eps)) fail[count++] = (int32_t)i;
  return count;
}

/* ------------------------------------------------------------ bit flips */

static float flip_f32(float v, int bit) {
  uint32_t w;
  memcpy(&w, &v, 4);
  w ^= (uint32_t)1u << bit;
  memcpy(&v, &w, 4);
  return v;
}

/* R6: perturb a double by the change a flip makes to its FP32 image */
static void apply_flip(double* v, int bit) {
  const float f = (float)*v;
  *v += (double)flip_f32(f, bit) - (double)f;
}

/* ------------------------------------------------------------ run state */

static void add_event(orc_out* r, int64_t step, int32_t z, int32_t y, int32_t x, int32_t kind,
                      double before, double after) {
  if (r->n_ev < r->ev_cap) {
    orc_event* e = &r->ev[r->n_ev];
    e->step = step; e->z = z; e->y = y; e->x = x; e->kind = kind; e->before = before; e->after = after;
  }
  r->n_ev++;
}

static void add_marginal(orc_out* r, int64_t step, int32_t z) {
  if (r->n_marg > 0 && r->n_marg <= r->marg_cap && r->marg_step[r->n_marg - 1] == step &&
      r->marg_z[r->n_marg - 1] == z)
    return;
  if (r->n_marg < r->marg_cap) { r->marg_step[r->n_marg] = step; r->marg_z[r->n_marg] = z; }
  r->n_marg++;
}

/* compare one plane's vector; record the largest residual and the guard band */
static int64_t compare_line(const orc_opts* o, orc_out* r, int64_t step, int32_t z, int64_t n,
                            const double* pred, const double* comp, int32_t* fail) {
  int marginal = 0;
  for (int64_t i = 0; i < n; i++) {
    const double rel = fabs(pred[i] - comp[i]) / fabs(comp[i]);
    if (rel == rel && rel > r->max_resid) r->max_resid = rel;
    const double ratio = rel / o->eps;
    if (ratio >= o->band_lo && ratio <= o->band_hi) marginal = 1;
  }
  if (marginal) add_marginal(r, step, z);
  return orc_detect(n, pred, comp, o->eps, fail);
}

/* Eq. (8) and Fig. 9 at (ex, ey) of plane z; uq holds u^{t+1} */
static void correct_point(const orc_stencil* s, const orc_opts* o, orc_out* r, int64_t step,
                          int32_t z, int32_t ex, int32_t ey, double* uq, double* A, double* B,
                          const double* Ap, const double* Bp) {
  const int64_t nx = s->nx, ny = s->ny;
  const int64_t c = lin(s, z, ey, ex);
  const double bad = uq[c];
  double others_a = 0.0, others_b = 0.0; /* sums of the line without the flagged point */
  for (int64_t y = 0; y < ny; y++)
    if (y != ey) others_a += uq[lin(s, z, y, ex)];
  for (int64_t x = 0; x < nx; x++)
    if (x != ex) others_b += uq[lin(s, z, ey, x)];
  double va, vb;
  if (o->literal_eq8) {
    va = Ap[z * nx + ex] - (A[z * nx + ex] - bad);
    vb = Bp[z * ny + ey] - (B[z * ny + ey] - bad);
  } else {
    va = Ap[z * nx + ex] - others_a;
    vb = Bp[z * ny + ey] - others_b;
  }
  const double corrected = (va + vb) / 2.0;
  uq[c] = corrected;
  A[z * nx + ex] = others_a + corrected; /* keep the checksums consistent (Sec. 3.5) */
  B[z * ny + ey] = others_b + corrected;
  add_event(r, step, z, ey, ex, ORC_EV_CORRECTED, bad, corrected);
}

/* R5: recompute flagged lines of plane z from the intact previous state */
static void recompute_lines(const orc_stencil* s, orc_out* r, int64_t step, int32_t z,
                            const int32_t* fa, int64_t nfa, const int32_t* fb, int64_t nfb,
                            const double* C, const double* u_prev, double* uq, double* A, double* B) {
  for (int64_t k = 0; k < nfb; k++) {
    const int32_t y = fb[k];
    for (int64_t x = 0; x < s->nx; x++) uq[lin(s, z, y, x)] = update_point(s, C, u_prev, z, y, x);
    add_event(r, step, z, y, -1, ORC_EV_RECOMPUTED, 0.0, 0.0);
  }
  for (int64_t k = 0; k < nfa; k++) {
    const int32_t x = fa[k];
    for (int64_t y = 0; y < s->ny; y++) uq[lin(s, z, y, x)] = update_point(s, C, u_prev, z, y, x);
    add_event(r, step, z, -1, x, ORC_EV_RECOMPUTED, 0.0, 0.0);
  }
  /* sum the plane's checksums again (Eq. 2, 3) */
  for (int64_t x = 0; x < s->nx; x++) {
    double t = 0.0;
    for (int64_t y = 0; y < s->ny; y++) t += uq[lin(s, z, y, x)];
    A[z * s->nx + x] = t;
  }
  for (int64_t y = 0; y < s->ny; y++) {
    double t = 0.0;
    for (int64_t x = 0; x < s->nx; x++) t += uq[lin(s, z, y, x)];
    B[z * s->ny + y] = t;
  }
}

/* apply the flips of step t to the grid (before the checksum) or to the checksums
   (after it); `k` walks a step-sorted list */
static void inject(const orc_stencil* s, const orc_flip* flips, int64_t nflips, int64_t t,
                   int32_t target, double* uq, double* A, double* B, orc_out* r) {
  for (int64_t k = 0; k < nflips; k++) {
    const orc_flip* f = &flips[k];
    if (f->step != t || f->target != target) continue;
    if (target == ORC_TARGET_GRID) apply_flip(&uq[lin(s, f->z, f->y, f->x)], f->bit);
    else if (target == ORC_TARGET_A) apply_flip(&A[(int64_t)f->z * s->nx + f->x], f->bit);
    else apply_flip(&B[(int64_t)f->z * s->ny + f->y], f->bit);
    r->n_flips_applied++;
  }
}

static int alpha_beta_vanish(const orc_stencil* s) {
  if (s->boundary == ORC_PERIODIC) return 1;
  if (s->boundary == ORC_ZERO || s->boundary == ORC_CONST) return 0;
  /* clamped: every point (i, j, k) needs a partner (i, -j, k) and (-i, j, k) of equal weight,
     and in-plane offsets of at most one: for |j| = 2 the clamped terms of Theorem 1 are
     2 u_0 - u_{n-2} - u_{n-1} and 2 u_{n-1} - u_0 - u_1, whose sum does not vanish */
  for (int k = 0; k < s->npts; k++) {
    const orc_point* p = &s->pts[k];
    if (abs(p->dx) > 1 || abs(p->dy) > 1) return 0;
    int mirror_y = 0, mirror_x = 0;
    for (int m = 0; m < s->npts; m++) {
      const orc_point* q = &s->pts[m];
      if (q->dx == p->dx && q->dy == -p->dy && q->dz == p->dz && q->w == p->w) mirror_y = 1;
      if (q->dx == -p->dx && q->dy == p->dy && q->dz == p->dz && q->w == p->w) mirror_x = 1;
    }
    if (!mirror_x || !mirror_y) return 0;
  }
  return 1;
}

int orc_run(const orc_stencil* s, const double* C, double* u, int64_t t0, int64_t nsteps,
            int32_t mode, const orc_flip* flips, int64_t nflips, const orc_opts* o, orc_out* r) {
  const int64_t nx = s->nx, ny = s->ny, nz = s->nz;
  const int64_t n = nx * ny * nz;
  if (mode == ORC_MODE_OFFLINE && o->delta < 1) return -1;
  const int simple_chain = alpha_beta_vanish(s); /* Eq. (6)/(7) suffice (Fig. 10) */

  double* uq = malloc(sizeof(double) * n);
  double* ck = malloc(sizeof(double) * n);
  double* cx = malloc(sizeof(double) * nz * nx);
  double* cy = malloc(sizeof(double) * nz * ny);
  double* A = malloc(sizeof(double) * nz * nx);
  double* B = malloc(sizeof(double) * nz * ny);
  double* An = malloc(sizeof(double) * nz * nx);
  double* Bn = malloc(sizeof(double) * nz * ny);
  double* Ap = malloc(sizeof(double) * nz * nx);
  double* Bp = malloc(sizeof(double) * nz * ny);
  double* Ack = malloc(sizeof(double) * nz * nx);
  double* Bck = malloc(sizeof(double) * nz * ny);
  int32_t* fa = malloc(sizeof(int32_t) * (nx > ny ? nx : ny));
  int32_t* fb = malloc(sizeof(int32_t) * (nx > ny ? nx : ny));
  int rc = 0;

  orc_checksums(s->nx, s->ny, s->nz, C, cx, cy);  /* c_x, c_y of Theorem 1 */
  orc_checksums(s->nx, s->ny, s->nz, u, A, B);    /* a^(t0), b^(t0) */

  if (mode == ORC_MODE_ONLINE) {
    for (int64_t t = t0; t < t0 + nsteps; t++) {
      orc_sweep(s, C, u, uq);                                       /* Eq. (1)       */
      inject(s, flips, nflips, t, ORC_TARGET_GRID, uq, An, Bn, r);  /* Sec. 5.1      */
      orc_checksums(s->nx, s->ny, s->nz, uq, An, Bn);               /* Eq. (2), (3)  */
      inject(s, flips, nflips, t, ORC_TARGET_A, uq, An, Bn, r);
      inject(s, flips, nflips, t, ORC_TARGET_B, uq, An, Bn, r);
      orc_interpolate(s, cx, cy, A, B, u, Ap, Bp);                  /* Theorem 1     */
      for (int32_t z = 0; z < nz; z++) {                            /* Theorem 2     */
        const int64_t nfb = compare_line(o, r, t, z, ny, Bp + z * ny, Bn + z * ny, fb);
        /* one-vector detection (Sec. 3.2): a is consulted only after b detected */
        const int64_t nfa = (o->vectors == 1 && nfb == 0)
                                ? 0 : compare_line(o, r, t, z, nx, Ap + z * nx, An + z * nx, fa);
        if (nfa == 1 && nfb == 1)
          correct_point(s, o, r, t, z, fa[0], fb[0], uq, An, Bn, Ap, Bp); /* Eq. (8) */
        else if (nfa + nfb > 0)
          recompute_lines(s, r, t, z, fa, nfa, fb, nfb, C, u, uq, An, Bn);
      }
      memcpy(u, uq, sizeof(double) * n);
      memcpy(A, An, sizeof(double) * nz * nx);
      memcpy(B, Bn, sizeof(double) * nz * ny);
    }
  } else if (mode == ORC_MODE_OFFLINE) {
    int64_t t = t0;
    while (t < t0 + nsteps) {
      const int64_t d = (t0 + nsteps - t) < o->delta ? (t0 + nsteps - t) : o->delta;
      memcpy(ck, u, sizeof(double) * n); /* checkpoint: grid and checksums (Sec. 5.4) */
      memcpy(Ack, A, sizeof(double) * nz * nx);
      memcpy(Bck, B, sizeof(double) * nz * ny);
      int attempt = 0;
      for (;;) {
        /* Fig. 10: interpolate Delta times from the checkpoint's checksums; with
           per-step boundary terms each link reads the state its step starts from */
        memcpy(Ap, Ack, sizeof(double) * nz * nx);
        memcpy(Bp, Bck, sizeof(double) * nz * ny);
        for (int64_t k = 0; k < d; k++) {
          if (!simple_chain) {
            orc_interpolate_chain(s, cx, cy, Ap, Bp, u, An, Bn);
            memcpy(Ap, An, sizeof(double) * nz * nx);
            memcpy(Bp, Bn, sizeof(double) * nz * ny);
          }
          orc_sweep(s, C, u, uq);
          if (attempt == 0) inject(s, flips, nflips, t + k, ORC_TARGET_GRID, uq, A, B, r);
          memcpy(u, uq, sizeof(double) * n);
        }
        orc_checksums(s->nx, s->ny, s->nz, u, A, B);
        for (int64_t k = 0; simple_chain && k < d; k++) {
          orc_interpolate_simple(s, cx, cy, Ap, Bp, An, Bn);
          memcpy(Ap, An, sizeof(double) * nz * nx);
          memcpy(Bp, Bn, sizeof(double) * nz * ny);
        }
        int64_t nfail = 0;
        for (int32_t z = 0; z < nz; z++) {
          nfail += compare_line(o, r, t + d - 1, z, nx, Ap + z * nx, A + z * nx, fa);
          nfail += compare_line(o, r, t + d - 1, z, ny, Bp + z * ny, B + z * ny, fb);
        }
        if (nfail == 0) break;
        if (attempt == 1) { rc = -2; break; } /* a fault-free recomputation must verify */
        add_event(r, t, -1, -1, -1, ORC_EV_ROLLBACK, (double)nfail, (double)d);
        r->n_rollbacks++;
        memcpy(u, ck, sizeof(double) * n); /* Sec. 4.2: restore and recompute */
        memcpy(A, Ack, sizeof(double) * nz * nx);
        memcpy(B, Bck, sizeof(double) * nz * ny);
        attempt = 1;
      }
      if (rc) break;
      t += d;
    }
  } else {
    for (int64_t t = t0; t < t0 + nsteps; t++) {
      orc_sweep(s, C, u, uq);
      inject(s, flips, nflips, t, ORC_TARGET_GRID, uq, A, B, r);
      memcpy(u, uq, sizeof(double) * n);
    }
  }

  free(uq); free(ck); free(cx); free(cy); free(A); free(B); free(An); free(Bn);
  free(Ap); free(Bp); free(Ack); free(Bck); free(fa); free(fb);
  return rc;
}

/* ------------------------------------------------ seeded flip schedule */

/* SplitMix64: state advances by the golden-ratio increment, output is the
   published 64-bit finaliser of the new state */
uint64_t orc_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Schedule recipe (shared definition, two implementations): stream s = t*n_grids + g,
   counters start at s*1024.  Draw 0 decides the count floor(rate) + [draw0>>11 <
   frac(rate)*2^53] (at most 511); flip i uses draw 1+2i for the point
   ((draw * N) >> 64) and draw 2+2i for the bit (the j-th set bit of `bitmask`,
   j = ((draw >> 32) * popcount) >> 32). */
int64_t orc_schedule(uint64_t seed, double rate, uint32_t bitmask, int32_t grid, int32_t n_grids,
                     int32_t nx, int32_t ny, int32_t nz, int64_t t_begin, int64_t t_end,
                     orc_flip* out, int64_t cap) {
  const uint64_t npts = (uint64_t)nx * (uint64_t)ny * (uint64_t)nz;
  int nbits = 0;
  for (int b = 0; b < 32; b++) nbits += (bitmask >> b) & 1u;
  if (nbits == 0 || rate <= 0.0) return 0;
  const double whole = floor(rate);
  const uint64_t thr = (uint64_t)((rate - whole) * 9007199254740992.0);
  int64_t count = 0;
  for (int64_t t = t_begin; t < t_end; t++) {
    const uint64_t c0 = ((uint64_t)t * (uint64_t)n_grids + (uint64_t)grid) * 1024ull;
    int64_t k = (int64_t)whole + (((orc_splitmix64(seed, c0) >> 11) < thr) ? 1 : 0);
    if (k > 511) k = 511;
    for (int64_t i = 0; i < k; i++) {
      const uint64_t r1 = orc_splitmix64(seed, c0 + 1 + 2 * (uint64_t)i);
      const uint64_t r2 = orc_splitmix64(seed, c0 + 2 + 2 * (uint64_t)i);
      const uint64_t p = (uint64_t)(((unsigned __int128)r1 * npts) >> 64);
      const uint32_t j = (uint32_t)(((r2 >> 32) * (uint64_t)nbits) >> 32);
      int bit = -1, seen = 0;
      for (int b = 0; b < 32; b++)
        if ((bitmask >> b) & 1u) {
          if (seen == (int)j) { bit = b; break; }
          seen++;
        }
      if (count < cap) {
        orc_flip* f = &out[count];
        f->step = t; f->grid = grid;
        f->z = (int32_t)(p / ((uint64_t)nx * ny));
        f->y = (int32_t)((p / (uint64_t)nx) % (uint64_t)ny);
        f->x = (int32_t)(p % (uint64_t)nx);
        f->bit = bit; f->target = ORC_TARGET_GRID;
      }
      count++;
    }
  }
  return count;
}
