/*
 * FP64 CPU oracle for batched LAD-LASSO coordinate descent.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or helper with the CUDA library; it is a plain, slow
 * restatement of the method, written for a reader to check against the
 * paper by eye.  Everything is double precision.
 *
 * Problem (Sections 1-2, combined LAD loss and L1 penalty):
 *
 *     F(b) = sum_i |y_i - x_i . b|  +  lambda * sum_j |b_j|
 *
 * The paper's LP (Section 3.1) puts the constant on the residual term; the
 * same argmin results with the constant moved onto the coefficient term,
 * lambda = 1/C.  No intercept is fitted.
 *
 * Two independent halves:
 *
 *   method (what the GPU path also computes)
 *     orc_axis_update  exact 1-D minimisation along one axis (Section 3.3/3.4:
 *                      the sub-search on the piecewise-linear objective),
 *                      written as its plain definition, a weighted median.
 *     orc_ccd          cyclical coordinate descent (Section 3.3).
 *     orc_chop         ternary search along one axis over the locus of
 *                      axis-wise minima, each probe a coordinate descent
 *                      restricted to the other axes (Sections 3.4-3.5),
 *                      with range extension (Section 3.5); option
 *                      chop_sections = 4 reads the paper's undefined
 *                      "quadrature" search (Sections 1, 5) as four equal
 *                      sections probed at the three inner points.
 *     orc_polish       exact finish: vertex-to-vertex edge line searches
 *                      (each itself a weighted median) until the
 *                      optimality multipliers certify the vertex.  The
 *                      paper's locus argument is unproven (Section 5) and
 *                      chop results are not always optimal; the polish makes
 *                      every result the LP optimum that Section 3.2
 *                      guarantees exists at a vertex.
 *     orc_fit_path     the above in order over a descending lambda path
 *                      with warm starts.
 *
 *   exact definitions (pin the method; none of the method's code is used)
 *     orc_brute_force  evaluate F at every vertex formed by p hyperplanes
 *                      from {x_i.b = y_i} U {b_j = 0} (Section 3.2).
 *     orc_simplex      dense primal simplex, Bland's rule, of the split-
 *                      variable LP of Section 3.1.
 *     orc_certify      duality-gap certificate from the dual LP
 *                      max y.u  s.t. |u_i| <= 1, |(X^T u)_j| <= lambda.
 *
 *   also: orc_lambda_max (smallest lambda with b = 0 optimal) and
 *   orc_grad (implicit-differentiation gradient of a validation LAD loss at
 *   the final vertex).
 *
 * Layout: each problem's design is a dense row-major n x p double matrix.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FIT_OK 0
#define ORC_FIT_MAX_ITERS 1
#define ORC_FIT_BAD_INPUT 2
#define ORC_FIT_NONUNIQUE 4

typedef struct {
  double tol_move;       /* CCD stops after a sweep with max|db| <= tol_move*max(1,|b|inf) */
  int max_sweeps;        /* CCD sweep cap */
  int chop;              /* run the ternary chop when a CCD stall is not optimal */
  double chop_bracket;   /* initial half-width of the search range, times max(1,|b_k|) */
  double chop_tol;       /* stop when the bracket is below chop_tol*max(1,|b_k|) */
  int chop_max_probes;   /* ternary probes after bracketing */
  int chop_max_extend;   /* range extensions */
  int probe_max_sweeps;  /* restricted-CCD sweep cap inside one probe */
  int polish;            /* run the exact vertex polish */
  int max_pivots;        /* polish step cap */
  double tol_opt;        /* multiplier tolerance, times max(1,lambda) */
  double lambda_min_floor; /* Section 3.5: a small minimum lambda disambiguates flat LAD minima */
  int chop_sections;     /* 3: ternary chop; 4: the "quadrature" reading (3 interior probes) */
} orc_opts;

typedef struct {
  int sweeps;          /* CCD sweeps (all phases) */
  int probes;          /* chop probes */
  int extends;         /* chop range extensions */
  int pivots;          /* polish steps */
  int ccd_optimal;     /* CCD fixed point already optimal */
  int chop_ran;        /* chop executed */
  int chop_optimal;    /* point after chop + CCD already optimal */
} orc_stats;

void orc_default_opts(orc_opts* o) {
  o->tol_move = 1e-12;
  o->max_sweeps = 1000;
  o->chop = 1;
  o->chop_bracket = 0.05;
  o->chop_tol = 1e-3;
  o->chop_max_probes = 12;
  o->chop_max_extend = 20;
  o->chop_sections = 3;
  o->probe_max_sweeps = 4;
  o->polish = 1;
  o->max_pivots = 2000;
  o->tol_opt = 1e-10;
  o->lambda_min_floor = 0.0;
}

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double sgn(double v) { return (v > 0) - (v < 0); }

/* F(b) = sum |y - X b| + lambda |b|_1, evaluated from scratch. */
double orc_objective(int n, int p, const double* X, const double* y,
                     const double* b, double lam) {
  double f = 0.0;
  for (int i = 0; i < n; ++i) {
    double ri = y[i];
    for (int j = 0; j < p; ++j) ri -= X[(size_t)i * p + j] * b[j];
    f += fabs(ri);
  }
  for (int j = 0; j < p; ++j) f += lam * fabs(b[j]);
  return f;
}

static void residual(int n, int p, const double* X, const double* y,
                     const double* b, double* r) {
  for (int i = 0; i < n; ++i) {
    double ri = y[i];
    for (int j = 0; j < p; ++j) ri -= X[(size_t)i * p + j] * b[j];
    r[i] = ri;
  }
}

/* Solve A x = rhs (m x m, row-major, destroyed) by Gaussian elimination with
 * partial pivoting.  Returns 0 on success, -1 when a pivot is below
 * rel_tol * max|A|. */
static int gauss_solve(int m, double* A, double* rhs, double rel_tol) {
  double amax = 0.0;
  for (int i = 0; i < m * m; ++i) amax = fmax(amax, fabs(A[i]));
  if (amax == 0.0) return m == 0 ? 0 : -1;
  for (int k = 0; k < m; ++k) {
    int piv = k;
    double best = fabs(A[k * m + k]);
    for (int i = k + 1; i < m; ++i)
      if (fabs(A[i * m + k]) > best) { best = fabs(A[i * m + k]); piv = i; }
    if (best <= rel_tol * amax) return -1;
    if (piv != k) {
      for (int c = 0; c < m; ++c) {
        double t = A[k * m + c]; A[k * m + c] = A[piv * m + c]; A[piv * m + c] = t;
      }
      double t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
    }
    for (int i = k + 1; i < m; ++i) {
      double l = A[i * m + k] / A[k * m + k];
      if (l == 0.0) continue;
      for (int c = k; c < m; ++c) A[i * m + c] -= l * A[k * m + c];
      rhs[i] -= l * rhs[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double s = rhs[k];
    for (int c = k + 1; c < m; ++c) s -= A[k * m + c] * rhs[c];
    rhs[k] = s / A[k * m + k];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* weighted median: the exact minimiser of a 1-D sum of |.| terms     */
/* ------------------------------------------------------------------ */

typedef struct { double z, w; int id; } bp_t; /* breakpoint, weight, owner */

static int bp_cmp(const void* a, const void* b) {
  const bp_t* u = (const bp_t*)a;
  const bp_t* v = (const bp_t*)b;
  if (u->z < v->z) return -1;
  if (u->z > v->z) return 1;
  return (u->id > v->id) - (u->id < v->id);
}

/* phi(t) = sum_k w_k |t - z_k| is convex and piecewise linear; its slope
 * between breakpoints is (weight left) - (weight right).  A minimiser is
 * the smallest z whose cumulative weight reaches half the total.  When the
 * cumulative weight equals exactly half, every t between that breakpoint
 * and the next distinct one is a minimiser (a flat segment, Section 3.5);
 * then the current value `cur` is kept if it lies inside, else the nearer
 * end is taken.  Returns the minimiser; *owner is the id of the breakpoint
 * landed on, or INT32_MIN when the result is strictly inside a flat segment.
 * m == 0 or zero total weight returns cur. */
static double weighted_median(bp_t* bp, int m, double cur, int* owner) {
  *owner = INT32_MIN;
  if (m == 0) return cur;
  qsort(bp, (size_t)m, sizeof(bp_t), bp_cmp);
  double W = 0.0;
  for (int k = 0; k < m; ++k) W += bp[k].w;
  if (!(W > 0.0)) return cur;
  double half = 0.5 * W, cum = 0.0;
  int k = 0;
  while (k < m) {
    int g = k; /* group of equal breakpoints */
    double gw = 0.0;
    while (g < m && bp[g].z == bp[k].z) { gw += bp[g].w; ++g; }
    cum += gw;
    if (cum >= half) {
      /* owner: the first positive-weight member of the group */
      int own = k;
      for (int q = k; q < g; ++q) if (bp[q].w > 0.0) { own = q; break; }
      if (cum == half && g < m) {
        double lo = bp[k].z, hi = bp[g].z;
        if (cur > lo && cur < hi) return cur;
        if (cur >= hi) { *owner = bp[g].id; return hi; }
        *owner = bp[own].id;
        return lo;
      }
      *owner = bp[own].id;
      return bp[k].z;
    }
    k = g;
  }
  *owner = bp[m - 1].id;
  return bp[m - 1].z;
}

/* Breakpoint owner ids: rows are 0..n-1, coordinate j is -(j+1). */
#define COORD_ID(j) (-(j) - 1)

/* ------------------------------------------------------------------ */
/* Section 3.3: axis update and cyclical coordinate descent            */
/* ------------------------------------------------------------------ */

/* Minimise F exactly along axis j, all other coordinates held (Section 3.3).
 * Along the axis, F(b + (t - b_j) e_j) = sum_i |x_ij| |z_i - t| + lambda |t|
 * + const, with z_i = b_j + r_i / x_ij for x_ij != 0: a weighted median of
 * the z_i (weights |x_ij|) and of 0 (weight lambda).  Updates b_j and r.
 * Returns the move; *piv = row landed on, -1 for the penalty breakpoint 0,
 * -2 for none. */
double orc_axis_update(int n, int p, const double* X, double* b, double* r,
                       double lam, int j, int* piv, bp_t* work) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    double x = X[(size_t)i * p + j];
    if (x != 0.0) {
      work[m].z = b[j] + r[i] / x;
      work[m].w = fabs(x);
      work[m].id = i;
      ++m;
    }
  }
  if (lam > 0.0) { work[m].z = 0.0; work[m].w = lam; work[m].id = COORD_ID(j); ++m; }
  int own;
  double t = weighted_median(work, m, b[j], &own);
  *piv = own == INT32_MIN ? -2 : (own < 0 ? -1 : own);
  double d = t - b[j];
  if (d != 0.0) {
    for (int i = 0; i < n; ++i) r[i] -= X[(size_t)i * p + j] * d;
    b[j] = t;
  }
  return d;
}

/* Cyclical coordinate descent over j = 0..p-1, skipping axis `skip` (the
 * restricted sub-search of Section 3.5; skip = -1 for none), until a sweep
 * moves no coordinate by more than tol_move*max(1,|b|inf), or max_sweeps.
 * Returns sweeps done, negative when the cap was hit. */
int orc_ccd(int n, int p, const double* X, double* b, double* r, double lam,
            int skip, double tol_move, int max_sweeps, int* piv, bp_t* work) {
  for (int s = 1; s <= max_sweeps; ++s) {
    double mx = 0.0, bmax = 0.0;
    for (int j = 0; j < p; ++j) {
      if (j == skip) continue;
      int pv;
      double d = orc_axis_update(n, p, X, b, r, lam, j, &pv, work);
      if (piv) piv[j] = pv;
      mx = fmax(mx, fabs(d));
    }
    for (int j = 0; j < p; ++j) bmax = fmax(bmax, fabs(b[j]));
    if (mx <= tol_move * fmax(1.0, bmax)) return s;
  }
  return -max_sweeps;
}

static double objective_r(int n, int p, const double* r, const double* b, double lam) {
  double f = 0.0;
  for (int i = 0; i < n; ++i) f += fabs(r[i]);
  for (int j = 0; j < p; ++j) f += lam * fabs(b[j]);
  return f;
}

/* ------------------------------------------------------------------ */
/* Sections 3.4-3.5: ternary chop along the locus of axis-wise minima  */
/* ------------------------------------------------------------------ */

typedef struct {
  int n, p; const double* X; const double* y; double lam;
  int k; const orc_opts* o; orc_stats* st;
  double* b; double* r;        /* working point, carried probe to probe */
  double* best_b; double best_f;
  int* piv; bp_t* work;
} chop_ctx;

/* One probe g(t): fix b_k = t (Section 3.5: the sub-search may not vary the
 * search axis), run coordinate descent on the other axes from the previous
 * probe's point, return F there. */
static double probe(chop_ctx* c, double t) {
  int n = c->n, p = c->p, k = c->k;
  double d = t - c->b[k];
  if (d != 0.0) {
    for (int i = 0; i < n; ++i) c->r[i] -= c->X[(size_t)i * p + k] * d;
    c->b[k] = t;
  }
  int s = orc_ccd(n, p, c->X, c->b, c->r, c->lam, k, c->o->tol_move,
                  c->o->probe_max_sweeps, NULL, c->work);
  c->st->sweeps += s < 0 ? -s : s;
  c->st->probes += 1;
  double f = objective_r(n, p, c->r, c->b, c->lam);
  if (f < c->best_f) { c->best_f = f; memcpy(c->best_b, c->b, sizeof(double) * p); }
  return f;
}

/* Ternary search on axis k starting from a CCD fixed point b (Sections
 * 3.4-3.5).  The initial range is centred on b_k with half-width
 * chop_bracket*max(1,|b_k|); while an end point is lower than the centre
 * the range is moved that way with doubled width (range extension,
 * Section 3.5).  Then the usual ternary step: probe the 1/3 and 2/3
 * points, drop the third beyond the higher probe (equal probes keep the
 * middle third).  The best probe seen is returned in b (and r recomputed).
 * Returns 1 if a probe improved on F(b). */
int orc_chop(int n, int p, const double* X, const double* y, double* b,
             double* r, double lam, int k, const orc_opts* o, orc_stats* st,
             bp_t* work) {
  double* wb = (double*)malloc(sizeof(double) * (size_t)(2 * p + n));
  double* bb = wb + p;
  double* wr = bb + p;
  memcpy(wb, b, sizeof(double) * p);
  memcpy(wr, r, sizeof(double) * n);
  chop_ctx c = {n, p, X, y, lam, k, o, st, wb, wr, bb, 0.0, NULL, work};
  double f0 = objective_r(n, p, r, b, lam);
  c.best_f = f0;
  memcpy(bb, b, sizeof(double) * p);

  double ck = b[k];
  double scale = fmax(1.0, fabs(ck));
  double delta = o->chop_bracket * scale;
  double a = ck - delta, m = ck, e = ck + delta;
  double gm = f0, ga = probe(&c, a), ge = probe(&c, e);
  int ext = 0;
  while (ext < o->chop_max_extend) {
    if (ga < gm) {             /* minimum lies left of the centre */
      e = m; ge = gm; m = a; gm = ga; delta *= 2.0; a = m - delta; ga = probe(&c, a);
    } else if (ge < gm) {      /* minimum lies right of the centre */
      a = m; ga = gm; m = e; gm = ge; delta *= 2.0; e = m + delta; ge = probe(&c, e);
    } else {
      break;
    }
    ++ext;
  }
  st->extends += ext;
  double lo = a, hi = e;
  int probes = 0;
  if (o->chop_sections == 4) {
    /* four equal sections, probes at the three inner points; for a convex
     * g the minimum lies within one section of the lowest probe, so keep
     * the two sections around it (the leftmost lowest on ties) */
    while (hi - lo > o->chop_tol * scale && probes + 3 <= o->chop_max_probes) {
      double h = (hi - lo) / 4.0;
      double t1 = lo + h, t2 = lo + 2.0 * h, t3 = hi - h;
      double g1 = probe(&c, t1), g2 = probe(&c, t2), g3 = probe(&c, t3);
      probes += 3;
      if (g1 <= g2 && g1 <= g3) hi = t2;
      else if (g2 <= g3) { lo = t1; hi = t3; }
      else lo = t2;
    }
  } else {
    while (hi - lo > o->chop_tol * scale && probes + 2 <= o->chop_max_probes) {
      double m1 = lo + (hi - lo) / 3.0, m2 = hi - (hi - lo) / 3.0;
      double g1 = probe(&c, m1), g2 = probe(&c, m2);
      probes += 2;
      if (g1 < g2) hi = m2;
      else if (g1 > g2) lo = m1;
      else { lo = m1; hi = m2; }
    }
  }
  int improved = c.best_f < f0;
  if (improved) {
    memcpy(b, bb, sizeof(double) * p);
    residual(n, p, X, y, b, r);
  }
  free(wb);
  return improved;
}

/* ------------------------------------------------------------------ */
/* exact finish: vertex polish                                         */
/* ------------------------------------------------------------------ */

/* A basis is p hyperplanes with linearly independent normals: row i
 * (normal x_i, x_i.b = y_i) or coordinate j (normal e_j, b_j = 0).  A
 * coordinate put in only to complete the basis while b_j != 0 is a
 * "phantom": it pins b_j at its current value, and its multiplier must
 * vanish at an optimum.  code >= 0 row, code < 0 coordinate -(code+1). */
typedef struct { int code; int phantom; } cons_t;

static void cons_normal(int p, const double* X, cons_t c, double* v) {
  if (c.code >= 0) {
    memcpy(v, X + (size_t)c.code * p, sizeof(double) * p);
  } else {
    memset(v, 0, sizeof(double) * p);
    v[-c.code - 1] = 1.0;
  }
}

/* Incremental independence test: reduce v against stored echelon rows. */
static int try_add(int p, double* ech, int* pcol, int* m, double* v, double tol) {
  double vmax0 = 0.0;
  for (int j = 0; j < p; ++j) vmax0 = fmax(vmax0, fabs(v[j]));
  if (vmax0 == 0.0) return 0;
  for (int q = 0; q < *m; ++q) {
    double f = v[pcol[q]] / ech[(size_t)q * p + pcol[q]];
    if (f != 0.0) for (int j = 0; j < p; ++j) v[j] -= f * ech[(size_t)q * p + j];
  }
  int best = -1; double bv = 0.0;
  for (int j = 0; j < p; ++j) if (fabs(v[j]) > bv) { bv = fabs(v[j]); best = j; }
  if (bv <= tol * vmax0) return 0;
  memcpy(ech + (size_t)(*m) * p, v, sizeof(double) * p);
  pcol[*m] = best;
  (*m)++;
  return 1;
}

/* Build a basis at a coordinate-descent fixed point: the hyperplanes each
 * axis update landed on (row piv[j], or b_j = 0 for the penalty
 * breakpoint), kept when independent, then completed with coordinate
 * hyperplanes j = 0,1,.. . */
static void build_basis(int p, const double* X, const double* b, const int* piv,
                        cons_t* basis) {
  double* ech = (double*)malloc(sizeof(double) * (size_t)(p * p + p));
  double* v = ech + (size_t)p * p;
  int* pcol = (int*)malloc(sizeof(int) * (size_t)p);
  int m = 0;
  for (int j = 0; j < p && m < p; ++j) {
    if (piv[j] == -2) continue;
    cons_t c = {piv[j] >= 0 ? piv[j] : COORD_ID(j), 0};
    int dup = 0;
    for (int q = 0; q < m; ++q) if (basis[q].code == c.code) dup = 1;
    if (dup) continue;
    cons_normal(p, X, c, v);
    if (try_add(p, ech, pcol, &m, v, 1e-9)) basis[m - 1] = c;
  }
  for (int j = 0; j < p && m < p; ++j) {
    cons_t c = {COORD_ID(j), b[j] != 0.0};
    int dup = 0;
    for (int q = 0; q < m; ++q) if (basis[q].code == c.code) dup = 1;
    if (dup) continue;
    cons_normal(p, X, c, v);
    if (try_add(p, ech, pcol, &m, v, 1e-9)) basis[m - 1] = c;
  }
  free(ech);
  free(pcol);
}

/* Polish from a basis to a certified optimal vertex.
 *
 * At the current point every basis hyperplane holds (phantoms hold b_j at
 * its value).  Off the basis F is differentiable near b with gradient
 *   g = -sum_{rows i not in basis} sign(r_i) x_i + lambda sign(b_j) e_j
 *       (the second sum over coordinates that are not real basis members).
 * Solving B^T mu = -g gives one multiplier per basis hyperplane; the point
 * is optimal iff |mu| <= 1 on rows, <= lambda on real coordinates and
 * == 0 on phantoms (0 is in the subdifferential).  Otherwise release the
 * most violating hyperplane q: direction d with B d = sign(mu_q) e_q keeps
 * the others, and F decreases along d at rate |mu_q| - cap_q.  Along d,
 * F(b + t d) = sum_i |r_i - t v_i| + lambda sum_j |b_j + t d_j| (v = X d),
 * again a weighted median; the breakpoint landed on enters the basis.
 * Returns the number of steps, or -1 when max_pivots was hit.  *nonunique is
 * set when the optimum found is not a strict vertex. */
int orc_polish(int n, int p, const double* X, const double* y, double* b,
               double* r, double lam, cons_t* basis, const orc_opts* o,
               int max_pivots, int* is_opt, int* nonunique) {
  size_t P = (size_t)p;
  double* B = (double*)malloc(sizeof(double) * (P * P * 2 + P * 6));
  double* Bt = B + P * P;
  double* h = Bt + P * P;
  double* g = h + P;
  double* mu = g + P;
  double* d = mu + P;
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  char* inb = (char*)calloc((size_t)n, 1);
  bp_t* bp = (bp_t*)malloc(sizeof(bp_t) * (size_t)(n + p));
  int it = 0;
  *is_opt = 0;
  *nonunique = 0;
  double tol = o->tol_opt * fmax(1.0, lam);
  for (;;) {
    /* snap b onto the basis hyperplanes and refresh r */
    for (int k = 0; k < p; ++k) {
      cons_normal(p, X, basis[k], B + (size_t)k * p);
      int c = basis[k].code;
      h[k] = c >= 0 ? y[c] : (basis[k].phantom ? b[-c - 1] : 0.0);
    }
    memcpy(Bt, B, sizeof(double) * P * P);
    memcpy(d, h, sizeof(double) * P);
    if (gauss_solve(p, Bt, d, 1e-13) == 0) memcpy(b, d, sizeof(double) * P);
    for (int k = 0; k < p; ++k)
      if (basis[k].code < 0 && !basis[k].phantom) b[-basis[k].code - 1] = 0.0;
    residual(n, p, X, y, b, r);
    memset(inb, 0, (size_t)n);
    for (int k = 0; k < p; ++k) if (basis[k].code >= 0) inb[basis[k].code] = 1;

    /* multipliers */
    for (int j = 0; j < p; ++j) g[j] = 0.0;
    for (int i = 0; i < n; ++i) {
      if (inb[i]) continue;
      double s = sgn(r[i]);
      if (s != 0.0) for (int j = 0; j < p; ++j) g[j] -= s * X[(size_t)i * p + j];
    }
    for (int j = 0; j < p; ++j) {
      int real = 0;
      for (int k = 0; k < p; ++k)
        if (basis[k].code == COORD_ID(j) && !basis[k].phantom) real = 1;
      if (!real) g[j] += lam * sgn(b[j]);
    }
    for (int k = 0; k < p; ++k)
      for (int c = 0; c < p; ++c) Bt[(size_t)c * p + k] = B[(size_t)k * p + c];
    for (int j = 0; j < p; ++j) mu[j] = -g[j];
    if (gauss_solve(p, Bt, mu, 1e-13) != 0) break;
    int q = -1; double worst = tol;
    int phantoms = 0, at_cap = 0;
    for (int k = 0; k < p; ++k) {
      double cap = basis[k].code >= 0 ? 1.0 : (basis[k].phantom ? 0.0 : lam);
      double viol = fabs(mu[k]) - cap;
      if (basis[k].phantom) phantoms++;
      else if (viol > -1e-9 * fmax(1.0, cap)) at_cap++;
      if (viol > worst) { worst = viol; q = k; }
    }
    if (q < 0) {
      *is_opt = 1;
      *nonunique = phantoms > 0 || at_cap > 0;
      break;
    }
    if (it >= max_pivots) break;

    /* edge direction and exact line search */
    double sg = mu[q] > 0 ? 1.0 : -1.0;
    memcpy(Bt, B, sizeof(double) * P * P);
    for (int k = 0; k < p; ++k) d[k] = 0.0;
    d[q] = sg;
    if (gauss_solve(p, Bt, d, 1e-13) != 0) break;
    int m = 0;
    for (int i = 0; i < n; ++i) {
      double vi = 0.0;
      for (int j = 0; j < p; ++j) vi += X[(size_t)i * p + j] * d[j];
      v[i] = vi;
      if (inb[i]) {
        if (i == basis[q].code) { bp[m].z = 0.0; bp[m].w = fabs(vi); bp[m].id = i; ++m; }
        continue; /* the other basis rows stay on their hyperplanes */
      }
      if (vi != 0.0) { bp[m].z = r[i] / vi; bp[m].w = fabs(vi); bp[m].id = i; ++m; }
    }
    for (int j = 0; j < p; ++j) {
      int kk = -1;
      for (int k = 0; k < p; ++k) if (basis[k].code == COORD_ID(j)) kk = k;
      if (kk >= 0 && kk != q) continue;
      if (kk == q && !basis[q].phantom) {
        bp[m].z = 0.0; bp[m].w = lam * fabs(d[j]); bp[m].id = COORD_ID(j); ++m;
        continue;
      }
      if (d[j] != 0.0) { bp[m].z = -b[j] / d[j]; bp[m].w = lam * fabs(d[j]); bp[m].id = COORD_ID(j); ++m; }
    }
    int own;
    double ts = weighted_median(bp, m, 0.0, &own);
    if (own == INT32_MIN) break; /* flat along the edge: cannot happen when F decreases */
    for (int j = 0; j < p; ++j) b[j] += ts * d[j];
    basis[q].code = own;
    basis[q].phantom = 0;
    ++it;
  }
  free(B); free(v); free(inb); free(bp);
  return *is_opt ? it : -1;
}

/* ------------------------------------------------------------------ */
/* one lambda: CCD, chop when not optimal, polish                       */
/* ------------------------------------------------------------------ */

static int fit_one(int n, int p, const double* X, const double* y, double lam,
                   double* b, double* r, const orc_opts* o, orc_stats* st,
                   cons_t* basis, int* piv, bp_t* work) {
  int status = ORC_FIT_OK;
  residual(n, p, X, y, b, r);
  for (int j = 0; j < p; ++j) piv[j] = -2;
  int s = orc_ccd(n, p, X, b, r, lam, -1, o->tol_move, o->max_sweeps, piv, work);
  st->sweeps += s < 0 ? -s : s;
  if (s < 0) status |= ORC_FIT_MAX_ITERS;
  int is_opt = 0, nonu = 0;
  double* bb = (double*)malloc(sizeof(double) * (size_t)(p + n));
  double* rr = bb + p;
  /* stall test: is the CCD fixed point already optimal? */
  memcpy(bb, b, sizeof(double) * p); memcpy(rr, r, sizeof(double) * n);
  build_basis(p, X, b, piv, basis);
  orc_polish(n, p, X, y, bb, rr, lam, basis, o, 0, &is_opt, &nonu);
  st->ccd_optimal = is_opt;
  if (is_opt) { memcpy(b, bb, sizeof(double) * p); memcpy(r, rr, sizeof(double) * n); }
  if (!is_opt && o->chop && p >= 2) {
    /* Section 3.4: it does not matter which axis; take the largest |b_k| */
    int k = 0;
    for (int j = 1; j < p; ++j) if (fabs(b[j]) > fabs(b[k])) k = j;
    st->chop_ran = 1;
    orc_chop(n, p, X, y, b, r, lam, k, o, st, work);
    for (int j = 0; j < p; ++j) piv[j] = -2;
    s = orc_ccd(n, p, X, b, r, lam, -1, o->tol_move, o->max_sweeps, piv, work);
    st->sweeps += s < 0 ? -s : s;
    memcpy(bb, b, sizeof(double) * p); memcpy(rr, r, sizeof(double) * n);
    build_basis(p, X, b, piv, basis);
    orc_polish(n, p, X, y, bb, rr, lam, basis, o, 0, &is_opt, &nonu);
    st->chop_optimal = is_opt;
    if (is_opt) { memcpy(b, bb, sizeof(double) * p); memcpy(r, rr, sizeof(double) * n); }
  }
  if (!is_opt && o->polish) {
    build_basis(p, X, b, piv, basis);
    int it = orc_polish(n, p, X, y, b, r, lam, basis, o, o->max_pivots, &is_opt, &nonu);
    st->pivots += it < 0 ? o->max_pivots : it;
    if (!is_opt) status |= ORC_FIT_MAX_ITERS;
  }
  if (is_opt && nonu) status |= ORC_FIT_NONUNIQUE;
  free(bb);
  return status;
}

/* Fit one problem along a lambda path (descending), warm-starting each
 * lambda from the previous solution.  b_init may be NULL (zeros).
 * Outputs: b_out [L x p], f_out [L], status_out [L], basis_out [L x p]
 * (constraint codes, may be NULL), stats (may be NULL: one per lambda). */
void orc_fit_path(int n, int p, const double* X, const double* y, int L,
                  const double* lambdas, const double* b_init,
                  const orc_opts* o, double* b_out, double* f_out,
                  int* status_out, int* basis_out, orc_stats* stats) {
  double* b = (double*)calloc((size_t)(p + n), sizeof(double));
  double* r = b + p;
  int* piv = (int*)malloc(sizeof(int) * (size_t)p);
  cons_t* basis = (cons_t*)malloc(sizeof(cons_t) * (size_t)p);
  bp_t* work = (bp_t*)malloc(sizeof(bp_t) * (size_t)(n + p + 1));
  if (b_init) memcpy(b, b_init, sizeof(double) * p);
  for (int l = 0; l < L; ++l) {
    orc_stats st;
    memset(&st, 0, sizeof st);
    double lam = lambdas[l];
    int status;
    if (!(lam >= 0.0) || !isfinite(lam)) {
      status = ORC_FIT_BAD_INPUT;
      memset(b_out + (size_t)l * p, 0, sizeof(double) * p);
      f_out[l] = 0.0;
      if (basis_out) for (int j = 0; j < p; ++j) basis_out[(size_t)l * p + j] = COORD_ID(j);
    } else {
      lam = fmax(lam, o->lambda_min_floor);
      status = fit_one(n, p, X, y, lam, b, r, o, &st, basis, piv, work);
      memcpy(b_out + (size_t)l * p, b, sizeof(double) * p);
      f_out[l] = orc_objective(n, p, X, y, b, lam);
      if (basis_out) for (int j = 0; j < p; ++j) basis_out[(size_t)l * p + j] = basis[j].code;
    }
    status_out[l] = status;
    if (stats) stats[l] = st;
  }
  free(b); free(piv); free(basis); free(work);
}

/* Many independent problems (OpenMP over problems).  Problem q's design is
 * X_cat + xoff[q] (n[q] x p[q] row-major), targets y_cat + yoff[q];
 * lambdas [B x L]; b_out [B x L x P] zero padded beyond p[q]; f_out and
 * status_out [B x L].  Returns the OpenMP thread count used. */
int orc_fit_batch(int B, const double* X_cat, const int64_t* xoff,
                  const double* y_cat, const int64_t* yoff, const int* n,
                  const int* p, int P, int L, const double* lambdas,
                  const orc_opts* o, double* b_out, double* f_out,
                  int* status_out, int nthreads) {
  int used = 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
  {
#pragma omp single
    used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
#endif
    for (int q = 0; q < B; ++q) {
      int pq = p[q];
      double* bo = (double*)malloc(sizeof(double) * (size_t)L * pq);
      orc_fit_path(n[q], pq, X_cat + xoff[q], y_cat + yoff[q], L,
                   lambdas + (size_t)q * L, NULL, o, bo, f_out + (size_t)q * L,
                   status_out + (size_t)q * L, NULL, NULL);
      for (int l = 0; l < L; ++l) {
        double* dst = b_out + ((size_t)q * L + l) * P;
        memset(dst, 0, sizeof(double) * P);
        memcpy(dst, bo + (size_t)l * pq, sizeof(double) * pq);
      }
      free(bo);
    }
#ifdef _OPENMP
  }
#endif
  return used;
}

/* ------------------------------------------------------------------ */
/* lambda_max                                                           */
/* ------------------------------------------------------------------ */

/* b = 0 is optimal iff 0 lies in -X^T s + lambda [-1,1]^p for some
 * s in sign(y); with no zero targets this is lambda >= |X^T sign(y)|_inf. */
double orc_lambda_max(int n, int p, const double* X, const double* y) {
  double best = 0.0;
  for (int j = 0; j < p; ++j) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += X[(size_t)i * p + j] * sgn(y[i]);
    best = fmax(best, fabs(c));
  }
  return best;
}

/* ------------------------------------------------------------------ */
/* Section 3.2: brute-force vertex evaluation                           */
/* ------------------------------------------------------------------ */

/* The optimum of the LP lies at a vertex; in b-space a vertex is where p
 * of the hyperplanes {x_i.b = y_i} U {b_j = 0} meet (Section 3.2).  Every
 * p-subset is solved (Gaussian elimination, partial pivoting; singular
 * subsets skipped) and F evaluated.  Returns min F; b_best gets the first
 * minimiser; *n_distinct counts distinct minimising vertices (up to 64;
 * > 1 means the optimum is not unique). */
double orc_brute_force(int n, int p, const double* X, const double* y,
                       double lam, double* b_best, int* n_distinct) {
  int H = n + p;
  int* idx = (int*)malloc(sizeof(int) * (size_t)p);
  double* A = (double*)malloc(sizeof(double) * (size_t)(p * p + 2 * p));
  double* rhs = A + p * p;
  double* opt = (double*)malloc(sizeof(double) * 64 * (size_t)p);
  int nopt = 0;
  double fbest = INFINITY;
  for (int k = 0; k < p; ++k) idx[k] = k;
  if (p > H) { free(idx); free(A); free(opt); *n_distinct = 0; return NAN; }
  for (;;) {
    for (int k = 0; k < p; ++k) {
      int hk = idx[k];
      if (hk < n) {
        memcpy(A + (size_t)k * p, X + (size_t)hk * p, sizeof(double) * p);
        rhs[k] = y[hk];
      } else {
        memset(A + (size_t)k * p, 0, sizeof(double) * p);
        A[(size_t)k * p + (hk - n)] = 1.0;
        rhs[k] = 0.0;
      }
    }
    if (gauss_solve(p, A, rhs, 1e-10) == 0) {
      double f = orc_objective(n, p, X, y, rhs, lam);
      double tolf = 1e-11 * fmax(1.0, fabs(f));
      if (f < fbest - tolf) {
        fbest = f;
        nopt = 1;
        memcpy(opt, rhs, sizeof(double) * p);
      } else if (fabs(f - fbest) <= tolf) {
        int same = 0;
        for (int q = 0; q < nopt && !same; ++q) {
          double dm = 0.0, sc = 1.0;
          for (int j = 0; j < p; ++j) {
            dm = fmax(dm, fabs(opt[(size_t)q * p + j] - rhs[j]));
            sc = fmax(sc, fabs(rhs[j]));
          }
          if (dm <= 1e-8 * sc) same = 1;
        }
        if (!same && nopt < 64) memcpy(opt + (size_t)(nopt++) * p, rhs, sizeof(double) * p);
      }
    }
    int k = p - 1;
    while (k >= 0 && idx[k] == H - p + k) --k;
    if (k < 0) break;
    idx[k]++;
    for (int q = k + 1; q < p; ++q) idx[q] = idx[q - 1] + 1;
  }
  if (nopt > 0) memcpy(b_best, opt, sizeof(double) * p);
  *n_distinct = nopt;
  free(idx); free(A); free(opt);
  return fbest;
}

/* ------------------------------------------------------------------ */
/* Section 3.1: dense simplex of the split-variable LP                  */
/* ------------------------------------------------------------------ */

/* Variables (all >= 0): x_p[0..p), x_n[0..p), r_p[0..n), r_n[0..n) with
 *   X (x_p - x_n) + r_p - r_n = y,
 *   minimise lambda * sum(x_p + x_n) + sum(r_p + r_n).
 * Start from the basis r_p (y_i >= 0) / r_n (y_i < 0); textbook tableau
 * simplex with Bland's rule (lowest-index entering variable, lowest-index
 * leaving variable among ratio ties).  Returns the optimum value, b in
 * b_out, or NAN if max_iter pivots did not finish. */
double orc_simplex(int n, int p, const double* X, const double* y, double lam,
                   double* b_out, int max_iter) {
  int m = 2 * p + 2 * n;
  int W = m + 1;
  double* T = (double*)calloc((size_t)(n + 1) * W, sizeof(double));
  int* bas = (int*)malloc(sizeof(int) * (size_t)n);
  double* cost = (double*)malloc(sizeof(double) * (size_t)m);
  for (int j = 0; j < 2 * p; ++j) cost[j] = lam;
  for (int j = 2 * p; j < m; ++j) cost[j] = 1.0;
  for (int i = 0; i < n; ++i) {
    double s = y[i] >= 0 ? 1.0 : -1.0;
    double* row = T + (size_t)i * W;
    for (int j = 0; j < p; ++j) {
      row[j] = s * X[(size_t)i * p + j];
      row[p + j] = -s * X[(size_t)i * p + j];
    }
    row[2 * p + i] = s;
    row[2 * p + n + i] = -s;
    row[m] = s * y[i];
    bas[i] = s > 0 ? 2 * p + i : 2 * p + n + i;
  }
  /* reduced-cost row: c_j - sum_i c_B(i) T[i][j]; last entry -objective */
  double* z = T + (size_t)n * W;
  for (int j = 0; j <= m; ++j) {
    double s = j < m ? cost[j] : 0.0;
    for (int i = 0; i < n; ++i) s -= cost[bas[i]] * T[(size_t)i * W + j];
    z[j] = s;
  }
  const double eps = 1e-11;
  int it = 0, done = 0;
  for (; it < max_iter; ++it) {
    int e = -1;
    for (int j = 0; j < m; ++j) if (z[j] < -eps) { e = j; break; }
    if (e < 0) { done = 1; break; }
    int l = -1; double best = INFINITY;
    for (int i = 0; i < n; ++i) {
      double a = T[(size_t)i * W + e];
      if (a > eps) {
        double ratio = T[(size_t)i * W + m] / a;
        if (ratio < best - 1e-14 || (fabs(ratio - best) <= 1e-14 && l >= 0 && bas[i] < bas[l])) {
          best = ratio; l = i;
        }
      }
    }
    if (l < 0) break; /* unbounded: impossible for this LP */
    double* pr = T + (size_t)l * W;
    double pv = pr[e];
    for (int j = 0; j <= m; ++j) pr[j] /= pv;
    for (int i = 0; i <= n; ++i) {
      if (i == l) continue;
      double* ri = T + (size_t)i * W;
      double f = ri[e];
      if (f != 0.0) for (int j = 0; j <= m; ++j) ri[j] -= f * pr[j];
    }
    bas[l] = e;
  }
  double val = NAN;
  if (done) {
    memset(b_out, 0, sizeof(double) * p);
    val = 0.0;
    for (int i = 0; i < n; ++i) {
      double xv = T[(size_t)i * W + m];
      val += cost[bas[i]] * xv;
      if (bas[i] < p) b_out[bas[i]] += xv;
      else if (bas[i] < 2 * p) b_out[bas[i] - p] -= xv;
    }
  }
  free(T); free(bas); free(cost);
  return val;
}

/* ------------------------------------------------------------------ */
/* optimality certificate (dual LP, duality gap)                        */
/* ------------------------------------------------------------------ */

/* Dual of min_b F(b):  max_u y.u  s.t. |u_i| <= 1, |(X^T u)_j| <= lambda.
 * Any feasible u gives F* >= y.u (weak duality), so F(b) - y.u bounds the
 * sub-optimality of b.  At b take N = rows with |r_i| > eps_r, E the rest,
 * S = {j : |b_j| > eps_b}; u_N = sign(r_N) and u_E solves (least squares,
 * minimum norm) X_{E,S}^T u_E = lambda sign(b_S) - X_{N,S}^T u_N, the
 * stationarity condition on S.  u is then scaled into the dual feasible
 * set.  Returns the gap F(b) - y.u; out[0] = y.u, out[1] = max|u_E|,
 * out[2] = max_{j not in S} |(X^T u)_j| / lambda, out[3] = |E|, out[4] = |S|,
 * out[5] = 1 if the certificate also shows the minimiser is unique (|E| =
 * |S|, X_{E,S} nonsingular, strict bounds). */
double orc_certify(int n, int p, const double* X, const double* y,
                   const double* b, double lam, double eps_r, double eps_b,
                   double* out) {
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* u = (double*)calloc((size_t)n, sizeof(double));
  int* E = (int*)malloc(sizeof(int) * (size_t)n);
  int* S = (int*)malloc(sizeof(int) * (size_t)p);
  residual(n, p, X, y, b, r);
  double ymax = 0.0;
  for (int i = 0; i < n; ++i) ymax = fmax(ymax, fabs(y[i]));
  double bmax = 0.0;
  for (int j = 0; j < p; ++j) bmax = fmax(bmax, fabs(b[j]));
  int ne = 0, ns = 0;
  for (int i = 0; i < n; ++i) {
    if (fabs(r[i]) > eps_r * fmax(1.0, ymax)) u[i] = sgn(r[i]);
    else E[ne++] = i;
  }
  for (int j = 0; j < p; ++j) if (fabs(b[j]) > eps_b * fmax(1.0, bmax)) S[ns++] = j;
  /* rhs_s = lambda sign(b_s) - sum_N u_i x_is */
  double* rhs = (double*)malloc(sizeof(double) * (size_t)(ns + 1));
  for (int a = 0; a < ns; ++a) {
    int j = S[a];
    double s = lam * sgn(b[j]);
    for (int i = 0; i < n; ++i) if (u[i] != 0.0) s -= u[i] * X[(size_t)i * p + j];
    rhs[a] = s;
  }
  int solved = 1, unique_ok = (ne == ns);
  if (ne > 0 && ns > 0) {
    /* A = X_{E,S}^T  (ns x ne); min-norm LS: if ne >= ns, u_E = A^T (A A^T)^-1 rhs,
     * else u_E = (A^T A)^-1 A^T rhs. */
    if (ne >= ns) {
      double* G = (double*)malloc(sizeof(double) * (size_t)ns * ns);
      double* t = (double*)malloc(sizeof(double) * (size_t)ns);
      for (int a = 0; a < ns; ++a)
        for (int c = 0; c < ns; ++c) {
          double s = 0.0;
          for (int e = 0; e < ne; ++e)
            s += X[(size_t)E[e] * p + S[a]] * X[(size_t)E[e] * p + S[c]];
          G[(size_t)a * ns + c] = s;
        }
      memcpy(t, rhs, sizeof(double) * ns);
      if (gauss_solve(ns, G, t, 1e-14) != 0) { solved = 0; unique_ok = 0; }
      else
        for (int e = 0; e < ne; ++e) {
          double s = 0.0;
          for (int a = 0; a < ns; ++a) s += X[(size_t)E[e] * p + S[a]] * t[a];
          u[E[e]] = s;
        }
      free(G); free(t);
    } else {
      double* G = (double*)malloc(sizeof(double) * (size_t)ne * ne);
      double* t = (double*)malloc(sizeof(double) * (size_t)ne);
      for (int a = 0; a < ne; ++a) {
        for (int c = 0; c < ne; ++c) {
          double s = 0.0;
          for (int q = 0; q < ns; ++q)
            s += X[(size_t)E[a] * p + S[q]] * X[(size_t)E[c] * p + S[q]];
          G[(size_t)a * ne + c] = s;
        }
        double s = 0.0;
        for (int q = 0; q < ns; ++q) s += X[(size_t)E[a] * p + S[q]] * rhs[q];
        t[a] = s;
      }
      if (gauss_solve(ne, G, t, 1e-14) != 0) solved = 0;
      else for (int a = 0; a < ne; ++a) u[E[a]] = t[a];
      free(G); free(t);
    }
  }
  /* scale into the dual feasible set */
  double umax = 0.0, cmax_off = 0.0, cmax = 0.0;
  for (int e = 0; e < ne; ++e) umax = fmax(umax, fabs(u[E[e]]));
  char* inS = (char*)calloc((size_t)p, 1);
  for (int a = 0; a < ns; ++a) inS[S[a]] = 1;
  for (int j = 0; j < p; ++j) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += X[(size_t)i * p + j] * u[i];
    cmax = fmax(cmax, fabs(c));
    if (!inS[j]) cmax_off = fmax(cmax_off, fabs(c));
  }
  double theta = 1.0;
  for (int i = 0; i < n; ++i) theta = fmax(theta, fabs(u[i]));
  if (lam > 0) theta = fmax(theta, cmax / lam);
  double yu = 0.0;
  for (int i = 0; i < n; ++i) yu += y[i] * u[i] / theta;
  double f = orc_objective(n, p, X, y, b, lam);
  if (out) {
    out[0] = yu;
    out[1] = umax;
    out[2] = lam > 0 ? cmax_off / lam : INFINITY;
    out[3] = ne;
    out[4] = ns;
    out[5] = (solved && unique_ok && umax < 1.0 - 1e-9 &&
              (lam > 0 ? cmax_off < lam * (1.0 - 1e-9) : 0)) ? 1.0 : 0.0;
  }
  free(r); free(u); free(E); free(S); free(rhs); free(inS);
  return f - yu;
}

/* ------------------------------------------------------------------ */
/* gradient of a validation LAD loss at the final vertex               */
/* ------------------------------------------------------------------ */

/* At a strict optimal vertex with basis rows R (|R| = |S|) and zero
 * coordinates Z, b_S = X_{R,S}^{-1} y_R and b_Z = 0 do not depend on lambda,
 * so locally b is a smooth function of (y_R, X_{R,S}) alone.
 * With L = sum_v |y_v - x_v.b| over validation rows:
 *   g_S = dL/db_S = -sum_v sign(r_v) x_{v,S}
 *   X_{R,S}^T w = g_S
 *   dL/dy_R = w,  dL/dX_{R,S} = -w b_S^T,  other training entries 0
 *   dL/dy_v = sign(r_v),  dL/dX_v = -sign(r_v) b^T,  dL/dlambda = 0.
 * All outputs are scaled by `up` (the upstream derivative).  `basis` holds
 * the p constraint codes of the vertex (rows >= 0, coordinate j as -(j+1)).
 * Returns 0, or -1 when the vertex is not strict (singular X_{R,S} or a
 * row count that does not match the support). */
int orc_grad(int n, int p, const double* X, const double* y, const double* b,
             const int* basis, int nv, const double* Xv, const double* yv,
             double up, double* gy, double* gX, double* gyv, double* gXv,
             double* glam) {
  (void)y; /* b already encodes y through the vertex equations */
  int* R = (int*)malloc(sizeof(int) * (size_t)p);
  int* S = (int*)malloc(sizeof(int) * (size_t)p);
  char* inZ = (char*)calloc((size_t)p, 1);
  int nr = 0, ns = 0;
  for (int k = 0; k < p; ++k) {
    if (basis[k] >= 0) R[nr++] = basis[k];
    else inZ[-basis[k] - 1] = 1;
  }
  for (int j = 0; j < p; ++j) if (!inZ[j]) S[ns++] = j;
  memset(gy, 0, sizeof(double) * (size_t)n);
  memset(gX, 0, sizeof(double) * (size_t)n * p);
  *glam = 0.0;
  double* gS = (double*)calloc((size_t)p, sizeof(double));
  for (int v = 0; v < nv; ++v) {
    double rv = yv[v];
    for (int j = 0; j < p; ++j) rv -= Xv[(size_t)v * p + j] * b[j];
    double s = sgn(rv);
    gyv[v] = up * s;
    for (int j = 0; j < p; ++j) gXv[(size_t)v * p + j] = -up * s * b[j];
    for (int a = 0; a < ns; ++a) gS[a] -= s * Xv[(size_t)v * p + S[a]];
  }
  int rc = 0;
  if (nr != ns) rc = -1;
  else if (ns > 0) {
    double* M = (double*)malloc(sizeof(double) * (size_t)ns * ns);
    for (int a = 0; a < ns; ++a)      /* M = X_{R,S}^T */
      for (int c = 0; c < ns; ++c) M[(size_t)a * ns + c] = X[(size_t)R[c] * p + S[a]];
    if (gauss_solve(ns, M, gS, 1e-13) != 0) rc = -1;
    else
      for (int c = 0; c < ns; ++c) {
        gy[R[c]] = up * gS[c];
        for (int a = 0; a < ns; ++a) gX[(size_t)R[c] * p + S[a]] = -up * gS[c] * b[S[a]];
      }
    free(M);
  }
  free(R); free(S); free(inZ); free(gS);
  return rc;
}
