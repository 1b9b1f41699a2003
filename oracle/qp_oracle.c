/*
 * qp_oracle.c -- plain, slow FP64 CPU oracle for the implicit-complementarity
 * interior-point method for dense convex QPs (paper: "A Differentiable
 * Interior-Point Method in Single Precision").
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA path.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Problem (eq. 1):  min 1/2 x'Qx + q'x  s.t.  A x = b (p rows),  G x <= h (m rows),
 * slack form G x + s = h, s >= 0.  Matrices are dense, row-major, FP64.
 * Letters: n variables, p equality rows, m inequality rows (the paper writes
 * m for the equality count and p for the inequality count; only the letters
 * differ).
 *
 * Every function follows the paper's steps in its order and notation:
 *   - retraction b_k(v) and its derivatives: eq. 11, eq. 12, App. C;
 *   - residuals: eq. 4 and eq. 10;
 *   - Newton system: eq. 14 (partially condensed, symmetric), solved here as a
 *     full (n+m+p)-square system by Gaussian elimination with partial
 *     pivoting -- no Schur complement, no Cholesky -- then the remaining
 *     direction components recovered from the rows of eq. 13;
 *   - step length: eq. 7;
 *   - Alg. 1 (solve), Alg. 2 (relax), Alg. 3 (gradients);
 *   - standard formulation (ablation): eq. 6 / eq. 8 with a textbook
 *     Mehrotra predictor-corrector.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   R1  kappa = s'z / m with m = number of inequalities (the mean
 *       complementarity; the printed divisor names the equality count).
 *   R2  c in eq. 13/14 is the vector c_i = d/dkappa b_k(v_i) = 1/sqrt(v_i^2+4k).
 *   R3  Alg. 3's adjoint solve uses right-hand side (-grad_x l, 0, 0): the
 *       eq. 14 matrix is symmetric, so this is the transpose solve of the
 *       implicit function theorem (App. A); dz is recovered from eq. 13's
 *       fourth row with zero residuals, dz = B_k(v) dv.
 *   R5  sigma: Mehrotra's (mu_aff/kappa)^3 clipped to [0,1] by default, or a
 *       constant; kappa_target is floored at kappa_min.
 *   R6  predictor (kappa_target = 0) only sets sigma; the corrector re-solves
 *       the same matrix with kappa_target = sigma*kappa; no second-order term
 *       (z.*s = kappa holds exactly through the retraction).
 *   R7  eq. 7 unscaled for the implicit method (step_frac = 1); the standard
 *       ablation uses fraction-to-boundary 0.99.
 *   R8  convergence on the scaled infinity-norm residual (or absolute).
 *   R13 initial point: CVXOPT's cone-QP start (the paper cites it for Alg. 1).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OQP_SOLVED 0
#define OQP_MAX_ITER 1
#define OQP_STALLED 2
#define OQP_NUMERICAL 3
#define OQP_BAD_INPUT 4

typedef struct {
  int n, p, m; /* variables, equality rows, inequality rows */
  const double *Q, *q, *A, *b, *G, *h;
} oqp_problem;

typedef struct {
  double tol;        /* stop when the residual measure is below tol            */
  int max_iter;      /* iteration cap (the paper uses 100)                      */
  int sigma_mode;    /* 0: Mehrotra (mu_aff/kappa)^3, 1: constant sigma         */
  double sigma;      /* constant sigma                                          */
  double kappa_min;  /* floor on kappa_target                                   */
  int scaled;        /* 1: scaled residual measure, 0: absolute (paper's)       */
  double step_frac;  /* multiplies eq. 7's alpha (1 for the implicit method)    */
} oqp_settings;

#define IX(i, j, ld) ((size_t)(i) * (size_t)(ld) + (size_t)(j))

static double vmax_abs(int k, const double* a) {
  double r = 0.0;
  for (int i = 0; i < k; ++i) r = fmax(r, fabs(a[i]));
  return r;
}

/* ---------------------------------------------------------------------------
 * Retraction map (eq. 11) and its derivatives, cancellation-free (App. C).
 *   b_k(v)      = (v + sqrt(v^2+4k))/2            v >= 0
 *               = 2k / (sqrt(v^2+4k) - v)         v <  0
 *   d/dv b_k(v) = (1 + v/sqrt(v^2+4k))/2          v >= 0
 *               = 2k / (v^2 + 4k - v sqrt(v^2+4k)) v < 0
 *   d/dk b_k(v) = 1/sqrt(v^2+4k)                   (R2)
 * ------------------------------------------------------------------------- */
double oqp_retract(double v, double kappa) {
  double r = sqrt(v * v + 4.0 * kappa);
  if (v >= 0.0) return 0.5 * (v + r);
  return 2.0 * kappa / (r - v);
}

double oqp_retract_dv(double v, double kappa) {
  double r = sqrt(v * v + 4.0 * kappa);
  if (v >= 0.0) return 0.5 * (1.0 + v / r);
  return 2.0 * kappa / (v * v + 4.0 * kappa - v * r);
}

double oqp_retract_dk(double v, double kappa) { return 1.0 / sqrt(v * v + 4.0 * kappa); }

/* ---------------------------------------------------------------------------
 * Dense Gaussian elimination with partial pivoting (whole-row swaps).
 * ------------------------------------------------------------------------- */
static int lu_factor(int N, double* M, int* piv) {
  for (int k = 0; k < N; ++k) {
    int pr = k;
    double best = fabs(M[IX(k, k, N)]);
    for (int i = k + 1; i < N; ++i) {
      double a = fabs(M[IX(i, k, N)]);
      if (a > best) { best = a; pr = i; }
    }
    piv[k] = pr;
    if (!(best > 0.0) || !isfinite(best)) return -1;
    if (pr != k)
      for (int j = 0; j < N; ++j) {
        double t = M[IX(k, j, N)];
        M[IX(k, j, N)] = M[IX(pr, j, N)];
        M[IX(pr, j, N)] = t;
      }
    double inv = 1.0 / M[IX(k, k, N)];
    for (int i = k + 1; i < N; ++i) {
      double l = M[IX(i, k, N)] * inv;
      M[IX(i, k, N)] = l;
      if (l != 0.0)
        for (int j = k + 1; j < N; ++j) M[IX(i, j, N)] -= l * M[IX(k, j, N)];
    }
  }
  return 0;
}

static void lu_solve(int N, const double* M, const int* piv, double* r) {
  for (int k = 0; k < N; ++k)
    if (piv[k] != k) { double t = r[k]; r[k] = r[piv[k]]; r[piv[k]] = t; }
  for (int i = 0; i < N; ++i) {
    double acc = r[i];
    for (int j = 0; j < i; ++j) acc -= M[IX(i, j, N)] * r[j];
    r[i] = acc;
  }
  for (int i = N - 1; i >= 0; --i) {
    double acc = r[i];
    for (int j = i + 1; j < N; ++j) acc -= M[IX(i, j, N)] * r[j];
    r[i] = acc / M[IX(i, i, N)];
  }
}

/* ---------------------------------------------------------------------------
 * Residuals (eq. 4):  r_t = Qx + q + G'z + A'y,  r_e = Ax - b,  r_i = Gx + s - h,
 * and the terms the scaled measure divides by.
 * ------------------------------------------------------------------------- */
typedef struct {
  double *rt, *re, *ri;           /* n, p, m */
  double *Qx, *Gtz, *Aty, *Ax, *Gx; /* n, n, n, p, m */
} oqp_resid;

static void residuals(const oqp_problem* P, const double* x, const double* y,
                      const double* z, const double* s, oqp_resid* R) {
  int n = P->n, p = P->p, m = P->m;
  for (int i = 0; i < n; ++i) {
    double a = 0.0;
    for (int j = 0; j < n; ++j) a += P->Q[IX(i, j, n)] * x[j];
    R->Qx[i] = a;
    double c = 0.0;
    for (int k = 0; k < m; ++k) c += P->G[IX(k, i, n)] * z[k];
    R->Gtz[i] = c;
    double d = 0.0;
    for (int k = 0; k < p; ++k) d += P->A[IX(k, i, n)] * y[k];
    R->Aty[i] = d;
    R->rt[i] = a + P->q[i] + c + d;
  }
  for (int k = 0; k < p; ++k) {
    double a = 0.0;
    for (int j = 0; j < n; ++j) a += P->A[IX(k, j, n)] * x[j];
    R->Ax[k] = a;
    R->re[k] = a - P->b[k];
  }
  for (int k = 0; k < m; ++k) {
    double a = 0.0;
    for (int j = 0; j < n; ++j) a += P->G[IX(k, j, n)] * x[j];
    R->Gx[k] = a;
    R->ri[k] = a + s[k] - P->h[k];
  }
}

/* Residual measure (R8).  Scaled:
 *   max( |r_t| / max(1,|Qx|,|q|,|A'y|,|G'z|), |r_e| / max(1,|Ax|,|b|),
 *        |r_i| / max(1,|Gx|,|h|,|s|), max_i z_i s_i, |r_z|,|r_s| rel. to max(1,|z|,|s|) )
 * Absolute: max(|r_t|,|r_e|,|r_i|,|z.*s|,|r_z|,|r_s|), all infinity norms. */
static double residual_measure(const oqp_problem* P, const oqp_resid* R, const double* z,
                               const double* s, const double* rz, const double* rs,
                               int scaled) {
  int n = P->n, p = P->p, m = P->m;
  double et = vmax_abs(n, R->rt), ee = vmax_abs(p, R->re), ei = vmax_abs(m, R->ri);
  double ec = 0.0, ezs = 0.0;
  for (int k = 0; k < m; ++k) {
    ec = fmax(ec, fabs(z[k] * s[k]));
    if (rz) ezs = fmax(ezs, fmax(fabs(rz[k]), fabs(rs[k])));
  }
  if (!scaled) return fmax(fmax(fmax(et, ee), fmax(ei, ec)), ezs);
  double dt = fmax(1.0, fmax(fmax(vmax_abs(n, R->Qx), vmax_abs(n, P->q)),
                             fmax(vmax_abs(n, R->Aty), vmax_abs(n, R->Gtz))));
  double de = fmax(1.0, fmax(vmax_abs(p, R->Ax), vmax_abs(p, P->b)));
  double di = fmax(1.0, fmax(fmax(vmax_abs(m, R->Gx), vmax_abs(m, P->h)), vmax_abs(m, s)));
  double dz = fmax(1.0, fmax(vmax_abs(m, z), vmax_abs(m, s)));
  return fmax(fmax(fmax(et / dt, ee / de), fmax(ei / di, ec)), ezs / dz);
}

double oqp_kkt_measure(const oqp_problem* P, const double* x, const double* y,
                       const double* z, const double* s, int scaled) {
  int n = P->n, p = P->p, m = P->m;
  double* buf = (double*)calloc((size_t)(4 * n + 2 * p + 2 * m + 1), sizeof(double));
  oqp_resid R = {buf, buf + n, buf + n + p, buf + n + p + m, buf + 2 * n + p + m,
                 buf + 3 * n + p + m, buf + 4 * n + p + m, buf + 4 * n + 2 * p + m};
  residuals(P, x, y, z, s, &R);
  double r = residual_measure(P, &R, z, s, NULL, NULL, scaled);
  free(buf);
  return r;
}

/* Step length, eq. 7:  alpha = min(1, min_{ds<0} -s/ds, min_{dz<0} -z/dz). */
static double step_length(int m, const double* s, const double* z, const double* ds,
                          const double* dz) {
  double a = 1.0;
  for (int k = 0; k < m; ++k) {
    if (ds[k] < 0.0) a = fmin(a, -s[k] / ds[k]);
    if (dz[k] < 0.0) a = fmin(a, -z[k] / dz[k]);
  }
  return a;
}

/* ---------------------------------------------------------------------------
 * Initial point (R13, CVXOPT's cone-QP start):
 *   solve [Q A' G'; A 0 0; G 0 -I] (x, y, z) = (-q, b, h),  s = -z,
 *   then shift s (resp. z) by (1 + a) e when a = -min(s) (resp. -min(z)) is
 *   not clearly negative (a >= -1e-8 max(1, |s|_inf)).
 * ------------------------------------------------------------------------- */
static int initialize(const oqp_problem* P, double* x, double* y, double* z, double* s) {
  int n = P->n, p = P->p, m = P->m, N = n + p + m;
  double* M = (double*)calloc((size_t)N * N + N, sizeof(double));
  int* piv = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
  double* r = M + (size_t)N * N;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[IX(i, j, N)] = P->Q[IX(i, j, n)];
  for (int k = 0; k < p; ++k)
    for (int j = 0; j < n; ++j) {
      M[IX(n + k, j, N)] = P->A[IX(k, j, n)];
      M[IX(j, n + k, N)] = P->A[IX(k, j, n)];
    }
  for (int k = 0; k < m; ++k) {
    for (int j = 0; j < n; ++j) {
      M[IX(n + p + k, j, N)] = P->G[IX(k, j, n)];
      M[IX(j, n + p + k, N)] = P->G[IX(k, j, n)];
    }
    M[IX(n + p + k, n + p + k, N)] = -1.0;
  }
  for (int i = 0; i < n; ++i) r[i] = -P->q[i];
  for (int k = 0; k < p; ++k) r[n + k] = P->b[k];
  for (int k = 0; k < m; ++k) r[n + p + k] = P->h[k];
  int rc = lu_factor(N, M, piv);
  if (rc == 0) lu_solve(N, M, piv, r);
  if (rc == 0) {
    for (int i = 0; i < n; ++i) x[i] = r[i];
    for (int k = 0; k < p; ++k) y[k] = r[n + k];
    for (int k = 0; k < m; ++k) { z[k] = r[n + p + k]; s[k] = -z[k]; }
    if (m > 0) {
      double ap = -INFINITY, ad = -INFINITY;
      for (int k = 0; k < m; ++k) { ap = fmax(ap, -s[k]); ad = fmax(ad, -z[k]); }
      if (ap >= -1e-8 * fmax(1.0, vmax_abs(m, s)))
        for (int k = 0; k < m; ++k) s[k] += 1.0 + ap;
      if (ad >= -1e-8 * fmax(1.0, vmax_abs(m, z)))
        for (int k = 0; k < m; ++k) z[k] += 1.0 + ad;
    }
  }
  free(M);
  free(piv);
  return rc;
}

/* ---------------------------------------------------------------------------
 * One implicit Newton system (eq. 14) at manifold coordinates (v, kappa),
 * factored once and solved for any kappa_target.
 *   [ Q - G'G   G'      A' ] [dx]     [ r_t - G'(r_i + r_z - r_s) ]
 *   [ G        -B_k(-v)  0 ] [dv] = - [ r_i - r_s - c .* r_kappa  ]
 *   [ A         0        0 ] [dy]     [ r_e                       ]
 * then (eq. 13 rows 4-6)  dkappa = -r_kappa,
 *   dz = -r_z + B_k(v) dv + c dkappa,   ds = -r_s - B_k(-v) dv + c dkappa.
 * ------------------------------------------------------------------------- */
typedef struct {
  int N;
  double *M, *rhs;
  int* piv;
  double *Bp, *Bm, *c; /* B_k(v), B_k(-v), c  (m each) */
} oqp_newton;

static int newton_factor(const oqp_problem* P, const double* v, double kappa, oqp_newton* W) {
  int n = P->n, p = P->p, m = P->m, N = n + m + p;
  double* M = W->M;
  memset(M, 0, sizeof(double) * (size_t)N * N);
  for (int k = 0; k < m; ++k) {
    W->Bp[k] = oqp_retract_dv(v[k], kappa);
    W->Bm[k] = oqp_retract_dv(-v[k], kappa);
    W->c[k] = oqp_retract_dk(v[k], kappa);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double gg = 0.0;
      for (int k = 0; k < m; ++k) gg += P->G[IX(k, i, n)] * P->G[IX(k, j, n)];
      M[IX(i, j, N)] = P->Q[IX(i, j, n)] - gg;
    }
  for (int k = 0; k < m; ++k) {
    for (int j = 0; j < n; ++j) {
      M[IX(n + k, j, N)] = P->G[IX(k, j, n)];
      M[IX(j, n + k, N)] = P->G[IX(k, j, n)];
    }
    M[IX(n + k, n + k, N)] = -W->Bm[k];
  }
  for (int k = 0; k < p; ++k)
    for (int j = 0; j < n; ++j) {
      M[IX(n + m + k, j, N)] = P->A[IX(k, j, n)];
      M[IX(j, n + m + k, N)] = P->A[IX(k, j, n)];
    }
  W->N = N;
  return lu_factor(N, M, W->piv);
}

/* Solve eq. 14 for a given r_kappa and recover (dz, ds, dkappa) from eq. 13. */
static void newton_solve(const oqp_problem* P, oqp_newton* W, const double* rt,
                         const double* re, const double* ri, const double* rz,
                         const double* rs, double rkappa, double* dx, double* dv,
                         double* dy, double* dz, double* ds, double* dkappa) {
  int n = P->n, p = P->p, m = P->m, N = W->N;
  double* r = W->rhs;
  for (int i = 0; i < n; ++i) {
    double g = 0.0;
    for (int k = 0; k < m; ++k) g += P->G[IX(k, i, n)] * (ri[k] + rz[k] - rs[k]);
    r[i] = -(rt[i] - g);
  }
  for (int k = 0; k < m; ++k) r[n + k] = -(ri[k] - rs[k] - W->c[k] * rkappa);
  for (int k = 0; k < p; ++k) r[n + m + k] = -re[k];
  lu_solve(N, W->M, W->piv, r);
  for (int i = 0; i < n; ++i) dx[i] = r[i];
  for (int k = 0; k < m; ++k) dv[k] = r[n + k];
  for (int k = 0; k < p; ++k) dy[k] = r[n + m + k];
  *dkappa = -rkappa;
  for (int k = 0; k < m; ++k) {
    dz[k] = -rz[k] + W->Bp[k] * dv[k] + W->c[k] * (*dkappa);
    ds[k] = -rs[k] - W->Bm[k] * dv[k] + W->c[k] * (*dkappa);
  }
}

/* Work arrays for one problem. */
typedef struct {
  double* mem;
  oqp_resid R;
  oqp_newton W;
  double *v, *rz, *rs, *dx, *dv, *dy, *dz, *ds;
} oqp_work;

static int work_alloc(const oqp_problem* P, oqp_work* w) {
  int n = P->n, p = P->p, m = P->m, N = n + m + p;
  size_t tot = (size_t)N * N + N + 3 * (size_t)m + (4 * n + 2 * p + 2 * m + 1) +
               (3 * (size_t)m + 2 * n + 2 * p + 4 * (size_t)m + 8);
  w->mem = (double*)calloc(tot, sizeof(double));
  w->W.piv = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
  if (!w->mem || !w->W.piv) return -1;
  double* c = w->mem;
  w->W.M = c; c += (size_t)N * N;
  w->W.rhs = c; c += N;
  w->W.Bp = c; c += m;
  w->W.Bm = c; c += m;
  w->W.c = c; c += m;
  w->R.rt = c; c += n;
  w->R.re = c; c += p;
  w->R.ri = c; c += m;
  w->R.Qx = c; c += n;
  w->R.Gtz = c; c += n;
  w->R.Aty = c; c += n;
  w->R.Ax = c; c += p;
  w->R.Gx = c; c += m;
  w->v = c; c += m;
  w->rz = c; c += m;
  w->rs = c; c += m;
  w->dx = c; c += n;
  w->dv = c; c += m;
  w->dy = c; c += p;
  w->dz = c; c += m;
  w->ds = c; c += m;
  return 0;
}

static void work_free(oqp_work* w) {
  free(w->mem);
  free(w->W.piv);
}

static int finite_vec(int k, const double* a) {
  for (int i = 0; i < k; ++i)
    if (!isfinite(a[i])) return 0;
  return 1;
}

/* Equality-only problem (m = 0): one Newton step of [Q A'; A 0] is exact. */
static int solve_eq_only(const oqp_problem* P, const oqp_settings* S, double* x, double* y,
                         int* iters) {
  int n = P->n, p = P->p, N = n + p;
  double* M = (double*)calloc((size_t)N * N + N, sizeof(double));
  int* piv = (int*)malloc(sizeof(int) * (size_t)N);
  double* r = M + (size_t)N * N;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[IX(i, j, N)] = P->Q[IX(i, j, n)];
  for (int k = 0; k < p; ++k)
    for (int j = 0; j < n; ++j) {
      M[IX(n + k, j, N)] = P->A[IX(k, j, n)];
      M[IX(j, n + k, N)] = P->A[IX(k, j, n)];
    }
  for (int i = 0; i < n; ++i) r[i] = -P->q[i];
  for (int k = 0; k < p; ++k) r[n + k] = P->b[k];
  int rc = lu_factor(N, M, piv);
  if (rc == 0) {
    lu_solve(N, M, piv, r);
    for (int i = 0; i < n; ++i) x[i] = r[i];
    for (int k = 0; k < p; ++k) y[k] = r[n + k];
  }
  free(M);
  free(piv);
  *iters = 1;
  (void)S;
  return rc == 0 ? OQP_SOLVED : OQP_NUMERICAL;
}

/* ---------------------------------------------------------------------------
 * Alg. 1 (solve_qp) with the predictor-corrector extension (R5, R6).
 * x, y, z, s are outputs.
 * ------------------------------------------------------------------------- */
int oqp_solve(const oqp_problem* P, const oqp_settings* S, double* x, double* y, double* z,
              double* s, int* iters_out, double* res_out) {
  int n = P->n, p = P->p, m = P->m;
  *iters_out = 0;
  if (n < 1 || p < 0 || m < 0 || p > n) return OQP_BAD_INPUT;
  if (m == 0) {
    int st = solve_eq_only(P, S, x, y, iters_out);
    if (res_out) *res_out = oqp_kkt_measure(P, x, y, z, s, S->scaled);
    return st;
  }
  if (initialize(P, x, y, z, s) != 0) return OQP_NUMERICAL;
  oqp_work w;
  if (work_alloc(P, &w) != 0) return OQP_NUMERICAL;
  int status = OQP_MAX_ITER, it;
  double res = INFINITY;
  for (it = 0; it < S->max_iter; ++it) {
    /* manifold coordinates */
    double kappa = 0.0;
    for (int k = 0; k < m; ++k) { w.v[k] = z[k] - s[k]; kappa += s[k] * z[k]; }
    kappa /= (double)m; /* R1 */
    /* residuals (eq. 4, eq. 10) and convergence check */
    residuals(P, x, y, z, s, &w.R);
    for (int k = 0; k < m; ++k) {
      w.rz[k] = z[k] - oqp_retract(w.v[k], kappa);
      w.rs[k] = s[k] - oqp_retract(-w.v[k], kappa);
    }
    res = residual_measure(P, &w.R, z, s, w.rz, w.rs, S->scaled);
    if (!isfinite(res)) { status = OQP_NUMERICAL; break; }
    if (res < S->tol) { status = OQP_SOLVED; break; }
    /* Newton system at (v, kappa) */
    if (newton_factor(P, w.v, kappa, &w.W) != 0) { status = OQP_NUMERICAL; break; }
    double dk, sigma;
    /* predictor: kappa_target = 0 */
    newton_solve(P, &w.W, w.R.rt, w.R.re, w.R.ri, w.rz, w.rs, kappa, w.dx, w.dv, w.dy, w.dz,
                 w.ds, &dk);
    if (S->sigma_mode == 1) {
      sigma = S->sigma;
    } else {
      double aa = step_length(m, s, z, w.ds, w.dz);
      double mu = 0.0;
      for (int k = 0; k < m; ++k) mu += (s[k] + aa * w.ds[k]) * (z[k] + aa * w.dz[k]);
      mu /= (double)m;
      double ratio = mu / kappa;
      sigma = ratio * ratio * ratio;
      if (!(sigma >= 0.0)) sigma = 0.0;
      if (sigma > 1.0) sigma = 1.0;
    }
    double kt = fmax(sigma * kappa, S->kappa_min);
    /* corrector: same matrix, kappa_target = sigma * kappa */
    newton_solve(P, &w.W, w.R.rt, w.R.re, w.R.ri, w.rz, w.rs, kappa - kt, w.dx, w.dv, w.dy,
                 w.dz, w.ds, &dk);
    double alpha = S->step_frac * step_length(m, s, z, w.ds, w.dz);
    for (int i = 0; i < n; ++i) x[i] += alpha * w.dx[i];
    for (int k = 0; k < p; ++k) y[k] += alpha * w.dy[k];
    double knew = kappa + alpha * dk;
    for (int k = 0; k < m; ++k) {
      double vn = w.v[k] + alpha * w.dv[k];
      z[k] = oqp_retract(vn, knew);
      s[k] = oqp_retract(-vn, knew);
    }
    if (!finite_vec(n, x) || !finite_vec(m, z) || !finite_vec(m, s)) {
      status = OQP_NUMERICAL;
      break;
    }
  }
  *iters_out = it;
  if (res_out) *res_out = res;
  work_free(&w);
  return status;
}

/* ---------------------------------------------------------------------------
 * One direction of Alg. 1 at (x, y, z, s), on its own: v = z - s and
 * kappa = s'z/m as the iteration forms them, eq. 14 factored and solved for
 * r_kappa = kappa - kappa_target, and (dz, ds, dkappa) recovered from eq. 13.
 * The tests hold it to the linearisation of eq. 4 and eq. 11 that it solves.
 * ------------------------------------------------------------------------- */
int oqp_newton_direction(const oqp_problem* P, const double* x, const double* y,
                         const double* z, const double* s, double kappa_target, double* dx,
                         double* dy, double* dv, double* dz, double* ds, double* dkappa) {
  int n = P->n, p = P->p, m = P->m;
  if (n < 1 || p < 0 || m < 1 || p > n) return OQP_BAD_INPUT;
  oqp_work w;
  if (work_alloc(P, &w) != 0) return OQP_NUMERICAL;
  double kappa = 0.0;
  for (int k = 0; k < m; ++k) { w.v[k] = z[k] - s[k]; kappa += s[k] * z[k]; }
  kappa /= (double)m; /* R1 */
  residuals(P, x, y, z, s, &w.R);
  for (int k = 0; k < m; ++k) {
    w.rz[k] = z[k] - oqp_retract(w.v[k], kappa);
    w.rs[k] = s[k] - oqp_retract(-w.v[k], kappa);
  }
  int status = OQP_SOLVED;
  if (newton_factor(P, w.v, kappa, &w.W) != 0)
    status = OQP_NUMERICAL;
  else
    newton_solve(P, &w.W, w.R.rt, w.R.re, w.R.ri, w.rz, w.rs, kappa - kappa_target, dx, dv, dy,
                 dz, ds, dkappa);
  work_free(&w);
  return status;
}

/* ---------------------------------------------------------------------------
 * Alg. 2 (relax_qp): warm start from (x, y, z, s), Newton steps with
 * kappa_target = kappa_relax, refactoring every iteration (exact Newton).
 * Converged when the residual measure of (r_t, r_e, r_i) is below tol and
 * |kappa - kappa_relax| <= tol * kappa_relax.
 * ------------------------------------------------------------------------- */
int oqp_relax(const oqp_problem* P, const oqp_settings* S, double kappa_relax, double* x,
              double* y, double* z, double* s, int* iters_out, double* res_out) {
  int n = P->n, p = P->p, m = P->m;
  *iters_out = 0;
  if (m == 0) return OQP_SOLVED;
  oqp_work w;
  if (work_alloc(P, &w) != 0) return OQP_NUMERICAL;
  int status = OQP_MAX_ITER, it;
  double res = INFINITY;
  for (it = 0; it < S->max_iter; ++it) {
    double kappa = 0.0;
    for (int k = 0; k < m; ++k) { w.v[k] = z[k] - s[k]; kappa += s[k] * z[k]; }
    kappa /= (double)m;
    residuals(P, x, y, z, s, &w.R);
    for (int k = 0; k < m; ++k) {
      w.rz[k] = z[k] - oqp_retract(w.v[k], kappa);
      w.rs[k] = s[k] - oqp_retract(-w.v[k], kappa);
    }
    /* complementarity enters through |kappa - kappa_relax| instead of z.*s */
    double* zero = w.dz;
    for (int k = 0; k < m; ++k) zero[k] = 0.0;
    double r1 = residual_measure(P, &w.R, zero, s, w.rz, w.rs, S->scaled);
    double rk = fabs(kappa - kappa_relax) / kappa_relax;
    res = fmax(r1, rk);
    if (!isfinite(res)) { status = OQP_NUMERICAL; break; }
    if (res < S->tol) { status = OQP_SOLVED; break; }
    if (newton_factor(P, w.v, kappa, &w.W) != 0) { status = OQP_NUMERICAL; break; }
    double dk;
    newton_solve(P, &w.W, w.R.rt, w.R.re, w.R.ri, w.rz, w.rs, kappa - kappa_relax, w.dx, w.dv,
                 w.dy, w.dz, w.ds, &dk);
    double alpha = S->step_frac * step_length(m, s, z, w.ds, w.dz);
    for (int i = 0; i < n; ++i) x[i] += alpha * w.dx[i];
    for (int k = 0; k < p; ++k) y[k] += alpha * w.dy[k];
    double knew = kappa + alpha * dk;
    for (int k = 0; k < m; ++k) {
      double vn = w.v[k] + alpha * w.dv[k];
      z[k] = oqp_retract(vn, knew);
      s[k] = oqp_retract(-vn, knew);
    }
  }
  *iters_out = it;
  if (res_out) *res_out = res;
  work_free(&w);
  return status;
}

/* ---------------------------------------------------------------------------
 * Alg. 3 (compute_qp_gradients) at a relaxed point (x, y, z, s), kappa_relax.
 * Solves eq. 14 (symmetric) at v = z - s with right-hand side (-g, 0, 0) (R3),
 * dz = B_k(v) dv (eq. 13 row 4 with zero residuals), then
 *   dQ = (dx x' + x dx')/2, dq = dx, dA = dy x' + y dx', db = -dy,
 *   dG = dz x' + z dx', dh = -dz.
 * Equality-only problems use [Q A'; A 0] (dx, dy) = (-g, 0).
 * ------------------------------------------------------------------------- */
int oqp_gradients(const oqp_problem* P, double kappa_relax, const double* x, const double* y,
                  const double* z, const double* s, const double* g, double* dQ, double* dq,
                  double* dA, double* db, double* dG, double* dh) {
  int n = P->n, p = P->p, m = P->m, N = n + m + p;
  oqp_work w;
  if (work_alloc(P, &w) != 0) return OQP_NUMERICAL;
  for (int k = 0; k < m; ++k) w.v[k] = z[k] - s[k];
  if (newton_factor(P, w.v, kappa_relax, &w.W) != 0) { work_free(&w); return OQP_NUMERICAL; }
  double* r = w.W.rhs;
  for (int i = 0; i < N; ++i) r[i] = 0.0;
  for (int i = 0; i < n; ++i) r[i] = -g[i];
  lu_solve(N, w.W.M, w.W.piv, r);
  double *dx = w.dx, *dy = w.dy, *dzv = w.dz;
  for (int i = 0; i < n; ++i) dx[i] = r[i];
  for (int k = 0; k < p; ++k) dy[k] = r[n + m + k];
  for (int k = 0; k < m; ++k) dzv[k] = w.W.Bp[k] * r[n + k];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) dQ[IX(i, j, n)] = 0.5 * (dx[i] * x[j] + x[i] * dx[j]);
  for (int i = 0; i < n; ++i) dq[i] = dx[i];
  for (int k = 0; k < p; ++k) {
    for (int j = 0; j < n; ++j) dA[IX(k, j, n)] = dy[k] * x[j] + y[k] * dx[j];
    db[k] = -dy[k];
  }
  for (int k = 0; k < m; ++k) {
    for (int j = 0; j < n; ++j) dG[IX(k, j, n)] = dzv[k] * x[j] + z[k] * dx[j];
    dh[k] = -dzv[k];
  }
  work_free(&w);
  return OQP_SOLVED;
}

/* ---------------------------------------------------------------------------
 * Standard formulation (ablation): explicit complementarity z.*s = kappa,
 * Newton system eq. 8 solved as a full (n+p+m)-square system,
 *   [Q A' G'; A 0 0; G 0 -D(s./z)] (dx, dy, dz) = -(r_t, r_e, r_i - r_c ./ z),
 *   ds = -(r_c + s.*dz) ./ z          (eq. 6 fourth row),
 * Mehrotra predictor-corrector (r_c = z.*s, then z.*s + ds_a.*dz_a - sigma mu),
 * fraction-to-boundary 0.99 on eq. 7.
 * ------------------------------------------------------------------------- */
int oqp_solve_standard(const oqp_problem* P, const oqp_settings* S, double* x, double* y,
                       double* z, double* s, int* iters_out, double* res_out) {
  int n = P->n, p = P->p, m = P->m, N = n + p + m;
  *iters_out = 0;
  if (n < 1 || p < 0 || m < 0 || p > n) return OQP_BAD_INPUT;
  if (m == 0) return solve_eq_only(P, S, x, y, iters_out);
  if (initialize(P, x, y, z, s) != 0) return OQP_NUMERICAL;
  oqp_work w;
  if (work_alloc(P, &w) != 0) return OQP_NUMERICAL;
  double* rc = w.rz;
  double* dsa = w.rs;
  double* dza = w.v;
  int status = OQP_MAX_ITER, it;
  double res = INFINITY;
  double* M = w.W.M;
  double* r = w.W.rhs;
  for (it = 0; it < S->max_iter; ++it) {
    double mu = 0.0;
    for (int k = 0; k < m; ++k) mu += s[k] * z[k];
    mu /= (double)m;
    residuals(P, x, y, z, s, &w.R);
    res = residual_measure(P, &w.R, z, s, NULL, NULL, S->scaled);
    if (!isfinite(res)) { status = OQP_NUMERICAL; break; }
    if (res < S->tol) { status = OQP_SOLVED; break; }
    memset(M, 0, sizeof(double) * (size_t)N * N);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) M[IX(i, j, N)] = P->Q[IX(i, j, n)];
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < n; ++j) {
        M[IX(n + k, j, N)] = P->A[IX(k, j, n)];
        M[IX(j, n + k, N)] = P->A[IX(k, j, n)];
      }
    for (int k = 0; k < m; ++k) {
      for (int j = 0; j < n; ++j) {
        M[IX(n + p + k, j, N)] = P->G[IX(k, j, n)];
        M[IX(j, n + p + k, N)] = P->G[IX(k, j, n)];
      }
      M[IX(n + p + k, n + p + k, N)] = -s[k] / z[k];
    }
    if (lu_factor(N, M, w.W.piv) != 0) { status = OQP_NUMERICAL; break; }
    double sigma_mu = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = 0; k < m; ++k)
        rc[k] = pass == 0 ? z[k] * s[k] : z[k] * s[k] + dsa[k] * dza[k] - sigma_mu;
      for (int i = 0; i < n; ++i) r[i] = -w.R.rt[i];
      for (int k = 0; k < p; ++k) r[n + k] = -w.R.re[k];
      for (int k = 0; k < m; ++k) r[n + p + k] = -(w.R.ri[k] - rc[k] / z[k]);
      lu_solve(N, M, w.W.piv, r);
      double* dzp = pass == 0 ? dza : w.dz;
      double* dsp = pass == 0 ? dsa : w.ds;
      for (int k = 0; k < m; ++k) {
        dzp[k] = r[n + p + k];
        dsp[k] = -(rc[k] + s[k] * dzp[k]) / z[k];
      }
      if (pass == 0) {
        double aa = step_length(m, s, z, dsa, dza);
        double mua = 0.0;
        for (int k = 0; k < m; ++k) mua += (s[k] + aa * dsa[k]) * (z[k] + aa * dza[k]);
        mua /= (double)m;
        double ratio = mua / mu;
        double sigma = S->sigma_mode == 1 ? S->sigma : ratio * ratio * ratio;
        if (!(sigma >= 0.0)) sigma = 0.0;
        if (sigma > 1.0) sigma = 1.0;
        sigma_mu = sigma * mu;
      } else {
        for (int i = 0; i < n; ++i) w.dx[i] = r[i];
        for (int k = 0; k < p; ++k) w.dy[k] = r[n + k];
      }
    }
    double alpha = fmin(1.0, 0.99 * step_length(m, s, z, w.ds, w.dz));
    for (int i = 0; i < n; ++i) x[i] += alpha * w.dx[i];
    for (int k = 0; k < p; ++k) y[k] += alpha * w.dy[k];
    for (int k = 0; k < m; ++k) { z[k] += alpha * w.dz[k]; s[k] += alpha * w.ds[k]; }
    if (!finite_vec(n, x) || !finite_vec(m, z) || !finite_vec(m, s)) {
      status = OQP_NUMERICAL;
      break;
    }
  }
  *iters_out = it;
  if (res_out) *res_out = res;
  work_free(&w);
  return status;
}

/* ---------------------------------------------------------------------------
 * Batched driver: B independent problems of one size, contiguous, run by a
 * pool of POSIX threads (one problem per task).
 *   mode bit 0: solve (implicit; or standard when bit 3 is set)
 *   mode bit 1: relax to kappa_relax after the solve
 *   mode bit 2: gradients at the relaxed point (needs g)
 * x, y, z, s receive the solution; xr, yr, zr, sr (optional) the relaxed point.
 * ------------------------------------------------------------------------- */
typedef struct {
  int B, n, p, m, mode;
  const double *Q, *q, *A, *b, *G, *h, *g;
  oqp_settings S;
  double kappa_relax;
  double *x, *y, *z, *s, *res;
  double *xr, *yr, *zr, *sr; /* relaxed point (optional) */
  double *dQ, *dq, *dA, *db, *dG, *dh;
  int *status, *iters, *relax_iters;
  int next;
} oqp_batch_job;

static void* batch_worker(void* arg) {
  oqp_batch_job* J = (oqp_batch_job*)arg;
  int n = J->n, p = J->p, m = J->m;
  for (;;) {
    int i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (i >= J->B) break;
    oqp_problem P = {n, p, m, J->Q + (size_t)i * n * n, J->q + (size_t)i * n,
                     J->A + (size_t)i * p * n, J->b + (size_t)i * p,
                     J->G + (size_t)i * m * n, J->h + (size_t)i * m};
    double* x = J->x + (size_t)i * n;
    double* y = J->y + (size_t)i * p;
    double* z = J->z + (size_t)i * m;
    double* s = J->s + (size_t)i * m;
    int it = 0, st = OQP_SOLVED, rit = 0;
    double res = 0.0;
    if (J->mode & 8)
      st = oqp_solve_standard(&P, &J->S, x, y, z, s, &it, &res);
    else
      st = oqp_solve(&P, &J->S, x, y, z, s, &it, &res);
    /* the relaxed point lives in xr..sr (a copy of the solution when not relaxing) */
    double* xr = J->xr ? J->xr + (size_t)i * n : x;
    double* yr = J->yr ? J->yr + (size_t)i * p : y;
    double* zr = J->zr ? J->zr + (size_t)i * m : z;
    double* sr = J->sr ? J->sr + (size_t)i * m : s;
    if (xr != x) memcpy(xr, x, sizeof(double) * (size_t)n);
    if (yr != y) memcpy(yr, y, sizeof(double) * (size_t)p);
    if (zr != z) memcpy(zr, z, sizeof(double) * (size_t)m);
    if (sr != s) memcpy(sr, s, sizeof(double) * (size_t)m);
    if ((J->mode & 2) && st == OQP_SOLVED && m > 0) {
      double rres;
      int rst = oqp_relax(&P, &J->S, J->kappa_relax, xr, yr, zr, sr, &rit, &rres);
      if (rst != OQP_SOLVED) st = rst;
    }
    if ((J->mode & 4) && J->g) {
      double kr = (J->mode & 2) ? J->kappa_relax : 0.0;
      if (!(J->mode & 2) && m > 0) {
        for (int k = 0; k < m; ++k) kr += z[k] * s[k];
        kr /= (double)m;
      }
      oqp_gradients(&P, kr, xr, yr, zr, sr, J->g + (size_t)i * n, J->dQ + (size_t)i * n * n,
                    J->dq + (size_t)i * n, J->dA + (size_t)i * p * n, J->db + (size_t)i * p,
                    J->dG + (size_t)i * m * n, J->dh + (size_t)i * m);
    }
    J->status[i] = st;
    J->iters[i] = it;
    if (J->relax_iters) J->relax_iters[i] = rit;
    if (J->res) J->res[i] = res;
  }
  return NULL;
}

int oqp_batch(int B, int n, int p, int m, int mode, const double* Q, const double* q,
              const double* A, const double* b, const double* G, const double* h,
              const double* g, const oqp_settings* S, double kappa_relax, double* x, double* y,
              double* z, double* s, double* res, int* status, int* iters, int* relax_iters,
              double* xr, double* yr, double* zr, double* sr, double* dQ, double* dq,
              double* dA, double* db, double* dG, double* dh, int nthreads) {
  oqp_batch_job J = {B, n, p, m, mode, Q, q, A, b, G, h, g, *S, kappa_relax, x, y, z, s, res,
                     xr, yr, zr, sr, dQ, dq, dA, db, dG, dh, status, iters, relax_iters, 0};
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nthreads == 1) {
    batch_worker(&J);
    return 0;
  }
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, batch_worker, &J) != 0) break;
    ++started;
  }
  if (started == 0) batch_worker(&J);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return 0;
}
