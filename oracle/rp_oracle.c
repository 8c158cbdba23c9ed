/*
 * FP64 CPU oracle for the rational-program fit and MWP-CWP search.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes.  Only tests/, the smoke check
 * and the bench's CPU-baseline leg load it.  It shares no code, header or
 * table with the CUDA library.
 *
 * What it follows:
 *  - Rational model f = p/q with degree bounds (Sec. 4.2, "Rational function
 *    estimation"): p and q are polynomials in the data and program
 *    parameters (N, B0, B1).
 *  - Linearisation: the model is linear in the coefficients, giving
 *    A x = b (Sec. 4.2), a homogeneous system (footnote in Sec. 4.2) that
 *    needs one normalisation.  Reading used here: the mean of q over the
 *    fit's own samples equals 1 (q = 1 + sum_j gamma_j (phi_j - mean_j)).
 *  - Least squares min ||b - A x||_2 solved with the SVD (Sec. 4.2), which
 *    copes with the rank-deficient, ill-conditioned sample matrices the
 *    paper describes; minimum-norm solution with singular values below
 *    rcond * sigma_max dropped.  The SVD is a one-sided Jacobi SVD
 *    (Hestenes 1958; Demmel & Veselic 1992).
 *  - Rows weighted by 1/|y| (relative error); variables mapped affinely per
 *    fit to [-1, 1].
 *  - Hardware occupancy (Sec. 2, Example 1, Eq. for W_active) and the
 *    MWP-CWP execution-time model (Sec. 2, Example 2), whose formulas the
 *    paper cites (Hong & Kim, ISCA 2009) but does not print: restated here.
 *    PARITY UNPINNED BY THE PAPER for the MWP-CWP constants and case
 *    details; pinned only by hand-worked examples and invariants.
 *  - Exhaustive evaluation over all admissible configurations and argmin
 *    (Sec. 3.3, Steps 4-5); ties go to the lowest configuration index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RPO_MAXD 4
#define RPO_MAXNM 35
#define RPO_NCFG 66
#define RPO_NMET 8

/* fit status bits */
#define FS_RANK_DEFICIENT 1
#define FS_NOT_CONVERGED 2
#define FS_POLE 4
#define FS_NONFINITE 8
#define FS_NONPOS_Y 16
#define FS_EMPTY 32

static int g_threads = 1;
void rpo_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int rpo_get_threads(void) { return g_threads; }

int rpo_num_monomials(int d) { return (d + 1) * (d + 2) * (d + 3) / 6; }

/* Graded-lex exponents of total degree <= d: degree ascending, then e_N
 * descending, then e_B0 descending. */
int rpo_exponents(int d, int *e) {
  int k = 0;
  for (int t = 0; t <= d; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) {
        e[3 * k] = a;
        e[3 * k + 1] = b;
        e[3 * k + 2] = t - a - b;
        ++k;
      }
  return k;
}

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* ------------------------------------------------------------------ */
/* One-sided Jacobi SVD: W (m x n, row-major) is overwritten by U*Sigma,
 * V (n x n) receives the right singular vectors.  Returns sweeps used, or
 * -1 if it did not converge. */
static int jacobi_svd(int m, int n, double *W, double *V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  const double eps = 1e-15;
  /* columns whose squared norm is below 1e-30 of the matrix's squared
   * Frobenius norm are numerically zero and take no part in rotations */
  double fro2 = 0;
  for (int i = 0; i < m * n; ++i) fro2 += W[i] * W[i];
  const double tiny = 1e-30 * fro2;
  for (int sweep = 1; sweep <= 80; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, b = 0, g = 0;
        for (int i = 0; i < m; ++i) {
          double wp = W[i * n + p], wq = W[i * n + q];
          a += wp * wp;
          b += wq * wq;
          g += wp * wq;
        }
        if (a <= tiny || b <= tiny) continue;
        if (fabs(g) <= eps * sqrt(a * b)) continue;
        rotated = 1;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < m; ++i) {
          double wp = W[i * n + p], wq = W[i * n + q];
          W[i * n + p] = c * wp - s * wq;
          W[i * n + q] = s * wp + c * wq;
        }
        for (int i = 0; i < n; ++i) {
          double vp = V[i * n + p], vq = V[i * n + q];
          V[i * n + p] = c * vp - s * vq;
          V[i * n + q] = s * vp + c * vq;
        }
      }
    if (!rotated) return sweep;
  }
  return -1;
}

/* Singular values of A (m x n row-major), unsorted order of Jacobi columns,
 * written sorted descending into sv[min(m,n)..n]. */
int rpo_svd_values(int m, int n, const double *A, double *sv) {
  double *W = malloc(sizeof(double) * (size_t)m * n), *V = malloc(sizeof(double) * (size_t)n * n);
  memcpy(W, A, sizeof(double) * (size_t)m * n);
  int sw = jacobi_svd(m, n, W, V);
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < m; ++i) s += W[i * n + j] * W[i * n + j];
    sv[j] = sqrt(s);
  }
  for (int i = 0; i < n; ++i) /* insertion sort, descending */
    for (int j = i; j > 0 && sv[j] > sv[j - 1]; --j) {
      double t = sv[j]; sv[j] = sv[j - 1]; sv[j - 1] = t;
    }
  free(W); free(V);
  return sw;
}

/* Minimum-norm least squares x = V Sigma^+ U^T b with rcond truncation. */
int rpo_lstsq_svd(int m, int n, const double *A, const double *b, double rcond,
                  double *x, int *rank) {
  double *W = malloc(sizeof(double) * (size_t)m * n), *V = malloc(sizeof(double) * (size_t)n * n);
  double *sig = malloc(sizeof(double) * n), *c = malloc(sizeof(double) * n);
  memcpy(W, A, sizeof(double) * (size_t)m * n);
  int sw = jacobi_svd(m, n, W, V);
  double smax = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0, t = 0;
    for (int i = 0; i < m; ++i) {
      s += W[i * n + j] * W[i * n + j];
      t += W[i * n + j] * b[i];
    }
    sig[j] = sqrt(s);
    c[j] = t; /* = sigma_j * (u_j . b) */
    if (sig[j] > smax) smax = sig[j];
  }
  int r = 0;
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    if (sig[j] <= rcond * smax || sig[j] == 0.0) continue;
    ++r;
    double coef = c[j] / (sig[j] * sig[j]);
    for (int i = 0; i < n; ++i) x[i] += V[i * n + j] * coef;
  }
  *rank = r;
  free(W); free(V); free(sig); free(c);
  return sw;
}

/* Householder QR least squares for full column rank (m >= n).  Returns 0,
 * or 1 if a zero column is met. */
int rpo_lstsq_qr(int m, int n, const double *A, const double *b, double *x) {
  double *R = malloc(sizeof(double) * (size_t)m * n), *y = malloc(sizeof(double) * m);
  memcpy(R, A, sizeof(double) * (size_t)m * n);
  memcpy(y, b, sizeof(double) * m);
  int bad = 0;
  for (int k = 0; k < n && k < m; ++k) {
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += R[i * n + k] * R[i * n + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { bad = 1; continue; }
    double alpha = R[k * n + k] > 0 ? -nrm : nrm;
    /* v = a_k - alpha e_k, stored in column k below the diagonal */
    double v0 = R[k * n + k] - alpha;
    double vnorm2 = v0 * v0;
    for (int i = k + 1; i < m; ++i) vnorm2 += R[i * n + k] * R[i * n + k];
    R[k * n + k] = v0;
    for (int j = k + 1; j < n; ++j) {
      double s = 0;
      for (int i = k; i < m; ++i) s += R[i * n + k] * R[i * n + j];
      s = 2.0 * s / vnorm2;
      for (int i = k; i < m; ++i) R[i * n + j] -= s * R[i * n + k];
    }
    double s = 0;
    for (int i = k; i < m; ++i) s += R[i * n + k] * y[i];
    s = 2.0 * s / vnorm2;
    for (int i = k; i < m; ++i) y[i] -= s * R[i * n + k];
    R[k * n + k] = alpha;
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = y[k];
    for (int j = k + 1; j < n; ++j) s -= R[k * n + j] * x[j];
    x[k] = (R[k * n + k] != 0.0) ? s / R[k * n + k] : 0.0;
  }
  free(R); free(y);
  return bad;
}

/* ------------------------------------------------------------------ */
/* Fit.  x is [3][S], y [S] (FP64; FP32 inputs are widened by the caller), fit f owns samples
 * [off[f], off[f+1]).  coef row f: alpha_j at [0, nm), beta_j at
 * [stride/2, stride/2 + nm) in the normalised monomial basis; box row f:
 * (lo_N, hi_N, lo_B0, hi_B0, lo_B1, hi_B1). */
static void fit_one(int64_t f, const int64_t *off, const double *x, const double *y,
                    int64_t S, const int8_t *deg, int weighted, double rcond,
                    int use_qr, int64_t stride, double *coef, double *box,
                    int32_t *rank, int32_t *status) {
  int64_t b0 = off[f], b1 = off[f + 1];
  int m = (int)(b1 - b0);
  int d = deg[f];
  int nm = rpo_num_monomials(d);
  int n = 2 * nm - 1;
  double *cf = coef + f * stride;
  for (int64_t j = 0; j < stride; ++j) cf[j] = 0.0;
  double *bx = box + 6 * f;
  for (int j = 0; j < 6; ++j) bx[j] = 0.0;
  rank[f] = 0;
  status[f] = 0;
  if (m <= 0) { status[f] = FS_EMPTY; return; }
  for (int i = 0; i < m; ++i) {
    for (int v = 0; v < 3; ++v)
      if (!isfinite(x[v * S + b0 + i])) { status[f] = FS_NONFINITE; return; }
    if (!isfinite(y[b0 + i])) { status[f] = FS_NONFINITE; return; }
    if (weighted && !(y[b0 + i] > 0.0)) { status[f] = FS_NONPOS_Y; return; }
  }
  int e[3 * RPO_MAXNM];
  rpo_exponents(d, e);
  /* affine map of each variable to [-1, 1] */
  double lo[3], hi[3];
  for (int v = 0; v < 3; ++v) {
    lo[v] = hi[v] = (double)x[v * S + b0];
    for (int i = 1; i < m; ++i) {
      double t = (double)x[v * S + b0 + i];
      if (t < lo[v]) lo[v] = t;
      if (t > hi[v]) hi[v] = t;
    }
    bx[2 * v] = lo[v];
    bx[2 * v + 1] = hi[v];
  }
  double *phi = malloc(sizeof(double) * (size_t)m * nm);
  for (int i = 0; i < m; ++i) {
    double xn[3];
    for (int v = 0; v < 3; ++v) {
      double t = (double)x[v * S + b0 + i];
      xn[v] = (hi[v] > lo[v]) ? 2.0 * (t - lo[v]) / (hi[v] - lo[v]) - 1.0 : 0.0;
    }
    for (int j = 0; j < nm; ++j)
      phi[i * nm + j] = ipow(xn[0], e[3 * j]) * ipow(xn[1], e[3 * j + 1]) * ipow(xn[2], e[3 * j + 2]);
  }
  double mu[RPO_MAXNM];
  for (int j = 0; j < nm; ++j) {
    double s = 0;
    for (int i = 0; i < m; ++i) s += phi[i * nm + j];
    mu[j] = s / m;
  }
  /* rows w_i [phi_0..phi_{nm-1}, -y_i (phi_1 - mu_1) .. ], rhs w_i y_i */
  double *A = malloc(sizeof(double) * (size_t)m * n), *b = malloc(sizeof(double) * m);
  for (int i = 0; i < m; ++i) {
    double yi = (double)y[b0 + i];
    double w = weighted ? 1.0 / fabs(yi) : 1.0;
    for (int j = 0; j < nm; ++j) A[i * n + j] = w * phi[i * nm + j];
    for (int j = 1; j < nm; ++j) A[i * n + nm + j - 1] = -w * yi * (phi[i * nm + j] - mu[j]);
    b[i] = w * yi;
  }
  double xs[2 * RPO_MAXNM];
  int r = n;
  if (use_qr) {
    if (m < n || rpo_lstsq_qr(m, n, A, b, xs)) status[f] |= FS_RANK_DEFICIENT;
  } else {
    int sw = rpo_lstsq_svd(m, n, A, b, rcond, xs, &r);
    if (sw < 0) status[f] |= FS_NOT_CONVERGED;
    if (r < n) status[f] |= FS_RANK_DEFICIENT;
  }
  rank[f] = r;
  int64_t hb = stride / 2;
  double beta0 = 1.0;
  for (int j = 0; j < nm; ++j) cf[j] = xs[j];
  for (int j = 1; j < nm; ++j) {
    cf[hb + j] = xs[nm + j - 1];
    beta0 -= xs[nm + j - 1] * mu[j];
  }
  cf[hb] = beta0;
  /* pole check: q must stay positive at every sample */
  for (int i = 0; i < m; ++i) {
    double q = 0;
    for (int j = 0; j < nm; ++j) q += cf[hb + j] * phi[i * nm + j];
    if (!(q > 0.0)) { status[f] |= FS_POLE; break; }
  }
  free(phi); free(A); free(b);
}

static int fit_all(int64_t F, const int64_t *off, const double *x, const double *y,
                   int64_t S, const int8_t *deg, int weighted, double rcond, int use_qr,
                   int64_t stride, double *coef, double *box, int32_t *rank,
                   int32_t *status) {
  for (int64_t f = 0; f < F; ++f)
    if (deg[f] < 0 || deg[f] > RPO_MAXD || 2 * rpo_num_monomials(deg[f]) > stride) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
  for (int64_t f = 0; f < F; ++f)
    fit_one(f, off, x, y, S, deg, weighted, rcond, use_qr, stride, coef, box, rank, status);
  return 0;
}

int rpo_fit(int64_t F, const int64_t *off, const double *x, const double *y, int64_t S,
            const int8_t *deg, int weighted, double rcond, int64_t stride, double *coef,
            double *box, int32_t *rank, int32_t *status) {
  return fit_all(F, off, x, y, S, deg, weighted, rcond, 0, stride, coef, box, rank, status);
}

int rpo_fit_qr(int64_t F, const int64_t *off, const double *x, const double *y, int64_t S,
               const int8_t *deg, int weighted, int64_t stride, double *coef, double *box,
               int32_t *rank, int32_t *status) {
  return fit_all(F, off, x, y, S, deg, weighted, 0.0, 1, stride, coef, box, rank, status);
}

/* Evaluate one fitted p/q at raw points pts[P][3]. */
void rpo_predict(int64_t P, const double *pts, int d, const double *cf, int64_t stride,
                 const double *bx, double *out) {
  int e[3 * RPO_MAXNM];
  int nm = rpo_exponents(d, e);
  int64_t hb = stride / 2;
  for (int64_t i = 0; i < P; ++i) {
    double xn[3];
    for (int v = 0; v < 3; ++v) {
      double lo = bx[2 * v], hi = bx[2 * v + 1];
      xn[v] = (hi > lo) ? 2.0 * (pts[3 * i + v] - lo) / (hi - lo) - 1.0 : 0.0;
    }
    double p = 0, q = 0;
    for (int j = 0; j < nm; ++j) {
      double ph = ipow(xn[0], e[3 * j]) * ipow(xn[1], e[3 * j + 1]) * ipow(xn[2], e[3 * j + 2]);
      p += cf[j] * ph;
      q += cf[hb + j] * ph;
    }
    out[i] = p / q;
  }
}

/* ------------------------------------------------------------------ */
/* Relative mean squared error of each fit on its samples, and its gradient
 * with respect to alpha_j and beta_j (j >= 1; beta_0 held fixed):
 *   L = (1/m) sum r_i^2,  r_i = (p_i/q_i - y_i)/y_i
 *   dL/dalpha_j = (2/m) sum r_i phi_ij / (y_i q_i)
 *   dL/dbeta_j  = -(2/m) sum r_i p_i phi_ij / (y_i q_i^2) */
int rpo_relmse(int64_t F, const int64_t *off, const double *x, const double *y, int64_t S,
               const int8_t *deg, const double *coef, int64_t stride, const double *box,
               double *loss, double *grad) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
  for (int64_t f = 0; f < F; ++f) {
    int d = deg[f];
    int e[3 * RPO_MAXNM];
    int nm = rpo_exponents(d, e);
    int64_t hb = stride / 2;
    const double *cf = coef + f * stride;
    const double *bx = box + 6 * f;
    double *g = grad + f * stride;
    for (int64_t j = 0; j < stride; ++j) g[j] = 0.0;
    int64_t b0 = off[f];
    int m = (int)(off[f + 1] - b0);
    double L = 0;
    for (int i = 0; i < m; ++i) {
      double xn[3], ph[RPO_MAXNM];
      for (int v = 0; v < 3; ++v) {
        double lo = bx[2 * v], hi = bx[2 * v + 1];
        xn[v] = (hi > lo) ? 2.0 * ((double)x[v * S + b0 + i] - lo) / (hi - lo) - 1.0 : 0.0;
      }
      double p = 0, q = 0;
      for (int j = 0; j < nm; ++j) {
        ph[j] = ipow(xn[0], e[3 * j]) * ipow(xn[1], e[3 * j + 1]) * ipow(xn[2], e[3 * j + 2]);
        p += cf[j] * ph[j];
        q += cf[hb + j] * ph[j];
      }
      double yi = (double)y[b0 + i];
      double r = (p / q - yi) / yi;
      L += r * r;
      for (int j = 0; j < nm; ++j) {
        g[j] += 2.0 * r * ph[j] / (yi * q);
        if (j >= 1) g[hb + j] -= 2.0 * r * p * ph[j] / (yi * q * q);
      }
    }
    if (m > 0) {
      loss[f] = L / m;
      for (int64_t j = 0; j < stride; ++j) g[j] /= m;
    } else {
      loss[f] = 0.0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Pack ("code generation", Sec. 3.3 Step 3 and Sec. 4.3.1): for each
 * kernel, configuration and metric, fold the thread-block monomials of the
 * fitted p and q into univariate polynomials in t = aN*N + bN (the
 * normalised N).  All arithmetic in FP64, stored as FP32.
 * table layout: [K][66][8][2][d+1]; metric_map[K][8] = fit index or -1. */
static void cfg_dims(int c, int *b0, int *b1) {
  int k = 0;
  for (int a = 0; a <= 10; ++a)
    for (int b = 0; b <= 10 - a; ++b) {
      if (k == c) { *b0 = 1 << a; *b1 = 1 << b; return; }
      ++k;
    }
}

int rpo_pack(int64_t K, int d, const double *coef, int64_t stride, const double *box,
             const int8_t *deg, const int32_t *metric_map, float *aN, float *bN,
             float *table) {
  int64_t hb = stride / 2;
  int D1 = d + 1;
  for (int64_t k = 0; k < K; ++k)
    for (int mt = 0; mt < RPO_NMET; ++mt) {
      int fi = metric_map[k * RPO_NMET + mt];
      if (fi >= 0 && (deg[fi] > d || deg[fi] < 0)) return -1;
    }
  for (int64_t k = 0; k < K; ++k)
    for (int mt = 0; mt < RPO_NMET; ++mt) {
      int fi = metric_map[k * RPO_NMET + mt];
      double a = 0.0, bb = 0.0;
      if (fi >= 0) {
        const double *bx = box + 6 * (int64_t)fi;
        if (bx[1] > bx[0]) {
          a = 2.0 / (bx[1] - bx[0]);
          bb = -1.0 - 2.0 * bx[0] / (bx[1] - bx[0]);
        }
      }
      aN[k * RPO_NMET + mt] = (float)a;
      bN[k * RPO_NMET + mt] = (float)bb;
      for (int c = 0; c < RPO_NCFG; ++c) {
        float *num = table + ((((k * RPO_NCFG + c) * RPO_NMET + mt) * 2 + 0) * D1);
        float *den = num + D1;
        double pn[RPO_MAXD + 1] = {0}, pd[RPO_MAXD + 1] = {0};
        if (fi < 0) {
          pd[0] = 1.0;
        } else {
          int B0 = 1, B1 = 1;
          cfg_dims(c, &B0, &B1);
          const double *bx = box + 6 * (int64_t)fi;
          const double *cf = coef + (int64_t)fi * stride;
          double u = (bx[3] > bx[2]) ? 2.0 * (B0 - bx[2]) / (bx[3] - bx[2]) - 1.0 : 0.0;
          double w = (bx[5] > bx[4]) ? 2.0 * (B1 - bx[4]) / (bx[5] - bx[4]) - 1.0 : 0.0;
          int e[3 * RPO_MAXNM];
          int nm = rpo_exponents(deg[fi], e);
          for (int j = 0; j < nm; ++j) {
            double s = ipow(u, e[3 * j + 1]) * ipow(w, e[3 * j + 2]);
            pn[e[3 * j]] += cf[j] * s;
            pd[e[3 * j]] += cf[hb + j] * s;
          }
        }
        for (int i = 0; i < D1; ++i) {
          num[i] = (float)pn[i];
          den[i] = (float)pd[i];
        }
      }
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* MWP-CWP evaluation.  hw[7] = {warp_size, t_max, b_max, w_max, r_sm,
 * z_sm, issue_cycles}.  Query q[8] = {N, n_SM, f_GHz, Mem_LD, BW_GBs,
 * dd_coal, dd_uncoal, kernel_id (int32 bits)}.
 *
 * Per (query, configuration):
 *  metrics (Sec. 4.1): m0 Comp_insts, m1 Coal_Mem_insts, m2 Uncoal_Mem_insts,
 *  m3 Uncoal_per_mw, m4 Synch_insts, m5 Load_bytes_per_warp, m6 regs/thread,
 *  m7 smem words/block, each the packed univariate rational at t, clamped at
 *  0 (m3 at 1); q <= 0 marks a pole and the configuration invalid.
 *  Occupancy (Example 1, W_active = min(floor(B_active T / 32), W_max)):
 *  R and Z are taken to the nearest integer; B_active = 0 if the block
 *  cannot be resident, else min(B_max, floor(W_max/wpb),
 *  floor(R_SM/(R*wpb*32)) [R>0], floor(Z_SM/Z) [Z>0]); Nw = min(B_active*wpb,
 *  W_max) with wpb = ceil(T/32).
 *  #Blocks = ceil(N/B0)*ceil(N/B1) (2-D grid) or ceil(N/T) (1-D grid);
 *  #Active_SMs = min(n_SM, #Blocks); #Rep = ceil(#Blocks/(B_active *
 *  #Active_SMs)) -- exact integer arithmetic.
 *  Memory model, parallelism and the three cases as in Hong & Kim 2009,
 *  with the overlap terms (MWP - 1) taken as max(MWP - 1, 0);
 *  exec = (cycles + Synch_cost) * #Rep.  No memory instructions: exec =
 *  Comp_cycles * #Rep.
 * margin: smallest relative distance of any discrete decision to its
 * boundary; cond: largest Horner condition number of the 16 polynomials. */
static double horner(const float *c, int D1, double t, double *absum) {
  double v = 0, a = 0, at = fabs(t);
  for (int i = D1 - 1; i >= 0; --i) {
    v = v * t + (double)c[i];
    a = a * at + fabs((double)c[i]);
  }
  *absum = a;
  return v;
}

static double rel_gap(double a, double b) {
  double s = fmax(fabs(a), fabs(b));
  return s > 0 ? fabs(a - b) / s : 1.0;
}

/* B_active for integer registers per thread Ri and shared words per block Zi
 * (0 = the block cannot be resident) */
static int64_t occupancy(double Ri, double Zi, int64_t T, int64_t wpb, double warp, double bmax,
                         double wmax, double rsm, double zsm) {
  if (Ri * (double)T > rsm || Zi > zsm) return 0;
  int64_t bact = (int64_t)bmax;
  int64_t t1 = (int64_t)wmax / wpb;
  if (t1 < bact) bact = t1;
  if (Ri > 0) {
    int64_t t2 = (int64_t)(rsm / (Ri * (double)wpb * warp));
    if (t2 < bact) bact = t2;
  }
  if (Zi > 0) {
    int64_t t3 = (int64_t)floor(zsm / Zi);
    if (t3 < bact) bact = t3;
  }
  return bact > 0 ? bact : 0;
}

#define EV_INVALID -1
#define EV_POLE -2
#define EV_BADQ -3

static void eval_one(int64_t K, int d, const float *aN, const float *bN, const float *table,
                     const int32_t *grid_dims, const double *hw, const float *q, int c,
                     double *exec_out, int *case_out, double *margin_out, double *cond_out,
                     double *diag /* MWP, CWP, Nw, B_active or NULL */) {
  int D1 = d + 1;
  double margin = INFINITY, cond = 1.0;
  *exec_out = INFINITY;
  *case_out = EV_BADQ;
  *margin_out = INFINITY;
  *cond_out = 1.0;
  int32_t kid;
  memcpy(&kid, &q[7], 4);
  double N = q[0], nsm = q[1], fghz = q[2], memld = q[3], bw = q[4], ddc = q[5], ddu = q[6];
  for (int i = 0; i < 7; ++i)
    if (!isfinite(q[i])) return;
  if (kid < 0 || kid >= K || !(N >= 1.0) || !(nsm >= 1.0) || !(fghz > 0) || !(bw > 0) ||
      !(memld >= 0) || !(ddc >= 0) || !(ddu >= 0) || N > 4294967295.0 ||
      nsm > 1048576.0)
    return;
  int B0 = 1, B1 = 1;
  cfg_dims(c, &B0, &B1);
  double mv[RPO_NMET];
  for (int mt = 0; mt < RPO_NMET; ++mt) {
    double t = (double)aN[kid * RPO_NMET + mt] * N + (double)bN[kid * RPO_NMET + mt];
    const float *num = table + ((((int64_t)kid * RPO_NCFG + c) * RPO_NMET + mt) * 2) * D1;
    double ap, aq;
    double P = horner(num, D1, t, &ap);
    double Q = horner(num + D1, D1, t, &aq);
    if (P != 0) cond = fmax(cond, ap / fabs(P));
    if (Q != 0) cond = fmax(cond, aq / fabs(Q));
    if (aq > 0) margin = fmin(margin, fabs(Q) / aq);
    if (!(Q > 0.0)) {
      *case_out = EV_POLE;
      *margin_out = margin;
      *cond_out = cond;
      return;
    }
    mv[mt] = P / Q;
  }
  double comp = fmax(0.0, mv[0]), Cm = fmax(0.0, mv[1]), U = fmax(0.0, mv[2]);
  double upm = fmax(1.0, mv[3]), synch = fmax(0.0, mv[4]), lbw = fmax(0.0, mv[5]);
  double Rf = fmax(0.0, mv[6]), Zf = fmax(0.0, mv[7]);
  double warp = hw[0], tmax = hw[1], bmax = hw[2], wmax = hw[3], rsm = hw[4], zsm = hw[5],
         issue = hw[6];
  int64_t T = (int64_t)B0 * B1;
  *margin_out = margin;
  *cond_out = cond;
  *case_out = EV_INVALID;
  if (diag) diag[3] = 0.0;
  if ((double)T > tmax) return;
  int64_t wpb = (T + (int64_t)warp - 1) / (int64_t)warp;
  double Ri = floor(Rf + 0.5), Zi = floor(Zf + 0.5);
  int64_t bact = occupancy(Ri, Zi, T, wpb, warp, bmax, wmax, rsm, zsm);
  /* the nearest-integer roundings of R and Z are decisions only where the
   * other rounding would change residency */
  if (fabs(Rf - floor(Rf) - 0.5) < 1e-5 * fmax(1.0, Rf)) {
    double alt = (Rf - floor(Rf) >= 0.5) ? Ri - 1.0 : Ri + 1.0;
    if (occupancy(alt, Zi, T, wpb, warp, bmax, wmax, rsm, zsm) != bact)
      margin = fmin(margin, fabs(Rf - floor(Rf) - 0.5) / fmax(1.0, Rf));
  }
  if (fabs(Zf - floor(Zf) - 0.5) < 1e-5 * fmax(1.0, Zf)) {
    double alt = (Zf - floor(Zf) >= 0.5) ? Zi - 1.0 : Zi + 1.0;
    if (occupancy(Ri, alt, T, wpb, warp, bmax, wmax, rsm, zsm) != bact)
      margin = fmin(margin, fabs(Zf - floor(Zf) - 0.5) / fmax(1.0, Zf));
  }
  *margin_out = margin;
  if (diag) diag[3] = (double)bact;
  if (bact <= 0) return;
  int64_t nw_i = bact * wpb;
  if (nw_i > (int64_t)wmax) nw_i = (int64_t)wmax;
  double Nw = (double)nw_i;
  uint64_t Ni = (uint64_t)ceil(N);
  uint64_t blocks;
  if (grid_dims[kid] == 1)
    blocks = (Ni + (uint64_t)T - 1) / (uint64_t)T;
  else
    blocks = ((Ni + B0 - 1) / B0) * ((Ni + B1 - 1) / B1);
  uint64_t nsm_i = (uint64_t)floor(nsm);
  uint64_t asm_ = blocks < nsm_i ? blocks : nsm_i;
  uint64_t den = (uint64_t)bact * asm_;
  uint64_t rep_i = (blocks + den - 1) / den;
  double rep = (double)rep_i;
  double mem_insts = U + Cm;
  double comp_cycles = issue * (comp + mem_insts);
  double exec;
  int cs;
  /* the no-memory-instruction branch is a discrete decision at U + Cm = 0 */
  if (fabs(mv[1]) + fabs(mv[2]) < 1e-6 * (comp + 1.0) && (mv[1] > 0.0 || mv[2] > 0.0 || fmax(mv[1], mv[2]) > -1e-6 * (comp + 1.0)))
    margin = 0.0;
  if (mem_insts == 0.0) {
    exec = comp_cycles * rep;
    cs = 0;
  } else {
    double wu = U / mem_insts, wc = Cm / mem_insts;
    double ml_unc = memld + (upm - 1.0) * ddu;
    double ml_coal = memld;
    double ml = ml_unc * wu + ml_coal * wc;
    double dd = ddu * upm * wu + ddc * wc;
    double mwp_nobw = ml / dd; /* dd == 0 gives +inf */
    double bwpw = fghz * lbw / ml;
    double mwp_bw = bw / (bwpw * (double)asm_);
    double mwp_u = fmin(mwp_nobw, mwp_bw);
    int mwp_cap = (Nw <= mwp_u);
    double MWP = fmin(mwp_u, Nw);
    double mem_cycles = ml_unc * U + ml_coal * Cm;
    double cwp_full = (mem_cycles + comp_cycles) / comp_cycles;
    int cwp_cap = (Nw <= cwp_full);
    double CWP = fmin(cwp_full, Nw);
    double per = comp_cycles / mem_insts;
    /* warps overlapping with the first one: never negative (MWP can fall
     * below 1 when bandwidth-bound; the overlap terms then vanish) */
    double over = MWP > 1.0 ? MWP - 1.0 : 0.0;
    margin = fmin(margin, rel_gap(mwp_u, Nw));
    margin = fmin(margin, rel_gap(cwp_full, Nw));
    double cyc;
    if (mwp_cap && cwp_cap) {
      cyc = mem_cycles + comp_cycles + per * over;
      cs = 1;
    } else {
      margin = fmin(margin, fmax(rel_gap(CWP, MWP), rel_gap(comp_cycles, mem_cycles)));
      if (CWP >= MWP || comp_cycles > mem_cycles) {
        cyc = mem_cycles * Nw / MWP + per * over;
        cs = 2;
      } else {
        cyc = memld + comp_cycles * Nw;
        cs = 3;
      }
    }
    double synch_cost = dd * over * synch * (double)bact;
    exec = (cyc + synch_cost) * rep;
    /* (MWP - 1) loses digits when MWP is close to 1: the relative error of
     * MWP is amplified by MWP / (MWP - 1) in the overlap terms */
    if (over > 0.0) {
      double over_terms = (cs == 3 ? 0.0 : per * over) + synch_cost;
      cond = fmax(cond, (MWP / over) * (over_terms / (cyc + synch_cost)));
      *cond_out = cond;
    }
    if (diag) {
      diag[0] = MWP;
      diag[1] = CWP;
    }
  }
  if (diag) diag[2] = Nw;
  *exec_out = exec;
  *case_out = cs;
  *margin_out = margin;
}

int rpo_eval(int64_t K, int d, const float *aN, const float *bN, const float *table,
             const int32_t *grid_dims, const double *hw, int64_t Q, const float *queries,
             double *exec, int32_t *cas, double *margin, double *cond, double *diag) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int64_t i = 0; i < Q; ++i)
    for (int c = 0; c < RPO_NCFG; ++c) {
      int cs;
      double *dg = diag + 4 * (i * RPO_NCFG + c);
      dg[0] = dg[1] = dg[2] = dg[3] = NAN;
      eval_one(K, d, aN, bN, table, grid_dims, hw, queries + 8 * i, c, &exec[i * RPO_NCFG + c],
               &cs, &margin[i * RPO_NCFG + c], &cond[i * RPO_NCFG + c], dg);
      cas[i * RPO_NCFG + c] = cs;
    }
  return 0;
}

/* query status bits */
#define QS_NO_VALID 1
#define QS_POLE 2
#define QS_BAD 4

int rpo_search(int64_t K, int d, const float *aN, const float *bN, const float *table,
               const int32_t *grid_dims, const double *hw, int64_t Q, const float *queries,
               int32_t *argmin, double *best, double *second, int32_t *status) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (int64_t i = 0; i < Q; ++i) {
    double b1 = INFINITY, b2 = INFINITY;
    int arg = -1, st = 0;
    for (int c = 0; c < RPO_NCFG; ++c) {
      double ex, mg, cd;
      int cs;
      eval_one(K, d, aN, bN, table, grid_dims, hw, queries + 8 * i, c, &ex, &cs, &mg, &cd, NULL);
      if (cs == EV_BADQ) { st |= QS_BAD; break; }
      if (cs == EV_POLE) st |= QS_POLE;
      if (cs < 0) continue;
      if (ex < b1) { b2 = b1; b1 = ex; arg = c; }
      else if (ex < b2) b2 = ex;
    }
    if (arg < 0 && !(st & QS_BAD)) st |= QS_NO_VALID;
    argmin[i] = arg;
    best[i] = b1;
    second[i] = b2;
    status[i] = st;
  }
  return 0;
}
