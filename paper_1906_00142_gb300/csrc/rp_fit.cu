// Batched least-squares fitting of rational functions (Sec. 4.2).
//
// One CTA owns one fit.  The linearised problem of Sec. 4.2 -- minimise
// sum_i w_i^2 (p(x_i) - y_i q(x_i))^2 over the coefficients of p and q, with
// the homogeneous system normalised by mean(q) = 1 over the fit's samples --
// is solved through its normal equations, but in a basis chosen per fit so
// that the Gram matrix is well conditioned:
//
//  1. each variable is mapped affinely to [-1, 1] over the fit's samples
//     (box), then standardised (u = (x' - mean) / std);
//  2. per variable, polynomials Q_0 = 1, Q_1 .. Q_d orthonormal for the
//     empirical distribution of u (Cholesky of the Hankel moment matrix);
//  3. Psi_j = Q_a(u_N) Q_b(u_B0) Q_c(u_B1) for the graded-lex exponents
//     (a, b, c) -- a basis of the same polynomial space as the monomials;
//  4. the non-constant Psi_j are centred on the samples and whitened with
//     the inverse Cholesky factor of their Gram matrix (Psi~);
//  5. the design rows w_i [1, Psi~_1.., -y_i Psi~_1..] and right-hand side
//     w_i y_i give the augmented Gram matrix, which is equilibrated and
//     factored in FP64 (columns whose pivot falls below a drop tolerance are
//     removed, recorded as rank deficiency);
//  6. iterative refinement recomputes the residual from the samples
//     (compensated FP32 dot products for the FP32 path, FP64 for the plain
//     path) and corrects the solution with the FP64 factor;
//  7. the solution is mapped back to the monomial basis of the box-normalised
//     variables in FP64.
//
// Since every step is an exact change of basis of the same function space
// and the same normalisation, the fitted p/q is (up to rounding) the
// least-squares solution the paper's SVD formulation defines.
#include <math.h>
#include <stdint.h>

#include "rp_internal.cuh"

namespace rpk {
namespace {

constexpr int kThreads = 256;
constexpr int kSampleCache = 1024;   // samples per fit kept in shared memory

__constant__ int8_t c_exp[kMaxNm][3];        // graded-lex exponents
__constant__ int8_t c_idx[5][5][5];          // exponent triple -> monomial index

struct FitArgs {
  int64_t F, S;
  const float *x, *y;
  const int64_t *off;
  const int8_t *degs;
  int d_uniform;
  int max_refine;
  int weighted;
  double tol;
  double drop_tol;          // relative pivot drop tolerance of the design Gram
  double *coef;
  float *coef32;
  double *box;
  int32_t *status;
  int32_t *rank;
};

// ---------------------------------------------------------------------
// small helpers

__device__ __forceinline__ float two_prod_err(float a, float b, float p) { return fmaf(a, b, -p); }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of n values held by every thread in v[] (n <= 32).  Result
// in out[] (shared), valid after the call for all threads.
template <class T, int NMAX>
__device__ void block_sum(T (&v)[NMAX], int n, T *scratch /* [8][NMAX] */, T *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < n; ++i) {
    T s = warp_sum(v[i]);
    if (lane == 0) scratch[wid * NMAX + i] = s;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    T s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += scratch[w * NMAX + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------
// Per-fit shared state

template <class Real>
struct FitShared {
  // per-variable standardisation and orthonormal marginal polynomials
  float mu_v[3], isg_v[3];
  float Tm[3][kMaxDeg + 1][kMaxDeg + 1];   // Q_k(u) = sum_l Tm[l][k] u^l
  float sc_v[3], of_v[3];                  // x' = x*sc + of
  double lo[3], hi[3];
  float mupsi[kMaxNm];                     // sample means of Psi_j
  float W[kMaxNm][kMaxNm];                 // whitening (upper triangular, rows/cols 1..nm-1)
  double xsol[2 * kMaxNm];                 // current solution (design basis, unscaled)
  double gvec[2 * kMaxNm];                 // normal-equation residual / rhs
  double scl[2 * kMaxNm];                  // equilibration
  double invd[2 * kMaxNm];                 // 1/L_kk (0 = dropped)
  float xhi[2 * kMaxNm], xlo[2 * kMaxNm];  // split solution for compensated residuals
  int keep_cnt;
  int flags;
  int m, d, nm, naug;
  double red_d[8][32];
  float red_f[8][32];
  double dnorm, xnorm;
  int bad;
};

// Per-thread evaluation of the (unwhitened) basis Psi at one sample.
template <class Real>
__device__ __forceinline__ void eval_psi(const FitShared<Real> &sh, int d, int nm, float x0, float x1,
                                         float x2, Real *psi) {
  Real Q[3][kMaxDeg + 1];
  const float xv[3] = {x0, x1, x2};
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const Real xn = (Real)fmaf(xv[v], sh.sc_v[v], sh.of_v[v]);
    const Real u = (xn - (Real)sh.mu_v[v]) * (Real)sh.isg_v[v];
    Real pw[kMaxDeg + 1];
    pw[0] = 1;
#pragma unroll
    for (int l = 1; l <= kMaxDeg; ++l) pw[l] = pw[l - 1] * u;
#pragma unroll
    for (int k = 0; k <= kMaxDeg; ++k) {
      Real s = 0;
#pragma unroll
      for (int l = 0; l <= kMaxDeg; ++l)
        if (l <= k) s += (Real)sh.Tm[v][l][k] * pw[l];
      Q[v][k] = (k <= d) ? s : (Real)0;
    }
  }
  for (int j = 0; j < nm; ++j) psi[j] = Q[0][c_exp[j][0]] * Q[1][c_exp[j][1]] * Q[2][c_exp[j][2]];
}

// Whitened non-constant basis: out[j] for j = 1..nm-1 (out[0] = 1).
template <class Real>
__device__ __forceinline__ void whiten(const FitShared<Real> &sh, int nm, const Real *psi, Real *out) {
  out[0] = 1;
  for (int j = 1; j < nm; ++j) out[j] = 0;
  for (int i = 1; i < nm; ++i) {
    const Real c = psi[i] - (Real)sh.mupsi[i];
    for (int j = i; j < nm; ++j) out[j] += c * (Real)sh.W[i][j];
  }
}

// Accumulate the lower triangle of the Gram matrix of `ncols` columns of the
// rows in shared memory (rows[s*ld + c], s < cnt) into per-thread 4x4 tile
// accumulators (Kahan-compensated across chunks for float).
template <class Real>
struct GramAcc {
  Real s[16];
  Real c[16];
};

__device__ __forceinline__ void tile_of(int t, int &rb, int &cb) {
  // t-th lower-triangle tile in row-major order: rb >= cb
  int r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  rb = r;
  cb = t - r * (r + 1) / 2;
}

template <class Real>
__device__ void gram_chunk(const Real *rows, int ld, int cnt, int ntiles, int sg_count,
                           GramAcc<Real> &acc) {
  const int item = threadIdx.x;
  if (item >= ntiles * sg_count) return;
  const int tile = item % ntiles, sg = item / ntiles;
  int rb, cb;
  tile_of(tile, rb, cb);
  Real part[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) part[i] = 0;
  for (int s = sg; s < cnt; s += sg_count) {
    const Real *row = rows + (size_t)s * ld;
    Real a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = row[4 * rb + i];
      b[i] = row[4 * cb + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[4 * i + j] = fma(a[i], b[j], part[4 * i + j]);
  }
  // Kahan accumulation of the chunk partial
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const Real y = part[i] - acc.c[i];
    const Real t = acc.s[i] + y;
    acc.c[i] = (t - acc.s[i]) - y;
    acc.s[i] = t;
  }
}

// Sum the per-thread tile partials into G (FP64, full symmetric n x n).
template <class Real>
__device__ void gram_finish(const GramAcc<Real> &acc, int ntiles, int sg_count, int n, double *G,
                            double *red /* >= ntiles*sg_count*16 doubles */) {
  const int item = threadIdx.x;
  if (item < ntiles * sg_count)
#pragma unroll
    for (int i = 0; i < 16; ++i) red[(size_t)item * 16 + i] = (double)acc.s[i] - (double)acc.c[i];
  __syncthreads();
  for (int e = threadIdx.x; e < ntiles * 16; e += kThreads) {
    const int tile = e / 16, k = e % 16;
    int rb, cb;
    tile_of(tile, rb, cb);
    const int r = 4 * rb + k / 4, c = 4 * cb + k % 4;
    double s = 0;
    for (int g = 0; g < sg_count; ++g) s += red[((size_t)g * ntiles + tile) * 16 + k];
    if (r < n && c < n) {
      G[r * n + c] = s;
      G[c * n + r] = s;
    }
  }
  __syncthreads();
}

// In-place Cholesky (lower) of the equilibrated n x n matrix G with column
// dropping: a pivot <= tol removes the column (invd = 0).  Returns kept count
// through sh.keep_cnt.
template <class Real>
__device__ void chol_drop(double *G, int n, double tol, FitShared<Real> &sh) {
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double p = G[k * n + k];
      if (p > tol) {
        const double l = sqrt(p);
        G[k * n + k] = l;
        sh.invd[k] = 1.0 / l;
      } else {
        G[k * n + k] = 0.0;
        sh.invd[k] = 0.0;
      }
    }
    __syncthreads();
    const double inv = sh.invd[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += kThreads) G[i * n + k] *= inv;
    __syncthreads();
    const int r = n - k - 1;
    const int np = r * (r + 1) / 2;
    for (int e = threadIdx.x; e < np; e += kThreads) {
      int ii = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      while (ii * (ii + 1) / 2 > e) --ii;
      const int jj = e - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      G[i * n + j] -= G[i * n + k] * G[j * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int k = 0; k < n; ++k) kept += sh.invd[k] != 0.0;
    sh.keep_cnt = kept;
  }
  __syncthreads();
}

// Solve (L L^T) z = b for the factored G (dropped columns give z = 0).
// Executed by warp 0; b and z may alias.
__device__ void chol_solve(const double *L, const double *invd, int n, double *b) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int j = lane; j < i; j += 32) s += L[i * n + j] * b[j];
    s = warp_sum(s);
    if (lane == 0) b[i] = (b[i] - s) * invd[i];
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = 0;
    for (int j = i + 1 + lane; j < n; j += 32) s += L[j * n + i] * b[j];
    s = warp_sum(s);
    if (lane == 0) b[i] = (b[i] - s) * invd[i];
    __syncwarp();
  }
}

// FP64 Cholesky of a small SPD (d+1)x(d+1) Hankel matrix -> inverse factor
// columns (orthonormal polynomial coefficients).  Single thread.
__device__ void marginal_transform(const double *M /* moments M_0..M_2d */, int d, float T[][kMaxDeg + 1]) {
  double H[kMaxDeg + 1][kMaxDeg + 1], R[kMaxDeg + 1][kMaxDeg + 1], Ti[kMaxDeg + 1][kMaxDeg + 1];
  bool ok[kMaxDeg + 1];
  for (int i = 0; i <= d; ++i)
    for (int j = 0; j <= d; ++j) {
      H[i][j] = M[i + j];
      R[i][j] = 0.0;
      Ti[i][j] = 0.0;
    }
  // H = R^T R (R upper), degenerate pivots (below 1e-5 of the diagonal) dropped
  for (int k = 0; k <= d; ++k) {
    double p = H[k][k];
    for (int l = 0; l < k; ++l) p -= R[l][k] * R[l][k];
    ok[k] = p > 1e-5 * H[k][k] && H[k][k] > 0.0;
    if (!ok[k]) continue;
    R[k][k] = sqrt(p);
    for (int j = k + 1; j <= d; ++j) {
      double s = H[k][j];
      for (int l = 0; l < k; ++l) s -= R[l][k] * R[l][j];
      R[k][j] = s / R[k][k];
    }
  }
  // inverse of R restricted to kept indices: column k of Ti solves R Ti = I
  for (int k = 0; k <= d; ++k) {
    if (!ok[k]) continue;
    Ti[k][k] = 1.0 / R[k][k];
    for (int i = k - 1; i >= 0; --i) {
      if (!ok[i]) continue;
      double s = 0;
      for (int l = i + 1; l <= k; ++l) s += R[i][l] * Ti[l][k];
      Ti[i][k] = -s / R[i][i];
    }
  }
  for (int l = 0; l <= kMaxDeg; ++l)
    for (int k = 0; k <= kMaxDeg; ++k) T[l][k] = (l <= d && k <= d) ? (float)Ti[l][k] : 0.0f;
  T[0][0] = 1.0f;  // Q_0 = 1
  for (int k = 1; k <= kMaxDeg; ++k) T[0][k] = (k <= d) ? (float)Ti[0][k] : 0.0f;
}

// ---------------------------------------------------------------------
// The fit kernel.  Real = double: plain FP64 path; Real = float: FP32 path.

template <class Real, int DMAX>
struct Layout {
  static constexpr int NM = (DMAX + 1) * (DMAX + 2) * (DMAX + 3) / 6;
  static constexpr int NAUG = 2 * NM;
  // row stride: multiple of 4 with an odd quotient (fewer bank conflicts)
  static constexpr int LD = (((NAUG + 3) / 4) % 2 == 1) ? ((NAUG + 3) / 4) * 4 : ((NAUG + 3) / 4 + 1) * 4;
  static constexpr int CH = sizeof(Real) == 8 ? 128 : 256;
  static constexpr size_t rows_bytes = sizeof(Real) * (size_t)CH * LD;
  static constexpr size_t red_bytes = sizeof(double) * (size_t)kThreads * 16;
  static constexpr size_t buf_bytes = rows_bytes > red_bytes ? rows_bytes : red_bytes;
  static constexpr size_t G_bytes = sizeof(double) * (size_t)NAUG * NAUG;
  static constexpr size_t samples_bytes = sizeof(float) * 4 * kSampleCache;
  static constexpr size_t rvec_bytes = sizeof(Real) * CH;
  static constexpr size_t total =
      sizeof(FitShared<Real>) + 16 + buf_bytes + G_bytes + samples_bytes + rvec_bytes + 64;
};

template <class Real, int DMAX>
__global__ void __launch_bounds__(kThreads) fit_kernel(FitArgs a) {
  using L = Layout<Real, DMAX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FitShared<Real> &sh = *reinterpret_cast<FitShared<Real> *>(smem_raw);
  unsigned char *p = smem_raw + ((sizeof(FitShared<Real>) + 15) & ~size_t(15));
  Real *rows = reinterpret_cast<Real *>(p);
  double *red = reinterpret_cast<double *>(p);
  p += (L::buf_bytes + 15) & ~size_t(15);
  double *G = reinterpret_cast<double *>(p);
  p += (L::G_bytes + 15) & ~size_t(15);
  float *xs = reinterpret_cast<float *>(p);  // [4][kSampleCache]
  p += L::samples_bytes;
  Real *rvec = reinterpret_cast<Real *>(p);

  const int tid = threadIdx.x;
  for (int64_t f = blockIdx.x; f < a.F; f += gridDim.x) {
    // ---------------- phase 0: range, degree, validation, box
    const int64_t b0 = a.off[f], b1 = a.off[f + 1];
    const int d = a.degs ? (int)a.degs[f] : a.d_uniform;
    const bool range_ok = b0 >= 0 && b1 >= b0 && b1 <= a.S;
    const int m = range_ok ? (int)(b1 - b0) : 0;
    double *cf = a.coef + f * kStride;
    for (int j = tid; j < kStride; j += kThreads) {
      cf[j] = 0.0;
      if (a.coef32) a.coef32[f * kStride + j] = 0.0f;
    }
    if (tid < 6) a.box[f * 6 + tid] = 0.0;
    if (d < 1 || d > DMAX || m == 0) {
      if (tid == 0) {
        a.status[f] = RP_FIT_EMPTY;
        a.rank[f] = 0;
      }
      __syncthreads();
      continue;
    }
    const int nm = num_monomials(d);
    const int naug = 2 * nm;
    const int n = naug - 1;
    const bool cached = m <= kSampleCache;
    const float *gx0 = a.x + b0, *gx1 = a.x + a.S + b0, *gx2 = a.x + 2 * a.S + b0, *gy = a.y + b0;
    float lmin[3] = {INFINITY, INFINITY, INFINITY}, lmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    int lbad = 0;
    for (int i = tid; i < m; i += kThreads) {
      const float v0 = gx0[i], v1 = gx1[i], v2 = gx2[i], yy = gy[i];
      if (cached) {
        xs[i] = v0;
        xs[kSampleCache + i] = v1;
        xs[2 * kSampleCache + i] = v2;
        xs[3 * kSampleCache + i] = yy;
      }
      if (!(isfinite(v0) && isfinite(v1) && isfinite(v2) && isfinite(yy))) lbad |= RP_FIT_NONFINITE;
      else if (a.weighted && !(yy > 0.0f)) lbad |= RP_FIT_NONPOS_Y;
      lmin[0] = fminf(lmin[0], v0); lmax[0] = fmaxf(lmax[0], v0);
      lmin[1] = fminf(lmin[1], v1); lmax[1] = fmaxf(lmax[1], v1);
      lmin[2] = fminf(lmin[2], v2); lmax[2] = fmaxf(lmax[2], v2);
    }
    {
      const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          lmin[v] = fminf(lmin[v], __shfl_xor_sync(0xffffffffu, lmin[v], o));
          lmax[v] = fmaxf(lmax[v], __shfl_xor_sync(0xffffffffu, lmax[v], o));
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lbad |= __shfl_xor_sync(0xffffffffu, lbad, o);
      if (tid == 0) sh.bad = 0;
      __syncthreads();
      if (lane == 0) {
        for (int v = 0; v < 3; ++v) {
          sh.red_f[wid][v] = lmin[v];
          sh.red_f[wid][3 + v] = lmax[v];
        }
        atomicOr(&sh.bad, lbad);
      }
      __syncthreads();
      if (tid < 3) {
        float mn = INFINITY, mx = -INFINITY;
        for (int w = 0; w < kThreads / 32; ++w) {
          mn = fminf(mn, sh.red_f[w][tid]);
          mx = fmaxf(mx, sh.red_f[w][3 + tid]);
        }
        sh.lo[tid] = mn;
        sh.hi[tid] = mx;
        if (mx > mn) {
          // x' = 2 (x - lo) / (hi - lo) - 1 = x * sc + of
          const double sc = 2.0 / ((double)mx - (double)mn);
          sh.sc_v[tid] = (float)sc;
          sh.of_v[tid] = (float)(-1.0 - (double)mn * sc);
        } else {
          sh.sc_v[tid] = 0.0f;
          sh.of_v[tid] = 0.0f;
        }
      }
      __syncthreads();
    }
    if (sh.bad) {
      if (tid == 0) {
        a.status[f] = (sh.bad & RP_FIT_NONFINITE) ? RP_FIT_NONFINITE : RP_FIT_NONPOS_Y;
        a.rank[f] = 0;
      }
      __syncthreads();
      continue;
    }
    if (tid < 3) {
      a.box[f * 6 + 2 * tid] = sh.lo[tid];
      a.box[f * 6 + 2 * tid + 1] = sh.hi[tid];
    }
    const float *sx0 = cached ? xs : gx0;
    const float *sx1 = cached ? xs + kSampleCache : gx1;
    const float *sx2 = cached ? xs + 2 * kSampleCache : gx2;
    const float *sy = cached ? xs + 3 * kSampleCache : gy;

    // ---------------- phase 1: standardisation and marginal orthonormal polys
    {
      float acc[3] = {0, 0, 0};
      for (int i = tid; i < m; i += kThreads) {
        acc[0] += fmaf(sx0[i], sh.sc_v[0], sh.of_v[0]);
        acc[1] += fmaf(sx1[i], sh.sc_v[1], sh.of_v[1]);
        acc[2] += fmaf(sx2[i], sh.sc_v[2], sh.of_v[2]);
      }
      float r3[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) r3[v] = warp_sum(acc[v]);
      const int lane = tid & 31, wid = tid >> 5;
      if (lane == 0)
        for (int v = 0; v < 3; ++v) sh.red_f[wid][v] = r3[v];
      __syncthreads();
      if (tid < 3) {
        float s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh.red_f[w][tid];
        sh.mu_v[tid] = s / (float)m;
      }
      __syncthreads();
      // central moments k = 2 .. 2d (FP32 per thread, FP64 across threads)
      float mom[3][2 * kMaxDeg + 1];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k <= 2 * kMaxDeg; ++k) mom[v][k] = 0.0f;
      for (int i = tid; i < m; i += kThreads) {
        const float xv[3] = {sx0[i], sx1[i], sx2[i]};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const float c = fmaf(xv[v], sh.sc_v[v], sh.of_v[v]) - sh.mu_v[v];
          float pw = c;
#pragma unroll
          for (int k = 1; k <= 2 * kMaxDeg; ++k) {
            mom[v][k] += pw;
            pw *= c;
          }
        }
      }
      // reduce 3 x 8 values in FP64
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 1; k <= 2 * kMaxDeg; ++k) {
          const float s = warp_sum(mom[v][k]);
          if (lane == 0) sh.red_d[wid][v * 8 + (k - 1)] = (double)s;
        }
      __syncthreads();
      if (tid < 3) {
        const int v = tid;
        double M[2 * kMaxDeg + 1];
        for (int k = 1; k <= 2 * kMaxDeg; ++k) {
          double s = 0;
          for (int w = 0; w < kThreads / 32; ++w) s += sh.red_d[w][v * 8 + (k - 1)];
          M[k] = s / (double)m;
        }
        const double var = M[2];
        if (sh.sc_v[v] == 0.0f || !(var > 0.0)) {
          sh.isg_v[v] = 0.0f;
          for (int l = 0; l <= kMaxDeg; ++l)
            for (int k = 0; k <= kMaxDeg; ++k) sh.Tm[v][l][k] = (l == 0 && k == 0) ? 1.0f : 0.0f;
        } else {
          const double isg = 1.0 / sqrt(var);
          sh.isg_v[v] = (float)isg;
          // standardised moments (u = c / sigma); M_0 = 1, M_1 = mean of c / sigma
          double Ms[2 * kMaxDeg + 1];
          Ms[0] = 1.0;
          double pw = isg;
          for (int k = 1; k <= 2 * kMaxDeg; ++k) {
            Ms[k] = M[k] * pw;
            pw *= isg;
          }
          marginal_transform(Ms, d, sh.Tm[v]);
        }
      }
      __syncthreads();
    }

    // ---------------- phase 2: Gram of Psi (nm columns), means, whitening
    const int ld = L::LD;
    {
      const int side = (nm + 3) / 4;
      const int ntiles = side * (side + 1) / 2;
      const int sgc = max(1, kThreads / ntiles);
      GramAcc<Real> acc;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc.s[i] = acc.c[i] = 0;
      for (int base = 0; base < m; base += L::CH) {
        const int cnt = min(L::CH, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[kMaxNm];
          eval_psi<Real>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
          Real *row = rows + (size_t)tid * ld;
          for (int j = 0; j < 4 * side; ++j) row[j] = (j < nm) ? psi[j] : (Real)0;
        }
        __syncthreads();
        gram_chunk<Real>(rows, ld, cnt, ntiles, sgc, acc);
        __syncthreads();
      }
      gram_finish<Real>(acc, ntiles, sgc, nm, G, red);
      // means and centred Gram of the non-constant functions
      if (tid < nm) sh.mupsi[tid] = (float)(G[tid] / (double)m);  // row 0 = sums of Psi_j
      __syncthreads();
      const int nc = nm - 1;
      for (int e = tid; e < nc * nc; e += kThreads) {
        const int i = e / nc + 1, j = e % nc + 1;
        const double gc = (G[i * nm + j] - (double)m * (double)sh.mupsi[i] * (double)sh.mupsi[j]) / (double)m;
        red[e] = gc;
      }
      __syncthreads();
      // equilibrate and factor the centred Gram (nc x nc) in place in `red`
      for (int e = tid; e < nc; e += kThreads) {
        const double dg = red[e * nc + e];
        sh.scl[e] = dg > 0.0 ? 1.0 / sqrt(dg) : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kThreads) red[e] *= sh.scl[e / nc] * sh.scl[e % nc];
      __syncthreads();
      chol_drop<Real>(red, nc, 1e-9, sh);
      // W = D R^{-1}, with R = L^T (upper).  Column j of R^{-1} by back
      // substitution (one thread per column).
      for (int jj = tid; jj < nm; jj += kThreads)
        for (int ii = 0; ii < nm; ++ii) sh.W[ii][jj] = 0.0f;
      __syncthreads();
      if (tid < nc) {
        const int j = tid;
        double col[kMaxNm];
        for (int i = 0; i < nc; ++i) col[i] = 0.0;
        if (sh.invd[j] != 0.0) {
          col[j] = sh.invd[j];
          for (int i = j - 1; i >= 0; --i) {
            if (sh.invd[i] == 0.0) continue;
            double s = 0;
            for (int l = i + 1; l <= j; ++l) s += red[l * nc + i] * col[l];  // R[i][l] = L[l][i]
            col[i] = -s * sh.invd[i];
          }
        }
        for (int i = 0; i <= j; ++i) sh.W[i + 1][j + 1] = (float)(col[i] * sh.scl[i]);
      }
      __syncthreads();
    }

    // ---------------- phase 3: design Gram [num (nm) | den (nm-1) | rhs]
    {
      const int side = (naug + 3) / 4;
      const int ntiles = side * (side + 1) / 2;
      const int sgc = max(1, kThreads / ntiles);
      GramAcc<Real> acc;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc.s[i] = acc.c[i] = 0;
      for (int base = 0; base < m; base += L::CH) {
        const int cnt = min(L::CH, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[kMaxNm], pt[kMaxNm];
          eval_psi<Real>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
          whiten<Real>(sh, nm, psi, pt);
          const Real yy = (Real)sy[i];
          const Real w = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
          Real *row = rows + (size_t)tid * ld;
          for (int j = 0; j < nm; ++j) row[j] = w * pt[j];
          for (int j = 1; j < nm; ++j) row[nm + j - 1] = -w * yy * pt[j];
          row[n] = w * yy;
          for (int j = naug; j < 4 * side; ++j) row[j] = 0;
        }
        __syncthreads();
        gram_chunk<Real>(rows, ld, cnt, ntiles, sgc, acc);
        __syncthreads();
      }
      gram_finish<Real>(acc, ntiles, sgc, naug, G, red);
    }

    // ---------------- phase 4: equilibrate, factor, first solve
    // G is naug x naug; its leading n x n block is the normal matrix and
    // column n holds A^T b.  The scaled n x n block is factored in G's
    // storage with row stride n.
    {
      for (int e = tid; e < n; e += kThreads) {
        const double dg = G[e * naug + e];
        sh.scl[e] = dg > 0.0 ? 1.0 / sqrt(dg) : 0.0;
        sh.gvec[e] = G[e * naug + n];
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += kThreads) {
        const int i = e / n, j = e % n;
        red[e] = G[i * naug + j] * sh.scl[i] * sh.scl[j];
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += kThreads) G[e] = red[e];
      __syncthreads();
      chol_drop<Real>(G, n, a.drop_tol, sh);
      if (tid < n) sh.gvec[tid] *= sh.scl[tid];
      __syncthreads();
      chol_solve(G, sh.invd, n, sh.gvec);
      __syncthreads();
      if (tid < n) sh.xsol[tid] = sh.gvec[tid] * sh.scl[tid];
      if (tid == 0) sh.flags = (sh.keep_cnt < n) ? RP_FIT_RANK_DEFICIENT : 0;
      __syncthreads();
    }

    // ---------------- phase 5: iterative refinement from the samples,
    // then a final pass that checks q > 0 at every sample
    const int sgc = max(1, kThreads / n);
    double prev_rel = INFINITY;
    int refine_state = 0;  // 0 running, 1 converged, 2 stalled
    for (int it = 0; it <= a.max_refine; ++it) {
      const bool final_pass = (it == a.max_refine) || refine_state != 0;
      if (tid < n) {
        const double xv = sh.xsol[tid];
        const float h = (float)xv;
        sh.xhi[tid] = h;
        sh.xlo[tid] = (float)(xv - (double)h);
      }
      if (tid == 0) sh.bad = 0;
      __syncthreads();
      Real gacc = 0, gcmp = 0;
      int pole = 0;
      for (int base = 0; base < m; base += L::CH) {
        const int cnt = min(L::CH, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[kMaxNm], pt[kMaxNm];
          eval_psi<Real>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
          whiten<Real>(sh, nm, psi, pt);
          if (final_pass) {
            // q = 1 + sum_j g_j Psi~_j must stay positive
            double q = 1.0;
            for (int j = 1; j < nm; ++j) q += sh.xsol[nm + j - 1] * (double)pt[j];
            pole |= !(q > 0.0);
          } else {
            const Real yy = (Real)sy[i];
            const Real w = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
            Real *row = rows + (size_t)tid * ld;
            for (int j = 0; j < nm; ++j) row[j] = w * pt[j];
            for (int j = 1; j < nm; ++j) row[nm + j - 1] = -w * yy * pt[j];
            const Real bi = w * yy;
            Real r;
            if constexpr (sizeof(Real) == 8) {
              double sacc = bi;
              for (int j = 0; j < n; ++j) sacc -= row[j] * sh.xsol[j];
              r = sacc;
            } else {
              // compensated dot product (Ogita, Rump & Oishi 2005, "Dot2")
              // of the float row with the split solution xhi + xlo
              float sacc = (float)bi, c = 0.0f;
              for (int j = 0; j < n; ++j) {
                const float av = (float)row[j];
                const float pr = av * sh.xhi[j];
                const float pe = two_prod_err(av, sh.xhi[j], pr);
                float t, e;
                two_sum(sacc, -pr, t, e);
                sacc = t;
                c += e - pe - av * sh.xlo[j];
              }
              r = sacc + c;
            }
            rvec[tid] = r;
          }
        }
        __syncthreads();
        if (!final_pass && tid < n * sgc) {
          const int j = tid % n, g = tid / n;
          Real part = 0;
          for (int s2 = g; s2 < cnt; s2 += sgc) part = fma(rows[(size_t)s2 * ld + j], rvec[s2], part);
          const Real yk = part - gcmp;
          const Real tk = gacc + yk;
          gcmp = (tk - gacc) - yk;
          gacc = tk;
        }
        __syncthreads();
      }
      if (final_pass) {
        if (pole) atomicOr(&sh.bad, 1);
        __syncthreads();
        if (tid == 0) {
          if (sh.bad) sh.flags |= RP_FIT_POLE;
          if (refine_state != 1 && a.max_refine > 0) sh.flags |= RP_FIT_NOT_CONVERGED;
        }
        __syncthreads();
        break;
      }
      if (tid < n * sgc) red[tid] = (double)gacc - (double)gcmp;
      __syncthreads();
      if (tid < n) {
        double sum = 0;
        for (int g = 0; g < sgc; ++g) sum += red[g * n + tid];
        sh.gvec[tid] = sum * sh.scl[tid];
      }
      __syncthreads();
      chol_solve(G, sh.invd, n, sh.gvec);
      __syncthreads();
      if (tid < 32) {
        double dn = 0, xn = 0;
        for (int j = tid; j < n; j += 32) {
          const double dx = sh.gvec[j] * sh.scl[j];
          const double xv = sh.xsol[j] + dx;
          sh.xsol[j] = xv;
          dn += dx * dx;
          xn += xv * xv;
        }
        dn = warp_sum(dn);
        xn = warp_sum(xn);
        if (tid == 0) {
          sh.dnorm = sqrt(dn);
          sh.xnorm = sqrt(xn);
        }
      }
      __syncthreads();
      const double rel = sh.xnorm > 0 ? sh.dnorm / sh.xnorm : 0.0;
      if (rel <= a.tol) refine_state = 1;
      else if (it >= 1 && rel > 0.5 * prev_rel) refine_state = (rel <= 1e-5) ? 1 : 2;
      prev_rel = rel;
    }

    // ---------------- phase 6: back to the monomial basis (FP64)
    // Psi coefficients: numerator c_i, denominator e_i.
    {
      double *cpsi = red;              // [2][kMaxNm]
      double *P = red + 2 * kMaxNm;    // P[v][k][i]: Q_k as a polynomial in x'
      if (tid < 2 * nm) {
        const int which = tid / nm, i = tid % nm;   // 0 numerator, 1 denominator
        if (i >= 1) {
          double u = 0;
          for (int j = i; j < nm; ++j) {
            const double coefj = which == 0 ? sh.xsol[j] : sh.xsol[nm + j - 1];
            u += (double)sh.W[i][j] * coefj;
          }
          cpsi[which * kMaxNm + i] = u;
        }
      }
      if (tid < 3 * (kMaxDeg + 1)) {
        // Q_k(u), u = (x' - mu) * isg, expanded in powers of x'
        const int v = tid / (kMaxDeg + 1), k = tid % (kMaxDeg + 1);
        const double mu = sh.mu_v[v], isg = sh.isg_v[v];
        double out[kMaxDeg + 1] = {0, 0, 0, 0, 0};
        if (k <= d) {
          for (int l = 0; l <= k; ++l) {
            const double t = sh.Tm[v][l][k];
            if (t == 0.0) continue;
            // t * (isg (x' - mu))^l = t isg^l sum_i C(l,i) x'^i (-mu)^(l-i)
            double isgl = 1.0;
            for (int q = 0; q < l; ++q) isgl *= isg;
            double binom = 1.0;
            for (int ii = 0; ii <= l; ++ii) {
              double mpow = 1.0;
              for (int q = 0; q < l - ii; ++q) mpow *= -mu;
              out[ii] += t * isgl * binom * mpow;
              binom = binom * (double)(l - ii) / (double)(ii + 1);
            }
          }
        }
        for (int i2 = 0; i2 <= kMaxDeg; ++i2) P[(v * (kMaxDeg + 1) + k) * (kMaxDeg + 1) + i2] = out[i2];
      }
      __syncthreads();
      if (tid < 2) {
        const int which = tid;
        double c0 = which == 0 ? sh.xsol[0] : 1.0;
        for (int i = 1; i < nm; ++i) c0 -= (double)sh.mupsi[i] * cpsi[which * kMaxNm + i];
        cpsi[which * kMaxNm + 0] = c0;
      }
      __syncthreads();
      // target monomial (one thread each for numerator and denominator)
      if (tid < 2 * nm) {
        const int which = tid / nm, t = tid % nm;
        const int i0 = c_exp[t][0], i1 = c_exp[t][1], i2 = c_exp[t][2];
        double s = 0;
        for (int j = 0; j < nm; ++j) {
          const int e0 = c_exp[j][0], e1 = c_exp[j][1], e2 = c_exp[j][2];
          if (e0 < i0 || e1 < i1 || e2 < i2) continue;
          s += cpsi[which * kMaxNm + j] * P[(0 * (kMaxDeg + 1) + e0) * (kMaxDeg + 1) + i0] *
               P[(1 * (kMaxDeg + 1) + e1) * (kMaxDeg + 1) + i1] *
               P[(2 * (kMaxDeg + 1) + e2) * (kMaxDeg + 1) + i2];
        }
        const int o = which == 0 ? t : kHalf + t;
        cf[o] = s;
        if (a.coef32) a.coef32[f * kStride + o] = (float)s;
      }
      if (tid == 0) {
        a.status[f] = sh.flags;
        a.rank[f] = sh.keep_cnt;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------

void set_tables() {
  static bool done = false;
  if (done) return;
  int8_t e[kMaxNm][3];
  int8_t idx[5][5][5];
  for (int i = 0; i < 125; ++i) (&idx[0][0][0])[i] = -1;
  int k = 0;
  for (int s = 0; s <= kMaxDeg; ++s)
    for (int a = s; a >= 0; --a)
      for (int b = s - a; b >= 0; --b) {
        e[k][0] = (int8_t)a;
        e[k][1] = (int8_t)b;
        e[k][2] = (int8_t)(s - a - b);
        idx[a][b][s - a - b] = (int8_t)k;
        ++k;
      }
  cudaMemcpyToSymbol(c_exp, e, sizeof(e));
  cudaMemcpyToSymbol(c_idx, idx, sizeof(idx));
  done = true;
}

template <class Real, int DMAX>
cudaError_t launch_t(const FitArgs &a, cudaStream_t s) {
  using L = Layout<Real, DMAX>;
  const size_t smem = L::total;
  cudaError_t e = cudaFuncSetAttribute(fit_kernel<Real, DMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fit_kernel<Real, DMAX>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > a.F) grid = a.F;
  fit_kernel<Real, DMAX><<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t fit_workspace_bytes(const rp_fit_desc &) { return 0; }

bool fit_precision_supported(int precision) {
  return precision == RP_PREC_FP64 || precision == RP_PREC_FP32;
}

cudaError_t launch_fit(const rp_fit_desc &desc, const float *x, const float *y,
                       const int64_t *fit_off, double *coef, float *coef32, double *box,
                       int32_t *status, int32_t *rank, void *, cudaStream_t s) {
  if (desc.num_fits == 0) return cudaSuccess;
  set_tables();
  FitArgs a;
  a.F = desc.num_fits;
  a.S = desc.num_samples;
  a.x = x;
  a.y = y;
  a.off = fit_off;
  a.degs = desc.degrees;
  a.d_uniform = desc.degree;
  a.max_refine = desc.max_refine;
  a.weighted = (desc.flags & RP_FIT_UNWEIGHTED) ? 0 : 1;
  a.tol = desc.tol;
  a.coef = coef;
  a.coef32 = coef32;
  a.box = box;
  a.status = status;
  a.rank = rank;
  const int dmax = desc.degree;
  if (desc.precision == RP_PREC_FP64) {
    a.drop_tol = 1e-13;
    switch (dmax) {
      case 1: case 2: return launch_t<double, 2>(a, s);
      case 3: return launch_t<double, 3>(a, s);
      default: return launch_t<double, 4>(a, s);
    }
  }
  a.drop_tol = 1e-7;
  switch (dmax) {
    case 1: case 2: return launch_t<float, 2>(a, s);
    case 3: return launch_t<float, 3>(a, s);
    default: return launch_t<float, 4>(a, s);
  }
}

}  // namespace rpk
