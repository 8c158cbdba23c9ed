// Batched least-squares fitting of rational functions (Sec. 4.2).
//
// One CTA owns one fit at a time (persistent over fits).  The linearised
// problem of Sec. 4.2 -- minimise sum_i w_i^2 (p(x_i) - y_i q(x_i))^2 over the
// coefficients of p and q, the homogeneous system normalised by mean(q) = 1
// over the fit's samples -- is solved through its normal equations in a basis
// chosen per fit so that the Gram matrix is well conditioned:
//
//  1. each variable is mapped affinely to [-1, 1] over the fit's samples
//     (the box), then standardised, u = (x' - mean) / std;
//  2. per variable, polynomials Q_0 = 1, Q_1 .. Q_d orthonormal for the
//     empirical distribution of u (Cholesky of the Hankel moment matrix);
//  3. Psi_j = Q_a(u_N) Q_b(u_B0) Q_c(u_B1) over the graded-lex exponents
//     (a, b, c): a basis of the same polynomial space as the monomials;
//  4. the non-constant Psi_j are centred on the samples and whitened with the
//     inverse Cholesky factor of their Gram matrix (Psi~), cached in shared
//     memory when the fit is small enough;
//  5. the design rows w_i [1, Psi~.., -y_i Psi~..] with right-hand side
//     w_i y_i give the augmented Gram matrix, which is equilibrated and
//     factored with column dropping (pivot below a drop tolerance: column
//     removed, reported as rank deficiency);
//  6. iterative refinement recomputes the residual from the samples
//     (compensated FP32 dot products against the FP64 solution -- Ogita,
//     Rump & Oishi's Dot2 -- on the FP32 path, plain FP64 on the FP64 path),
//     stopping at ||dx|| <= tol ||x|| or when the corrections stop shrinking;
//  7. the solution is mapped back to the monomial basis of the box-normalised
//     variables in FP64 and the fitted q is checked to be positive at every
//     sample.
//
// Each step is a change of basis of the same function space under the same
// normalisation, so the fitted p/q is the least-squares solution the paper's
// SVD formulation defines (up to rounding).  The FP32 path factors in FP32
// (GB300's FP64 rate is ~1/58 of FP32): the factor only preconditions the
// refinement, whose residuals carry the accuracy.
#include <math.h>
#include <stdint.h>

#include "rp_internal.cuh"

namespace rpk {
namespace {

constexpr int kThreads = 256;
constexpr int kSampleCache = 1024;    // samples kept in shared memory
constexpr int kCacheFloats = 12288;   // whitened-basis cache (FP32 path): 48 KB
constexpr int kCh = 128;              // samples per row chunk
constexpr int kChP = kCh + 1;         // padded chunk stride (bank-conflict free)

__constant__ int8_t c_exp[kMaxNm][3];   // graded-lex exponents

struct FitArgs {
  int64_t F, S;
  const float *x, *y;
  const int64_t *off;
  const int8_t *degs;
  int d_uniform;
  int max_refine;
  int weighted;
  double tol;
  double drop_tol;   // relative pivot drop tolerance of the equilibrated design Gram
  double *coef;
  float *coef32;
  double *box;
  int32_t *status;
  int32_t *rank;
};

// ---------------------------------------------------------------------
// helpers

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

template <class T>
__device__ __forceinline__ T rsqrt_pos(T v);
template <>
__device__ __forceinline__ float rsqrt_pos<float>(float v) { return 1.0f / sqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_pos<double>(double v) { return 1.0 / sqrt(v); }

// Warp-synchronous Cholesky (lower) of the n x n matrix G (row stride ld) in
// place, with column dropping: a pivot <= tol removes the column (invd = 0).
// Called by one full warp.
template <class SR>
__device__ void warp_chol(SR *G, int n, int ld, SR tol, SR *invd, int *keep_cnt) {
  const int lane = threadIdx.x & 31;
  int kept = 0;
  for (int k = 0; k < n; ++k) {
    __syncwarp();
    const SR p = G[k * ld + k];
    const bool keep = p > tol;
    const SR inv = keep ? rsqrt_pos<SR>(p) : (SR)0;
    kept += keep;
    __syncwarp();
    if (lane == 0) {
      G[k * ld + k] = keep ? p * inv : (SR)0;
      invd[k] = inv;
    }
    for (int i = k + 1 + lane; i < n; i += 32) G[i * ld + k] *= inv;
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) {
      const SR lik = G[i * ld + k];
      for (int j = k + 1; j <= i; ++j) G[i * ld + j] -= lik * G[j * ld + k];
    }
  }
  __syncwarp();
  if (lane == 0) *keep_cnt = kept;
  __syncwarp();
}

// Solve (L L^T) z = b in place (one warp; dropped columns give z = 0).
template <class SR>
__device__ void warp_solve(const SR *L, int n, int ld, const SR *invd, SR *b) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < n; ++k) {
    __syncwarp();
    const SR yk = b[k] * invd[k];
    __syncwarp();
    if (lane == 0) b[k] = yk;
    for (int i = k + 1 + lane; i < n; i += 32) b[i] -= L[i * ld + k] * yk;
  }
  for (int k = n - 1; k >= 0; --k) {
    __syncwarp();
    const SR xk = b[k] * invd[k];
    __syncwarp();
    if (lane == 0) b[k] = xk;
    for (int i = lane; i < k; i += 32) b[i] -= L[k * ld + i] * xk;
  }
  __syncwarp();
}

// FP64 Cholesky of the (d+1) x (d+1) Hankel moment matrix of a standardised
// variable -> coefficients of the orthonormal polynomials (columns of the
// inverse factor).  A variable with only q distinct sample values supports
// polynomials of degree < q on the samples: Q_k for k > deg_eff (= q - 1) is
// set to 0, as is any Q_k whose pivot is not positive.  Single thread.
__device__ void marginal_transform(const double *M, int d, int deg_eff, float T[][kMaxDeg + 1]) {
  double R[kMaxDeg + 1][kMaxDeg + 1], Ti[kMaxDeg + 1][kMaxDeg + 1];
  bool ok[kMaxDeg + 1];
  for (int i = 0; i <= kMaxDeg; ++i)
    for (int j = 0; j <= kMaxDeg; ++j) R[i][j] = Ti[i][j] = 0.0;
  for (int k = 0; k <= d; ++k) {
    double p = M[2 * k];
    for (int l = 0; l < k; ++l) p -= R[l][k] * R[l][k];
    ok[k] = k <= deg_eff && M[2 * k] > 0.0 && p > 1e-12 * M[2 * k];
    if (!ok[k]) continue;
    R[k][k] = sqrt(p);
    for (int j = k + 1; j <= d; ++j) {
      double s = M[k + j];
      for (int l = 0; l < k; ++l) s -= R[l][k] * R[l][j];
      R[k][j] = s / R[k][k];
    }
  }
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
  T[0][0] = 1.0f;  // Q_0 = 1 (M_0 = 1)
}

// Insert a value into a small lock-free set of at most kMaxDeg + 1 distinct
// values (slots claimed in order with compare-and-swap; once full, further
// values are ignored -- kMaxDeg + 1 distinct values are all a degree-kMaxDeg
// marginal basis needs).
constexpr unsigned kEmpty = 0xFFFFFFFFu;
__device__ __forceinline__ void distinct_insert(unsigned *slots, float x) {
  const unsigned v = (x == 0.0f) ? 0u : __float_as_uint(x);
#pragma unroll
  for (int k = 0; k < kMaxDeg + 1; ++k) {
    const unsigned cur = *((volatile unsigned *)&slots[k]);
    if (cur == v) return;
    if (cur == kEmpty) {
      const unsigned old = atomicCAS(&slots[k], kEmpty, v);
      if (old == kEmpty || old == v) return;
    }
  }
}

// ---------------------------------------------------------------------
// Per-fit shared state

template <class Real>
struct FitShared {
  float mu_v[3], isg_v[3], sc_v[3], of_v[3];
  float Tm[3][kMaxDeg + 1][kMaxDeg + 1];   // Q_k(u) = sum_l Tm[l][k] u^l
  double lo[3], hi[3];
  Real mupsi[kMaxNm];                      // sample means of Psi_j
  Real W[kMaxNm][kMaxNm];                  // whitening, upper triangular on 1..nm-1
  double xsol[2 * kMaxNm];                 // solution, design basis, unscaled
  Real gvec[2 * kMaxNm];                   // right-hand side / correction
  Real scl[2 * kMaxNm];                    // equilibration
  Real invd[2 * kMaxNm];                   // 1/L_kk (0 = dropped)
  Real invw[2 * kMaxNm];                   // same for the whitening factor
  float xhi[2 * kMaxNm], xlo[2 * kMaxNm];  // split solution for compensated residuals
  float red_f[8][32];
  double red_d[8][32];
  unsigned dslot[3][kMaxDeg + 1];          // distinct raw values per variable (saturating)
  int keep_cnt, keep_w, flags, bad;
  float dnorm, xnorm;
};

template <class Real, int DMAX>
struct Layout {
  static constexpr int NM = (DMAX + 1) * (DMAX + 2) * (DMAX + 3) / 6;
  static constexpr int NAUG = 2 * NM;
  static constexpr int ROWS = ((NAUG + 3) / 4) * 4;             // padded feature count
  static constexpr size_t rows_bytes = sizeof(Real) * (size_t)ROWS * kChP;
  static constexpr size_t red_bytes = sizeof(Real) * (size_t)kThreads * 16;
  static constexpr size_t buf_bytes = rows_bytes > red_bytes ? rows_bytes : red_bytes;
  static constexpr size_t G_bytes = sizeof(Real) * (size_t)NAUG * NAUG;
  static constexpr size_t samples_bytes = sizeof(float) * 4 * kSampleCache;
  static constexpr size_t cache_bytes = sizeof(Real) == 4 ? sizeof(float) * kCacheFloats : 0;
  static constexpr size_t rvec_bytes = 2 * sizeof(Real) * kCh;
  static constexpr size_t total = ((sizeof(FitShared<Real>) + 15) & ~size_t(15)) + buf_bytes +
                                  G_bytes + samples_bytes + cache_bytes + rvec_bytes + 64;
};

// Unwhitened basis Psi at one sample (compile-time bound NM, runtime nm).
template <class Real, int NM>
__device__ __forceinline__ void eval_psi(const FitShared<Real> &sh, int d, int nm, float x0, float x1,
                                         float x2, Real (&psi)[NM]) {
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
      for (int l = 0; l <= k; ++l) s += (Real)sh.Tm[v][l][k] * pw[l];
      Q[v][k] = (k <= d) ? s : (Real)0;
    }
  }
#pragma unroll
  for (int j = 0; j < NM; ++j)
    psi[j] = (j < nm) ? Q[0][c_exp[j][0]] * Q[1][c_exp[j][1]] * Q[2][c_exp[j][2]] : (Real)0;
}

// Whitened basis: pt[0] = 1, pt[j] = sum_{1<=i<=j} (Psi_i - mean_i) W[i][j].
template <class Real, int NM>
__device__ __forceinline__ void whiten(const FitShared<Real> &sh, const Real (&psi)[NM],
                                       Real (&pt)[NM]) {
  pt[0] = 1;
#pragma unroll
  for (int j = 1; j < NM; ++j) pt[j] = 0;
#pragma unroll
  for (int i = 1; i < NM; ++i) {
    const Real c = psi[i] - sh.mupsi[i];
#pragma unroll
    for (int j = i; j < NM; ++j) pt[j] = fma(c, sh.W[i][j], pt[j]);
  }
}

// Accumulate lower-triangle 4x4 tiles of the Gram of `rows` (feature-major,
// stride kChP) over `cnt` samples into per-thread accumulators.
template <class Real>
struct GramAcc {
  Real s[16], c[16];
};

__device__ __forceinline__ void tile_of(int t, int &rb, int &cb) {
  int r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  rb = r;
  cb = t - r * (r + 1) / 2;
}

template <class Real>
__device__ void gram_chunk(const Real *rows, int cnt, int ntiles, int sgc, GramAcc<Real> &acc) {
  const int item = threadIdx.x;
  if (item >= ntiles * sgc) return;
  const int tile = item % ntiles, sg = item / ntiles;
  int rb, cb;
  tile_of(tile, rb, cb);
  Real part[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) part[i] = 0;
  for (int s = sg; s < cnt; s += sgc) {
    Real a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = rows[(4 * rb + i) * kChP + s];
      b[i] = rows[(4 * cb + i) * kChP + s];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[4 * i + j] = fma(a[i], b[j], part[4 * i + j]);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {  // Kahan accumulation of chunk partials
    const Real y = part[i] - acc.c[i];
    const Real t = acc.s[i] + y;
    acc.c[i] = (t - acc.s[i]) - y;
    acc.s[i] = t;
  }
}

// Combine per-thread tiles into the full symmetric n x n Gram G (stride n).
template <class Real>
__device__ void gram_finish(const GramAcc<Real> &acc, int ntiles, int sgc, int n, Real *G,
                            Real *red) {
  const int item = threadIdx.x;
  if (item < ntiles * sgc)
#pragma unroll
    for (int i = 0; i < 16; ++i) red[(size_t)item * 16 + i] = acc.s[i] - acc.c[i];
  __syncthreads();
  for (int e = threadIdx.x; e < ntiles * 16; e += kThreads) {
    const int tile = e / 16, k = e % 16;
    int rb, cb;
    tile_of(tile, rb, cb);
    const int r = 4 * rb + k / 4, c = 4 * cb + k % 4;
    Real s = 0;
    for (int g = 0; g < sgc; ++g) s += red[((size_t)g * ntiles + tile) * 16 + k];
    if (r < n && c < n) {
      G[r * n + c] = s;
      G[c * n + r] = s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------
// The fit kernel.  Real = double: plain FP64 path; Real = float: FP32 path.

template <class Real, int DMAX>
__global__ void __launch_bounds__(kThreads) fit_kernel(FitArgs a) {
  using L = Layout<Real, DMAX>;
  constexpr int NM = L::NM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FitShared<Real> &sh = *reinterpret_cast<FitShared<Real> *>(smem_raw);
  unsigned char *p = smem_raw + ((sizeof(FitShared<Real>) + 15) & ~size_t(15));
  Real *rows = reinterpret_cast<Real *>(p);   // [ROWS][kChP], also reduction scratch
  Real *red = rows;
  p += L::buf_bytes;
  Real *G = reinterpret_cast<Real *>(p);
  p += L::G_bytes;
  float *xs = reinterpret_cast<float *>(p);   // [4][kSampleCache]
  p += L::samples_bytes;
  Real *bcache = reinterpret_cast<Real *>(p); // [(nm-1)][mc]
  p += L::cache_bytes;
  Real *rvec = reinterpret_cast<Real *>(p);   // [2][kCh]

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
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
    const int nc = nm - 1;
    const int naug = 2 * nm;
    const int n = naug - 1;
    const bool cached = m <= kSampleCache;
    const int mc = (sizeof(Real) == 4 && m * nc <= kCacheFloats) ? m : 0;  // basis cache
    const float *gx0 = a.x + b0, *gx1 = a.x + a.S + b0, *gx2 = a.x + 2 * a.S + b0, *gy = a.y + b0;
    float lmin[3] = {INFINITY, INFINITY, INFINITY}, lmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    int lbad = 0;
    if (tid == 0) sh.bad = 0;
    if (tid < 3 * (kMaxDeg + 1)) (&sh.dslot[0][0])[tid] = kEmpty;
    __syncthreads();
    for (int i = tid; i < m; i += kThreads) {
      const float v0 = gx0[i], v1 = gx1[i], v2 = gx2[i], yy = gy[i];
      distinct_insert(sh.dslot[0], v0);
      distinct_insert(sh.dslot[1], v1);
      distinct_insert(sh.dslot[2], v2);
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
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lmin[v] = fminf(lmin[v], __shfl_xor_sync(0xffffffffu, lmin[v], o));
        lmax[v] = fmaxf(lmax[v], __shfl_xor_sync(0xffffffffu, lmax[v], o));
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lbad |= __shfl_xor_sync(0xffffffffu, lbad, o);
    __syncthreads();
    if (lane == 0) {
      for (int v = 0; v < 3; ++v) {
        sh.red_f[wid][v] = lmin[v];
        sh.red_f[wid][3 + v] = lmax[v];
      }
      if (lbad) atomicOr(&sh.bad, lbad);
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
      if (mx > mn) {   // x' = 2 (x - lo) / (hi - lo) - 1 = x * sc + of
        const double sc = 2.0 / ((double)mx - (double)mn);
        sh.sc_v[tid] = (float)sc;
        sh.of_v[tid] = (float)(-1.0 - (double)mn * sc);
      } else {
        sh.sc_v[tid] = 0.0f;
        sh.of_v[tid] = 0.0f;
      }
    }
    __syncthreads();
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

    // ---------------- phase 1: standardisation, marginal orthonormal polynomials
    {
      float acc[3] = {0, 0, 0};
      for (int i = tid; i < m; i += kThreads) {
        acc[0] += fmaf(sx0[i], sh.sc_v[0], sh.of_v[0]);
        acc[1] += fmaf(sx1[i], sh.sc_v[1], sh.of_v[1]);
        acc[2] += fmaf(sx2[i], sh.sc_v[2], sh.of_v[2]);
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) acc[v] = warp_sum(acc[v]);
      if (lane == 0)
        for (int v = 0; v < 3; ++v) sh.red_f[wid][v] = acc[v];
      __syncthreads();
      if (tid < 3) {
        float s = 0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh.red_f[w][tid];
        sh.mu_v[tid] = s / (float)m;
      }
      __syncthreads();
      float mom[3][2 * kMaxDeg];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < 2 * kMaxDeg; ++k) mom[v][k] = 0.0f;
      for (int i = tid; i < m; i += kThreads) {
        const float xv[3] = {sx0[i], sx1[i], sx2[i]};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const float c = fmaf(xv[v], sh.sc_v[v], sh.of_v[v]) - sh.mu_v[v];
          float pw = c;
#pragma unroll
          for (int k = 0; k < 2 * kMaxDeg; ++k) {
            mom[v][k] += pw;
            pw *= c;
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < 2 * kMaxDeg; ++k) {
          const float s = warp_sum(mom[v][k]);
          if (lane == 0) sh.red_d[wid][v * 8 + k] = (double)s;
        }
      __syncthreads();
      if (tid < 3) {
        const int v = tid;
        double M[2 * kMaxDeg + 1];
        M[0] = 1.0;
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
          double Ms[2 * kMaxDeg + 1];
          Ms[0] = 1.0;
          double pw = isg;
          for (int k = 1; k <= 2 * kMaxDeg; ++k) {
            Ms[k] = M[k] * pw;
            pw *= isg;
          }
          int cnt = 0;
          for (int k = 0; k <= kMaxDeg; ++k) cnt += sh.dslot[v][k] != kEmpty;
          marginal_transform(Ms, d, min(d, cnt - 1), sh.Tm[v]);
        }
      }
      __syncthreads();
    }

    // ---------------- phase 2: Gram of Psi (nm columns), means, whitening
    {
      const int side = (nm + 3) / 4;
      const int ntiles = side * (side + 1) / 2;
      const int sgc = max(1, kThreads / ntiles);
      GramAcc<Real> acc;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc.s[i] = acc.c[i] = 0;
      for (int base = 0; base < m; base += kCh) {
        const int cnt = min(kCh, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[NM];
          eval_psi<Real, NM>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < 4 * side) rows[j * kChP + tid] = psi[j];
          for (int j = NM; j < 4 * side; ++j) rows[j * kChP + tid] = 0;
        }
        __syncthreads();
        gram_chunk<Real>(rows, cnt, ntiles, sgc, acc);
        __syncthreads();
      }
      gram_finish<Real>(acc, ntiles, sgc, nm, G, red);
      // means (row 0 holds the sums of Psi_j) and the centred Gram / m of the
      // non-constant functions, equilibrated and factored by warp 0
      if (tid < NM) sh.mupsi[tid] = (tid < nm) ? G[tid] / (Real)m : (Real)0;
      for (int e = tid; e < NM * NM; e += kThreads) (&sh.W[0][0])[e] = 0;
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kThreads) {
        const int i = e / nc + 1, j = e % nc + 1;
        red[e] = (G[i * nm + j] - (Real)m * sh.mupsi[i] * sh.mupsi[j]) / (Real)m;
      }
      __syncthreads();
      if (tid < nc) {
        const Real dg = red[tid * nc + tid];
        sh.scl[tid] = dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0;
      }
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kThreads) red[e] *= sh.scl[e / nc] * sh.scl[e % nc];
      __syncthreads();
      // the whitening only preconditions: any positive pivot is kept (the
      // basis stays a basis of the same space); only exactly dependent
      // directions (pivot at rounding level or below) are dropped
      if (wid == 0)
        warp_chol<Real>(red, nc, nc, sizeof(Real) == 8 ? (Real)1e-14 : (Real)1e-10, sh.invw,
                        &sh.keep_w);
      __syncthreads();
      // R^{-1} (R = L^T, R[i][l] = L[l][i]), column j by back substitution,
      // one thread per column, into G (free now); then W = D R^{-1}
      if (tid < nc) {
        const int j = tid;
        for (int i = j; i >= 0; --i) {
          Real s = (i == j) ? (Real)1 : (Real)0;
          for (int l = i + 1; l <= j; ++l) s -= red[l * nc + i] * G[l * nc + j];
          G[i * nc + j] = s * sh.invw[i];
        }
      }
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kThreads) {
        const int i = e / nc, j = e % nc;
        if (i <= j) sh.W[i + 1][j + 1] = G[i * nc + j] * sh.scl[i];
      }
      __syncthreads();
    }

    // ---------------- phase 3: whitened basis (cached) and the design Gram
    // columns: [num (nm) | den (nm-1) | rhs]
    {
      const int side = (naug + 3) / 4;
      const int ntiles = side * (side + 1) / 2;
      const int sgc = max(1, kThreads / ntiles);
      GramAcc<Real> acc;
#pragma unroll
      for (int i = 0; i < 16; ++i) acc.s[i] = acc.c[i] = 0;
      for (int base = 0; base < m; base += kCh) {
        const int cnt = min(kCh, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[NM], pt[NM];
          eval_psi<Real, NM>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
          whiten<Real, NM>(sh, psi, pt);
          if (i < mc) {
#pragma unroll
            for (int j = 1; j < NM; ++j)
              if (j < nm) bcache[(j - 1) * mc + i] = pt[j];
          }
          const Real yy = (Real)sy[i];
          const Real w = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < nm) rows[j * kChP + tid] = w * pt[j];
#pragma unroll
          for (int j = 1; j < NM; ++j)
            if (j < nm) rows[(nm + j - 1) * kChP + tid] = -w * yy * pt[j];
          rows[n * kChP + tid] = w * yy;
          for (int j = naug; j < 4 * side; ++j) rows[j * kChP + tid] = 0;
        }
        __syncthreads();
        gram_chunk<Real>(rows, cnt, ntiles, sgc, acc);
        __syncthreads();
      }
      gram_finish<Real>(acc, ntiles, sgc, naug, G, red);
    }

    // ---------------- phase 4: equilibrate, factor, first solve
    // The leading n x n block of G (stride naug) is the normal matrix and
    // column n holds A^T b; the scaled block is factored in G with stride n.
    {
      if (tid < n) {
        const Real dg = G[tid * naug + tid];
        sh.scl[tid] = dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0;
        sh.gvec[tid] = G[tid * naug + n];
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += kThreads) {
        const int i = e / n, j = e % n;
        red[e] = G[i * naug + j] * sh.scl[i] * sh.scl[j];
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += kThreads) G[e] = red[e];
      if (tid < n) sh.gvec[tid] *= sh.scl[tid];
      __syncthreads();
      if (wid == 0) {
        warp_chol<Real>(G, n, n, (Real)a.drop_tol, sh.invd, &sh.keep_cnt);
        warp_solve<Real>(G, n, n, sh.invd, sh.gvec);
      }
      __syncthreads();
      if (tid < n) sh.xsol[tid] = (double)(sh.gvec[tid] * sh.scl[tid]);
      if (tid == 0) sh.flags = (sh.keep_cnt < n) ? RP_FIT_RANK_DEFICIENT : 0;
      __syncthreads();
    }

    // ---------------- phase 5: refinement from the samples, then a final
    // pass checking q > 0 at every sample
    const int sgc = max(1, kThreads / nm);
    float prev_rel = INFINITY;
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
      // g = A^T r, r = b - A x.  With rows w [pt, -y pt'],
      // g_num_j = sum_i (w r)_i pt_ij and g_den_j = -sum_i (w y r)_i pt_ij.
      Real gn = 0, gd = 0, cn = 0, cd = 0;
      int pole = 0;
      for (int base = 0; base < m; base += kCh) {
        const int cnt = min(kCh, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real pt[NM];
          if (i < mc) {
            pt[0] = 1;
#pragma unroll
            for (int j = 1; j < NM; ++j) pt[j] = (j < nm) ? bcache[(j - 1) * mc + i] : (Real)0;
          } else {
            Real psi[NM];
            eval_psi<Real, NM>(sh, d, nm, sx0[i], sx1[i], sx2[i], psi);
            whiten<Real, NM>(sh, psi, pt);
#pragma unroll
            for (int j = 1; j < NM; ++j)
              if (j < nm) rows[(j - 1) * kChP + tid] = pt[j];
          }
          if (final_pass) {
            double q = 1.0;
#pragma unroll
            for (int j = 1; j < NM; ++j)
              if (j < nm) q += sh.xsol[nm + j - 1] * (double)pt[j];
            pole |= !(q > 0.0);
          } else {
            const Real yy = (Real)sy[i];
            const Real w = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
            Real r;
            if constexpr (sizeof(Real) == 8) {
              double s = w * yy;
#pragma unroll
              for (int j = 0; j < NM; ++j)
                if (j < nm) s -= w * pt[j] * sh.xsol[j];
#pragma unroll
              for (int j = 1; j < NM; ++j)
                if (j < nm) s += w * yy * pt[j] * sh.xsol[nm + j - 1];
              r = s;
            } else {
              // compensated dot product (Ogita, Rump & Oishi 2005, "Dot2") of
              // the float row with the split solution xhi + xlo
              const float wy = w * yy;
              float s = wy, c = 0.0f;
#pragma unroll
              for (int j = 0; j < 2 * NM - 1; ++j) {
                const bool num = j < NM;
                const int jj = num ? j : j - NM + 1;
                if (jj < nm) {
                  const int col = num ? jj : nm + jj - 1;
                  const float av = num ? w * pt[jj] : -wy * pt[jj];
                  const float pr = av * sh.xhi[col];
                  const float pe = fmaf(av, sh.xhi[col], -pr);
                  float t, e;
                  two_sum(s, -pr, t, e);
                  s = t;
                  c += e - pe - av * sh.xlo[col];
                }
              }
              r = s + c;
            }
            rvec[tid] = w * r;
            rvec[kCh + tid] = w * yy * r;
          }
        }
        __syncthreads();
        if (!final_pass && tid < nm * sgc) {
          const int j = tid % nm, g = tid / nm;
          Real pn = 0, pd = 0;
          for (int s2 = g; s2 < cnt; s2 += sgc) {
            const int i2 = base + s2;
            const Real bv = (j == 0) ? (Real)1
                                     : (i2 < mc ? bcache[(j - 1) * mc + i2] : rows[(j - 1) * kChP + s2]);
            pn = fma(bv, rvec[s2], pn);
            pd = fma(bv, rvec[kCh + s2], pd);
          }
          const Real y1 = pn - cn, t1 = gn + y1;
          cn = (t1 - gn) - y1;
          gn = t1;
          const Real y2 = pd - cd, t2 = gd + y2;
          cd = (t2 - gd) - y2;
          gd = t2;
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
      if (tid < nm * sgc) {
        red[tid] = gn - cn;
        red[kThreads + tid] = gd - cd;
      }
      __syncthreads();
      if (tid < nm) {
        Real sn = 0, sd = 0;
        for (int g = 0; g < sgc; ++g) {
          sn += red[g * nm + tid];
          sd += red[kThreads + g * nm + tid];
        }
        sh.gvec[tid] = sn * sh.scl[tid];
        if (tid >= 1) sh.gvec[nm + tid - 1] = -sd * sh.scl[nm + tid - 1];
      }
      __syncthreads();
      if (wid == 0) {
        warp_solve<Real>(G, n, n, sh.invd, sh.gvec);
        float dn = 0, xn = 0;
        for (int j = lane; j < n; j += 32) {
          const double dx = (double)(sh.gvec[j] * sh.scl[j]);
          const double xv = sh.xsol[j] + dx;
          sh.xsol[j] = xv;
          dn += (float)(dx * dx);
          xn += (float)(xv * xv);
        }
        dn = warp_sum(dn);
        xn = warp_sum(xn);
        if (lane == 0) {
          sh.dnorm = sqrtf(dn);
          sh.xnorm = sqrtf(xn);
        }
      }
      __syncthreads();
      const float rel = sh.xnorm > 0.0f ? sh.dnorm / sh.xnorm : 0.0f;
      if (rel <= (float)a.tol) refine_state = 1;
      else if (it >= 1 && rel > 0.5f * prev_rel) refine_state = (rel <= 1e-5f) ? 1 : 2;
      prev_rel = rel;
    }

    // ---------------- phase 6: back to the monomial basis (FP64)
    {
      double *cpsi = reinterpret_cast<double *>(red);   // [2][kMaxNm]
      double *P = cpsi + 2 * kMaxNm;                      // [3][5][5]
      if (tid < 2 * nm) {
        const int which = tid / nm, i = tid % nm;   // 0 numerator, 1 denominator
        if (i >= 1) {
          double u = 0;
          for (int j = i; j < nm; ++j) {
            const double cj = which == 0 ? sh.xsol[j] : sh.xsol[nm + j - 1];
            u += (double)sh.W[i][j] * cj;
          }
          cpsi[which * kMaxNm + i] = u;
        }
      }
      if (tid >= 96 && tid < 96 + 3 * (kMaxDeg + 1)) {
        // Q_k(u), u = (x' - mu) isg, as a polynomial in x'
        const int v = (tid - 96) / (kMaxDeg + 1), k = (tid - 96) % (kMaxDeg + 1);
        const double mu = sh.mu_v[v], isg = sh.isg_v[v];
        double out[kMaxDeg + 1] = {0, 0, 0, 0, 0};
        if (k <= d) {
          double isgl = 1.0;
          for (int l = 0; l <= k; ++l) {
            const double t = sh.Tm[v][l][k];
            if (t != 0.0) {
              double binom = 1.0;
              for (int ii = 0; ii <= l; ++ii) {
                double mpow = 1.0;
                for (int q = 0; q < l - ii; ++q) mpow *= -mu;
                out[ii] += t * isgl * binom * mpow;
                binom = binom * (double)(l - ii) / (double)(ii + 1);
              }
            }
            isgl *= isg;
          }
        }
        for (int i2 = 0; i2 <= kMaxDeg; ++i2) P[(v * (kMaxDeg + 1) + k) * (kMaxDeg + 1) + i2] = out[i2];
      }
      __syncthreads();
      if (tid < 2) {
        double c0 = tid == 0 ? sh.xsol[0] : 1.0;
        for (int i = 1; i < nm; ++i) c0 -= (double)sh.mupsi[i] * cpsi[tid * kMaxNm + i];
        cpsi[tid * kMaxNm] = c0;
      }
      __syncthreads();
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
  int k = 0;
  for (int s = 0; s <= kMaxDeg; ++s)
    for (int a = s; a >= 0; --a)
      for (int b = s - a; b >= 0; --b) {
        e[k][0] = (int8_t)a;
        e[k][1] = (int8_t)b;
        e[k][2] = (int8_t)(s - a - b);
        ++k;
      }
  cudaMemcpyToSymbol(c_exp, e, sizeof(e));
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
