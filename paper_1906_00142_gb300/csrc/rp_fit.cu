// Batched least-squares fitting of rational functions (Sec. 4.2).
//
// One warp owns one fit at a time (persistent over fits).  The linearised
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
//     inverse Cholesky factor of their Gram matrix (Psi~);
//  5. the design rows w_i [1, Psi~.., -y_i Psi~..] with right-hand side
//     w_i y_i give the augmented Gram matrix, which is equilibrated and
//     factored with column dropping (pivot below a drop tolerance: column
//     removed, reported as rank deficiency);
//  6. iterative refinement recomputes the residual from the samples
//     (compensated FP32 dot products against the FP64 solution -- Ogita,
//     Rump & Oishi's Dot2 -- on the FP32 path, plain FP64 on the FP64 path),
//     stopping at ||dx|| <= tol ||x|| or when the corrections stop shrinking;
//  7. the solution is mapped back to the monomial basis of the box-normalised
//     variables in FP64.  Every refinement pass also checks that q is positive
//     at every sample for the solution the pass starts from.
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
// Per-warp fit state.  One warp owns one fit at a time; all its state lives
// in a private slice of shared memory, so no block-wide barrier is needed
// and the serial steps of one fit overlap with other warps' fits.

template <class Real, int DMAX>
struct WarpFit {
  static constexpr int NM = (DMAX + 1) * (DMAX + 2) * (DMAX + 3) / 6;
  static constexpr int NAUG = 2 * NM;
  // staging stride: >= NAUG, multiple of 4, odd multiple of 4 (LDS.128 reads
  // of one row by many lanes spread over banks)
  static constexpr int LDS = (((NAUG + 3) / 4) % 2 == 1) ? ((NAUG + 3) / 4) * 4 : ((NAUG + 3) / 4 + 1) * 4;
  static constexpr int WS = ((NM + 3) / 4) * 4;   // row stride of W (16-byte rows)
  double xsol[NAUG];                  // solution (design basis, unscaled)
  double lo[3], hi[3];
  Real G[NAUG * NAUG];                // Gram, then factor (stride n)
  Real stage[32 * LDS];               // 32 staged rows / scratch
  Real W[NM * WS];                    // whitening, upper triangular on 1..nm-1, stride WS
  Real mupsi[NM];
  Real gvec[NAUG], scl[NAUG], invd[NAUG], invw[NM];
  Real rbuf[2][32];
  Real Tm[3][kMaxDeg + 1][kMaxDeg + 1];  // Q_k(u) = sum_l Tm[l][k] u^l
  Real mu_v[3], isg_v[3], sc_v[3], of_v[3];
  double xprev[NAUG];                 // best solution so far (refinement)
  double uv[2][NM];                   // solution in the unwhitened basis: p = c_p + psi.u, q = c_q + psi.v
  Real HK[2][NM];                     // sum_s (w r)_s psi_s and sum_s (w y r)_s psi_s
  float uvhi[2][NM], uvlo[2][NM];     // split u, v (compensated residuals)
  float xhi[NAUG], xlo[NAUG];
  unsigned dslot[3][kMaxDeg + 1];
  int keep_cnt, keep_w;
};

template <class Real, int DMAX>
__host__ __device__ constexpr size_t warpfit_bytes() {
  return (sizeof(WarpFit<Real, DMAX>) + 15) & ~size_t(15);
}

// Unwhitened basis Psi at one sample (compile-time bound NM, runtime nm).
template <class Real, int DMAX, int NM>
__device__ __forceinline__ void eval_psi(const WarpFit<Real, DMAX> &w, int d, int nm, float x0,
                                         float x1, float x2, Real (&psi)[NM]) {
  Real Q[3][kMaxDeg + 1];
  const float xv[3] = {x0, x1, x2};
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const Real xn = fma((Real)xv[v], w.sc_v[v], w.of_v[v]);
    const Real u = (xn - w.mu_v[v]) * w.isg_v[v];
    Real pw[kMaxDeg + 1];
    pw[0] = 1;
#pragma unroll
    for (int l = 1; l <= DMAX; ++l) pw[l] = pw[l - 1] * u;
#pragma unroll
    for (int k = 0; k <= DMAX; ++k) {
      Real s = 0;
#pragma unroll
      for (int l = 0; l <= k; ++l) s = fma(w.Tm[v][l][k], pw[l], s);
      Q[v][k] = (k <= d) ? s : (Real)0;
    }
  }
#pragma unroll
  for (int j = 0; j < NM; ++j)
    psi[j] = (j < nm) ? Q[0][c_exp[j][0]] * Q[1][c_exp[j][1]] * Q[2][c_exp[j][2]] : (Real)0;
}

// Whitened basis: pt[0] = 1, pt[j] = sum_{1<=i<=j} (Psi_i - mean_i) W[i][j].
// W is zero below the diagonal, so rows are read from the aligned 4-block
// that holds the diagonal (128-bit loads on the FP32 path).
template <class Real, int DMAX, int NM>
__device__ __forceinline__ void whiten(const WarpFit<Real, DMAX> &w, const Real (&psi)[NM],
                                       Real (&pt)[NM]) {
  constexpr int WS = WarpFit<Real, DMAX>::WS;
  Real acc[WS];
#pragma unroll
  for (int j = 0; j < WS; ++j) acc[j] = 0;
#pragma unroll
  for (int i = 1; i < NM; ++i) {
    const Real c = psi[i] - w.mupsi[i];
    if constexpr (sizeof(Real) == 4) {
#pragma unroll
      for (int j4 = (i / 4) * 4; j4 < WS; j4 += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(&w.W[i * WS + j4]);
        acc[j4] = fmaf(c, v.x, acc[j4]);
        acc[j4 + 1] = fmaf(c, v.y, acc[j4 + 1]);
        acc[j4 + 2] = fmaf(c, v.z, acc[j4 + 2]);
        acc[j4 + 3] = fmaf(c, v.w, acc[j4 + 3]);
      }
    } else {
#pragma unroll
      for (int j = i; j < NM; ++j) acc[j] = fma(c, w.W[i * WS + j], acc[j]);
    }
  }
  pt[0] = 1;
#pragma unroll
  for (int j = 1; j < NM; ++j) pt[j] = acc[j];
}

// t-th tile of the lower triangle (row-major): rb >= cb
__device__ __forceinline__ void tile_of(int t, int &rb, int &cb) {
  int r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  rb = r;
  cb = t - r * (r + 1) / 2;
}

// Accumulate the 32 staged rows (stride LDS) into this lane's TS x TS tiles
// of the lower triangle of the Gram; tile t of lane = lane + 32 k.
template <class Real, int TS, int TPL, int LDS>
__device__ __forceinline__ void gram_stage(const Real *stage, int ntiles, Real (&acc)[TPL][TS * TS]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    const int t = lane + 32 * k;
    if (t >= ntiles) break;
    int rb, cb;
    tile_of(t, rb, cb);
    // partial over the 32 staged samples, then one add into the running sum
    // (blocked summation: error ~ (32 + m/32) u instead of m u)
    Real part[TS * TS];
#pragma unroll
    for (int i = 0; i < TS * TS; ++i) part[i] = 0;
#pragma unroll 4
    for (int s = 0; s < 32; ++s) {
      Real av[TS], bv[TS];
      if constexpr (TS == 4 && sizeof(Real) == 4) {
        const float4 va = *reinterpret_cast<const float4 *>(stage + s * LDS + 4 * rb);
        const float4 vb = *reinterpret_cast<const float4 *>(stage + s * LDS + 4 * cb);
        av[0] = va.x; av[1] = va.y; av[2] = va.z; av[3] = va.w;
        bv[0] = vb.x; bv[1] = vb.y; bv[2] = vb.z; bv[3] = vb.w;
      } else {
#pragma unroll
        for (int i = 0; i < TS; ++i) {
          av[i] = stage[s * LDS + TS * rb + i];
          bv[i] = stage[s * LDS + TS * cb + i];
        }
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) part[TS * i + j] = fma(av[i], bv[j], part[TS * i + j]);
    }
#pragma unroll
    for (int i = 0; i < TS * TS; ++i) acc[k][i] += part[i];
  }
}

template <class Real, int TS, int TPL>
__device__ __forceinline__ void gram_store(const Real (&acc)[TPL][TS * TS], int ntiles, int n, Real *G) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < TPL; ++k) {
    const int t = lane + 32 * k;
    if (t >= ntiles) break;
    int rb, cb;
    tile_of(t, rb, cb);
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) {
        const int r = TS * rb + i, c = TS * cb + j;
        if (r < n && c < n) {
          G[r * n + c] = acc[k][TS * i + j];
          G[c * n + r] = acc[k][TS * i + j];
        }
      }
  }
}

// ---------------------------------------------------------------------
// The fit kernel.  Real = double: plain FP64 path; Real = float: FP32 path.

constexpr int kMaxWarps = 8;

template <class Real, int DMAX>
__global__ void __launch_bounds__(kMaxWarps * 32) fit_kernel(FitArgs a, int warps_per_cta) {
  using WF = WarpFit<Real, DMAX>;
  constexpr int NM = WF::NM;
  constexpr int NAUG = WF::NAUG;
  constexpr int LDS = WF::LDS;
  constexpr int WS = WF::WS;
  constexpr int S2 = (NM + 1) / 2;                       // 2x2 tiles of the Psi Gram
  constexpr int T2 = (S2 * (S2 + 1) / 2 + 31) / 32;
  constexpr int S4 = (NAUG + 3) / 4;                     // 4x4 tiles of the design Gram
  constexpr int T4 = (S4 * (S4 + 1) / 2 + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid >= warps_per_cta) return;
  WF &w = *reinterpret_cast<WF *>(smem_raw + warpfit_bytes<Real, DMAX>() * wid);
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_cta;
  for (int64_t f = (int64_t)blockIdx.x * warps_per_cta + wid; f < a.F; f += nwarps) {
    // ---------------- phase 0: range, degree, validation, box, distinct values
    const int64_t b0 = a.off[f], b1 = a.off[f + 1];
    const int d = a.degs ? (int)a.degs[f] : a.d_uniform;
    const bool range_ok = b0 >= 0 && b1 >= b0 && b1 <= a.S;
    const int m = range_ok ? (int)(b1 - b0) : 0;
    double *cf = a.coef + f * kStride;
    for (int j = lane; j < kStride; j += 32) {
      cf[j] = 0.0;
      if (a.coef32) a.coef32[f * kStride + j] = 0.0f;
    }
    if (lane < 6) a.box[f * 6 + lane] = 0.0;
    if (d < 1 || d > DMAX || m == 0) {
      if (lane == 0) {
        a.status[f] = RP_FIT_EMPTY;
        a.rank[f] = 0;
      }
      continue;
    }
    const int nm = num_monomials(d);
    const int nc = nm - 1;
    const int naug = 2 * nm;
    const int n = naug - 1;
    const float *gx0 = a.x + b0, *gx1 = a.x + a.S + b0, *gx2 = a.x + 2 * a.S + b0, *gy = a.y + b0;
    if (lane < 3 * (kMaxDeg + 1)) (&w.dslot[0][0])[lane] = kEmpty;
    __syncwarp();
    float lmin[3] = {INFINITY, INFINITY, INFINITY}, lmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int i = lane; i < m; i += 32) {
      const float v0 = gx0[i], v1 = gx1[i], v2 = gx2[i], yy = gy[i];
      distinct_insert(w.dslot[0], v0);
      distinct_insert(w.dslot[1], v1);
      distinct_insert(w.dslot[2], v2);
      if (!(isfinite(v0) && isfinite(v1) && isfinite(v2) && isfinite(yy))) bad |= RP_FIT_NONFINITE;
      else if (a.weighted && !(yy > 0.0f)) bad |= RP_FIT_NONPOS_Y;
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
    for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (bad) {
      if (lane == 0) {
        a.status[f] = (bad & RP_FIT_NONFINITE) ? RP_FIT_NONFINITE : RP_FIT_NONPOS_Y;
        a.rank[f] = 0;
      }
      continue;
    }
    if (lane < 3) {
      const double mn = lmin[lane], mx = lmax[lane];
      w.lo[lane] = mn;
      w.hi[lane] = mx;
      a.box[f * 6 + 2 * lane] = mn;
      a.box[f * 6 + 2 * lane + 1] = mx;
      if (mx > mn) {   // x' = 2 (x - lo) / (hi - lo) - 1 = x * sc + of
        const double sc = 2.0 / (mx - mn);
        w.sc_v[lane] = (Real)sc;
        w.of_v[lane] = (Real)(-1.0 - mn * sc);
      } else {
        w.sc_v[lane] = 0;
        w.of_v[lane] = 0;
      }
    }
    __syncwarp();

    // ---------------- phase 1: standardisation, marginal orthonormal polynomials
    {
      Real acc[3] = {0, 0, 0};
      for (int i = lane; i < m; i += 32) {
        acc[0] += fma((Real)gx0[i], w.sc_v[0], w.of_v[0]);
        acc[1] += fma((Real)gx1[i], w.sc_v[1], w.of_v[1]);
        acc[2] += fma((Real)gx2[i], w.sc_v[2], w.of_v[2]);
      }
      Real mu[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) mu[v] = warp_sum(acc[v]) / (Real)m;
      Real mom[3][2 * kMaxDeg];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < 2 * kMaxDeg; ++k) mom[v][k] = 0;
      for (int i = lane; i < m; i += 32) {
        const float xv[3] = {gx0[i], gx1[i], gx2[i]};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const Real c = fma((Real)xv[v], w.sc_v[v], w.of_v[v]) - mu[v];
          Real pw = c;
#pragma unroll
          for (int k = 0; k < 2 * DMAX; ++k) {
            mom[v][k] += pw;
            pw *= c;
          }
        }
      }
      double M[3][2 * kMaxDeg + 1];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        M[v][0] = 1.0;
#pragma unroll
        for (int k = 0; k < 2 * DMAX; ++k) M[v][k + 1] = (double)warp_sum(mom[v][k]) / (double)m;
      }
      if (lane < 3) {
        const int v = lane;
        const double var = M[v][2];
        w.mu_v[v] = mu[v];
        for (int l = 0; l <= kMaxDeg; ++l)
          for (int k = 0; k <= kMaxDeg; ++k) w.Tm[v][l][k] = (l == 0 && k == 0) ? (Real)1 : (Real)0;
        if (w.sc_v[v] == (Real)0 || !(var > 0.0)) {
          w.isg_v[v] = 0;
        } else {
          const double isg = 1.0 / sqrt(var);
          w.isg_v[v] = (Real)isg;
          double Ms[2 * kMaxDeg + 1];
          Ms[0] = 1.0;
          double pw = isg;
          for (int k = 1; k <= 2 * DMAX; ++k) {
            Ms[k] = M[v][k] * pw;
            pw *= isg;
          }
          int cnt = 0;
          for (int k = 0; k <= kMaxDeg; ++k) cnt += w.dslot[v][k] != kEmpty;
          float T[kMaxDeg + 1][kMaxDeg + 1];
          marginal_transform(Ms, d, min(d, cnt - 1), T);
          for (int l = 0; l <= kMaxDeg; ++l)
            for (int k = 0; k <= kMaxDeg; ++k) w.Tm[v][l][k] = (Real)T[l][k];
        }
      }
      __syncwarp();
    }

    // ---------------- phase 2: Gram of Psi (nm columns), means, whitening
    {
      const int side = (nm + 1) / 2;
      const int ntiles = side * (side + 1) / 2;
      Real acc[T2][4];
#pragma unroll
      for (int k = 0; k < T2; ++k)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[k][i] = 0;
      for (int base = 0; base < m; base += 32) {
        const int i = base + lane;
        Real psi[NM];
        if (i < m) {
          eval_psi<Real, DMAX, NM>(w, d, nm, gx0[i], gx1[i], gx2[i], psi);
        } else {
#pragma unroll
          for (int j = 0; j < NM; ++j) psi[j] = 0;
        }
#pragma unroll
        for (int j = 0; j < 2 * S2; ++j) w.stage[lane * LDS + j] = (j < NM) ? psi[j] : (Real)0;
        __syncwarp();
        gram_stage<Real, 2, T2, LDS>(w.stage, ntiles, acc);
        __syncwarp();
      }
      gram_store<Real, 2, T2>(acc, ntiles, nm, w.G);
      __syncwarp();
      // means (row 0 holds the sums of Psi_j) and the centred Gram / m of the
      // non-constant functions, equilibrated, in `stage`
      for (int j = lane; j < NM; j += 32) w.mupsi[j] = (j < nm) ? w.G[j] / (Real)m : (Real)0;
      for (int e = lane; e < NM * WS; e += 32) w.W[e] = 0;
      __syncwarp();
      for (int e = lane; e < nc * nc; e += 32) {
        const int i = e / nc + 1, j = e % nc + 1;
        w.stage[e] = (w.G[i * nm + j] - (Real)m * w.mupsi[i] * w.mupsi[j]) / (Real)m;
      }
      __syncwarp();
      for (int j = lane; j < nc; j += 32) {
        const Real dg = w.stage[j * nc + j];
        w.scl[j] = dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0;
      }
      __syncwarp();
      for (int e = lane; e < nc * nc; e += 32) w.stage[e] *= w.scl[e / nc] * w.scl[e % nc];
      // the whitening only preconditions: any positive pivot is kept (the
      // basis stays a basis of the same space); only directions whose pivot
      // is at rounding level or below are dropped
      warp_chol<Real>(w.stage, nc, nc, sizeof(Real) == 8 ? (Real)1e-14 : (Real)1e-10, w.invw,
                      &w.keep_w);
      // R^{-1} (R = L^T, R[i][l] = L[l][i]) column by column into G; W = D R^{-1}
      for (int j = lane; j < nc; j += 32)
        for (int i = j; i >= 0; --i) {
          Real s = (i == j) ? (Real)1 : (Real)0;
          for (int l = i + 1; l <= j; ++l) s -= w.stage[l * nc + i] * w.G[l * nc + j];
          w.G[i * nc + j] = s * w.invw[i];
        }
      __syncwarp();
      for (int e = lane; e < nc * nc; e += 32) {
        const int i = e / nc, j = e % nc;
        if (i <= j) w.W[(i + 1) * WS + (j + 1)] = w.G[i * nc + j] * w.scl[i];
      }
      __syncwarp();
    }

    // ---------------- phase 3: the design Gram [num (nm) | den (nm-1) | rhs]
    {
      const int side = (naug + 3) / 4;
      const int ntiles = side * (side + 1) / 2;
      Real acc[T4][16];
#pragma unroll
      for (int k = 0; k < T4; ++k)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[k][i] = 0;
      for (int base = 0; base < m; base += 32) {
        const int i = base + lane;
        Real *row = w.stage + lane * LDS;
        if (i < m) {
          Real psi[NM], pt[NM];
          eval_psi<Real, DMAX, NM>(w, d, nm, gx0[i], gx1[i], gx2[i], psi);
          whiten<Real, DMAX, NM>(w, psi, pt);
          const Real yy = (Real)gy[i];
          const Real wt = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < nm) row[j] = wt * pt[j];
#pragma unroll
          for (int j = 1; j < NM; ++j)
            if (j < nm) row[nm + j - 1] = -wt * yy * pt[j];
          row[n] = wt * yy;
          for (int j = naug; j < 4 * S4; ++j) row[j] = 0;
        } else {
          for (int j = 0; j < 4 * S4; ++j) row[j] = 0;
        }
        __syncwarp();
        gram_stage<Real, 4, T4, LDS>(w.stage, ntiles, acc);
        __syncwarp();
      }
      gram_store<Real, 4, T4>(acc, ntiles, naug, w.G);
      __syncwarp();
    }

    // ---------------- phase 4: equilibrate, factor, first solve
    // The leading n x n block of G (stride naug) is the normal matrix and
    // column n holds A^T b; the scaled block is compacted in place to stride n
    // (row by row: each destination row ends before the next source row).
    {
      for (int j = lane; j < n; j += 32) {
        const Real dg = w.G[j * naug + j];
        w.scl[j] = dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0;
        w.gvec[j] = w.G[j * naug + n];
      }
      __syncwarp();
      for (int i = 0; i < n; ++i) {
        Real v[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int j = lane + 32 * r;
          v[r] = (j < n) ? w.G[i * naug + j] * w.scl[i] * w.scl[j] : (Real)0;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int j = lane + 32 * r;
          if (j < n) w.G[i * n + j] = v[r];
        }
        __syncwarp();
      }
      for (int j = lane; j < n; j += 32) w.gvec[j] *= w.scl[j];
      warp_chol<Real>(w.G, n, n, (Real)a.drop_tol, w.invd, &w.keep_cnt);
      warp_solve<Real>(w.G, n, n, w.invd, w.gvec);
      for (int j = lane; j < n; j += 32) w.xsol[j] = (double)(w.gvec[j] * w.scl[j]);
      __syncwarp();
    }

    // ---------------- phase 5: refinement from the samples.
    // With u = W x_num, v = W x_den (index 1..nm-1) and
    //   c_p = x_num[0] - mu.u, c_q = 1 - mu.v,
    // the fit's p and q at a sample are p = c_p + psi.u, q = c_q + psi.v, and
    // the design residual is r = w (y q - p).  The normal-equation residual
    // g = A^T r follows from H_i = sum (w r) psi_i and K_i = sum (w y r) psi_i:
    //   g_num_0 = H_0, g_num_j = sum_{i<=j} W_ij (H_i - mu_i H_0),
    //   g_den_j = -sum_{i<=j} W_ij (K_i - mu_i K_0),
    // so the passes work in the unwhitened basis.  Each pass also returns the
    // objective sum r^2 (a step that increases it is undone) and whether
    // q > 0 at every sample.  Residuals are plain FP32 until the corrections
    // fall below 1e-4 relative, then compensated (Dot2).
    int flags = (w.keep_cnt < n) ? RP_FIT_RANK_DEFICIENT : 0;
    float prev_rel = INFINITY, obj_prev = INFINITY;
    bool compensated = sizeof(Real) == 8, done = false, converged = false;
    int pole_prev = 0, it = 0;
    for (;; ++it) {
      const bool update = it < a.max_refine && !done;
      // u, v, c_p, c_q (FP64) and their float splits
      for (int e = lane; e < 2 * NM; e += 32) {
        const int which = e / NM, i2 = e % NM;
        double acc = 0.0;
        if (i2 >= 1 && i2 < nm)
          for (int j2 = i2; j2 < nm; ++j2)
            acc += (double)w.W[i2 * WS + j2] * (which == 0 ? w.xsol[j2] : w.xsol[nm + j2 - 1]);
        w.uv[which][i2] = acc;
      }
      __syncwarp();
      if (lane < 2) {
        double c = lane == 0 ? w.xsol[0] : 1.0;
        for (int i2 = 1; i2 < nm; ++i2) c -= (double)w.mupsi[i2] * w.uv[lane][i2];
        w.uv[lane][0] = c;
      }
      __syncwarp();
      for (int e = lane; e < 2 * NM; e += 32) {
        const int which = e / NM, i2 = e % NM;
        const double v = w.uv[which][i2];
        const float h = (float)v;
        w.uvhi[which][i2] = h;
        w.uvlo[which][i2] = (float)(v - (double)h);
      }
      __syncwarp();
      Real hk[2][2] = {{0, 0}, {0, 0}};
      float obj = 0.0f;
      int pole = 0;
      for (int base = 0; base < m; base += 32) {
        const int i = base + lane;
        Real psi[NM];
        Real r = 0, yy = 0, wt = 0;
        if (i < m) {
          eval_psi<Real, DMAX, NM>(w, d, nm, gx0[i], gx1[i], gx2[i], psi);
          psi[0] = 1;
          yy = (Real)gy[i];
          wt = a.weighted ? (Real)1 / fabs(yy) : (Real)1;
          if constexpr (sizeof(Real) == 8) {
            double p = w.uv[0][0], q = w.uv[1][0];
#pragma unroll
            for (int j2 = 1; j2 < NM; ++j2) {
              p = fma(psi[j2], w.uv[0][j2], p);
              q = fma(psi[j2], w.uv[1][j2], q);
            }
            pole |= !(q > 0.0);
            r = wt * (yy * q - p);
          } else {
            float qf = w.uvhi[1][0];
#pragma unroll
            for (int j2 = 1; j2 < NM; ++j2) qf = fmaf(psi[j2], w.uvhi[1][j2], qf);
            pole |= !(qf > 0.0f);
            if (compensated) {
              // e = y q - p = sum over (y psi_j) v_j - psi_j u_j, j = 0..nm-1
              // (psi_0 = 1), Dot2 against the split u, v
              float sacc = 0.0f, c = 0.0f;
#pragma unroll
              for (int j2 = 0; j2 < 2 * NM; ++j2) {
                const int jj = j2 >> 1;
                const bool den = (j2 & 1) == 0;
                const float av = den ? yy * psi[jj] : -psi[jj];
                const float xh = den ? w.uvhi[1][jj] : w.uvhi[0][jj];
                const float xl = den ? w.uvlo[1][jj] : w.uvlo[0][jj];
                const float pr = av * xh;
                const float pe = fmaf(av, xh, -pr);
                float t, e;
                two_sum(sacc, pr, t, e);
                sacc = t;
                c += e + pe + av * xl;
              }
              r = wt * (sacc + c);
            } else {
              float p = w.uvhi[0][0];
#pragma unroll
              for (int j2 = 1; j2 < NM; ++j2) p = fmaf(psi[j2], w.uvhi[0][j2], p);
              r = wt * fmaf(yy, qf, -p);
            }
          }
          obj += (float)(r * r);
        } else {
#pragma unroll
          for (int j2 = 0; j2 < NM; ++j2) psi[j2] = 0;
        }
        if (update) {
#pragma unroll
          for (int j2 = 0; j2 < NM; ++j2) w.stage[lane * LDS + j2] = psi[j2];
          w.rbuf[0][lane] = wt * r;
          w.rbuf[1][lane] = wt * yy * r;
          __syncwarp();
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int j2 = lane + 32 * rr;
            if (j2 < nm) {
              Real pn = 0, pd = 0;
#pragma unroll 8
              for (int s2 = 0; s2 < 32; ++s2) {
                const Real bv = w.stage[s2 * LDS + j2];
                pn = fma(bv, w.rbuf[0][s2], pn);
                pd = fma(bv, w.rbuf[1][s2], pd);
              }
              hk[rr][0] += pn;
              hk[rr][1] += pd;
            }
          }
          __syncwarp();
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pole |= __shfl_xor_sync(0xffffffffu, pole, o);
      obj = warp_sum(obj);
      // a step that increases the objective by more than the objective's own
      // rounding level (plain FP32 residuals: ~1e-4 relative) is undone
      if (it > 0 && obj > obj_prev * (compensated ? 1.00001f : 1.0001f)) {
        for (int j2 = lane; j2 < n; j2 += 32) w.xsol[j2] = w.xprev[j2];
        pole = pole_prev;
        converged = converged || prev_rel <= 1e-4f;
        __syncwarp();
        break;
      }
      for (int j2 = lane; j2 < n; j2 += 32) w.xprev[j2] = w.xsol[j2];
      obj_prev = obj;
      pole_prev = pole;
      __syncwarp();
      if (!update) break;
      // g from H, K; scaled for the factored (equilibrated) system
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int j2 = lane + 32 * rr;
        if (j2 < nm) {
          w.HK[0][j2] = hk[rr][0];
          w.HK[1][j2] = hk[rr][1];
        }
      }
      __syncwarp();
      for (int e = lane; e < n; e += 32) {
        Real g;
        if (e < nm) {
          if (e == 0) {
            g = w.HK[0][0];
          } else {
            g = 0;
            for (int i2 = 1; i2 <= e; ++i2) g += w.W[i2 * WS + e] * (w.HK[0][i2] - w.mupsi[i2] * w.HK[0][0]);
          }
        } else {
          const int jd = e - nm + 1;
          g = 0;
          for (int i2 = 1; i2 <= jd; ++i2) g -= w.W[i2 * WS + jd] * (w.HK[1][i2] - w.mupsi[i2] * w.HK[1][0]);
        }
        w.gvec[e] = g * w.scl[e];
      }
      __syncwarp();
      warp_solve<Real>(w.G, n, n, w.invd, w.gvec);
      float dn = 0, xn = 0;
      for (int j2 = lane; j2 < n; j2 += 32) {
        const double dx = (double)(w.gvec[j2] * w.scl[j2]);
        const double xv = w.xsol[j2] + dx;
        w.xsol[j2] = xv;
        dn += (float)(dx * dx);
        xn += (float)(xv * xv);
      }
      dn = warp_sum(dn);
      xn = warp_sum(xn);
      __syncwarp();
      const float rel = xn > 0.0f ? sqrtf(dn / xn) : 0.0f;
      const bool was_compensated = compensated;
      if (!compensated && rel < 1e-4f) compensated = true;
      if (rel <= (float)a.tol) {
        done = converged = true;
      } else if (was_compensated && rel > 0.9f * prev_rel) {
        // corrections stopped shrinking: at the noise floor of the residuals
        done = true;
        converged = rel <= 1e-4f;
      }
      prev_rel = rel;
    }
    flags |= (pole_prev ? RP_FIT_POLE : 0);
    if (a.max_refine > 0 && !converged && !(prev_rel <= 1e-4f)) flags |= RP_FIT_NOT_CONVERGED;
    flags |= min(it, 255) << RP_FIT_ITER_SHIFT;

    // ---------------- phase 6: back to the monomial basis (FP64)
    {
      double *cpsi = reinterpret_cast<double *>(w.stage);   // [2][kMaxNm]
      double *P = cpsi + 2 * kMaxNm;                          // [3][5][5]
      for (int e = lane; e < 2 * nm; e += 32) {
        const int which = e / nm, i = e % nm;   // 0 numerator, 1 denominator
        if (i >= 1) {
          double u = 0;
          for (int j = i; j < nm; ++j) {
            const double cj = which == 0 ? w.xsol[j] : w.xsol[nm + j - 1];
            u += (double)w.W[i * WS + j] * cj;
          }
          cpsi[which * kMaxNm + i] = u;
        }
      }
      if (lane < 3 * (kMaxDeg + 1)) {
        // Q_k(u), u = (x' - mu) isg, as a polynomial in x'
        const int v = lane / (kMaxDeg + 1), k = lane % (kMaxDeg + 1);
        const double mu = w.mu_v[v], isg = w.isg_v[v];
        double out[kMaxDeg + 1] = {0, 0, 0, 0, 0};
        if (k <= d) {
          double isgl = 1.0;
          for (int l = 0; l <= k; ++l) {
            const double t = w.Tm[v][l][k];
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
      __syncwarp();
      if (lane < 2) {
        double c0 = lane == 0 ? w.xsol[0] : 1.0;
        for (int i = 1; i < nm; ++i) c0 -= (double)w.mupsi[i] * cpsi[lane * kMaxNm + i];
        cpsi[lane * kMaxNm] = c0;
      }
      __syncwarp();
      for (int e = lane; e < 2 * nm; e += 32) {
        const int which = e / nm, t = e % nm;
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
      if (lane == 0) {
        a.status[f] = flags;
        a.rank[f] = w.keep_cnt;
      }
      __syncwarp();
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

// Choose warps per CTA (1..8) to maximise resident warps per SM under the
// per-warp shared-memory slice, then launch a persistent grid.
template <class Real, int DMAX>
cudaError_t launch_t(const FitArgs &a, cudaStream_t s) {
  const size_t per_warp = warpfit_bytes<Real, DMAX>();
  int best_w = 1, best_total = 0, best_ctas = 1;
  for (int wpc = kMaxWarps; wpc >= 1; wpc /= 2) {
    const size_t smem = per_warp * wpc;
    if (smem > 227 * 1024) continue;
    cudaError_t e = cudaFuncSetAttribute(fit_kernel<Real, DMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fit_kernel<Real, DMAX>, wpc * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm * wpc > best_total) {
      best_total = per_sm * wpc;
      best_w = wpc;
      best_ctas = per_sm;
    }
  }
  if (best_total == 0) return cudaErrorInvalidConfiguration;
  const size_t smem = per_warp * best_w;
  cudaError_t e = cudaFuncSetAttribute(fit_kernel<Real, DMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)num_sms() * best_ctas;
  const int64_t need = (a.F + best_w - 1) / best_w;
  if (grid > need) grid = need;
  fit_kernel<Real, DMAX><<<(unsigned)grid, best_w * 32, smem, s>>>(a, best_w);
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
