#pragma once
// Batched least-squares fitting of rational functions (Sec. 4.2).
//
// One 128-thread CTA owns one fit at a time (persistent over fits; several
// CTAs per SM).  The linearised
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
//  6. iterative refinement recomputes the residual from the samples (FP32
//     paths: plain FP32 passes while the steps are large, then accurate
//     passes in double-float arithmetic -- head + tail FP32 pairs built from
//     error-free sums and products, ~2^-44 relative -- in which the basis
//     functions, the residual, the normal-equation residual's sums and the
//     sample means of the basis are all carried in pairs; plain FP64 on the
//     FP64 path), stopping at ||dx|| <= tol ||x|| or when the corrections
//     stop shrinking.  The first accurate pass also fixes the normalisation
//     mean(q) = 1 with the exact sample means;
//  7. the solution is mapped back to the monomial basis of the box-normalised
//     variables in FP64.  Every refinement pass also checks that q is positive
//     at every sample for the solution the pass starts from.
//
// Each step is a change of basis of the same function space under the same
// normalisation, so the fitted p/q is the least-squares solution the paper's
// SVD formulation defines (up to rounding).  The FP32 path factors in FP32
// (GB300's FP64 rate is ~1/58 of FP32): the factor only preconditions the
// refinement, whose residuals carry the accuracy.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "rp_fit.cuh"
#include "rp_internal.cuh"
#include "rp_tc.cuh"

namespace rpk {
namespace {


__constant__ int8_t c_exp[kMaxNm][3];   // graded-lex exponents
__constant__ int8_t c_idx[kMaxDeg + 1][kMaxDeg + 1][kMaxDeg + 1];   // exponents -> graded-lex index


// ---------------------------------------------------------------------
// helpers

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// ---- double-float arithmetic: a value is a pair (h, l) of FP32 numbers with
// |l| <= ulp(h) / 2, worth ~44 bits.  Error-free transformations of a sum
// (two_sum, Knuth) and of a product (two_prod via FMA), Dekker's
// renormalisation, and Ogita-Rump-Oishi's compensated dot product.  Products
// are formed with __fmul_rn so that the compiler never fuses them into a
// following addition (which would break the error-free identities).
struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl df_norm(float h, float l) {
  dfl r;
  r.h = h + l;
  r.l = l - (r.h - h);
  return r;
}
__device__ __forceinline__ dfl df_make(float h) { return dfl{h, 0.0f}; }
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_norm(p, e);
}
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return df_norm(p, e);
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return df_norm(s, e + (a.l + b.l));
}
__device__ __forceinline__ dfl df_addf(dfl a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  return df_norm(s, e + a.l);
}
// 1 / a as a pair (one Newton correction of the correctly rounded reciprocal)
__device__ __forceinline__ dfl df_recip(dfl a) {
  const float h = __frcp_rn(a.h);
  const float r = fmaf(-a.h, h, 1.0f) - __fmul_rn(a.l, h);
  return df_norm(h, __fmul_rn(r, h));
}
// Running compensated sum s + c of pair products (Dot2): each product's
// rounding error and each addition's error go to c.
struct dacc {
  float s, c;
};
__device__ __forceinline__ void dacc_fma(dacc &a, dfl x, dfl y) {
  const float p = __fmul_rn(x.h, y.h);
  float pe = fmaf(x.h, y.h, -p);
  pe = fmaf(x.h, y.l, pe);
  pe = fmaf(x.l, y.h, pe);
  float t, e;
  two_sum(a.s, p, t, e);
  a.s = t;
  a.c += e + pe;
}
__device__ __forceinline__ dfl dacc_get(const dacc &a) { return df_norm(a.s, a.c); }

// A double as a head + tail pair of FP32 numbers, read from its bit pattern
// with integer operations only (GB300 runs FP64 arithmetic and conversions
// at a small fraction of its FP32 rate): the head is v truncated to 24
// significant bits, the tail the remaining 29 mantissa bits truncated to
// 23 (relative error below 2^-46).  |v| outside [2^-80, 2^127) (zero
// included) takes the conversions instead.
__device__ __forceinline__ dfl split_d(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const int E = (int)((hw >> 20) & 0x7FFu);
  if (E < 1023 - 80 || E > 1023 + 126) {
    const float h = __double2float_rz(v);
    return dfl{h, __double2float_rn(v - (double)h)};
  }
  const unsigned sign = hw & 0x80000000u;
  // head: sign, exponent E - 1023 + 127, mantissa bits 51..29
  const float h = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // tail: mantissa bits 28..0 (the integer R, worth R 2^(E - 1075)); R >> 6
  // (< 2^23) becomes a float exactly through the 2^23 bias, then 2^(E - 1069)
  const float r = __uint_as_float(0x4B000000u | ((lw & 0x1FFFFFFFu) >> 6)) - 8388608.0f;
  const float l = __fmul_rn(r, __uint_as_float((unsigned)(E - 1069 + 127) << 23));
  return dfl{h, __uint_as_float(__float_as_uint(l) | sign)};
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

// Cholesky (lower) of the n x n matrix G (row stride ld) by all NT threads of
// the block, with column dropping: a pivot <= tol removes the column
// (invd = 0).  Step k scales column k, then updates the trailing lower
// triangle with one thread per entry.
template <class SR, int NT>
__device__ void cta_chol(SR *G, int n, int ld, SR tol, SR *invd, int *keep_cnt) {
  const int tid = threadIdx.x;
  for (int k = 0; k < n; ++k) {
    const SR p = G[k * ld + k];
    const bool keep = p > tol;
    const SR inv = keep ? rsqrt_pos<SR>(p) : (SR)0;
    __syncthreads();
    if (tid == 0) {
      G[k * ld + k] = keep ? p * inv : (SR)0;
      invd[k] = inv;
    }
    for (int i = k + 1 + tid; i < n; i += NT) G[i * ld + k] *= inv;
    __syncthreads();
    const int r = n - k - 1;
    const int np = r * (r + 1) / 2;
    for (int e = tid; e < np; e += NT) {
      int ii = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      ii += ((ii + 1) * (ii + 2) / 2 <= e);
      ii -= (ii * (ii + 1) / 2 > e);
      const int jj = e - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      G[i * ld + j] -= G[i * ld + k] * G[j * ld + k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    int kept = 0;
    for (int k = 0; k < n; ++k) kept += invd[k] != (SR)0;
    *keep_cnt = kept;
  }
  __syncthreads();
}

// Cholesky of the (d+1) x (d+1) Hankel moment matrix of a standardised
// variable -> coefficients of the orthonormal polynomials (columns of the
// inverse factor).  A variable with only q distinct sample values supports
// polynomials of degree < q on the samples: Q_k for k > deg_eff (= q - 1) is
// set to 0.  Single thread, FP32 (the transform only has to give a
// well-scaled basis; it is used consistently wherever the basis is).
__device__ void marginal_transform(const float *M, int d, int deg_eff, float T[][kMaxDeg + 1]) {
  float R[kMaxDeg + 1][kMaxDeg + 1], Ti[kMaxDeg + 1][kMaxDeg + 1];
  bool ok[kMaxDeg + 1];
  for (int i = 0; i <= kMaxDeg; ++i)
    for (int j = 0; j <= kMaxDeg; ++j) R[i][j] = Ti[i][j] = 0.0f;
  for (int k = 0; k <= d; ++k) {
    float p = M[2 * k];
    for (int l = 0; l < k; ++l) p -= R[l][k] * R[l][k];
    ok[k] = k <= deg_eff && M[2 * k] > 0.0f;
    if (!ok[k]) continue;
    // a supported direction whose pivot rounding has eaten is regularised
    // (any positive pivot keeps the polynomial basis a basis)
    p = fmaxf(p, 1e-6f * M[2 * k]);
    R[k][k] = sqrtf(p);
    const float inv = 1.0f / R[k][k];
    for (int j = k + 1; j <= d; ++j) {
      float s = M[k + j];
      for (int l = 0; l < k; ++l) s -= R[l][k] * R[l][j];
      R[k][j] = s * inv;
    }
  }
  for (int k = 0; k <= d; ++k) {
    if (!ok[k]) continue;
    Ti[k][k] = 1.0f / R[k][k];
    for (int i = k - 1; i >= 0; --i) {
      if (!ok[i]) continue;
      float s = 0;
      for (int l = i + 1; l <= k; ++l) s += R[i][l] * Ti[l][k];
      Ti[i][k] = -s / R[i][i];
    }
  }
  for (int l = 0; l <= kMaxDeg; ++l)
    for (int k = 0; k <= kMaxDeg; ++k) T[l][k] = (l <= d && k <= d) ? Ti[l][k] : 0.0f;
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
// Per-fit state of one CTA (128 threads).  Shared memory and registers are
// sized so that several CTAs share an SM: while one CTA runs the serial
// steps of its fit (factorisations, triangular solves) on one warp, the
// others' sample passes keep the SM busy.

constexpr int kT = 128;       // threads per CTA (one fit at a time)
constexpr int kMC = 512;      // samples per fit kept in shared memory
constexpr int kJacobiSweeps = 16;   // bound on the SVD route's Jacobi sweeps

// Tensor-core Gram shapes (Sec. 4.2 normal equations on tcgen05).  A Gram
// X^T X over the samples is one MMA chain D = A B^T with A = B = X^T stored
// K-major (K = samples): the B operand holds the NPAD padded columns, the A
// operand (M = 128 rows) reads the same tile and the shared memory after it
// (rows >= NPAD of D are never read).  One K-block = 32 samples = NPAD/8
// swizzle atoms.
template <int DMAX>
struct TcShape {
  static constexpr int NM = (DMAX + 1) * (DMAX + 2) * (DMAX + 3) / 6;
  static constexpr int NAUG = 2 * NM;
  static constexpr int NDES = ((NAUG + 15) / 16) * 16;
  static constexpr int NB_DES = NDES / 8 * 1024;
  static constexpr int TMEM_COLS = NDES <= 64 ? 64 : 128;
};

// GM: 0 = design Gram on CUDA cores (FP32 or FP64), 1 = design Gram on the
// tensor cores in one TF32 pass, 2 = in three TF32 passes (hi.hi + hi.lo +
// lo.hi), 3 = one BF16 pass, 4 = three BF16 passes.  The basis Gram (whitening) is always formed on CUDA cores: its
// condition number (~1e6 for the correlated B0, B1 of the 66 formats) needs
// round-to-nearest FP32 accumulation.
template <class Real, int DMAX, int GM>
struct CtaFit {
  static constexpr int NM = (DMAX + 1) * (DMAX + 2) * (DMAX + 3) / 6;
  static constexpr int NAUG = 2 * NM;
  // row stride of the staged rows: >= NAUG, an odd multiple of 4 (16-byte
  // rows; 128-bit reads of the same row by many threads spread over banks)
  static constexpr int LDS = (((NAUG + 3) / 4) % 2 == 1) ? ((NAUG + 3) / 4) * 4 : ((NAUG + 3) / 4 + 1) * 4;
  static constexpr int WS = ((NM + 3) / 4) * 4;   // row stride of W (16-byte rows)
  using TS = TcShape<DMAX>;
  static constexpr int ROWS_BYTES = kT * LDS * (int)sizeof(Real);
  // staging: hi then lo K-blocks (4 TF32 or 2 BF16 K-blocks per chunk)
  static constexpr int TC_NKB = (GM == 3 || GM == 4) ? 2 : 4;
  static constexpr bool TC_X3 = GM == 2 || GM == 4;
  static constexpr int TC_BYTES = GM == 0 ? 0 : (TC_X3 ? 2 : 1) * TC_NKB * TS::NB_DES;
  // accurate pass rows: the basis as (head, tail) pairs, then from DF_AO the
  // pairs a = w r and b = w y r; stride an odd multiple of 4 floats
  static constexpr int DF_AO = ((2 * NM + 3) / 4) * 4;
  static constexpr int DF_LDD = ((DF_AO / 4 + 1) % 2 == 1) ? DF_AO + 4 : DF_AO + 8;
  static constexpr int DF_BYTES = sizeof(Real) == 4 ? kT * DF_LDD * 4 : 0;
  static constexpr int RB_BYTES = ROWS_BYTES > DF_BYTES ? ROWS_BYTES : DF_BYTES;
  static constexpr int STAGE_BYTES = RB_BYTES > TC_BYTES ? RB_BYTES : TC_BYTES;
  // furthest byte the M = 128 A operand reads, from the start of `stage`
  static constexpr int TC_REACH = GM == 0 ? 0 : ((TC_X3 ? 2 : 1) * TC_NKB - 1) * TS::NB_DES + 16384;
  alignas(16) Real stage[STAGE_BYTES / sizeof(Real)];   // first member: 1024-byte aligned
  double uv[2][NM], uvp[2][NM];       // FP64 path: (c, u) and (c, v) of p and q; previous
  double lo[3], hi[3];
  Real redr[4][32];                   // per-warp partial sums (phase 1)
  uint64_t mbar;                      // tensor-core completion barrier
  alignas(16) Real G[NAUG * NAUG];    // Gram, then factor (stride n)
  alignas(16) Real W[NM * WS];        // whitening, upper triangular on 1..nm-1 (128-bit loads)
  Real mupsi[NM];
  Real gvec[NAUG], scl[NAUG], invd[NAUG], invw[NM];
  Real xw[NAUG], xwp[NAUG], dxw[NAUG];  // iterate in the design basis (norms), previous, step
  // pivot rows of the sweep, padded to whole 8-column blocks (16-byte rows)
  static constexpr int RBW = ((NAUG + 7) / 8) * 8;
  alignas(16) Real rowb[2][RBW];
  Real duv[2][NM];                    // step of (c, u), (c, v)
  Real HK[2][NM];
  Real rbuf[2][kT];
  // Q_k(u) = sum_l Tm[l][k] u^l (rows padded to 8: 128-bit loads of k = 0..3)
  alignas(16) Real Tm[3][kMaxDeg + 1][8];
  Real mu_v[3], isg_v[3], sc_v[3], of_v[3];
  alignas(16) Real vc[3][4];          // per variable: sc, of, mu, isg
  alignas(16) float uvhi[2][NM];      // FP32 path: (c, u), (c, v) as head + tail
  alignas(16) float uvlo[2][NM];
  float uvphi[2][NM], uvplo[2][NM];   // previous
  float2 uvq[2][NM];                  // accurate pass: the iterate (head, tail) interleaved
  float mulo[NM];                     // FP32 path: tails of the exact sample means (mupsi: heads)
  float hkd[3][NM][2];                // accurate pass: H, K and the basis sums as pairs
  Real HKc[2][NM];                    // H_0, H_i - mu_i H_0 and K_0, K_i - mu_i K_0
  float redv[4][((2 * NM + 2 + 15) / 16) * 16];
  // sample cache (N, B0, B1, y) of fits with at most MC samples; none on the
  // FP32 degree-4 path, whose shared memory then admits 3 CTAs per SM
  static constexpr int MC = (sizeof(Real) == 4 && DMAX == 4 && GM == 0) ? 0 : kMC;
  float xs[4][MC > 0 ? MC : 1];
  float redf[4][32];
  unsigned dslot[3][kMaxDeg + 1];
  uint32_t tmem_base;
  long long next_fit[2];              // claimed point-set indices (alternating slots)
  int keep_cnt, keep_w, bad, set_deg;
  float fscal[4];
};

// Dynamic shared memory of one CTA: the state, at least TC_REACH bytes from
// its start, plus 1 KB to align the start to 1024 bytes.
template <class Real, int DMAX, int GM>
__host__ __device__ constexpr size_t ctafit_bytes() {
  using WF = CtaFit<Real, DMAX, GM>;
  // the 1 KB alignment slack only where swizzle atoms are staged
  return ((sizeof(WF) > (size_t)WF::TC_REACH ? sizeof(WF) : (size_t)WF::TC_REACH) + 15 & ~size_t(15)) +
         (GM > 0 ? 1024 : 0);
}

// Block-wide sum of one float per thread; result returned to every thread.
template <class S>
__device__ __forceinline__ float block_sum_f(S &w, float v, int slot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) w.redf[wid][slot] = v;
  __syncthreads();
  const float r = w.redf[0][slot] + w.redf[1][slot] + w.redf[2][slot] + w.redf[3][slot];
  return r;
}

// Shared-memory row of N floats into registers: 128-bit loads where the
// rows are 16-byte aligned (N a multiple of 4; the arrays are 16-byte
// aligned), else 32-bit loads.
template <int N>
__device__ __forceinline__ void ld_row(const float *src, float (&dst)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 v = reinterpret_cast<const float4 *>(src)[q];
      dst[4 * q] = v.x;
      dst[4 * q + 1] = v.y;
      dst[4 * q + 2] = v.z;
      dst[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) dst[j] = src[j];
  }
}

// 1 / x, correctly rounded (the same value as the IEEE division)
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Unwhitened basis Psi at one sample (compile-time bound NM, runtime nm).
template <class Real, int DMAX, int NM, class S>
__device__ __forceinline__ void eval_psi(const S &w, int d, int nm, float x0, float x1, float x2,
                                         Real (&psi)[NM]) {
  Real Q[3][kMaxDeg + 1];
  const float xv[3] = {x0, x1, x2};
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    Real pw[kMaxDeg + 1];
    if constexpr (sizeof(Real) == 4) {
      const float4 c = *reinterpret_cast<const float4 *>(&w.vc[v][0]);   // sc, of, mu, isg
      const float xn = fmaf(xv[v], c.x, c.y);
      pw[1] = (xn - c.z) * c.w;
    } else {
      const Real xn = fma((Real)xv[v], w.sc_v[v], w.of_v[v]);
      pw[1] = (xn - w.mu_v[v]) * w.isg_v[v];
    }
    pw[0] = 1;
#pragma unroll
    for (int l = 2; l <= DMAX; ++l) pw[l] = pw[l - 1] * pw[1];
    // Q_k = sum_{l <= k} Tm[l][k] u^l, summed over l ascending
    Real s[kMaxDeg + 1];
#pragma unroll
    for (int k = 0; k <= DMAX; ++k) s[k] = 0;
#pragma unroll
    for (int l = 0; l <= DMAX; ++l) {
      Real t[8];
      if constexpr (sizeof(Real) == 4) {
        ld_row<(DMAX >= 4 ? 8 : 4)>(&w.Tm[v][l][0], reinterpret_cast<float (&)[(DMAX >= 4 ? 8 : 4)]>(t));
      } else {
#pragma unroll
        for (int k = 0; k <= DMAX; ++k) t[k] = w.Tm[v][l][k];
      }
#pragma unroll
      for (int k = l; k <= DMAX; ++k) s[k] = fma(t[k], pw[l], s[k]);
    }
#pragma unroll
    for (int k = 0; k <= DMAX; ++k) Q[v][k] = (k <= d) ? s[k] : (Real)0;
  }
  // graded-lex order (degree s ascending, exponent a of N descending, b of
  // B0 descending) with compile-time exponents: Q stays in registers
  int j = 0;
#pragma unroll
  for (int s = 0; s <= DMAX; ++s)
#pragma unroll
    for (int a = s; a >= 0; --a)
#pragma unroll
      for (int b = s - a; b >= 0; --b, ++j)
        psi[j] = (j < nm) ? Q[0][a] * Q[1][b] * Q[2][s - a - b] : (Real)0;
}

// Whitened basis: pt[0] = 1, pt[j] = sum_{1<=i<=j} (Psi_i - mean_i) W[i][j].
// W is zero below the diagonal, so each row is read from the aligned 4-block
// holding the diagonal on (128-bit loads on the FP32 path).
template <class Real, int NM, int WS, class S>
__device__ __forceinline__ void whiten(const S &w, const Real (&psi)[NM], Real (&pt)[NM]) {
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

// t-th 4x4 tile of the lower triangle (row-major): rb >= cb
__device__ __forceinline__ void tile_of(int t, int &rb, int &cb) {
  int r = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  rb = r;
  cb = t - r * (r + 1) / 2;
}

// Gram of `cols` columns of the staged rows: work item = (4x4 tile, sample
// group); each thread holds up to IPT items.  Chunk partials are summed
// into the per-item accumulators (blocked summation).
template <class Real, int IPT, int LDS>
struct TileGram {
  Real acc[IPT][16];
  int ntiles, groups;

  __device__ void init(int cols) {
    const int side = (cols + 3) / 4;
    ntiles = side * (side + 1) / 2;
    groups = max(1, kT / ntiles);
#pragma unroll
    for (int k = 0; k < IPT; ++k)
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[k][i] = 0;
  }

  __device__ void chunk(const Real *stage, int cnt) {
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int item = threadIdx.x + kT * k;
      if (item >= ntiles * groups) break;
      const int tile = item % ntiles, g = item / ntiles;
      int rb, cb;
      tile_of(tile, rb, cb);
      Real part[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) part[i] = 0;
#pragma unroll 2
      for (int s = g; s < cnt; s += groups) {
        Real av[4], bv[4];
        if constexpr (sizeof(Real) == 4) {
          const float4 va = *reinterpret_cast<const float4 *>(stage + s * LDS + 4 * rb);
          const float4 vb = *reinterpret_cast<const float4 *>(stage + s * LDS + 4 * cb);
          av[0] = va.x; av[1] = va.y; av[2] = va.z; av[3] = va.w;
          bv[0] = vb.x; bv[1] = vb.y; bv[2] = vb.z; bv[3] = vb.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            av[i] = stage[s * LDS + 4 * rb + i];
            bv[i] = stage[s * LDS + 4 * cb + i];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) part[4 * i + j] = fma(av[i], bv[j], part[4 * i + j]);
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[k][i] += part[i];
    }
  }

  // The same Gram of FP64 rows staged as head + tail FP32 pairs (split_d):
  // products and per-chunk sums in double-float arithmetic (Dot2) on the
  // FP32 pipe, chunk totals added in FP64.  Used by the FP64 launch that
  // re-fits the fits an FP32 / tensor-core launch passed on: it is
  // accurate to ~1e-14 relative, like the FP64 sums, at a fraction of the
  // FP64 pipe's time.
  __device__ void chunk_split(const Real *stage, int cnt) {
    static_assert(sizeof(Real) == 8, "FP64 rows only");
    const float2 *st2 = reinterpret_cast<const float2 *>(stage);
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int item = threadIdx.x + kT * k;
      if (item >= ntiles * groups) break;
      const int tile = item % ntiles, g = item / ntiles;
      int rb, cb;
      tile_of(tile, rb, cb);
      dacc part[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) part[i] = dacc{0.0f, 0.0f};
      for (int s = g; s < cnt; s += groups) {
        const float4 *pa = reinterpret_cast<const float4 *>(st2 + s * LDS + 4 * rb);
        const float4 *pb = reinterpret_cast<const float4 *>(st2 + s * LDS + 4 * cb);
        const float4 a01 = pa[0], a23 = pa[1], b01 = pb[0], b23 = pb[1];
        const dfl av[4] = {{a01.x, a01.y}, {a01.z, a01.w}, {a23.x, a23.y}, {a23.z, a23.w}};
        const dfl bv[4] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) dacc_fma(part[4 * i + j], av[i], bv[j]);
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[k][i] += (double)part[i].s + (double)part[i].c;
    }
  }

  // Sum the sample groups and write the symmetric cols x cols Gram into G
  // (stride cols).  `scratch` needs ntiles * groups * 16 entries.
  __device__ void finish(int cols, Real *G, Real *scratch) {
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int item = threadIdx.x + kT * k;
      if (item < ntiles * groups)
#pragma unroll
        for (int i = 0; i < 16; ++i) scratch[(size_t)item * 16 + i] = acc[k][i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ntiles * 16; e += kT) {
      const int tile = e / 16, q = e % 16;
      int rb, cb;
      tile_of(tile, rb, cb);
      const int r = 4 * rb + q / 4, c = 4 * cb + q % 4;
      Real sum = 0;
      for (int g = 0; g < groups; ++g) sum += scratch[((size_t)g * ntiles + tile) * 16 + q];
      if (r < cols && c < cols) {
        G[r * cols + c] = sum;
        G[c * cols + r] = sum;
      }
    }
    __syncthreads();
  }
};

// One entry of a staged row: the value, or (FP64 rows for chunk_split) its
// head + tail FP32 pair in the same 8 bytes.
template <class Real>
__device__ __forceinline__ void stage_put(Real *row, int j, Real v, bool split) {
  if constexpr (sizeof(Real) == 8) {
    if (split) {
      const dfl p = split_d(v);
      reinterpret_cast<float2 *>(row)[j] = make_float2(p.h, p.l);
      return;
    }
  }
  row[j] = v;
}

// Warp reduce-scatter of V values per lane (V a multiple of 16): four
// halving exchanges (offsets 16, 8, 4, 2) and one full exchange (offset 1).
// Afterwards lane l holds, in v[0 .. V/16), the warp totals of the original
// indices rs_base<V>(l) + q (lanes l and l ^ 1 hold the same totals).
template <int V>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[V]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int o = 16 >> step;
    const int half = V >> (step + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float send = up ? v[j] : v[j + half];
      const float keep = up ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int j = 0; j < V / 16; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1);
}
template <int V>
__device__ __forceinline__ int rs_base(int lane) {
  return ((lane >> 4) & 1) * (V / 2) + ((lane >> 3) & 1) * (V / 4) + ((lane >> 2) & 1) * (V / 8) +
         ((lane >> 1) & 1) * (V / 16);
}

// x += dx in head + tail form (FP32 pairs carrying ~46 bits)
__device__ __forceinline__ void df_add(float &h, float &l, float d) {
  float s, e;
  two_sum(h, d, s, e);
  const float t = l + e;
  h = s + t;
  l = t - (h - s);
}

// Apply the design-basis step dxw (n entries: numerator 0..nm-1, denominator
// 1..nm-1 at nm..2nm-2) to the fitted function: with u = W x_num and
// v = W x_den on the non-constant basis functions, du = W dx_num,
// dv = W dx_den, dc_p = dx_num_0 - mu.du, dc_q = -mu.dv.  The iterate
// (c_p, u), (c_q, v) is kept in FP64 (FP64 path) or as FP32 head + tail
// pairs (FP32 paths); dxw itself is FP32 there.  Returns ||dx|| / ||x||
// for the updated x (block-wide; contains barriers).
template <class Real, int NM, int WS, class S>
__device__ float apply_step(S &w, int nm, int n) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < 2 * NM; e += kT) {
    const int which = e / NM, i = e % NM;
    Real acc = 0;
    if (i >= 1 && i < nm)
      for (int j = i; j < nm; ++j)
        acc = fma(w.W[i * WS + j], which == 0 ? w.dxw[j] : w.dxw[nm + j - 1], acc);
    w.duv[which][i] = acc;
  }
  __syncthreads();
  if (wid < 2) {
    Real c = 0;
    for (int i = 1 + lane; i < nm; i += 32) c = fma(-w.mupsi[i], w.duv[wid][i], c);
    c = warp_sum(c);
    if (lane == 0) w.duv[wid][0] = c + (wid == 0 ? w.dxw[0] : (Real)0);
  } else if (wid == 2) {
    // norms of the step and of the updated iterate
    float dn = 0.0f, xn = 0.0f;
    for (int j = lane; j < n; j += 32) {
      const Real xv = w.xw[j] + w.dxw[j];
      w.xw[j] = xv;
      dn += (float)(w.dxw[j] * w.dxw[j]);
      xn += (float)(xv * xv);
    }
    dn = warp_sum(dn);
    xn = warp_sum(xn);
    if (lane == 0) w.fscal[0] = xn > 0.0f ? sqrtf(dn / xn) : 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < 2 * NM; e += kT) {
    const int which = e / NM, i = e % NM;
    if (sizeof(Real) == 8) {
      w.uv[which][i] += (double)w.duv[which][i];
    } else {
      df_add(w.uvhi[which][i], w.uvlo[which][i], (float)w.duv[which][i]);
    }
  }
  __syncthreads();
  return w.fscal[0];
}

// Accurate refinement pass of the FP32 paths (double-float arithmetic).
// Every thread takes one sample of a 128-sample chunk (row phase):
//   basis variable t_v = (x_v sc_v + of_v - mu_v) isg_v as a pair (the exact
//   affine map of the FP32 constants that define the basis),
//   Q_k(t_v) = sum_l Tm[l][k] t_v^l, Psi_j = Q_a Q_b Q_c (pairs),
//   p = c_p + Psi.u, q = c_q + Psi.v (compensated dot products against the
//   head + tail iterate), r = w (y q - p), a = w r, b = w y r (pairs),
// and stages its row: the pairs (head, tail) of Psi_0.. interleaved, then a
// and b at DF_AO (16-byte stores; the row stride is an odd multiple of 16
// bytes, so 8 consecutive rows fill distinct banks).  Then thread (column,
// group) adds a Psi_j (H_j), b Psi_j (K_j) and, on the first accurate pass,
// Psi_j (the basis sums, for the exact sample means) over the group's rows
// with Dot2 (column phase; 64-bit loads of the pairs).  Results: hkd[0..2][j]
// (pairs, block totals), the objective sum r^2 and whether q <= 0 at some
// sample.
// slab (or null): this CTA's basis cache, float4 q (pairs 2q, 2q + 1) of
// sample i at q kCacheSamples + i (a warp's accesses are consecutive
// 16-byte words).  The basis pairs depend only on
// the point set's samples and basis (degree D, the set's largest), not on
// the fit: the first accurate pass of a claim computes them and writes them
// there (slab_full false), the claim's later accurate passes read them back
// (slab_full true).  Both give the same values; a fit of degree d < D uses
// the leading nm of them.
template <int DMAX, int NM, class S>
__device__ void df_pass(S &w, int d, int nm, int m, bool weighted, bool first, const float *sx0,
                        const float *sx1, const float *sx2, const float *sy, float &obj_out,
                        int &pole_out, float4 *slab, bool slab_full, int D) {
  constexpr int NP4 = (NM + 1) / 2;   // float4 of the slab per sample (two pairs each)
  constexpr int LDD = S::DF_LDD, AO = S::DF_AO;
  static_assert(AO % 4 == 0 && LDD % 4 == 0 && AO + 4 <= LDD && 2 * NM <= AO, "accurate pass rows");
  const int tid = threadIdx.x;
  float *stage = reinterpret_cast<float *>(w.stage);
  // the iterate as interleaved pairs (one 64-bit broadcast load per term)
  for (int e = tid; e < 2 * NM; e += kT) {
    const int which = e / NM, i2 = e % NM;
    w.uvq[which][i2] = make_float2(w.uvhi[which][i2], w.uvlo[which][i2]);
  }
  __syncthreads();
  const int ncol = (first ? 3 : 2) * nm;
  const int groups = max(1, kT / ncol);
  const int col = tid % ncol, grp = tid / ncol;
  const int which = col / nm, jc = col % nm;
  const bool colw = tid < groups * ncol;
  const int wo = which == 2 ? 0 : AO + 2 * which;   // weight pair of the column
  dacc ca = {0.0f, 0.0f}, cb = {0.0f, 0.0f};        // two chains (alternate rows)
  dacc objacc = {0.0f, 0.0f};   // the objective, compensated (its changes near
                                // convergence are far below FP32 summation noise)
  int pole = 0;
  for (int base = 0; base < m; base += kT) {
    const int cnt = min(kT, m - base);
    if (tid < cnt) {
      const int i = base + tid;
      const float yy = sy[i];
      float *row = stage + tid * LDD;
      dacc P = {0.0f, 0.0f}, Qs = {0.0f, 0.0f};
      if (slab && slab_full) {
        // the sample's basis pairs from the slab
#pragma unroll
        for (int q4 = 0; q4 < NP4; ++q4) {
          float4 v4 = __ldcg(slab + (size_t)q4 * kCacheSamples + i);   // L2 only
          const int j0 = 2 * q4, j1 = 2 * q4 + 1;
          if (j0 >= nm) v4.x = v4.y = 0.0f;
          if (j1 >= nm) v4.z = v4.w = 0.0f;
          *reinterpret_cast<float4 *>(row + 4 * q4) = v4;
          {
            const float2 u = w.uvq[0][j0], v = w.uvq[1][j0];
            dacc_fma(P, dfl{u.x, u.y}, dfl{v4.x, v4.y});
            dacc_fma(Qs, dfl{v.x, v.y}, dfl{v4.x, v4.y});
          }
          if (j1 < NM) {
            const float2 u = w.uvq[0][j1], v = w.uvq[1][j1];
            dacc_fma(P, dfl{u.x, u.y}, dfl{v4.z, v4.w});
            dacc_fma(Qs, dfl{v.x, v.y}, dfl{v4.z, v4.w});
          }
        }
      } else {
      const float xv[3] = {sx0[i], sx1[i], sx2[i]};
      dfl Q[3][DMAX + 1];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const float4 c = *reinterpret_cast<const float4 *>(&w.vc[v][0]);   // sc, of, mu, isg
        const float ph = __fmul_rn(xv[v], c.x);
        const float pl = fmaf(xv[v], c.x, -ph);
        float s1, e1, s2, e2;
        two_sum(ph, c.y, s1, e1);
        two_sum(s1, -c.z, s2, e2);
        const dfl t = df_mulf(df_norm(s2, e2 + (e1 + pl)), c.w);
        dfl pw[DMAX + 1];
        pw[1] = t;
#pragma unroll
        for (int l = 2; l <= DMAX; ++l) pw[l] = df_mul(pw[l - 1], t);
        Q[v][0] = df_make(1.0f);
#pragma unroll
        for (int k = 1; k <= DMAX; ++k) {
          dfl sk = df_make(w.Tm[v][0][k]);
#pragma unroll
          for (int l = 1; l <= k; ++l) sk = df_add(sk, df_mulf(pw[l], w.Tm[v][l][k]));
          Q[v][k] = (k <= D) ? sk : df_make(0.0f);
        }
      }
      const int nmD = num_monomials(D);
      float2 prev = make_float2(0.0f, 0.0f), prevs = prev;
      int j = 0;
#pragma unroll
      for (int sd = 0; sd <= DMAX; ++sd)
#pragma unroll
        for (int ea = sd; ea >= 0; --ea)
#pragma unroll
          for (int eb = sd - ea; eb >= 0; --eb, ++j) {
            const int ec = sd - ea - eb;
            dfl ps = df_make(1.0f);
            if (ea) ps = Q[0][ea];
            if (eb) ps = ea ? df_mul(ps, Q[1][eb]) : Q[1][eb];
            if (ec) ps = (ea || eb) ? df_mul(ps, Q[2][ec]) : Q[2][ec];
            // the set's basis (degree D) to the slab, the fit's (degree d) here
            const dfl pss = j < nmD ? ps : df_make(0.0f);
            if (j >= nm) ps = df_make(0.0f);
            if (j & 1) {
              *reinterpret_cast<float4 *>(row + 2 * (j - 1)) = make_float4(prev.x, prev.y, ps.h, ps.l);
              if (slab) __stcg(slab + (size_t)(j >> 1) * kCacheSamples + i, make_float4(prevs.x, prevs.y, pss.h, pss.l));
            } else {
              prev = make_float2(ps.h, ps.l);
              prevs = make_float2(pss.h, pss.l);
            }
            const float2 u = w.uvq[0][j], v = w.uvq[1][j];
            dacc_fma(P, dfl{u.x, u.y}, ps);
            dacc_fma(Qs, dfl{v.x, v.y}, ps);
          }
      if (NM & 1) {
        *reinterpret_cast<float4 *>(row + 2 * (NM - 1)) = make_float4(prev.x, prev.y, 0.0f, 0.0f);
        if (slab) __stcg(slab + (size_t)(NP4 - 1) * kCacheSamples + i, make_float4(prevs.x, prevs.y, 0.0f, 0.0f));
      }
      }   // basis pairs
      const dfl pv = dacc_get(P), qv = dacc_get(Qs);
      pole |= !(qv.h > 0.0f);
      const dfl e = df_add(df_mulf(qv, yy), df_neg(pv));
      dfl ra, rb, r;
      if (weighted) {   // y > 0 here; w = 1 / y, so w y = 1
        const dfl wt = df_recip(df_make(yy));
        r = df_mul(wt, e);
        ra = df_mul(wt, r);
        rb = r;
      } else {
        r = e;
        ra = e;
        rb = df_mulf(e, yy);
      }
      dacc_fma(objacc, r, r);
      *reinterpret_cast<float4 *>(row + AO) = make_float4(ra.h, ra.l, rb.h, rb.l);
    }
    __syncthreads();
    if (colw) {
      auto term = [&](dacc &acc, int s2) {
        const float *rw = stage + s2 * LDD;
        const float2 ps = *reinterpret_cast<const float2 *>(rw + 2 * jc);
        const float2 wt = which == 2 ? make_float2(1.0f, 0.0f) : *reinterpret_cast<const float2 *>(rw + wo);
        dacc_fma(acc, dfl{wt.x, wt.y}, dfl{ps.x, ps.y});
      };
      int s2 = grp;
      for (; s2 + groups < cnt; s2 += 2 * groups) {
        term(ca, s2);
        term(cb, s2 + groups);
      }
      if (s2 < cnt) term(ca, s2);
    }
    __syncthreads();
  }
  // group partials -> block totals (pairs)
  if (colw) {
    const dfl t = df_add(dacc_get(ca), dacc_get(cb));
    stage[2 * tid] = t.h;
    stage[2 * tid + 1] = t.l;
  }
  __syncthreads();
  if (tid < ncol) {
    dfl t = dfl{stage[2 * tid], stage[2 * tid + 1]};
    for (int g = 1; g < groups; ++g) t = df_add(t, dfl{stage[2 * (g * ncol + tid)], stage[2 * (g * ncol + tid) + 1]});
    w.hkd[which][jc][0] = t.h;
    w.hkd[which][jc][1] = t.l;
  }
  pole_out = __syncthreads_or(pole);
  {   // block total of the objective (pairs)
    const int lane = tid & 31, wd = tid >> 5;
    dfl t = dacc_get(objacc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      t = df_add(t, dfl{__shfl_xor_sync(0xffffffffu, t.h, o), __shfl_xor_sync(0xffffffffu, t.l, o)});
    if (lane == 0) {
      w.redf[wd][10] = t.h;
      w.redf[wd][11] = t.l;
    }
    __syncthreads();
    dfl tot = dfl{w.redf[0][10], w.redf[0][11]};
    for (int k = 1; k < kT / 32; ++k) tot = df_add(tot, dfl{w.redf[k][10], w.redf[k][11]});
    obj_out = tot.h;
  }
  __syncthreads();
}

// Tensor-core Gram X^T X of up to NPAD columns over 128-sample chunks: each
// thread stages its sample's row (column j at row j of the K-major tile,
// K slot = the thread), one thread issues the MMAs of the chunk's K-blocks
// and commits them to an mbarrier.  X3: the staged values are split into a
// TF32 head and tail and D accumulates hi.hi + hi.lo + lo.hi.
constexpr uint32_t kTcWaitLimit = 1u << 22;   // mbarrier polls before giving up

template <int NPAD, bool X3, bool BF16 = false>
struct TcGram {
  static constexpr int NB = NPAD / 8 * 1024;   // bytes per K-block (128-byte rows)
  static constexpr int KB = BF16 ? 64 : 32;    // samples per K-block
  static constexpr int NKB = kT / KB;          // K-blocks per 128-sample chunk
  uint32_t base;                               // this thread's K slot
  uint32_t xo[8];                              // swizzled chunk offset per row % 8

  __device__ __forceinline__ void init() {
    const int t = threadIdx.x;
    const int k = t % KB;                      // sample slot within the K-block
    constexpr int es = BF16 ? 2 : 4;
    base = (uint32_t)((t / KB) * NB + (k * es) % 16);
    const int c = (k * es) / 16;
#pragma unroll
    for (int r = 0; r < 8; ++r) xo[r] = (uint32_t)(((c ^ r) & 7) << 4);
  }
  // column j (a compile-time index after unrolling) of this thread's sample
  __device__ __forceinline__ void put(unsigned char *st, int j, float v) const {
    const uint32_t o = base + (uint32_t)((j >> 3) * 1024 + (j & 7) * 128) + xo[j & 7];
    if constexpr (BF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      *reinterpret_cast<__nv_bfloat16 *>(st + o) = h;
      if (X3) *reinterpret_cast<__nv_bfloat16 *>(st + NKB * NB + o) = __float2bfloat16_rn(v - __bfloat162float(h));
    } else {
      float h, l;
      tc::split_tf32(v, h, l);
      *reinterpret_cast<float *>(st + o) = h;
      if (X3) *reinterpret_cast<float *>(st + NKB * NB + o) = l;
    }
  }
  // one thread: D = (first ? 0 : D) + X^T X over nkb K-blocks (each 4 MMAs
  // of K = 32 bytes of the 128-byte rows)
  __device__ static void issue(const unsigned char *st, uint32_t tmem, int nkb, bool first) {
    constexpr uint32_t id = tc::idesc(BF16 ? tc::kFmtBF16 : tc::kFmtTF32, 128, NPAD);
    const uint32_t b = tc::smem_u32(st);
    for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const uint32_t off = (uint32_t)(kb * NB + 32 * s);
        const uint64_t ah = tc::sw128_desc(b + off);
        const uint32_t acc0 = (first && kb == 0 && s == 0) ? 0u : 1u;
        if constexpr (BF16) tc::mma_f16(tmem, ah, ah, id, acc0);
        else tc::mma_tf32(tmem, ah, ah, id, acc0);
        if (X3) {
          const uint64_t al = tc::sw128_desc(b + NKB * NB + off);
          if constexpr (BF16) {
            tc::mma_f16(tmem, ah, al, id, 1u);
            tc::mma_f16(tmem, al, ah, id, 1u);
          } else {
            tc::mma_tf32(tmem, ah, al, id, 1u);
            tc::mma_tf32(tmem, al, ah, id, 1u);
          }
        }
      }
  }
  // Warps holding padded rows < rows copy D into G: padded index j maps to
  // map(j) (< 0: unused), G[map(r) * ld + map(c)].
  template <class Real, class Map>
  __device__ static void read(uint32_t tmem, int rows, Real *G, int ld, Map map) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (32 * wid < rows) {
      const int r = 32 * wid + lane;
      const int rc = r < rows ? map(r) : -1;
#pragma unroll
      for (int c0 = 0; c0 < NPAD; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0, v);
        if (rc >= 0)
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int cc = map(c0 + q);
            if (cc >= 0) G[rc * ld + cc] = (Real)v[q];
          }
      }
    }
    tc::fence_before_sync();
  }
};

// Staged values visible to the tensor core, MMAs of one chunk issued by
// thread 0 and committed, completion awaited by every thread (bounded).
template <class TG>
__device__ __forceinline__ bool tc_chunk(const unsigned char *st, uint32_t tmem, uint64_t *mbar,
                                         int nkb, bool first, uint32_t &phase) {
  tc::fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::fence_after_sync();
    TG::issue(st, tmem, nkb, first);
    tc::mma_commit(mbar);
  }
  const bool ok = tc::mbar_wait(mbar, phase, kTcWaitLimit);
  tc::fence_after_sync();
  const bool all = __syncthreads_and(ok);
  if (all) phase ^= 1u;
  return all;
}

// ---------------------------------------------------------------------
// The fit kernel.  Real = double: plain FP64 path; Real = float: FP32 path.

template <class Real, int DMAX, int GM>
__global__ void __launch_bounds__(kT, (sizeof(Real) == 4 && DMAX <= 3) ? (GM == 2 ? 3 : 4)
                                          : (DMAX <= 3 ? 2 : (sizeof(Real) == 4 && GM == 0 ? 3 : 1)))
    fit_kernel(FitArgs a) {
  using WF = CtaFit<Real, DMAX, GM>;
  using TS = TcShape<DMAX>;
  constexpr int NM = WF::NM;
  constexpr int NAUG = WF::NAUG;
  constexpr int LDS = WF::LDS;
  constexpr int WS = WF::WS;
  constexpr int S4 = (NAUG + 3) / 4;
  constexpr int IPT = ((S4 * (S4 + 1) / 2) + kT - 1) / kT;   // design-Gram items per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the state starts at the first 1024-byte boundary (swizzle atoms of the
  // tensor-core paths; 16-byte alignment suffices otherwise)
  const uint32_t raw_s = tc::smem_u32(smem_raw);
  WF &w = *reinterpret_cast<WF *>(smem_raw + (GM > 0 ? (((raw_s + 1023u) & ~1023u) - raw_s) : 0u));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // the FP64 launch for fits an FP32 / tensor-core launch passed on forms
  // its two Grams in double-float arithmetic (chunk_split)
  const bool split_gram = sizeof(Real) == 8 && a.esc_mode == 2;
  // the FP64 pass over the fits passed on by an FP32 / tensor-core launch:
  // nothing to do when none was (the count is final: same stream, earlier
  // launch)
  if (a.esc_mode == 2 && a.esc_count && *a.esc_count == 0ull) return;
  // tensor memory for the Gram accumulators, held for the whole launch
  uint32_t tmem = 0, tc_phase = 0;
  bool tc_dead = false;
  if constexpr (GM > 0) {
    if (wid == 0) {
      tc::tmem_alloc(&w.tmem_base, TS::TMEM_COLS);
      tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&w.mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem = w.tmem_base;
  }
  // Point sets are claimed from the workspace counter (CTAs that draw large
  // sets take fewer), else every gridDim.x-th set.  A set is the fits that
  // share one block of sample points (fits_per_set consecutive fits with a
  // point_off array, else a single fit with its own points): phases 0-2
  // (box, marginal polynomials, basis Gram and whitening) depend only on
  // the points and run once per set, at the set's largest degree D; a fit
  // of degree d < D uses the leading block of that basis (graded-lex order
  // puts lower total degrees first and every factorisation of phases 1-2 is
  // triangular, so the leading block is the degree-d basis itself).
  // A claim is one of set_parts runs of a set's fits (the host splits sets
  // when there are too few of them to keep every CTA busy to the end; each
  // run repeats phases 0-2).
  const int64_t G = a.point_off ? (int64_t)a.fits_per_set : 1;
  const int64_t nsets = (a.F + G - 1) / G;
  const int64_t parts = a.point_off ? max(a.set_parts, 1) : 1;
  const int64_t run = (G + parts - 1) / parts;
  int64_t unit = blockIdx.x;
  // this CTA's slab of the basis cache (accurate passes of the FP32 paths,
  // point sets of at most MC samples), or null
  float4 *slab = nullptr;
  if constexpr (sizeof(Real) == 4 && WF::MC > 0) {
    static_assert(WF::MC == kCacheSamples, "slab size");
    constexpr size_t kSlabF4 = (size_t)WF::MC * ((NM + 1) / 2);
    if (a.psi_cache && (size_t)(blockIdx.x + 1) * kSlabF4 * sizeof(float4) <= a.psi_cache_bytes)
      slab = a.psi_cache + (size_t)blockIdx.x * kSlabF4;
  }
  for (int claim = 0;; ++claim) {
    bool psi_in_slab = false;   // the slab holds this claim's basis pairs
    if (a.counter) {
      if (tid == 0) w.next_fit[claim & 1] = (long long)atomicAdd(a.counter, 1ull);
      __syncthreads();
      unit = w.next_fit[claim & 1];
    } else if (claim > 0) {
      unit += gridDim.x;
    }
    if (unit >= nsets * parts) break;
    const int64_t ps = unit / parts;
    const int64_t f0 = min(a.F, ps * G + (unit % parts) * run);
    const int64_t f1 = min(min(a.F, ps * G + G), f0 + run);
    // ---------------- phase 0: the set's fits in this launch and its degree
    // (a launch of a split batch takes only its degrees; invalid degrees go
    // to the launch that starts at 1; the others' outputs are not touched)
    if (tid == 0) {
      int D = 0, any = 0;
      for (int64_t f = f0; f < f1; ++f) {
        if (a.esc_mode == 2 && !(a.status[f] & kPending64)) continue;
        const int d = a.degs ? (int)a.degs[f] : a.d_uniform;
        const bool valid_d = d >= 1 && d <= a.d_uniform;
        if (valid_d ? (d < a.deg_lo || d > a.deg_hi) : a.deg_lo > 1) continue;
        any = 1;
        if (valid_d && d <= DMAX) D = max(D, d);
      }
      w.set_deg = any ? D : -1;
    }
    __syncthreads();
    const int D = w.set_deg;
    if (D < 0) continue;
    int64_t xb0, xb1, xS;
    if (a.point_off) {
      xb0 = a.point_off[ps];
      xb1 = a.point_off[ps + 1];
      xS = a.num_points;
    } else {
      xb0 = a.off[ps];
      xb1 = a.off[ps + 1];
      xS = a.S;
    }
    const bool prange_ok = xb0 >= 0 && xb1 >= xb0 && xb1 <= xS;
    const int m = prange_ok ? (int)(xb1 - xb0) : 0;
    const bool cached = m <= WF::MC;
    const float *gx0 = a.x + xb0, *gx1 = a.x + xS + xb0, *gx2 = a.x + 2 * xS + xb0;
    // ---------------- phase 0: range, validation, box, distinct values of the points
    int xbad = 0;
    if (D >= 1 && m > 0) {
      if (tid < 3 * (kMaxDeg + 1)) (&w.dslot[0][0])[tid] = kEmpty;
      if (tid == 0) w.bad = 0;
      __syncthreads();
      float lmin[3] = {INFINITY, INFINITY, INFINITY}, lmax[3] = {-INFINITY, -INFINITY, -INFINITY};
      int bad = 0;
      // loads (unrolled so that several samples' loads are in flight), the
      // sample cache, validity and range; then the distinct values from the
      // cached copy (the set's atomics would otherwise serialise the loads)
#pragma unroll 4
      for (int i = tid; i < m; i += kT) {
        const float v0 = __ldg(gx0 + i), v1 = __ldg(gx1 + i), v2 = __ldg(gx2 + i);
        if (cached) {
          w.xs[0][i] = v0;
          w.xs[1][i] = v1;
          w.xs[2][i] = v2;
        }
        if (!(isfinite(v0) && isfinite(v1) && isfinite(v2))) bad = 1;
        lmin[0] = fminf(lmin[0], v0); lmax[0] = fmaxf(lmax[0], v0);
        lmin[1] = fminf(lmin[1], v1); lmax[1] = fmaxf(lmax[1], v1);
        lmin[2] = fminf(lmin[2], v2); lmax[2] = fmaxf(lmax[2], v2);
      }
      for (int i = tid; i < m; i += kT) {
        distinct_insert(w.dslot[0], cached ? w.xs[0][i] : gx0[i]);
        distinct_insert(w.dslot[1], cached ? w.xs[1][i] : gx1[i]);
        distinct_insert(w.dslot[2], cached ? w.xs[2][i] : gx2[i]);
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
      if (lane == 0) {
        for (int v = 0; v < 3; ++v) {
          w.redf[wid][v] = lmin[v];
          w.redf[wid][3 + v] = lmax[v];
        }
        if (bad) atomicOr(&w.bad, bad);
      }
      __syncthreads();
      xbad = w.bad;
      if (!xbad && tid < 3) {
        double mn = w.redf[0][tid], mx = w.redf[0][3 + tid];
        for (int k = 1; k < 4; ++k) {
          mn = fmin(mn, (double)w.redf[k][tid]);
          mx = fmax(mx, (double)w.redf[k][3 + tid]);
        }
        w.lo[tid] = mn;
        w.hi[tid] = mx;
        if (mx > mn) {   // x' = 2 (x - lo) / (hi - lo) - 1 = x * sc + of
          // in Real: the FP32 paths normalise in FP32, so FP32 sc and of (a
          // consistent normalisation; lo and hi are kept exactly)
          const Real sc = (Real)2 / (Real)(mx - mn);
          w.sc_v[tid] = sc;
          w.of_v[tid] = fma(-(Real)mn, sc, (Real)-1);
        } else {
          w.sc_v[tid] = 0;
          w.of_v[tid] = 0;
        }
      }
      __syncthreads();
    }
    const bool basis_ok = D >= 1 && m > 0 && !xbad;
    const float *sx0 = cached ? w.xs[0] : gx0;
    const float *sx1 = cached ? w.xs[1] : gx1;
    const float *sx2 = cached ? w.xs[2] : gx2;
    if (basis_ok) {
    const int d = D;                       // phases 1-2: the set's degree
    const int nm = num_monomials(d);
    const int nc = nm - 1;

    // ---------------- phase 1: standardisation, marginal orthonormal polynomials
    {
      Real acc[3] = {0, 0, 0};
      for (int i = tid; i < m; i += kT) {
        acc[0] += fma((Real)sx0[i], w.sc_v[0], w.of_v[0]);
        acc[1] += fma((Real)sx1[i], w.sc_v[1], w.of_v[1]);
        acc[2] += fma((Real)sx2[i], w.sc_v[2], w.of_v[2]);
      }
      // sums and moments in Real (FP32 on the FP32 paths: they only choose
      // the per-fit basis, which is used consistently; FP64 divisions at
      // GB300's FP64 rate would cost more than the whole phase)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const Real sv = warp_sum(acc[v]);
        if (lane == 0) w.redr[wid][v] = sv;
      }
      __syncthreads();
      const Real inv_m = (Real)1 / (Real)m;
      Real mu[3];
#pragma unroll
      for (int v = 0; v < 3; ++v)
        mu[v] = (w.redr[0][v] + w.redr[1][v] + w.redr[2][v] + w.redr[3][v]) * inv_m;
      Real mom[3][2 * DMAX];
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < 2 * DMAX; ++k) mom[v][k] = 0;
      for (int i = tid; i < m; i += kT) {
        const float xv[3] = {sx0[i], sx1[i], sx2[i]};
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
      // (slots 3.. : the means' slots 0..2 may still be being read)
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = 0; k < 2 * DMAX; ++k) {
          const Real sv = warp_sum(mom[v][k]);
          if (lane == 0) w.redr[wid][3 + v * 2 * DMAX + k] = sv;
        }
      __syncthreads();
      if (tid < 3) {
        const int v = tid;
        Real M[2 * kMaxDeg + 1];
        M[0] = 1;
        for (int k = 0; k < 2 * DMAX; ++k) {
          const int o = 3 + v * 2 * DMAX + k;
          M[k + 1] = (w.redr[0][o] + w.redr[1][o] + w.redr[2][o] + w.redr[3][o]) * inv_m;
        }
        const Real var = M[2];
        w.mu_v[v] = mu[v];
        for (int l = 0; l <= kMaxDeg; ++l)
          for (int k = 0; k <= kMaxDeg; ++k) w.Tm[v][l][k] = (l == 0 && k == 0) ? (Real)1 : (Real)0;
        if (w.sc_v[v] == (Real)0 || !(var > (Real)0)) {
          w.isg_v[v] = 0;
        } else {
          const Real isg = rsqrt_pos<Real>(var);
          w.isg_v[v] = isg;
          float Ms[2 * kMaxDeg + 1];
          Ms[0] = 1.0f;
          Real pw = isg;
          for (int k = 1; k <= 2 * DMAX; ++k) {
            Ms[k] = (float)(M[k] * pw);
            pw *= isg;
          }
          int cnt = 0;
          for (int k = 0; k <= kMaxDeg; ++k) cnt += w.dslot[v][k] != kEmpty;
          float T[kMaxDeg + 1][kMaxDeg + 1];
          marginal_transform(Ms, d, min(d, cnt - 1), T);
          for (int l = 0; l <= kMaxDeg; ++l)
            for (int k = 0; k <= kMaxDeg; ++k) w.Tm[v][l][k] = (Real)T[l][k];
        }
        w.vc[v][0] = w.sc_v[v];
        w.vc[v][1] = w.of_v[v];
        w.vc[v][2] = w.mu_v[v];
        w.vc[v][3] = w.isg_v[v];
      }
      __syncthreads();
    }

    // ---------------- phase 2: Gram of Psi (nm columns), means, whitening
    {
      TileGram<Real, IPT, LDS> tg;
      tg.init(nm);
      const int cols4 = 4 * ((nm + 3) / 4);
      for (int base = 0; base < m; base += kT) {
        const int cnt = min(kT, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[NM];
          eval_psi<Real, DMAX, NM>(w, d, nm, sx0[i], sx1[i], sx2[i], psi);
          Real *row = w.stage + tid * LDS;
#pragma unroll
          for (int j = 0; j < NM; ++j) stage_put(row, j, psi[j], split_gram);
          for (int j = NM; j < cols4; ++j) row[j] = 0;
        }
        __syncthreads();
        if constexpr (sizeof(Real) == 8) {
          if (split_gram) tg.chunk_split(w.stage, cnt);
          else tg.chunk(w.stage, cnt);
        } else {
          tg.chunk(w.stage, cnt);
        }
        __syncthreads();
      }
      tg.finish(nm, w.G, w.stage);

      // means (row 0 holds the sums of Psi_j), the centred Gram / m of the
      // non-constant functions, equilibrated, in `stage`
      for (int j = tid; j < NM; j += kT) {
        w.mupsi[j] = (j < nm) ? w.G[j] / (Real)m : (Real)0;
        w.mulo[j] = 0.0f;   // tails of the exact means: none known yet
      }
      for (int e = tid; e < NM * WS; e += kT) w.W[e] = 0;
      __syncthreads();
      // the centred Gram / m of the non-constant functions, equilibrated, in
      // `stage`; its Cholesky factor (block-wide); R^-1 (R = L^T) column by
      // column into G; W = D R^-1.  The whitening only preconditions: any
      // positive pivot is kept (the basis stays a basis of the same space);
      // only directions whose pivot is at rounding level or below are dropped.
      for (int e = tid; e < nc * nc; e += kT) {
        const int i = e / nc + 1, j = e % nc + 1;
        w.stage[e] = (w.G[i * nm + j] - (Real)m * w.mupsi[i] * w.mupsi[j]) / (Real)m;
      }
      __syncthreads();
      for (int j = tid; j < nc; j += kT) {
        const Real dg = w.stage[j * nc + j];
        w.scl[j] = dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0;
      }
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kT) w.stage[e] *= w.scl[e / nc] * w.scl[e % nc];
      __syncthreads();
      cta_chol<Real, kT>(w.stage, nc, nc, sizeof(Real) == 8 ? (Real)1e-14 : (Real)1e-10, w.invw,
                         &w.keep_w);
      for (int j = tid; j < nc; j += kT)
        for (int i = j; i >= 0; --i) {
          Real s = (i == j) ? (Real)1 : (Real)0;
          for (int l = i + 1; l <= j; ++l) s -= w.stage[l * nc + i] * w.G[l * nc + j];
          w.G[i * nc + j] = s * w.invw[i];
        }
      __syncthreads();
      for (int e = tid; e < nc * nc; e += kT) {
        const int i = e / nc, j = e % nc;
        if (i <= j) w.W[(i + 1) * WS + (j + 1)] = w.G[i * nc + j] * w.scl[i];
      }
      __syncthreads();
    }

    }   // phases 1-2

    // ---------------- each fit of the set: its values, then phases 3-6
    int mu_known = 0;   // basis functions [0, mu_known) have exact sample means
    for (int64_t f = f0; f < f1; ++f) {
    if (a.esc_mode == 2) {
      const bool pend = (a.status[f] & kPending64) != 0;
      __syncthreads();   // every thread has read status[f] before it is rewritten
      if (!pend) continue;
    }
    const int d = a.degs ? (int)a.degs[f] : a.d_uniform;
    const bool valid_d = d >= 1 && d <= a.d_uniform;
    if (valid_d ? (d < a.deg_lo || d > a.deg_hi) : a.deg_lo > 1) continue;
    double *cf = a.coef + f * kStride;
    for (int j = tid; j < kStride; j += kT) {
      cf[j] = 0.0;
      if (a.coef32) a.coef32[f * kStride + j] = 0.0f;
    }
    if (tid < 6) a.box[f * 6 + tid] = 0.0;
    // the fit's values, one per point of its set
    const int64_t yb0 = a.off[f], yb1 = a.off[f + 1];
    const bool yrange_ok = yb0 >= 0 && yb1 >= yb0 && yb1 <= a.S && yb1 - yb0 == (int64_t)m;
    if (d < 1 || d > DMAX || m == 0 || !yrange_ok) {
      if (tid == 0) {
        a.status[f] = RP_FIT_EMPTY;
        a.rank[f] = 0;
      }
      continue;
    }
    if (xbad) {
      if (tid == 0) {
        a.status[f] = RP_FIT_NONFINITE;
        a.rank[f] = 0;
      }
      continue;
    }
    // ---------------- phase 0 (values): load, cache, validate
    const float *gy = a.y + yb0;
    if (tid == 0) w.bad = 0;
    __syncthreads();
    {
      int bad = 0;
#pragma unroll 4
      for (int i = tid; i < m; i += kT) {
        const float yy = __ldg(gy + i);
        if (cached) w.xs[3][i] = yy;
        if (!isfinite(yy)) bad |= RP_FIT_NONFINITE;
        else if (a.weighted && !(yy > 0.0f)) bad |= RP_FIT_NONPOS_Y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
      if (lane == 0 && bad) atomicOr(&w.bad, bad);
    }
    __syncthreads();
    if (w.bad) {
      if (tid == 0) {
        a.status[f] = (w.bad & RP_FIT_NONFINITE) ? RP_FIT_NONFINITE : RP_FIT_NONPOS_Y;
        a.rank[f] = 0;
      }
      __syncthreads();
      continue;
    }
    if (tid < 3) {
      a.box[f * 6 + 2 * tid] = w.lo[tid];
      a.box[f * 6 + 2 * tid + 1] = w.hi[tid];
    }
    const float *sy = cached ? w.xs[3] : gy;
    const int nm = num_monomials(d);
    const int naug = 2 * nm;
    const int n = naug - 1;

    // Phases 3-5, attempted first with the tensor-core design Gram (GM > 0)
    // and, for a fit whose refinement stops short of its tolerance or whose
    // factorisation drops pivots there, again with the FP32 Gram on CUDA
    // cores (the low-precision Gram was too coarse to precondition it).
    int flags = 0;
    bool escalated = false;
    for (int attempt = 0;; ++attempt) {
    const bool use_tc = GM > 0 && attempt == 0;
    // ---------------- phase 3: the design Gram [num (nm) | den (nm-1) | rhs]
    if (use_tc) {
      if constexpr (GM > 0) {
      // staged in the padded layout num [0, NM), den [NM, 2 NM - 1), rhs
      // 2 NM - 1 (compile-time columns); read back compacted to stride naug
      using TG = TcGram<TS::NDES, WF::TC_X3, (GM == 3 || GM == 4)>;
      TG tg;
      tg.init();
      unsigned char *st = reinterpret_cast<unsigned char *>(w.stage);
      for (int base = 0; base < m && !tc_dead; base += kT) {
        const int cnt = min(kT, m - base);
        const int nkb = (cnt + TG::KB - 1) / TG::KB;
        if (tid < nkb * TG::KB) {
          Real pt[NM];
          Real wt = 0, yy = 0;
          if (tid < cnt) {
            const int i = base + tid;
            Real psi[NM];
            eval_psi<Real, DMAX, NM>(w, d, nm, sx0[i], sx1[i], sx2[i], psi);
            whiten<Real, NM, WS>(w, psi, pt);
            yy = (Real)sy[i];
            wt = a.weighted ? recip(fabs(yy)) : (Real)1;
          } else {
#pragma unroll
            for (int j = 0; j < NM; ++j) pt[j] = 0;
          }
#pragma unroll
          for (int j = 0; j < NM; ++j) tg.put(st, j, j < nm ? (float)(wt * pt[j]) : 0.0f);
#pragma unroll
          for (int j = 1; j < NM; ++j) tg.put(st, NM + j - 1, j < nm ? (float)(-wt * yy * pt[j]) : 0.0f);
          tg.put(st, 2 * NM - 1, (float)(wt * yy));
#pragma unroll
          for (int j = 2 * NM; j < TS::NDES; ++j) tg.put(st, j, 0.0f);
        }
        tc_dead = !tc_chunk<TG>(st, tmem, &w.mbar, nkb, base == 0, tc_phase);
      }
      if (tc_dead) break;
      TG::read(tmem, 2 * NM, w.G, naug, [nm](int j) {
        return j < nm ? j : (j < NM ? -1 : (j < NM + nm - 1 ? nm + (j - NM) : (j == 2 * NM - 1 ? 2 * nm - 1 : -1)));
      });
      __syncthreads();
      }
    } else {
      TileGram<Real, IPT, LDS> tg;
      tg.init(naug);
      const int cols4 = 4 * ((naug + 3) / 4);
      for (int base = 0; base < m; base += kT) {
        const int cnt = min(kT, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[NM], pt[NM];
          eval_psi<Real, DMAX, NM>(w, d, nm, sx0[i], sx1[i], sx2[i], psi);
          whiten<Real, NM, WS>(w, psi, pt);
          const Real yy = (Real)sy[i];
          const Real wt = a.weighted ? recip(fabs(yy)) : (Real)1;
          Real *row = w.stage + tid * LDS;
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < nm) stage_put(row, j, wt * pt[j], split_gram);
#pragma unroll
          for (int j = 1; j < NM; ++j)
            if (j < nm) stage_put(row, nm + j - 1, -wt * yy * pt[j], split_gram);
          stage_put(row, n, wt * yy, split_gram);
          for (int j = naug; j < cols4; ++j) row[j] = 0;
        }
        __syncthreads();
        if constexpr (sizeof(Real) == 8) {
          if (split_gram) tg.chunk_split(w.stage, cnt);
          else tg.chunk(w.stage, cnt);
        } else {
          tg.chunk(w.stage, cnt);
        }
        __syncthreads();
      }
      tg.finish(naug, w.G, w.stage);
    }

    // ---------------- phase 4: equilibrate and sweep
    // S = D G D (D = diag(G_jj^-1/2) on the n normal columns, 1 on the
    // right-hand side), in place in G (stride naug).  Sweeping the pivots
    // 0..n-1 (the sweep operator of least-squares regression: Gauss-Jordan
    // on the SPD normal matrix) leaves -S^-1 in the n x n block and the
    // least-squares solution in column n.  A pivot <= drop_tol (relative to
    // the unit equilibrated diagonal) is not swept: its column is dropped
    // (rank deficiency).  Afterwards G holds Q = D S^-1 D on the kept columns
    // (0 elsewhere), the refinement's preconditioner, and dxw the first step.
    {
      const int N1 = naug;
      for (int j = tid; j < N1; j += kT) {
        const Real dg = w.G[j * N1 + j];
        w.scl[j] = (j == n) ? (Real)1 : (dg > 0 ? rsqrt_pos<Real>(dg) : (Real)0);
      }
      __syncthreads();
      if (!a.svd) {
      if constexpr (DMAX <= 3) {
      // Degree <= 3 (at most 40 columns): thread t holds one chunk of the
      // upper triangle in registers -- row ci, the 8-column block starting
      // at cj0, clipped to columns [max(cj0, ci), N1) -- 120 chunks for 40
      // columns.  Per pivot a thread loads the pivot row's block once and
      // updates its row with one FMA per entry; the pivot's own row and
      // column and the writes of the next pivot row touch few threads.
      constexpr int CW = 8;
      static_assert(NAUG <= 40 && kT >= 120, "one chunk per thread (120 chunks for 40 columns)");
      const int nblk = (N1 + CW - 1) / CW;
      int ci = -1, cj0 = 0;
      {
        int t = tid;
        for (int i = 0; i < N1; ++i) {
          const int nb = nblk - i / CW;
          if (t < nb) {
            ci = i;
            cj0 = (i / CW + t) * CW;
            break;
          }
          t -= nb;
        }
      }
      const bool have = ci >= 0;
      const int jlo = have ? max(cj0, ci) : 0, jhi = have ? min(cj0 + CW, N1) : 0;
      Real v[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const int j = cj0 + c;
        v[c] = (j >= jlo && j < jhi) ? w.G[ci * N1 + j] * w.scl[ci] * w.scl[j] : (Real)0;
        if (ci == 0 && j >= jlo && j < jhi) w.rowb[0][j] = v[c];
      }
      __syncthreads();
      int kept = 0;
      for (int k = 0; k < n; ++k) {
        const Real *rk = w.rowb[k & 1];
        Real *rn = w.rowb[(k + 1) & 1];
        const Real piv = rk[k];
        const bool keep = piv > (Real)a.drop_tol;
        kept += keep;
        if (have) {
          if (keep) {
            const Real ip = recip(piv);
            Real rj[CW];
            if constexpr (sizeof(Real) == 4) {
              ld_row<CW>(rk + cj0, reinterpret_cast<float (&)[CW]>(rj));
            } else {
#pragma unroll
              for (int c = 0; c < CW; ++c) rj[c] = rk[cj0 + c];
            }
            if (ci == k) {
              // the pivot's row: S'_kj = S_kj / p, S'_kk = -1 / p
#pragma unroll
              for (int c = 0; c < CW; ++c) v[c] = (cj0 + c == k) ? -ip : rj[c] * ip;
            } else {
              // S'_ij = S_ij - S_ik S_kj / p; the pivot's column S'_ik = S_ik / p
              const Real rip = rk[ci] * ip;
#pragma unroll
              for (int c = 0; c < CW; ++c) v[c] = fma(-rip, rj[c], v[c]);
              const int ck = k - cj0;
              if (ck >= 0 && ck < CW) {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                  if (c == ck) v[c] = rip;
              }
            }
          }
          // the next pivot row: its entries (k+1, j >= k+1) and (i, k+1), i <= k
          if (ci == k + 1) {
#pragma unroll
            for (int c = 0; c < CW; ++c)
              if (cj0 + c >= jlo && cj0 + c < jhi) rn[cj0 + c] = v[c];
          }
          const int c1 = k + 1 - cj0;
          if (ci <= k && c1 >= 0 && c1 < CW && k + 1 < jhi) {
            Real val = v[0];
#pragma unroll
            for (int c = 1; c < CW; ++c)
              if (c == c1) val = v[c];
            rn[ci] = val;
          }
        }
        if (tid == 0) w.invd[k] = keep ? (Real)1 : (Real)0;
        __syncthreads();
      }
      // Q = -D S D on the kept columns, both triangles; the first step
      if (have) {
        const Real si = w.invd[ci] * w.scl[ci];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int j = cj0 + c;
          if (j < jlo || j >= jhi) continue;
          if (j < n) {
            const Real qv = -v[c] * si * w.invd[j] * w.scl[j];
            w.G[ci * N1 + j] = qv;
            w.G[j * N1 + ci] = qv;
          } else if (j == n && ci < n) {
            w.dxw[ci] = v[c] * si;
          }
        }
      }
      if (tid == 0) w.keep_cnt = kept;
      } else {
      // the upper triangle (i <= j), EPT entries per thread, decoded once
      constexpr int EPT = (NAUG * (NAUG + 1) / 2 + kT - 1) / kT;
      const int ntri = N1 * (N1 + 1) / 2;
      int ent[EPT];   // i << 16 | j, or -1
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + kT * q;
        if (e < ntri) {
          // e = i N1 - i (i - 1) / 2 + (j - i): row i holds N1 - i entries
          int i = (int)((2.0f * N1 + 1.0f - sqrtf((2.0f * N1 + 1.0f) * (2.0f * N1 + 1.0f) - 8.0f * e)) * 0.5f);
          while (i > 0 && i * N1 - i * (i - 1) / 2 > e) --i;
          while ((i + 1) * N1 - (i + 1) * i / 2 <= e) ++i;
          const int j = i + (e - (i * N1 - i * (i - 1) / 2));
          ent[q] = (i << 16) | j;
        } else {
          ent[q] = -1;
        }
      }
      // the entries stay in registers through the elimination; shared memory
      // holds only the pivot rows
      Real v[EPT];
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        v[q] = 0;
        if (ent[q] >= 0) {
          const int i = ent[q] >> 16, j = ent[q] & 0xFFFF;
          v[q] = w.G[i * N1 + j] * w.scl[i] * w.scl[j];
          if (i == 0) w.rowb[0][j] = v[q];
        }
      }
      __syncthreads();
      int kept = 0;
      for (int k = 0; k < n; ++k) {
        const Real *rk = w.rowb[k & 1];
        Real *rn = w.rowb[(k + 1) & 1];
        const Real piv = rk[k];
        const bool keep = piv > (Real)a.drop_tol;
        kept += keep;
        const Real ip = keep ? recip(piv) : (Real)0;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          if (ent[q] < 0) continue;
          const int i = ent[q] >> 16, j = ent[q] & 0xFFFF;
          if (keep) {
            // S'_ij = S_ij - S_ik S_kj / p; S'_ik = S_ik / p; S'_kk = -1 / p
            const Real ri = rk[i], rj = rk[j];
            const Real gen = fma(-ri * ip, rj, v[q]);
            v[q] = (j == k) ? ((i == k) ? -ip : ri * ip) : ((i == k) ? rj * ip : gen);
          }
          if (i == k + 1) rn[j] = v[q];
          if (j == k + 1) rn[i] = v[q];
        }
        if (tid == 0) w.invd[k] = keep ? (Real)1 : (Real)0;
        __syncthreads();
      }
      // Q = -D S D on the kept columns, both triangles; the first step
#pragma unroll
      for (int q = 0; q < EPT; ++q)
        if (ent[q] >= 0) {
          const int i = ent[q] >> 16, j = ent[q] & 0xFFFF;
          const Real si = w.invd[i] * w.scl[i];
          if (j < n) {
            const Real qv = -v[q] * si * w.invd[j] * w.scl[j];
            w.G[i * N1 + j] = qv;
            w.G[j * N1 + i] = qv;
          } else if (j == n && i < n) {
            w.dxw[i] = v[q] * si;
          }
        }
      if (tid == 0) w.keep_cnt = kept;
      }   // degree bound
      } else {
        // The SVD route (the paper's solver, Sec. 4.2): the right singular
        // vectors of the equilibrated design and its squared singular values
        // are the eigenvectors and eigenvalues of S = D G D, found by cyclic
        // Jacobi rotations of S (the rotations Hestenes' one-sided method
        // applies to the design's columns; pairs in round-robin order, the
        // disjoint pairs of a round in parallel); V accumulates them.
        // Directions with an eigenvalue <= drop_tol times the largest are
        // dropped (the SVD's rank); Q = D V L+ V^T D on the kept ones is the
        // refinement's preconditioner and Q times the right-hand-side column
        // the first step (the truncated least-squares solution).
        Real *V = w.stage;                     // n x n, stride n
        for (int e = tid; e < n * n; e += kT) {
          const int i = e / n, j = e % n;
          w.G[i * N1 + j] *= w.scl[i] * w.scl[j];
          V[e] = (i == j) ? (Real)1 : (Real)0;
        }
        const int n2 = n + (n & 1);            // even (one padding index when n is odd)
        const int npair = n2 / 2;
        // a pair is rotated while its coupling exceeds off_tol relative to its
        // diagonal (high relative accuracy) and the rounding level of the
        // unit-diagonal matrix (the sweeps then end in either arithmetic)
        const Real off_tol = sizeof(Real) == 8 ? (Real)1e-15 : (Real)1e-7;
        const Real abs_tol = sizeof(Real) == 8 ? (Real)4e-16 : (Real)2.4e-7;
        // pair i of round r (circle method: n2 - 1 fixed, the others rotate)
        auto pair_of = [n2](int r, int i, int &p, int &q) {
          const int u = i == 0 ? n2 - 1 : (r + i) % (n2 - 1);
          const int v = i == 0 ? r : (r - i + n2 - 1) % (n2 - 1);
          p = min(u, v);
          q = max(u, v);
        };
        for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
          __syncthreads();
          if (tid == 0) w.bad = 0;             // set when a rotation is applied
          __syncthreads();
          for (int r = 0; r < n2 - 1; ++r) {
            for (int i = tid; i < npair; i += kT) {
              int p, q;
              pair_of(r, i, p, q);
              Real c = 1, sn = 0;
              if (q < n) {
                const Real spp = w.G[p * N1 + p], sqq = w.G[q * N1 + q], spq = w.G[p * N1 + q];
                if (fabs(spq) > abs_tol && fabs(spq) > off_tol * sqrt(fabs(spp * sqq))) {
                  // symmetric 2 x 2 Schur decomposition (Golub & Van Loan)
                  const Real zeta = (sqq - spp) / (2 * spq);
                  const Real t = copysign((Real)1, zeta) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                  c = rsqrt_pos<Real>(1 + t * t);
                  sn = c * t;
                  w.bad = 1;
                }
              }
              w.rowb[0][i] = c;
              w.rowb[1][i] = sn;
            }
            __syncthreads();
            // S J and V J: columns p, q of every row
            for (int e = tid; e < npair * n; e += kT) {
              const int i = e / n, k = e % n;
              const Real sn = w.rowb[1][i];
              if (sn == (Real)0) continue;
              const Real c = w.rowb[0][i];
              int p, q;
              pair_of(r, i, p, q);
              const Real akp = w.G[k * N1 + p], akq = w.G[k * N1 + q];
              w.G[k * N1 + p] = c * akp - sn * akq;
              w.G[k * N1 + q] = sn * akp + c * akq;
              const Real vkp = V[k * n + p], vkq = V[k * n + q];
              V[k * n + p] = c * vkp - sn * vkq;
              V[k * n + q] = sn * vkp + c * vkq;
            }
            __syncthreads();
            // J^T (S J): rows p, q of every column
            for (int e = tid; e < npair * n; e += kT) {
              const int i = e / n, k = e % n;
              const Real sn = w.rowb[1][i];
              if (sn == (Real)0) continue;
              const Real c = w.rowb[0][i];
              int p, q;
              pair_of(r, i, p, q);
              const Real apk = w.G[p * N1 + k], aqk = w.G[q * N1 + k];
              w.G[p * N1 + k] = c * apk - sn * aqk;
              w.G[q * N1 + k] = sn * apk + c * aqk;
            }
            __syncthreads();
          }
          if (!w.bad) break;                   // a sweep without rotations: converged
        }
        __syncthreads();
        // eigenvalues, their largest, the kept directions' 1 / lambda
        if (tid == 0) {
          Real lmax = 0;
          for (int j = 0; j < n; ++j) lmax = fmax(lmax, w.G[j * N1 + j]);
          int kept = 0;
          for (int j = 0; j < n; ++j) {
            const Real l = w.G[j * N1 + j];
            const bool keep = l > (Real)a.drop_tol * lmax;
            w.invd[j] = keep ? (Real)1 / l : (Real)0;
            kept += keep;
          }
          w.keep_cnt = kept;
        }
        __syncthreads();
        // Q = D V L+ V^T D into the n x n block of G; the first step
        for (int e = tid; e < n * n; e += kT) {
          const int i = e / n, j = e % n;
          Real acc = 0;
          for (int k = 0; k < n; ++k) acc = fma(V[i * n + k] * w.invd[k], V[j * n + k], acc);
          w.G[i * N1 + j] = acc * w.scl[i] * w.scl[j];
        }
        __syncthreads();
        for (int i = tid; i < n; i += kT) {
          Real acc = 0;
          for (int k = 0; k < n; ++k) acc = fma(w.G[i * N1 + k], w.G[k * N1 + n], acc);
          w.gvec[i] = acc;
        }
        __syncthreads();
        for (int i = tid; i < n; i += kT) w.dxw[i] = w.gvec[i];
      }
      // the iterate starts at 0: (c_p, u) = 0, (c_q, v) = (1, 0)
      for (int e = tid; e < 2 * NM; e += kT) {
        const int which = e / NM, i = e % NM;
        const float c = (which == 1 && i == 0) ? 1.0f : 0.0f;
        w.uvhi[which][i] = c;
        w.uvlo[which][i] = 0.0f;
        w.uv[which][i] = c;
      }
      for (int j = tid; j < NAUG; j += kT) w.xw[j] = 0;
      __syncthreads();
      (void)apply_step<Real, NM, WS>(w, nm, n);
    }

    // ---------------- phase 5: refinement from the samples.
    // The iterate is the function pair p = c_p + psi.u, q = c_q + psi.v in
    // the unwhitened basis; each pass computes at every sample the design
    // residual r = w (y q - p), the objective sum r^2, whether q > 0, and
    // H_i = sum (w r) psi_i, K_i = sum (w y r) psi_i.  FP32 paths: plain
    // FP32 passes while the steps are large, then accurate passes (df_pass,
    // double-float; the first of them also computes the exact sample means
    // mu_i of the basis and rescales the iterate so that q averages to 1
    // over the samples exactly); FP64 path: FP64 passes.  With the mu_i of
    // the pass, the normal-equation residual in the design basis is
    //   g_num_0 = H_0, g_num_j = sum_{i<=j} W_ij (H_i - mu_i H_0),
    //   g_den_j = -sum_{i<=j} W_ij (K_i - mu_i K_0),
    // and the step dx = Q g.  A step that raises the objective is undone and
    // retried at half length.  The refinement stops once an accurate pass's
    // step, times the contraction estimated from the steps, is at most tol
    // relative (or such steps stop shrinking: their rounding floor), or
    // after max_refine steps.
    flags = (w.keep_cnt < n) ? RP_FIT_RANK_DEFICIENT : 0;
    float prev_rel = INFINITY, obj_prev = INFINITY;
    bool accurate = sizeof(Real) == 8, prev_accurate = false, done = false;
    // exact means of the set's basis carry over from the set's earlier fits
    bool have_mu = mu_known >= nm;
    int pole_prev = 0, it = 0, acc_passes = 0;
    float omega = 1.0f;   // step length (halved after an objective increase)
    float contr = 1.0f;   // estimated contraction per step
    constexpr bool kRegAcc = sizeof(Real) == 4 && DMAX <= 3;
    constexpr int VP = ((2 * NM + 2 + 15) / 16) * 16;   // register accumulators
    const int hk_groups = max(1, kT / nm);
    bool last_acc = sizeof(Real) == 8;   // the previous evaluation pass was accurate
    for (;; ++it) {
      const bool update = it < a.max_refine && !done;
      const bool dfp = sizeof(Real) == 4 && accurate;
      const bool first_df = dfp && !have_mu;
      // the first accurate pass: its exact objective is not compared with the
      // plain passes' (their residuals carry FP32 rounding)
      const bool fresh = dfp && !last_acc;
      last_acc = last_acc || dfp;
      float obj = 0.0f;
      int pole = 0;
      if (dfp) {
        if constexpr (sizeof(Real) == 4)
          df_pass<DMAX, NM>(w, d, nm, m, a.weighted != 0, first_df, sx0, sx1, sx2, sy, obj, pole,
                            cached ? slab : nullptr, psi_in_slab, D);
        psi_in_slab = psi_in_slab || (slab != nullptr && cached);
        ++acc_passes;
        if (first_df) {
          // exact sample means mu_j = S_j / m (pairs; mu_0 = 1), then the
          // iterate, the sums and the objective scaled by 1 / mean(q), with
          // mean(q) = sum_j mu_j V_j (V: the denominator's coefficients)
          if (wid == 0) {
            const float mh = (float)m;
            const dfl rm = df_recip(df_make(mh));
            dfl t = df_make(0.0f);
            for (int j2 = lane; j2 < nm; j2 += 32) {
              const dfl mu = df_mul(dfl{w.hkd[2][j2][0], w.hkd[2][j2][1]}, rm);
              w.mupsi[j2] = mu.h;
              w.mulo[j2] = mu.l;
              t = df_add(t, df_mul(mu, dfl{w.uvhi[1][j2], w.uvlo[1][j2]}));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
              t = df_add(t, dfl{__shfl_xor_sync(0xffffffffu, t.h, o), __shfl_xor_sync(0xffffffffu, t.l, o)});
            if (lane == 0) {
              const dfl sc = df_recip(t);
              w.fscal[1] = sc.h;
              w.fscal[2] = sc.l;
            }
          }
          __syncthreads();
          const dfl sc = dfl{w.fscal[1], w.fscal[2]};
          for (int e = tid; e < 2 * NM; e += kT) {
            const int which = e / NM, i2 = e % NM;
            const dfl u = df_mul(dfl{w.uvhi[which][i2], w.uvlo[which][i2]}, sc);
            w.uvhi[which][i2] = u.h;
            w.uvlo[which][i2] = u.l;
            const dfl hk = df_mul(dfl{w.hkd[which][i2][0], w.hkd[which][i2][1]}, sc);
            w.hkd[which][i2][0] = hk.h;
            w.hkd[which][i2][1] = hk.l;
          }
          for (int j2 = tid; j2 < n; j2 += kT) w.xw[j2] *= (Real)sc.h;
          obj *= sc.h * sc.h;
          have_mu = true;
          mu_known = nm;
          __syncthreads();
        }
      } else {
      Real hk0 = 0, hk1 = 0;    // staged path: this thread's column partials
      float acc[kRegAcc ? VP : 1];
#pragma unroll
      for (int j = 0; j < (kRegAcc ? VP : 1); ++j) acc[j] = 0.0f;
      for (int base = 0; base < m; base += kT) {
        const int cnt = min(kT, m - base);
        if (tid < cnt) {
          const int i = base + tid;
          Real psi[NM];
          eval_psi<Real, DMAX, NM>(w, d, nm, sx0[i], sx1[i], sx2[i], psi);
          psi[0] = 1;
          const Real yy = (Real)sy[i];
          const Real wt = a.weighted ? recip(fabs(yy)) : (Real)1;
          Real r;
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
            float hq[NM], hp[NM];
            ld_row<NM>(w.uvhi[1], hq);
            ld_row<NM>(w.uvhi[0], hp);
            float qf = hq[0], p = hp[0];
#pragma unroll
            for (int j2 = 1; j2 < NM; ++j2) {
              qf = fmaf(psi[j2], hq[j2], qf);
              p = fmaf(psi[j2], hp[j2], p);
            }
            pole |= !(qf > 0.0f);
            r = wt * fmaf(yy, qf, -p);
          }
          obj += (float)(r * r);
          if constexpr (kRegAcc) {
            if (update) {
              const float rn = (float)(wt * r), rd = (float)(wt * yy * r);
#pragma unroll
              for (int j2 = 0; j2 < NM; ++j2) {
                acc[j2] = fmaf(rn, (float)psi[j2], acc[j2]);
                acc[NM + j2] = fmaf(rd, (float)psi[j2], acc[NM + j2]);
              }
            }
          } else if (update) {
            Real *row = w.stage + tid * LDS;
#pragma unroll
            for (int j2 = 0; j2 < NM; ++j2) row[j2] = psi[j2];
            w.rbuf[0][tid] = wt * r;
            w.rbuf[1][tid] = wt * yy * r;
          }
        }
        if constexpr (!kRegAcc) {
          if (update) {
            __syncthreads();
            if (tid < nm * hk_groups) {
              const int j2 = tid % nm, g = tid / nm;
              Real pn = 0, pd = 0;
              for (int s2 = g; s2 < cnt; s2 += hk_groups) {
                const Real bv = w.stage[s2 * LDS + j2];
                pn = fma(bv, w.rbuf[0][s2], pn);
                pd = fma(bv, w.rbuf[1][s2], pd);
              }
              hk0 += pn;
              hk1 += pd;
            }
            __syncthreads();
          }
        }
      }
      // block totals: objective, pole, and (when stepping) H and K
      if constexpr (kRegAcc) {
        acc[2 * NM] = obj;
        acc[2 * NM + 1] = pole ? 1.0f : 0.0f;
        warp_reduce_scatter<VP>(acc);
        if ((lane & 1) == 0) {
          const int b = rs_base<VP>(lane);
#pragma unroll
          for (int q = 0; q < VP / 16; ++q) w.redv[wid][b + q] = acc[q];
        }
        __syncthreads();
        obj = w.redv[0][2 * NM] + w.redv[1][2 * NM] + w.redv[2][2 * NM] + w.redv[3][2 * NM];
        pole = (w.redv[0][2 * NM + 1] + w.redv[1][2 * NM + 1] + w.redv[2][2 * NM + 1] +
                w.redv[3][2 * NM + 1]) > 0.0f;
        if (update && tid < 2 * NM) {
          const Real v = w.redv[0][tid] + w.redv[1][tid] + w.redv[2][tid] + w.redv[3][tid];
          w.HK[tid / NM][tid % NM] = v;
        }
      } else {
        pole = __syncthreads_or(pole);
        obj = block_sum_f(w, obj, 8);
        if (update) {
          __syncthreads();
          if (tid < nm * hk_groups) {
            w.stage[tid] = hk0;
            w.stage[kT + tid] = hk1;
          }
          __syncthreads();
          if (tid < nm) {
            Real h = 0, k2 = 0;
            for (int g = 0; g < hk_groups; ++g) {
              h += w.stage[g * nm + tid];
              k2 += w.stage[kT + g * nm + tid];
            }
            w.HK[0][tid] = h;
            w.HK[1][tid] = k2;
          }
        }
      }
      __syncthreads();
      }   // plain pass
      // (the first accurate pass starts a new comparison: its objective is
      // exact, and on a set's first fit its iterate was rescaled)
      const bool worse = it > 0 && !fresh && obj > obj_prev * (accurate ? 1.00001f : 1.0001f);
      if (worse) {
        // the last step increased the objective: undo it, then retry it at
        // half length (a preconditioner that overestimates curvature in some
        // direction makes the full step overshoot); the halving persists
        // for the fit's later steps; below 1/16 the refinement stops
        for (int e = tid; e < 2 * NM; e += kT) {
          const int which = e / NM, i2 = e % NM;
          w.uv[which][i2] = w.uvp[which][i2];
          w.uvhi[which][i2] = w.uvphi[which][i2];
          w.uvlo[which][i2] = w.uvplo[which][i2];
        }
        for (int j2 = tid; j2 < n; j2 += kT) w.xw[j2] = w.xwp[j2];
        omega *= 0.5f;
        if (omega < 0.0625f || it >= a.max_refine) {
          pole = pole_prev;
          __syncthreads();
          break;
        }
        for (int j2 = tid; j2 < n; j2 += kT) w.dxw[j2] *= (Real)0.5;
        __syncthreads();
        (void)apply_step<Real, NM, WS>(w, nm, n);
        continue;
      }
      for (int e = tid; e < 2 * NM; e += kT) {
        const int which = e / NM, i2 = e % NM;
        w.uvp[which][i2] = w.uv[which][i2];
        w.uvphi[which][i2] = w.uvhi[which][i2];
        w.uvplo[which][i2] = w.uvlo[which][i2];
      }
      for (int j2 = tid; j2 < n; j2 += kT) w.xwp[j2] = w.xw[j2];
      obj_prev = obj;
      pole_prev = pole;
      if (!update) {
        __syncthreads();
        break;
      }
      // centred sums H_0, H_i - mu_i H_0 and K_0, K_i - mu_i K_0 (pairs on
      // an accurate pass: the fixed point K_i = mu_i K_0 carries the
      // normalisation, so mu_i K_0 is formed to the pass's accuracy)
      for (int e = tid; e < 2 * NM; e += kT) {
        const int which = e / NM, i2 = e % NM;
        Real v = 0;
        if (i2 < nm) {
          if (dfp) {
            const dfl h0 = dfl{w.hkd[which][0][0], w.hkd[which][0][1]};
            const dfl hi = dfl{w.hkd[which][i2][0], w.hkd[which][i2][1]};
            const dfl c = i2 == 0 ? h0 : df_add(hi, df_neg(df_mul(dfl{(float)w.mupsi[i2], w.mulo[i2]}, h0)));
            v = (Real)c.h;
          } else {
            v = i2 == 0 ? w.HK[which][0] : w.HK[which][i2] - w.mupsi[i2] * w.HK[which][0];
          }
        }
        w.HKc[which][i2] = v;
      }
      __syncthreads();
      // g, then the step dx = Q g
      for (int e = tid; e < n; e += kT) {
        Real g;
        if (e < nm) {
          if (e == 0) {
            g = w.HKc[0][0];
          } else {
            g = 0;
            for (int i2 = 1; i2 <= e; ++i2) g = fma(w.W[i2 * WS + e], w.HKc[0][i2], g);
          }
        } else {
          const int jd = e - nm + 1;
          g = 0;
          for (int i2 = 1; i2 <= jd; ++i2) g = fma(-w.W[i2 * WS + jd], w.HKc[1][i2], g);
        }
        w.gvec[e] = g;
      }
      __syncthreads();
      for (int e = tid; e < n; e += kT) {
        // Q is symmetric: read column e (consecutive threads, consecutive words)
        Real z = 0;
        for (int k2 = 0; k2 < n; ++k2) z = fma(w.G[k2 * naug + e], w.gvec[k2], z);
        w.dxw[e] = z * (Real)omega;
      }
      __syncthreads();
      const float rel = apply_step<Real, NM, WS>(w, nm, n);
      // contraction of the preconditioned iteration, estimated from the
      // steps: the first step's relative size (the error of the factor's
      // solution) and the ratios of later steps while they are above the
      // FP32 rounding floor (plain passes) or of successive accurate steps
      const bool was_accurate = accurate;
      if (it == 0) contr = rel;
      else if (was_accurate ? prev_accurate : rel > 1e-5f) contr = fmaxf(contr, rel / prev_rel);
      // accurate from here on once the plain steps are small, stop
      // shrinking (the FP32 rounding floor), or the budget nears its end
      if (!accurate && (rel < 1e-4f || (it > 0 && rel > 0.5f * prev_rel) || it + 2 >= a.max_refine))
        accurate = true;
      // stop once an accurate step leaves an estimated relative error
      // (contraction x step, the contraction taken as at least 1e-3) of at
      // most tol, or once accurate corrections stop shrinking at their
      // rounding floor (below 1e-8 relative: above it, slow shrinking is a
      // weak preconditioner's contraction, and the refinement goes on)
      if (was_accurate && (fminf(fmaxf(contr, 1e-3f), 1.0f) * rel <= (float)a.tol ||
                           (prev_accurate && rel > 0.9f * prev_rel && rel < 1e-8f)))
        done = true;
      prev_rel = rel;
      prev_accurate = was_accurate;
      if (done) {
        // converged: the last correction is below tol (or at the residuals'
        // noise floor); it is kept without another evaluation pass
        ++it;
        break;
      }
    }
    flags |= (pole_prev ? RP_FIT_POLE : 0);
    // not converged: the refinement ended (max_refine steps, or steps that
    // kept raising the objective) before its stop test was met
    if (a.max_refine > 0 && !done) flags |= RP_FIT_NOT_CONVERGED;
    flags |= min(it, 255) << RP_FIT_ITER_SHIFT;
    flags |= min(acc_passes, 255) << RP_FIT_ACC_SHIFT;
    if (use_tc && a.max_refine > 0 && (!done || (flags & RP_FIT_RANK_DEFICIENT))) {
      escalated = true;
      continue;
    }
    break;
    }   // attempts
    if (tc_dead) {
      if (tid == 0) {
        a.status[f] = RP_FIT_TIMEOUT;
        a.rank[f] = 0;
      }
      continue;
    }
    if (escalated) flags |= RP_FIT_ESCALATED;

    // ---------------- phase 6: back to the monomial basis (FP64)
    {
      double *cpsi = reinterpret_cast<double *>(w.stage);   // [2][kMaxNm]
      double *P = cpsi + 2 * kMaxNm;                          // [3][5][5]
      // the iterate's coefficients on Psi (index 0: the constants c_p, c_q)
      for (int e = tid; e < 2 * nm; e += kT) {
        const int which = e / nm, i = e % nm;   // 0 numerator, 1 denominator
        cpsi[which * kMaxNm + i] = sizeof(Real) == 8
                                       ? w.uv[which][i]
                                       : (double)w.uvhi[which][i] + (double)w.uvlo[which][i];
      }
      if (tid >= kT - 3 * (kMaxDeg + 1) * (kMaxDeg + 1) + 0 && tid < kT) {
        // P[v][k][i]: coefficient of x'^i in Q_k(u) for the box-normalised
        // x' = 2 (x - lo) / (hi - lo) - 1, where the basis variable is
        // u = (x sc + of - mu) isg with the kernel's own constants, i.e.
        // u = A x' + B, A = isg sc (hi - lo) / 2, B = isg (sc (hi + lo) / 2 + of - mu)
        // (exactly the map the accurate passes evaluate); one entry per
        // thread: sum_{l=i..k} Tm[l][k] C(l, i) A^i B^(l-i)
        const int e = tid - (kT - 3 * (kMaxDeg + 1) * (kMaxDeg + 1));
        const int v = e / ((kMaxDeg + 1) * (kMaxDeg + 1));
        const int k = (e / (kMaxDeg + 1)) % (kMaxDeg + 1), i = e % (kMaxDeg + 1);
        const double isg = w.isg_v[v], scv = w.sc_v[v];
        const double A = isg * scv * (w.hi[v] - w.lo[v]) * 0.5;
        const double B = isg * (scv * (w.hi[v] + w.lo[v]) * 0.5 + (double)w.of_v[v] - (double)w.mu_v[v]);
        double acc = 0.0;
        if (k <= d && i <= k) {
          double pw = 1.0;   // A^i B^(l - i), starting at l = i
          for (int l = 0; l < i; ++l) pw *= A;
          const double step = B;
          int binom = 1;     // C(l, i), starting at C(i, i)
          for (int l = i; l <= k; ++l) {
            acc = fma((double)w.Tm[v][l][k] * (double)binom, pw, acc);
            pw *= step;
            binom = binom * (l + 1) / (l + 1 - i);
          }
        }
        P[(v * (kMaxDeg + 1) + k) * (kMaxDeg + 1) + i] = acc;
      }
      __syncthreads();
      // the basis change is a tensor product: three 1-D passes, one per
      // variable (N last), each summing <= d + 1 terms per coefficient
      double *buf[2] = {cpsi, P + 3 * (kMaxDeg + 1) * (kMaxDeg + 1)};
      int cur = 0;
#pragma unroll
      for (int v = 2; v >= 0; --v) {
        for (int e = tid; e < 2 * nm; e += kT) {
          const int which = e / nm, t = e % nm;
          int ex[3] = {c_exp[t][0], c_exp[t][1], c_exp[t][2]};
          const int ov = ex[v];
          const int room = d - (ex[0] + ex[1] + ex[2] - ov);
          double acc = 0.0;
          for (int k = ov; k <= room; ++k) {
            ex[v] = k;
            acc = fma(buf[cur][which * kMaxNm + c_idx[ex[0]][ex[1]][ex[2]]],
                      P[(v * (kMaxDeg + 1) + k) * (kMaxDeg + 1) + ov], acc);
          }
          buf[cur ^ 1][which * kMaxNm + t] = acc;
        }
        cur ^= 1;
        __syncthreads();
      }
      for (int e = tid; e < 2 * nm; e += kT) {
        const int which = e / nm, t = e % nm;
        const double s = buf[cur][which * kMaxNm + t];
        const int o = which == 0 ? t : kHalf + t;
        cf[o] = s;
        if (a.coef32) a.coef32[f * kStride + o] = (float)s;
      }
      if (tid == 0) {
        int32_t st = flags;
        if (a.esc_mode == 2) st |= RP_FIT_FP64_PASS;
        // dropped pivots or refinement short of tol: solved again on the
        // FP64 path by the launch that follows
        if (a.esc_mode == 1 && a.max_refine > 0 && (flags & (RP_FIT_RANK_DEFICIENT | RP_FIT_NOT_CONVERGED))) {
          st |= kPending64;
          if (a.esc_count) atomicAdd(a.esc_count, 1ull);
        }
        a.status[f] = st;
        a.rank[f] = w.keep_cnt;
      }
      __syncthreads();
    }
    }   // fits of the set
  }
  if constexpr (GM > 0) {
    // after a wait that gave up, wait (bounded) once more for the MMAs still
    // in flight before the tensor memory is released
    if (tc_dead && tid == 0) (void)tc::mbar_wait(&w.mbar, tc_phase, kTcWaitLimit);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (wid == 0) tc::tmem_dealloc(tmem, TS::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------

void set_tables() {
  static bool done[16] = {};   // per device (constant memory is per context)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) dev = 0;
  if (done[dev]) return;
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
  int8_t idx[kMaxDeg + 1][kMaxDeg + 1][kMaxDeg + 1];
  for (int i = 0; i <= kMaxDeg; ++i)
    for (int j = 0; j <= kMaxDeg; ++j)
      for (int l = 0; l <= kMaxDeg; ++l) idx[i][j][l] = -1;
  for (int t = 0; t < kMaxNm; ++t) idx[e[t][0]][e[t][1]][e[t][2]] = (int8_t)t;
  cudaMemcpyToSymbol(c_idx, idx, sizeof(idx));
  done[dev] = true;
}

// Resident CTAs per SM of one fit-kernel variant: registers, shared memory,
// threads and (tensor-core variants) tensor-memory columns.
template <class Real, int DMAX, int GM>
int residency() {
  using WF = CtaFit<Real, DMAX, GM>;
  const size_t smem = ctafit_bytes<Real, DMAX, GM>();
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fit_kernel<Real, DMAX, GM>) != cudaSuccess) return 1;
  int dev = 0;
  cudaGetDevice(&dev);
  int smem_sm = 0, smem_rsv = 0, regs_sm = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  const int regs_cta = ((fa.numRegs * 32 + 255) / 256 * 256) * (kT / 32);
  int per_sm = smem_sm / (int)(smem + smem_rsv);
  per_sm = min(per_sm, regs_sm / max(regs_cta, 1));
  per_sm = min(per_sm, 2048 / kT);
  if (GM > 0) per_sm = min(per_sm, 512 / TcShape<DMAX>::TMEM_COLS);
  (void)sizeof(WF);
  return per_sm < 1 ? 1 : per_sm;
}

template <class Real, int DMAX, int GM>
cudaError_t launch_t(const FitArgs &a, int precision, cudaStream_t s) {
  using WF = CtaFit<Real, DMAX, GM>;
  // 128-bit shared-memory loads of the staged rows and of W; 8-byte mbarrier
  static_assert(offsetof(WF, stage) == 0, "stage must start the state");
  static_assert(offsetof(WF, W) % 16 == 0 && offsetof(WF, G) % 16 == 0, "W, G: 16-byte aligned");
  static_assert(offsetof(WF, mbar) % 8 == 0, "mbarrier: 8-byte aligned");
  set_tables();
  const size_t smem = ctafit_bytes<Real, DMAX, GM>();
  cudaError_t e = cudaFuncSetAttribute(fit_kernel<Real, DMAX, GM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = residency<Real, DMAX, GM>();
  const int cap = fit_ctas_cap(precision, DMAX);
  if (cap > 0 && cap < per_sm) per_sm = cap;
  int64_t grid = (int64_t)num_sms() * per_sm;
  const int64_t nsets = a.point_off ? (a.F + a.fits_per_set - 1) / a.fits_per_set : a.F;
  // split point sets into runs only while there are fewer claims than
  // resident CTAs: a whole set computes its box, basis and whitening once
  // for all of its fits (and its basis cache serves them all), and the
  // dynamic claims balance whole sets well (1024 sets of 8 fits on 608
  // CTAs: 2.38 ms, against 2.48 ms for runs of 4 fits)
  FitArgs b = a;
  b.set_parts = 1;
  if (a.point_off)
    while (b.set_parts < a.fits_per_set && nsets * b.set_parts < grid) b.set_parts *= 2;
  const int64_t units = nsets * b.set_parts;
  if (grid > units) grid = units;
  if (a.counter) {
    e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  fit_kernel<Real, DMAX, GM><<<(unsigned)grid, kT, smem, s>>>(b);
  return cudaGetLastError();
}

// One precision family (Real, GM) for the degree bound dmax of a launch.
template <class Real, int GM>
cudaError_t launch_family(const FitArgs &a, int dmax, int precision, cudaStream_t s) {
  switch (dmax) {
    case 1: case 2: return launch_t<Real, 2, GM>(a, precision, s);
    case 3: return launch_t<Real, 3, GM>(a, precision, s);
    default: return launch_t<Real, 4, GM>(a, precision, s);
  }
}
template <class Real, int GM>
int residency_family(int dmax) {
  return dmax <= 2 ? residency<Real, 2, GM>() : dmax == 3 ? residency<Real, 3, GM>() : residency<Real, 4, GM>();
}

}  // namespace
}  // namespace rpk
