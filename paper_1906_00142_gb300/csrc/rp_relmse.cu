// Nonlinear refinement of fitted rational functions on the mean squared
// relative error (no counterpart in the paper; it refines the linearised
// least-squares solution of Sec. 4.2):
//   L_f = (1/m) sum_i r_i^2,  r_i = (p(x_i)/q(x_i) - y_i) / y_i
//   dL/dalpha_j = (2/m) sum_i r_i phi_j(x_i) / (y_i q_i)
//   dL/dbeta_j  = -(2/m) sum_i r_i p_i phi_j(x_i) / (y_i q_i^2)   (j >= 1)
// beta_0 is held fixed (it fixes the scale of the homogeneous pair p, q).
// One CTA per fit, deterministic reductions.  The coefficients are the
// fit's FP64 output and p and q are evaluated in FP64 (the fitted monomial
// coefficients can cancel by 1e3-1e9, so neither an FP32 copy of them nor an
// FP32 evaluation keeps the residual's leading digits); the residual, loss
// and gradient sums are FP32.  Adam updates the FP64 coefficients with FP32
// moments.
#include <math.h>
#include <stdint.h>

#include "rp_internal.cuh"

namespace rpk {
namespace {

constexpr int kT = 256;

struct Exps {
  int8_t e[kMaxNm][3];
};

Exps exps_table() {
  Exps t{};
  int k = 0;
  for (int s = 0; s <= kMaxDeg; ++s)
    for (int a = s; a >= 0; --a)
      for (int b = s - a; b >= 0; --b) {
        t.e[k][0] = (int8_t)a;
        t.e[k][1] = (int8_t)b;
        t.e[k][2] = (int8_t)(s - a - b);
        ++k;
      }
  return t;
}

// Powers of the sample's normalised coordinates, 0..kMaxDeg, per variable.
constexpr int kPw = kMaxDeg + 1;

struct RelShared {
  double cf[kStride];
  double scd[3], ofd[3];
  float red[kT / 32];
  float xp[kT][3][kPw];               // chunk samples: powers of x', B0', B1'
  float sp[kT], sq[kT];
  float part[kT];                     // gradient partials per (entry, sample group)
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Graded-lex index of the monomial x^a y^b z^c (degree ascending, then a
// descending, then b descending): the same for every degree bound.
__host__ __device__ constexpr int glex(int a, int b, int c) {
  return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// sum_j c_j x^a_j y^b_j z^c_j of total degree <= D as nested Horner
// polynomials (one FMA per coefficient plus one per inner polynomial), FP64.
template <int D>
__device__ __forceinline__ double horner3(const double *c, double x, double y, double z) {
  double p = 0.0;
#pragma unroll
  for (int a = D; a >= 0; --a) {
    double pa = 0.0;
#pragma unroll
    for (int b = D - a; b >= 0; --b) {
      double pab = 0.0;
#pragma unroll
      for (int cc = D - a - b; cc >= 0; --cc) pab = fma(pab, z, c[glex(a, b, cc)]);
      pa = fma(pa, y, pab);
    }
    p = fma(p, x, pa);
  }
  return p;
}

__device__ __forceinline__ double horner_d(int d, const double *c, double x, double y, double z) {
  switch (d) {
    case 1: return horner3<1>(c, x, y, z);
    case 2: return horner3<2>(c, x, y, z);
    case 3: return horner3<3>(c, x, y, z);
    default: return horner3<4>(c, x, y, z);
  }
}

__global__ void __launch_bounds__(kT) relmse_kernel(bool backward, int64_t F, int64_t S,
                                                    const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    const int64_t *__restrict__ off,
                                                    const int8_t *__restrict__ degs,
                                                    const double *__restrict__ coef,
                                                    const double *__restrict__ box,
                                                    const float *__restrict__ grad_loss,
                                                    float *__restrict__ out, Exps et) {
  __shared__ RelShared sh;
  const int tid = threadIdx.x;
  for (int64_t f = blockIdx.x; f < F; f += gridDim.x) {
    const int64_t b0 = off[f];
    const int m = (int)(off[f + 1] - b0);
    const int d = degs[f];
    const int nm = (d >= 1 && d <= kMaxDeg) ? num_monomials(d) : 0;
    if (tid < kStride) sh.cf[tid] = coef[f * kStride + tid];
    if (tid < 3) {
      const double lo = box[f * 6 + 2 * tid], hi = box[f * 6 + 2 * tid + 1];
      if (hi > lo) {
        const double s = 2.0 / (hi - lo);
        sh.scd[tid] = s;
        sh.ofd[tid] = -1.0 - lo * s;
      } else {
        sh.scd[tid] = 0.0;
        sh.ofd[tid] = 0.0;
      }
    }
    __syncthreads();
    const float gscale = backward ? grad_loss[f] : 1.0f;
    float lsum = 0.0f;
    // backward: gradient entry e (numerator e < nm, denominator nm + e) is
    // summed by `groups` threads over interleaved samples of each chunk
    const int ne = 2 * nm;
    const int groups = ne > 0 ? max(1, kT / ne) : 1;
    const int my_e = tid % max(ne, 1), my_g = tid / max(ne, 1);
    const bool has_e = ne > 0 && tid < ne * groups;
    const int e0 = has_e ? et.e[my_e % nm][0] : 0, e1 = has_e ? et.e[my_e % nm][1] : 0,
              e2 = has_e ? et.e[my_e % nm][2] : 0;
    const bool den = my_e >= nm;
    float gacc = 0.0f;
    for (int base = 0; base < m; base += kT) {
      const int cnt = min(kT, m - base);
      if (tid < cnt && nm > 0) {
        const int64_t i = b0 + base + tid;
        const double xd0 = fma((double)x[i], sh.scd[0], sh.ofd[0]);
        const double xd1 = fma((double)x[S + i], sh.scd[1], sh.ofd[1]);
        const double xd2 = fma((double)x[2 * S + i], sh.scd[2], sh.ofd[2]);
        // p and q in FP64: fitted monomial coefficients can cancel heavily
        const double p = horner_d(d, sh.cf, xd0, xd1, xd2);
        const double q = horner_d(d, sh.cf + kHalf, xd0, xd1, xd2);
        const float yy = y[i];
        const float r = (float)((p / q - (double)yy) / (double)yy);
        lsum = fmaf(r, r, lsum);
        if (backward) {
          const float pf = (float)p, qf = (float)q;
          const float iyq = 1.0f / (yy * qf);
          sh.sp[tid] = r * iyq;
          sh.sq[tid] = -r * pf * iyq / qf;
          const float xv[3] = {(float)xd0, (float)xd1, (float)xd2};
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            float pw = 1.0f;
#pragma unroll
            for (int l = 0; l < kPw; ++l) {
              sh.xp[tid][v][l] = pw;
              pw *= xv[v];
            }
          }
        }
      }
      if (backward) {
        __syncthreads();
        if (has_e) {
          const float *s_r = den ? sh.sq : sh.sp;
          float part = 0.0f;
          for (int s2 = my_g; s2 < cnt; s2 += groups)
            part = fmaf(s_r[s2], sh.xp[s2][0][e0] * sh.xp[s2][1][e1] * sh.xp[s2][2][e2], part);
          gacc += part;
        }
        __syncthreads();
      }
    }
    if (!backward) {
      lsum = warp_sum_f(lsum);
      if ((tid & 31) == 0) sh.red[tid >> 5] = lsum;
      __syncthreads();
      if (tid == 0) {
        float s = 0.0f;
        for (int w = 0; w < kT / 32; ++w) s += sh.red[w];
        out[f] = m > 0 ? s / (float)m : 0.0f;
      }
    } else {
      // sum the sample groups of each entry (fixed order: deterministic)
      sh.part[tid] = has_e ? gacc : 0.0f;
      if (tid < kStride) out[f * kStride + tid] = 0.0f;
      __syncthreads();
      const float scale = m > 0 ? 2.0f * gscale / (float)m : 0.0f;
      if (tid < ne) {
        float g = 0.0f;
        for (int g2 = 0; g2 < groups; ++g2) g += sh.part[g2 * ne + tid];
        const int j = tid % nm;
        if (!(tid >= nm && j == 0)) out[f * kStride + (tid >= nm ? kHalf + j : j)] = scale * g;
      }
    }
    __syncthreads();
  }
}

__global__ void adam_kernel(int64_t n, double *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v,
                            const uint8_t *__restrict__ mask, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask && !mask[i]) continue;
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= (double)(lr * (mi / c1) / (sqrtf(vi / c2) + eps));
  }
}

}  // namespace

cudaError_t launch_relmse(bool backward, int64_t F, int64_t S, const float *x, const float *y,
                          const int64_t *fit_off, const int8_t *degrees, const double *coef,
                          const double *box, const float *grad_loss, float *out,
                          cudaStream_t s) {
  if (F == 0) return cudaSuccess;
  static const Exps et = exps_table();
  int64_t grid = (int64_t)num_sms() * 4;
  if (grid > F) grid = F;
  relmse_kernel<<<(unsigned)grid, kT, 0, s>>>(backward, F, S, x, y, fit_off, degrees, coef, box,
                                              grad_loss, out, et);
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, double *p, const float *g, float *m, float *v,
                        const uint8_t *mask, int t, float lr, float b1, float b2, float eps,
                        cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  int64_t grid = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (grid > cap) grid = cap;
  adam_kernel<<<(unsigned)grid, 256, 0, s>>>(n, p, g, m, v, mask, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace rpk
