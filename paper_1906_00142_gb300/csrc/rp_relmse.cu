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

struct RelShared {
  double cf[kStride];
  double scd[3], ofd[3];
  float red[kT / 32];
  float xn[kT][3];
  float sp[kT], sq[kT];
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
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
    // backward: thread j owns gradient entry j (numerator j < nm, denominator
    // nm + j); accumulated over chunks of kT samples.
    float gacc = 0.0f;
    for (int base = 0; base < m; base += kT) {
      const int cnt = min(kT, m - base);
      if (tid < cnt && nm > 0) {
        const int64_t i = b0 + base + tid;
        // p and q in FP64: fitted monomial coefficients can cancel heavily,
        // so an FP32 evaluation would lose the residual's leading digits
        double xd[3];
        xd[0] = fma((double)x[i], sh.scd[0], sh.ofd[0]);
        xd[1] = fma((double)x[S + i], sh.scd[1], sh.ofd[1]);
        xd[2] = fma((double)x[2 * S + i], sh.scd[2], sh.ofd[2]);
        double pw[3][kMaxDeg + 1];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          pw[v][0] = 1.0;
#pragma unroll
          for (int l = 1; l <= kMaxDeg; ++l) pw[v][l] = pw[v][l - 1] * xd[v];
        }
        double p = 0.0, q = 0.0;
        for (int j = 0; j < nm; ++j) {
          const double ph = pw[0][et.e[j][0]] * pw[1][et.e[j][1]] * pw[2][et.e[j][2]];
          p = fma(sh.cf[j], ph, p);
          q = fma(sh.cf[kHalf + j], ph, q);
        }
        const float yy = y[i];
        const float r = (float)((p / q - (double)yy) / (double)yy);
        lsum = fmaf(r, r, lsum);
        if (backward) {
          const float pf = (float)p, qf = (float)q;
          const float iyq = 1.0f / (yy * qf);
          sh.sp[tid] = r * iyq;
          sh.sq[tid] = -r * pf * iyq / qf;
          sh.xn[tid][0] = (float)xd[0];
          sh.xn[tid][1] = (float)xd[1];
          sh.xn[tid][2] = (float)xd[2];
        }
      }
      if (backward) {
        __syncthreads();
        if (tid < 2 * nm) {
          const int j = tid % nm;
          const bool den = tid >= nm;
          const int e0 = et.e[j][0], e1 = et.e[j][1], e2 = et.e[j][2];
          float part = 0.0f;
          for (int s = 0; s < cnt; ++s) {
            float ph = 1.0f;
            for (int l = 0; l < e0; ++l) ph *= sh.xn[s][0];
            for (int l = 0; l < e1; ++l) ph *= sh.xn[s][1];
            for (int l = 0; l < e2; ++l) ph *= sh.xn[s][2];
            part = fmaf(den ? sh.sq[s] : sh.sp[s], ph, part);
          }
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
      const float scale = m > 0 ? 2.0f * gscale / (float)m : 0.0f;
      if (tid < kStride) out[f * kStride + tid] = 0.0f;
      __syncthreads();
      if (tid < 2 * nm) {
        const int j = tid % nm;
        const bool den = tid >= nm;
        if (!(den && j == 0)) out[f * kStride + (den ? kHalf + j : j)] = scale * gacc;
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
