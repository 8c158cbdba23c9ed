// Rational-program table packing and the FP32 evaluate-and-argmin kernel.
//
// Pack: Sec. 3.3 Step 3 (code generation) / Sec. 4.3.1 -- the fitted metric
// functions of each kernel become, per thread-block configuration, univariate
// rationals in the normalised data parameter.
// Search: Sec. 3.3 Steps 4-5 / Sec. 4.3.2 -- the MWP-CWP rational program
// (Sec. 2 Example 2, occupancy Example 1) is evaluated at every admissible
// configuration and the best one is selected.
#include <math.h>
#include <stdint.h>

#include "rp_internal.cuh"

namespace rpk {
namespace {

// Graded-lex exponents, degree ascending, e_N descending, e_B0 descending.
struct ExpTab {
  int8_t e[kMaxNm][3];
};

ExpTab make_exponents() {
  ExpTab t{};
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

// One thread per (kernel, configuration, metric).  FP64 arithmetic.
__global__ void pack_kernel(int64_t K, int d, const double *__restrict__ coef,
                            const double *__restrict__ box, const int8_t *__restrict__ degrees,
                            const int32_t *__restrict__ metric_map,
                            const int32_t *__restrict__ grid_dims, ProgramMut prog, ExpTab et) {
  const int64_t total = K * kNcfg * kNmet;
  const int D1 = d + 1;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int mt = (int)(id % kNmet);
    const int c = (int)((id / kNmet) % kNcfg);
    const int64_t k = id / (kNmet * kNcfg);
    const int fi = metric_map[k * kNmet + mt];
    double pn[kMaxDeg + 1], pd[kMaxDeg + 1];
#pragma unroll
    for (int i = 0; i <= kMaxDeg; ++i) pn[i] = pd[i] = 0.0;
    if (fi < 0) {
      pd[0] = 1.0;
    } else {
      // configuration index -> (a, b) with B0 = 2^a, B1 = 2^b
      int a = 0, rem = c;
      while (rem >= 11 - a) { rem -= 11 - a; ++a; }
      const double B0 = (double)(1 << a), B1 = (double)(1 << rem);
      const double *bx = box + 6 * (int64_t)fi;
      const double u = (bx[3] > bx[2]) ? 2.0 * (B0 - bx[2]) / (bx[3] - bx[2]) - 1.0 : 0.0;
      const double w = (bx[5] > bx[4]) ? 2.0 * (B1 - bx[4]) / (bx[5] - bx[4]) - 1.0 : 0.0;
      double up[kMaxDeg + 1], wp[kMaxDeg + 1];
      up[0] = wp[0] = 1.0;
#pragma unroll
      for (int i = 1; i <= kMaxDeg; ++i) {
        up[i] = up[i - 1] * u;
        wp[i] = wp[i - 1] * w;
      }
      const int df = degrees[fi];
      const int nm = num_monomials(df);
      const double *cf = coef + (int64_t)fi * kStride;
      for (int j = 0; j < nm; ++j) {
        const double sB = up[et.e[j][1]] * wp[et.e[j][2]];
        const int e0 = et.e[j][0];
        pn[e0] += cf[j] * sB;
        pd[e0] += cf[kHalf + j] * sB;
      }
    }
    float *row = prog.table + ((k * kNcfg + c) * kNmet + mt) * 2 * D1;
    for (int i = 0; i < D1; ++i) {
      row[i] = (float)pn[i];
      row[D1 + i] = (float)pd[i];
    }
    if (c == 0) {
      double A = 0.0, Bc = 0.0;
      if (fi >= 0) {
        const double *bx = box + 6 * (int64_t)fi;
        if (bx[1] > bx[0]) {
          A = 2.0 / (bx[1] - bx[0]);
          Bc = -1.0 - 2.0 * bx[0] / (bx[1] - bx[0]);
        }
      }
      prog.aN[k * kNmet + mt] = (float)A;
      prog.bN[k * kNmet + mt] = (float)Bc;
      if (mt == 0) prog.grid[k] = grid_dims[k];
    }
  }
}

// ---------------------------------------------------------------------
// Search

struct CfgTab {
  int8_t la[kNcfg];        // log2 B0
  int8_t lb[kNcfg];        // log2 B1
  int32_t wpb[kNcfg];      // warps per block, ceil(T / warp)
  int32_t bact_w[kNcfg];   // min(B_max, floor(W_max / wpb)), 0 if T > T_max
};

struct HwC {
  int32_t warp, wmax, rsm, zsm;
  float issue;
};

// #Rep = ceil(blocks / D) for blocks = c0 * c1 (each < 2^32) and
// 1 <= D < 2^25.  Exact (integer remainder correction of a float estimate)
// when the quotient is below 2^22; above that the float estimate (relative
// error < 2^-21) is used.  Only 32-bit int<->float conversions are used.
__device__ __forceinline__ float rep_count(uint32_t c0, uint32_t c1, uint32_t D) {
  const float qf = __fdividef((float)c0 * (float)c1, (float)D);
  const uint64_t blocks = (uint64_t)c0 * c1;
  const uint32_t q0 = (uint32_t)fminf(qf, 4194304.0f);
  int64_t r = (int64_t)(blocks - (uint64_t)q0 * D);
  int64_t q = q0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool lo = r < 0;
    q -= lo;
    r += lo ? (int64_t)D : 0;
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = r >= (int64_t)D;
    q += hi;
    r -= hi ? (int64_t)D : 0;
  }
  const float exact = (float)(uint32_t)(q + (r > 0));
  return qf < 4194304.0f ? exact : ceilf(qf);
}

// floor(a / b) for 0 <= a < 2^24, 1 <= b < 2^24 (exact).
__device__ __forceinline__ int floor_div_small(int a, int b) {
  int q = (int)(__fdividef((float)a, (float)b));
  q -= (q * b > a);
  q += ((q + 1) * b <= a);
  return q;
}

// ceil(n / 2^s) without overflow
__device__ __forceinline__ uint32_t ceil_shift(uint32_t n, int s) {
  return (n >> s) + ((n & ((1u << s) - 1u)) != 0u);
}

// x / y with y >= 0; +inf where y == 0
__device__ __forceinline__ float div_pos(float x, float y) {
  return y > 0.0f ? __fdividef(x, y) : INFINITY;
}

template <int D1>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&c)[2 * D1]) {
  if constexpr ((2 * D1) % 4 == 0) {
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < (2 * D1) / 4; ++i) {
      const float4 v = __ldg(p4 + i);
      c[4 * i] = v.x;
      c[4 * i + 1] = v.y;
      c[4 * i + 2] = v.z;
      c[4 * i + 3] = v.w;
    }
  } else {
    const float2 *p2 = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      const float2 v = __ldg(p2 + i);
      c[2 * i] = v.x;
      c[2 * i + 1] = v.y;
    }
  }
}

// One thread per query; persistent grid-stride loop.  Every configuration is
// evaluated in registers without data-dependent branches (invalid and pole
// configurations evaluate to +inf), and the running (best, second, argmin) is
// kept in registers, so no cross-thread reduction is needed.
template <int D1>
__global__ void __launch_bounds__(256) search_kernel(ProgramView P, int64_t K, CfgTab cfg, HwC hw,
                                                     const float4 *__restrict__ q, int64_t Q,
                                                     int32_t *__restrict__ argmin,
                                                     float *__restrict__ best,
                                                     float *__restrict__ second,
                                                     int32_t *__restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 q0 = __ldg(q + 2 * i);
    const float4 q1 = __ldg(q + 2 * i + 1);
    const float N = q0.x, nsm = q0.y, fghz = q0.z, memld = q0.w;
    const float bw = q1.x, ddc = q1.y, ddu = q1.z;
    const int32_t kid = __float_as_int(q1.w);
    float b1 = INFINITY, b2 = INFINITY;
    int arg = -1, st = 0;
    const bool finite = isfinite(N) && isfinite(nsm) && isfinite(fghz) && isfinite(memld) &&
                        isfinite(bw) && isfinite(ddc) && isfinite(ddu);
    if (!finite || kid < 0 || kid >= K || !(N >= 1.0f) || !(nsm >= 1.0f) || !(fghz > 0.0f) ||
        !(bw > 0.0f) || !(memld >= 0.0f) || !(ddc >= 0.0f) || !(ddu >= 0.0f) ||
        !(N <= 4294967040.0f) || !(nsm <= 1048576.0f)) {
      st = RP_Q_BAD;
    } else {
      float t[kNmet];
#pragma unroll
      for (int m = 0; m < kNmet; ++m)
        t[m] = fmaf(__ldg(P.aN + kid * kNmet + m), N, __ldg(P.bN + kid * kNmet + m));
      const uint32_t Ni = (uint32_t)ceilf(N);
      const uint32_t nsm_i = (uint32_t)nsm;
      const bool grid1 = __ldg(P.grid + kid) == 1;
      const float *tab = P.table + (int64_t)kid * kNcfg * kNmet * 2 * D1;
      bool any_pole = false;
      for (int c = 0; c < kNcfg; ++c) {
        float mv[kNmet];
        bool pole = false;
        const float *row = tab + c * kNmet * 2 * D1;
#pragma unroll
        for (int m = 0; m < kNmet; ++m) {
          float cf[2 * D1];
          load_row<D1>(row + m * 2 * D1, cf);
          float p = cf[D1 - 1], d = cf[2 * D1 - 1];
#pragma unroll
          for (int j = D1 - 2; j >= 0; --j) {
            p = fmaf(p, t[m], cf[j]);
            d = fmaf(d, t[m], cf[D1 + j]);
          }
          pole |= !(d > 0.0f) || !(d < 8.5e37f);
          mv[m] = __fdividef(p, d);
        }
        const float comp = fmaxf(mv[0], 0.0f), Cm = fmaxf(mv[1], 0.0f),
                    U = fmaxf(mv[2], 0.0f), upm = fmaxf(mv[3], 1.0f),
                    synch = fmaxf(mv[4], 0.0f), lbw = fmaxf(mv[5], 0.0f);
        // clamped at 2^24: above every admissible R_SM / Z_SM (< 2^24), so
        // the configuration is invalid either way
        const float Rf = fminf(fmaxf(mv[6], 0.0f), 16777216.0f);
        const float Zf = fminf(fmaxf(mv[7], 0.0f), 16777216.0f);
        const int Ri = (int)floorf(Rf + 0.5f), Zi = (int)floorf(Zf + 0.5f);
        const int la = cfg.la[c], lb = cfg.lb[c];
        const int T = 1 << (la + lb);
        const int wpb = cfg.wpb[c];
        const int64_t bR = (int64_t)max(Ri, 1) * wpb * hw.warp;
        const int tR = bR > hw.rsm ? 0 : floor_div_small(hw.rsm, (int)bR);
        const int tZ = floor_div_small(hw.zsm, max(Zi, 1));
        int bact = cfg.bact_w[c];
        bact = Ri > 0 ? min(bact, tR) : bact;
        bact = Zi > 0 ? min(bact, tZ) : bact;
        const bool valid = !pole && bact > 0 && (int64_t)Ri * T <= hw.rsm && Zi <= hw.zsm;
        bact = max(bact, 1);
        const float Nw = (float)min(bact * wpb, hw.wmax);
        const uint32_t c0 = grid1 ? ceil_shift(Ni, la + lb) : ceil_shift(Ni, la);
        const uint32_t c1 = grid1 ? 1u : ceil_shift(Ni, lb);
        const bool few = (uint64_t)c0 * c1 < (uint64_t)nsm_i;
        const uint32_t asm_ = few ? c0 * c1 : nsm_i;
        const float rep = rep_count(c0, c1, (uint32_t)bact * asm_);
        const float mem_insts = U + Cm;
        const float comp_cycles = hw.issue * (comp + mem_insts);
        const bool has_mem = mem_insts > 0.0f;
        const float inv_mi = has_mem ? __fdividef(1.0f, mem_insts) : 0.0f;
        const float wu = U * inv_mi, wc = Cm * inv_mi;
        const float ml_unc = fmaf(upm - 1.0f, ddu, memld);
        const float ml = fmaf(ml_unc, wu, memld * wc);
        const float dd = fmaf(ddu * upm, wu, ddc * wc);
        const float mwp_nobw = div_pos(ml, dd);
        const float bwpw = div_pos(fghz * lbw, ml);
        const float mwp_bw = div_pos(bw, bwpw * (float)asm_);
        const float mwp_u = fminf(mwp_nobw, mwp_bw);
        const bool mwp_cap = Nw <= mwp_u;
        const float MWP = fminf(mwp_u, Nw);
        const float mem_cycles = fmaf(ml_unc, U, memld * Cm);
        const float cwp_full = div_pos(mem_cycles + comp_cycles, comp_cycles);
        const bool cwp_cap = Nw <= cwp_full;
        const float CWP = fminf(cwp_full, Nw);
        const float per = comp_cycles * inv_mi;
        const float over = fmaxf(MWP - 1.0f, 0.0f);
        const float cy1 = fmaf(per, over, mem_cycles + comp_cycles);
        const float cy2 = fmaf(per, over, div_pos(mem_cycles * Nw, MWP));
        const float cy3 = fmaf(comp_cycles, Nw, memld);
        const float cyc = (mwp_cap && cwp_cap) ? cy1 : ((CWP >= MWP || comp_cycles > mem_cycles) ? cy2 : cy3);
        const float synch_cost = dd * over * synch * (float)bact;
        float ex = has_mem ? (cyc + synch_cost) * rep : comp_cycles * rep;
        ex = valid ? ex : INFINITY;
        any_pole |= pole;
        const bool better = ex < b1;
        const bool second_better = !better && ex < b2;
        b2 = better ? b1 : (second_better ? ex : b2);
        arg = better ? c : arg;
        b1 = better ? ex : b1;
      }
      st |= any_pole ? RP_Q_POLE : 0;
      if (arg < 0) st |= RP_Q_NO_VALID;
    }
    argmin[i] = arg;
    best[i] = b1;
    second[i] = b2;
    status[i] = st;
  }
}

}  // namespace

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
  }
  return n;
}

namespace {
constexpr int kMaxDev = 16;
SearchShape g_search_shape[kMaxDev][kMaxDeg + 1];
int g_fit_cap[kMaxDev][RP_PREC_BF16X3 + 1][kMaxDeg + 1];
int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
  return dev;
}
}  // namespace

SearchShape search_shape(int degree) {
  SearchShape s = g_search_shape[current_device()][degree];
  if (s.threads <= 0) s = SearchShape{256, 8};
  return s;
}
void set_search_shape(int degree, SearchShape s) { g_search_shape[current_device()][degree] = s; }
int fit_ctas_cap(int precision, int dmax) { return g_fit_cap[current_device()][precision][dmax]; }
void set_fit_ctas_cap(int precision, int dmax, int cap) {
  g_fit_cap[current_device()][precision][dmax] = cap;
}

cudaError_t launch_pack(int64_t K, int d, const double *coef, const double *box,
                        const int8_t *degrees, const int32_t *metric_map, const int32_t *grid_dims,
                        ProgramMut prog, cudaStream_t s) {
  static const ExpTab et = make_exponents();
  const int64_t total = K * kNcfg * kNmet;
  if (total == 0) return cudaSuccess;
  const int threads = 128;
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  pack_kernel<<<(unsigned)blocks, threads, 0, s>>>(K, d, coef, box, degrees, metric_map,
                                                   grid_dims, prog, et);
  return cudaGetLastError();
}

cudaError_t launch_search(ProgramView prog, int64_t K, int d, const rp_hw_fixed &hw,
                          const float *queries, int64_t Q, int32_t *argmin, float *best,
                          float *second, int32_t *status, cudaStream_t s) {
  if (Q == 0) return cudaSuccess;
  CfgTab cfg{};
  int c = 0;
  for (int a = 0; a <= 10; ++a)
    for (int b = 0; b <= 10 - a; ++b, ++c) {
      const int T = 1 << (a + b);
      cfg.la[c] = (int8_t)a;
      cfg.lb[c] = (int8_t)b;
      const int wpb = (T + hw.warp_size - 1) / hw.warp_size;
      cfg.wpb[c] = wpb;
      int bw = hw.b_max < hw.w_max / wpb ? hw.b_max : hw.w_max / wpb;
      cfg.bact_w[c] = (T > hw.t_max) ? 0 : bw;
    }
  HwC h{hw.warp_size, hw.w_max, hw.r_sm, hw.z_sm, hw.issue_cycles};
  const SearchShape shape = search_shape(d);
  const int threads = shape.threads;
  int64_t blocks = (Q + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * shape.ctas_per_sm;
  if (blocks > cap) blocks = cap;
  const float4 *q4 = reinterpret_cast<const float4 *>(queries);
  switch (d + 1) {
    case 1: search_kernel<1><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best, second, status); break;
    case 2: search_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best, second, status); break;
    case 3: search_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best, second, status); break;
    case 4: search_kernel<4><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best, second, status); break;
    case 5: search_kernel<5><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best, second, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rpk
