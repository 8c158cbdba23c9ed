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

// Index of the monomial N^a B0^b B1^c in the graded-lex order of the fit's
// coefficients (degree ascending, then exponent of N descending, then of B0
// descending): the C(s+2, 3) monomials of lower degree s = a + b + c, then
// (b + c)(b + c + 1) / 2 monomials of degree s with a larger exponent of N,
// then c.
__host__ __device__ constexpr int glex_index(int a, int b, int c) {
  return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// out[a] = sum over b + c <= D - a of cf[glex(a, b, c)] u^b w^c: the
// coefficient of t^a once B0 and B1 are fixed, by nested Horner in u and w
// (one FMA per monomial); only the fit's own nm monomials are read.
template <int D>
__device__ __forceinline__ void fold_b(const double *__restrict__ cf, int nm, double u, double w,
                                       double (&out)[D + 1]) {
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    double acc = 0.0;
#pragma unroll
    for (int b = D - a; b >= 0; --b) {
      double inner = 0.0;
#pragma unroll
      for (int c = D - a - b; c >= 0; --c) {
        const int j = glex_index(a, b, c);
        inner = fma(inner, w, j < nm ? __ldg(cf + j) : 0.0);
      }
      acc = fma(acc, u, inner);
    }
    out[a] = acc;
  }
}

// One thread per (kernel, metric, run of kPackRun consecutive
// configurations): the fit's normalisation of B0 and B1 (two FP64 divisions)
// is set up once for the run; per configuration the normalised B0, B1 cost
// one FMA each and the fold one FMA per monomial.  FP64 arithmetic.  D: the
// program's degree bound.
constexpr int kPackRun = 11;   // 66 configurations = 6 runs
template <int D>
__global__ void pack_kernel(int64_t K, const double *__restrict__ coef,
                            const double *__restrict__ box, const int8_t *__restrict__ degrees,
                            const int32_t *__restrict__ metric_map,
                            const int32_t *__restrict__ grid_dims, ProgramMut prog) {
  constexpr int D1 = D + 1;
  constexpr int kRuns = kNcfg / kPackRun;
  const int64_t total = K * kRuns * kNmet;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int mt = (int)(id % kNmet);
    const int run = (int)((id / kNmet) % kRuns);
    const int64_t k = id / (kNmet * kRuns);
    const int fi = metric_map[k * kNmet + mt];
    // x' = x s + o maps the fit's [lo, hi] to [-1, 1] (0 for a constant variable)
    double s0 = 0.0, o0 = 0.0, s1 = 0.0, o1 = 0.0;
    const double *cf = coef;
    int nm = 0;
    if (fi >= 0) {
      const double *bx = box + 6 * (int64_t)fi;
      if (bx[3] > bx[2]) {
        s0 = 2.0 / (bx[3] - bx[2]);
        o0 = -1.0 - bx[2] * s0;
      }
      if (bx[5] > bx[4]) {
        s1 = 2.0 / (bx[5] - bx[4]);
        o1 = -1.0 - bx[4] * s1;
      }
      cf = coef + (int64_t)fi * kStride;
      nm = num_monomials(degrees[fi]);
    }
    // first configuration of the run -> (a, b) with B0 = 2^a, B1 = 2^b
    int a = 0, b = run * kPackRun;
    while (b >= 11 - a) { b -= 11 - a; ++a; }
    for (int r = 0; r < kPackRun; ++r) {
      const int c = run * kPackRun + r;
      double pn[D1], pd[D1];
      if (fi < 0) {
#pragma unroll
        for (int i = 0; i < D1; ++i) pn[i] = pd[i] = 0.0;
        pd[0] = 1.0;
      } else {
        const double u = fma((double)(1 << a), s0, o0);
        const double w = fma((double)(1 << b), s1, o1);
        fold_b<D>(cf, nm, u, w, pn);
        fold_b<D>(cf + kHalf, nm, u, w, pd);
      }
      float *row = prog.table + ((k * kNcfg + c) * kNmet + mt) * 2 * D1;
#pragma unroll
      for (int i = 0; i < D1; ++i) {
        row[i] = (float)pn[i];
        row[D1 + i] = (float)pd[i];
      }
      if (++b > 10 - a) {   // next configuration: b ascending, then a
        b = 0;
        ++a;
      }
    }
    if (run == 0) {
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

#include "rp_eval_cfg.cuh"

// The evaluate-and-argmin of one query (Sec. 3.3 Steps 4-5): every
// configuration is evaluated in registers without data-dependent branches
// (invalid and pole configurations evaluate to +inf) and the running (best,
// second, argmin) is kept in registers.  aN8, bN8, grid and tab are the
// query's kernel's sections of the program (global memory, or a shared-memory
// copy when SH); kid_ok: the query's kernel id names a kernel of the program.
template <int D1, bool SH>
__device__ __forceinline__ void eval_query(const float4 q0, const float4 q1, bool kid_ok,
                                           const float *aN8, const float *bN8, int32_t grid,
                                           const float *tab, const CfgTab &cfg, const HwC &hw,
                                           int &arg_out, float &b1_out, float &b2_out,
                                           int &st_out) {
  const float N = q0.x, nsm = q0.y, fghz = q0.z, memld = q0.w;
  const float bw = q1.x, ddc = q1.y, ddu = q1.z;
  float b1 = INFINITY, b2 = INFINITY;
  int arg = -1, st = 0;
  const bool finite = isfinite(N) && isfinite(nsm) && isfinite(fghz) && isfinite(memld) &&
                      isfinite(bw) && isfinite(ddc) && isfinite(ddu);
  if (!finite || !kid_ok || !(N >= 1.0f) || !(nsm >= 1.0f) || !(fghz > 0.0f) ||
      !(bw > 0.0f) || !(memld >= 0.0f) || !(ddc >= 0.0f) || !(ddu >= 0.0f) ||
      !(N <= 4294967040.0f) || !(nsm <= 1048576.0f)) {
    st = RP_Q_BAD;
  } else {
    float t[kNmet];
#pragma unroll
    for (int m = 0; m < kNmet; ++m) t[m] = fmaf(ld1<SH>(aN8 + m), N, ld1<SH>(bN8 + m));
    const uint32_t Ni = (uint32_t)ceilf(N);
    const uint32_t nsm_i = (uint32_t)nsm;
    const bool grid1 = grid == 1;
    bool any_pole = false;
    for (int c = 0; c < kNcfg; ++c) {
      float mv[kNmet];
      unsigned dbits = 0u;
      const float *row = tab + c * kNmet * 2 * D1;
#pragma unroll
      for (int m = 0; m < kNmet; ++m) {
        float cf[2 * D1];
        load_row<D1, SH>(row + m * 2 * D1, cf);
        float p = cf[D1 - 1], d = cf[2 * D1 - 1];
#pragma unroll
        for (int j = D1 - 2; j >= 0; --j) {
          p = fmaf(p, t[m], cf[j]);
          d = fmaf(d, t[m], cf[D1 + j]);
        }
        // 0 < d < 8.5e37 (NaN excluded) <=> bits(d) - 1 < bits(8.5e37) - 1,
        // unsigned: one running maximum instead of two compares per metric
        dbits = max(dbits, __float_as_uint(d) - 1u);
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
      const bool pole = dbits >= __float_as_uint(8.5e37f) - 1u;
      const int la = cfg.la[c], lb = cfg.lb[c];
      const int wpb = cfg.wpb[c];
      // floor(R_SM / (R wpb warp)) = floor(floor(R_SM / (wpb warp)) / R)
      const int tR = floor_div_small(cfg.rsm_w[c], max(Ri, 1));
      const int tZ = floor_div_small(hw.zsm, max(Zi, 1));
      int bact = cfg.bact_w[c];
      bact = Ri > 0 ? min(bact, tR) : bact;
      bact = Zi > 0 ? min(bact, tZ) : bact;
      const bool valid = !pole && bact > 0 && Ri <= cfg.rsm_t[c] && Zi <= hw.zsm;
      bact = max(bact, 1);
      const float Nw = (float)min(bact * wpb, hw.wmax);
      // ceil(N / 2^s) = ((N - 1) >> s) + 1 for N >= 1
      const uint32_t c0 = ((Ni - 1u) >> (grid1 ? la + lb : la)) + 1u;
      const uint32_t c1 = grid1 ? 1u : ((Ni - 1u) >> lb) + 1u;
      // fewer blocks than SMs (decided exactly in FP32: below 2^24 the
      // product is exact, above it is >= 2^24 > SMs): every block runs in
      // one round, #Rep = 1
      const float blocks = (float)c0 * (float)c1;
      const bool few = blocks < (float)nsm_i;
      const float asm_ = few ? blocks : (float)nsm_i;
      const float rep = few ? 1.0f : rep_count(c0, c1, (uint32_t)bact * nsm_i);
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
      const float mwp_bw = div_pos(bw, bwpw * asm_);
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
  arg_out = arg;
  b1_out = b1;
  b2_out = b2;
  st_out = st;
}

// eval_query with Step 5's choice among several optimal configurations made
// by a second metric: of the configurations within (1 + tie_rel) of the
// best cycles, the one with the most active warps per SM (lowest index among
// equals), found in a second pass over the configurations.  The first pass
// gives the same best, second and (before the choice) argmin as eval_query.
template <int D1, bool SH, bool TIE>
__device__ __forceinline__ void eval_query_tie(const float4 q0, const float4 q1, bool kid_ok,
                                           const float *aN8, const float *bN8, int32_t grid,
                                           const float *tab, const CfgTab &cfg, const HwC &hw,
                                           int &arg_out, float &b1_out, float &b2_out,
                                           int &st_out, float tie_rel = 0.0f) {
  float b1 = INFINITY, b2 = INFINITY;
  int arg = -1, st = 0;
  QState s;
  if (!query_state<SH>(q0, q1, kid_ok, aN8, bN8, grid, s)) {
    st = RP_Q_BAD;
  } else {
    bool any_pole = false;
    for (int c = 0; c < kNcfg; ++c) {
      const CfgOut o = eval_cfg<D1, SH>(c, s, tab, cfg, hw);
      any_pole |= o.pole;
      const float ex = o.ex;
      const bool better = ex < b1;
      const bool second_better = !better && ex < b2;
      b2 = better ? b1 : (second_better ? ex : b2);
      arg = better ? c : arg;
      b1 = better ? ex : b1;
    }
    if (TIE) {
      if (arg >= 0) {
        const float lim = b1 * (1.0f + tie_rel);
        int best_nw = -1;
        for (int c = 0; c < kNcfg; ++c) {
          const CfgOut o = eval_cfg<D1, SH, true>(c, s, tab, cfg, hw);
          const bool take = o.ex <= lim && o.nw > best_nw;
          best_nw = take ? o.nw : best_nw;
          arg = take ? c : arg;
        }
      }
    }
    st |= any_pole ? RP_Q_POLE : 0;
    if (arg < 0) st |= RP_Q_NO_VALID;
  }
  arg_out = arg;
  b1_out = b1;
  b2_out = b2;
  st_out = st;
}

// Occupancy of every configuration of every query (Sec. 2 Example 1, as a
// rational program of the fitted registers per thread and shared words per
// block): B_active and W_active per (query, configuration), 0 where the
// configuration is not resident, invalid or a pole; a bad query gets 0
// everywhere and RP_Q_BAD.  One thread per query.
template <int D1>
__global__ void __launch_bounds__(256) occupancy_kernel(ProgramView P, int64_t K,
                                                        const __grid_constant__ CfgTab cfg, HwC hw,
                                                        const float4 *__restrict__ q, int64_t Q,
                                                        int32_t *__restrict__ b_active,
                                                        int32_t *__restrict__ w_active,
                                                        int32_t *__restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 q0 = __ldg(q + 2 * i);
    const float4 q1 = __ldg(q + 2 * i + 1);
    const int32_t kid = __float_as_int(q1.w);
    const bool kid_ok = kid >= 0 && kid < K;
    const int64_t k = kid_ok ? kid : 0;
    QState s;
    const bool ok = query_state<false>(q0, q1, kid_ok, P.aN + k * kNmet, P.bN + k * kNmet,
                                       kid_ok ? __ldg(P.grid + k) : 0, s);
    const float *tab = P.table + k * kNcfg * kNmet * 2 * D1;
    int st = ok ? 0 : RP_Q_BAD;
    for (int c = 0; c < kNcfg; ++c) {
      CfgOut o = CfgOut{INFINITY, false, 0, 0};
      if (ok) o = eval_cfg<D1, false, true>(c, s, tab, cfg, hw);
      st |= o.pole ? RP_Q_POLE : 0;
      b_active[i * kNcfg + c] = o.bact;
      w_active[i * kNcfg + c] = o.nw;
    }
    status[i] = st;
  }
}

// One thread per query, queries in input order; persistent grid-stride
// loop.  Each query gathers its kernel's table rows from global memory (L2).
template <int D1, bool TIE>
__global__ void __launch_bounds__(256) search_kernel(ProgramView P, int64_t K,
                                                     const __grid_constant__ CfgTab cfg, HwC hw,
                                                     const float4 *__restrict__ q, int64_t Q,
                                                     int32_t *__restrict__ argmin,
                                                     float *__restrict__ best,
                                                     float *__restrict__ second,
                                                     int32_t *__restrict__ status, float tie_rel) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 q0 = __ldg(q + 2 * i);
    const float4 q1 = __ldg(q + 2 * i + 1);
    const int32_t kid = __float_as_int(q1.w);
    const bool kid_ok = kid >= 0 && kid < K;
    const int64_t k = kid_ok ? kid : 0;
    int arg, st;
    float b1, b2;
    if constexpr (TIE)
      eval_query_tie<D1, false, true>(q0, q1, kid_ok, P.aN + k * kNmet, P.bN + k * kNmet,
                                      kid_ok ? __ldg(P.grid + k) : 0,
                                      P.table + k * kNcfg * kNmet * 2 * D1, cfg, hw, arg, b1, b2,
                                      st, tie_rel);
    else
      eval_query<D1, false>(q0, q1, kid_ok, P.aN + k * kNmet, P.bN + k * kNmet,
                            kid_ok ? __ldg(P.grid + k) : 0,
                            P.table + k * kNcfg * kNmet * 2 * D1, cfg, hw, arg, b1, b2, st);
    argmin[i] = arg;
    best[i] = b1;
    second[i] = b2;
    status[i] = st;
  }
}

// ---------------------------------------------------------------------
// Grouped search: the queries are bucketed by kernel id on the device
// (count, exclusive scan, scatter of query indices), then each CTA takes a
// tile of consecutive bucketed positions, stages the table of each kernel
// that occurs in the tile in shared memory once, and evaluates that
// kernel's queries from there (every lane of a warp reads the same row:
// shared-memory broadcasts).  Bucket K collects queries whose kernel id is
// out of range.  Results do not depend on the order within a bucket.

// bucket of query i: its kernel id, or K if out of range
__device__ __forceinline__ int query_bucket(const float *__restrict__ q, int64_t i, int64_t K) {
  const int32_t kid = __float_as_int(__ldg(q + 8 * i + 7));
  return (kid >= 0 && kid < K) ? kid : (int)K;
}

constexpr int kBucketSmem = 8192;   // buckets counted in shared memory up to this many

// cnt[b] += number of queries in bucket b (cnt zeroed by the caller)
__global__ void bucket_count_kernel(const float *__restrict__ q, int64_t Q, int64_t K,
                                    int32_t *__restrict__ cnt) {
  extern __shared__ int32_t hist[];
  const bool local = K + 1 <= kBucketSmem;
  if (local)
    for (int j = threadIdx.x; j <= K; j += blockDim.x) hist[j] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // whole warps iterate (blockDim.x is a multiple of 32, so a warp's 32
  // indices are consecutive): the loop condition is the same for every lane
  // and every warp-collective call below uses the full mask; lanes past Q
  // take the bucket -1, which no query has, and do nothing
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - lane < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    // warp-aggregated: one atomic per distinct bucket in the warp (queries
    // in kernel order would otherwise serialise 32 atomics on one counter)
    const bool valid = i < Q;
    const int b = valid ? query_bucket(q, i, K) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (valid && lane == __ffs(peers) - 1) {
      if (local) atomicAdd(&hist[b], __popc(peers));
      else atomicAdd(&cnt[b], __popc(peers));
    }
  }
  __syncthreads();
  if (local)
    for (int j = threadIdx.x; j <= K; j += blockDim.x)
      if (hist[j]) atomicAdd(&cnt[j], hist[j]);
}

// In place: off[0..n) counts -> off[0..n] exclusive offsets (off[n] = total);
// cur[0..n) = off[0..n) (the scatter's cursors).  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) bucket_scan_kernel(int32_t *__restrict__ off,
                                                           int32_t *__restrict__ cur, int n) {
  __shared__ int32_t wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t carry = 0;
  for (int base = 0; base < n; base += 1024) {
    const int j = base + threadIdx.x;
    const int32_t v = j < n ? off[j] : 0;
    int32_t x = v;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int32_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int32_t before = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    if (j < n) {
      off[j] = before;
      cur[j] = before;
    }
    carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

// perm[cur[b]++] = i for every query i of bucket b
__global__ void bucket_scatter_kernel(const float *__restrict__ q, int64_t Q, int64_t K,
                                      int32_t *__restrict__ cur, int32_t *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  // whole warps iterate, as in bucket_count_kernel (full-mask collectives;
  // lanes past Q: bucket -1, no claim, no write)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - lane < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    // warp-aggregated: the lowest lane of each bucket's group claims the
    // group's slots, the others take consecutive ones after it
    const bool valid = i < Q;
    const int b = valid ? query_bucket(q, i, K) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&cur[b], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) perm[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
  }
}

// Dynamic shared memory of the grouped kernel: one kernel's table, its aN
// and bN, and one bucket id per thread.
template <int D1>
__host__ __device__ constexpr int grouped_table_floats() { return kNcfg * kNmet * 2 * D1; }
template <int D1>
size_t grouped_smem(int threads) {
  return (size_t)(grouped_table_floats<D1>() + 2 * kNmet) * sizeof(float) + (size_t)threads * 4;
}

template <int D1, bool TIE>
__global__ void __launch_bounds__(256, 3) search_grouped_kernel(
    ProgramView P, int64_t K, const __grid_constant__ CfgTab cfg, HwC hw,
    const float4 *__restrict__ q, int64_t Q, const int32_t *__restrict__ perm,
    int32_t *__restrict__ argmin, float *__restrict__ best, float *__restrict__ second,
    int32_t *__restrict__ status, float tie_rel) {
  constexpr int TF = grouped_table_floats<D1>();
  extern __shared__ float4 smem4[];
  float *tab_s = reinterpret_cast<float *>(smem4);   // TF floats (a multiple of 4)
  float *ab_s = tab_s + TF;                           // aN[8], bN[8]
  int32_t *bk_s = reinterpret_cast<int32_t *>(ab_s + 2 * kNmet);
  __shared__ int32_t grid_s;
  const int T = blockDim.x;
  const int64_t ntiles = (Q + T - 1) / T;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * T + threadIdx.x;
    const bool act = p < Q;
    int32_t qi = 0;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
    int b = (int)K + 1;   // past every bucket: inactive
    if (act) {
      qi = __ldg(perm + p);
      q0 = __ldg(q + 2 * (int64_t)qi);
      q1 = __ldg(q + 2 * (int64_t)qi + 1);
      const int32_t kid = __float_as_int(q1.w);
      b = (kid >= 0 && kid < K) ? kid : (int)K;
    }
    bk_s[threadIdx.x] = b;
    __syncthreads();
    // the tile's positions are bucket-sorted with the inactive ones last:
    // one run per bucket present
    for (int pos = 0; pos < T;) {
      const int cb = bk_s[pos];
      if (cb > K) break;
      const int nrun = __syncthreads_count(b == cb);
      if (cb < K) {
        const float4 *src = reinterpret_cast<const float4 *>(P.table + (int64_t)cb * TF);
        for (int j = threadIdx.x; j < TF / 4; j += T) smem4[j] = __ldg(src + j);
        if (threadIdx.x < 2 * kNmet)
          ab_s[threadIdx.x] = threadIdx.x < kNmet ? __ldg(P.aN + (int64_t)cb * kNmet + threadIdx.x)
                                                  : __ldg(P.bN + (int64_t)cb * kNmet + threadIdx.x - kNmet);
        if (threadIdx.x == 0) grid_s = __ldg(P.grid + cb);
        __syncthreads();
      }
      if (b == cb) {
        int arg, st;
        float b1, b2;
        if constexpr (TIE)
          eval_query_tie<D1, true, true>(q0, q1, cb < K, ab_s, ab_s + kNmet, grid_s, tab_s, cfg, hw,
                                         arg, b1, b2, st, tie_rel);
        else
          eval_query<D1, true>(q0, q1, cb < K, ab_s, ab_s + kNmet, grid_s, tab_s, cfg, hw, arg, b1,
                               b2, st);
        argmin[qi] = arg;
        best[qi] = b1;
        second[qi] = b2;
        status[qi] = st;
      }
      __syncthreads();   // the next run restages the table
      pos += nrun;
    }
    __syncthreads();     // bk_s is rewritten by the next tile
  }
}

// Error % of a chosen configuration (Sec. 5): per query, over the finite
// runtimes of its 66 configurations, B = the smallest, W = the largest, and
// (t[choice] - B) / (W - B) * 100 (0 when W == B).  One thread per query.
__global__ void error_pct_kernel(const float *__restrict__ rt, const int32_t *__restrict__ choice,
                                 int64_t Q, float *__restrict__ err, int32_t *__restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float *r = rt + i * kNcfg;
    float lo = INFINITY, hi = -INFINITY;
    for (int c = 0; c < kNcfg; ++c) {
      const float v = __ldg(r + c);
      if (isfinite(v)) {
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
      }
    }
    const int32_t c = __ldg(choice + i);
    int st = 0;
    float e = NAN;
    if (!(lo <= hi)) {
      st = RP_EP_NO_RUNTIME;
    } else if (c < 0 || c >= kNcfg || !isfinite(__ldg(r + c))) {
      st = RP_EP_BAD_CHOICE;
    } else {
      const float t = __ldg(r + c);
      e = hi > lo ? (t - lo) / (hi - lo) * 100.0f : 0.0f;
    }
    err[i] = e;
    status[i] = st;
  }
}

}  // namespace

cudaError_t launch_error_pct(const float *runtimes, const int32_t *choice, int64_t Q,
                             float *err_pct, int32_t *status, cudaStream_t s) {
  if (Q == 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (Q + threads - 1) / threads;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  error_pct_kernel<<<(unsigned)blocks, threads, 0, s>>>(runtimes, choice, Q, err_pct, status);
  return cudaGetLastError();
}

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
  static_assert(kNcfg % kPackRun == 0, "whole runs of configurations");
  const int64_t total = K * (kNcfg / kPackRun) * kNmet;
  if (total == 0) return cudaSuccess;
  const int threads = 128;
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  switch (d) {
    case 1: pack_kernel<1><<<(unsigned)blocks, threads, 0, s>>>(K, coef, box, degrees, metric_map, grid_dims, prog); break;
    case 2: pack_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(K, coef, box, degrees, metric_map, grid_dims, prog); break;
    case 3: pack_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(K, coef, box, degrees, metric_map, grid_dims, prog); break;
    case 4: pack_kernel<4><<<(unsigned)blocks, threads, 0, s>>>(K, coef, box, degrees, metric_map, grid_dims, prog); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Workspace of the grouped search: offsets int32[K+2], cursors int32[K+1],
// the bucketed query indices int32[Q], each section 16-byte aligned.  0 (no
// grouping) for fewer than kGroupMinPerKernel queries per kernel on average
// (a tile would then stage a table for only a few queries) or sizes that
// int32 positions cannot index.
constexpr int64_t kGroupMinPerKernel = 32;
size_t search_workspace_bytes(int64_t K, int64_t Q) {
  if (Q <= 0 || K < 1 || Q >= ((int64_t)1 << 31) - 1 || K >= ((int64_t)1 << 30) ||
      Q < kGroupMinPerKernel * K)
    return 0;
  return align16((size_t)(K + 2) * 4) + align16((size_t)(K + 1) * 4) + align16((size_t)Q * 4);
}

template <int D1, bool TIE>
static cudaError_t launch_d(ProgramView prog, int64_t K, const CfgTab &cfg, const HwC &h,
                            const float *queries, int64_t Q, int32_t *argmin, float *best,
                            float *second, int32_t *status, void *ws, cudaStream_t s,
                            float tie_rel) {
  const SearchShape shape = search_shape(D1 - 1);
  const int threads = shape.threads;
  const float4 *q4 = reinterpret_cast<const float4 *>(queries);
  int64_t blocks = (Q + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * shape.ctas_per_sm;
  if (blocks > cap) blocks = cap;
  if (!ws) {
    search_kernel<D1, TIE><<<(unsigned)blocks, threads, 0, s>>>(prog, K, cfg, h, q4, Q, argmin, best,
                                                                second, status, tie_rel);
    return cudaGetLastError();
  }
  unsigned char *w = static_cast<unsigned char *>(ws);
  int32_t *off = reinterpret_cast<int32_t *>(w);
  int32_t *cur = reinterpret_cast<int32_t *>(w + align16((size_t)(K + 2) * 4));
  int32_t *perm = reinterpret_cast<int32_t *>(w + align16((size_t)(K + 2) * 4) +
                                              align16((size_t)(K + 1) * 4));
  cudaError_t e = cudaMemsetAsync(off, 0, (size_t)(K + 1) * 4, s);
  if (e != cudaSuccess) return e;
  const int bt = 512;
  int64_t bb = (Q + bt - 1) / bt;
  if (bb > (int64_t)num_sms() * 4) bb = (int64_t)num_sms() * 4;
  const size_t hist = K + 1 <= kBucketSmem ? (size_t)(K + 1) * 4 : 0;
  bucket_count_kernel<<<(unsigned)bb, bt, hist, s>>>(queries, Q, K, off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bucket_scan_kernel<<<1, 1024, 0, s>>>(off, cur, (int)(K + 1));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bucket_scatter_kernel<<<(unsigned)bb, bt, 0, s>>>(queries, Q, K, cur, perm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  search_grouped_kernel<D1, TIE><<<(unsigned)blocks, threads, grouped_smem<D1>(threads), s>>>(
      prog, K, cfg, h, q4, Q, perm, argmin, best, second, status, tie_rel);
  return cudaGetLastError();
}

// Per-configuration constants of the occupancy arithmetic (host).
static CfgTab make_cfg(const rp_hw_fixed &hw);

void search_cfg_table(const rp_hw_fixed &hw, int8_t *la, int8_t *lb, int32_t *wpb, int32_t *bact_w,
                      int32_t *rsm_w, int32_t *rsm_t) {
  const CfgTab c = make_cfg(hw);
  for (int i = 0; i < kNcfg; ++i) {
    la[i] = c.la[i];
    lb[i] = c.lb[i];
    wpb[i] = c.wpb[i];
    bact_w[i] = c.bact_w[i];
    rsm_w[i] = c.rsm_w[i];
    rsm_t[i] = c.rsm_t[i];
  }
}

static CfgTab make_cfg(const rp_hw_fixed &hw) {
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
      const int64_t wpbw = (int64_t)wpb * hw.warp_size;
      cfg.rsm_w[c] = (int32_t)(hw.r_sm / wpbw);
      cfg.rsm_t[c] = hw.r_sm / T;
    }
  return cfg;
}

template <int D1>
static cudaError_t launch_occ_d(ProgramView prog, int64_t K, const CfgTab &cfg, const HwC &h,
                                const float *queries, int64_t Q, int32_t *b_active,
                                int32_t *w_active, int32_t *status, cudaStream_t s) {
  const int threads = 128;
  int64_t blocks = (Q + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  occupancy_kernel<D1><<<(unsigned)blocks, threads, 0, s>>>(
      prog, K, cfg, h, reinterpret_cast<const float4 *>(queries), Q, b_active, w_active, status);
  return cudaGetLastError();
}

cudaError_t launch_occupancy(ProgramView prog, int64_t K, int d, const rp_hw_fixed &hw,
                             const float *queries, int64_t Q, int32_t *b_active, int32_t *w_active,
                             int32_t *status, cudaStream_t s) {
  if (Q == 0) return cudaSuccess;
  const CfgTab cfg = make_cfg(hw);
  HwC h{hw.warp_size, hw.w_max, hw.r_sm, hw.z_sm, hw.issue_cycles};
  switch (d + 1) {
    case 1: return launch_occ_d<1>(prog, K, cfg, h, queries, Q, b_active, w_active, status, s);
    case 2: return launch_occ_d<2>(prog, K, cfg, h, queries, Q, b_active, w_active, status, s);
    case 3: return launch_occ_d<3>(prog, K, cfg, h, queries, Q, b_active, w_active, status, s);
    case 4: return launch_occ_d<4>(prog, K, cfg, h, queries, Q, b_active, w_active, status, s);
    case 5: return launch_occ_d<5>(prog, K, cfg, h, queries, Q, b_active, w_active, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_search(ProgramView prog, int64_t K, int d, const rp_hw_fixed &hw,
                          const float *queries, int64_t Q, int32_t *argmin, float *best,
                          float *second, int32_t *status, void *workspace, cudaStream_t s,
                          float tie_rel) {
  if (Q == 0) return cudaSuccess;
  const CfgTab cfg = make_cfg(hw);
  HwC h{hw.warp_size, hw.w_max, hw.r_sm, hw.z_sm, hw.issue_cycles};
  void *ws = search_workspace_bytes(K, Q) > 0 ? workspace : nullptr;
  const bool tie = tie_rel >= 0.0f;
#define RP_LAUNCH(D1)                                                                          \
  return tie ? launch_d<D1, true>(prog, K, cfg, h, queries, Q, argmin, best, second, status, ws, s, \
                                  tie_rel)                                                     \
             : launch_d<D1, false>(prog, K, cfg, h, queries, Q, argmin, best, second, status, ws,   \
                                   s, tie_rel)
  switch (d + 1) {
    case 1: RP_LAUNCH(1);
    case 2: RP_LAUNCH(2);
    case 3: RP_LAUNCH(3);
    case 4: RP_LAUNCH(4);
    case 5: RP_LAUNCH(5);
    default: return cudaErrorInvalidValue;
  }
#undef RP_LAUNCH
}

}  // namespace rpk
