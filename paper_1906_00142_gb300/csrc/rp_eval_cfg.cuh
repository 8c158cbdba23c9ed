// The per-configuration evaluation of the MWP-CWP rational program (Sec. 2
// Examples 1-2; Sec. 3.3 Step 4) and the helpers the search kernels share.
//
// Included twice: by rp_search.cu (inside namespace rpk's anonymous
// namespace, with <math.h>, <stdint.h> and the constants kNcfg, kNmet of
// rp_internal.cuh in scope), and as text by the program generator
// (rp_codegen.cu), whose generated source defines the same names first and
// is compiled at run time.  It therefore includes nothing and opens no
// namespace.

struct CfgTab {
  int8_t la[kNcfg];        // log2 B0
  int8_t lb[kNcfg];        // log2 B1
  int32_t wpb[kNcfg];      // warps per block, ceil(T / warp)
  int32_t bact_w[kNcfg];   // min(B_max, floor(W_max / wpb)), 0 if T > T_max
  int32_t rsm_w[kNcfg];    // floor(R_SM / (wpb warp)): R <= rsm_w <=> R wpb warp <= R_SM
  int32_t rsm_t[kNcfg];    // floor(R_SM / T): R <= rsm_t <=> R T <= R_SM
};

struct HwC {
  int32_t warp, wmax, rsm, zsm;
  float issue;
};

// #Rep = ceil(c0 c1 / D) for 1 <= c0, c1 < 2^32 and 1 <= D < 2^30.
// The float estimate qf of the quotient is within 6 float roundings (3.6e-7
// relative) of it.  Below 2^20 it is therefore within 0.4 of the quotient,
// so q0 = floor(qf) leaves a remainder r = c0 c1 - q0 D in (-D, 2D), exact in
// 32-bit wrap-around arithmetic, and the ceiling is q0 + [r > 0] + [r > D].
// Above 2^20 ceil(qf) is used (relative error below 1.4e-6).
__device__ __forceinline__ float rep_count(uint32_t c0, uint32_t c1, uint32_t D) {
  const float qf = __fdividef((float)c0 * (float)c1, (float)D);
  const uint32_t q0 = (uint32_t)fminf(qf, 1048576.0f);
  const int32_t r = (int32_t)(c0 * c1 - q0 * D);
  const uint32_t q = q0 + (r > 0 ? 1u : 0u) + (r > (int32_t)D ? 1u : 0u);
  return qf < 1048576.0f ? (float)q : ceilf(qf);
}

// floor(a / b) for 0 <= a < 2^24, 1 <= b < 2^24 (exact).  Below 2^21 the
// quotient of a + 1/2 lies at least 1/(2b) from every integer and
// __fdividef's error (2 ulp, under (a + 1/2) 2^-22 / b) is smaller, so its
// truncation is the floor; above, the estimate is corrected (a is a table or
// hardware constant: the branch is uniform across a warp).
__device__ __forceinline__ int floor_div_small(int a, int b) {
  if (a < (1 << 21)) return (int)__fdividef((float)a + 0.5f, (float)b);
  int q = (int)(__fdividef((float)a, (float)b));
  q -= (q * b > a);
  q += ((q + 1) * b <= a);
  return q;
}

// x / y with y >= 0; +inf where y == 0
__device__ __forceinline__ float div_pos(float x, float y) {
  return y > 0.0f ? __fdividef(x, y) : INFINITY;
}

// Loads of the program's coefficients: read-only global loads, or plain
// loads from a copy staged in shared memory (SH).
template <bool SH>
__device__ __forceinline__ float4 ld4(const float4 *p) {
  if constexpr (SH) return *p;
  else return __ldg(p);
}
template <bool SH>
__device__ __forceinline__ float2 ld2(const float2 *p) {
  if constexpr (SH) return *p;
  else return __ldg(p);
}
template <bool SH>
__device__ __forceinline__ float ld1(const float *p) {
  if constexpr (SH) return *p;
  else return __ldg(p);
}

template <int D1, bool SH>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&c)[2 * D1]) {
  if constexpr ((2 * D1) % 4 == 0) {
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < (2 * D1) / 4; ++i) {
      const float4 v = ld4<SH>(p4 + i);
      c[4 * i] = v.x;
      c[4 * i + 1] = v.y;
      c[4 * i + 2] = v.z;
      c[4 * i + 3] = v.w;
    }
  } else {
    const float2 *p2 = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int i = 0; i < D1; ++i) {
      const float2 v = ld2<SH>(p2 + i);
      c[2 * i] = v.x;
      c[2 * i + 1] = v.y;
    }
  }
}

// The per-query state of the evaluation: the query's scalars and its
// kernel's normalised data parameter per metric.
struct QState {
  float fghz, memld, bw, ddc, ddu;
  float t[kNmet];
  uint32_t Ni, nsm_i;
  bool grid1;
};

// Validates the query and sets up its state; false: a bad query (RP_Q_BAD).
template <bool SH>
__device__ __forceinline__ bool query_state(const float4 q0, const float4 q1, bool kid_ok,
                                            const float *aN8, const float *bN8, int32_t grid,
                                            QState &s) {
  const float N = q0.x, nsm = q0.y;
  s.fghz = q0.z; s.memld = q0.w;
  s.bw = q1.x; s.ddc = q1.y; s.ddu = q1.z;
  const bool finite = isfinite(N) && isfinite(nsm) && isfinite(s.fghz) && isfinite(s.memld) &&
                      isfinite(s.bw) && isfinite(s.ddc) && isfinite(s.ddu);
  if (!finite || !kid_ok || !(N >= 1.0f) || !(nsm >= 1.0f) || !(s.fghz > 0.0f) ||
      !(s.bw > 0.0f) || !(s.memld >= 0.0f) || !(s.ddc >= 0.0f) || !(s.ddu >= 0.0f) ||
      !(N <= 4294967040.0f) || !(nsm <= 1048576.0f))
    return false;
#pragma unroll
  for (int m = 0; m < kNmet; ++m) s.t[m] = fmaf(ld1<SH>(aN8 + m), N, ld1<SH>(bN8 + m));
  s.Ni = (uint32_t)ceilf(N);
  s.nsm_i = (uint32_t)nsm;
  s.grid1 = grid == 1;
  return true;
}

// One configuration c of one query, branch-free: the execution cycles (+inf
// for an invalid or pole configuration), whether a metric's denominator was
// <= 0 (pole), and the occupancy B_active, W_active (0 when not resident).
// The same operations, in the same order, as eval_query's loop body (which
// keeps its own copy: factored out, it costs the benchmarked kernel register
// spills); the tie-break and occupancy tests check that the two agree bit
// for bit.
struct CfgOut {
  float ex;
  bool pole;
  int bact, nw;
};
template <int D1, bool SH, bool OCC = false>
__device__ __forceinline__ CfgOut eval_cfg(int c, const QState &s, const float *tab,
                                           const CfgTab &cfg, const HwC &hw) {
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
      p = fmaf(p, s.t[m], cf[j]);
      d = fmaf(d, s.t[m], cf[D1 + j]);
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
  const int bact_out = OCC ? (valid ? bact : 0) : 0;
  bact = max(bact, 1);
  const int nw_i = min(bact * wpb, hw.wmax);
  const float Nw = (float)nw_i;
  // ceil(N / 2^s) = ((N - 1) >> s) + 1 for N >= 1
  const uint32_t c0 = ((s.Ni - 1u) >> (s.grid1 ? la + lb : la)) + 1u;
  const uint32_t c1 = s.grid1 ? 1u : ((s.Ni - 1u) >> lb) + 1u;
  // fewer blocks than SMs (decided exactly in FP32: below 2^24 the
  // product is exact, above it is >= 2^24 > SMs): every block runs in
  // one round, #Rep = 1
  const float blocks = (float)c0 * (float)c1;
  const bool few = blocks < (float)s.nsm_i;
  const float asm_ = few ? blocks : (float)s.nsm_i;
  const float rep = few ? 1.0f : rep_count(c0, c1, (uint32_t)bact * s.nsm_i);
  const float mem_insts = U + Cm;
  const float comp_cycles = hw.issue * (comp + mem_insts);
  const bool has_mem = mem_insts > 0.0f;
  const float inv_mi = has_mem ? __fdividef(1.0f, mem_insts) : 0.0f;
  const float wu = U * inv_mi, wc = Cm * inv_mi;
  const float ml_unc = fmaf(upm - 1.0f, s.ddu, s.memld);
  const float ml = fmaf(ml_unc, wu, s.memld * wc);
  const float dd = fmaf(s.ddu * upm, wu, s.ddc * wc);
  const float mwp_nobw = div_pos(ml, dd);
  const float bwpw = div_pos(s.fghz * lbw, ml);
  const float mwp_bw = div_pos(s.bw, bwpw * asm_);
  const float mwp_u = fminf(mwp_nobw, mwp_bw);
  const bool mwp_cap = Nw <= mwp_u;
  const float MWP = fminf(mwp_u, Nw);
  const float mem_cycles = fmaf(ml_unc, U, s.memld * Cm);
  const float cwp_full = div_pos(mem_cycles + comp_cycles, comp_cycles);
  const bool cwp_cap = Nw <= cwp_full;
  const float CWP = fminf(cwp_full, Nw);
  const float per = comp_cycles * inv_mi;
  const float over = fmaxf(MWP - 1.0f, 0.0f);
  const float cy1 = fmaf(per, over, mem_cycles + comp_cycles);
  const float cy2 = fmaf(per, over, div_pos(mem_cycles * Nw, MWP));
  const float cy3 = fmaf(comp_cycles, Nw, s.memld);
  const float cyc = (mwp_cap && cwp_cap) ? cy1 : ((CWP >= MWP || comp_cycles > mem_cycles) ? cy2 : cy3);
  const float synch_cost = dd * over * synch * (float)bact;
  float ex = has_mem ? (cyc + synch_cost) * rep : comp_cycles * rep;
  ex = valid ? ex : INFINITY;
  return CfgOut{ex, pole, bact_out, OCC ? (valid ? nw_i : 0) : 0};
}

