// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rp.h"

namespace rpk {

constexpr int kMaxDeg = RP_MAX_DEGREE;
constexpr int kMaxNm = 35;                 // monomials of total degree <= 4 in 3 variables
constexpr int kStride = RP_COEF_STRIDE;    // 70
constexpr int kHalf = kStride / 2;         // beta offset
constexpr int kNcfg = RP_NUM_CONFIGS;      // 66
constexpr int kNmet = RP_NUM_METRICS;      // 8

__host__ __device__ inline int num_monomials(int d) { return (d + 1) * (d + 2) * (d + 3) / 6; }

// Packed program sections (see rp_program_size in rp.h).
struct ProgramView {
  const float *aN;       // [K][8]
  const float *bN;       // [K][8]
  const int32_t *grid;   // [K]
  const float *table;    // [K][66][8][2][d+1]
};
struct ProgramMut {
  float *aN;
  float *bN;
  int32_t *grid;
  float *table;
};

inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

inline size_t program_size(int64_t K, int d) {
  size_t s = align16(sizeof(float) * K * kNmet) * 2 + align16(sizeof(int32_t) * K);
  s += sizeof(float) * (size_t)K * kNcfg * kNmet * 2 * (d + 1);
  return s;
}

template <class V, class B>
inline V program_sections(B *base, int64_t K) {
  char *p = (char *)base;
  V v;
  v.aN = (decltype(v.aN))p;
  p += align16(sizeof(float) * K * kNmet);
  v.bN = (decltype(v.bN))p;
  p += align16(sizeof(float) * K * kNmet);
  v.grid = (decltype(v.grid))p;
  p += align16(sizeof(int32_t) * K);
  v.table = (decltype(v.table))p;
  return v;
}

// Host-side launchers (return the CUDA error of the launch).
cudaError_t launch_pack(int64_t K, int d, const double *coef, const double *box,
                        const int8_t *degrees, const int32_t *metric_map, const int32_t *grid_dims,
                        ProgramMut prog, cudaStream_t s);

// workspace: NULL (queries in input order) or search_workspace_bytes(K, Q)
// bytes, 16-byte aligned (queries bucketed by kernel first); ignored when
// search_workspace_bytes is 0.
// tie_rel >= 0: Step 5's second-metric choice among the configurations within
// (1 + tie_rel) of the best (the most active warps; lowest index among equals).
cudaError_t launch_search(ProgramView prog, int64_t K, int d, const rp_hw_fixed &hw,
                          const float *queries, int64_t Q, int32_t *argmin, float *best,
                          float *second, int32_t *status, void *workspace, cudaStream_t s,
                          float tie_rel = -1.0f);
cudaError_t launch_occupancy(ProgramView prog, int64_t K, int d, const rp_hw_fixed &hw,
                             const float *queries, int64_t Q, int32_t *b_active, int32_t *w_active,
                             int32_t *status, cudaStream_t s);
cudaError_t launch_error_pct(const float *runtimes, const int32_t *choice, int64_t Q,
                             float *err_pct, int32_t *status, cudaStream_t s);
// The rational program of one kernel as generated source (rp_codegen.cu).
std::string codegen_source(const void *program_host, int64_t K, int d, int64_t kid,
                           const rp_hw_fixed &hw);
int codegen_compile(const char *src, void **handle, char *log, size_t log_len);
cudaError_t codegen_search(void *handle, const float *queries, int64_t Q, int32_t *argmin,
                           float *best, float *second, int32_t *status, cudaStream_t s);
void codegen_free(void *handle);
// The search's per-configuration constants for hw (host; 66 entries each).
void search_cfg_table(const rp_hw_fixed &hw, int8_t *la, int8_t *lb, int32_t *wpb, int32_t *bact_w,
                      int32_t *rsm_w, int32_t *rsm_t);
size_t search_workspace_bytes(int64_t K, int64_t Q);

cudaError_t launch_fit(const rp_fit_desc &desc, const float *x, const float *y,
                       const int64_t *fit_off, double *coef, float *coef32, double *box,
                       int32_t *status, int32_t *rank, void *workspace, size_t workspace_bytes,
                       cudaStream_t s);
size_t fit_workspace_bytes(const rp_fit_desc &desc);
size_t fit_cache_workspace_bytes(const rp_fit_desc &desc);   // + the basis cache
cudaError_t fit_static_scratch(void **ptr, size_t *bytes);   // rp_fit_noalloc's scratch
bool fit_precision_supported(int precision);
int fit_max_ctas_per_sm(const rp_fit_desc &desc);   // residency limit of the launch desc selects

// Launch shapes chosen by the autotuner, per device (0 = built-in default).
struct SearchShape {
  int threads;        // threads per CTA (<= 256)
  int ctas_per_sm;    // persistent grid = SMs x this
};
SearchShape search_shape(int degree);
void set_search_shape(int degree, SearchShape s);
int fit_ctas_cap(int precision, int dmax);           // 0: the residency limit
void set_fit_ctas_cap(int precision, int dmax, int cap);

cudaError_t launch_relmse(bool backward, int64_t F, int64_t S, const float *x, const float *y,
                          const int64_t *fit_off, const int8_t *degrees, const double *coef,
                          const double *box, const float *grad_loss, float *out,
                          cudaStream_t s);

cudaError_t launch_adam(int64_t n, double *p, const float *g, float *m, float *v,
                        const uint8_t *mask, int t, float lr, float b1, float b2, float eps,
                        cudaStream_t s);

int num_sms();

}  // namespace rpk
