// Fit launch interface shared by the fit translation units: the kernel
// arguments and one launcher / residency query per precision family (each
// family is compiled in its own translation unit, rp_fit_<family>.cu).
#pragma once
#include <stdint.h>

#include "rp_internal.cuh"

namespace rpk {

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
  unsigned long long *counter;   // dynamic fit schedule (workspace), or null
  int deg_lo, deg_hi;            // degrees this launch fits (valid ones outside: skipped)
  // Fits the FP32 and tensor-core kernels cannot finish (pivots dropped at
  // their drop tolerance, or refinement stopped short of tol) are solved
  // again by the FP64 kernel: esc_mode 1 marks them (kPending64) and counts
  // them in *esc_count (workspace, or null); esc_mode 2 (the FP64 kernel)
  // fits only marked fits, and returns at once when *esc_count is 0.
  int esc_mode;
  unsigned long long *esc_count;
  // shared sample points: null, or int64 [ceil(F / fits_per_set) + 1]
  // offsets into x (float [3][num_points]); fit f uses point set
  // f / fits_per_set and its values y[off[f] .. off[f+1])
  const int64_t *point_off;
  int64_t num_points;
  int fits_per_set;
  int set_parts;      // claims per point set (its fits split into this many runs)
  int svd;            // solve by the SVD route (Jacobi) instead of the sweep
  // basis cache of the accurate refinement passes (FP32 paths): one slab
  // per CTA of kCacheSamples x ceil(NM / 2) float4 (the basis pairs of a
  // point set's samples), or null; the bytes available from psi_cache
  float4 *psi_cache;
  size_t psi_cache_bytes;
};

// samples per point set whose basis values the cache holds (the kernels'
// shared-memory sample cache size)
constexpr int kCacheSamples = 512;
// offset of the basis cache in the workspace (after the two counters)
constexpr size_t kCacheOffset = 256;

constexpr int32_t kPending64 = 1 << 25;   // status bit between the two launches

// Real = double, design Gram on CUDA cores (RP_PREC_FP64)
cudaError_t fit_launch_f64(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_f64(int dmax);
// Real = float: CUDA-core Gram (FP32), tcgen05 TF32, split TF32, BF16, split BF16
cudaError_t fit_launch_f32(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_f32(int dmax);
cudaError_t fit_launch_tf32(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_tf32(int dmax);
cudaError_t fit_launch_tf32x3(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_tf32x3(int dmax);
cudaError_t fit_launch_bf16(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_bf16(int dmax);
cudaError_t fit_launch_bf16x3(const FitArgs &a, int dmax, int precision, cudaStream_t s);
int fit_residency_bf16x3(int dmax);

}  // namespace rpk
