// Batched least-squares fitting of rational functions (Sec. 4.2): the host
// side of rp_fit -- argument bundling, dispatch to the precision family's
// launcher (rp_fit_<family>.cu, kernel in rp_fit_kernel.cuh), the optional
// workspace of the dynamic fit schedule and rp_fit_noalloc's static scratch.
#include <stdint.h>

#include "rp_fit.cuh"

namespace rpk {

// Scratch of rp_fit_noalloc: the dynamic schedule's counter in a statically
// allocated device array (one per process and device; calls that overlap
// in time share it).
static __device__ __align__(256) unsigned long long g_fit_scratch[4];

cudaError_t fit_static_scratch(void **ptr, size_t *bytes) {
  static void *addr[16] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fit_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  *bytes = sizeof(g_fit_scratch);
  return cudaSuccess;
}

// Two 64-bit counters, 16 bytes apart: the dynamic fit schedule's claims
// and the number of fits passed on to the FP64 path.
size_t fit_workspace_bytes(const rp_fit_desc &desc) { return desc.num_fits > 0 ? 32 : 0; }

// The counters, then (FP32 and tensor-core precisions) one basis-cache slab
// per resident CTA of the largest launch the batch makes: kCacheSamples
// samples x ceil(NM / 2) float4, NM the launch's monomial count.  The FP32
// degree-4 variant keeps no sample cache and takes no slab.
size_t fit_cache_workspace_bytes(const rp_fit_desc &desc) {
  const size_t base = fit_workspace_bytes(desc);
  if (base == 0 || desc.precision == RP_PREC_FP64) return base;
  auto res = [&](int dmax) {
    switch (desc.precision) {
      case RP_PREC_TF32: return fit_residency_tf32(dmax);
      case RP_PREC_TF32X3: return fit_residency_tf32x3(dmax);
      case RP_PREC_BF16: return fit_residency_bf16(dmax);
      case RP_PREC_BF16X3: return fit_residency_bf16x3(dmax);
      default: return fit_residency_f32(dmax);
    }
  };
  auto slab = [](int dmax) {
    const int nm = (dmax + 1) * (dmax + 2) * (dmax + 3) / 6;
    return (size_t)kCacheSamples * (size_t)((nm + 1) / 2) * 16;
  };
  const int dmax = desc.degree;
  size_t per_sm = (size_t)res(dmax <= 3 ? dmax : 3) * slab(dmax <= 3 ? dmax : 3);
  if (dmax == 4 && desc.precision != RP_PREC_FP32) {
    const size_t d4 = (size_t)res(4) * slab(4);
    if (d4 > per_sm) per_sm = d4;
  }
  return kCacheOffset + (size_t)num_sms() * per_sm;
}

int fit_max_ctas_per_sm(const rp_fit_desc &desc) {
  const int dmax = desc.degree;
  switch (desc.precision) {
    case RP_PREC_FP64: return fit_residency_f64(dmax);
    case RP_PREC_TF32: return fit_residency_tf32(dmax);
    case RP_PREC_TF32X3: return fit_residency_tf32x3(dmax);
    case RP_PREC_BF16: return fit_residency_bf16(dmax);
    case RP_PREC_BF16X3: return fit_residency_bf16x3(dmax);
    default: return fit_residency_f32(dmax);
  }
}


bool fit_precision_supported(int precision) {
  return precision >= RP_PREC_FP64 && precision <= RP_PREC_BF16X3;
}

cudaError_t launch_fit(const rp_fit_desc &desc, const float *x, const float *y,
                       const int64_t *fit_off, double *coef, float *coef32, double *box,
                       int32_t *status, int32_t *rank, void *workspace, size_t workspace_bytes,
                       cudaStream_t s) {
  if (desc.num_fits == 0) return cudaSuccess;
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
  a.svd = (desc.flags & RP_FIT_SOLVER_SVD) ? 1 : 0;
  a.tol = desc.tol;
  a.coef = coef;
  a.coef32 = coef32;
  a.box = box;
  a.status = status;
  a.rank = rank;
  a.point_off = desc.point_off;
  a.num_points = desc.num_points;
  a.fits_per_set = desc.point_off ? desc.fits_per_point_set : 1;
  a.counter = reinterpret_cast<unsigned long long *>(workspace);
  a.esc_count = workspace ? reinterpret_cast<unsigned long long *>(static_cast<char *>(workspace) + 16)
                          : nullptr;
  // the basis cache when the workspace holds it (results do not depend on it)
  a.psi_cache = nullptr;
  a.psi_cache_bytes = 0;
  if (workspace && desc.precision != RP_PREC_FP64 && workspace_bytes > kCacheOffset &&
      workspace_bytes >= fit_cache_workspace_bytes(desc)) {
    a.psi_cache = reinterpret_cast<float4 *>(static_cast<char *>(workspace) + kCacheOffset);
    a.psi_cache_bytes = workspace_bytes - kCacheOffset;
  }
  const int dmax = desc.degree;
  const int p0 = desc.precision;
  int p = p0;
  a.drop_tol = (p == RP_PREC_FP64) ? 1e-13 : 1e-7;
  a.esc_mode = (p == RP_PREC_FP64) ? 0 : 1;
  if (a.esc_count) {
    cudaError_t e = cudaMemsetAsync(a.esc_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  auto go = [&](int variant) {
    switch (p) {
      case RP_PREC_FP64: return fit_launch_f64(a, variant, p, s);
      case RP_PREC_TF32: return fit_launch_tf32(a, variant, p, s);
      case RP_PREC_TF32X3: return fit_launch_tf32x3(a, variant, p, s);
      case RP_PREC_BF16: return fit_launch_bf16(a, variant, p, s);
      case RP_PREC_BF16X3: return fit_launch_bf16x3(a, variant, p, s);
      default: return fit_launch_f32(a, variant, p, s);
    }
  };
  // A batch of per-fit degrees up to 4 runs as two launches on the stream:
  // the degree-3 variant (4 CTAs/SM on the FP32 path) for degrees <= 3, the
  // degree-4 variant (its basis needs ~250 registers) for degree 4 only.
  auto all = [&]() -> cudaError_t {
    if (desc.degrees && dmax == 4) {
      a.deg_lo = 1;
      a.deg_hi = 3;
      cudaError_t e = go(3);
      if (e != cudaSuccess) return e;
      a.deg_lo = 4;
      a.deg_hi = 4;
      return go(4);
    }
    a.deg_lo = 1;
    a.deg_hi = dmax;
    return go(dmax);
  };
  cudaError_t e = all();
  if (e != cudaSuccess || p0 == RP_PREC_FP64) return e;
  // the fits the FP32 / tensor-core launch passed on, on the FP64 path
  p = RP_PREC_FP64;
  a.drop_tol = 1e-13;
  a.esc_mode = 2;
  return all();
}

}  // namespace rpk
