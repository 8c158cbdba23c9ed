// extern "C" entry points: argument checks, then launches on the caller's
// stream.  Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include "rp_internal.cuh"

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int from_cuda(cudaError_t e) { return e == cudaSuccess ? RP_OK : RP_ERR_CUDA; }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool device_ok() {
  int n = 0;
  return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
}

// Mean device time (ms) of `reps` calls of fn on the stream, after one
// untimed call; a negative value reports a launch or CUDA error.
template <class Fn>
float time_calls(Fn fn, int reps, cudaStream_t s) {
  if (fn() != RP_OK) return -1.0f;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.0f;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return -1.0f;
  }
  float ms = -1.0f;
  bool ok = cudaEventRecord(a, s) == cudaSuccess;
  for (int r = 0; r < reps && ok; ++r) ok = fn() == RP_OK;
  ok = ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
       cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ok ? ms / (float)reps : -1.0f;
}

}  // namespace

extern "C" {

int rp_version(void) { return RP_VERSION; }

const char *rp_strerror(int code) {
  switch (code) {
    case RP_OK: return "ok";
    case RP_ERR_INVALID_ARG: return "invalid argument";
    case RP_ERR_UNSUPPORTED: return "unsupported configuration";
    case RP_ERR_WORKSPACE: return "workspace too small";
    case RP_ERR_CUDA: return "CUDA error";
    case RP_ERR_ALIGNMENT: return "misaligned pointer";
    case RP_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
  }
}

int rp_fit_workspace_size(const rp_fit_desc *desc, size_t *bytes) {
  if (!desc || !bytes) return RP_ERR_INVALID_ARG;
  *bytes = rpk::fit_workspace_bytes(*desc);
  return RP_OK;
}

int rp_fit_cache_workspace_size(const rp_fit_desc *desc, size_t *bytes) {
  if (!desc || !bytes) return RP_ERR_INVALID_ARG;
  if (desc->degree < 1 || desc->degree > RP_MAX_DEGREE) return RP_ERR_INVALID_ARG;
  if (desc->precision < RP_PREC_FP64 || desc->precision > RP_PREC_BF16X3) return RP_ERR_INVALID_ARG;
  *bytes = rpk::fit_cache_workspace_bytes(*desc);
  return RP_OK;
}

int rp_fit(const rp_fit_desc *desc, const float *x, const float *y, const int64_t *fit_off,
           double *coef, float *coef32, double *box, int32_t *status, int32_t *rank,
           void *workspace, size_t workspace_bytes, void *stream) {
  if (!desc || desc->num_fits < 0 || desc->num_samples < 0) return RP_ERR_INVALID_ARG;
  if (desc->degree < 1 || desc->degree > RP_MAX_DEGREE) return RP_ERR_INVALID_ARG;
  if (desc->precision < RP_PREC_FP64 || desc->precision > RP_PREC_BF16X3) return RP_ERR_INVALID_ARG;
  if (desc->max_refine < 0 || desc->max_refine > 64 || !(desc->tol >= 0.0)) return RP_ERR_INVALID_ARG;
  if (desc->reserved != 0 || (desc->flags & ~(RP_FIT_UNWEIGHTED | RP_FIT_SOLVER_SVD)))
    return RP_ERR_INVALID_ARG;
  if (desc->point_off && (desc->fits_per_point_set < 1 || desc->num_points < 0)) return RP_ERR_INVALID_ARG;
  if (desc->num_fits == 0) return RP_OK;
  if (!fit_off || !coef || !box || !status || !rank) return RP_ERR_INVALID_ARG;
  if (desc->num_samples > 0 && !y) return RP_ERR_INVALID_ARG;
  if ((desc->point_off ? desc->num_points : desc->num_samples) > 0 && !x) return RP_ERR_INVALID_ARG;
  if (workspace && workspace_bytes < rpk::fit_workspace_bytes(*desc)) return RP_ERR_WORKSPACE;
  if (workspace && !aligned(workspace, 16)) return RP_ERR_ALIGNMENT;
  if (!rpk::fit_precision_supported(desc->precision)) return RP_ERR_UNSUPPORTED;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_fit(*desc, x, y, fit_off, coef, coef32, box, status, rank, workspace,
                                   workspace ? workspace_bytes : 0, as_stream(stream)));
}

int rp_fit_noalloc(const rp_fit_desc *desc, const float *x, const float *y,
                   const int64_t *fit_off, double *coef, float *coef32, double *box,
                   int32_t *status, int32_t *rank, void *stream) {
  if (!desc) return RP_ERR_INVALID_ARG;
  if (desc->num_fits == 0)   // nothing to launch; arguments checked as rp_fit does
    return rp_fit(desc, x, y, fit_off, coef, coef32, box, status, rank, nullptr, 0, stream);
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  if (rpk::fit_static_scratch(&scratch, &scratch_bytes) != cudaSuccess) return RP_ERR_CUDA;
  if (rpk::fit_workspace_bytes(*desc) > scratch_bytes) return RP_ERR_WORKSPACE;
  return rp_fit(desc, x, y, fit_off, coef, coef32, box, status, rank, scratch, scratch_bytes,
                stream);
}

size_t rp_program_size(int64_t num_kernels, int32_t degree) {
  if (num_kernels < 0 || degree < 0 || degree > RP_MAX_DEGREE) return 0;
  return rpk::program_size(num_kernels, degree);
}

int rp_program_pack(int64_t num_kernels, int32_t degree, const double *coef, const double *box,
                    const int8_t *degrees, const int32_t *metric_map, const int32_t *grid_dims,
                    void *program, size_t program_bytes, void *stream) {
  if (num_kernels < 0 || degree < 1 || degree > RP_MAX_DEGREE) return RP_ERR_INVALID_ARG;
  if (num_kernels == 0) return RP_OK;
  if (!coef || !box || !degrees || !metric_map || !grid_dims || !program) return RP_ERR_INVALID_ARG;
  if (program_bytes < rpk::program_size(num_kernels, degree)) return RP_ERR_INVALID_ARG;
  if (!aligned(program, 16)) return RP_ERR_ALIGNMENT;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  auto pm = rpk::program_sections<rpk::ProgramMut>(program, num_kernels);
  return from_cuda(rpk::launch_pack(num_kernels, degree, coef, box, degrees, metric_map, grid_dims,
                                    pm, as_stream(stream)));
}

int rp_search_workspace_size(int64_t num_kernels, int64_t num_queries, size_t *bytes) {
  if (!bytes || num_kernels < 0 || num_queries < 0) return RP_ERR_INVALID_ARG;
  *bytes = rpk::search_workspace_bytes(num_kernels, num_queries);
  return RP_OK;
}

int rp_eval_search(const void *program, int64_t num_kernels, int32_t degree,
                   const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                   int32_t *argmin, float *best, float *second, int32_t *status,
                   void *workspace, size_t workspace_bytes, void *stream) {
  if (num_kernels < 0 || num_queries < 0 || degree < 0 || degree > RP_MAX_DEGREE || !hw)
    return RP_ERR_INVALID_ARG;
  if (hw->warp_size < 1 || hw->t_max < 1 || hw->b_max < 1 || hw->w_max < 1 || hw->r_sm < 1 ||
      hw->z_sm < 1 || !(hw->issue_cycles > 0.0f) || hw->reserved != 0 || hw->r_sm >= (1 << 24) ||
      hw->z_sm >= (1 << 24))
    return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!program || !queries || !argmin || !best || !second || !status) return RP_ERR_INVALID_ARG;
  if (!aligned(program, 16) || !aligned(queries, 16)) return RP_ERR_ALIGNMENT;
  if (workspace) {
    if (workspace_bytes < rpk::search_workspace_bytes(num_kernels, num_queries))
      return RP_ERR_WORKSPACE;
    if (!aligned(workspace, 16)) return RP_ERR_ALIGNMENT;
  }
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  auto pv = rpk::program_sections<rpk::ProgramView>(program, num_kernels);
  return from_cuda(rpk::launch_search(pv, num_kernels, degree, *hw, queries, num_queries, argmin,
                                      best, second, status, workspace, as_stream(stream)));
}

static bool hw_ok(const rp_hw_fixed *hw) {
  return hw && hw->warp_size >= 1 && hw->t_max >= 1 && hw->b_max >= 1 && hw->w_max >= 1 &&
         hw->r_sm >= 1 && hw->z_sm >= 1 && hw->issue_cycles > 0.0f && hw->reserved == 0 &&
         hw->r_sm < (1 << 24) && hw->z_sm < (1 << 24);
}

int rp_eval_search_tiebreak(const void *program, int64_t num_kernels, int32_t degree,
                            const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                            float tie_rel, int32_t *argmin, float *best, float *second,
                            int32_t *status, void *workspace, size_t workspace_bytes,
                            void *stream) {
  if (!(tie_rel >= 0.0f) || !(tie_rel < 1.0f)) return RP_ERR_INVALID_ARG;
  if (num_kernels < 0 || num_queries < 0 || degree < 0 || degree > RP_MAX_DEGREE || !hw_ok(hw))
    return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!program || !queries || !argmin || !best || !second || !status) return RP_ERR_INVALID_ARG;
  if (!aligned(program, 16) || !aligned(queries, 16)) return RP_ERR_ALIGNMENT;
  if (workspace) {
    if (workspace_bytes < rpk::search_workspace_bytes(num_kernels, num_queries))
      return RP_ERR_WORKSPACE;
    if (!aligned(workspace, 16)) return RP_ERR_ALIGNMENT;
  }
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  auto pv = rpk::program_sections<rpk::ProgramView>(program, num_kernels);
  return from_cuda(rpk::launch_search(pv, num_kernels, degree, *hw, queries, num_queries, argmin,
                                      best, second, status, workspace, as_stream(stream), tie_rel));
}

int rp_eval_occupancy(const void *program, int64_t num_kernels, int32_t degree,
                      const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                      int32_t *b_active, int32_t *w_active, int32_t *status, void *stream) {
  if (num_kernels < 0 || num_queries < 0 || degree < 0 || degree > RP_MAX_DEGREE || !hw_ok(hw))
    return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!program || !queries || !b_active || !w_active || !status) return RP_ERR_INVALID_ARG;
  if (!aligned(program, 16) || !aligned(queries, 16)) return RP_ERR_ALIGNMENT;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  auto pv = rpk::program_sections<rpk::ProgramView>(program, num_kernels);
  return from_cuda(rpk::launch_occupancy(pv, num_kernels, degree, *hw, queries, num_queries,
                                         b_active, w_active, status, as_stream(stream)));
}

int rp_error_pct(const float *runtimes, const int32_t *choice, int64_t num_queries,
                 float *err_pct, int32_t *status, void *stream) {
  if (num_queries < 0) return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!runtimes || !choice || !err_pct || !status) return RP_ERR_INVALID_ARG;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_error_pct(runtimes, choice, num_queries, err_pct, status,
                                         as_stream(stream)));
}

int rp_codegen_source(const void *program_host, int64_t num_kernels, int32_t degree,
                      int64_t kernel_id, const rp_hw_fixed *hw, char *src, size_t *len) {
  if (!program_host || !len || num_kernels < 1 || kernel_id < 0 || kernel_id >= num_kernels ||
      degree < 0 || degree > RP_MAX_DEGREE || !hw_ok(hw))
    return RP_ERR_INVALID_ARG;
  const std::string code = rpk::codegen_source(program_host, num_kernels, degree, kernel_id, *hw);
  const size_t need = code.size() + 1;
  if (!src || *len < need) {
    *len = need;
    return src ? RP_ERR_WORKSPACE : RP_OK;
  }
  memcpy(src, code.c_str(), need);
  *len = need;
  return RP_OK;
}

int rp_codegen_compile(const char *src, void **handle, char *log, size_t log_len) {
  if (!src || !handle) return RP_ERR_INVALID_ARG;
  *handle = nullptr;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return rpk::codegen_compile(src, handle, log, log_len);
}

int rp_codegen_search(void *handle, const float *queries, int64_t num_queries, int32_t *argmin,
                      float *best, float *second, int32_t *status, void *stream) {
  if (!handle || num_queries < 0) return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!queries || !argmin || !best || !second || !status) return RP_ERR_INVALID_ARG;
  if (!aligned(queries, 16)) return RP_ERR_ALIGNMENT;
  return from_cuda(rpk::codegen_search(handle, queries, num_queries, argmin, best, second, status,
                                       as_stream(stream)));
}

int rp_codegen_free(void *handle) {
  rpk::codegen_free(handle);
  return RP_OK;
}

int rp_tune_search(const void *program, int64_t num_kernels, int32_t degree,
                   const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                   int32_t *argmin, float *best, float *second, int32_t *status,
                   void *workspace, size_t workspace_bytes, void *stream, int32_t *threads,
                   int32_t *ctas_per_sm) {
  if (!threads || !ctas_per_sm) return RP_ERR_INVALID_ARG;
  // validates everything once (and is the first, untimed call)
  int rc = rp_eval_search(program, num_kernels, degree, hw, queries, num_queries, argmin, best,
                          second, status, workspace, workspace_bytes, stream);
  if (rc != RP_OK) return rc;
  static const rpk::SearchShape cand[] = {{256, 8}, {256, 4}, {256, 2}, {128, 16}, {128, 8},
                                          {128, 4}, {64, 32}, {64, 16}};
  const rpk::SearchShape keep = rpk::search_shape(degree);
  rpk::SearchShape best_shape = keep;
  float best_ms = 0.0f;
  for (const auto &c : cand) {
    rpk::set_search_shape(degree, c);
    const float ms = time_calls(
        [&] {
          return rp_eval_search(program, num_kernels, degree, hw, queries, num_queries, argmin,
                                best, second, status, workspace, workspace_bytes, stream);
        },
        3, as_stream(stream));
    if (ms < 0.0f) {
      rpk::set_search_shape(degree, keep);
      return RP_ERR_CUDA;
    }
    if (best_ms == 0.0f || ms < best_ms) {
      best_ms = ms;
      best_shape = c;
    }
  }
  rpk::set_search_shape(degree, best_shape);
  *threads = best_shape.threads;
  *ctas_per_sm = best_shape.ctas_per_sm;
  return RP_OK;
}

int rp_tune_fit(const rp_fit_desc *desc, const float *x, const float *y, const int64_t *fit_off,
                double *coef, float *coef32, double *box, int32_t *status, int32_t *rank,
                void *workspace, size_t workspace_bytes, void *stream, int32_t *ctas_per_sm) {
  if (!ctas_per_sm) return RP_ERR_INVALID_ARG;
  int rc = rp_fit(desc, x, y, fit_off, coef, coef32, box, status, rank, workspace, workspace_bytes,
                  stream);
  if (rc != RP_OK) return rc;
  if (desc->num_fits == 0) {
    *ctas_per_sm = 0;
    return RP_OK;
  }
  const int dmax = desc->degree;
  const int keep = rpk::fit_ctas_cap(desc->precision, dmax);
  const int top = rpk::fit_max_ctas_per_sm(*desc);
  int best_cap = keep;
  float best_ms = 0.0f;
  for (int c = top; c >= 1; --c) {
    rpk::set_fit_ctas_cap(desc->precision, dmax, c);
    const float ms = time_calls(
        [&] {
          return rp_fit(desc, x, y, fit_off, coef, coef32, box, status, rank, workspace,
                        workspace_bytes, stream);
        },
        2, as_stream(stream));
    if (ms < 0.0f) {
      rpk::set_fit_ctas_cap(desc->precision, dmax, keep);
      return RP_ERR_CUDA;
    }
    if (best_ms == 0.0f || ms < best_ms) {
      best_ms = ms;
      best_cap = c;
    }
  }
  rpk::set_fit_ctas_cap(desc->precision, dmax, best_cap);
  *ctas_per_sm = best_cap;
  return RP_OK;
}

int rp_relmse_fwd(int64_t num_fits, int64_t num_samples, const float *x, const float *y,
                  const int64_t *fit_off, const int8_t *degrees, const double *coef,
                  const double *box, float *loss, void *stream) {
  if (num_fits < 0 || num_samples < 0) return RP_ERR_INVALID_ARG;
  if (num_fits == 0) return RP_OK;
  if (!x || !y || !fit_off || !degrees || !coef || !box || !loss) return RP_ERR_INVALID_ARG;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_relmse(false, num_fits, num_samples, x, y, fit_off, degrees, coef,
                                      box, nullptr, loss, as_stream(stream)));
}

int rp_relmse_bwd(int64_t num_fits, int64_t num_samples, const float *x, const float *y,
                  const int64_t *fit_off, const int8_t *degrees, const double *coef,
                  const double *box, const float *grad_loss, float *grad, void *stream) {
  if (num_fits < 0 || num_samples < 0) return RP_ERR_INVALID_ARG;
  if (num_fits == 0) return RP_OK;
  if (!x || !y || !fit_off || !degrees || !coef || !box || !grad_loss || !grad)
    return RP_ERR_INVALID_ARG;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_relmse(true, num_fits, num_samples, x, y, fit_off, degrees, coef,
                                      box, grad_loss, grad, as_stream(stream)));
}

int rp_adam_step(int64_t n, double *param, const float *grad, float *m, float *v,
                 const uint8_t *mask, int32_t t, float lr, float beta1, float beta2, float eps,
                 void *stream) {
  if (n < 0 || t < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
    return RP_ERR_INVALID_ARG;
  if (n == 0) return RP_OK;
  if (!param || !grad || !m || !v) return RP_ERR_INVALID_ARG;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_adam(n, param, grad, m, v, mask, t, lr, beta1, beta2, eps,
                                    as_stream(stream)));
}

}  // extern "C"
