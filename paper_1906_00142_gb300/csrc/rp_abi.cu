// extern "C" entry points: argument checks, then launches on the caller's
// stream.  Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rp_internal.cuh"

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int from_cuda(cudaError_t e) { return e == cudaSuccess ? RP_OK : RP_ERR_CUDA; }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool device_ok() {
  int n = 0;
  return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
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

int rp_fit(const rp_fit_desc *desc, const float *x, const float *y, const int64_t *fit_off,
           double *coef, float *coef32, double *box, int32_t *status, int32_t *rank,
           void *workspace, size_t workspace_bytes, void *stream) {
  if (!desc || desc->num_fits < 0 || desc->num_samples < 0) return RP_ERR_INVALID_ARG;
  if (desc->degree < 1 || desc->degree > RP_MAX_DEGREE) return RP_ERR_INVALID_ARG;
  if (desc->precision < RP_PREC_FP64 || desc->precision > RP_PREC_BF16X3) return RP_ERR_INVALID_ARG;
  if (desc->max_refine < 0 || desc->max_refine > 64 || !(desc->tol >= 0.0)) return RP_ERR_INVALID_ARG;
  if (desc->num_fits == 0) return RP_OK;
  if (!fit_off || !coef || !box || !status || !rank) return RP_ERR_INVALID_ARG;
  if (desc->num_samples > 0 && (!x || !y)) return RP_ERR_INVALID_ARG;
  if (workspace_bytes < rpk::fit_workspace_bytes(*desc)) return RP_ERR_WORKSPACE;
  if (!rpk::fit_precision_supported(desc->precision)) return RP_ERR_UNSUPPORTED;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  return from_cuda(rpk::launch_fit(*desc, x, y, fit_off, coef, coef32, box, status, rank, workspace,
                                   as_stream(stream)));
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

int rp_eval_search(const void *program, int64_t num_kernels, int32_t degree,
                   const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                   int32_t *argmin, float *best, float *second, int32_t *status, void *stream) {
  if (num_kernels < 0 || num_queries < 0 || degree < 0 || degree > RP_MAX_DEGREE || !hw)
    return RP_ERR_INVALID_ARG;
  if (hw->warp_size < 1 || hw->t_max < 1 || hw->b_max < 1 || hw->w_max < 1 || hw->r_sm < 1 ||
      hw->z_sm < 1 || !(hw->issue_cycles > 0.0f) || hw->reserved != 0 || hw->r_sm >= (1 << 24) ||
      hw->z_sm >= (1 << 24))
    return RP_ERR_INVALID_ARG;
  if (num_queries == 0) return RP_OK;
  if (!program || !queries || !argmin || !best || !second || !status) return RP_ERR_INVALID_ARG;
  if (!aligned(program, 16) || !aligned(queries, 16)) return RP_ERR_ALIGNMENT;
  if (!device_ok()) return RP_ERR_NO_DEVICE;
  auto pv = rpk::program_sections<rpk::ProgramView>(program, num_kernels);
  return from_cuda(rpk::launch_search(pv, num_kernels, degree, *hw, queries, num_queries, argmin,
                                      best, second, status, as_stream(stream)));
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
