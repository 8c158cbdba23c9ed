// Fit kernel instantiations of one precision family (FP32: FP32 design, Gram on CUDA cores),
// degree bounds 2, 3 and 4; compiled on their own so the families build in
// parallel.
#include "rp_fit_kernel.cuh"

namespace rpk {

cudaError_t fit_launch_f32(const FitArgs &a, int dmax, int precision, cudaStream_t s) {
  return launch_family<float, 0>(a, dmax, precision, s);
}

int fit_residency_f32(int dmax) { return residency_family<float, 0>(dmax); }

}  // namespace rpk
