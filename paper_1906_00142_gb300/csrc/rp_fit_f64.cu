// Fit kernel instantiations of one precision family (FP64: FP64 design, Gram and factor on CUDA cores),
// degree bounds 2, 3 and 4; compiled on their own so the families build in
// parallel.
#include "rp_fit_kernel.cuh"

namespace rpk {

cudaError_t fit_launch_f64(const FitArgs &a, int dmax, int precision, cudaStream_t s) {
  return launch_family<double, 0>(a, dmax, precision, s);
}

int fit_residency_f64(int dmax) { return residency_family<double, 0>(dmax); }

}  // namespace rpk
