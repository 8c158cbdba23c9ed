// Fit kernel instantiations of one precision family (TF32: design Gram in one TF32 tensor-core pass),
// degree bounds 2, 3 and 4; compiled on their own so the families build in
// parallel.
#include "rp_fit_kernel.cuh"

namespace rpk {

cudaError_t fit_launch_tf32(const FitArgs &a, int dmax, int precision, cudaStream_t s) {
  return launch_family<float, 1>(a, dmax, precision, s);
}

int fit_residency_tf32(int dmax) { return residency_family<float, 1>(dmax); }

}  // namespace rpk
