// Fit kernel instantiations of one precision family (split BF16: design Gram in three BF16 tensor-core passes),
// degree bounds 2, 3 and 4; compiled on their own so the families build in
// parallel.
#include "rp_fit_kernel.cuh"

namespace rpk {

cudaError_t fit_launch_bf16x3(const FitArgs &a, int dmax, int precision, cudaStream_t s) {
  return launch_family<float, 4>(a, dmax, precision, s);
}

int fit_residency_bf16x3(int dmax) { return residency_family<float, 4>(dmax); }

}  // namespace rpk
