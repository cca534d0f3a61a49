// Instantiates part of the spin-summation kernels (see ss_k2.cuh): d = 2.
#include "ss_k2.cuh"

namespace ss {

cudaError_t launch_k2_d2(const KParams& kp, int ar, cudaStream_t st) {
  if (ar == AR_EXACT) return launch_k2_impl<2, AR_EXACT, double>(kp, st);
  if (ar == AR_STRICT) return launch_k2_impl<2, AR_STRICT, double>(kp, st);
  return launch_k2_impl<2, AR_F32, float>(kp, st);
}
}  // namespace ss
