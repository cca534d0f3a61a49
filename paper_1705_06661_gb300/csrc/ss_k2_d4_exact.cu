// Instantiates part of the spin-summation kernels (see ss_k2.cuh).
#include "ss_k2.cuh"

namespace ss {

cudaError_t launch_k2_d4_exact(const KParams& kp, cudaStream_t st) {
  if (kp.flags & KF_WHT) return launch_k2_impl<4, AR_EXACT_XW, double>(kp, st);
  return launch_k2_impl<4, AR_EXACT, double>(kp, st);
}
}  // namespace ss
