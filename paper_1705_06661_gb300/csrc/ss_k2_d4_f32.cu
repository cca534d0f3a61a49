// Instantiates part of the spin-summation kernels (see ss_k2.cuh).
#include "ss_k2.cuh"

namespace ss {

cudaError_t launch_k2_d4_f32(const KParams& kp, cudaStream_t st) {
  return launch_k2_impl<4, AR_F32, float>(kp, st);
}
}  // namespace ss
