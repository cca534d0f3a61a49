// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_k1_d4_f32(const KParams& kp, int vec, cudaStream_t st) {
  const dim3 grid((unsigned)kp.pre[npatterns(4)]), block(256);
  (void)vec;
  k1_kernel<4, AR_F32, 1, float><<<grid, block, 0, st>>>(kp);
  return cudaGetLastError();
}
}  // namespace ss
