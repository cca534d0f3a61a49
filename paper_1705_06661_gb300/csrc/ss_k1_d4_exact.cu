// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_k1_d4_exact(const KParams& kp, cudaStream_t st) {
  const dim3 grid((unsigned)kp.pre[npatterns(4)]), block(256);
  if (kp.flags & KF_WHT) k1_kernel<4, AR_EXACT, 1, double, 1><<<grid, block, 0, st>>>(kp);
  else k1_kernel<4, AR_EXACT, 1, double, 0><<<grid, block, 0, st>>>(kp);
  return cudaGetLastError();
}
}  // namespace ss
