// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_k1_d3(const KParams& kp, int ar, int vec, cudaStream_t st) {
  const dim3 grid((unsigned)kp.pre[npatterns(3)]), block(256);
  if (ar == AR_EXACT) {
    if (vec == 2) k1_kernel<3, AR_EXACT, 2, double><<<grid, block, 0, st>>>(kp);
    else k1_kernel<3, AR_EXACT, 1, double><<<grid, block, 0, st>>>(kp);
  } else if (ar == AR_STRICT) {
    if (vec == 2) k1_kernel<3, AR_STRICT, 2, double><<<grid, block, 0, st>>>(kp);
    else k1_kernel<3, AR_STRICT, 1, double><<<grid, block, 0, st>>>(kp);
  } else {
    if (vec == 4) k1_kernel<3, AR_F32, 4, float><<<grid, block, 0, st>>>(kp);
    else if (vec == 2) k1_kernel<3, AR_F32, 2, float><<<grid, block, 0, st>>>(kp);
    else k1_kernel<3, AR_F32, 1, float><<<grid, block, 0, st>>>(kp);
  }
  return cudaGetLastError();
}
}  // namespace ss
