// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_kg_d4(const KParams& kp, int ar, cudaStream_t st) {
  const dim3 grid((unsigned)((kp.ngroup + 255) / 256)), block(256);
  // FP64 runs the strict core here (the exact core needs coalesced orbit runs to pay off)
  if (ar == AR_F32) kg_kernel<4, AR_F32, float><<<grid, block, 0, st>>>(kp);
  else kg_kernel<4, AR_STRICT, double><<<grid, block, 0, st>>>(kp);
  return cudaGetLastError();
}
}  // namespace ss
