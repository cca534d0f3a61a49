// Instantiates the fused summation-contraction kernels for d = 4 (see ss_contract.cuh).
#include "ss_contract.cuh"

namespace ss {

cudaError_t launch_kc_d4(const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                         int64_t ldc, cudaStream_t st) {
  return launch_kc_d<4>(kp, ar, sum, W, Y, ldw, C, ldc, st);
}
}  // namespace ss
