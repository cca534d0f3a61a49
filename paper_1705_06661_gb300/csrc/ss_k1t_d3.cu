// Instantiates part of the spin-summation kernels (see ss_tma.cuh).
#include "ss_tma.cuh"

namespace ss {

cudaError_t launch_k1t_d3(const KParams& kp, int ar, cudaStream_t st) {
  if (ar == AR_EXACT) return launch_k1t_impl<3, AR_EXACT, 2, double, SS_K1T3_NCW, SS_K1T3_NST>(kp, st);
  return launch_k1t_impl<3, AR_F32, 4, float, SS_K1T3_NCW, SS_K1T3_NST>(kp, st);
}

}  // namespace ss
