// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_kb_d4_strict(const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                              cudaStream_t st, const void** fn) {
  if (fn) {
    *fn = reinterpret_cast<const void*>(&kb_kernel<4, AR_STRICT, double>);
    return cudaSuccess;
  }
  kb_kernel<4, AR_STRICT, double><<<dim3((unsigned)grid), dim3(256), 0, st>>>(probs, prefix, vecs, n, ctr);
  return cudaGetLastError();
}
}  // namespace ss
