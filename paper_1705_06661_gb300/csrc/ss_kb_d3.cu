// Instantiates part of the spin-summation kernels (see ss_kernels.cuh).
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_kb_d3(int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                         cudaStream_t st, const void** fn) {
  const void* f;
  if (ar == AR_EXACT) f = reinterpret_cast<const void*>(&kb_kernel<3, AR_EXACT, double>);
  else if (ar == AR_STRICT) f = reinterpret_cast<const void*>(&kb_kernel<3, AR_STRICT, double>);
  else f = reinterpret_cast<const void*>(&kb_kernel<3, AR_F32, float>);
  if (fn) { *fn = f; return cudaSuccess; }
  const dim3 g((unsigned)grid), b(256);
  if (ar == AR_EXACT) kb_kernel<3, AR_EXACT, double><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  else if (ar == AR_STRICT) kb_kernel<3, AR_STRICT, double><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  else kb_kernel<3, AR_F32, float><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  return cudaGetLastError();
}
}  // namespace ss
