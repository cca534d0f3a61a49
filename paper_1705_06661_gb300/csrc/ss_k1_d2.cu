// Instantiates part of the spin-summation kernels (see ss_kernels.cuh): d = 2.
#include "ss_kernels.cuh"

namespace ss {

cudaError_t launch_k1_d2(const KParams& kp, int ar, int vec, cudaStream_t st) {
  const dim3 grid((unsigned)kp.pre[npatterns(2)]), block(256);
  if (ar == AR_EXACT) {
    if (vec == 2) k1_kernel<2, AR_EXACT, 2, double><<<grid, block, 0, st>>>(kp);
    else k1_kernel<2, AR_EXACT, 1, double><<<grid, block, 0, st>>>(kp);
  } else if (ar == AR_STRICT) {
    if (vec == 2) k1_kernel<2, AR_STRICT, 2, double><<<grid, block, 0, st>>>(kp);
    else k1_kernel<2, AR_STRICT, 1, double><<<grid, block, 0, st>>>(kp);
  } else {
    if (vec == 4) k1_kernel<2, AR_F32, 4, float><<<grid, block, 0, st>>>(kp);
    else if (vec == 2) k1_kernel<2, AR_F32, 2, float><<<grid, block, 0, st>>>(kp);
    else k1_kernel<2, AR_F32, 1, float><<<grid, block, 0, st>>>(kp);
  }
  return cudaGetLastError();
}

cudaError_t launch_kg_d2(const KParams& kp, int ar, cudaStream_t st) {
  const dim3 grid((unsigned)((kp.ngroup + 255) / 256)), block(256);
  // FP64 runs the strict core here (the exact core needs coalesced orbit runs to pay off)
  if (ar == AR_F32) kg_kernel<2, AR_F32, float><<<grid, block, 0, st>>>(kp);
  else kg_kernel<2, AR_STRICT, double><<<grid, block, 0, st>>>(kp);
  return cudaGetLastError();
}

cudaError_t launch_kb_d2(int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                         cudaStream_t st, const void** fn) {
  const void* f;
  if (ar == AR_EXACT) f = reinterpret_cast<const void*>(&kb_kernel<2, AR_EXACT, double>);
  else if (ar == AR_STRICT) f = reinterpret_cast<const void*>(&kb_kernel<2, AR_STRICT, double>);
  else f = reinterpret_cast<const void*>(&kb_kernel<2, AR_F32, float>);
  if (fn) { *fn = f; return cudaSuccess; }
  const dim3 g((unsigned)grid), b(256);
  if (ar == AR_EXACT) kb_kernel<2, AR_EXACT, double><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  else if (ar == AR_STRICT) kb_kernel<2, AR_STRICT, double><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  else kb_kernel<2, AR_F32, float><<<g, b, 0, st>>>(probs, prefix, vecs, n, ctr);
  return cudaGetLastError();
}
}  // namespace ss
