// Device status word and the dispatch from (d, arithmetic, vector width) to
// the kernel instantiations of the ss_k*.cu translation units.
#include <cuda_runtime.h>

#include "ss_internal.h"

namespace ss {

__device__ int g_status;

cudaError_t launch_k1_d3(const KParams& kp, int ar, int vec, cudaStream_t st);
cudaError_t launch_k1_d4_exact(const KParams& kp, cudaStream_t st);
cudaError_t launch_k1_d4_strict(const KParams& kp, cudaStream_t st);
cudaError_t launch_k1_d4_f32(const KParams& kp, int vec, cudaStream_t st);
cudaError_t launch_kg_d3(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_kg_d4(const KParams& kp, int ar, cudaStream_t st);

cudaError_t launch_k1(int d, const KParams& kp, int ar, int vec, cudaStream_t st) {
  if (d == 3) return launch_k1_d3(kp, ar, vec, st);
  if (ar == AR_EXACT) return launch_k1_d4_exact(kp, st);
  if (ar == AR_STRICT) return launch_k1_d4_strict(kp, st);
  return launch_k1_d4_f32(kp, vec, st);
}

cudaError_t launch_kg(int d, const KParams& kp, int ar, cudaStream_t st) {
  return d == 3 ? launch_kg_d3(kp, ar, st) : launch_kg_d4(kp, ar, st);
}

cudaError_t read_and_clear_status(int* out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_status, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
}

}  // namespace ss
