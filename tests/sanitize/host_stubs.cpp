// Stand-ins for the device-side translation units, so that the host planner
// (ss_host.cpp) links without a GPU build: every launch reports "no device"
// and the status word does not exist. Used only by the sanitizer test.
#include <cuda_runtime.h>

#include "../../paper_1705_06661_gb300/csrc/ss_internal.h"

namespace ss {
cudaError_t launch_k1(int, const KParams&, int, int, cudaStream_t) { return cudaErrorNoDevice; }
cudaError_t launch_k1t(int, const KParams&, int, cudaStream_t) { return cudaErrorNoDevice; }
cudaError_t launch_k2(int, const KParams&, int, cudaStream_t) { return cudaErrorNoDevice; }
cudaError_t launch_kg(int, const KParams&, int, cudaStream_t) { return cudaErrorNoDevice; }
cudaError_t launch_pack(int, const KParams&, bool, bool, int, cudaStream_t) { return cudaErrorNoDevice; }
cudaError_t launch_kb(int, int, const KParams*, const int64_t*, const int*, int, unsigned long long*, int, cudaStream_t, const void**) {
  return cudaErrorNoDevice;
}
cudaError_t launch_kc(int, const KParams&, int, bool, const double*, int64_t, int64_t, double*, int64_t, cudaStream_t) {
  return cudaErrorNoDevice;
}
int k1t_chunk(int d, int) { return d == 3 ? 512 : 256; }
int* status_ptr() { return nullptr; }
cudaError_t read_and_clear_status(int* out) {
  *out = 0;
  return cudaErrorNoDevice;
}
cudaError_t static_scratch_ptr(void** out) {
  *out = nullptr;
  return cudaErrorNoDevice;
}
}  // namespace ss
