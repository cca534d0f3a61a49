// Batched spin summation for callers that cannot allocate device memory.
//
// A batched plan keeps its problem parameters and K1-block prefix sums in
// device memory that spinsum_plan_create allocates. spinsum_batch_static runs
// the same batched kernel, but with that image in the fixed file-scope array
// below: the array exists on every GPU that loads this library, from load
// until process exit. On the host the array's name is only a stand-in symbol,
// never a device address, so host code looks the address up once per device
// with cudaGetSymbolAddress and passes it to the kernel.
#include <cuda_runtime.h>

#include "../../include/spinsum.h"
#include "ss_devcache.h"
#include "ss_internal.h"

namespace ss {

static __device__ __align__(256) unsigned char g_static_scratch[batch_image_bytes(SPINSUM_STATIC_MAX_PROBLEMS)];

// device address of the array on the current device, looked up once per
// device (several host threads may ask at once)
cudaError_t static_scratch_ptr(void** out) {
  static DeviceCache cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  long long v = 0;
  const int rc = cache.get(dev, &v, [](long long* val) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_static_scratch);
    *val = (long long)(uintptr_t)p;
    return (int)err;
  });
  if (rc != 0) return rc < 0 ? cudaErrorInvalidDevice : (cudaError_t)rc;
  *out = (void*)(uintptr_t)v;
  return cudaSuccess;
}

}  // namespace ss
