// Self-test of the device-side failure path: one thread waits, with the
// library's bounded wait, on an mbarrier phase that nothing completes. The
// wait runs out after `limit` polls, the kernel records SPINSUM_ERR_TIMEOUT
// in the status word and returns; the host reads it with
// spinsum_check_status(). Nothing faults, traps or hangs.
#include "ss_tma.cuh"

namespace ss {

__global__ void selftest_wait_kernel(int* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicExch(status, 1);
}

int* status_ptr();

}  // namespace ss

extern "C" int ss_selftest_wait_timeout(long long limit, void* stream) {
  int* st = ss::status_ptr();
  if (!st) return -4;
  ss::selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(st, limit);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}
