// Device status word and the dispatch from (d, arithmetic, vector width) to
// the kernel instantiations of the ss_k1_*, ss_k2_*, ss_kg_*, ss_kb_* and
// ss_kc_* translation units.
#include <cuda_runtime.h>

#include "ss_devcache.h"
#include "ss_internal.h"

namespace ss {

__device__ int g_status;

cudaError_t launch_k1_d2(const KParams& kp, int ar, int vec, cudaStream_t st);
cudaError_t launch_kg_d2(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k2_d2(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_kb_d2(int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                         cudaStream_t st, const void** fn);
cudaError_t launch_k1_d3(const KParams& kp, int ar, int vec, cudaStream_t st);
cudaError_t launch_k1_d4_exact(const KParams& kp, cudaStream_t st);
cudaError_t launch_k1_d4_strict(const KParams& kp, cudaStream_t st);
cudaError_t launch_k1_d4_f32(const KParams& kp, int vec, cudaStream_t st);
cudaError_t launch_kg_d3(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k2_d3(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k2_d4_exact(const KParams& kp, cudaStream_t st);
cudaError_t launch_k2_d4_strict(const KParams& kp, cudaStream_t st);
cudaError_t launch_k2_d4_f32(const KParams& kp, cudaStream_t st);
cudaError_t launch_kg_d4(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k1t_d3(const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_kb_d3(int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                         cudaStream_t st, const void** fn);
cudaError_t launch_kb_d4_exact(const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                              cudaStream_t st, const void** fn);
cudaError_t launch_kb_d4_strict(const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                              cudaStream_t st, const void** fn);
cudaError_t launch_kb_d4_f32(const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                              cudaStream_t st, const void** fn);

cudaError_t launch_kc_d2(const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                         int64_t ldc, cudaStream_t st);
cudaError_t launch_kc_d3(const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                         int64_t ldc, cudaStream_t st);
cudaError_t launch_kc_d4(const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                         int64_t ldc, cudaStream_t st);

// the summation fused into a contraction over the permuted group (or the contraction alone)
cudaError_t launch_kc(int d, const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                      int64_t ldc, cudaStream_t st) {
  if (d == 2) return launch_kc_d2(kp, ar, sum, W, Y, ldw, C, ldc, st);
  if (d == 3) return launch_kc_d3(kp, ar, sum, W, Y, ldw, C, ldc, st);
  return launch_kc_d4(kp, ar, sum, W, Y, ldw, C, ldc, st);
}

cudaError_t launch_k1(int d, const KParams& kp, int ar, int vec, cudaStream_t st) {
  if (d == 2) return launch_k1_d2(kp, ar, vec, st);
  if (d == 3) return launch_k1_d3(kp, ar, vec, st);
  if (ar == AR_EXACT) return launch_k1_d4_exact(kp, st);
  if (ar == AR_STRICT) return launch_k1_d4_strict(kp, st);
  return launch_k1_d4_f32(kp, vec, st);
}

// TMA-staged orbit stream (3D; exact FP64 or FP32 arithmetic)
cudaError_t launch_k1t(int d, const KParams& kp, int ar, cudaStream_t st) {
  if (d != 3) return cudaErrorInvalidValue;
  return launch_k1t_d3(kp, ar, st);
}

// elements per member chunk of the K1T instantiations
int k1t_chunk(int d, int ar) {
  (void)d;
  return SS_K1T3_NCW * 32 * (ar == AR_EXACT ? 2 : 4);
}

// device address of the status word, per device (looked up once per device;
// several host threads may ask at once)
int* status_ptr() {
  static DeviceCache cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  long long v = 0;
  const int rc = cache.get(dev, &v, [](long long* val) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_status);
    *val = (long long)(uintptr_t)p;
    return (int)err;
  });
  return rc == 0 ? reinterpret_cast<int*>((uintptr_t)v) : nullptr;
}

// tiled kernel for the paper's N^d layout
cudaError_t launch_k2(int d, const KParams& kp, int ar, cudaStream_t st) {
  if (d == 2) return launch_k2_d2(kp, ar, st);
  if (d == 3) return launch_k2_d3(kp, ar, st);
  if (ar == AR_EXACT) return launch_k2_d4_exact(kp, st);
  if (ar == AR_STRICT) return launch_k2_d4_strict(kp, st);
  return launch_k2_d4_f32(kp, st);
}

cudaError_t launch_kg(int d, const KParams& kp, int ar, cudaStream_t st) {
  if (d == 2) return launch_kg_d2(kp, ar, st);
  return d == 3 ? launch_kg_d3(kp, ar, st) : launch_kg_d4(kp, ar, st);
}

// batched kernel of class (d, ar); with fn != nullptr only reports the kernel symbol
cudaError_t launch_kb(int d, int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                      cudaStream_t st, const void** fn) {
  if (d == 2) return launch_kb_d2(ar, probs, prefix, vecs, n, ctr, grid, st, fn);
  if (d == 3) return launch_kb_d3(ar, probs, prefix, vecs, n, ctr, grid, st, fn);
  if (ar == AR_EXACT) return launch_kb_d4_exact(probs, prefix, vecs, n, ctr, grid, st, fn);
  if (ar == AR_STRICT) return launch_kb_d4_strict(probs, prefix, vecs, n, ctr, grid, st, fn);
  return launch_kb_d4_f32(probs, prefix, vecs, n, ctr, grid, st, fn);
}

cudaError_t read_and_clear_status(int* out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_status, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
}

}  // namespace ss
