#pragma once
// KC: the spin summation fused into the contraction it feeds (Sec. 1: the
// spin-summed intermediates of CC theory enter tensor contractions; Sec. 6).
//
//   C[s, y] = sum_t S(A)[s, t] * W[y, t]   (SUM = true)
//   C[s, y] = sum_t A[s, t] * W[y, t]      (SUM = false: the contraction alone)
//
// over the O^d tuples t of the permuted group, for every spectator position s
// (dense, column-major A: each tuple owns a contiguous run of S positions).
// A thread owns one position s and YT consecutive columns y of C, kept in
// FP64 registers. The CTA walks every orbit of every equality pattern (the
// same orbits as K1, in colex order of their canonical tuples); per orbit each
// thread loads its m member values (coalesced across the warp), applies the
// orbit operator in registers (the same cores as K1: exact fixed point or
// strict FP64), and multiplies the m results into its accumulators with the
// W entries of the m tuples (one address for the whole warp: a broadcast from
// L1). S(A) is never written: the summation costs one read of A instead of a
// write and a re-read of S(A). The FP64 multiply-adds (Y per element of A)
// run on the FP64 pipe, which bounds the kernel for Y >= 2; the exact core
// therefore converts its fixed-point sums to FP64 with integer instructions
// (fixed_to_double<true>), leaving the FP64 pipe to the multiply-adds.
#include "ss_kernels.cuh"

namespace ss {

constexpr int KC_THREADS = 64;

// next strictly increasing tuple of ND values in [0, O) in colex order
template <int ND>
__device__ __forceinline__ void colex_next(int (&v)[4], int O) {
#pragma unroll
  for (int i = 0; i < ND; i++) {
    const int lim = (i + 1 < ND) ? v[i + 1] : O;
    if (v[i] + 1 < lim) {
      v[i]++;
#pragma unroll
      for (int j = 0; j < i; j++) v[j] = j;
      return;
    }
  }
}

template <int D, int P, int AR, int YT, bool SUM>
__device__ __forceinline__ void kc_pattern(const KParams& kp, const double* __restrict__ W, int64_t ldw, int ny,
                                           int64_t s, bool act, double (&acc)[YT]) {
  constexpr int M = Pat<D, P>::M, ND = Pat<D, P>::ND;
  const double* A = static_cast<const double*>(kp.A);
  int64_t opow[4] = {1, 1, 1, 1};
#pragma unroll
  for (int k = 1; k < D; k++) opow[k] = opow[k - 1] * kp.O;
  int v[4] = {0, 1, 2, 3};
  const int64_t nor = kp.norb[P];
  for (int64_t o = 0; o < nor; o++) {
    int64_t offA[M], tw[M];
#pragma unroll
    for (int u = 0; u < M; u++) {
      int64_t a = 0, t = 0;
#pragma unroll
      for (int k = 0; k < D; k++) {
        const int x = v[Pat<D, P>::lab(u, k)];
        a += (int64_t)x * kp.lda[k];
        t += (int64_t)x * opow[k];
      }
      offA[u] = a;
      tw[u] = t;
    }
    double x[M], y[M];
#pragma unroll
    for (int u = 0; u < M; u++) x[u] = act ? A[offA[u] + s] : 0.0;
    if constexpr (SUM) {
      apply_group<D, P, AR, double, 0, true>(kp, x, y);
    } else {
#pragma unroll
      for (int u = 0; u < M; u++) y[u] = x[u];
    }
#pragma unroll
    for (int u = 0; u < M; u++) {
      const double* w = W + ldw * tw[u];
#pragma unroll
      for (int j = 0; j < YT; j++) acc[j] = fma(y[u], j < ny ? w[j] : 0.0, acc[j]);
    }
    colex_next<ND>(v, kp.O);
  }
}

template <int D, int AR, int YT, bool SUM>
__global__ void __launch_bounds__(KC_THREADS) kc_kernel(const __grid_constant__ KParams kp, const double* __restrict__ W,
                                                        int64_t Y, int64_t ldw, double* __restrict__ C, int64_t ldc) {
  const int64_t s = (int64_t)blockIdx.x * KC_THREADS + threadIdx.x;
  const int64_t y0 = (int64_t)blockIdx.y * YT;
  const int ny = (int)min((int64_t)YT, Y - y0);
  const bool act = s < kp.S;
  const double* Wt = W + y0;
  double acc[YT];
#pragma unroll
  for (int j = 0; j < YT; j++) acc[j] = 0.0;
  kc_pattern<D, 0, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
  kc_pattern<D, 1, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
  if constexpr (D >= 3) {
    kc_pattern<D, 2, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
    kc_pattern<D, 3, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
  }
  if constexpr (D == 4) {
    kc_pattern<D, 4, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
    kc_pattern<D, 5, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
    kc_pattern<D, 6, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
    kc_pattern<D, 7, AR, YT, SUM>(kp, Wt, ldw, ny, s, act, acc);
  }
  if (act) {
#pragma unroll
    for (int j = 0; j < YT; j++)
      if (j < ny) C[s + ldc * (y0 + j)] = acc[j];
  }
}

// one y-tile width per launch: 4, 8, 16 or 32 columns of C per thread
template <int D, int AR, bool SUM>
cudaError_t launch_kc_impl(const KParams& kp, const double* W, int64_t Y, int64_t ldw, double* C, int64_t ldc,
                           cudaStream_t st) {
  const int yt = Y <= 4 ? 4 : (Y <= 8 ? 8 : (Y <= 16 || D == 4 ? 16 : 32));
  const dim3 grid((unsigned)((kp.S + KC_THREADS - 1) / KC_THREADS), (unsigned)((Y + yt - 1) / yt));
  if (yt == 4) kc_kernel<D, AR, 4, SUM><<<grid, KC_THREADS, 0, st>>>(kp, W, Y, ldw, C, ldc);
  else if (yt == 8) kc_kernel<D, AR, 8, SUM><<<grid, KC_THREADS, 0, st>>>(kp, W, Y, ldw, C, ldc);
  else if (yt == 16) kc_kernel<D, AR, 16, SUM><<<grid, KC_THREADS, 0, st>>>(kp, W, Y, ldw, C, ldc);
  else if constexpr (D < 4) kc_kernel<D, AR, 32, SUM><<<grid, KC_THREADS, 0, st>>>(kp, W, Y, ldw, C, ldc);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_kc_d(const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                        int64_t ldc, cudaStream_t st) {
  if (!sum) return launch_kc_impl<D, AR_STRICT, false>(kp, W, Y, ldw, C, ldc, st);
  if (ar == AR_EXACT) return launch_kc_impl<D, AR_EXACT, true>(kp, W, Y, ldw, C, ldc, st);
  return launch_kc_impl<D, AR_STRICT, true>(kp, W, Y, ldw, C, ldc, st);
}

}  // namespace ss
