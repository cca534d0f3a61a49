// K1T: the orbit-stream kernel with TMA staging (sm_90+ bulk async copies,
// here for sm_103a).
//
// A persistent CTA = NCW consumer warps + 1 producer warp. Work is a sequence
// of tiles (orbit, spectator chunk of CH = NCW*32*VEC positions). For each
// tile the producer thread issues one cp.async.bulk per orbit member (m <= d!
// contiguous runs of CH elements) into a shared-memory stage and arms the
// stage's "full" mbarrier with the byte count; the consumers wait on it, read
// their positions of every member from shared memory, apply the orbit
// operator in registers, write the m results with coalesced vector stores,
// and release the stage through its "empty" mbarrier. NST stages form a ring,
// so the loads of the next tiles are in flight while the current one is
// computed: every element of A crosses HBM once (into shared memory) and every
// element of B once (from registers).
//
// Every wait is bounded (kp.wait_limit polls): when one runs out the kernel
// records SPINSUM_ERR_TIMEOUT in the status word, waits (bounded again) for
// its own copies in flight, and returns; nothing traps or hangs.
#pragma once
#include "ss_devcache.h"
#include "ss_kernels.cuh"

namespace ss {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void report_timeout(const KParams& kp) {
  if (kp.status) atomicExch(kp.status, 1);
}

// polls spent waiting for in-flight copies after a timeout
constexpr long long kDrainLimit = 1LL << 26;

struct TileMeta {
  int64_t offB[24];
  int64_t s0;
  int count;
  int p;
};

template <int D, int P>
__device__ __forceinline__ void member_offsets(const KParams& kp, int64_t orb, int64_t* offA, int64_t* offB) {
  constexpr int M = Pat<D, P>::M;
  int val[4] = {0, 0, 0, 0};
  unrank<Pat<D, P>::ND>(orb, kp.O, val);
#pragma unroll
  for (int u = 0; u < M; u++) {
    int64_t a = 0, b = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int t = val[Pat<D, P>::lab(u, k)];
      a += (int64_t)t * kp.lda[k];
      b += (int64_t)t * kp.ldb[k];
    }
    offA[u] = a;
    offB[u] = b;
  }
}

template <int D>
__device__ __forceinline__ int pattern_members(int p) {
  if constexpr (D == 3) {
    constexpr int m[4] = {6, 3, 3, 1};
    return m[p];
  } else {
    constexpr int m[8] = {24, 12, 12, 12, 6, 4, 4, 1};
    return m[p];
  }
}

template <int D>
__device__ __forceinline__ void tile_offsets(const KParams& kp, int p, int64_t orb, int64_t* offA, int64_t* offB) {
  switch (p) {
    case 0: member_offsets<D, 0>(kp, orb, offA, offB); break;
    case 1: member_offsets<D, 1>(kp, orb, offA, offB); break;
    case 2: member_offsets<D, 2>(kp, orb, offA, offB); break;
    case 3: member_offsets<D, 3>(kp, orb, offA, offB); break;
    default:
      if constexpr (D == 4) {
        switch (p) {
          case 4: member_offsets<D, 4>(kp, orb, offA, offB); break;
          case 5: member_offsets<D, 5>(kp, orb, offA, offB); break;
          case 6: member_offsets<D, 6>(kp, orb, offA, offB); break;
          case 7: member_offsets<D, 7>(kp, orb, offA, offB); break;
        }
      }
  }
}

// consumer side of one tile of pattern P: shared memory -> registers -> B
template <int D, int P, int AR, int VEC, typename T, int CH>
__device__ __forceinline__ void k1t_consume(const KParams& kp, const T* stage, const TileMeta& me, int tid) {
  constexpr int M = Pat<D, P>::M;
  const int e = tid * VEC;
  if (e >= me.count) return;
  T x[VEC][M], y[VEC][M];
#pragma unroll
  for (int u = 0; u < M; u++) {
    T v[VEC];
    vload<T, VEC>(stage + u * CH + e, v);
#pragma unroll
    for (int i = 0; i < VEC; i++) x[i][u] = v[i];
  }
#pragma unroll
  for (int i = 0; i < VEC; i++) apply_group<D, P, AR, T>(kp, x[i], y[i]);
  T* B = static_cast<T*>(kp.B);
  const bool beta = kp.flags & KF_BETA;
  const T bt = beta_of<T>(kp);
#pragma unroll
  for (int u = 0; u < M; u++) {
    T v[VEC];
    T* dst = B + me.offB[u] + me.s0 + e;
    if (beta) {
      vload<T, VEC>(dst, v);
#pragma unroll
      for (int i = 0; i < VEC; i++) v[i] = add_beta(y[i][u], v[i], bt);
    } else {
#pragma unroll
      for (int i = 0; i < VEC; i++) v[i] = y[i][u];
    }
    vstore<T, VEC>(dst, v);
  }
}

template <int D, int AR, int VEC, typename T, int NCW, int NST>
__global__ void __launch_bounds__((NCW + 1) * 32) k1t_kernel(const __grid_constant__ KParams kp) {
  constexpr int CH = NCW * 32 * VEC;
  constexpr int MMAX = fact(D);
  extern __shared__ __align__(128) unsigned char k1t_smem[];
  T* buf = reinterpret_cast<T*>(k1t_smem);
  __shared__ TileMeta meta[NST];
  __shared__ __align__(8) uint64_t full[NST];
  __shared__ __align__(8) uint64_t empty[NST];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t ntiles = kp.pre[npatterns(D)];
  if (warp == NCW) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    const T* A = static_cast<const T*>(kp.A);
    int k = 0;
    int64_t offA[24];
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, k++) {
      const int st = k % NST;
      if (k >= NST && !mbar_wait(&empty[st], ((k / NST) - 1) & 1, kp.wait_limit)) {
        report_timeout(kp);
        break;
      }
      const int p = find_pattern<D>(kp.pre, t);
      const int64_t local = t - kp.pre[p];
      const int64_t orb = local / kp.nchunk;
      const int64_t c = local - orb * kp.nchunk;
      TileMeta& me = meta[st];
      tile_offsets<D>(kp, p, orb, offA, me.offB);
      me.s0 = c * CH;
      me.count = (int)(kp.S - me.s0 < (int64_t)CH ? kp.S - me.s0 : (int64_t)CH);
      me.p = p;
      const int m = pattern_members<D>(p);
      const uint32_t bytes = (uint32_t)me.count * (uint32_t)sizeof(T);
      mbar_arrive_expect_tx(&full[st], bytes * (uint32_t)m);
      T* dst = buf + (size_t)st * MMAX * CH;
      for (int u = 0; u < m; u++) bulk_g2s(dst + u * CH, A + offA[u] + me.s0, bytes, &full[st]);
    }
    return;
  }
  // ---------------- consumers ----------------
  const int tid = threadIdx.x;
  int k = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, k++) {
    const int st = k % NST;
    if (!mbar_wait(&full[st], (k / NST) & 1, kp.wait_limit)) {
      report_timeout(kp);
      // let copies already issued into this CTA's shared memory land before exiting
      for (int j = 0; j < NST; j++) mbar_wait(&full[(k + j) % NST], ((k + j) / NST) & 1, kDrainLimit);
      return;
    }
    const TileMeta& me = meta[st];
    const T* stage = buf + (size_t)st * MMAX * CH;
    switch (me.p) {
      case 0: k1t_consume<D, 0, AR, VEC, T, CH>(kp, stage, me, tid); break;
      case 1: k1t_consume<D, 1, AR, VEC, T, CH>(kp, stage, me, tid); break;
      case 2: k1t_consume<D, 2, AR, VEC, T, CH>(kp, stage, me, tid); break;
      case 3: k1t_consume<D, 3, AR, VEC, T, CH>(kp, stage, me, tid); break;
      default:
        if constexpr (D == 4) {
          switch (me.p) {
            case 4: k1t_consume<D, 4, AR, VEC, T, CH>(kp, stage, me, tid); break;
            case 5: k1t_consume<D, 5, AR, VEC, T, CH>(kp, stage, me, tid); break;
            case 6: k1t_consume<D, 6, AR, VEC, T, CH>(kp, stage, me, tid); break;
            case 7: k1t_consume<D, 7, AR, VEC, T, CH>(kp, stage, me, tid); break;
          }
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

// launch configuration of one K1T instantiation
template <int D, int AR, int VEC, typename T, int NCW, int NST>
struct K1TConfig {
  static constexpr int CH = NCW * 32 * VEC;
  static constexpr int THREADS = (NCW + 1) * 32;
  static constexpr size_t SMEM = (size_t)NST * fact(D) * CH * sizeof(T);
};

template <int D, int AR, int VEC, typename T, int NCW, int NST>
cudaError_t launch_k1t_impl(const KParams& kp, cudaStream_t st) {
  using C = K1TConfig<D, AR, VEC, T, NCW, NST>;
  auto fn = k1t_kernel<D, AR, VEC, T, NCW, NST>;
  // resident CTAs per device (persistent grid), set up once per device
  static DeviceCache cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  long long ctas = 0;
  const int rc = cache.get(dev, &ctas, [&](long long* val) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (err != cudaSuccess) return (int)err;
    int sms = 0, nb = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return (int)err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, C::THREADS, C::SMEM);
    if (err != cudaSuccess) return (int)err;
    *val = (long long)sms * (nb > 0 ? nb : 1);
    return 0;
  });
  if (rc != 0) return rc < 0 ? cudaErrorInvalidDevice : (cudaError_t)rc;
  const int64_t ntiles = kp.pre[npatterns(D)];
  int64_t g = ctas;
  if (ntiles < g) g = ntiles;
  if (g < 1) g = 1;
  fn<<<(unsigned)g, C::THREADS, C::SMEM, st>>>(kp);
  return cudaGetLastError();
}

}  // namespace ss
