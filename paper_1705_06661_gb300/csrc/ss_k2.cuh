// K2: the tiled kernel for the paper's own layout, a dense N^d tensor whose
// permuted group includes the stride-1 index (Sec. 3.1), so that the members
// of an orbit are scattered single elements rather than contiguous runs.
//
// The index space is cut into tiles of BL^d elements (BL = 8 for d = 3,
// BL = 4 for d = 4). Tiles form orbits exactly as elements do: for a sorted
// tuple of block coordinates T0 the tiles T0 o tau hold, between them, every
// element orbit whose block coordinates are a rearrangement of T0 -- the
// d! blocks of Algorithm 5's macro-kernel (Sec. 4.5), all kept on chip at once.
// A CTA takes one block orbit:
//   1. copies its m_b <= d! tiles from HBM into shared memory (rows along the
//      stride-1 index, coalesced), with padded pitches so that the permuted
//      reads of step 2 hit few shared-memory banks;
//   2. each thread takes canonical in-tile offsets w of the first tile; the
//      element orbit of T0 * BL + w has its members in the tiles T0 o tau at
//      the permuted offsets w o tau (the renaming of Sec. 4.6.1, done per
//      element through shared memory). The thread reads them, applies the
//      orbit operator with the same cores as K1 and writes the results back to
//      the same shared-memory places (each place belongs to one orbit);
//   3. copies the tiles back to HBM (in place: the same addresses, after every
//      read of the block orbit is done).
// Partial tiles at the upper edge (N not a multiple of BL) are handled by
// bounds checks: an element orbit lies entirely inside or outside the tensor.
#pragma once
#include "ss_kernels.cuh"

namespace ss {

template <int D>
struct K2Shape;
template <>
struct K2Shape<3> {
  static constexpr int BL = 8, NT = 512;  // tile edge, elements per tile
  static constexpr int TS = 608;          // shared-memory slots per tile (padded)
  __device__ static constexpr int pitch(int k) { return k == 0 ? 1 : (k == 1 ? 9 : 76); }
};
template <>
struct K2Shape<4> {
  static constexpr int BL = 4, NT = 256;
  static constexpr int TS = 344;
  __device__ static constexpr int pitch(int k) { return k == 0 ? 1 : (k == 1 ? 4 : (k == 2 ? 21 : 87)); }
};

// For a block pattern BP and an element pattern EP (of a canonical element in
// a block orbit of pattern BP): member u of the element orbit lies in block
// member bm[u] of the block orbit, at in-tile offset w o tau[u].
template <int D>
struct K2Map {
  int bm[24] = {};
  int tau[24][4] = {};
  bool valid = false;
};

template <int D>
constexpr K2Map<D> make_k2map(int BP, int EP) {
  K2Map<D> r{};
  const Pattern<D> pe = make_pattern<D>(EP), pb = make_pattern<D>(BP);
  const Sym<D> S = make_sym<D>();
  // equal element values need equal blocks
  for (int i = 0; i < D; i++)
    for (int j = i + 1; j < D; j++)
      if (pe.lab[0][i] == pe.lab[0][j] && pb.lab[0][i] != pb.lab[0][j]) return r;
  for (int u = 0; u < pe.m; u++) {
    int tau = -1;
    for (int n = 0; n < fact(D) && tau < 0; n++) {
      bool same = true;
      for (int k = 0; k < D; k++) same = same && pe.lab[0][S.p[n][k]] == pe.lab[u][k];
      if (same) tau = n;
    }
    for (int k = 0; k < D; k++) r.tau[u][k] = S.p[tau][k];
    for (int v = 0; v < pb.m; v++) {
      bool same = true;
      for (int k = 0; k < D; k++) same = same && pb.lab[0][S.p[tau][k]] == pb.lab[v][k];
      if (same) r.bm[u] = v;
    }
  }
  r.valid = true;
  return r;
}

template <int D, int BP, int EP>
__device__ constexpr K2Map<D> kK2Map = make_k2map<D>(BP, EP);

// shared-memory slot of member u of an (BP, EP) element orbit at canonical offset w
template <int D, int BP, int EP>
__device__ __forceinline__ int k2_slot(int u, const int (&w)[4]) {
  int a = kK2Map<D, BP, EP>.bm[u] * K2Shape<D>::TS;
#pragma unroll
  for (int k = 0; k < D; k++) a += w[kK2Map<D, BP, EP>.tau[u][k]] * K2Shape<D>::pitch(k);
  return a;
}

template <int D, int BP, int EP, int AR, typename T>
__device__ __forceinline__ void k2_group(const KParams& kp, const int (&w)[4], T* sm) {
  constexpr int M = Pat<D, EP>::M;
  T x[M];
#pragma unroll
  for (int u = 0; u < M; u++) x[u] = sm[k2_slot<D, BP, EP>(u, w)];
  if constexpr (D == 4 && EP == 0 && AR == AR_EXACT) {
    const bool amul = kp.flags & KF_ALPHA_MUL;
    auto sink = [&](int u, double v) { sm[k2_slot<D, BP, EP>(u, w)] = amul ? __dmul_rn(kp.alpha, v) : v; };
    if (exact_core_grouped4<SS_4D_GROUPS>(kp, x, sink)) return;
    strict_core<D, EP>(kp, x);
#pragma unroll
    for (int u = 0; u < M; u++) sm[k2_slot<D, BP, EP>(u, w)] = __dmul_rn(kp.alpha, x[u]);
  } else {
    T y[M];
    apply_group<D, EP, AR, T>(kp, x, y);
#pragma unroll
    for (int u = 0; u < M; u++) sm[k2_slot<D, BP, EP>(u, w)] = y[u];
  }
}

// element pattern of the sorted tuple with adjacent-equality bits eq
template <int D>
__device__ __forceinline__ int k2_elem_pattern(unsigned eq) {
  if constexpr (D == 3) {
    constexpr int t[4] = {0, 1, 2, 3};  // bits: 1 = (0,1) equal, 2 = (1,2) equal
    return t[eq];
  } else {
    // bits 1 = (0,1), 2 = (1,2), 4 = (2,3) -> pattern index of ss_internal.h
    constexpr int t[8] = {0, 1, 2, 5, 3, 4, 6, 7};
    return t[eq];
  }
}

template <int D, int BP, int AR, typename T>
__device__ __forceinline__ void k2_dispatch(const KParams& kp, int ep, const int (&w)[4], T* sm) {
  switch (ep) {
    case 0: if constexpr (kK2Map<D, BP, 0>.valid) k2_group<D, BP, 0, AR, T>(kp, w, sm); break;
    case 1: if constexpr (kK2Map<D, BP, 1>.valid) k2_group<D, BP, 1, AR, T>(kp, w, sm); break;
    case 2: if constexpr (kK2Map<D, BP, 2>.valid) k2_group<D, BP, 2, AR, T>(kp, w, sm); break;
    case 3: if constexpr (kK2Map<D, BP, 3>.valid) k2_group<D, BP, 3, AR, T>(kp, w, sm); break;
    default:
      if constexpr (D == 4) {
        switch (ep) {
          case 4: if constexpr (kK2Map<D, BP, 4>.valid) k2_group<D, BP, 4, AR, T>(kp, w, sm); break;
          case 5: if constexpr (kK2Map<D, BP, 5>.valid) k2_group<D, BP, 5, AR, T>(kp, w, sm); break;
          case 6: if constexpr (kK2Map<D, BP, 6>.valid) k2_group<D, BP, 6, AR, T>(kp, w, sm); break;
          case 7: if constexpr (kK2Map<D, BP, 7>.valid) k2_group<D, BP, 7, AR, T>(kp, w, sm); break;
        }
      }
  }
}

template <int D, int BP, int AR, typename T>
__device__ __forceinline__ void k2_body(const KParams& kp, int64_t orb, T* sm) {
  using K = K2Shape<D>;
  constexpr int MB = Pat<D, BP>::M;
  const int N = kp.O;
  const int nb = (N + K::BL - 1) / K::BL;
  int val[4] = {0, 0, 0, 0};
  unrank<Pat<D, BP>::ND>(orb, nb, val);
  const T* A = static_cast<const T*>(kp.A);
  T* B = static_cast<T*>(kp.B);
  // block coordinates and origins (A and B element offsets) of the m_b tiles
  __shared__ int sblk[24][4];
  __shared__ int64_t sbase[2][24];
  __syncthreads();
  if (threadIdx.x < MB) {
    const int u = threadIdx.x;
    int64_t oa = 0, ob = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int bk = val[kPattern<D, BP>.lab[u][k]];
      sblk[u][k] = bk;
      oa += (int64_t)bk * K::BL * kp.lda[k];
      ob += (int64_t)bk * K::BL * kp.ldb[k];
    }
    sbase[0][u] = oa;
    sbase[1][u] = ob;
  }
  __syncthreads();
  // 1. tiles -> shared memory
  for (int i = threadIdx.x; i < MB * K::NT; i += blockDim.x) {
    const int u = i / K::NT;
    int e = i - u * K::NT;
    int64_t off = sbase[0][u];
    int slot = u * K::TS;
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int wk = e % K::BL;
      e /= K::BL;
      in = in && sblk[u][k] * K::BL + wk < N;
      off += (int64_t)wk * kp.lda[k];
      slot += wk * K::pitch(k);
    }
    if (in) sm[slot] = A[off];
  }
  __syncthreads();
  // 2. element orbits of the block orbit, in shared memory
  int T0[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; k++) T0[k] = val[Pat<D, BP>::lab(0, k)];
  for (int e0 = threadIdx.x; e0 < K::NT; e0 += blockDim.x) {
    int w[4] = {0, 0, 0, 0};
    int e = e0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      w[k] = e % K::BL;
      e /= K::BL;
    }
    bool ok = T0[D - 1] * K::BL + w[D - 1] < N;  // the largest coordinate of the sorted tuple
    unsigned eq = 0;
#pragma unroll
    for (int k = 0; k + 1 < D; k++) {
      if (T0[k] == T0[k + 1]) {
        ok = ok && w[k] <= w[k + 1];  // canonical: sorted within equal blocks
        if (w[k] == w[k + 1]) eq |= 1u << k;
      }
    }
    if (!ok) continue;
    k2_dispatch<D, BP, AR, T>(kp, k2_elem_pattern<D>(eq), w, sm);
  }
  __syncthreads();
  // 3. shared memory -> tiles (alpha applied; beta added here)
  const bool beta = kp.flags & KF_BETA;
  const T bt = beta_of<T>(kp);
  for (int i = threadIdx.x; i < MB * K::NT; i += blockDim.x) {
    const int u = i / K::NT;
    int e = i - u * K::NT;
    int64_t off = sbase[1][u];
    int slot = u * K::TS;
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int wk = e % K::BL;
      e /= K::BL;
      in = in && sblk[u][k] * K::BL + wk < N;
      off += (int64_t)wk * kp.ldb[k];
      slot += wk * K::pitch(k);
    }
    if (in) {
      T v = sm[slot];
      if (beta) v = add_beta(v, B[off], bt);
      B[off] = v;
    }
  }
}

template <int D, int AR, typename T>
__global__ void __launch_bounds__(256) k2_kernel(const __grid_constant__ KParams kp) {
  extern __shared__ __align__(16) unsigned char k2_smem[];
  T* sm = reinterpret_cast<T*>(k2_smem);
  const int64_t b = blockIdx.x;
  const int p = find_pattern<D>(kp.pre, b);
  const int64_t orb = b - kp.pre[p];
  switch (p) {
    case 0: k2_body<D, 0, AR, T>(kp, orb, sm); break;
    case 1: k2_body<D, 1, AR, T>(kp, orb, sm); break;
    case 2: k2_body<D, 2, AR, T>(kp, orb, sm); break;
    case 3: k2_body<D, 3, AR, T>(kp, orb, sm); break;
    default:
      if constexpr (D == 4) {
        switch (p) {
          case 4: k2_body<D, 4, AR, T>(kp, orb, sm); break;
          case 5: k2_body<D, 5, AR, T>(kp, orb, sm); break;
          case 6: k2_body<D, 6, AR, T>(kp, orb, sm); break;
          case 7: k2_body<D, 7, AR, T>(kp, orb, sm); break;
        }
      }
  }
}

template <int D, int AR, typename T>
cudaError_t launch_k2_impl(const KParams& kp, cudaStream_t st) {
  constexpr size_t smem = (size_t)fact(D) * K2Shape<D>::TS * sizeof(T);
  auto fn = k2_kernel<D, AR, T>;
  constexpr int MAXDEV = 64;
  static bool init[MAXDEV] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
  if (!init[dev]) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    init[dev] = true;
  }
  fn<<<(unsigned)kp.pre[npatterns(D)], 256, smem, st>>>(kp);
  return cudaGetLastError();
}

}  // namespace ss
