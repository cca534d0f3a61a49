// Packed antisymmetric storage (the tensor unpacking the paper names as a
// further use of its orbit traversal, Sec. 2 and Sec. 6): an antisymmetric
// tensor B over the permuted group is stored as P[s, r], one value per
// strictly increasing tuple t0 = (i_1 < .. < i_d) of colex rank
// r = sum_k C(i_k, k + 1) (the combinatorial number system).
//   unpack: B[s, t0 o tau] = sign(tau) P[s, r] for every tau in S_d, and
//           B[s, t] = 0 wherever t repeats an index;
//   pack:   P[s, r] = B[s, t0]  (the canonical member; the inverse of unpack
//           on antisymmetric tensors).
// Same traversal as the orbit-stream kernel: a block takes one orbit (one
// equality pattern) and a range of spectator chunks; the member offsets come
// from the unranked tuple; every element of P and B crosses HBM once.
#include "ss_kernels.cuh"

namespace ss {

// parity of permutation n of S_D in lexicographic order, as a sign
template <int D>
constexpr int perm_sign(int n) {
  const Sym<D> S = make_sym<D>();
  int inv = 0;
  for (int i = 0; i < D; i++)
    for (int j = i + 1; j < D; j++)
      if (S.p[n][i] > S.p[n][j]) inv++;
  return (inv & 1) ? -1 : 1;
}

template <int D>
struct SignTable {
  int s[fact(D)] = {};
};
template <int D>
constexpr SignTable<D> make_signs() {
  SignTable<D> t{};
  for (int n = 0; n < fact(D); n++) t.s[n] = perm_sign<D>(n);
  return t;
}
template <int D>
__device__ constexpr SignTable<D> kSigns = make_signs<D>();

// pattern P's block of the grid: members of the orbit, spectator chunks
template <int D, int P, bool UNPACK, int VEC, typename T>
__device__ __forceinline__ void pk_body(const KParams& kp, int64_t orb, int64_t c0, int64_t c1) {
  constexpr int M = Pat<D, P>::M;
  __shared__ int64_t soff[24];
  __syncthreads();
  if (threadIdx.x < 32) {
    int val[4] = {0, 0, 0, 0};
    unrank<Pat<D, P>::ND>(orb, kp.O, val);
#pragma unroll
    for (int u = 0; u < M; u++) {
      if (threadIdx.x == (u & 31)) {
        int64_t b = 0;
#pragma unroll
        for (int k = 0; k < D; k++) b += (int64_t)val[Pat<D, P>::lab(u, k)] * kp.ldb[k];
        soff[u] = b;
      }
    }
  }
  __syncthreads();
  const T* Pp = static_cast<const T*>(kp.A);
  T* Bp = static_cast<T*>(kp.B);
  const int64_t poff = orb * kp.lda[0];  // packed index stride (pattern 0 only)
  const int64_t step = (int64_t)blockDim.x * VEC;
  for (int64_t c = c0; c < c1; c++) {
    const int64_t s = c * step + (int64_t)threadIdx.x * VEC;
    if (s >= kp.S) break;
    if constexpr (UNPACK) {
      T x[VEC];
      if constexpr (P == 0) vload<T, VEC>(Pp + poff + s, x);
#pragma unroll
      for (int u = 0; u < M; u++) {
        T v[VEC];
#pragma unroll
        for (int e = 0; e < VEC; e++) v[e] = P == 0 ? (kSigns<D>.s[u] > 0 ? x[e] : -x[e]) : T(0);
        vstore<T, VEC>(Bp + soff[u] + s, v);
      }
    } else if constexpr (P == 0) {
      T x[VEC];
      vload<T, VEC>(static_cast<const T*>(kp.B) + soff[0] + s, x);
      vstore<T, VEC>(const_cast<T*>(Pp) + poff + s, x);
    }
  }
}

template <int D, bool UNPACK, int VEC, typename T>
__global__ void __launch_bounds__(256) pk_kernel(const __grid_constant__ KParams kp) {
  const int64_t b = blockIdx.x;
  const int p = find_pattern<D>(kp.pre, b);
  const int64_t bpo = (kp.nchunk + kp.cpb - 1) / kp.cpb;
  const int64_t local = b - kp.pre[p];
  const int64_t orb = local / bpo;
  const int64_t c0 = (local - orb * bpo) * kp.cpb;
  const int64_t c1 = min(kp.nchunk, c0 + kp.cpb);
  switch (p) {
    case 0: pk_body<D, 0, UNPACK, VEC, T>(kp, orb, c0, c1); break;
    case 1: pk_body<D, 1, UNPACK, VEC, T>(kp, orb, c0, c1); break;
    case 2: if constexpr (npatterns(D) > 2) pk_body<D, 2, UNPACK, VEC, T>(kp, orb, c0, c1); break;
    case 3: if constexpr (npatterns(D) > 3) pk_body<D, 3, UNPACK, VEC, T>(kp, orb, c0, c1); break;
    default:
      if constexpr (D == 4) {
        switch (p) {
          case 4: pk_body<D, 4, UNPACK, VEC, T>(kp, orb, c0, c1); break;
          case 5: pk_body<D, 5, UNPACK, VEC, T>(kp, orb, c0, c1); break;
          case 6: pk_body<D, 6, UNPACK, VEC, T>(kp, orb, c0, c1); break;
          case 7: pk_body<D, 7, UNPACK, VEC, T>(kp, orb, c0, c1); break;
        }
      }
  }
}

template <int D, bool UNPACK, typename T>
cudaError_t launch_pk_t(const KParams& kp, int vec, cudaStream_t st) {
  const dim3 grid((unsigned)kp.pre[npatterns(D)]), block(256);
  if (vec == 2) pk_kernel<D, UNPACK, 2, T><<<grid, block, 0, st>>>(kp);
  else pk_kernel<D, UNPACK, 1, T><<<grid, block, 0, st>>>(kp);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_pk_d(const KParams& kp, bool unpack, bool f64, int vec, cudaStream_t st) {
  if (f64) return unpack ? launch_pk_t<D, true, double>(kp, vec, st) : launch_pk_t<D, false, double>(kp, vec, st);
  return unpack ? launch_pk_t<D, true, float>(kp, vec, st) : launch_pk_t<D, false, float>(kp, vec, st);
}

// kp: A = P (packed), lda[0] = its packed-index stride; B = the full tensor,
// ldb[0..d-1] its permuted strides; S spectator positions (dense, stride 1)
cudaError_t launch_pack(int d, const KParams& kp, bool unpack, bool f64, int vec, cudaStream_t st) {
  if (d == 2) return launch_pk_d<2>(kp, unpack, f64, vec, st);
  if (d == 3) return launch_pk_d<3>(kp, unpack, f64, vec, st);
  return launch_pk_d<4>(kp, unpack, f64, vec, st);
}
}  // namespace ss
