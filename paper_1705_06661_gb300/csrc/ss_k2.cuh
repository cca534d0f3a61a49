// K2: the tiled kernel for the paper's own layout, a dense N^d tensor whose
// permuted group includes the stride-1 index (Sec. 3.1), so that the members
// of an orbit are scattered single elements rather than contiguous runs.
//
// The index space is cut into tiles of BL^d elements (BL = 8 for d = 3,
// BL = 4 for d = 4). Tiles form orbits exactly as elements do: for a sorted
// tuple of block coordinates T0 the tiles T0 o tau hold, between them, every
// element orbit whose block coordinates are a rearrangement of T0 -- the
// d! blocks of Algorithm 5's macro-kernel (Sec. 4.5), all kept on chip at once.
// A CTA works through block orbits:
//   1. copies the m_b <= d! tiles of a block orbit from HBM into shared memory
//      (rows along the stride-1 index, coalesced 16-byte copies; asynchronous,
//      one block orbit ahead of the one being computed);
//   2. each thread takes canonical in-tile offsets w of the first tile; the
//      element orbit of T0 * BL + w has its members in the tiles T0 o tau at
//      the permuted offsets w o tau (the renaming of Sec. 4.6.1, done per
//      element through shared memory). The thread reads them, applies the
//      orbit operator with the same cores as K1 and writes the results back to
//      the same shared-memory places (each place belongs to one orbit);
//   3. copies the tiles back to HBM (in place: the same addresses, after every
//      read of the block orbit is done).
// Tiles are stored densely in shared memory with an XOR swizzle of the 16-byte
// unit within each row (and, for d = 4, of the row within each 128-byte line),
// chosen so that the permuted reads of step 2 -- a warp takes a 4x4x2 (d = 3)
// or 4x2x2x2 (d = 4) block of canonical offsets -- touch every shared-memory
// bank equally for all d! permutations, while the copies of steps 1 and 3 keep
// 16-byte units whole.
// Partial tiles at the upper edge (N not a multiple of BL) are handled by
// bounds checks: an element orbit lies entirely inside or outside the tensor.
#pragma once
#include "ss_devcache.h"
#include "ss_kernels.cuh"

namespace ss {

template <int D>
struct K2Shape;
template <>
struct K2Shape<2> {
  static constexpr int BL = 32, NT = 1024;  // 32 x 32 tiles: 256-byte rows
  // the pair index c0 / 2 is XORed with c1 mod 16
  __device__ static __forceinline__ int phys(const int (&c)[4]) {
    return ((((c[0] >> 1) ^ (c[1] & 15)) << 1) | (c[0] & 1)) + 32 * c[1];
  }
  // warp e / 32 takes the 16 x 2 block ((e >> 5) & 1, e >> 6) of the tile,
  // lane l its element (l & 15, l >> 4)
  __host__ __device__ static constexpr void elem(int e, int (&w)[4]) {
    const int l = e & 31, b = e >> 5;
    w[0] = (l & 15) + 16 * (b & 1);
    w[1] = (l >> 4) + 2 * (b >> 1);
    w[2] = 0;
    w[3] = 0;
  }
};
template <>
struct K2Shape<3> {
  static constexpr int BL = 8, NT = 512;  // tile edge, elements per tile
  // shared-memory place of in-tile offset c: the pair index c0 / 2 is XORed
  // with (c1 ^ c2) mod 4
  __device__ static __forceinline__ int phys(const int (&c)[4]) {
    return ((((c[0] >> 1) ^ ((c[1] ^ c[2]) & 3)) << 1) | (c[0] & 1)) + 8 * c[1] + 64 * c[2];
  }
  // canonical offsets of element e (0..511): warp e / 32 takes the 4x4x2 block
  // ((e >> 5) & 1, (e >> 6) & 1, e >> 7) of the tile, lane l its element
  // (l & 3, (l >> 2) & 3, l >> 4)
  __host__ __device__ static constexpr void elem(int e, int (&w)[4]) {
    const int l = e & 31, b = e >> 5;
    w[0] = (l & 3) + 4 * (b & 1);
    w[1] = ((l >> 2) & 3) + 4 * ((b >> 1) & 1);
    w[2] = (l >> 4) + 2 * (b >> 2);
    w[3] = 0;
  }
};
template <>
struct K2Shape<4> {
  static constexpr int BL = 4, NT = 256;
  // pair bit c0 / 2 XORed with c1.0 ^ c3.0, row c1 XORed with
  // (c3.1, c2.0 ^ c2.1 ^ c3.1)
  __device__ static __forceinline__ int phys(const int (&c)[4]) {
    const int x = c[0] ^ (((c[1] ^ c[3]) & 1) << 1);
    const int g = (c[3] >> 1) | ((((c[2] ^ (c[2] >> 1)) ^ (c[3] >> 1)) & 1) << 1);
    return x + 4 * (c[1] ^ g) + 16 * c[2] + 64 * c[3];
  }
  // warp e / 32 takes the 4x2x2x2 block (0, b & 1, (b >> 1) & 1, b >> 2) * 2
  __host__ __device__ static constexpr void elem(int e, int (&w)[4]) {
    const int l = e & 31, b = e >> 5;
    w[0] = l & 3;
    w[1] = ((l >> 2) & 1) + 2 * (b & 1);
    w[2] = ((l >> 3) & 1) + 2 * ((b >> 1) & 1);
    w[3] = (l >> 4) + 2 * (b >> 2);
  }
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
  int c[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; k++) c[k] = w[kK2Map<D, BP, EP>.tau[u][k]];
  return kK2Map<D, BP, EP>.bm[u] * K2Shape<D>::NT + K2Shape<D>::phys(c);
}

// whether the kernel keeps a slot table for the generic orbits (d = 4, transform core)
template <int D, int AR>
__host__ __device__ constexpr bool k2_slot_table() {
  return SS_K2_SLOTS4 && D == 4 && AR == AR_EXACT_XW;
}

// the strict core for an element orbit whose exponents leave the fixed-point
// range: rare, kept out of line so that it holds no registers in the hot path
template <int D, int BP, int EP>
static __device__ __noinline__ void k2_strict_group(const KParams& kp, const int* wp, double* sm) {
  constexpr int M = Pat<D, EP>::M;
  const int w[4] = {wp[0], wp[1], wp[2], wp[3]};
  double x[M];
  for (int u = 0; u < M; u++) x[u] = sm[k2_slot<D, BP, EP>(u, w)];
  strict_core<D, EP>(kp, x);
  for (int u = 0; u < M; u++) sm[k2_slot<D, BP, EP>(u, w)] = __dmul_rn(kp.alpha, x[u]);
}

template <int D, int BP, int EP, int AR, typename T>
__device__ __forceinline__ void k2_group(const KParams& kp, const int (&w)[4], T* sm,
                                         const unsigned short* sl = nullptr) {
  constexpr int M = Pat<D, EP>::M;
  if constexpr (D == 4 && AR == AR_EXACT_XW) {
    // slots are recomputed where they are used rather than kept in registers
    // (the generic orbit of a generic block orbit reads them from the
    // thread's column of the slot table sl when there is one); the strict
    // core stays out of line (inlined, the compiler may predicate its FP64
    // operations into the common path)
    auto slot = [&](int u) {
      if constexpr (BP == 0 && EP == 0 && SS_K2_SLOTS4) return (int)sl[u * 256 + threadIdx.x];
      else return k2_slot<D, BP, EP>(u, w);
    };
    T x[M];
#pragma unroll
    for (int u = 0; u < M; u++) x[u] = sm[slot(u)];
    if constexpr (wht_ok<EP>()) {
      auto sink = [&](int u, double v) { sm[slot(u)] = v; };
      if (!exact_core_wht4<EP>(kp, x, sink)) k2_strict_group<D, BP, EP>(kp, w, sm);
    } else {
      T y[M];
      if (exact_core<D, EP>(kp, x, y)) {
#pragma unroll
        for (int u = 0; u < M; u++) sm[k2_slot<D, BP, EP>(u, w)] = y[u];
      } else {
        k2_strict_group<D, BP, EP>(kp, w, sm);
      }
    }
    return;
  }
  constexpr int ARC = AR == AR_EXACT_XW ? (int)AR_EXACT : AR;
  int s[M];
#pragma unroll
  for (int u = 0; u < M; u++) s[u] = k2_slot<D, BP, EP>(u, w);
  T x[M];
#pragma unroll
  for (int u = 0; u < M; u++) x[u] = sm[s[u]];
  if constexpr (D == 4 && EP == 0 && ARC == AR_EXACT) {
    auto sink = [&](int u, double v) { sm[s[u]] = v; };
    if (exact_core_grouped4<SS_4D_GROUPS>(kp, x, sink)) {
      if (kp.flags & KF_ALPHA_MUL) {  // alpha not a power of two: rare, a separate pass
#pragma unroll
        for (int u = 0; u < M; u++) sm[s[u]] = __dmul_rn(kp.alpha, sm[s[u]]);  // unrolled: s stays in registers
      }
      return;
    }
    strict_core<D, EP>(kp, x);
#pragma unroll
    for (int u = 0; u < M; u++) sm[s[u]] = __dmul_rn(kp.alpha, x[u]);
  } else {
    T y[M];
    apply_group<D, EP, ARC, T>(kp, x, y);
#pragma unroll
    for (int u = 0; u < M; u++) sm[s[u]] = y[u];
  }
}

// element pattern of the sorted tuple with adjacent-equality bits eq
// (d = 3: bit 0 = (0,1), bit 1 = (1,2) equal; d = 4: bits (0,1), (1,2), (2,3)),
// as a pattern index of ss_internal.h; a packed table, not a local-memory array
template <int D>
__host__ __device__ constexpr int k2_elem_pattern(unsigned eq) {
  if constexpr (D <= 3) {  // d = 2: bit 0 = (0,1) equal
    return (int)eq;
  } else {
    return (int)((0x76435210u >> (4 * eq)) & 0xFu);  // eq 0..7 -> 0 1 2 5 3 4 6 7
  }
}

// The canonical in-tile offsets of a block orbit of pattern BP > 0 (some
// block coordinates equal), with their element patterns, grouped by element
// pattern: threads take consecutive entries, so the warps of a degenerate
// block orbit mostly run one element pattern's code (in tile order they
// would branch into up to d! pattern bodies, each run with a few lanes).
// Entry: w_0 .. w_3 in bytes 0..3 (w_k < 32), element pattern in bits 29..31.
template <int D>
struct K2List {
  int n = 0;
  unsigned e[1024] = {};
};

template <int D, int BP>
constexpr K2List<D> make_k2list() {
  using K = K2Shape<D>;
  K2List<D> r{};
  const Pattern<D> pb = make_pattern<D>(BP);
  for (int ep = 0; ep < npatterns(D); ep++)
    for (int e0 = 0; e0 < K::NT; e0++) {
      int w[4] = {0, 0, 0, 0};
      K::elem(e0, w);
      bool ok = true;
      unsigned eq = 0;
      for (int k = 0; k + 1 < D; k++)
        if (pb.lab[0][k] == pb.lab[0][k + 1]) {
          ok = ok && w[k] <= w[k + 1];
          if (w[k] == w[k + 1]) eq |= 1u << k;
        }
      if (!ok || k2_elem_pattern<D>(eq) != ep) continue;
      r.e[r.n++] = (unsigned)w[0] | ((unsigned)w[1] << 8) | ((unsigned)w[2] << 16) | ((unsigned)w[3] << 24 & 0x1F000000u) |
                   ((unsigned)ep << 29);
    }
  return r;
}

template <int D, int BP>
__device__ constexpr K2List<D> kK2List = make_k2list<D, BP>();

template <int D, int BP, int AR, typename T>
__device__ __forceinline__ void k2_dispatch(const KParams& kp, int ep, const int (&w)[4], T* sm) {
  switch (ep) {
    case 0: if constexpr (kK2Map<D, BP, 0>.valid) k2_group<D, BP, 0, AR, T>(kp, w, sm); break;
    case 1: if constexpr (kK2Map<D, BP, 1>.valid) k2_group<D, BP, 1, AR, T>(kp, w, sm); break;
    case 2: if constexpr (npatterns(D) > 2) { if constexpr (kK2Map<D, BP, 2>.valid) k2_group<D, BP, 2, AR, T>(kp, w, sm); } break;
    case 3: if constexpr (npatterns(D) > 3) { if constexpr (kK2Map<D, BP, 3>.valid) k2_group<D, BP, 3, AR, T>(kp, w, sm); } break;
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

// asynchronous global -> shared copies (cp.async, completion by commit groups);
// 16-byte units bypass L1
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One block orbit as the CTA sees it: the sorted block tuple (pattern bp,
// distinct values val), and per tile member u its A and B origins, its extent
// left before the upper edge of the tensor per dimension, and whether it is a
// full tile. bp < 0 marks the end of the CTA's list.
struct K2Desc {
  int64_t base[2][24];
  int lim[24][4];
  unsigned char full[24];
  int64_t id;
  int bp, mb;
  int allfull;  // every tile of the block orbit is a full tile
  int val[4];
};

// lanes u < m_b of one warp fill the tile table of a block orbit of pattern BP
template <int D, int BP>
__device__ __forceinline__ void k2_fill(const KParams& kp, const int (&val)[4], K2Desc& dsc) {
  using K = K2Shape<D>;
  constexpr int MB = Pat<D, BP>::M;
  const int u = threadIdx.x & 31;
  if (u == 0) {
    dsc.bp = BP;
    dsc.mb = MB;
  }
  if (u < D) dsc.val[u] = u == 0 ? val[0] : (u == 1 ? val[1] : (u == 2 ? val[2] : val[3]));
  bool full = true;
  if (u < MB) {
    int64_t oa = 0, ob = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int l = kPattern<D, BP>.lab[u][k];  // selects, not a local-memory index
      const int bk = l == 0 ? val[0] : (l == 1 ? val[1] : (l == 2 ? val[2] : val[3]));
      dsc.lim[u][k] = kp.O - bk * K::BL;
      full = full && kp.O - bk * K::BL >= K::BL;
      oa += (int64_t)bk * K::BL * kp.lda[k];
      ob += (int64_t)bk * K::BL * kp.ldb[k];
    }
    dsc.base[0][u] = oa;
    dsc.base[1][u] = ob;
    dsc.full[u] = full;
  }
  const unsigned part = __ballot_sync(0xffffffffu, !full);
  if (u == 0) dsc.allfull = part == 0;
}

// Colex unranking as in unrank(), by a whole warp at once: the candidates c of
// each position are tested 32 at a time (C(c, i + 1) grows with c, so the
// qualifying c form a prefix and the answer is its last element). Every lane
// returns the same tuple; all 32 lanes must be active.
template <int ND>
__device__ __forceinline__ void unrank_warp(int64_t r, int O, int (&v)[4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = ND - 1; i >= 0; i--) {
    int cnt = 0;
    for (int c0 = i; c0 < O; c0 += 32) {
      const int c = c0 + lane;
      const unsigned m = __ballot_sync(0xffffffffu, c < O && binom(c, i + 1) <= r);
      cnt += __popc(m);
      if (m != 0xffffffffu) break;
    }
    v[i] = i + cnt - 1;
    r -= binom(v[i], i + 1);
  }
}

// Work ids and block orbits. Block orbits are visited in groups: the sorted
// tuple c of coarse blocks (F tiles per edge, F = 2^k2lf) is unranked from
// id / F^d as a multiset (colex rank of the strictly increasing c_k + k), and
// the F^d consecutive ids of the group take the fine tuples b_k = F c_k +
// delta_k. Sorted fine tuples need delta non-decreasing where c repeats; the
// other ids of a group are skipped. A CTA takes a run of consecutive ids
// (or, persistent, every G-th id); the hardware starts CTAs in order, so the
// ids in flight at any time form a compact window of consecutive groups:
// every tile row of the F^d tiles of a coarse tile (F x BL x sizeof(T)
// contiguous bytes) is read and written at about the same time, and the
// coarse block orbits in flight lie close together in the colex order.
// One whole warp finds the first valid id in [id, end) (step `step`) and
// fills dsc; bp = -1 when there is none.
template <int D>
__device__ __forceinline__ void k2_next(const KParams& kp, int64_t id, int64_t step, int64_t end, K2Desc& dsc) {
  const int lf = kp.k2lf;
  const int nb = (kp.O + K2Shape<D>::BL - 1) / K2Shape<D>::BL;
  const int nc = ((nb - 1) >> lf) + 1;
  const int fm = (1 << lf) - 1;
  for (; id < end; id += step) {
    int v[4] = {0, 0, 0, 0};
    unrank_warp<D>(id >> (D * lf), nc + D - 1, v);
    const unsigned dl = (unsigned)id & ((1u << (D * lf)) - 1u);
    int b[4] = {0, 0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; k++) {
      b[k] = ((v[k] - k) << lf) + (int)((dl >> (k * lf)) & fm);
      ok = ok && b[k] < nb;
    }
    unsigned eq = 0;
    int val[4] = {b[0], 0, 0, 0};
    int j = 0;
#pragma unroll
    for (int k = 0; k + 1 < D; k++) {
      ok = ok && b[k] <= b[k + 1];
      if (b[k] == b[k + 1]) {
        eq |= 1u << k;
      } else {
        j++;
        if (j == 1) val[1] = b[k + 1];
        if (j == 2) val[2] = b[k + 1];
        if (j == 3) val[3] = b[k + 1];
      }
    }
    if (!ok) continue;
    if ((threadIdx.x & 31) == 0) dsc.id = id;
    switch (k2_elem_pattern<D>(eq)) {
      case 0: k2_fill<D, 0>(kp, val, dsc); break;
      case 1: k2_fill<D, 1>(kp, val, dsc); break;
      case 2: if constexpr (npatterns(D) > 2) k2_fill<D, 2>(kp, val, dsc); break;
      case 3: if constexpr (npatterns(D) > 3) k2_fill<D, 3>(kp, val, dsc); break;
      default:
        if constexpr (D == 4) {
          switch (k2_elem_pattern<D>(eq)) {
            case 4: k2_fill<D, 4>(kp, val, dsc); break;
            case 5: k2_fill<D, 5>(kp, val, dsc); break;
            case 6: k2_fill<D, 6>(kp, val, dsc); break;
            case 7: k2_fill<D, 7>(kp, val, dsc); break;
          }
        }
    }
    return;
  }
  if ((threadIdx.x & 31) == 0) dsc.bp = -1;
}

// a stored unit with the beta term (U elements v0, v1 at g), out of line:
// inlined, the compiler may predicate its FP64 operations into the common
// beta = 0 path, where they would still occupy the FP64 pipe
template <typename T, int U>
static __device__ __noinline__ void k2_store_beta(T* g, T v0, T v1, T bt) {
  T v[U], o[U];
  v[0] = v0;
  if constexpr (U == 2) v[1] = v1;
  vload<T, U>(g, o);
#pragma unroll
  for (int i = 0; i < U; i++) v[i] = add_beta(v[i], o[i], bt);
  vstore<T, U>(g, v);
}

// Copy the m_b tiles of a block orbit between HBM and shared memory in units
// of U elements along the stride-1 index (U = 2: 16 bytes for FP64, 8 for
// FP32; U = 1 where the tensor's strides or base addresses do not allow
// pairs). Each thread owns fixed units at the same in-tile place of every
// tile (global offset from the tile origin and shared-memory place computed
// once); per tile it adds the tile's origin and checks the tile's bounds only
// at the upper edge. LOAD: asynchronous copies into shared memory (the caller
// commits and waits); store: shared memory -> HBM with the beta term.
template <int D, int U, bool LOAD, typename T>
__device__ __forceinline__ void k2_copy(const KParams& kp, T* sm, const K2Desc& dsc) {
  using K = K2Shape<D>;
  constexpr int CPR = K::BL / U;   // units per tile row
  constexpr int CPT = K::NT / U;   // units per tile
  // either several tiles per pass of 256 threads, or several units of one tile per thread
  constexpr int TPP = CPT <= 256 ? 256 / CPT : 1;
  constexpr int NCH = CPT <= 256 ? 1 : CPT / 256;
  static_assert(CPT <= 256 ? 256 % CPT == 0 : CPT % 256 == 0, "tile units must tile the block");
  const int64_t* ld = LOAD ? kp.lda : kp.ldb;
  const int64_t* base = dsc.base[LOAD ? 0 : 1];
  const int mb = dsc.mb;
  const int u0 = CPT <= 256 ? threadIdx.x / CPT : 0;
  int w[NCH][4];
  int64_t goff[NCH];
  int slot[NCH];
#pragma unroll
  for (int q = 0; q < NCH; q++) {
    const int c = (CPT <= 256 ? threadIdx.x % CPT : threadIdx.x) + q * 256;
    w[q][0] = (c % CPR) * U;
    int r = c / CPR;
#pragma unroll
    for (int k = 1; k < 4; k++) {
      w[q][k] = 0;
      if (k < D) {
        w[q][k] = r % K::BL;
        r /= K::BL;
      }
    }
    goff[q] = 0;
#pragma unroll
    for (int k = 0; k < D; k++) goff[q] += (int64_t)w[q][k] * ld[k];
    slot[q] = K::phys(w[q]);  // the swizzle keeps the pair (w0 even, w0 + 1) together
  }
  T* G = LOAD ? const_cast<T*>(static_cast<const T*>(kp.A)) : static_cast<T*>(kp.B);
  const bool beta = !LOAD && (kp.flags & KF_BETA);
  const T bt = beta_of<T>(kp);
  auto unit = [&](int u, int q) {
    T* g = G + base[u] + goff[q];
    T* sp = sm + u * K::NT + slot[q];
    if constexpr (LOAD) {
      cp_async<U * sizeof(T)>(sp, g);
    } else {
      T v[U];
      if constexpr (U == 2) {
        vload<T, 2>(sp, v);
      } else {
        v[0] = sp[0];
      }
#if SS_K2_BETA_CALL
      if (beta)
        k2_store_beta<T, U>(g, v[0], v[U - 1], bt);
      else
        vstore<T, U>(g, v);
#else
      if (beta) {
        T o[U];
        vload<T, U>(g, o);
#pragma unroll
        for (int i = 0; i < U; i++) v[i] = add_beta(v[i], o[i], bt);
      }
      vstore<T, U>(g, v);
#endif
    }
  };
#if SS_K2_COPY_FULL
  // d <= 3, every tile full (all block orbits away from the upper edge): the
  // m_b <= d! tiles unrolled, no bounds checks
  if constexpr (D <= 3 && TPP == 1) {
    if (dsc.allfull) {
#pragma unroll
      for (int u = 0; u < fact(D); u++) {
        if (u < mb) {
#pragma unroll
          for (int q = 0; q < NCH; q++) unit(u, q);
        }
      }
      return;
    }
  }
#endif
  for (int u = u0; u < mb; u += TPP) {
    const bool full_u = dsc.full[u];
#pragma unroll
    for (int q = 0; q < NCH; q++) {
      bool in = full_u;
      if (!in) {
        in = true;
#pragma unroll
        for (int k = 0; k < D; k++) in = in && w[q][k] < dsc.lim[u][k];
      }
      if (!in) continue;
      unit(u, q);
    }
  }
}

// the element orbits of one block orbit of pattern BP, in shared memory: each
// thread takes canonical in-tile offsets w of the first tile member
template <int D, int BP, int AR, typename T>
__device__ __forceinline__ void k2_orbits(const KParams& kp, const K2Desc& dsc, T* sm, const unsigned short* sl) {
  using K = K2Shape<D>;
  int T0[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < D; k++) T0[k] = dsc.val[Pat<D, BP>::lab(0, k)];
  // the equal block coordinates are those with equal labels in the block
  // pattern (compile time): for distinct blocks every offset is canonical and
  // the element pattern is the generic one
  const bool edge = T0[D - 1] * K::BL + K::BL > kp.O;  // the largest coordinate's tile is cut by the edge
  if constexpr (BP != 0 && SS_K2_SORTED) {
    constexpr int n = kK2List<D, BP>.n;
#pragma unroll 1
    for (int i = threadIdx.x; i < n; i += 256) {
      const unsigned pk = kK2List<D, BP>.e[i];
      const int w[4] = {(int)(pk & 0xFFu), (int)((pk >> 8) & 0xFFu), (int)((pk >> 16) & 0xFFu),
                        (int)((pk >> 24) & 0x1Fu)};
      if (edge && T0[D - 1] * K::BL + w[D - 1] >= kp.O) continue;
      k2_dispatch<D, BP, AR, T>(kp, (int)(pk >> 29), w, sm);
    }
    return;
  }
#pragma unroll 1
  for (int e0 = threadIdx.x; e0 < K::NT; e0 += 256) {
    int w[4];
    K::elem(e0, w);
    bool ok = !edge || T0[D - 1] * K::BL + w[D - 1] < kp.O;
    unsigned eq = 0;
#pragma unroll
    for (int k = 0; k + 1 < D; k++) {
      if (Pat<D, BP>::lab(0, k) == Pat<D, BP>::lab(0, k + 1)) {
        ok = ok && w[k] <= w[k + 1];  // canonical: sorted within equal blocks
        if (w[k] == w[k + 1]) eq |= 1u << k;
      }
    }
    if (!ok) continue;
    if constexpr (BP == 0) {
      if constexpr (kK2Map<D, BP, 0>.valid) k2_group<D, BP, 0, AR, T>(kp, w, sm, sl);
    } else {
      k2_dispatch<D, BP, AR, T>(kp, k2_elem_pattern<D>(eq), w, sm);
    }
  }
}

template <int D, int AR, typename T>
__device__ __forceinline__ void k2_compute(const KParams& kp, const K2Desc& dsc, T* sm, const unsigned short* sl) {
  switch (dsc.bp) {
    case 0: k2_orbits<D, 0, AR, T>(kp, dsc, sm, sl); break;
    case 1: k2_orbits<D, 1, AR, T>(kp, dsc, sm, sl); break;
    case 2: if constexpr (npatterns(D) > 2) k2_orbits<D, 2, AR, T>(kp, dsc, sm, sl); break;
    case 3: if constexpr (npatterns(D) > 3) k2_orbits<D, 3, AR, T>(kp, dsc, sm, sl); break;
    default:
      if constexpr (D == 4) {
        switch (dsc.bp) {
          case 4: k2_orbits<D, 4, AR, T>(kp, dsc, sm, sl); break;
          case 5: k2_orbits<D, 5, AR, T>(kp, dsc, sm, sl); break;
          case 6: k2_orbits<D, 6, AR, T>(kp, dsc, sm, sl); break;
          case 7: k2_orbits<D, 7, AR, T>(kp, dsc, sm, sl); break;
        }
      }
  }
}

// A CTA works through the block orbits of its ids. With NBUF = 2 the tiles of
// the next block orbit are copied asynchronously into the second buffer
// while the current one is computed and stored back; with NBUF = 1 the
// phases follow one another. Block orbits own disjoint tiles, so in place the
// prefetch of the next orbit never reads an element the current one writes.
// The tile tables rotate through three slots: the one being filled for the
// next orbit is neither the current one nor the one the previous orbit's
// stores may still be reading.
template <int D, int AR, int U, int NBUF, int RUN, int MINB, typename T>
__global__ void __launch_bounds__(256, MINB) k2_kernel(const __grid_constant__ KParams kp) {
  using K = K2Shape<D>;
  extern __shared__ __align__(16) unsigned char k2_smem[];
  T* const buf0 = reinterpret_cast<T*>(k2_smem);
  T* const buf1 = buf0 + (NBUF > 1 ? fact(D) * K::NT : 0);
  // d = 4 transform instantiation: after the buffers, each thread's slots of
  // the members of its generic orbit (in-tile offset of element threadIdx.x)
  // in a generic block orbit, one column per thread; read back only by the
  // same thread, so no barrier
  constexpr bool SLT = k2_slot_table<D, AR>();
  unsigned short* const sl = SLT ? reinterpret_cast<unsigned short*>(buf0 + NBUF * fact(D) * K::NT) : nullptr;
  if constexpr (SLT) {
    int w[4];
    K::elem(threadIdx.x, w);
#pragma unroll
    for (int u = 0; u < 24; u++) sl[u * 256 + threadIdx.x] = (unsigned short)k2_slot<4, 0, 0>(u, w);
  }
  __shared__ K2Desc dsc[3];
  const bool w0 = threadIdx.x < 32;
  // ids of this CTA: a run of RUN consecutive ids, or (RUN = 0) every
  // gridDim.x-th id from blockIdx.x
  const int64_t total = kp.pre[npatterns(D)];
  const int64_t first = RUN > 0 ? (int64_t)blockIdx.x * RUN : (int64_t)blockIdx.x;
  const int64_t step = RUN > 0 ? 1 : (int64_t)gridDim.x;
  const int64_t end = RUN > 0 ? (first + RUN < total ? first + RUN : total) : total;
  if (w0) k2_next<D>(kp, first, step, end, dsc[0]);
  __syncthreads();
  if (dsc[0].bp < 0) return;
  if constexpr (NBUF > 1) {
    k2_copy<D, U, true, T>(kp, buf0, dsc[0]);
    cp_async_commit();
  }
  for (int k = 0;; k++) {
    const K2Desc& cur = dsc[k % 3];
    K2Desc& nxt = dsc[(k + 1) % 3];
    T* const cb = NBUF > 1 && (k & 1) ? buf1 : buf0;
    if constexpr (NBUF > 1) {
      if (w0) k2_next<D>(kp, cur.id + step, step, end, nxt);
      __syncthreads();  // nxt ready; the previous orbit's stores from the other buffer are done
      if (nxt.bp >= 0) k2_copy<D, U, true, T>(kp, (k & 1) ? buf0 : buf1, nxt);
      cp_async_commit();
      cp_async_wait<1>();  // this thread's copies of the current orbit have landed
    } else {
      k2_copy<D, U, true, T>(kp, cb, cur);
      cp_async_commit();
      cp_async_wait<0>();
    }
    __syncthreads();
    k2_compute<D, AR, T>(kp, cur, cb, sl);
    __syncthreads();
    k2_copy<D, U, false, T>(kp, cb, cur);
    if constexpr (NBUF == 1) {
      if (w0) k2_next<D>(kp, cur.id + step, step, end, nxt);
      __syncthreads();  // nxt ready; the buffer is free again
    }
    if (nxt.bp < 0) break;
  }
}

// Launch shape per d: SS_K2_NBUF<d> buffers of d! dense tiles per CTA,
// SS_K2_RUN<d> consecutive ids per CTA (0: a persistent grid of the resident
// CTAs) and SS_K2_MINB<d> resident CTAs per SM for the register budget.
template <int D, int AR, int U, typename T>
cudaError_t launch_k2_vec(const KParams& kp, cudaStream_t st) {
  constexpr bool XW = AR == AR_EXACT_XW;
  constexpr int NBUF = D == 2 ? SS_K2_NBUF2 : (D == 3 ? SS_K2_NBUF3 : (XW ? SS_K2_NBUF4W : SS_K2_NBUF4));
  constexpr int MINB = D == 2 ? SS_K2_MINB2 : (D == 3 ? SS_K2_MINB3 : (XW ? SS_K2_MINB4W : SS_K2_MINB4));
  constexpr int RUN = D == 2 ? SS_K2_RUN2 : (D == 3 ? SS_K2_RUN3 : (XW ? SS_K2_RUN4W : SS_K2_RUN4));
  constexpr size_t smem = (size_t)NBUF * fact(D) * K2Shape<D>::NT * sizeof(T) +
                          (k2_slot_table<D, AR>() ? 24 * 256 * sizeof(unsigned short) : 0);
  auto fn = k2_kernel<D, AR, U, NBUF, RUN, MINB, T>;
  // resident CTAs per device (persistent grid), set up once per device
  static DeviceCache cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  long long ctas = 0;
  const int rc = cache.get(dev, &ctas, [&](long long* val) {
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    // all of the unified L1/shared array as shared memory: occupancy is set by the tiles
    err = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return (int)err;
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
    if (err != cudaSuccess) return (int)err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    *val = (long long)per_sm * sms;
    return 0;
  });
  if (rc != 0) return rc < 0 ? cudaErrorInvalidDevice : (cudaError_t)rc;
  const int64_t ids = kp.pre[npatterns(D)];
  if (ids == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(RUN > 0 ? (ids + RUN - 1) / RUN : (ids > ctas ? ctas : ids));
  fn<<<grid, 256, smem, st>>>(kp);
  return cudaGetLastError();
}

// element pairs along the stride-1 index when the tensor allows them
template <int D, int AR, typename T>
cudaError_t launch_k2_impl(const KParams& kp, cudaStream_t st) {
  constexpr uintptr_t PB = 2 * sizeof(T);
  bool pair = (kp.O % 2 == 0) && ((uintptr_t)kp.A % PB == 0) && ((uintptr_t)kp.B % PB == 0);
  for (int k = 1; k < D; k++) pair = pair && (kp.lda[k] % 2 == 0) && (kp.ldb[k] % 2 == 0);
  if (pair) return launch_k2_vec<D, AR, 2, T>(kp, st);
  return launch_k2_vec<D, AR, 1, T>(kp, st);
}

}  // namespace ss
