#pragma once
// CUDA kernel templates of the spin-summation library (sm_103a). Each
// ss_k_*.cu translation unit instantiates a few of them, so the kernels
// compile in parallel.
//
// K1 "orbit stream": the fast layout, where each permuted tuple owns a
// contiguous run of S spectator elements. A CTA takes one orbit (the m <= d!
// tuples t0 o tau of a canonical tuple t0, Sec. 4.2) and a range of spectator
// positions; each thread loads the m member values at its position(s) with
// coalesced vector loads, applies the m x m orbit operator in registers, and
// stores the m results. Every element of A is read once and every element of
// B written once (the temporal locality of Algorithm 2, at element level, with
// the spatial locality of Sec. 4.6 coming from the spectator run instead of a
// cache block). In place is safe: a thread reads all of its orbit positions
// before it writes any, and no other thread touches them (Sec. 4.6.5).
//
// KG "general": one thread per (orbit, spectator position) with arbitrary
// strides; used when the spectator block is not dense or too short.
//
// Arithmetic cores, per orbit element group x[0..m-1] -> y[0..m-1]:
//   AR_EXACT  FP64 via exact fixed-point integer limbs (see exact_core)
//   AR_STRICT FP64 natively, sigma in lexicographic order, multiply then add
//   AR_F32    FP32 storage and accumulation
#include <cuda_runtime.h>
#include <stdint.h>

#include "ss_internal.h"

namespace ss {

// pattern tables evaluated once per (D, P); loads from them fold to constants
// in the unrolled loops
template <int D, int P>
__device__ constexpr Pattern<D> kPattern = make_pattern<D>(P);

template <int D, int P>
struct Pat {
  static constexpr int M = make_pattern<D>(P).m;
  static constexpr int ND = make_pattern<D>(P).nd;
  __device__ __forceinline__ static int lab(int u, int k) { return kPattern<D, P>.lab[u][k]; }
  __device__ __forceinline__ static int idx(int u, int s) { return kPattern<D, P>.idx[u][s]; }
};

// Klein four-group tables of the 4D patterns (see Wht4)
template <int P>
__device__ constexpr Wht4 kWht = make_wht4(P);
template <int P>
constexpr bool wht_ok() { return make_wht4(P).ok; }

// C(n, k) for k <= 4 with constant divisors (no 64-bit division routine);
// k is a compile-time constant at every call site after unrolling
__device__ __forceinline__ int64_t binom(int64_t n, int k) {
  if (n < k) return 0;
  switch (k) {
    case 1: return n;
    case 2: return n * (n - 1) / 2;
    case 3: return n * (n - 1) * (n - 2) / 6;
    case 4: return n * (n - 1) * (n - 2) * (n - 3) / 24;
    default: return 1;
  }
}

// strictly increasing ND-tuple of values in [0, O) with colex rank r
// (combinatorial number system: r = sum_i C(v_i, i + 1))
template <int ND>
__device__ __forceinline__ void unrank(int64_t r, int O, int* v) {
#pragma unroll
  for (int i = ND - 1; i >= 0; i--) {
    int c = i;
    while (c + 1 < O && binom(c + 1, i + 1) <= r) c++;
    v[i] = c;
    r -= binom(c, i + 1);
  }
}

__device__ __forceinline__ unsigned long long shr64(unsigned long long x, unsigned k) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(k));  // amounts >= 64 give 0
  return r;
}

// ---------------------------------------------------------------------------
// strict FP64 core: the reference order, stage by stage
// ---------------------------------------------------------------------------
template <int D, int P>
__device__ __forceinline__ void strict_stage(const double* cd, double (&t)[Pat<D, P>::M]) {
  constexpr int M = Pat<D, P>::M;
  constexpr int NS = fact(D);
  double acc[M];
#pragma unroll
  for (int u = 0; u < M; u++) acc[u] = 0.0;
#pragma unroll
  for (int s = 0; s < NS; s++) {
    const double c = cd[s];
    if (c != 0.0) {
#pragma unroll
      for (int u = 0; u < M; u++) acc[u] = __dadd_rn(acc[u], __dmul_rn(c, t[Pat<D, P>::idx(u, s)]));
    }
  }
#pragma unroll
  for (int u = 0; u < M; u++) t[u] = acc[u];
}

template <int D, int P>
__device__ __forceinline__ void strict_core(const KParams& kp, double (&t)[Pat<D, P>::M]) {
  // the first three stages unrolled (coefficients become constant operands)
#pragma unroll
  for (int st = 0; st < 3; st++)
    if (st < kp.nstage) strict_stage<D, P>(kp.cd[st], t);
  for (int st = 3; st < kp.nstage; st++) strict_stage<D, P>(kp.cd[st], t);
}

// ---------------------------------------------------------------------------
// exact FP64 core.
// Let E be the largest biased exponent among the m inputs of the group. Every
// input is truncated to the grid 2^(E-1022-2W) (two signed W-bit limbs, i.e.
// 2W = 48..52 bits below the top of the largest input); the integer sums
// sum_v M[u][v] X_v are exact in int32 per limb because sum|M[u][.]| * 2^W <
// 2^31; the two limbs are joined into a 64-bit integer, rounded by kdrop bits
// to below 2^51, and converted to FP64 exactly with one subtraction of a
// magic constant C = 1.5 * 2^52 * ulp. Integer-valued inputs are therefore
// reproduced exactly, and the error of any output is at most sum|a| * 2^(-2W)
// times the largest input of its orbit plus 2^(kdrop-1) grid units.
// Returns false (and leaves y untouched) when E is outside [emin, emax]:
// zero or tiny groups, huge values, infinities and NaNs take the strict core.
// ---------------------------------------------------------------------------
// shared prologue: largest exponent field E of the group and the signed limbs
template <int M>
__device__ __forceinline__ bool exact_limbs(const KParams& kp, const double (&x)[M], int (&l0)[M], int (&l1)[M],
                                            unsigned& E) {
  unsigned hi[M], lo[M];
  E = 0;
#pragma unroll
  for (int v = 0; v < M; v++) {
    hi[v] = (unsigned)__double2hiint(x[v]);
    lo[v] = (unsigned)__double2loint(x[v]);
    E = max(E, hi[v] & 0x7FF00000u);
  }
  if (E < kp.emin || E > kp.emax) {
    // a group of exact zeros (signed or not) is exact on any grid: give it the
    // smallest valid exponent and let the fixed-point path produce +0
    unsigned any = 0;
    if (E == 0) {
#pragma unroll
      for (int v = 0; v < M; v++) any |= (hi[v] & 0x7FFFFFFFu) | lo[v];
    }
    if (E != 0 || any != 0) return false;
    E = kp.emin;
  }
  const int W = kp.W;
  const unsigned mask = (1u << W) - 1u;
#pragma unroll
  for (int v = 0; v < M; v++) {
    unsigned k = ((E - (hi[v] & 0x7FF00000u)) >> 20) + (unsigned)kp.s0;
    unsigned long long mant = ((unsigned long long)((hi[v] & 0x000FFFFFu) | 0x00100000u) << 32) | lo[v];
    unsigned long long q = shr64(mant, k);
    int a = (int)((unsigned)q & mask);
    int b = (int)(q >> W);
    int sg = (int)hi[v] >> 31;
    l0[v] = (a ^ sg) - sg;
    l1[v] = (b ^ sg) - sg;
  }
  return true;
}

// limbs (y1 * 2^W + y0) -> FP64: round off kdrop bits on the low limb
// ((y1 2^W + y0 + r) >> k = y1 2^(W-k) + ((y0 + r) >> k) for k <= W), then one
// subtraction of the magic constant C = chi:0
//
// INTCONV: build the same FP64 value with integer instructions instead (for
// kernels whose FP64 pipe is busy with other work): the value is
// Y * 2^(ef - 1075), ef = chi >> 20, |Y| < 2^50, so it is normalised by the
// position of Y's leading one and packed; exact whenever the result is a
// normal number (otherwise, which the exponent range allows only for tiny
// alpha, the subtraction above is used).
__device__ __forceinline__ double fixed_to_double_fp64(long long Y, unsigned chi, double C) {
  const double Dv = __hiloint2double((int)(chi + (unsigned)(Y >> 32)), (int)(unsigned)Y);
  return __dsub_rn(Dv, C);
}
// out of line, so that the compiler cannot predicate the subtraction into the
// common path (a predicated-off FP64 instruction still occupies the FP64 pipe)
static __device__ __noinline__ double fixed_to_double_fp64_call(long long Y, unsigned chi, double C) {
  return fixed_to_double_fp64(Y, chi, C);
}

template <bool INTCONV = false>
__device__ __forceinline__ double fixed_to_double(long long Y, unsigned chi, double C) {
  if constexpr (INTCONV) {
    const unsigned long long a = Y < 0 ? 0ull - (unsigned long long)Y : (unsigned long long)Y;
    const int p = 63 - __clzll((long long)a);
    const int e = p + (int)(chi >> 20) - 52;
    if (Y != 0 && e <= 0) return fixed_to_double_fp64_call(Y, chi, C);
    const unsigned long long m = (a << ((52 - p) & 63)) & 0x000FFFFFFFFFFFFFull;
    const unsigned long long bits =
        ((unsigned long long)Y & 0x8000000000000000ull) | ((unsigned long long)e << 52) | m;
    return __longlong_as_double(Y == 0 ? 0ll : (long long)bits);
  } else {
    return fixed_to_double_fp64(Y, chi, C);
  }
}

template <bool INTCONV = false>
__device__ __forceinline__ double exact_out(const KParams& kp, unsigned chi, double C, int y0, int y1) {
  const long long Y = ((long long)y1 << kp.wk) + (long long)((y0 + (int)kp.rnd) >> kp.kdrop);
  return fixed_to_double<INTCONV>(Y, chi, C);
}

template <int D, int P, int NST = 0, bool INTCONV = false>
__device__ __forceinline__ bool exact_core(const KParams& kp, const double (&x)[Pat<D, P>::M],
                                           double (&y)[Pat<D, P>::M]) {
  constexpr int M = Pat<D, P>::M;
  constexpr int NS = fact(D);
  int l0[M], l1[M];
  unsigned E;
  if (!exact_limbs<M>(kp, x, l0, l1, E)) return false;
  int y0[M], y1[M];
  if constexpr (P == 0) {
    // NST > 0: the stage count is a compile-time constant (only those stages are
    // compiled); NST == 0: up to MAXSTAGE_EXACT stages, count read at run time
#pragma unroll
    for (int st = 0; st < (NST > 0 ? NST : MAXSTAGE_EXACT); st++) {
      if (NST == 0 && st >= kp.nci) break;
#pragma unroll
      for (int u = 0; u < M; u++) { y0[u] = 0; y1[u] = 0; }
#pragma unroll
      for (int s = 0; s < NS; s++) {
        const int c = kp.ci[st][s];
        if (c != 0) {
#pragma unroll
          for (int u = 0; u < M; u++) {
            y0[u] += c * l0[Pat<D, P>::idx(u, s)];
            y1[u] += c * l1[Pat<D, P>::idx(u, s)];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < M; u++) { l0[u] = y0[u]; l1[u] = y1[u]; }
    }
  } else {
    const int* mp = kp.mp + mp_offset<D>(P);
#pragma unroll
    for (int u = 0; u < M; u++) {
      int a = 0, b = 0;
#pragma unroll
      for (int v = 0; v < M; v++) {
        a += mp[u * M + v] * l0[v];
        b += mp[u * M + v] * l1[v];
      }
      y0[u] = a;
      y1[u] = b;
    }
#pragma unroll
    for (int u = 0; u < M; u++) { l0[u] = y0[u]; l1[u] = y1[u]; }
  }
  const unsigned chi = E + (unsigned)kp.cexp;
  const double C = __hiloint2double((int)chi, 0);
#pragma unroll
  for (int u = 0; u < M; u++) y[u] = exact_out<INTCONV>(kp, chi, C, l0[u], l1[u]);
  return true;
}

// The generic 24-member orbit of d = 4 with the expanded operator (ci[0]),
// computed in G groups of 24 / G outputs: only the 48 input limbs and one
// group's accumulators are live, and each group's outputs go to `sink(u, y)`
// as soon as they are converted (register pressure, hence occupancy).
template <int G, class Sink>
__device__ __forceinline__ bool exact_core_grouped4(const KParams& kp, const double (&x)[24], Sink&& sink) {
  constexpr int M = 24, NU = M / G;
  int l0[M], l1[M];
  unsigned E;
  if (!exact_limbs<M>(kp, x, l0, l1, E)) return false;
  const unsigned chi = E + (unsigned)kp.cexp;
  const double C = __hiloint2double((int)chi, 0);
#pragma unroll
  for (int g = 0; g < G; g++) {
    int y0[NU], y1[NU];
#pragma unroll
    for (int j = 0; j < NU; j++) { y0[j] = 0; y1[j] = 0; }
#pragma unroll
    for (int s = 0; s < 24; s++) {
      const int c = kp.ci[0][s];
      if (c != 0) {
#pragma unroll
        for (int j = 0; j < NU; j++) {
          y0[j] += c * l0[Pat<4, 0>::idx(g * NU + j, s)];
          y1[j] += c * l1[Pat<4, 0>::idx(g * NU + j, s)];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NU; j++) sink(g * NU + j, exact_out(kp, chi, C, y0[j], y1[j]));
  }
  return true;
}

// The exact fixed-point core of a freely transformable d = 4 orbit through
// the Klein four-group transform (Wht4). Each input becomes one signed
// integer X on the 48-bit grid (kp.s0 = 5) of the largest input, exactly as
// the two limbs of exact_limbs join; every V-orbit's four X go through the
// 4-point Walsh-Hadamard transform (64-bit, below 2^50), whose results are
// split into a non-negative 25-bit low limb and a high limb; the sparse
// transformed operator (kp.wh) runs on int32 IMAD per limb (the planner
// keeps sum|a| <= 63, so both limb sums stay below 2^31); the two limb sums
// are joined in 64 bits and the inverse transform (the same butterflies)
// gives 4 Y, Y the integer sum sum_v M[u][v] X_v of the dense core. Rounding
// off kdrop + 2 bits of 4 Y is rounding off kdrop bits of Y, so outputs are
// bit-identical to exact_core on the same grid. Outputs go to sink(u, y).
template <int P, class Sink>
__device__ __forceinline__ bool exact_core_wht4(const KParams& kp, const double (&x)[Pat<4, P>::M], Sink&& sink) {
  constexpr int M = Pat<4, P>::M, NB = M / 4;
  constexpr int WOFF = wh_offset(P);
  unsigned E = 0;
#pragma unroll
  for (int v = 0; v < M; v++) E = max(E, (unsigned)__double2hiint(x[v]) & 0x7FF00000u);
  if (E < kp.emin || E > kp.emax) {
    unsigned any = 0;
    if (E == 0) {
#pragma unroll
      for (int v = 0; v < M; v++) any |= ((unsigned)__double2hiint(x[v]) & 0x7FFFFFFFu) | (unsigned)__double2loint(x[v]);
    }
    if (E != 0 || any != 0) return false;
    E = kp.emin;
  }
  int l0[M], l1[M];  // transformed values (row 4 o + k), low 25 bits and the rest
#pragma unroll
  for (int o = 0; o < NB; o++) {
    long long X[4];
#pragma unroll
    for (int vi = 0; vi < 4; vi++) {
      const double xv = x[kWht<P>.orb[o][vi]];
      const unsigned hi = (unsigned)__double2hiint(xv), lo = (unsigned)__double2loint(xv);
      const unsigned k = ((E - (hi & 0x7FF00000u)) >> 20) + (unsigned)kp.s0;
      const unsigned long long mant = ((unsigned long long)((hi & 0x000FFFFFu) | 0x00100000u) << 32) | lo;
      const long long q = (long long)shr64(mant, k);
      const long long sg = (long long)((int)hi >> 31);
      X[vi] = (q ^ sg) - sg;
    }
    const long long a0 = X[0] + X[1], a1 = X[0] - X[1], a2 = X[2] + X[3], a3 = X[2] - X[3];
    const long long xh[4] = {a0 + a2, a1 + a3, a0 - a2, a1 - a3};  // characters 0..3
#pragma unroll
    for (int k = 0; k < 4; k++) {
      l0[4 * o + k] = (int)((unsigned)xh[k] & 0x1FFFFFFu);
      l1[4 * o + k] = (int)(xh[k] >> 25);
    }
  }
  const unsigned chi = E + (unsigned)kp.cexp;
  const double C = __hiloint2double((int)chi, 0);
  const int sh = kp.kdrop + 2;
  const long long r4 = kp.rnd << 2;
#pragma unroll
  for (int o = 0; o < NB; o++) {
    long long yh[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int i = 4 * o + k;
      int a = 0, b = 0;
#pragma unroll
      for (int q = 0; q < 6; q++) {
        if (q < kWht<P>.nnz[i]) {
          const int w = kp.wh[WOFF + kWht<P>.woff[i] + q];
          a += w * l0[kWht<P>.col[i][q]];
          b += w * l1[kWht<P>.col[i][q]];
        }
      }
      yh[k] = ((long long)b << 25) + (long long)a;
    }
    const long long b0 = yh[0] + yh[1], b1 = yh[0] - yh[1], b2 = yh[2] + yh[3], b3 = yh[2] - yh[3];
    const long long y4[4] = {b0 + b2, b1 + b3, b0 - b2, b1 - b3};  // 4 Y at v_0..v_3
#pragma unroll
    for (int vi = 0; vi < 4; vi++) {
      const long long Y = (y4[vi] + r4) >> sh;
      sink(kWht<P>.orb[o][vi], fixed_to_double_fp64(Y, chi, C));
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// one orbit element group: x (inputs, m members) -> y (outputs), incl. alpha/beta
// ---------------------------------------------------------------------------
template <int D, int P, int AR, typename T, int NST = 0, bool INTCONV = false>
__device__ __forceinline__ void apply_group(const KParams& kp, T (&x)[Pat<D, P>::M], T (&y)[Pat<D, P>::M]) {
  constexpr int M = Pat<D, P>::M;
  constexpr int NS = fact(D);
  if constexpr (AR == AR_F32) {
    float t[M];
#pragma unroll
    for (int u = 0; u < M; u++) t[u] = x[u];
    auto stage = [&](const float* cf) {
      float acc[M];
#pragma unroll
      for (int u = 0; u < M; u++) acc[u] = 0.f;
#pragma unroll
      for (int s = 0; s < NS; s++) {
        const float c = cf[s];
        if (c != 0.f) {
#pragma unroll
          for (int u = 0; u < M; u++) acc[u] = fmaf(c, t[Pat<D, P>::idx(u, s)], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < M; u++) t[u] = acc[u];
    };
#pragma unroll
    for (int st = 0; st < 3; st++)
      if (st < kp.nstage) stage(kp.cf[st]);
    for (int st = 3; st < kp.nstage; st++) stage(kp.cf[st]);
    const float al = kp.alphaf;
#pragma unroll
    for (int u = 0; u < M; u++) y[u] = al * t[u];
  } else {
    bool done = false;
    if constexpr (AR == AR_EXACT) {
      done = exact_core<D, P, NST, INTCONV>(kp, x, y);
      if (done && (kp.flags & KF_ALPHA_MUL)) {
#pragma unroll
        for (int u = 0; u < M; u++) y[u] = __dmul_rn(kp.alpha, y[u]);
      }
    }
    if (!done) {
      strict_core<D, P>(kp, x);
#pragma unroll
      for (int u = 0; u < M; u++) y[u] = __dmul_rn(kp.alpha, x[u]);
    }
  }
}

template <typename T>
__device__ __forceinline__ T beta_of(const KParams& kp) {
  if constexpr (sizeof(T) == 8) return kp.beta;
  else return kp.betaf;
}

// B = alpha S(A) + beta B_old: the beta term, in the reference order for FP64
__device__ __forceinline__ double add_beta(double y, double b, double beta) { return __dadd_rn(y, __dmul_rn(beta, b)); }
__device__ __forceinline__ float add_beta(float y, float b, float beta) { return fmaf(beta, b, y); }

template <typename T, int VEC>
struct VecT;
template <>
struct VecT<double, 1> { using t = double; };
template <>
struct VecT<double, 2> { using t = double2; };
template <>
struct VecT<float, 1> { using t = float; };
template <>
struct VecT<float, 2> { using t = float2; };
template <>
struct VecT<float, 4> { using t = float4; };

template <typename T, int VEC>
__device__ __forceinline__ void vload(const T* p, T (&v)[VEC]) {
  using V = typename VecT<T, VEC>::t;
  V w = *reinterpret_cast<const V*>(p);
  const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
  for (int i = 0; i < VEC; i++) v[i] = e[i];
}
template <typename T, int VEC>
__device__ __forceinline__ void vstore(T* p, const T (&v)[VEC]) {
  using V = typename VecT<T, VEC>::t;
  V w;
  T* e = reinterpret_cast<T*>(&w);
#pragma unroll
  for (int i = 0; i < VEC; i++) e[i] = v[i];
  *reinterpret_cast<V*>(p) = w;
}

// The strict core for one generic d = 4 group whose exponents leave the
// fixed-point range (zeros, tiny or huge values, Inf, NaN): reloads its 24
// inputs (nothing of the group has been stored yet, so this is safe in place)
// and stores alpha S(x) + beta B. Kept out of line: it is rare, and inlining
// it would hold registers in the hot path.
static __device__ __noinline__ void strict_fallback_generic4(const KParams& kp, const int64_t* offA, const int64_t* offB,
                                                      int64_t s) {
  const double* A = static_cast<const double*>(kp.A);
  double* B = static_cast<double*>(kp.B);
  double x[24];
  for (int u = 0; u < 24; u++) x[u] = A[offA[u] + s];
  strict_core<4, 0>(kp, x);
  const bool beta = kp.flags & KF_BETA;
  for (int u = 0; u < 24; u++) {
    double* dst = B + offB[u] + s;
    double v = __dmul_rn(kp.alpha, x[u]);
    if (beta) v = add_beta(v, *dst, kp.beta);
    *dst = v;
  }
}

// The same for a d = 4 orbit of pattern P on the transformed path.
template <int P>
static __device__ __noinline__ void strict_fallback4(const KParams& kp, const int64_t* offA, const int64_t* offB,
                                                     int64_t s) {
  constexpr int M = Pat<4, P>::M;
  const double* A = static_cast<const double*>(kp.A);
  double* B = static_cast<double*>(kp.B);
  double x[M];
  for (int u = 0; u < M; u++) x[u] = A[offA[u] + s];
  strict_core<4, P>(kp, x);
  const bool beta = kp.flags & KF_BETA;
  for (int u = 0; u < M; u++) {
    double* dst = B + offB[u] + s;
    double v = __dmul_rn(kp.alpha, x[u]);
    if (beta) v = add_beta(v, *dst, kp.beta);
    *dst = v;
  }
}

// The generic d = 4 group when alpha is not a power of two (the fixed-point
// path cannot fold it into the conversion): reloads its inputs and stores
// alpha S(x) + beta B. Out of line and taken by a uniform branch before the
// loads, so the common path carries no FP64 multiply.
static __device__ __noinline__ void scaled_generic4(const KParams& kp, const int64_t* offA, const int64_t* offB,
                                                    int64_t s) {
  const double* A = static_cast<const double*>(kp.A);
  double* B = static_cast<double*>(kp.B);
  double x[24];
  for (int u = 0; u < 24; u++) x[u] = A[offA[u] + s];
  const bool beta = kp.flags & KF_BETA;
  auto sink = [&](int u, double v) {
    double* dst = B + offB[u] + s;
    v = __dmul_rn(kp.alpha, v);
    if (beta) v = add_beta(v, *dst, kp.beta);
    *dst = v;
  };
  if (!exact_core_grouped4<SS_4D_GROUPS>(kp, x, sink)) strict_fallback_generic4(kp, offA, offB, s);
}

// chunks a K1 thread takes at a time for an orbit of m members: the generic
// orbit's d! over m, at most kbmax
constexpr int k1_batch(int D, int m, int kbmax) {
  return m >= fact(D) ? 1 : (fact(D) / m < kbmax ? fact(D) / m : kbmax);
}

// ---------------------------------------------------------------------------
// K1 body for pattern P. Warp 0 unranks the orbit and writes the m member
// offsets of A and B to shared memory; the CTA then streams cpb chunks of
// VEC * blockDim spectator positions through registers.
// ---------------------------------------------------------------------------
//
// XW selects the Klein four-group path of d = 4 exact orbits: 0 never, 1 for
// every transformable pattern (the planner set KF_WHT), 2 when the problem's
// KF_WHT flag says so (batched kernels, whose problems differ).
// KBM: the most chunks a thread takes at a time (k1_batch).
template <int D, int P, int AR, int VEC, typename T, int NST = 0, int XW = 0, int KBM = 1>
__device__ __forceinline__ void k1_body(const KParams& kp, int64_t orb, int64_t c0, int64_t c1) {
  constexpr int M = Pat<D, P>::M;
  __shared__ int64_t soff[2][24];
  __syncthreads();
  if (threadIdx.x < 32) {
    int val[4] = {0, 0, 0, 0};
    unrank<Pat<D, P>::ND>(orb, kp.O, val);
#pragma unroll
    for (int u = 0; u < M; u++) {
      if (threadIdx.x == (u & 31)) {
        int64_t a = 0, b = 0;
#pragma unroll
        for (int k = 0; k < D; k++) {
          const int t = val[Pat<D, P>::lab(u, k)];
          a += (int64_t)t * kp.lda[k];
          b += (int64_t)t * kp.ldb[k];
        }
        soff[0][u] = a;
        soff[1][u] = b;
      }
    }
  }
  __syncthreads();
  const T* A = static_cast<const T*>(kp.A);
  T* B = static_cast<T*>(kp.B);
  const int64_t step = (int64_t)blockDim.x * VEC;
  if constexpr (D == 4 && AR == AR_EXACT && VEC == 1 && XW != 0) {
    if (XW == 1 || (kp.flags & KF_WHT)) {
      const bool beta = kp.flags & KF_BETA;
      constexpr int KB = k1_batch(D, M, KBM);
      for (int64_t c = c0; c < c1; c += KB) {
        if constexpr (SS_4DW_PREFETCH) {
          // thread u < M asks L2 for member u's runs SS_4DW_PREFETCH batches ahead
          const int64_t sn = (c + (int64_t)SS_4DW_PREFETCH * KB) * step;
          if (c + SS_4DW_PREFETCH * KB < c1 && threadIdx.x < M && sn < kp.S) {
            const int64_t n = min((int64_t)step * KB, kp.S - sn);
            const uintptr_t a = reinterpret_cast<uintptr_t>(A + soff[0][threadIdx.x] + sn);
            const unsigned bytes = (unsigned)(n * (int64_t)sizeof(T)) & ~15u;
            if ((a & 15) == 0 && bytes > 0) {
              if constexpr (SS_4DW_PFHINT) {
                unsigned long long pol;
                asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
                asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(a), "r"(bytes),
                             "l"(pol)
                             : "memory");
              } else {
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
              }
            }
          }
        }
        int64_t sk[KB];
        bool ok[KB];
#pragma unroll
        for (int k = 0; k < KB; k++) {
          sk[k] = (c + k) * step + (int64_t)threadIdx.x;
          ok[k] = c + k < c1 && sk[k] < kp.S;
        }
        if (!ok[0]) break;
        double x[KB][M];
#pragma unroll
        for (int k = 0; k < KB; k++)
          if (ok[k]) {
#pragma unroll
            for (int u = 0; u < M; u++) x[k][u] = A[soff[0][u] + sk[k]];
          }
#pragma unroll
        for (int k = 0; k < KB; k++) {
          if (!ok[k]) continue;
          const int64_t s = sk[k];
          auto sink = [&](int u, double v) {
            T* dst = B + soff[1][u] + s;
            if (beta) v = add_beta(v, *dst, kp.beta);
            *dst = v;
          };
          if constexpr (wht_ok<P>()) {
            if (!exact_core_wht4<P>(kp, x[k], sink)) strict_fallback4<P>(kp, soff[0], soff[1], s);
          } else {
            // the two patterns V does not act on freely: the dense core on the
            // same grid, with the strict core out of line (inlined, the compiler
            // may predicate its FP64 operations into the common path)
            double y[M];
            if (exact_core<4, P>(kp, x[k], y)) {
#pragma unroll
              for (int u = 0; u < M; u++) sink(u, y[u]);
            } else {
              strict_fallback4<P>(kp, soff[0], soff[1], s);
            }
          }
        }
      }
      return;
    }
  }
  // orbits with fewer members than the generic one take KB chunks at a time,
  // so that every thread has about the same number of loads in flight
  constexpr bool G4 = D == 4 && P == 0 && AR == AR_EXACT && VEC == 1;
  constexpr int KB = G4 ? 1 : k1_batch(D, M, KBM);
  for (int64_t c0k = c0; c0k < c1; c0k += KB) {
    int64_t sk[KB];
    bool ok[KB];
#pragma unroll
    for (int k = 0; k < KB; k++) {
      sk[k] = (c0k + k) * step + (int64_t)threadIdx.x * VEC;
      ok[k] = c0k + k < c1 && sk[k] < kp.S;
    }
    if (!ok[0]) break;
    const int64_t s = sk[0];
    if constexpr (SS_4D_SCALED_OUTOFLINE && G4) {
      if (kp.flags & KF_ALPHA_MUL) {
        scaled_generic4(kp, soff[0], soff[1], s);
        continue;
      }
    }
    T xk[KB][VEC][M];
#pragma unroll
    for (int k = 0; k < KB; k++)
      if (ok[k]) {
#pragma unroll
        for (int u = 0; u < M; u++) {
          T v[VEC];
          vload<T, VEC>(A + soff[0][u] + sk[k], v);
#pragma unroll
          for (int e = 0; e < VEC; e++) xk[k][e][u] = v[e];
        }
      }
    if constexpr (G4) {
      auto& x = xk[0];
      const bool beta = kp.flags & KF_BETA;
      bool done;
      if (!SS_4D_SCALED_OUTOFLINE && (kp.flags & KF_ALPHA_MUL)) {
        auto sink = [&](int u, double v) {
          T* dst = B + soff[1][u] + s;
          v = __dmul_rn(kp.alpha, v);
          if (beta) v = add_beta(v, *dst, kp.beta);
          *dst = v;
        };
        done = exact_core_grouped4<SS_4D_GROUPS>(kp, x[0], sink);
      } else {
        auto sink = [&](int u, double v) {
          T* dst = B + soff[1][u] + s;
          if (beta) v = add_beta(v, *dst, kp.beta);
          *dst = v;
        };
        done = exact_core_grouped4<SS_4D_GROUPS>(kp, x[0], sink);
      }
      if (!done) strict_fallback_generic4(kp, soff[0], soff[1], s);
      continue;
    }
    const bool beta = kp.flags & KF_BETA;
    const T bt = beta_of<T>(kp);
#pragma unroll
    for (int k = 0; k < KB; k++) {
      if (!ok[k]) continue;
      T y[VEC][M];
#pragma unroll
      for (int e = 0; e < VEC; e++) apply_group<D, P, AR, T, NST>(kp, xk[k][e], y[e]);
#pragma unroll
      for (int u = 0; u < M; u++) {
        T v[VEC];
        T* dst = B + soff[1][u] + sk[k];
        if (beta) {
          vload<T, VEC>(dst, v);
#pragma unroll
          for (int e = 0; e < VEC; e++) v[e] = add_beta(y[e][u], v[e], bt);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; e++) v[e] = y[e][u];
        }
        vstore<T, VEC>(dst, v);
      }
    }
  }
}

template <int D>
__device__ __forceinline__ int find_pattern(const int64_t* pre, int64_t b) {
  int p = 0;
#pragma unroll
  for (int q = 1; q < npatterns(D); q++)
    if (b >= pre[q]) p = q;
  return p;
}

// one K1 block of work: block index b of the problem's grid -> (pattern,
// orbit, chunk range)
template <int D, int AR, int VEC, typename T, int XW = 0, int KBM = 1>
__device__ __forceinline__ void k1_block(const KParams& kp, int64_t b) {
  const int p = find_pattern<D>(kp.pre, b);
  const int64_t bpo = (kp.nchunk + kp.cpb - 1) / kp.cpb;  // blocks per orbit
  const int64_t local = b - kp.pre[p];
  const int64_t orb = local / bpo;
  const int64_t cb = local - orb * bpo;
  const int64_t c0 = cb * kp.cpb;
  const int64_t c1 = min(kp.nchunk, c0 + kp.cpb);
  switch (p) {
    case 0: k1_body<D, 0, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
    case 1: k1_body<D, 1, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
    case 2: if constexpr (npatterns(D) > 2) k1_body<D, 2, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
    case 3: if constexpr (npatterns(D) > 3) k1_body<D, 3, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
    default:
      if constexpr (D == 4) {
        switch (p) {
          case 4: k1_body<D, 4, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
          case 5: k1_body<D, 5, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
          case 6: k1_body<D, 6, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
          case 7: k1_body<D, 7, AR, VEC, T, 0, XW, KBM>(kp, orb, c0, c1); break;
        }
      }
  }
}

template <int D, int AR, int VEC, typename T, int XW = 0>
__global__ void __launch_bounds__(256, (D == 4 && AR == AR_EXACT) ? (XW ? SS_4DW_MINBLOCKS : SS_4D_MINBLOCKS) : 1)
    k1_kernel(const __grid_constant__ KParams kp) {
  k1_block<D, AR, VEC, T, XW, D <= 3 ? SS_K1_KBMAX3 : SS_K1_KBMAX4>(kp, blockIdx.x);
}

// ---------------------------------------------------------------------------
// KB: batched persistent kernel. A fixed grid walks the K1 blocks of n
// problems; block g belongs to the problem i with prefix[i] <= g < prefix[i + 1]
// (binary search). CTAs take blocks from a work counter in global memory (one
// atomic per block), so a CTA that drew short blocks (orbits with few members,
// small problems) simply takes more: the blocks differ in size by up to d!
// and a fixed assignment left the grid waiting for its most loaded CTAs. A
// CTA copies a problem's parameters into shared memory when the problem
// changes, then runs that K1 block. One launch covers all problems of one
// (d, arithmetic) class. ctr[0] counts blocks taken and ctr[1] CTAs done; the
// last CTA to finish sets both back to zero for the next launch.
// ---------------------------------------------------------------------------
template <int D, int AR, typename T>
__device__ __forceinline__ void k1_block_anyvec(const KParams& kp, int vec, int64_t b) {
  constexpr int VMAX = sizeof(T) == 8 ? (D <= 3 ? 2 : 1) : (D <= 3 ? 4 : 1);
  constexpr int KBM = D <= 3 ? SS_KB_KBMAX3 : 1;
  if constexpr (VMAX >= 4) {
    if (vec == 4) { k1_block<D, AR, 4, T, 0, KBM>(kp, b); return; }
  }
  if constexpr (VMAX >= 2) {
    if (vec == 2) { k1_block<D, AR, 2, T, 0, KBM>(kp, b); return; }
  }
  k1_block<D, AR, 1, T, 2, KBM>(kp, b);
}

template <int D, int AR, typename T>
__global__ void __launch_bounds__(256, D <= 3 ? SS_KB_MINB3 : 1) kb_kernel(const KParams* __restrict__ probs, const int64_t* __restrict__ prefix,
                                                 const int* __restrict__ vecs, int n, unsigned long long* ctr) {
  __shared__ KParams skp;
  __shared__ unsigned long long next;
  const unsigned long long total = (unsigned long long)prefix[n];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(&ctr[0], 1ull);
    __syncthreads();
    const unsigned long long gu = next;
    __syncthreads();  // every thread has read `next` before thread 0 overwrites it
    if (gu >= total) break;
    const int64_t g = (int64_t)gu;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    if (lo != cur) {
      __syncthreads();
      const int4* src = reinterpret_cast<const int4*>(probs + lo);
      int4* dst = reinterpret_cast<int4*>(&skp);
      for (int i = threadIdx.x; i < (int)(sizeof(KParams) / 16); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      cur = lo;
    }
    k1_block_anyvec<D, AR, T>(skp, vecs[lo], g - prefix[lo]);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctr[1], 1ull) == (unsigned long long)gridDim.x - 1) {
      // every CTA has taken its last block: nothing reads the counters again in this launch
      ctr[0] = 0;
      ctr[1] = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// KG: general strides, one thread per orbit element group
// ---------------------------------------------------------------------------
template <int D, int P, int AR, typename T>
__device__ __forceinline__ void kg_body(const KParams& kp, int64_t g) {
  constexpr int M = Pat<D, P>::M;
  const int64_t orb = g / kp.S;
  int64_t s = g - orb * kp.S;
  int64_t sa = 0, sb = 0;
  for (int k = 0; k < kp.nspec; k++) {
    const int64_t q = s / kp.sext[k];
    const int64_t r = s - q * kp.sext[k];
    sa += r * kp.slda[k];
    sb += r * kp.sldb[k];
    s = q;
  }
  int val[4] = {0, 0, 0, 0};
  unrank<Pat<D, P>::ND>(orb, kp.O, val);
  const T* A = static_cast<const T*>(kp.A);
  T* B = static_cast<T*>(kp.B);
  int64_t offA[M], offB[M];
#pragma unroll
  for (int u = 0; u < M; u++) {
    int64_t a = sa, b = sb;
#pragma unroll
    for (int k = 0; k < D; k++) {
      const int t = val[Pat<D, P>::lab(u, k)];
      a += (int64_t)t * kp.lda[k];
      b += (int64_t)t * kp.ldb[k];
    }
    offA[u] = a;
    offB[u] = b;
  }
  T x[M], y[M];
#pragma unroll
  for (int u = 0; u < M; u++) x[u] = A[offA[u]];
  apply_group<D, P, AR, T>(kp, x, y);
  const T bt = beta_of<T>(kp);
#pragma unroll
  for (int u = 0; u < M; u++) B[offB[u]] = (kp.flags & KF_BETA) ? add_beta(y[u], B[offB[u]], bt) : y[u];
}

template <int D, int AR, typename T>
__global__ void __launch_bounds__(256) kg_kernel(const __grid_constant__ KParams kp) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= kp.ngroup) return;
  const int p = find_pattern<D>(kp.gpre, g);
  const int64_t lg = g - kp.gpre[p];
  switch (p) {
    case 0: kg_body<D, 0, AR, T>(kp, lg); break;
    case 1: kg_body<D, 1, AR, T>(kp, lg); break;
    case 2: if constexpr (npatterns(D) > 2) kg_body<D, 2, AR, T>(kp, lg); break;
    case 3: if constexpr (npatterns(D) > 3) kg_body<D, 3, AR, T>(kp, lg); break;
    default:
      if constexpr (D == 4) {
        switch (p) {
          case 4: kg_body<D, 4, AR, T>(kp, lg); break;
          case 5: kg_body<D, 5, AR, T>(kp, lg); break;
          case 6: kg_body<D, 6, AR, T>(kp, lg); break;
          case 7: kg_body<D, 7, AR, T>(kp, lg); break;
        }
      }
  }
}

}  // namespace ss
