// Internal definitions shared by the host planner and the CUDA kernels of the
// spin-summation library (not part of the public C-ABI).
//
// Orbits. For a canonical (sorted) permuted tuple t0 the tensor elements
// A[s, t0 o tau], tau in S_d, form one orbit: the d! update statements of the
// innermost loop of Algorithm 2 read and write exactly these elements, and
// every A element is reused by all of them (Sec. 4.2). The members are the
// distinct rearrangements of t0; their number m depends only on which entries
// of t0 are equal (the "pattern"): {6, 3, 3, 1} for d = 3, and
// {24, 12, 12, 12, 6, 4, 4, 1} for d = 4 (footnotes 3-4: equal-index cases
// drop redundant updates). A pattern is given by a label tuple, e.g. (0,0,1)
// for i = j < k; the orbits of a pattern are the strictly increasing choices
// of its distinct values.
//
// Within an orbit, output member u of the summation needs input member
// idx[u][sigma], the member equal to t_u o sigma (Def. 2), for every sigma in
// lexicographic order. These tables are computed at compile time.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace ss {

constexpr int fact(int n) { return n <= 1 ? 1 : n * fact(n - 1); }
constexpr int npatterns(int D) { return D == 2 ? 2 : (D == 3 ? 4 : 8); }

// label tuple of pattern P (sorted, labels 0..nd-1)
constexpr int pattern_label(int D, int P, int m) {
  if (D == 2) {
    constexpr int t[2][2] = {{0, 1}, {0, 0}};
    return t[P][m];
  }
  if (D == 3) {
    constexpr int t[4][3] = {{0, 1, 2}, {0, 0, 1}, {0, 1, 1}, {0, 0, 0}};
    return t[P][m];
  }
  constexpr int t[8][4] = {{0, 1, 2, 3}, {0, 0, 1, 2}, {0, 1, 1, 2}, {0, 1, 2, 2},
                           {0, 0, 1, 1}, {0, 0, 0, 1}, {0, 1, 1, 1}, {0, 0, 0, 0}};
  return t[P][m];
}

template <int D>
struct Sym {
  int p[fact(D)][D] = {};
};

// S_D in lexicographic one-line order (0-based images), id first
template <int D>
constexpr Sym<D> make_sym() {
  Sym<D> s{};
  int a[D] = {};
  for (int i = 0; i < D; i++) a[i] = i;
  for (int n = 0; n < fact(D); n++) {
    for (int i = 0; i < D; i++) s.p[n][i] = a[i];
    int i = D - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) break;
    int j = D - 1;
    while (a[j] < a[i]) j--;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int x = i + 1, y = D - 1; x < y; x++, y--) { t = a[x]; a[x] = a[y]; a[y] = t; }
  }
  return s;
}

template <int D>
struct Pattern {
  int m = 0;                    // orbit members
  int nd = 0;                   // distinct values
  int lab[fact(D)][D] = {};     // member label tuples, member 0 = canonical
  int idx[fact(D)][fact(D)] = {};  // idx[u][sigma]: member equal to (member u) o sigma
};

template <int D>
constexpr Pattern<D> make_pattern(int P) {
  Pattern<D> r{};
  Sym<D> S = make_sym<D>();
  int base[D] = {};
  int nd = 0;
  for (int m = 0; m < D; m++) {
    base[m] = pattern_label(D, P, m);
    if (base[m] + 1 > nd) nd = base[m] + 1;
  }
  r.nd = nd;
  // members: distinct base o tau, tau in lex order
  for (int n = 0; n < fact(D); n++) {
    int t[D] = {};
    for (int m = 0; m < D; m++) t[m] = base[S.p[n][m]];
    bool seen = false;
    for (int u = 0; u < r.m; u++) {
      bool same = true;
      for (int m = 0; m < D; m++) same = same && r.lab[u][m] == t[m];
      seen = seen || same;
    }
    if (!seen) {
      for (int m = 0; m < D; m++) r.lab[r.m][m] = t[m];
      r.m++;
    }
  }
  for (int u = 0; u < r.m; u++) {
    for (int n = 0; n < fact(D); n++) {
      int t[D] = {};
      for (int m = 0; m < D; m++) t[m] = r.lab[u][S.p[n][m]];
      int v = -1;
      for (int w = 0; w < r.m; w++) {
        bool same = true;
        for (int m = 0; m < D; m++) same = same && r.lab[w][m] == t[m];
        if (same) v = w;
      }
      r.idx[u][n] = v;
    }
  }
  return r;
}

template <int D, int P>
struct PT {
  static constexpr Pattern<D> t = make_pattern<D>(P);
};

// ---------------------------------------------------------------------------
// Klein four-group transform of 4D orbits. V = {e, (01)(23), (02)(13),
// (03)(12)} (0-based places) is a normal subgroup of S_4. Where no double
// transposition fixes the orbit's canonical tuple (every pattern but
// (0,0,1,1) and (0,0,0,0)), V acts freely on the members from the right
// (t -> t o v), so they fall into m/4 V-orbits of 4. Transforming each
// V-orbit with the characters of V = Z_2 x Z_2 (a 4-point Walsh-Hadamard
// transform, entries +-1) turns every pi_sigma into a signed permutation of
// the transformed values (pi_sigma o pi_v = pi_(sigma v sigma^-1) o pi_sigma
// maps V-orbits to V-orbits and characters to characters), so the orbit
// operator sum_sigma a_sigma pi_sigma becomes a sparse matrix whose entries
// are signed sums of the a_sigma: 6 nonzeros per row for the 24-member orbit
// (144 products instead of 576), 3 or 6 for the 12-member orbits (54 instead
// of 144), 1 or 3 for the 4-member orbits (10 instead of 16). The inverse
// transform is the transpose divided by 4.
// ---------------------------------------------------------------------------
constexpr int KLEIN[4] = {0, 7, 16, 23};  // lex indices of e, (01)(23), (02)(13), (03)(12); v_a o v_b = v_(a xor b)

constexpr int chi4(int k, int vi) {  // character k of V at v_vi: (-1)^popcount(k & vi)
  return ((k & vi & 1) ^ ((k & vi) >> 1 & 1)) ? -1 : 1;
}

struct Wht4 {
  bool ok = false;        // V acts freely on the members
  int m = 0, nb = 0;      // members, V-orbits (m = 4 nb)
  int orb[6][4] = {};     // member of V-orbit o at v_vi: (representative) o v_vi
  int nnz[24] = {};       // transformed row i = 4 o + k (character k of V-orbit o): nonzeros
  int col[24][6] = {};    // their transformed columns
  int woff[25] = {};      // row i's weights: w[woff[i] .. woff[i] + nnz[i])
  int jmap[24][24] = {};  // pi_sigma (lex index s) sends row i to column jmap[i][s] ...
  int smap[24][24] = {};  // ... with sign smap[i][s]; the weight of (i, j) is sum over s with
                          // jmap[i][s] = j of smap[i][s] * a_s
};

constexpr Wht4 make_wht4(int P) {
  Wht4 w{};
  const Pattern<4> pt = make_pattern<4>(P);
  w.m = pt.m;
  int memorb[24] = {}, memvi[24] = {};
  for (int u = 0; u < 24; u++) memorb[u] = -1;
  for (int u = 0; u < pt.m; u++) {
    if (memorb[u] >= 0) continue;
    if (w.nb >= 6) return w;
    for (int vi = 0; vi < 4; vi++) {
      const int v = pt.idx[u][KLEIN[vi]];
      if (memorb[v] >= 0) return w;  // a double transposition fixes a member: not free
      memorb[v] = w.nb;
      memvi[v] = vi;
      w.orb[w.nb][vi] = v;
    }
    w.nb++;
  }
  for (int o = 0; o < w.nb; o++)
    for (int k = 0; k < 4; k++) {
      const int i = 4 * o + k;
      for (int s = 0; s < 24; s++) {
        // M_s[i][4 o' + k'] = 1/4 sum_vi chi_k(vi) chi_k'(vi'), where member
        // orb[o][vi] o sigma = orb[o'][vi']
        const int o2 = memorb[pt.idx[w.orb[o][0]][s]];
        for (int k2 = 0; k2 < 4; k2++) {
          int acc = 0;
          for (int vi = 0; vi < 4; vi++) acc += chi4(k, vi) * chi4(k2, memvi[pt.idx[w.orb[o][vi]][s]]);
          if (acc == 4 || acc == -4) {
            w.jmap[i][s] = 4 * o2 + k2;
            w.smap[i][s] = acc / 4;
          }
        }
        bool seen = false;
        for (int q = 0; q < w.nnz[i]; q++) seen = seen || w.col[i][q] == w.jmap[i][s];
        if (!seen) {
          if (w.nnz[i] >= 6) return Wht4{};
          w.col[i][w.nnz[i]++] = w.jmap[i][s];
        }
      }
      w.woff[i + 1] = w.woff[i] + w.nnz[i];
    }
  w.ok = true;
  return w;
}

// offsets of each transformable pattern's weights in the wh table
constexpr int wh_offset(int P) {
  int o = 0;
  for (int q = 0; q < P; q++) {
    const Wht4 w = make_wht4(q);
    if (w.ok) o += w.woff[w.m];
  }
  return o;
}
constexpr int WH_TOTAL = 144 + 3 * 54 + 2 * 10;

// offsets of each pattern's dense expanded matrix in the M table
template <int D>
constexpr int mp_offset(int P) {
  int o = 0;
  for (int q = 1; q < P; q++) {
    int m = make_pattern<D>(q).m;
    o += m * m;
  }
  return o;
}
constexpr int MP_TOTAL_3 = 9 + 9 + 1;
constexpr int MP_TOTAL_4 = 3 * 144 + 36 + 16 + 16 + 1;
constexpr int MP_MAX = MP_TOTAL_4;

// K1T pipeline shape: consumer warps and stages per CTA (3D / 4D)
#ifndef SS_K1T3_NCW
#define SS_K1T3_NCW 8
#endif
#ifndef SS_K1T3_NST
#define SS_K1T3_NST 4
#endif
#ifndef SS_K1T4_NCW
#define SS_K1T4_NCW 8
#endif
#ifndef SS_K1T4_NST
#define SS_K1T4_NST 3
#endif

// K2 CTA grouping: log2 of the tiles per coarse-block edge (2D / 3D / 4D)
#ifndef SS_K2_LF2
#define SS_K2_LF2 0
#endif
#ifndef SS_K2_LF3
#define SS_K2_LF3 1
#endif
#ifndef SS_K2_LF4
#define SS_K2_LF4 2
#endif
// K2: buffers of d! tiles per CTA (2 = the next block orbit is copied while the
// current one is computed) and resident CTAs per SM the register budget is
// sized for
#ifndef SS_K2_NBUF2
#define SS_K2_NBUF2 2
#endif
#ifndef SS_K2_RUN2
#define SS_K2_RUN2 4
#endif
#ifndef SS_K2_MINB2
#define SS_K2_MINB2 4
#endif
#ifndef SS_K2_NBUF3
#define SS_K2_NBUF3 2
#endif
#ifndef SS_K2_NBUF4
#define SS_K2_NBUF4 1
#endif
// K2: consecutive work ids per CTA (0 = persistent grid of the resident CTAs
// taking every G-th id). Hardware dispatches CTAs in order, so runs keep the
// ids in flight a compact window; a persistent round robin lets it spread.
#ifndef SS_K2_RUN3
#define SS_K2_RUN3 4
#endif
#ifndef SS_K2_RUN4
#define SS_K2_RUN4 1
#endif
#ifndef SS_K2_MINB3
#define SS_K2_MINB3 4
#endif
#ifndef SS_K2_MINB4
#define SS_K2_MINB4 2
#endif
// K2: degenerate block orbits take their canonical offsets grouped by element
// pattern (1) or in tile order (0)
#ifndef SS_K2_SORTED
#define SS_K2_SORTED 1
#endif
// K2, d = 4 through the Klein four-group transform: buffers, ids per CTA and
// resident CTAs per SM
#ifndef SS_K2_NBUF4W
#define SS_K2_NBUF4W 1
#endif
#ifndef SS_K2_RUN4W
#define SS_K2_RUN4W 1
#endif
#ifndef SS_K2_MINB4W
#define SS_K2_MINB4W 3
#endif

// generic d = 4 orbits with a non-power-of-two alpha: 1 = an out-of-line
// path that reloads the inputs (the common path stays 2 % faster; a
// non-power-of-two alpha runs at about 2/3 of the inline copy's speed),
// 0 = a second inline copy of the core
#ifndef SS_4D_SCALED_OUTOFLINE
#define SS_4D_SCALED_OUTOFLINE 1
#endif

// batched kernel (3D): resident CTAs per SM the register budget is sized for,
// and the most chunks a thread takes at a time (as SS_K1_KBMAX3)
#ifndef SS_KB_MINB3
#define SS_KB_MINB3 4
#endif
#ifndef SS_KB_KBMAX3
#define SS_KB_KBMAX3 1
#endif

// K2: the beta term of the copy-out in an out-of-line call (1) or inline (0)
#ifndef SS_K2_BETA_CALL
#define SS_K2_BETA_CALL 1
#endif
// K2, d = 4 through the Klein four-group transform: slots of the generic
// orbit's members from a per-thread table in shared memory (1) or recomputed (0)
#ifndef SS_K2_SLOTS4
#define SS_K2_SLOTS4 1
#endif
// K2: block orbits whose tiles are all full copied by an unrolled loop
// without bounds checks (d <= 3)
#ifndef SS_K2_COPY_FULL
#define SS_K2_COPY_FULL 1
#endif
// 4D generic orbit in the exact core: outputs per register group (24 / G)
// and the CTAs per SM the kernel is compiled for
#ifndef SS_4D_GROUPS
#define SS_4D_GROUPS 3
#endif
#ifndef SS_4D_MINBLOCKS
#define SS_4D_MINBLOCKS 3
#endif
// K1 (single problems): most chunks a thread takes at a time for orbits with
// fewer members than the generic one, for d <= 3 and d = 4 (1 = one chunk at
// a time for every orbit; the batched kernel always takes one)
#ifndef SS_K1_KBMAX3
#define SS_K1_KBMAX3 2
#endif
#ifndef SS_K1_KBMAX4
#define SS_K1_KBMAX4 1
#endif
// K1, d = 4 transform path: spectator positions per member per block
#ifndef SS_K1_POS4
#define SS_K1_POS4 5120
#endif
// K1, d = 4 transform path: bulk L2 prefetch of the member runs this many
// chunks ahead (0: none)
#ifndef SS_4DW_PREFETCH
#define SS_4DW_PREFETCH 1
#endif
// ... with an evict-last L2 policy on the prefetched lines (1)
#ifndef SS_4DW_PFHINT
#define SS_4DW_PFHINT 1
#endif
// the same for the K1 kernel of d = 4 orbits through the Klein four-group transform
#ifndef SS_4DW_MINBLOCKS
#define SS_4DW_MINBLOCKS 3
#endif

constexpr int MAXSTAGE = 8;
constexpr int MAXSTAGE_EXACT = 3;  // the exact core unrolls at most this many stages
constexpr int MAXSPEC = 4;

enum Arith {
  AR_EXACT = 0,
  AR_STRICT = 1,
  AR_F32 = 2,
  AR_EXACT_XW = 3,  // kernel-template choice only: AR_EXACT with d = 4 orbits through the Klein four-group transform
};

// flags
enum {
  KF_BETA = 1,        // beta != 0: read B_old
  KF_ALPHA_MUL = 2,   // exact path: alpha is not a power of two, multiply at the end
  KF_KDROP = 4,       // exact path: round the fixed-point sum before conversion
  KF_WHT = 8,         // exact path, d = 4: freely transformable orbits through the Klein four-group transform
};

// Kernel parameters (passed by value as a __grid_constant__, or from a
// device array in batched plans; 16-byte aligned so CTAs copy it as int4).
struct alignas(16) KParams {
  const void* A;
  void* B;
  int64_t S;                    // spectator elements per permuted tuple
  int64_t lda[4], ldb[4];       // permuted-index strides (elements)
  // general spectator layout (used when the spectator block is not dense)
  int64_t sext[MAXSPEC];        // spectator extents
  int64_t slda[MAXSPEC], sldb[MAXSPEC];
  int nspec;
  int O;                        // permuted extent
  int nstage;                   // stages of the FP64/FP32 sigma lists cd (1 = expanded)
  int nci;                      // stages of the exact integer sigma lists ci (<= MAXSTAGE_EXACT)
  int flags;
  double alpha, beta;
  // exact fixed-point path
  int W;                        // limb width; grid = 2^(E+1-2W) of the orbit element's max
  int s0;                       // 53 - 2W
  int kdrop;                    // low bits rounded off the sum before conversion
  int wk;                       // W - kdrop
  long long rnd;                // 2^(kdrop-1) or 0
  int cexp;                     // added to the max exponent field to build the conversion constant
  unsigned emin, emax;          // fast path when the max exponent field lies in [emin, emax]
  int ci[MAXSTAGE][24];         // sigma-list coefficients per stage, scaled integers (application order)
  int mp[MP_MAX];               // degenerate patterns: expanded orbit matrices M_p, scaled integers
  int wh[WH_TOTAL];             // d = 4 with KF_WHT: transformed orbit operators (Wht4), scaled integers
  double cd[MAXSTAGE][24];      // sigma-list coefficients per stage (strict path, application order)
  float cf[MAXSTAGE][24];       // the same rounded to FP32 (FP32 path)
  float alphaf, betaf;
  int* status;                  // device status word (bounded waits report here)
  long long wait_limit;         // iterations of a bounded wait before it gives up
  // block mapping: pattern p owns blocks [pre[p], pre[p+1]); each block covers
  // one orbit and cpb chunks of VEC*blockDim spectator elements
  int64_t pre[9];
  int64_t nchunk;               // chunks per orbit
  int cpb;                      // chunks per block
  int k2lf;                     // K2: log2 of the tiles per coarse-block edge (CTA grouping)
  int64_t norb[8];              // orbits per pattern
  int64_t ngroup;               // general kernel: total orbit-element groups
  int64_t gpre[9];              // general kernel: group prefix per pattern
};

// a planned single problem (host side)
struct Launch {
  KParams kp;
  int ar = AR_STRICT;
  int kernel = 0;  // 0 = K1 (registers), 1 = KG (general strides), 2 = K1T (TMA-staged), 3 = K2 (N^d tiles)
  int vec = 1;
  bool empty = false;
};

// byte layout of a batch image (plan memory, or the library's fixed array)
// for at most n problems: KParams[n], then the K1-block prefix segments of the
// (d, arithmetic) classes (class c has n_c + 1 entries, so n +
// BATCH_MAX_CLASSES int64 in all), then the vector widths (n int)
constexpr size_t batch_offset_probs(int n) { return (void)n, 0; }
constexpr size_t batch_offset_prefix(int n) { return sizeof(KParams) * (size_t)n; }
constexpr int BATCH_MAX_CLASSES = 12;  // (d, arithmetic) classes: 3 x 3, with room
constexpr size_t batch_offset_vec(int n) {
  return batch_offset_prefix(n) + sizeof(int64_t) * (size_t)(n + BATCH_MAX_CLASSES);
}
// then, 16-byte aligned, two work counters per class for the batched kernel's
// dynamic schedule (zero between launches: the last CTA of a launch resets them)
constexpr size_t batch_offset_ctr(int n) { return (batch_offset_vec(n) + sizeof(int) * (size_t)n + 15) / 16 * 16; }
constexpr size_t batch_image_bytes(int n) {
  return batch_offset_ctr(n) + 2 * sizeof(unsigned long long) * (size_t)BATCH_MAX_CLASSES;
}

}  // namespace ss
