// Host side of the spin-summation library: argument checks, coefficient
// algebra (product rule, adjoint, orbit matrices), choice of arithmetic and
// kernel, and the extern "C" entry points declared in include/spinsum.h.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/spinsum.h"
#include "ss_internal.h"

namespace ss {
cudaError_t launch_k1(int d, const KParams& kp, int ar, int vec, cudaStream_t st);
cudaError_t launch_kg(int d, const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k1t(int d, const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_k2(int d, const KParams& kp, int ar, cudaStream_t st);
cudaError_t launch_pack(int d, const KParams& kp, bool unpack, bool f64, int vec, cudaStream_t st);
cudaError_t launch_kc(int d, const KParams& kp, int ar, bool sum, const double* W, int64_t Y, int64_t ldw, double* C,
                      int64_t ldc, cudaStream_t st);
int k1t_chunk(int d, int ar);

int* status_ptr();
cudaError_t static_scratch_ptr(void** out);
cudaError_t read_and_clear_status(int* out);
}  // namespace ss

using namespace ss;

namespace {

thread_local std::string t_err;
thread_local int64_t t_launches = 0;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SPINSUM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// permutation group tables (lexicographic order, 0-based images)
// ---------------------------------------------------------------------------
struct Group {
  int d = 0, n = 0;
  int p[24][4] = {};
  int inv[24] = {};       // index of the inverse permutation
  int comp[24][24] = {};  // index of phi o psi, (phi o psi)(m) = phi(psi(m))
};

Group make_group(int d) {
  Group g;
  g.d = d;
  int a[4] = {0, 1, 2, 3};
  for (;;) {
    for (int m = 0; m < d; m++) g.p[g.n][m] = a[m];
    g.n++;
    int i = d - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) break;
    int j = d - 1;
    while (a[j] < a[i]) j--;
    std::swap(a[i], a[j]);
    for (int x = i + 1, y = d - 1; x < y; x++, y--) std::swap(a[x], a[y]);
  }
  auto find = [&](const int* q) {
    for (int k = 0; k < g.n; k++) {
      bool same = true;
      for (int m = 0; m < d; m++) same = same && g.p[k][m] == q[m];
      if (same) return k;
    }
    return -1;
  };
  for (int k = 0; k < g.n; k++) {
    int q[4] = {};
    for (int m = 0; m < d; m++) q[g.p[k][m]] = m;
    g.inv[k] = find(q);
    for (int l = 0; l < g.n; l++) {
      int c[4] = {};
      for (int m = 0; m < d; m++) c[m] = g.p[k][g.p[l][m]];
      g.comp[k][l] = find(c);
    }
  }
  return g;
}

const Group& group(int d) {
  static const Group g2 = make_group(2), g3 = make_group(3), g4 = make_group(4);
  return d == 2 ? g2 : (d == 3 ? g3 : g4);
}

// product of a chain F_1 .. F_k (B = F_1(...F_k(A))): left fold, each entry
// summed over (phi, psi) pairs in lexicographic order, zero terms skipped.
std::vector<double> expand_chain(const Group& g, const std::vector<std::vector<double>>& chain) {
  std::vector<double> P = chain[0];
  for (size_t f = 1; f < chain.size(); f++) {
    std::vector<double> Q(g.n, 0.0);
    for (int a = 0; a < g.n; a++) {
      if (P[a] == 0.0) continue;
      for (int b = 0; b < g.n; b++) {
        if (chain[f][b] == 0.0) continue;
        double prod = P[a] * chain[f][b];
        Q[g.comp[a][b]] = Q[g.comp[a][b]] + prod;
      }
    }
    P = Q;
  }
  return P;
}

// smallest e >= -40 such that every c * 2^e is an integer of magnitude < 2^24;
// returns false if there is none
bool int_scale(const std::vector<double>& c, int* e_out) {
  for (int e = -40; e <= 60; e++) {
    bool ok = true;
    for (double v : c) {
      double s = std::ldexp(v, e);
      if (std::fabs(s) >= 16777216.0 || s != std::floor(s)) { ok = false; break; }
    }
    if (ok) { *e_out = e; return true; }
  }
  return false;
}

// integer exponent a with alpha == +-2^a, else false
bool pow2(double x, int* a) {
  if (x == 0.0 || !std::isfinite(x)) return false;
  int e;
  double m = std::frexp(std::fabs(x), &e);
  if (m != 0.5) return false;
  *a = e - 1;
  return true;
}

int64_t binom(int n, int k) {
  if (n < k || k < 0) return 0;
  int64_t r = 1;
  for (int i = 0; i < k; i++) r = r * (n - i) / (i + 1);
  return r;
}

// the pattern tables and matrix offsets, built once per process (building
// them per call cost about 0.5 ms of host time for d = 4)
template <int D>
const Pattern<D>& host_pattern(int P) {
  static const std::array<Pattern<D>, 8> t = [] {
    std::array<Pattern<D>, 8> a{};
    for (int p = 0; p < npatterns(D); p++) a[p] = make_pattern<D>(p);
    return a;
  }();
  return t[P];
}
template <int D>
int host_mp_offset(int P) {
  static const std::array<int, 9> t = [] {
    std::array<int, 9> a{};
    for (int p = 0; p < npatterns(D); p++) a[p] = mp_offset<D>(p);
    return a;
  }();
  return t[P];
}

template <int D>
int pattern_nd(int P) { return host_pattern<D>(P).nd; }
template <int D>
int pattern_m(int P) { return host_pattern<D>(P).m; }

int nd_of(int d, int P) { return d == 2 ? pattern_nd<2>(P) : (d == 3 ? pattern_nd<3>(P) : pattern_nd<4>(P)); }

// dense expanded orbit matrices of the degenerate patterns
template <int D>
void fill_mp(const std::vector<long long>& a, int* mp) {
  for (int P = 1; P < npatterns(D); P++) {
    const Pattern<D>& pt = host_pattern<D>(P);
    int* M = mp + host_mp_offset<D>(P);
    for (int u = 0; u < pt.m; u++)
      for (int v = 0; v < pt.m; v++) M[u * pt.m + v] = 0;
    for (int u = 0; u < pt.m; u++)
      for (int s = 0; s < fact(D); s++) M[u * pt.m + pt.idx[u][s]] += (int)a[s];
  }
}

// the transformed orbit operators of the Klein four-group transform (d = 4):
// weight (i, q) = sum over sigma with jmap[i][sigma] = col[i][q] of
// smap[i][sigma] * a_sigma
const std::array<Wht4, 8>& host_wht4() {
  static const std::array<Wht4, 8> t = [] {
    std::array<Wht4, 8> a{};
    for (int p = 0; p < 8; p++) a[p] = make_wht4(p);
    return a;
  }();
  return t;
}

// SPINSUM_4D_DENSE_CORE set to a nonzero value: d = 4 orbits take the dense
// fixed-point core on the grid the transform would use (read on every call)
bool dense_4d_requested() {
  const char* e = getenv("SPINSUM_4D_DENSE_CORE");
  return e && atoi(e) != 0;
}

void fill_wh(const std::vector<long long>& a, int* wh) {
  int off = 0;
  for (int P = 0; P < 8; P++) {
    const Wht4& w = host_wht4()[P];
    if (!w.ok) continue;
    for (int i = 0; i < w.m; i++)
      for (int q = 0; q < w.nnz[i]; q++) {
        long long v = 0;
        for (int s = 0; s < 24; s++)
          if (w.jmap[i][s] == w.col[i][q]) v += w.smap[i][s] * a[s];
        wh[off + w.woff[i] + q] = (int)v;
      }
    off += w.woff[w.m];
  }
}

// polls of a bounded device-side wait before it reports SPINSUM_ERR_TIMEOUT;
// SPINSUM_WAIT_LIMIT overrides the default (2^22 polls, well under a minute)
long long wait_limit() {
  static long long v = [] {
    const char* e = getenv("SPINSUM_WAIT_LIMIT");
    long long x = e ? atoll(e) : 0;
    return x > 0 ? x : (1LL << 22);
  }();
  return v;
}

struct Request {
  int d, dtype;
  const int64_t* ext;
  const void* A;
  const int64_t* lda;
  void* B;
  const int64_t* ldb;
  const double* coef;
  int nfactors, mode;
  double alpha, beta;
  int inplace;
};

// byte span [lo, hi) touched by a strided tensor
void span(int n, const int64_t* ext, const int64_t* ld, const void* base, size_t es, uintptr_t* lo,
          uintptr_t* hi) {
  int64_t mx = 0;
  for (int k = 0; k < n; k++) mx += (ext[k] - 1) * ld[k];
  *lo = (uintptr_t)base;
  *hi = (uintptr_t)base + (uintptr_t)((mx + 1) * (int64_t)es);
}

int plan_one(const Request& r, Launch* L) {
  const int d = r.d;
  if (d < 2 || d > 4) return fail(SPINSUM_ERR_ARG, "d must be 2, 3 or 4");
  if (r.dtype != SPINSUM_F64 && r.dtype != SPINSUM_F32) return fail(SPINSUM_ERR_ARG, "unknown dtype %d", r.dtype);
  if (r.mode & ~(SPINSUM_FACTORIZED | SPINSUM_ADJOINT | SPINSUM_STRICT | SPINSUM_TMA))
    return fail(SPINSUM_ERR_ARG, "unknown mode bits 0x%x", r.mode);
  if ((r.mode & SPINSUM_STRICT) && r.dtype != SPINSUM_F64)
    return fail(SPINSUM_ERR_ARG, "SPINSUM_STRICT applies to FP64 only");
  if (!r.ext || !r.lda || !r.ldb) return fail(SPINSUM_ERR_ARG, "null extent or stride array");
  if (r.nfactors < 1 || r.nfactors > MAXSTAGE) return fail(SPINSUM_ERR_ARG, "nfactors must be 1..%d", MAXSTAGE);
  if (!r.coef) return fail(SPINSUM_ERR_ARG, "null coefficient array");
  if (!std::isfinite(r.alpha) || !std::isfinite(r.beta)) return fail(SPINSUM_ERR_ARG, "alpha/beta must be finite");
  const int nidx = 2 * d;
  int64_t total = 1;
  for (int k = 0; k < nidx; k++) {
    if (r.ext[k] < 0) return fail(SPINSUM_ERR_ARG, "negative extent at index %d", k);
    total *= r.ext[k];
  }
  const int O = (int)r.ext[d];
  for (int k = d; k < nidx; k++)
    if (r.ext[k] != r.ext[d]) return fail(SPINSUM_ERR_ARG, "permuted extents must be equal (index %d)", k);
  const int64_t omax = d == 2 ? 65536 : 4096;
  if (r.ext[d] > omax) return fail(SPINSUM_ERR_UNSUPPORTED, "permuted extent above %lld", (long long)omax);
  const Group& g = group(d);
  for (int i = 0; i < r.nfactors * g.n; i++)
    if (!std::isfinite(r.coef[i])) return fail(SPINSUM_ERR_ARG, "non-finite coefficient at %d", i);
  for (int k = 0; k < nidx; k++)
    if (r.lda[k] < 0 || r.ldb[k] < 0) return fail(SPINSUM_ERR_UNSUPPORTED, "negative strides are not supported");
  if (total == 0) { L->empty = true; return SPINSUM_OK; }
  if (!r.A || !r.B) return fail(SPINSUM_ERR_ARG, "null tensor pointer");
  const size_t es = r.dtype == SPINSUM_F64 ? 8 : 4;
  if (((uintptr_t)r.A % es) || ((uintptr_t)r.B % es)) return fail(SPINSUM_ERR_ARG, "misaligned tensor pointer");
  if (r.inplace) {
    if (r.A != r.B) return fail(SPINSUM_ERR_ALIAS, "inplace requires A == B");
    for (int k = 0; k < nidx; k++)
      if (r.lda[k] != r.ldb[k]) return fail(SPINSUM_ERR_ALIAS, "inplace requires lda == ldb");
  } else {
    uintptr_t alo, ahi, blo, bhi;
    span(nidx, r.ext, r.lda, r.A, es, &alo, &ahi);
    span(nidx, r.ext, r.ldb, r.B, es, &blo, &bhi);
    if (alo < bhi && blo < ahi) return fail(SPINSUM_ERR_ALIAS, "A and B overlap (use inplace = 1 for A == B)");
  }

  // ---- coefficients: chain in application order (innermost first) ----
  std::vector<std::vector<double>> chain(r.nfactors, std::vector<double>(g.n));
  for (int f = 0; f < r.nfactors; f++)
    for (int s = 0; s < g.n; s++) chain[f][s] = r.coef[f * g.n + s];
  if (r.mode & SPINSUM_ADJOINT) {
    // (F_1 ... F_k)^T = F_k^T ... F_1^T, F^T[sigma] = F[sigma^-1]
    std::vector<std::vector<double>> t(r.nfactors, std::vector<double>(g.n));
    for (int f = 0; f < r.nfactors; f++)
      for (int s = 0; s < g.n; s++) t[f][s] = chain[r.nfactors - 1 - f][g.inv[s]];
    chain = t;
  }
  const bool factorized = (r.mode & SPINSUM_FACTORIZED) && r.nfactors > 1;
  std::vector<std::vector<double>> stages;  // application order
  const std::vector<double> full = expand_chain(g, chain);
  if (factorized) {
    for (int f = r.nfactors - 1; f >= 0; f--) stages.push_back(chain[f]);
  } else {
    stages.push_back(full);
  }

  KParams& kp = L->kp;
  memset(&kp, 0, sizeof kp);
  kp.A = r.A;
  kp.B = r.B;
  kp.O = O;
  kp.alpha = r.alpha;
  kp.beta = r.beta;
  kp.nstage = (int)stages.size();
  kp.flags = r.beta != 0.0 ? KF_BETA : 0;
  for (int st = 0; st < kp.nstage; st++)
    for (int s = 0; s < g.n; s++) {
      kp.cd[st][s] = stages[st][s];
      kp.cf[st][s] = (float)stages[st][s];
    }
  kp.alphaf = (float)r.alpha;
  kp.betaf = (float)r.beta;
  kp.wait_limit = wait_limit();
  for (int k = 0; k < d; k++) {
    kp.lda[k] = r.lda[d + k];
    kp.ldb[k] = r.ldb[d + k];
  }

  // ---- arithmetic ----
  if (r.dtype == SPINSUM_F32) {
    L->ar = AR_F32;
  } else if (r.mode & SPINSUM_STRICT) {
    L->ar = AR_STRICT;
  } else {
    L->ar = AR_STRICT;
    // exact fixed-point path: integer stage coefficients up to a power-of-two scale
    // in exact arithmetic a chain and its expansion give identical results,
    // so a chain longer than the exact core unrolls is applied expanded
    std::vector<std::vector<double>> istages = stages;
    if (istages.size() > (size_t)MAXSTAGE_EXACT) istages.assign(1, full);
    bool ok = true;
    int escale = 0;
    double Lnorm = 1.0;
    std::vector<std::vector<long long>> ist(istages.size());
    for (size_t st = 0; st < istages.size() && ok; st++) {
      int e;
      if (!int_scale(istages[st], &e)) { ok = false; break; }
      escale += e;
      double n1 = 0;
      for (int s = 0; s < g.n; s++) {
        ist[st].push_back((long long)std::ldexp(istages[st][s], e));
        n1 += std::fabs(std::ldexp(istages[st][s], e));
      }
      Lnorm *= n1;
    }
    int a = 0;
    const bool apow2 = pow2(r.alpha, &a);
    if (ok && Lnorm >= 1.0 && Lnorm <= 127.0) {
      // limb width W: every limb sum, plus the rounding increment of the low
      // limb, stays below 2^31; kdrop rounds the joined sum to below 2^50
      int W = 26, kdrop = 0;
      for (;;) {
        kdrop = 0;
        const double ymax = Lnorm * (std::ldexp(1.0, 2 * W) + std::ldexp(1.0, W));
        while (ymax / std::ldexp(1.0, kdrop) + 1.0 >= std::ldexp(1.0, 50)) kdrop++;
        const double rnd = kdrop ? std::ldexp(1.0, kdrop - 1) : 0.0;
        if (W == 0 || Lnorm * std::ldexp(1.0, W) + rnd <= 2147483647.0) break;
        W--;
      }
      if (2 * W >= 48) {
        // expanded integer coefficients for the orbit matrices: product of the scaled stages
        std::vector<long long> ex(g.n, 0);
        {
          std::vector<long long> P = ist[0];
          for (size_t st = 1; st < ist.size(); st++) {
            std::vector<long long> Q(g.n, 0);
            // stage st is applied after stage st-1: operator = S_st o S_(st-1)
            for (int x = 0; x < g.n; x++)
              for (int y = 0; y < g.n; y++) Q[g.comp[x][y]] += ist[st][x] * P[y];
            P = Q;
          }
          ex = P;
        }
        // d = 4: the Klein four-group transform (Wht4) needs the transformed
        // low limbs (25 bits, non-negative) and high limbs (the 50-bit
        // transformed values shifted down by 25) times the coefficient 1-norm
        // to stay below 2^31, i.e. sum|a| <= 63 on a 48-bit grid; the other
        // patterns then use the same grid (W = 24)
        // (SPINSUM_4D_DENSE_CORE=1 keeps the 48-bit grid but applies the dense
        // orbit matrices instead: the results must then be bit-identical, which
        // the GPU tests check)
        bool wht = false;
        if (d == 4 && apow2) {
          long long lx = 0;
          for (long long v : ex) lx += v < 0 ? -v : v;
          if (lx <= 63) {
            wht = true;
            W = 24;
            kdrop = 0;
            const double ymax = Lnorm * (std::ldexp(1.0, 2 * W) + std::ldexp(1.0, W));
            while (ymax / std::ldexp(1.0, kdrop) + 1.0 >= std::ldexp(1.0, 50)) kdrop++;
          }
        }
        const bool neg = apow2 && r.alpha < 0;
        int aexp = -escale + (apow2 ? a : 0);
        const int cshift = 53 - 2 * W + kdrop + aexp;
        const int emin = std::max(64, 1 - cshift), emax = std::min(2046, 2046 - cshift);
        if (emin <= emax) {
          L->ar = AR_EXACT;
          kp.nci = (int)ist.size();
          kp.W = W;
          kp.s0 = 53 - 2 * W;
          kp.kdrop = kdrop;
          kp.wk = W - kdrop;
          kp.rnd = kdrop ? (1LL << (kdrop - 1)) : 0;
          if (kdrop) kp.flags |= KF_KDROP;
          if (!apow2) kp.flags |= KF_ALPHA_MUL;
          kp.cexp = (int)((unsigned)cshift << 20) + 0x80000;
          kp.emin = (unsigned)emin << 20;
          kp.emax = (unsigned)emax << 20;
          // sign of alpha folded into the last stage / the orbit matrices
          for (size_t st = 0; st < ist.size(); st++)
            for (int s = 0; s < g.n; s++)
              kp.ci[st][s] = (int)((neg && st + 1 == ist.size()) ? -ist[st][s] : ist[st][s]);
          if (neg)
            for (auto& v : ex) v = -v;
          if (d == 4) {
            // d = 4: the generic orbit always applies the expanded operator (identical
            // results in exact arithmetic), which lets the kernel keep one group of
            // outputs live at a time
            kp.nci = 1;
            for (int s = 0; s < g.n; s++) kp.ci[0][s] = (int)ex[s];
          }
          if (d == 2) fill_mp<2>(ex, kp.mp);
          else if (d == 3) fill_mp<3>(ex, kp.mp);
          else fill_mp<4>(ex, kp.mp);
          if (wht && !dense_4d_requested()) {
            kp.flags |= KF_WHT;
            fill_wh(ex, kp.wh);
          }
        }
      }
    }
  }

  // ---- layout and launch shape ----
  int64_t S = 1;
  bool dense = true;
  for (int k = 0; k < d; k++) {
    if (r.ext[k] != 1 && (r.lda[k] != S || r.ldb[k] != S)) dense = false;
    S *= r.ext[k];
  }
  kp.S = S;
  kp.nspec = d;
  for (int k = 0; k < d; k++) {
    kp.sext[k] = r.ext[k];
    kp.slda[k] = r.lda[k];
    kp.sldb[k] = r.ldb[k];
  }
  const int np = npatterns(d);
  for (int p = 0; p < np; p++) kp.norb[p] = binom(O, nd_of(d, p));
  if (dense && S >= 64) {
    L->kernel = 0;
    int vec = 1;
    const int want = d <= 3 ? (r.dtype == SPINSUM_F64 ? 2 : 4) : 1;
    bool aligned = (S % want == 0) && ((uintptr_t)r.A % (es * want) == 0) && ((uintptr_t)r.B % (es * want) == 0);
    for (int k = 0; k < d; k++) aligned = aligned && (kp.lda[k] % want == 0) && (kp.ldb[k] % want == 0);
    if (aligned && want > 1) vec = want;
    L->vec = vec;
    // TMA staging: every member run must start on a 16-byte boundary and span a
    // multiple of 16 bytes (bulk-copy rule), and the vector width must divide S
    bool tma = (r.mode & SPINSUM_TMA) && d == 3 && L->ar != AR_STRICT && aligned && (S * (int64_t)es) % 16 == 0 &&
               (uintptr_t)r.A % 16 == 0 && (uintptr_t)r.B % 16 == 0;
    for (int k = 0; k < d; k++) tma = tma && (kp.lda[k] * (int64_t)es) % 16 == 0;
    if (tma) {
      L->kernel = 2;
      const int ch = k1t_chunk(d, L->ar);
      kp.nchunk = (S + ch - 1) / ch;
      kp.cpb = 1;
      kp.pre[0] = 0;
      for (int p = 0; p < np; p++) kp.pre[p + 1] = kp.pre[p] + kp.norb[p] * kp.nchunk;
      for (int p = np; p < 8; p++) kp.pre[p + 1] = kp.pre[p];
    } else {
      const int64_t per = 256LL * vec;
      kp.nchunk = (S + per - 1) / per;
      // about 8192 positions per member per block, spread evenly over the
      // blocks of an orbit (40 chunks: 20 + 20, not 32 + 8)
      // (d = 4 through the Klein four-group transform: SS_K1_POS4, measured best
      // with the L2 prefetch of the next chunk)
      const int64_t pos = (d == 4 && (kp.flags & KF_WHT)) ? SS_K1_POS4 : 8192;
      const int64_t cpb0 = std::min<int64_t>(kp.nchunk, std::max<int64_t>(1, pos / per));
      const int64_t nbo = (kp.nchunk + cpb0 - 1) / cpb0;
      kp.cpb = (int)((kp.nchunk + nbo - 1) / nbo);
      const int64_t bpo = (kp.nchunk + kp.cpb - 1) / kp.cpb;
      kp.pre[0] = 0;
      for (int p = 0; p < np; p++) kp.pre[p + 1] = kp.pre[p] + kp.norb[p] * bpo;
      for (int p = np; p < 8; p++) kp.pre[p + 1] = kp.pre[p];
    }
    if (kp.pre[np] > 0x7FFFFFFFLL) return fail(SPINSUM_ERR_UNSUPPORTED, "problem too large for one launch");
  } else if (S == 1 && kp.lda[0] == 1 && kp.ldb[0] == 1) {
    // the paper's layout: no spectators, the first permuted index at stride 1 --
    // tiled block orbits through shared memory (K2)
    L->kernel = 3;
    const int bl = d == 2 ? 32 : (d == 3 ? 8 : 4);
    const int nb = (O + bl - 1) / bl;
    // CTAs in groups of F^d over sorted coarse tuples (multisets of d of nc values)
    kp.k2lf = d == 2 ? SS_K2_LF2 : (d == 3 ? SS_K2_LF3 : SS_K2_LF4);
    const int64_t nc = ((nb - 1) >> kp.k2lf) + 1;
    const int64_t grid = binom(nc + d - 1, d) << (d * kp.k2lf);
    for (int p = 0; p <= 8; p++) kp.pre[p] = p < np ? 0 : grid;
    if (grid > 0x7FFFFFFFLL) return fail(SPINSUM_ERR_UNSUPPORTED, "problem too large for one launch");
  } else {
    L->kernel = 1;
    kp.gpre[0] = 0;
    for (int p = 0; p < np; p++) kp.gpre[p + 1] = kp.gpre[p] + kp.norb[p] * S;
    for (int p = np; p < 8; p++) kp.gpre[p + 1] = kp.gpre[p];
    kp.ngroup = kp.gpre[np];
    if ((kp.ngroup + 255) / 256 > 0x7FFFFFFFLL) return fail(SPINSUM_ERR_UNSUPPORTED, "problem too large");
  }
  return SPINSUM_OK;
}

// Packed antisymmetric storage: B (2d indices, dense spectators at stride 1)
// and P (d spectator indices with B's dense strides, then the packed index
// r = colex rank of i_1 < .. < i_d). unpack: P -> B, pack: B -> P.
int run_pack(bool unpack, int d, int dtype, const int64_t* ext, const void* P, const int64_t* ldp, const void* B,
             const int64_t* ldb, cudaStream_t st) {
  t_err.clear();
  if (d < 2 || d > 4) return fail(SPINSUM_ERR_ARG, "d must be 2, 3 or 4");
  if (dtype != SPINSUM_F64 && dtype != SPINSUM_F32) return fail(SPINSUM_ERR_ARG, "unknown dtype %d", dtype);
  if (!ext || !ldp || !ldb) return fail(SPINSUM_ERR_ARG, "null extent or stride array");
  const size_t es = dtype == SPINSUM_F64 ? 8 : 4;
  int64_t S = 1;
  for (int k = 0; k < d; k++) {
    if (ext[k] < 0) return fail(SPINSUM_ERR_ARG, "negative extent at index %d", k);
    if (ext[k] != 1 && (ldb[k] != S || ldp[k] != S))
      return fail(SPINSUM_ERR_UNSUPPORTED, "spectator indices must be dense and fastest in P and B");
    S *= ext[k];
  }
  const int64_t O = ext[d];
  for (int k = d; k < 2 * d; k++) {
    if (ext[k] != O) return fail(SPINSUM_ERR_ARG, "permuted extents must be equal (index %d)", k);
    if (ldb[k] < 0) return fail(SPINSUM_ERR_UNSUPPORTED, "negative strides are not supported");
  }
  if (O > 4096) return fail(SPINSUM_ERR_UNSUPPORTED, "permuted extent above 4096");
  if (ldp[d] < S) return fail(SPINSUM_ERR_ARG, "packed-index stride below the spectator block");
  const int64_t npack = binom((int)O, d);
  if (S == 0 || O == 0) return SPINSUM_OK;
  if (!P || !B) return fail(SPINSUM_ERR_ARG, "null tensor pointer");
  // P and B must not overlap
  uintptr_t plo = (uintptr_t)P, phi = plo + (uintptr_t)(((npack > 0 ? (npack - 1) * ldp[d] : 0) + S) * (int64_t)es);
  uintptr_t blo = 0, bhi = 0;
  span(2 * d, ext, ldb, B, es, &blo, &bhi);
  if (npack > 0 && plo < bhi && blo < phi) return fail(SPINSUM_ERR_ALIAS, "P and B overlap");
  KParams kp{};
  kp.A = P;
  kp.B = const_cast<void*>(B);
  kp.S = S;
  kp.O = (int)O;
  kp.lda[0] = ldp[d];
  for (int k = 0; k < d; k++) kp.ldb[k] = ldb[d + k];
  const int np = npatterns(d);
  for (int p = 0; p < np; p++) kp.norb[p] = (unpack || p == 0) ? binom((int)O, nd_of(d, p)) : 0;
  const int want = 2;  // pairs: 16 bytes (FP64) or 8 bytes (FP32)
  bool pair = S % want == 0 && (uintptr_t)P % (es * want) == 0 && (uintptr_t)B % (es * want) == 0 &&
              ldp[d] % want == 0;
  for (int k = d; k < 2 * d; k++) pair = pair && ldb[k] % want == 0;
  const int vec = pair ? want : 1;
  const int64_t per = 256LL * vec;
  kp.nchunk = (S + per - 1) / per;
  const int64_t cpb0 = std::min<int64_t>(kp.nchunk, std::max<int64_t>(1, 8192 / per));
  const int64_t nbo = (kp.nchunk + cpb0 - 1) / cpb0;
  kp.cpb = (int)((kp.nchunk + nbo - 1) / nbo);
  const int64_t bpo = (kp.nchunk + kp.cpb - 1) / kp.cpb;
  kp.pre[0] = 0;
  for (int p = 0; p < np; p++) kp.pre[p + 1] = kp.pre[p] + kp.norb[p] * bpo;
  for (int p = np; p < 8; p++) kp.pre[p + 1] = kp.pre[p];
  if (kp.pre[np] == 0) return SPINSUM_OK;
  if (kp.pre[np] > 0x7FFFFFFFLL) return fail(SPINSUM_ERR_UNSUPPORTED, "problem too large for one launch");
  kp.status = status_ptr();
  cudaError_t e = launch_pack(d, kp, unpack, dtype == SPINSUM_F64, vec, st);
  t_launches++;
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SPINSUM_OK;
}

int run(const Request& r, cudaStream_t st) {
  t_err.clear();
  Launch L;
  int rc = plan_one(r, &L);
  if (rc != SPINSUM_OK || L.empty) return rc;
  L.kp.status = status_ptr();
  cudaError_t e = L.kernel == 0   ? launch_k1(r.d, L.kp, L.ar, L.vec, st)
                  : L.kernel == 2 ? launch_k1t(r.d, L.kp, L.ar, st)
                  : L.kernel == 3 ? launch_k2(r.d, L.kp, L.ar, st)
                                  : launch_kg(r.d, L.kp, L.ar, st);
  t_launches++;
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SPINSUM_OK;
}

// The summation fused into a contraction over the permuted group:
// C[s, y] = sum_t S(A)[s, t] W[y, t] (coef == NULL: sum_t A[s, t] W[y, t]).
int run_contract(int d, const int64_t* ext, const void* A, const double* coef, int nfactors, int mode, const void* W,
                 int64_t Y, int64_t ldw, void* C, int64_t ldc, cudaStream_t st) {
  t_err.clear();
  if (d < 2 || d > 4) return fail(SPINSUM_ERR_ARG, "d must be 2, 3 or 4");
  if (!ext) return fail(SPINSUM_ERR_ARG, "null extent array");
  if (Y < 0) return fail(SPINSUM_ERR_ARG, "negative Y");
  if (mode & ~(SPINSUM_FACTORIZED | SPINSUM_ADJOINT | SPINSUM_STRICT))
    return fail(SPINSUM_ERR_ARG, "unknown mode bits 0x%x for a contraction", mode);
  int64_t ld[8], total = 1;
  for (int k = 0; k < 2 * d; k++) {
    if (ext[k] < 0) return fail(SPINSUM_ERR_ARG, "negative extent at index %d", k);
    ld[k] = total;
    total *= ext[k];
  }
  int64_t S = 1, T = 1;
  for (int k = 0; k < d; k++) S *= ext[k];
  for (int k = d; k < 2 * d; k++) T *= ext[k];
  if (ldw < std::max<int64_t>(Y, 1)) return fail(SPINSUM_ERR_ARG, "ldw below Y");
  if (ldc < std::max<int64_t>(S, 1)) return fail(SPINSUM_ERR_ARG, "ldc below the spectator block");
  if (S == 0 || Y == 0) return SPINSUM_OK;
  if (!C || (T > 0 && (!W || !A))) return fail(SPINSUM_ERR_ARG, "null pointer");
  if ((uintptr_t)A % 8 || (uintptr_t)W % 8 || (uintptr_t)C % 8) return fail(SPINSUM_ERR_ARG, "misaligned pointer");
  // C is written while A and W are read: no overlap
  const uintptr_t c0 = (uintptr_t)C, c1 = c0 + (uintptr_t)(((Y - 1) * ldc + S) * 8);
  const uintptr_t a0 = (uintptr_t)A, a1 = a0 + (uintptr_t)(total * 8);
  const uintptr_t w0 = (uintptr_t)W, w1 = w0 + (uintptr_t)(T > 0 ? ((T - 1) * ldw + Y) * 8 : 0);
  if ((T > 0 && c0 < a1 && a0 < c1) || (T > 0 && c0 < w1 && w0 < c1))
    return fail(SPINSUM_ERR_ALIAS, "C overlaps A or W");
  // the summation's arithmetic and orbit tables, planned as an in-place call
  // on A (nothing is written to A)
  const bool sum = coef != nullptr;
  double ident[24] = {1.0};
  Request r{d, SPINSUM_F64, ext, T > 0 ? A : C, ld, T > 0 ? const_cast<void*>(A) : C, ld, sum ? coef : ident,
            sum ? nfactors : 1, sum ? mode : 0, 1.0, 0.0, 1};
  Launch L;
  if (T > 0) {
    const int rc = plan_one(r, &L);
    if (rc != SPINSUM_OK) return rc;
  } else {
    memset(&L.kp, 0, sizeof L.kp);
    L.kp.S = S;
    L.kp.O = (int)ext[d];
  }
  L.kp.S = S;
  L.kp.status = status_ptr();
  if ((Y + 3) / 4 > 65535) return fail(SPINSUM_ERR_UNSUPPORTED, "Y too large for one launch");
  cudaError_t e = launch_kc(d, L.kp, L.ar, sum, static_cast<const double*>(W), Y, ldw, static_cast<double*>(C), ldc, st);
  t_launches++;
  if (e != cudaSuccess) return cuda_fail(e, "contraction kernel launch");
  return SPINSUM_OK;
}

}  // namespace

extern "C" {

int spinsum_contract(int d, const int64_t ext[], const void* A, const double* coef, int nfactors, int mode,
                     const void* W, int64_t Y, int64_t ldw, void* C, int64_t ldc, spinsum_stream_t stream) {
  return run_contract(d, ext, A, coef, nfactors, mode, W, Y, ldw, C, ldc, (cudaStream_t)stream);
}

int spinsum_unpack(int d, int dtype, const int64_t ext[], const void* P, const int64_t ldp[], void* B,
                   const int64_t ldb[], spinsum_stream_t stream) {
  return run_pack(true, d, dtype, ext, P, ldp, B, ldb, (cudaStream_t)stream);
}

int spinsum_pack(int d, int dtype, const int64_t ext[], const void* B, const int64_t ldb[], void* P,
                 const int64_t ldp[], spinsum_stream_t stream) {
  return run_pack(false, d, dtype, ext, P, ldp, B, ldb, (cudaStream_t)stream);
}

int spinsum_2d(int dtype, const int64_t ext[4], const void* A, const int64_t lda[4], void* B,
               const int64_t ldb[4], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream) {
  Request r{2, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run(r, (cudaStream_t)stream);
}

int spinsum_3d(int dtype, const int64_t ext[6], const void* A, const int64_t lda[6], void* B,
               const int64_t ldb[6], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream) {
  Request r{3, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run(r, (cudaStream_t)stream);
}

int spinsum_4d(int dtype, const int64_t ext[8], const void* A, const int64_t lda[8], void* B,
               const int64_t ldb[8], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream) {
  Request r{4, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run(r, (cudaStream_t)stream);
}

int spinsum_check_status(spinsum_stream_t stream) {
  t_err.clear();
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int st = 0;
  e = read_and_clear_status(&st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
  if (st == 1) return fail(SPINSUM_ERR_TIMEOUT, "a device-side bounded wait ran out");
  if (st != 0) return fail(SPINSUM_ERR_DEVICE, "device status %d", st);
  return SPINSUM_OK;
}

const char* spinsum_last_error(void) { return t_err.c_str(); }

int64_t spinsum_launch_count(int reset) {
  int64_t v = t_launches;
  if (reset) t_launches = 0;
  return v;
}

const char* spinsum_version(void) { return "spinsum-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// host-resident tensors: the summation of a column-major host tensor, in
// chunks along the slowest spectator index; each chunk is copied in (one 2D
// copy: a row per permuted tuple), summed on the device and copied out, on
// three internal streams so that copy-in, compute and copy-out of successive
// chunks overlap. The device memory is the caller's workspace.
// ---------------------------------------------------------------------------
namespace {

struct HostPipe {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};   // copy-in, compute, copy-out
  std::vector<cudaEvent_t> ev;                       // per slot: in, done, free
  cudaEvent_t start = nullptr, end = nullptr;
};

int host_pipe(HostPipe** out) {
  static HostPipe pipes[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(SPINSUM_ERR_UNSUPPORTED, "device index above 63");
  HostPipe& P = pipes[dev];
  if (!P.s[0]) {
    for (auto& st : P.s)
      if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "creating the pipeline streams");
    if ((e = cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&P.end, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "creating the pipeline events");
  }
  *out = &P;
  return SPINSUM_OK;
}

int run_host(const Request& r, void* ws, size_t ws_bytes, cudaStream_t user) {
  t_err.clear();
  const int d = r.d;
  if (d < 2 || d > 4) return fail(SPINSUM_ERR_ARG, "d must be 2, 3 or 4");
  if (!r.ext || !r.lda || !r.ldb) return fail(SPINSUM_ERR_ARG, "null extent or stride array");
  if (r.dtype != SPINSUM_F64 && r.dtype != SPINSUM_F32) return fail(SPINSUM_ERR_ARG, "unknown dtype %d", r.dtype);
  const size_t es = r.dtype == SPINSUM_F64 ? 8 : 4;
  const int nidx = 2 * d;
  int64_t total = 1, dense[8];
  for (int k = 0; k < nidx; k++) {
    if (r.ext[k] < 0) return fail(SPINSUM_ERR_ARG, "negative extent at index %d", k);
    dense[k] = total;
    total *= r.ext[k];
  }
  if (total == 0) return SPINSUM_OK;
  for (int k = 0; k < nidx; k++)
    if ((r.ext[k] > 1 && r.lda[k] != dense[k]) || (r.ext[k] > 1 && r.ldb[k] != dense[k]))
      return fail(SPINSUM_ERR_UNSUPPORTED, "host tensors must be dense column-major");
  if (!r.A || !r.B) return fail(SPINSUM_ERR_ARG, "null tensor pointer");
  if (r.inplace && r.A != r.B) return fail(SPINSUM_ERR_ALIAS, "inplace requires A == B");
  if (!r.inplace) {
    const uintptr_t a0 = (uintptr_t)r.A, b0 = (uintptr_t)r.B, n = (uintptr_t)(total * es);
    if (a0 < b0 + n && b0 < a0 + n) return fail(SPINSUM_ERR_ALIAS, "A and B overlap (use inplace = 1 for A == B)");
  }
  // page-locked host memory mapped into the device address space: the orbit
  // kernel reads A and writes B in place over the host link (zero-copy), in
  // one launch that streams both directions at once
  {
    cudaPointerAttributes pa, pb;
    if (cudaPointerGetAttributes(&pa, r.A) == cudaSuccess && cudaPointerGetAttributes(&pb, r.B) == cudaSuccess &&
        pa.type == cudaMemoryTypeHost && pb.type == cudaMemoryTypeHost && pa.devicePointer && pb.devicePointer) {
      Request q = r;
      q.A = pa.devicePointer;
      q.B = pb.devicePointer;
      return run(q, user);
    }
    cudaGetLastError();  // clear a sticky "invalid value" from probing pageable memory
  }
  if (!ws) return fail(SPINSUM_ERR_ARG, "null workspace");
  // chunk = a range of the slowest spectator index; three slots, each with the
  // A chunk (summed in place on the device) and, when beta != 0 out of place,
  // the B chunk
  const int64_t slow = r.ext[d - 1];
  const int64_t inner = dense[d - 1];            // spectator elements per slow index value
  const int64_t rows = total / (inner * slow);   // permuted tuples
  const int per_slot = (r.beta != 0.0 && !r.inplace) ? 2 : 1;
  const int64_t slice_bytes = inner * rows * (int64_t)es * per_slot;
  int64_t delta = (int64_t)(ws_bytes / 3) / std::max<int64_t>(1, slice_bytes);
  if (delta < 1) return fail(SPINSUM_ERR_ARG, "workspace too small: at least %lld bytes", (long long)(3 * slice_bytes));
  delta = std::min(delta, std::max<int64_t>(1, (slow + 7) / 8));   // at least ~8 chunks to overlap
  const int64_t nchunks = (slow + delta - 1) / delta;
  const size_t slot_bytes = (size_t)(delta * slice_bytes);
  HostPipe* P = nullptr;
  int rc = host_pipe(&P);
  if (rc != SPINSUM_OK) return rc;
  while (P->ev.size() < 9) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "creating the pipeline events");
    P->ev.push_back(ev);
  }
  cudaError_t e = cudaEventRecord(P->start, user);
  for (int k = 0; k < 3 && e == cudaSuccess; k++) e = cudaStreamWaitEvent(P->s[k], P->start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "ordering after the caller's stream");
  const unsigned char* hA = static_cast<const unsigned char*>(r.A);
  unsigned char* hB = static_cast<unsigned char*>(r.B);
  const size_t pitch = (size_t)(inner * slow) * es;
  for (int64_t c = 0; c < nchunks; c++) {
    const int slot = (int)(c % 3);
    const int64_t c0 = c * delta, dc = std::min(delta, slow - c0);
    const size_t width = (size_t)(inner * dc) * es;
    unsigned char* dA = static_cast<unsigned char*>(ws) + slot * slot_bytes;
    unsigned char* dB = per_slot == 2 ? dA + slot_bytes / 2 : dA;
    cudaEvent_t ev_in = P->ev[slot * 3], ev_done = P->ev[slot * 3 + 1], ev_free = P->ev[slot * 3 + 2];
    if (c >= 3 && (e = cudaStreamWaitEvent(P->s[0], ev_free, 0)) != cudaSuccess) break;
    e = cudaMemcpy2DAsync(dA, width, hA + (size_t)(c0 * inner) * es, pitch, width, (size_t)rows,
                          cudaMemcpyHostToDevice, P->s[0]);
    if (e == cudaSuccess && per_slot == 2)
      e = cudaMemcpy2DAsync(dB, width, hB + (size_t)(c0 * inner) * es, pitch, width, (size_t)rows,
                            cudaMemcpyHostToDevice, P->s[0]);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, P->s[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s[1], ev_in, 0);
    if (e != cudaSuccess) break;
    // the chunk as a dense device tensor: slow spectator extent dc
    int64_t cext[8], cld[8], s1 = 1;
    for (int k = 0; k < nidx; k++) {
      cext[k] = (k == d - 1) ? dc : r.ext[k];
      cld[k] = s1;
      s1 *= cext[k];
    }
    Request q = r;
    q.ext = cext;
    q.lda = cld;
    q.ldb = cld;
    q.A = dA;
    q.B = dB;
    q.inplace = per_slot == 1;
    rc = run(q, P->s[1]);
    if (rc != SPINSUM_OK) return rc;
    if ((e = cudaEventRecord(ev_done, P->s[1])) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(P->s[2], ev_done, 0)) != cudaSuccess) break;
    e = cudaMemcpy2DAsync(hB + (size_t)(c0 * inner) * es, pitch, dB, width, width, (size_t)rows,
                          cudaMemcpyDeviceToHost, P->s[2]);
    if (e == cudaSuccess) e = cudaEventRecord(ev_free, P->s[2]);
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "host pipeline");
  for (int k = 0; k < 3 && e == cudaSuccess; k++) {
    e = cudaEventRecord(P->end, P->s[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, P->end, 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ordering the caller's stream after the pipeline");
  return SPINSUM_OK;
}

}  // namespace

extern "C" {

int spinsum_2d_host(int dtype, const int64_t ext[4], const void* A, const int64_t lda[4], void* B,
                    const int64_t ldb[4], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream) {
  Request r{2, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run_host(r, workspace, workspace_bytes, (cudaStream_t)stream);
}

int spinsum_3d_host(int dtype, const int64_t ext[6], const void* A, const int64_t lda[6], void* B,
                    const int64_t ldb[6], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream) {
  Request r{3, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run_host(r, workspace, workspace_bytes, (cudaStream_t)stream);
}

int spinsum_4d_host(int dtype, const int64_t ext[8], const void* A, const int64_t lda[8], void* B,
                    const int64_t ldb[8], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream) {
  Request r{4, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace};
  return run_host(r, workspace, workspace_bytes, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched plans: problems grouped by (d, arithmetic); each class runs as one
// persistent launch of the batched kernel over its problems' K1 blocks.
// Problems whose layout needs the general kernel are launched one by one.
// ---------------------------------------------------------------------------
namespace ss {
cudaError_t launch_kb(int d, int ar, const KParams* probs, const int64_t* prefix, const int* vecs, int n, unsigned long long* ctr, int grid,
                      cudaStream_t st, const void** fn);
}

namespace {

// K1 blocks of one problem for a given number of chunks per block
void set_cpb(KParams& kp, int d, int cpb) {
  kp.cpb = (int)std::max<int64_t>(1, std::min<int64_t>(cpb, kp.nchunk));
  const int64_t bpo = (kp.nchunk + kp.cpb - 1) / kp.cpb;
  const int np = npatterns(d);
  kp.pre[0] = 0;
  for (int p = 0; p < np; p++) kp.pre[p + 1] = kp.pre[p] + kp.norb[p] * bpo;
  for (int p = np; p < 8; p++) kp.pre[p + 1] = kp.pre[p];
}

// a batch image in host memory (same layout as the device copy)
struct BatchLayout {
  KParams* probs;
  int64_t* prefix;
  int* vec;
};

struct ClassRange {
  int d, ar, first, pfirst, n;
  int64_t blocks;
};

// bytes and field offsets of an image for n problems
struct ImageShape {
  size_t probs, prefix, vec, ctr, bytes;
};
ImageShape image_shape(int n) {
  return ImageShape{batch_offset_probs(n), batch_offset_prefix(n), batch_offset_vec(n), batch_offset_ctr(n),
                    batch_image_bytes(n)};
}

// Fill the image with the K1-capable launches in the given order, grouped by
// class, each with K1 chunking and `cpb` chunks per block (cpb <= 0: the
// single-call heuristic of 8192 positions per block).
std::vector<ClassRange> fill_batch(const std::vector<Launch>& ls, const std::vector<int>& order, int cpb,
                                   BatchLayout out, int* status) {
  std::vector<ClassRange> cls;
  int next = 0, pnext = 0;
  for (int d : {2, 3, 4})
    for (int ar : {(int)AR_EXACT, (int)AR_STRICT, (int)AR_F32}) {
      ClassRange c{d, ar, next, pnext, 0, 0};
      for (int i : order) {
        const Launch& L = ls[i];
        if (L.kernel == 1 || L.kernel == 3 || L.kp.nspec != d || L.ar != ar) continue;
        KParams kp = L.kp;
        kp.status = status;
        const int vec = (L.vec > 1 && !(d == 4 && L.ar == AR_F32)) ? L.vec : 1;
        kp.nchunk = (kp.S + 256LL * vec - 1) / (256LL * vec);
        set_cpb(kp, d, cpb > 0 ? cpb : (int)std::max<int64_t>(1, 8192 / (256LL * vec)));
        out.probs[next] = kp;
        out.vec[next] = vec;
        out.prefix[pnext + c.n] = c.blocks;
        c.blocks += kp.pre[npatterns(d)];
        next++;
        c.n++;
      }
      if (c.n == 0) continue;
      out.prefix[pnext + c.n] = c.blocks;
      pnext += c.n + 1;
      cls.push_back(c);
    }
  return cls;
}

int64_t problem_bytes(const Launch& L) {
  int64_t n = L.kp.S;
  for (int k = 0; k < L.kp.nspec; k++) n *= L.kp.O;
  return n;
}

}  // namespace

struct spinsum_plan {
  int device = 0;
  int dtype = SPINSUM_F64;
  std::vector<Launch> launches;      // one per non-empty problem
  std::vector<int> general;          // problems run by the general kernel
  std::vector<ClassRange> classes;
  std::vector<int> grid;             // per class
  unsigned char* d_image = nullptr;  // device copy of the batch image (owned)
  ImageShape shape{};
  int cpb_scale = 3;                 // chunks per block = 2^cpb_scale
  int order = 0;                     // 0 as given, 1 largest problems first
  int occ = 1;                       // grid = SMs * max blocks per SM / occ
  std::string desc;
};

namespace {

int plan_build(spinsum_plan* P, int cpb_scale, int order, int occ, cudaStream_t st) {
  const int n = (int)P->launches.size();
  std::vector<int> idx(n);
  for (int i = 0; i < n; i++) idx[i] = i;
  if (order == 1)
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return problem_bytes(P->launches[a]) > problem_bytes(P->launches[b]); });
  std::vector<unsigned char> img(P->shape.bytes, 0);
  BatchLayout lay{reinterpret_cast<KParams*>(img.data() + P->shape.probs),
                  reinterpret_cast<int64_t*>(img.data() + P->shape.prefix),
                  reinterpret_cast<int*>(img.data() + P->shape.vec)};
  P->classes = fill_batch(P->launches, idx, 1 << cpb_scale, lay, status_ptr());
  cudaError_t e = cudaMemcpyAsync(P->d_image, img.data(), img.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "uploading the plan");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  P->grid.clear();
  for (const ClassRange& c : P->classes) {
    const void* fn = nullptr;
    launch_kb(c.d, c.ar, nullptr, nullptr, nullptr, 0, nullptr, 0, st, &fn);
    int nb = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    const int64_t full = (int64_t)sms * std::max(1, nb) / occ;
    P->grid.push_back((int)std::max<int64_t>(1, std::min<int64_t>(c.blocks, full)));
  }
  P->cpb_scale = cpb_scale;
  P->order = order;
  P->occ = occ;
  return SPINSUM_OK;
}

int plan_launch(spinsum_plan* P, cudaStream_t st) {
  const KParams* probs = reinterpret_cast<const KParams*>(P->d_image + P->shape.probs);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(P->d_image + P->shape.prefix);
  const int* vec = reinterpret_cast<const int*>(P->d_image + P->shape.vec);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(P->d_image + P->shape.ctr);
  for (size_t k = 0; k < P->classes.size(); k++) {
    const ClassRange& c = P->classes[k];
    cudaError_t e = launch_kb(c.d, c.ar, probs + c.first, prefix + c.pfirst, vec + c.first, c.n, ctr + 2 * k,
                              P->grid[k], st, nullptr);
    t_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
  }
  for (int i : P->general) {
    Launch L = P->launches[i];
    L.kp.status = status_ptr();
    cudaError_t e = L.kernel == 3 ? launch_k2(L.kp.nspec, L.kp, L.ar, st) : launch_kg(L.kp.nspec, L.kp, L.ar, st);
    t_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "general kernel launch");
  }
  return SPINSUM_OK;
}

// autotune cache: key -> (cpb_scale, order, occ); kept for the process, and
// in the file named by SPINSUM_AUTOTUNE_CACHE when set
std::string tune_key(const spinsum_plan* P) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, P->device);
  std::string k = std::string(prop.name) + "|dt" + std::to_string(P->dtype);
  for (const Launch& L : P->launches) {
    char buf[96];
    snprintf(buf, sizeof buf, "|%d:%lld:%d:%d:%d", L.kp.nspec, (long long)L.kp.S, L.kp.O, L.ar, L.vec);
    k += buf;
  }
  return k;
}

std::vector<std::pair<std::string, std::array<int, 3>>>& tune_cache() {
  static std::vector<std::pair<std::string, std::array<int, 3>>> c;
  static bool loaded = false;
  if (!loaded) {
    loaded = true;
    if (const char* f = getenv("SPINSUM_AUTOTUNE_CACHE")) {
      if (FILE* fp = fopen(f, "r")) {
        char line[8192];
        while (fgets(line, sizeof line, fp)) {
          char* tab = strrchr(line, '\t');
          if (!tab) continue;
          *tab = 0;
          int a, b, cc;
          if (sscanf(tab + 1, "%d %d %d", &a, &b, &cc) == 3) c.push_back({line, {a, b, cc}});
        }
        fclose(fp);
      }
    }
  }
  return c;
}

void tune_store(const std::string& key, int a, int b, int c) {
  tune_cache().push_back({key, {a, b, c}});
  if (const char* f = getenv("SPINSUM_AUTOTUNE_CACHE")) {
    if (FILE* fp = fopen(f, "a")) {
      fprintf(fp, "%s\t%d %d %d\n", key.c_str(), a, b, c);
      fclose(fp);
    }
  }
}

void plan_free(spinsum_plan* P) {
  if (P->d_image) cudaFree(P->d_image);
  P->d_image = nullptr;
}

}  // namespace

extern "C" {

int spinsum_plan_create(spinsum_plan** plan, const spinsum_problem* problems, int nproblems, int dtype,
                        int allow_tuning_runs, spinsum_stream_t stream) {
  t_err.clear();
  if (!plan) return fail(SPINSUM_ERR_ARG, "null plan pointer");
  *plan = nullptr;
  if (nproblems < 0 || (nproblems > 0 && !problems)) return fail(SPINSUM_ERR_ARG, "bad problem list");
  cudaStream_t st = (cudaStream_t)stream;
  auto* P = new spinsum_plan();
  P->dtype = dtype;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) { delete P; return cuda_fail(e, "cudaGetDevice"); }
  for (int i = 0; i < nproblems; i++) {
    const spinsum_problem& q = problems[i];
    Request r{q.d, dtype, q.ext, q.A, q.lda, q.B, q.ldb, q.coef, q.nfactors, q.mode & ~SPINSUM_TMA, q.alpha,
              q.beta, q.inplace};
    Launch L;
    int rc = plan_one(r, &L);
    if (rc != SPINSUM_OK) {
      std::string m = "problem " + std::to_string(i) + ": " + t_err;
      delete P;
      return fail(rc, "%s", m.c_str());
    }
    if (L.empty) continue;
    if (L.kernel == 1 || L.kernel == 3) P->general.push_back((int)P->launches.size());
    P->launches.push_back(L);
  }
  P->shape = image_shape((int)P->launches.size());
  e = cudaMalloc(&P->d_image, std::max<size_t>(P->shape.bytes, 16));
  if (e != cudaSuccess) { delete P; return cuda_fail(e, "allocating the plan image"); }
  int best[3] = {3, 0, 1};
  const std::string key = tune_key(P);
  bool cached = false;
  for (auto& kv : tune_cache())
    if (kv.first == key) {
      best[0] = kv.second[0]; best[1] = kv.second[1]; best[2] = kv.second[2];
      cached = true;
    }
  const bool any_k1 = P->general.size() < P->launches.size();
  if (!cached && allow_tuning_runs && any_k1) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int cs = 0; cs <= 5; cs++)
      for (int order = 0; order <= 1; order++)
        for (int occ = 1; occ <= 2; occ++) {
          int rc = plan_build(P, cs, order, occ, st);
          if (rc != SPINSUM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); plan_free(P); delete P; return rc; }
          float ms = 1e30f;
          for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, st);
            rc = plan_launch(P, st);
            cudaEventRecord(e1, st);
            if (rc != SPINSUM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); plan_free(P); delete P; return rc; }
            cudaEventSynchronize(e1);
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
          }
          if (ms < best_ms) { best_ms = ms; best[0] = cs; best[1] = order; best[2] = occ; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, best[0], best[1], best[2]);
  }
  int rc = plan_build(P, best[0], best[1], best[2], st);
  if (rc != SPINSUM_OK) { plan_free(P); delete P; return rc; }
  char buf[256];
  int64_t blocks = 0;
  for (auto& c : P->classes) blocks += c.blocks;
  snprintf(buf, sizeof buf,
           "problems=%zu classes=%zu general=%zu blocks=%lld chunks_per_block=%d order=%s occupancy=1/%d%s",
           P->launches.size(), P->classes.size(), P->general.size(), (long long)blocks, 1 << best[0],
           best[1] ? "largest-first" : "as-given", best[2],
           cached ? " (cached)" : (allow_tuning_runs ? " (tuned)" : " (heuristic)"));
  P->desc = buf;
  *plan = P;
  return SPINSUM_OK;
}

int spinsum_plan_execute(spinsum_plan* plan, spinsum_stream_t stream) {
  t_err.clear();
  if (!plan) return fail(SPINSUM_ERR_ARG, "null plan");
  return plan_launch(plan, (cudaStream_t)stream);
}

int spinsum_plan_destroy(spinsum_plan* plan) {
  t_err.clear();
  if (!plan) return SPINSUM_OK;
  plan_free(plan);
  delete plan;
  return SPINSUM_OK;
}

const char* spinsum_plan_describe(const spinsum_plan* plan) { return plan ? plan->desc.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// spinsum_batch_static: the batched kernel with its image in the library's
// fixed device array (ss_static.cu) instead of plan memory. Nothing is
// allocated: the image is built on the host, copied into the array with
// cudaMemcpyAsync on the caller's stream, and the kernels read it there.
// ---------------------------------------------------------------------------
extern "C" int spinsum_batch_static(const spinsum_problem* problems, int nproblems, int dtype,
                                    spinsum_stream_t stream) {
  t_err.clear();
  if (nproblems < 0 || (nproblems > 0 && !problems)) return fail(SPINSUM_ERR_ARG, "bad problem list");
  if (nproblems > SPINSUM_STATIC_MAX_PROBLEMS)
    return fail(SPINSUM_ERR_ARG, "spinsum_batch_static takes at most %d problems (got %d)",
                SPINSUM_STATIC_MAX_PROBLEMS, nproblems);
  cudaStream_t st = (cudaStream_t)stream;
  // the parameter upload below reads a host buffer that lives only for this
  // call, so a capturing stream (whose graph would read it at replay) is refused
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "querying the stream's capture status");
    if (cs != cudaStreamCaptureStatusNone)
      return fail(SPINSUM_ERR_ARG, "spinsum_batch_static does not run on a stream that is being captured");
  }
  std::vector<Launch> launches;
  for (int i = 0; i < nproblems; i++) {
    const spinsum_problem& q = problems[i];
    Request r{q.d, dtype, q.ext, q.A, q.lda, q.B, q.ldb, q.coef, q.nfactors, q.mode & ~SPINSUM_TMA, q.alpha,
              q.beta, q.inplace};
    Launch L;
    int rc = plan_one(r, &L);
    if (rc != SPINSUM_OK) {
      std::string m = "problem " + std::to_string(i) + ": " + t_err;
      return fail(rc, "%s", m.c_str());
    }
    if (!L.empty) launches.push_back(L);
  }
  if (launches.empty()) return SPINSUM_OK;
  void* dimg = nullptr;
  cudaError_t e = static_scratch_ptr(&dimg);
  if (e != cudaSuccess) return cuda_fail(e, "looking up the static scratch array");
  const int nmax = SPINSUM_STATIC_MAX_PROBLEMS;
  const ImageShape sh = image_shape(nmax);
  std::vector<unsigned char> img(sh.bytes, 0);
  BatchLayout lay{reinterpret_cast<KParams*>(img.data() + sh.probs), reinterpret_cast<int64_t*>(img.data() + sh.prefix),
                  reinterpret_cast<int*>(img.data() + sh.vec)};
  std::vector<int> order(launches.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
  const std::vector<ClassRange> cls = fill_batch(launches, order, 0, lay, status_ptr());
  if (!cls.empty()) {
    // only the entries the kernels read: the parameters and vector widths of
    // the n problems and the class prefix segments (n + classes entries); the
    // rest of the array keeps whatever an earlier call left there
    const ClassRange& last = cls.back();
    const size_t n = (size_t)(last.first + last.n), np = (size_t)(last.pfirst + last.n + 1);
    const size_t parts[3][2] = {{sh.probs, n * sizeof(KParams)}, {sh.prefix, np * sizeof(int64_t)},
                                {sh.vec, n * sizeof(int)}};
    for (const auto& pt : parts) {
      e = cudaMemcpyAsync(static_cast<unsigned char*>(dimg) + pt[0], img.data() + pt[0], pt[1],
                          cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "uploading the batch parameters");
    }
  }
  const unsigned char* base = static_cast<const unsigned char*>(dimg);
  const KParams* probs = reinterpret_cast<const KParams*>(base + sh.probs);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(base + sh.prefix);
  const int* vec = reinterpret_cast<const int*>(base + sh.vec);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(dimg) + sh.ctr);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (size_t k = 0; k < cls.size(); k++) {
    const ClassRange& c = cls[k];
    const void* fn = nullptr;
    launch_kb(c.d, c.ar, nullptr, nullptr, nullptr, 0, nullptr, 0, st, &fn);
    int nb = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(c.blocks, (int64_t)sms * std::max(1, nb)));
    e = launch_kb(c.d, c.ar, probs + c.first, prefix + c.pfirst, vec + c.first, c.n, ctr + 2 * k, grid, st, nullptr);
    t_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "static batched kernel launch");
  }
  for (const Launch& L : launches) {
    if (L.kernel != 1 && L.kernel != 3) continue;
    KParams kp = L.kp;
    kp.status = status_ptr();
    e = L.kernel == 3 ? launch_k2(kp.nspec, kp, L.ar, st) : launch_kg(kp.nspec, kp, L.ar, st);
    t_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "general kernel launch");
  }
  return SPINSUM_OK;
}

// ---------------------------------------------------------------------------
// Planner introspection for host-side tests (not part of the public ABI):
// plans a d-dimensional problem with permuted extent O and spectator extent V
// (fake device addresses, nothing is launched) and reports the expanded
// coefficients, the arithmetic choice and the launch shape.
// info: [arith, W, kdrop, nstage, kernel, vec, flags, cexp, emin>>20, emax>>20,
//        norb[0..7], blocks]
// ---------------------------------------------------------------------------
extern "C" int ss_debug_plan(int d, int O, int V, const double* coef, int nfactors, int mode, double alpha,
                             double beta, double* expanded, int64_t* info, int* ci, int* mp) {
  int64_t ext[8], ld[8];
  int64_t s = 1;
  for (int k = 0; k < 2 * d; k++) {
    ext[k] = k < d ? V : O;
    ld[k] = s;
    s *= ext[k];
  }
  Request r{d, SPINSUM_F64, ext, (const void*)0x100000, ld, (void*)(0x100000 + 8 * s + 4096), ld,
            coef, nfactors, mode, alpha, beta, 0};
  Launch L;
  int rc = plan_one(r, &L);
  if (rc != SPINSUM_OK) return rc;
  const Group& g = group(d);
  std::vector<std::vector<double>> chain(nfactors, std::vector<double>(g.n));
  for (int f = 0; f < nfactors; f++)
    for (int x = 0; x < g.n; x++) chain[f][x] = coef[f * g.n + x];
  std::vector<double> full = expand_chain(g, chain);
  for (int x = 0; x < g.n; x++) expanded[x] = full[x];
  const KParams& kp = L.kp;
  int64_t v[32] = {L.ar, kp.W, kp.kdrop, kp.nstage, L.kernel, L.vec, kp.flags, kp.cexp, (int64_t)(kp.emin >> 20),
                   (int64_t)(kp.emax >> 20)};
  for (int p = 0; p < 8; p++) v[10 + p] = kp.norb[p];
  v[18] = L.kernel == 1 ? (kp.ngroup + 255) / 256 : kp.pre[npatterns(d)];
  v[19] = L.kernel == 3 ? kp.k2lf : 0;
  for (int k = 0; k < 20; k++) info[k] = v[k];
  for (int st = 0; st < MAXSTAGE; st++)
    for (int x = 0; x < 24; x++) ci[st * 24 + x] = kp.ci[st][x];
  for (int k = 0; k < MP_MAX; k++) mp[k] = kp.mp[k];
  return SPINSUM_OK;
}

// Planner introspection for host-side tests (not part of the public ABI): the
// Klein four-group tables of 4D pattern P as
// [ok, m, nb, orb[6][4], nnz[24], col[24][6], woff[25]] (223 ints), and, for a
// planned d = 4 problem (as ss_debug_plan), [flags, W, kdrop] and the wh
// weights (WH_TOTAL ints).
extern "C" int ss_debug_wht_tables(int P, int* out) {
  if (P < 0 || P >= 8) return SPINSUM_ERR_ARG;
  const Wht4& w = host_wht4()[P];
  int k = 0;
  out[k++] = w.ok;
  out[k++] = w.m;
  out[k++] = w.nb;
  for (int o = 0; o < 6; o++)
    for (int vi = 0; vi < 4; vi++) out[k++] = w.orb[o][vi];
  for (int i = 0; i < 24; i++) out[k++] = w.nnz[i];
  for (int i = 0; i < 24; i++)
    for (int q = 0; q < 6; q++) out[k++] = w.col[i][q];
  for (int i = 0; i < 25; i++) out[k++] = w.woff[i];
  return SPINSUM_OK;
}

extern "C" int ss_debug_plan_wh(int O, int V, const double* coef, int nfactors, int mode, double alpha, double beta,
                                int64_t* info, int* wh) {
  int64_t ext[8], ld[8];
  int64_t s = 1;
  for (int k = 0; k < 8; k++) {
    ext[k] = k < 4 ? V : O;
    ld[k] = s;
    s *= ext[k];
  }
  Request r{4, SPINSUM_F64, ext, (const void*)0x100000, ld, (void*)(0x100000 + 8 * s + 4096), ld,
            coef, nfactors, mode, alpha, beta, 0};
  Launch L;
  int rc = plan_one(r, &L);
  if (rc != SPINSUM_OK) return rc;
  info[0] = L.kp.flags;
  info[1] = L.kp.W;
  info[2] = L.kp.kdrop;
  info[3] = L.ar;
  for (int k = 0; k < WH_TOTAL; k++) wh[k] = L.kp.wh[k];
  return SPINSUM_OK;
}
