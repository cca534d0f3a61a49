// The paper's Algorithm 2 (Sec. 4.2): temporal locality in A and B, the
// spin summation of the NCC quantum-chemistry code that the paper measures
// its blocked algorithm against. See spinsum_alg6.h for the operation and the
// rounding order.
//
// Structure: the loops run over the sorted tuples t0 = (i_1 <= ... <= i_d)
// only (the tetrahedral iteration space); for each t0 the innermost loop
// visits the distinct rearrangements t = t0 o tau (every member of the
// element orbit once; repeated indices drop the duplicate updates) and
// computes B[t] = sum_sigma a_sigma A[t o sigma]. All d! outputs of the orbit
// read the same m <= d! elements of A, so each element of A is loaded once
// and reused for every update of its orbit (the temporal locality of the
// algorithm's name), while consecutive orbits touch scattered cache lines (no
// spatial locality: that is what the blocked algorithm adds). The outermost
// index is split cyclically over the threads, as the paper's
// "omp parallel for schedule(static, 1)" does. A factor chain is applied as
// its expanded product (one stage). In place is safe: an orbit's outputs are
// formed in registers before any of them is stored.
#include "spinsum_alg6.h"

#include <array>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

namespace {

constexpr int kD = 4;
constexpr int kN = 24;

struct Perms {
  int n = 0;
  int p[kN][kD] = {};
};

// S_d in lexicographic one-line order (0-based images)
Perms lex_perms(int d) {
  Perms S;
  int a[kD] = {0, 1, 2, 3};
  for (;;) {
    for (int m = 0; m < d; m++) S.p[S.n][m] = a[m];
    S.n++;
    int i = d - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) break;
    int j = d - 1;
    while (a[j] < a[i]) j--;
    std::swap(a[i], a[j]);
    for (int x = i + 1, y = d - 1; x < y; x++, y--) std::swap(a[x], a[y]);
  }
  return S;
}

// product of the chain F_1 .. F_k, (phi o psi)(m) = phi(psi(m)), each entry
// summed over (phi, psi) pairs in lexicographic order, zero terms skipped
std::vector<double> expand(const Perms& S, int d, const double* coef, int nf) {
  auto index_of = [&](const int* q) {
    for (int s = 0; s < S.n; s++) {
      bool same = true;
      for (int m = 0; m < d; m++) same = same && S.p[s][m] == q[m];
      if (same) return s;
    }
    return -1;
  };
  std::vector<double> P(coef, coef + S.n);
  for (int f = 1; f < nf; f++) {
    std::vector<double> Q(S.n, 0.0);
    const double* F = coef + f * S.n;
    for (int a = 0; a < S.n; a++) {
      if (P[a] == 0.0) continue;
      for (int b = 0; b < S.n; b++) {
        if (F[b] == 0.0) continue;
        int c[kD];
        for (int m = 0; m < d; m++) c[m] = S.p[a][S.p[b][m]];
        const int k = index_of(c);
        const double prod = P[a] * F[b];
        Q[k] = Q[k] + prod;
      }
    }
    P = Q;
  }
  return P;
}

struct Job {
  int d;
  int64_t N;
  const double* A;
  double* B;
  double alpha, beta;
  Perms S;
  std::vector<double> c;
};

// all sorted tuples with last index i_d = v, each orbit's updates in turn
void slab(const Job& jb, int64_t v) {
  const int d = jb.d;
  const int n = jb.S.n;
  int64_t pw[kD] = {1, 1, 1, 1};
  for (int m = 1; m < d; m++) pw[m] = pw[m - 1] * jb.N;
  int64_t t0[kD] = {0, 0, 0, 0};
  t0[d - 1] = v;
  for (;;) {
    // the distinct members t = t0 o tau (tau in lexicographic order)
    int64_t mem[kN][kD];
    int64_t off[kN];
    int m = 0;
    for (int s = 0; s < n; s++) {
      int64_t t[kD];
      for (int k = 0; k < d; k++) t[k] = t0[jb.S.p[s][k]];
      bool seen = false;
      for (int u = 0; u < m && !seen; u++) {
        bool same = true;
        for (int k = 0; k < d; k++) same = same && mem[u][k] == t[k];
        seen = same;
      }
      if (seen) continue;
      int64_t o = 0;
      for (int k = 0; k < d; k++) {
        mem[m][k] = t[k];
        o += t[k] * pw[k];
      }
      off[m++] = o;
    }
    // B[t] = alpha * sum_sigma a_sigma A[t o sigma] (+ beta B[t]) for every member
    double out[kN];
    for (int u = 0; u < m; u++) {
      double acc = 0.0;
      for (int s = 0; s < n; s++) {
        const double cs = jb.c[s];
        if (cs == 0.0) continue;
        int64_t o = 0;
        for (int k = 0; k < d; k++) o += mem[u][jb.S.p[s][k]] * pw[k];
        const double prod = cs * jb.A[o];
        acc = acc + prod;
      }
      out[u] = jb.alpha * acc;
    }
    for (int u = 0; u < m; u++) {
      double r = out[u];
      if (jb.beta != 0.0) {
        const double bo = jb.beta * jb.B[off[u]];
        r = r + bo;
      }
      jb.B[off[u]] = r;
    }
    // next sorted tuple i_1 <= ... <= i_(d-1) <= v
    int k = 0;
    while (k < d - 1 && t0[k] == t0[k + 1]) k++;
    if (k == d - 1) break;
    t0[k]++;
    for (int q = 0; q < k; q++) t0[q] = 0;
  }
}

}  // namespace

extern "C" int spinsum_alg2(int d, int64_t N, const double* A, double* B, const double* coef, int nfactors,
                            double alpha, double beta, int nthreads) {
  if (d < 2 || d > kD || N < 0 || nfactors < 1 || nfactors > 8 || nthreads < 0) return -1;
  if (!coef || (N > 0 && (!A || !B))) return -1;
  int64_t total = 1;
  for (int m = 0; m < d; m++) {
    if (N > 0 && total > INT64_MAX / N) return -1;
    total *= N;
  }
  if (total == 0) return 0;
  Job jb;
  jb.d = d;
  jb.N = N;
  jb.A = A;
  jb.B = B;
  jb.alpha = alpha;
  jb.beta = beta;
  jb.S = lex_perms(d);
  try {
    jb.c = expand(jb.S, d, coef, nfactors);
  } catch (const std::bad_alloc&) {
    return -2;
  }
  int nt = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > N) nt = (int)N;
  auto worker = [&jb, nt](int id) {
    for (int64_t v = id; v < jb.N; v += nt) slab(jb, v);
  };
  std::vector<std::thread> pool;
  try {
    for (int i = 1; i < nt; i++) pool.emplace_back(worker, i);
  } catch (const std::system_error&) {
    for (auto& th : pool) th.join();
    return -2;
  }
  worker(0);
  for (auto& th : pool) th.join();
  return 0;
}
