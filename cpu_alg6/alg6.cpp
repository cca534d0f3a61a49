// The paper's blocked CPU spin summation (Sec. 4.5 Algorithm 5a/5b, Sec. 4.6
// Algorithm 6) for the dense column-major N^d tensor; see spinsum_alg6.h for
// the operation, arguments and rounding order.
//
// Structure:
//  * tasks (Algorithm 5a): one per block orbit, i.e. per sorted tuple of tile
//    coordinates T_1 <= ... <= T_d; a pool of threads takes them from an
//    atomic counter (dynamic, task-based parallelism);
//  * macro-kernel (Algorithm 5b): the m_b <= d! distinct tiles T o tau of the
//    orbit are copied into a per-thread buffer; each factor stage maps one
//    buffer to the next (the auxiliary T of Algorithm 5b, d! tiles in size)
//    and the last stage writes B; in place is safe because every tile of the
//    orbit has been read before any of them is written;
//  * traversal (Algorithm 6): every output tile is visited row by row along
//    its stride-1 index i_1, so B is written contiguously, and a row's d!
//    terms are accumulated term by term over the whole row (a vectorisable
//    loop: stride 1 in the buffer for the permutations that keep i_1 in
//    place, a stride of bl^m for the ones that move it to position m).
//
// Not reproduced: the paper's x86 mechanisms (AVX transposes, non-temporal
// stores, NUMA-aware first touch); the compiler vectorises the row loops for
// the host it is built on.
#include "spinsum_alg6.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

namespace {

constexpr int kMaxD = 4;
constexpr int kMaxPerm = 24;
constexpr int kMaxBl = 64;
constexpr int kMaxFactors = 8;

using Tuple = std::array<int64_t, kMaxD>;

struct Sym {
  int n = 0;                       // d!
  int p[kMaxPerm][kMaxD] = {};     // p[s][m] = phi_s(m) (0-based images), lexicographic order
};

Sym make_sym(int d) {
  Sym S;
  int a[kMaxD];
  for (int m = 0; m < d; m++) a[m] = m;
  // lexicographic enumeration: the next permutation after a is found by the
  // longest non-increasing suffix, a swap with its smallest larger element
  // and a reversal of the suffix
  for (;;) {
    for (int m = 0; m < d; m++) S.p[S.n][m] = a[m];
    S.n++;
    int i = d - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) break;
    int j = d - 1;
    while (a[j] < a[i]) j--;
    std::swap(a[i], a[j]);
    std::reverse(a + i + 1, a + d);
  }
  return S;
}

int index_of(const Sym& S, int d, const int* q) {
  for (int s = 0; s < S.n; s++) {
    bool same = true;
    for (int m = 0; m < d; m++) same = same && S.p[s][m] == q[m];
    if (same) return s;
  }
  return -1;
}

// The product of the chain in the group algebra: applying pi_psi and then
// pi_phi is pi_{phi o psi}, so (sum a_phi pi_phi)(sum b_psi pi_psi) has
// a_phi b_psi on phi o psi; folded from F_1, products added in lexicographic
// order of phi, then psi, zero coefficients skipped.
std::vector<double> expand_chain(const Sym& S, int d, const double* coef, int nfactors) {
  std::vector<double> P(coef, coef + S.n);
  for (int f = 1; f < nfactors; f++) {
    const double* F = coef + (size_t)f * S.n;
    std::vector<double> Q(S.n, 0.0);
    for (int a = 0; a < S.n; a++) {
      if (P[a] == 0.0) continue;
      for (int b = 0; b < S.n; b++) {
        if (F[b] == 0.0) continue;
        int c[kMaxD];
        for (int m = 0; m < d; m++) c[m] = S.p[a][S.p[b][m]];
        const int k = index_of(S, d, c);
        const double prod = P[a] * F[b];
        Q[k] = Q[k] + prod;
      }
    }
    P.swap(Q);
  }
  return P;
}

struct Problem {
  int d;
  int64_t N;
  int bl;
  int64_t V;               // bl^d, the buffer size of one tile
  int64_t pw[kMaxD];       // bl^m
  int64_t gs[kMaxD];       // N^m
  const double* A;
  double* B;
  double alpha, beta;
  Sym S;
  int inv0[kMaxPerm];      // position m with phi_s(m) = 0
  std::vector<std::vector<double>> stages;  // applied in this order; the last one writes B
};

struct Buffers {
  std::vector<double> buf[3];
};

// one block orbit: sorted tile tuple T
void macro_kernel(const Problem& pb, const Tuple& T, Buffers& bf) {
  const int d = pb.d;
  const Sym& S = pb.S;
  // the distinct tiles T o tau of the orbit
  Tuple tiles[kMaxPerm];
  int nt = 0;
  for (int s = 0; s < S.n; s++) {
    Tuple t{};
    for (int m = 0; m < d; m++) t[m] = T[S.p[s][m]];
    bool seen = false;
    for (int q = 0; q < nt && !seen; q++) seen = tiles[q] == t;
    if (!seen) tiles[nt++] = t;
  }
  // source tile of term s for output tile b: (T_b o phi_s)
  int src[kMaxPerm][kMaxPerm];
  for (int b = 0; b < nt; b++)
    for (int s = 0; s < S.n; s++) {
      Tuple t{};
      for (int m = 0; m < d; m++) t[m] = tiles[b][S.p[s][m]];
      int q = 0;
      while (tiles[q] != t) q++;
      src[b][s] = q;
    }
  auto extent = [&](const Tuple& t, int m) { return std::min<int64_t>(pb.bl, pb.N - t[m] * pb.bl); };

  // copy in: the orbit's tiles, row by row
  double* L = bf.buf[0].data();
  for (int q = 0; q < nt; q++) {
    int64_t e[kMaxD] = {1, 1, 1, 1};
    for (int m = 0; m < d; m++) e[m] = extent(tiles[q], m);
    int64_t j[kMaxD] = {0, 0, 0, 0};
    for (;;) {
      int64_t g = tiles[q][0] * pb.bl, l = 0;
      for (int m = 1; m < d; m++) {
        g += (tiles[q][m] * pb.bl + j[m]) * pb.gs[m];
        l += j[m] * pb.pw[m];
      }
      const double* a = pb.A + g;
      double* o = L + q * pb.V + l;
      for (int64_t x = 0; x < e[0]; x++) o[x] = a[x];
      int m = 1;
      while (m < d && ++j[m] == e[m]) j[m++] = 0;
      if (m >= d) break;
    }
  }

  // the stages: buffer -> buffer, the last one buffer -> B
  const int nst = (int)pb.stages.size();
  int cur = 0;
  for (int st = 0; st < nst; st++) {
    const bool last = st == nst - 1;
    const double* c = pb.stages[st].data();
    const double* in = bf.buf[cur].data();
    const int nxt = cur == 1 ? 2 : 1;
    double* out = last ? nullptr : bf.buf[nxt].data();
    for (int b = 0; b < nt; b++) {
      const Tuple& Tb = tiles[b];
      int64_t e[kMaxD] = {1, 1, 1, 1};
      for (int m = 0; m < d; m++) e[m] = extent(Tb, m);
      int64_t j[kMaxD] = {0, 0, 0, 0};
      for (;;) {
        double acc[kMaxBl];
        for (int64_t x = 0; x < e[0]; x++) acc[x] = 0.0;
        for (int s = 0; s < S.n; s++) {
          const double cs = c[s];
          if (cs == 0.0) continue;
          // element j o phi_s of the source tile: sum_m j[phi_s(m)] bl^m; j[0]
          // sits at position inv0[s]
          int64_t base = 0;
          for (int m = 0; m < d; m++) {
            const int k = S.p[s][m];
            if (k != 0) base += j[k] * pb.pw[m];
          }
          const double* a = in + src[b][s] * pb.V + base;
          const int64_t str = pb.pw[pb.inv0[s]];
          for (int64_t x = 0; x < e[0]; x++) {
            const double prod = cs * a[x * str];
            acc[x] = acc[x] + prod;
          }
        }
        if (!last) {
          int64_t l = 0;
          for (int m = 1; m < d; m++) l += j[m] * pb.pw[m];
          double* o = out + b * pb.V + l;
          for (int64_t x = 0; x < e[0]; x++) o[x] = acc[x];
        } else {
          int64_t g = Tb[0] * pb.bl;
          for (int m = 1; m < d; m++) g += (Tb[m] * pb.bl + j[m]) * pb.gs[m];
          double* o = pb.B + g;
          if (pb.beta != 0.0) {
            for (int64_t x = 0; x < e[0]; x++) {
              double r = pb.alpha * acc[x];
              const double bo = pb.beta * o[x];
              r = r + bo;
              o[x] = r;
            }
          } else {
            for (int64_t x = 0; x < e[0]; x++) o[x] = pb.alpha * acc[x];
          }
        }
        int m = 1;
        while (m < d && ++j[m] == e[m]) j[m++] = 0;
        if (m >= d) break;
      }
    }
    cur = nxt;
  }
}

// sorted tuples T_1 <= ... <= T_d over nt tiles (Algorithm 5a's task list),
// by an odometer over non-decreasing tuples
std::vector<Tuple> block_orbits(int d, int64_t nt) {
  std::vector<Tuple> r;
  if (nt == 0) return r;
  Tuple v{};
  for (;;) {
    r.push_back(v);
    int m = d - 1;
    while (m >= 0 && v[m] == nt - 1) m--;
    if (m < 0) break;
    v[m]++;
    for (int k = m + 1; k < d; k++) v[k] = v[m];
  }
  return r;
}

}  // namespace

extern "C" int spinsum_alg6(int d, int64_t N, const double* A, double* B, const double* coef, int nfactors,
                            int factorized, double alpha, double beta, int bl, int nthreads) {
  if (d < 2 || d > kMaxD || N < 0 || nfactors < 1 || nfactors > kMaxFactors || bl < 0 || bl > kMaxBl ||
      nthreads < 0 || (factorized != 0 && factorized != 1))
    return -1;
  if (!coef || (N > 0 && (!A || !B))) return -1;
  // N^d must be addressable
  int64_t total = 1;
  for (int m = 0; m < d; m++) {
    if (N > 0 && total > INT64_MAX / N) return -1;
    total *= N;
  }
  if (total == 0) return 0;
  if (bl == 0) bl = d == 2 ? 64 : (d == 3 ? 16 : 8);

  Problem pb;
  pb.d = d;
  pb.N = N;
  pb.bl = bl;
  pb.A = A;
  pb.B = B;
  pb.alpha = alpha;
  pb.beta = beta;
  pb.S = make_sym(d);
  pb.V = 1;
  for (int m = 0; m < kMaxD; m++) {
    pb.pw[m] = m < d ? pb.V : 0;
    if (m < d) pb.V *= bl;
  }
  pb.gs[0] = 1;
  for (int m = 1; m < kMaxD; m++) pb.gs[m] = pb.gs[m - 1] * N;
  for (int s = 0; s < pb.S.n; s++)
    for (int m = 0; m < d; m++)
      if (pb.S.p[s][m] == 0) pb.inv0[s] = m;
  try {
    if (factorized && nfactors > 1) {
      // innermost factor first: F_k, ..., F_2, then F_1 with alpha and beta
      for (int f = nfactors - 1; f >= 0; f--)
        pb.stages.emplace_back(coef + (size_t)f * pb.S.n, coef + (size_t)(f + 1) * pb.S.n);
    } else {
      pb.stages.push_back(expand_chain(pb.S, d, coef, nfactors));
    }
    const int64_t nt = (N + bl - 1) / bl;
    const std::vector<Tuple> tasks = block_orbits(d, nt);
    int nth = nthreads > 0 ? nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
    nth = (int)std::min<int64_t>(nth, (int64_t)tasks.size());
    const int nbuf = pb.stages.size() == 1 ? 1 : (pb.stages.size() == 2 ? 2 : 3);
    std::vector<Buffers> bufs(nth);
    for (auto& b : bufs)
      for (int k = 0; k < nbuf; k++) b.buf[k].assign((size_t)pb.S.n * pb.V, 0.0);
    std::atomic<int64_t> next{0};
    auto worker = [&](int w) {
      for (;;) {
        const int64_t i = next.fetch_add(1, std::memory_order_relaxed);
        if (i >= (int64_t)tasks.size()) break;
        macro_kernel(pb, tasks[i], bufs[w]);
      }
    };
    std::vector<std::thread> th;
    th.reserve(nth);
    try {
      for (int w = 1; w < nth; w++) th.emplace_back(worker, w);
    } catch (const std::system_error&) {
      // fewer threads than asked: the ones started and this one take all tasks
    }
    worker(0);
    for (auto& t : th) t.join();
  } catch (const std::bad_alloc&) {
    return -2;
  }
  return 0;
}
