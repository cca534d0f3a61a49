// Drives the host blocked algorithm (cpu_alg6/alg6.cpp) under AddressSanitizer
// and UndefinedBehaviorSanitizer: every d, tiles cut by the tensor's edge,
// tile edges 1..bl > N, expanded and factorized chains, in place, several
// threads, and the invalid-argument returns. Prints "ok" at the end.
#include <cmath>
#include <cstdio>
#include <vector>

#include "spinsum_alg6.h"

static int fact(int d) { return d == 2 ? 2 : (d == 3 ? 6 : 24); }

int main() {
  unsigned long long state = 12345;
  auto rnd = [&]() {
    state = state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (double)((state >> 11) & ((1ULL << 52) - 1)) / (double)(1ULL << 52) - 0.5;
  };
  const int cases[][3] = {{2, 9, 4}, {2, 3, 5}, {3, 7, 3}, {3, 5, 1}, {3, 6, 16}, {4, 5, 2}, {4, 6, 4}, {4, 3, 8}};
  for (const auto& c : cases) {
    const int d = c[0], N = c[1], bl = c[2], n = fact(d);
    long long total = 1;
    for (int m = 0; m < d; m++) total *= N;
    std::vector<double> A(total), B(total), B2(total), coef(3 * n);
    for (auto& v : A) v = rnd();
    for (auto& v : coef) v = std::floor(4 * rnd());
    for (int fac = 0; fac < 2; fac++) {
      for (int nth = 1; nth <= 3; nth += 2) {
        if (spinsum_alg6(d, N, A.data(), B.data(), coef.data(), 3, fac, 0.5, 0.0, bl, nth) != 0) return 1;
        for (long long i = 0; i < total; i++) B2[i] = B[i];
        if (spinsum_alg6(d, N, A.data(), B2.data(), coef.data(), 3, fac, 1.0, -2.0, bl, nth) != 0) return 2;
        std::vector<double> Ai(A);
        if (spinsum_alg6(d, N, Ai.data(), Ai.data(), coef.data(), 3, fac, 1.0, 0.25, bl, nth) != 0) return 3;
      }
    }
    // factorized and expanded agree on integer coefficients (exact sums)
    std::vector<double> E(total), F(total);
    if (spinsum_alg6(d, N, A.data(), E.data(), coef.data(), 3, 0, 1.0, 0.0, bl, 2) != 0) return 4;
    if (spinsum_alg6(d, N, A.data(), F.data(), coef.data(), 3, 1, 1.0, 0.0, bl, 2) != 0) return 5;
    double scale = 0;
    for (long long i = 0; i < total; i++) scale = std::fmax(scale, std::fabs(E[i]));
    for (long long i = 0; i < total; i++)
      if (std::fabs(E[i] - F[i]) > 1e-12 * (1.0 + scale)) return 6;
    // Algorithm 2 (expanded chain), out of place and in place, one and several threads
    std::vector<double> G(total), H(A);
    if (spinsum_alg2(d, N, A.data(), G.data(), coef.data(), 3, 1.0, 0.0, 1) != 0) return 7;
    if (spinsum_alg2(d, N, H.data(), H.data(), coef.data(), 3, 1.0, 0.0, 3) != 0) return 8;
    for (long long i = 0; i < total; i++)
      if (G[i] != H[i] || std::fabs(E[i] - G[i]) > 1e-12 * (1.0 + scale)) return 9;
  }
  if (spinsum_alg2(5, 2, nullptr, nullptr, nullptr, 1, 1.0, 0.0, 1) != -1) return 15;
  double A[8] = {}, B[8] = {}, c[6] = {1, 0, 0, 0, 0, 0};
  if (spinsum_alg6(1, 2, A, B, c, 1, 0, 1.0, 0.0, 0, 1) != -1) return 10;
  if (spinsum_alg6(3, 2, A, B, c, 1, 0, 1.0, 0.0, 65, 1) != -1) return 11;
  if (spinsum_alg6(3, 2, nullptr, B, c, 1, 0, 1.0, 0.0, 0, 1) != -1) return 12;
  if (spinsum_alg6(3, 2, A, B, nullptr, 1, 0, 1.0, 0.0, 0, 1) != -1) return 13;
  if (spinsum_alg6(3, 0, nullptr, nullptr, c, 1, 0, 1.0, 0.0, 0, 1) != 0) return 14;
  std::printf("ok\n");
  return 0;
}
