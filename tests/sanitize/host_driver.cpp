// Runs the host planner (ss_host.cpp, linked with device stand-ins) under
// AddressSanitizer and UndefinedBehaviorSanitizer: the plan of every Table II
// style chain shape for d = 3 and 4 (expanded, factorized, adjoint, strict,
// alpha and beta variants, spectator and paper layouts), and the public entry
// points on invalid arguments and without a device. Prints "ok" on success.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/spinsum.h"

extern "C" int ss_debug_plan(int d, int O, int V, const double* coef, int nfactors, int mode, double alpha,
                             double beta, double* expanded, int64_t* info, int* ci, int* mp);

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static int irand(int n) {
  rng ^= rng << 13;
  rng ^= rng >> 7;
  rng ^= rng << 17;
  return (int)(rng % (uint64_t)n);
}

int main() {
  int bad = 0;
  double ex[24];
  int64_t info[32];
  std::vector<int> ci(8 * 24), mp(501);
  const double alphas[] = {1.0, 0.5, 0.3, -2.0};
  const double betas[] = {0.0, 1.0, -0.25};
  for (int d = 3; d <= 4; d++) {
    const int np = d == 3 ? 6 : 24;
    for (int nf = 1; nf <= 9; nf += 2) {
      std::vector<double> coef(np * nf);
      for (int trial = 0; trial < 6; trial++) {
        for (auto& c : coef) c = trial == 5 ? 0.37 * (irand(9) - 4) : (double)(irand(5) - 2);
        for (int mode = 0; mode < 8; mode++)
          for (double a : alphas)
            for (double b : betas)
              for (int O : {1, 2, 5, 12})
                for (int V : {1, 3, 16}) {
                  const int rc = ss_debug_plan(d, O, V, coef.data(), nf, mode, a, b, ex, info, ci.data(), mp.data());
                  if (rc != SPINSUM_OK && rc != SPINSUM_ERR_ARG && rc != SPINSUM_ERR_UNSUPPORTED) {
                    std::printf("FAIL plan d=%d nf=%d mode=%d rc=%d\n", d, nf, mode, rc);
                    bad = 1;
                  }
                }
      }
    }
  }
  // public entry points: invalid arguments, and valid ones with no device
  double A[4096] = {0}, B[4096] = {0}, c6[6] = {4, -2, -2, 1, 1, -2};
  int64_t ext[6] = {2, 2, 2, 3, 3, 3}, ld[6] = {1, 2, 4, 8, 24, 72};
  int64_t bad_ext[6] = {2, 2, 2, 3, 3, 4};
  if (spinsum_3d(SPINSUM_F64, bad_ext, A, ld, B, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr) == SPINSUM_OK) bad = 1;
  if (spinsum_3d(SPINSUM_F64, ext, nullptr, ld, B, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr) == SPINSUM_OK) bad = 1;
  if (spinsum_3d(SPINSUM_F64, ext, A, ld, B, ld, nullptr, 1, 0, 1.0, 0.0, 0, nullptr) == SPINSUM_OK) bad = 1;
  if (spinsum_3d(SPINSUM_F64, ext, A, ld, A + 1, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr) == SPINSUM_OK) bad = 1;
  if (spinsum_3d(7, ext, A, ld, B, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr) == SPINSUM_OK) bad = 1;
  (void)spinsum_3d(SPINSUM_F64, ext, A, ld, B, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr);
  (void)spinsum_3d_host(SPINSUM_F64, ext, A, ld, B, ld, c6, 1, 0, 1.0, 0.0, 0, nullptr, 0, nullptr);
  spinsum_problem pr{};
  pr.d = 3;
  for (int k = 0; k < 6; k++) {
    pr.ext[k] = ext[k];
    pr.lda[k] = ld[k];
    pr.ldb[k] = ld[k];
  }
  pr.A = A;
  pr.B = B;
  pr.coef = c6;
  pr.nfactors = 1;
  pr.alpha = 1.0;
  spinsum_plan* plan = nullptr;
  if (spinsum_plan_create(&plan, &pr, 1, SPINSUM_F64, 0, nullptr) == SPINSUM_OK) {
    (void)spinsum_plan_execute(plan, nullptr);
    (void)spinsum_plan_describe(plan);
    (void)spinsum_plan_destroy(plan);
  }
  (void)spinsum_batch_static(&pr, 1, SPINSUM_F64, nullptr);
  // packed antisymmetric storage: invalid arguments, and valid ones with no device
  {
    // arrays sized for d = 4 (2d extents and strides, d + 1 packed strides)
    int64_t pext[8] = {2, 2, 2, 5, 5, 5, 5, 5}, pldb[8] = {1, 2, 4, 8, 40, 200, 1000, 5000};
    int64_t pldp[5] = {1, 2, 4, 8, 8};
    double Pk[1024] = {0}, Bk[2048] = {0};
    for (int d = 1; d <= 5; d++) {
      (void)spinsum_unpack(d, SPINSUM_F64, pext, Pk, pldp, Bk, pldb, nullptr);
      (void)spinsum_pack(d, SPINSUM_F32, pext, Bk, pldb, Pk, pldp, nullptr);
    }
    if (spinsum_unpack(3, SPINSUM_F64, pext, Pk, pldp, Pk + 4, pldb, nullptr) == SPINSUM_OK) bad = 1;
    int64_t short_ldp[5] = {1, 2, 4, 7, 7};
    if (spinsum_pack(3, SPINSUM_F64, pext, Bk, pldb, Pk, short_ldp, nullptr) == SPINSUM_OK) bad = 1;
  }
  if (spinsum_last_error() == nullptr || spinsum_version() == nullptr) bad = 1;
  if (!bad) std::puts("ok");
  return bad;
}
