/* Runs the oracle's entry points on small inputs so that a build with
 * AddressSanitizer and UndefinedBehaviorSanitizer checks every access and
 * operation of the C oracle: d = 3 and 4, 0..2 spectator indices, expanded
 * and factorized chains, in place and out of place, beta, strided and empty
 * tensors, and the transpose. The results are checked for internal
 * consistency on integer-valued inputs (factorized == expanded, in place ==
 * out of place, <S x, y> == <x, S^T y>). Prints "ok" and exits 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_perms(int d, int* out);
int oracle_expand(int d, const double* coef, int nfactors, double* out);
int oracle_spinsum(int d, int nspec, const int64_t* ext, const double* A, const int64_t* lda, double* B,
                   const int64_t* ldb, const double* coef, int nfactors, int factorized, double alpha, double beta,
                   int inplace);
int oracle_spinsum_transpose(int d, int nspec, const int64_t* ext, const double* Y, double* X, const double* coef,
                             int nfactors, double alpha);

static uint64_t rng = 88172645463325252ull;
static int64_t irand(int64_t n) {
  rng ^= rng << 13;
  rng ^= rng >> 7;
  rng ^= rng << 17;
  return (int64_t)(rng % (uint64_t)n);
}

static int fail(const char* what, int d, int nspec) {
  fprintf(stderr, "FAIL %s (d=%d nspec=%d)\n", what, d, nspec);
  return 1;
}

static int run_case(int d, int nspec, int O, int V, int nfactors) {
  const int np = d == 3 ? 6 : 24, nidx = nspec + d;
  int64_t ext[8], ld[8], n = 1;
  for (int k = 0; k < nidx; k++) {
    ext[k] = k < nspec ? V : O;
    ld[k] = n;
    n *= ext[k];
  }
  double* coef = (double*)malloc(sizeof(double) * np * nfactors);
  for (int i = 0; i < np * nfactors; i++) coef[i] = (double)(irand(5) - 2);
  double* A = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* B1 = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* B2 = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* C = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* Y = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* X = (double*)malloc(sizeof(double) * (n ? n : 1));
  for (int64_t e = 0; e < n; e++) {
    A[e] = (double)(irand(7) - 3);
    Y[e] = (double)(irand(7) - 3);
    B1[e] = B2[e] = 1.0;
  }
  int bad = 0;
  if (oracle_spinsum(d, nspec, ext, A, ld, B1, ld, coef, nfactors, 0, 2.0, 0.5, 0)) bad |= fail("expanded", d, nspec);
  if (oracle_spinsum(d, nspec, ext, A, ld, B2, ld, coef, nfactors, 1, 2.0, 0.5, 0)) bad |= fail("factorized", d, nspec);
  for (int64_t e = 0; e < n && !bad; e++)
    if (B1[e] != B2[e]) bad |= fail("factorized != expanded", d, nspec);
  memcpy(C, A, sizeof(double) * (n ? n : 1));
  for (int64_t e = 0; e < n; e++) B1[e] = A[e];
  if (oracle_spinsum(d, nspec, ext, A, ld, B1, ld, coef, nfactors, 1, 1.0, -1.0, 0)) bad |= fail("oop", d, nspec);
  if (oracle_spinsum(d, nspec, ext, C, ld, C, ld, coef, nfactors, 1, 1.0, -1.0, 1)) bad |= fail("in place", d, nspec);
  for (int64_t e = 0; e < n && !bad; e++)
    if (B1[e] != C[e]) bad |= fail("in place != out of place", d, nspec);
  /* <S A, Y> == <A, S^T Y> */
  if (oracle_spinsum(d, nspec, ext, A, ld, B1, ld, coef, nfactors, 1, 1.0, 0.0, 0)) bad |= fail("S", d, nspec);
  if (oracle_spinsum_transpose(d, nspec, ext, Y, X, coef, nfactors, 1.0)) bad |= fail("S^T", d, nspec);
  double l = 0, r = 0;
  for (int64_t e = 0; e < n; e++) {
    l += B1[e] * Y[e];
    r += A[e] * X[e];
  }
  if (l != r) bad |= fail("adjoint identity", d, nspec);
  /* strided: every index at twice its dense stride, the gaps untouched */
  int64_t lds[8];
  for (int k = 0; k < nidx; k++) lds[k] = 2 * ld[k];
  double* As = (double*)calloc((size_t)(2 * (n ? n : 1)), sizeof(double));
  double* Bs = (double*)calloc((size_t)(2 * (n ? n : 1)), sizeof(double));
  for (int64_t e = 0; e < n; e++) As[2 * e] = A[e];
  for (int64_t e = 0; e < 2 * n; e++) Bs[e] = -7.0;
  if (oracle_spinsum(d, nspec, ext, As, lds, Bs, lds, coef, nfactors, 1, 1.0, 0.0, 0)) bad |= fail("strided", d, nspec);
  for (int64_t e = 0; e < n && !bad; e++)
    if (Bs[2 * e] != B1[e] || Bs[2 * e + 1] != -7.0) bad |= fail("strided result", d, nspec);
  free(coef); free(A); free(B1); free(B2); free(C); free(Y); free(X); free(As); free(Bs);
  return bad;
}

int main(void) {
  int bad = 0;
  int perms[24 * 4];
  double full[24], ch[3 * 24];
  for (int d = 3; d <= 4; d++) {
    if (oracle_perms(d, perms) != (d == 3 ? 6 : 24)) bad |= fail("perms", d, 0);
    for (int i = 0; i < 3 * 24; i++) ch[i] = (double)(irand(5) - 2);
    if (oracle_expand(d, ch, 3, full) != (d == 3 ? 6 : 24)) bad |= fail("expand", d, 0);
  }
  /* argument errors are rejected, not crashed on */
  int64_t ext0[8] = {2, 2, 2, 3, 3, 4}, ld0[8] = {1, 2, 4, 8, 24, 72};
  double c6[6] = {1, 1, 1, 1, 1, 1}, a[4096], b[4096];
  if (oracle_spinsum(3, 3, ext0, a, ld0, b, ld0, c6, 1, 0, 1.0, 0.0, 0) == 0) bad |= fail("unequal extents accepted", 3, 3);
  if (oracle_spinsum(5, 0, ext0, a, ld0, b, ld0, c6, 1, 0, 1.0, 0.0, 0) == 0) bad |= fail("d = 5 accepted", 5, 0);
  for (int d = 3; d <= 4; d++)
    for (int nspec = 0; nspec <= 2; nspec++)
      for (int nf = 1; nf <= 3; nf++) {
        bad |= run_case(d, nspec, d == 3 ? 4 : 3, 3, nf);
        bad |= run_case(d, nspec, 0, 3, nf);   /* empty */
        bad |= run_case(d, nspec, 1, 2, nf);   /* a single orbit, all indices equal */
      }
  if (!bad) puts("ok");
  return bad;
}
