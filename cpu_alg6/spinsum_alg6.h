/*
 * The paper's blocked CPU algorithm for the spin summation (Sec. 4.5
 * Algorithm 5a: one task per block orbit, taken dynamically by a pool of
 * threads; Sec. 4.6 Algorithm 6: the macro-kernel traverses every output tile
 * along its stride-1 index), as a native host library. It is a comparison
 * point for the GPU library on the same machine's host cores, not a part of
 * the GPU path: the GPU entry points never call it.
 *
 * Layout: the paper's dense N^d tensor (Sec. 3.1), column-major, element
 * (i_1, ..., i_d) at i_1 + N i_2 + N^2 i_3 (+ N^3 i_4).
 *
 * Operation (Def. 3-4, Eq. 4-6; in place Sec. 4.6.5):
 *   B = alpha * F_1(F_2(...F_k(A))) + beta * B_old
 * with pi_phi(A)[t] = A[t_phi(1), ..., t_phi(d)] and each factor F_j given as
 * d! coefficients in lexicographic one-line order of S_d (identity first).
 * factorized = 0 applies the expanded product of the chain (one stage);
 * factorized = 1 applies the factors stage by stage, F_k first, on the
 * block orbit's tiles held in per-thread buffers (Algorithm 5b's auxiliary T).
 * Every output element is the sum of its terms in lexicographic order of
 * sigma, multiply then add, one rounding each, no fused multiply-add; zero
 * coefficients are skipped; then alpha * sum, then + beta * B_old (B_old not
 * read when beta == 0).
 */
#ifndef SPINSUM_ALG6_H
#define SPINSUM_ALG6_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * d        2, 3 or 4.
 * N        extent of every index (N >= 0; N = 0 is a no-op).
 * A        input, N^d doubles (host memory, read only unless A == B).
 * B        output, N^d doubles; B == A runs in place (each block orbit's
 *          tiles are read completely before any of them is written).
 * coef     nfactors * d! doubles, factor F_1 first.
 * nfactors 1..8.
 * bl       tile edge (1..64); 0 picks 64 / 16 / 8 for d = 2 / 3 / 4.
 * nthreads worker threads (>= 1); 0 uses the hardware concurrency.
 * Returns 0; -1 on an invalid argument (nothing written); -2 if a per-thread
 * buffer could not be allocated (B may be partly written).
 */
int spinsum_alg6(int d, int64_t N, const double* A, double* B, const double* coef, int nfactors,
                 int factorized, double alpha, double beta, int bl, int nthreads);

/*
 * spinsum_alg2 -- the paper's Algorithm 2 (Sec. 4.2), the spin summation of
 * the NCC code that Algorithm 6 is measured against: loops over the sorted
 * tuples i_1 <= ... <= i_d, and for each the d! (fewer where indices repeat)
 * update statements of its element orbit, which share their operands. No
 * blocking; the outermost index is split cyclically over `nthreads` threads
 * (0: the hardware concurrency). A chain is applied as its expanded product;
 * rounding order as above (factorized is not an option). Same layout, in
 * place rule and return codes as spinsum_alg6.
 */
int spinsum_alg2(int d, int64_t N, const double* A, double* B, const double* coef, int nfactors, double alpha,
                 double beta, int nthreads);

#ifdef __cplusplus
}
#endif

#endif /* SPINSUM_ALG6_H */
