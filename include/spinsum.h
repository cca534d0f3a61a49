/*
 * spinsum.h -- C-ABI of the GB300 spin-summation library.
 *
 * The operation (Def. 3, Eq. 4 of Springer, Matthews & Bientinesi, "Spin
 * Summations: A High-Performance Perspective", arXiv 1705.06661):
 *
 *   B = alpha * sum_{sigma in S_d} a_sigma * pi_sigma(A) + beta * B
 *
 * over one group of d permuted indices of a tensor that also carries d
 * spectator indices (CCSD: d = 2, A[a,b,i,j]; CCSDT: d = 3, A[a,b,c,i,j,k];
 * CCSDTQ: d = 4, A[a,b,c,d,i,j,k,l]). pi_phi acts on the permuted group as in Def. 1-2
 * (Eq. 1-3): pi_phi(A)[s, i_1..i_d] = A[s, i_phi(1), ..., i_phi(d)].
 *
 * Coefficients. `coef` holds `nfactors` rows of d! doubles each; the columns
 * are the permutations of S_d in lexicographic one-line order, identity first
 * (for d = 3: 123, 132, 213, 231, 312, 321 -- the order of Algorithms 2 and 4).
 * The rows are a factor chain F_1 .. F_k meaning B = F_1(F_2(...F_k(A)))
 * (Def. 4, Eq. 5-6); composition follows Eq. 9-10: pi_phi(pi_psi(A)) =
 * pi_{phi o psi}(A). With one row the chain is a plain coefficient vector.
 *
 * Tensor layout. Every index has an extent and an element stride (int64,
 * counted in elements, not bytes). Indices 0..d-1 are the spectators, indices
 * d..2d-1 the permuted group; the d permuted extents must be equal (Sec. 3.1).
 * Column-major storage with the spectators fastest is the fast layout: each
 * permuted tuple then owns a contiguous run of ext[0]*..*ext[d-1] elements.
 * The paper's own N^d layout is spectator extents 1 with the permuted group at
 * strides 1, N, N^2 (, N^3); any other non-overlapping strides also work.
 *
 * Ownership. The caller owns every buffer. A and B are device pointers; calls
 * are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream)
 * and allocate nothing. Coefficients, extents and strides are host memory,
 * read during the call only.
 *
 * Errors. Every entry point returns SPINSUM_OK (0) or a negative status and
 * never aborts, exits or traps the GPU. spinsum_last_error() gives a message
 * for the calling thread's last failure. Device-side failures (a bounded wait
 * that ran out, an element outside the fast path's range that could not be
 * handled) set a device status word that spinsum_check_status() reads.
 *
 * Threads. The error message and the launch count are per thread. Calls on
 * device tensors (spinsum_2d/3d/4d, spinsum_unpack/pack) and
 * spinsum_plan_execute on distinct plans may run concurrently from several
 * threads. Three things are shared per process and must not be used from two
 * threads at once: the staging pipeline of the host-tensor calls
 * (spinsum_*_host, one per device), the parameter array of
 * spinsum_batch_static (one per device), and the autotuning cache that every
 * spinsum_plan_create reads (and extends when it tunes), so plans are created
 * from one thread at a time.
 */
#ifndef SPINSUM_H
#define SPINSUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* spinsum_stream_t; /* same type as cudaStream_t */

enum spinsum_status {
  SPINSUM_OK = 0,
  SPINSUM_ERR_ARG = -1,         /* bad extent, stride, pointer, dtype, mode or coefficient */
  SPINSUM_ERR_ALIAS = -2,       /* A and B overlap without inplace = 1 (or inplace with A != B) */
  SPINSUM_ERR_UNSUPPORTED = -3, /* valid request this build does not implement */
  SPINSUM_ERR_CUDA = -4,        /* a CUDA runtime call failed (message has the CUDA error) */
  SPINSUM_ERR_TIMEOUT = -5,     /* a device-side bounded wait ran out */
  SPINSUM_ERR_DEVICE = -6       /* another device-side check failed */
};

enum spinsum_dtype { SPINSUM_F64 = 0, SPINSUM_F32 = 1 };

/* mode bits */
enum spinsum_mode {
  SPINSUM_EXPANDED = 0,   /* multiply the chain out on the host (product rule), one pass of d!-term sums */
  SPINSUM_FACTORIZED = 1, /* apply the factors stage by stage on chip, innermost first (Def. 4) */
  SPINSUM_ADJOINT = 2,    /* apply the transpose S^T = F_k^T ... F_1^T, F^T(sigma) = F(sigma^-1) */
  SPINSUM_STRICT = 4,     /* FP64 only: native FP64 arithmetic in the reference order (lex sigma,
                             multiply then add, no FMA), bit-identical to a plain loop nest */
  SPINSUM_TMA = 8         /* 3D, exact FP64 or FP32: stage orbits through shared memory with TMA bulk
                             copies (producer warp + mbarrier ring) instead of the default
                             register-streaming kernel; same results. Ignored where it does not apply
                             (4D, strict, unaligned or odd spectator blocks) and in batched plans. */
};

/*
 * spinsum_3d -- 3D spin summation on a 6-index tensor (Def. 3 with d = 3).
 *
 * dtype : SPINSUM_F64 (double in, double out) or SPINSUM_F32 (float in, float
 *         out, float accumulation).
 * ext   : 6 extents; ext[0..2] spectators a,b,c; ext[3..5] permuted i,j,k,
 *         ext[3] == ext[4] == ext[5].
 * A,lda : input tensor and its 6 element strides.
 * B,ldb : output tensor and its 6 element strides.
 * coef  : nfactors x 6 doubles (see above); 1 <= nfactors <= 8; finite.
 * mode  : SPINSUM_EXPANDED or SPINSUM_FACTORIZED, optionally | SPINSUM_ADJOINT,
 *         | SPINSUM_STRICT.
 * alpha, beta : B = alpha * S(A) + beta * B_old; beta == 0 never reads B.
 * inplace : 1 computes A = alpha * S(A) + beta * A (Sec. 4.6.5); then B must
 *           equal A and ldb equal lda. 0 requires A and B not to overlap.
 * stream : cudaStream_t to launch on.
 *
 * FP64 arithmetic. With integer coefficients (up to a common power-of-two
 * scale) and a chain 1-norm below 128, the sums run in exact fixed-point
 * integer arithmetic on a per-element grid of 2^-48 of the largest input of
 * the permutation orbit: integer-valued inputs give exact results, other
 * inputs are within 2^-47 * sum|a| * max|A| (plus the final rounding).
 * Otherwise, or with SPINSUM_STRICT, native FP64 in the reference order.
 */
int spinsum_3d(int dtype, const int64_t ext[6], const void* A, const int64_t lda[6], void* B,
               const int64_t ldb[6], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream);

/* spinsum_2d -- 2D spin summation on a 4-index tensor (Def. 3 with d = 2, the
 * CCSD case of Sec. 1): ext[0..1] spectators a,b; ext[2..3] permuted i,j
 * (equal); coef is nfactors x 2 doubles (identity, then the transposition).
 * Otherwise as spinsum_3d. */
int spinsum_2d(int dtype, const int64_t ext[4], const void* A, const int64_t lda[4], void* B,
               const int64_t ldb[4], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream);

/* spinsum_4d -- 4D spin summation on an 8-index tensor (Def. 3 with d = 4):
 * ext[0..3] spectators a,b,c,d; ext[4..7] permuted i,j,k,l (all equal);
 * coef is nfactors x 24 doubles. Otherwise as spinsum_3d. */
int spinsum_4d(int dtype, const int64_t ext[8], const void* A, const int64_t lda[8], void* B,
               const int64_t ldb[8], const double* coef, int nfactors, int mode, double alpha, double beta,
               int inplace, spinsum_stream_t stream);

/*
 * spinsum_3d_host / spinsum_4d_host -- the same summation on tensors in host
 * memory (pinned memory lets the copies run asynchronously and overlap).
 *
 * A and B are host pointers to dense column-major tensors (strides must be
 * the dense ones; SPINSUM_ERR_UNSUPPORTED otherwise).
 * Page-locked memory (cudaHostAlloc / cudaHostRegister, mapped): the orbit
 * kernel reads A and writes B directly over the host link, in one launch that
 * uses both directions of the link at once; `workspace` is not used and may
 * be NULL.
 * Pageable memory: the work is split along the slowest spectator index into
 * chunks; each chunk is copied to the device (one 2D copy with a row per
 * permuted tuple), summed there, and copied back, with copy-in, compute and
 * copy-out of successive chunks overlapped on three internal streams (created
 * on the first call on each device and kept). The device memory is the
 * caller's `workspace` of `workspace_bytes` (three chunk slots;
 * SPINSUM_ERR_ARG with the minimum size if it cannot hold one slice).
 * The call is asynchronous: `stream` is ordered before and after the whole
 * pipeline, so a synchronize on `stream` waits for B. Other arguments as for
 * spinsum_3d / spinsum_4d.
 */
int spinsum_3d_host(int dtype, const int64_t ext[6], const void* A, const int64_t lda[6], void* B,
                    const int64_t ldb[6], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream);
int spinsum_2d_host(int dtype, const int64_t ext[4], const void* A, const int64_t lda[4], void* B,
                    const int64_t ldb[4], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream);
int spinsum_4d_host(int dtype, const int64_t ext[8], const void* A, const int64_t lda[8], void* B,
                    const int64_t ldb[8], const double* coef, int nfactors, int mode, double alpha, double beta,
                    int inplace, void* workspace, size_t workspace_bytes, spinsum_stream_t stream);

/*
 * spinsum_contract -- the spin summation fused into the contraction it feeds.
 * The spin-summed amplitudes of CC theory are intermediates of tensor
 * contractions (Sec. 1; Sec. 6 names the kernels around the summation as the
 * next target). This call contracts the summed tensor over its whole permuted
 * group without storing it:
 *
 *   C[s, y] = sum_t S(A)[s, t] * W[y, t]      (coef != NULL)
 *   C[s, y] = sum_t A[s, t] * W[y, t]         (coef == NULL: the contraction alone)
 *
 * s runs over the S = ext[0] * .. * ext[d-1] spectator positions, t over the
 * O^d tuples of the permuted group (column-major index t = i_1 + O i_2 + ...),
 * y over 0 .. Y-1.
 *
 * d      : 2, 3 or 4.
 * ext    : 2d extents: d spectators, then d equal permuted extents O.
 * A      : FP64 device tensor, dense column-major (spectators fastest).
 * coef, nfactors, mode : the operator, as for spinsum_3d (EXPANDED or
 *          FACTORIZED, optionally | ADJOINT, | STRICT); ignored when coef is
 *          NULL. alpha = 1, beta = 0.
 * W      : FP64 device matrix W[y + ldw * t] (y fastest), ldw >= Y.
 * C      : FP64 device matrix C[s + ldc * y] (s fastest), ldc >= S; written,
 *          never read; must not overlap A or W.
 * stream : cudaStream_t to launch on.
 *
 * Every element of S(A) is formed in registers (the cores of spinsum_3d, so
 * with the exact core S(A) equals what spinsum_3d/4d would store) and
 * multiplied into FP64 accumulators in orbit order; A is read once per group
 * of 16 columns of C. FP64 only. Errors: SPINSUM_ERR_ARG (bad d, extents,
 * leading dimensions, pointers or mode bits), SPINSUM_ERR_ALIAS (C overlaps A
 * or W), SPINSUM_ERR_CUDA. Asynchronous on `stream`; allocates nothing.
 */
int spinsum_contract(int d, const int64_t ext[], const void* A, const double* coef, int nfactors, int mode,
                     const void* W, int64_t Y, int64_t ldw, void* C, int64_t ldc, spinsum_stream_t stream);

/*
 * Packed antisymmetric storage (tensor unpacking, named in Sec. 2 and Sec. 6
 * as a further use of the orbit traversal). An antisymmetric tensor B over
 * its d permuted indices is stored as P[s, r]: one value per strictly
 * increasing tuple t0 = (i_1 < .. < i_d), r = sum_k C(i_k, k + 1) (the colex
 * rank), C(O, d) values per spectator position s.
 *
 * spinsum_unpack -- B[s, t0 o tau] = sign(tau) * P[s, r] for every
 *   permutation tau, and B[s, t] = 0 where t repeats an index. Writes all of B.
 * spinsum_pack -- P[s, r] = B[s, t0] (the canonical member): the inverse of
 *   unpack on antisymmetric tensors.
 *
 * d      : 2, 3 or 4.
 * dtype  : SPINSUM_F64 or SPINSUM_F32 (P and B alike).
 * ext    : 2d extents of B: d spectators, then d permuted extents (equal, O).
 * B, ldb : the full tensor and its 2d element strides; the spectator indices
 *          must be dense and fastest (stride 1, then products of extents).
 * P, ldp : the packed tensor and its d + 1 element strides: the d spectator
 *          strides (equal to B's) and the stride of the packed index
 *          (at least the spectator block).
 * stream : cudaStream_t to launch on.
 * Errors: SPINSUM_ERR_ARG (bad d, dtype, extents or strides),
 * SPINSUM_ERR_UNSUPPORTED (non-dense spectators, O > 4096),
 * SPINSUM_ERR_ALIAS (P and B overlap), SPINSUM_ERR_CUDA. Caller-owned memory;
 * nothing is allocated; asynchronous on `stream`.
 */
int spinsum_unpack(int d, int dtype, const int64_t ext[], const void* P, const int64_t ldp[], void* B,
                   const int64_t ldb[], spinsum_stream_t stream);
int spinsum_pack(int d, int dtype, const int64_t ext[], const void* B, const int64_t ldb[], void* P,
                 const int64_t ldp[], spinsum_stream_t stream);

/*
 * Batched plans: many independent spin summations (uneven extents, mixed d,
 * mixed coefficient sets) run by one persistent kernel launch. The plan's work
 * list is the GPU form of the task-based scheduling of Sec. 4.5 (Algorithm
 * 5a): every (problem, block of orbits) pair is a task, and the persistent
 * CTAs take tasks in a fixed order instead of from a dynamic queue.
 *
 * spinsum_problem describes one summation exactly as the arguments of
 * spinsum_2d / spinsum_3d / spinsum_4d do (d = 2 uses the first 4 entries of
 * ext/lda/ldb, d = 3 the first 6).
 * spinsum_plan_create validates every problem, builds the device work list
 * (the plan allocates and owns that device memory until destroyed), copies the
 * coefficients, and picks tile sizes with its autotuner (which times
 * candidates on `stream` and may therefore run the problems: inputs must be
 * valid and in-place problems are restored only if `allow_tuning_runs` is 0,
 * in which case a fixed heuristic is used). dtype applies to all problems.
 * spinsum_plan_execute launches the whole batch as one kernel on `stream`;
 * it allocates nothing and may be captured in a CUDA graph. The kernel's CTAs
 * take work from counters in the plan's device memory (the last CTA of a
 * launch resets them), so two executions of one plan must not overlap on the
 * GPU; distinct plans are independent.
 */
typedef struct spinsum_problem {
  int d;            /* 2, 3 or 4 */
  int64_t ext[8];   /* d spectators then d permuted extents */
  const void* A;
  int64_t lda[8];
  void* B;
  int64_t ldb[8];
  const double* coef; /* nfactors x d! */
  int nfactors;
  int mode;
  double alpha;
  double beta;
  int inplace;
} spinsum_problem;

typedef struct spinsum_plan spinsum_plan;

int spinsum_plan_create(spinsum_plan** plan, const spinsum_problem* problems, int nproblems, int dtype,
                        int allow_tuning_runs, spinsum_stream_t stream);
int spinsum_plan_execute(spinsum_plan* plan, spinsum_stream_t stream);
int spinsum_plan_destroy(spinsum_plan* plan);
/* description of the plan's tuning choice, e.g. "vec=2 block=256 split=1" */
const char* spinsum_plan_describe(const spinsum_plan* plan);

/*
 * spinsum_batch_static -- the batched summation without any device allocation.
 * The paper has no counterpart: this is a deployment feature of the library.
 *
 * Some callers cannot call cudaMalloc: codes that reserve nearly all of HBM
 * for their amplitude tensors up front and hand out memory only from their
 * own pool, and latency-bound services where a cudaMalloc (and the device
 * synchronization it can imply) may not happen on the request path. For them
 * this entry point runs the same batched kernel as a plan, but reads the
 * per-problem parameters and block prefix sums from one fixed array that the
 * library keeps in device memory from load until process exit (about 430 KB
 * on every GPU that loads the library). The caller still owns and passes every
 * input and output tensor.
 *
 * problems, nproblems, dtype: as for spinsum_plan_create; at most
 *   SPINSUM_STATIC_MAX_PROBLEMS problems, else SPINSUM_ERR_ARG.
 * The call copies the parameters of the problems it is given (not the whole
 * array) into the array with cudaMemcpyAsync on `stream`, then launches
 * there; it calls no allocating routine. The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress), so make that first
 * call before any stream capture. The copy reads a host buffer that lives only
 * for the duration of the call, so the call returns SPINSUM_ERR_ARG on a
 * stream that is being captured. All calls share the one array and overwrite
 * what they use: calls whose work can overlap on the GPU (for example on two
 * streams at once) race on it, and the caller must order them.
 */
#define SPINSUM_STATIC_MAX_PROBLEMS 64
int spinsum_batch_static(const spinsum_problem* problems, int nproblems, int dtype, spinsum_stream_t stream);

/*
 * Error reporting and bookkeeping. These four calls are API additions with no
 * counterpart in the paper, which describes the computation only.
 */

/* Synchronizes `stream`, then reads and clears the device status word:
 * SPINSUM_OK, SPINSUM_ERR_TIMEOUT or SPINSUM_ERR_DEVICE. */
int spinsum_check_status(spinsum_stream_t stream);

/* Message for the calling thread's last failed call ("" if none). */
const char* spinsum_last_error(void);

/* Number of kernel launches the calling thread has issued through this
 * library since the last reset (for launch accounting in benchmarks). */
int64_t spinsum_launch_count(int reset);

/* Library version string. */
const char* spinsum_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPINSUM_H */
