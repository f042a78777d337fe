/*
 * gcge.h -- C ABI of the GB300 (sm_103a) GCG eigensolver.
 *
 * Computes the smallest `nev` eigenpairs of the sparse symmetric pencil
 *     A x = lambda B x,   A symmetric, B symmetric positive definite
 * (GCGE paper, Section 2, Eq. (1)) by the generalized conjugate gradient
 * (block damping inverse power) method of Algorithm 1, with the implementing
 * techniques of Section 3: internal locking, blockSize-wide P and W, dynamic
 * shift theta (Section 3.2, Eq. compW), B-orthogonalisation by Algorithm 3
 * (RecursiveOrthSVD), the structured Rayleigh-Ritz matrix of
 * Eq. (struct_bar_A_new), and the moving mechanism (Section 3.3).
 *
 * Conventions for every entry point
 *   - Every function returns an int status: GCGE_OK (0) or a negative code
 *     below.  Nothing is thrown across the ABI.  gcge_error_string() gives a
 *     static description; gcge_last_error_message() the detail of the most
 *     recent failure in the calling process.
 *   - Sparse matrices are CSR, 0-based, int32 row pointers and column indices,
 *     columns sorted within each row, full symmetric storage, FP64 values.
 *   - Multivectors ("blocks" of k vectors of length n) are ROW-MAJOR n x k
 *     with a leading dimension ld >= k (element (i, j) at X[i*ld + j]).
 *   - Small dense matrices (Gram blocks, Rayleigh-Ritz matrices) are FP64,
 *     COLUMN-MAJOR with a leading dimension (element (i, j) at C[i + j*ldc]).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device-pointer entry points are asynchronous on that stream
 *     unless stated otherwise; host-pointer arguments are read before return.
 *   - Pointers named d_* are device memory of the current CUDA device; all
 *     others are host memory.  The caller keeps ownership of every buffer it
 *     passes; the library owns what a handle allocates and frees it in
 *     gcge_destroy().
 */
#ifndef GCGE_H
#define GCGE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define GCGE_OK 0
#define GCGE_EINVAL (-1)      /* bad argument: sizes, CSR structure, nev/blockSize */
#define GCGE_ENOMEM (-2)      /* device allocation failed */
#define GCGE_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define GCGE_ENOTCONV (-4)    /* max_iter reached; results for the nconv locked pairs are valid */
#define GCGE_EBREAKDOWN (-5)  /* orthogonalisation lost the whole block (rank collapse) */
#define GCGE_ETIMEOUT (-6)    /* a bounded device-side wait ran out (grid barrier) */
#define GCGE_ENAN (-7)        /* NaN/Inf met in a Gram or Rayleigh-Ritz matrix */
#define GCGE_ENOTREADY (-8)   /* result queried before a successful gcge_solve() */

#define GCGE_FP64 0           /* every step in FP64 */
#define GCGE_MIXED 1          /* FP32 n-sized work, FP64 small dense work, FP64 refinement */

/* ----------------------------------------------------------------- types */
typedef struct gcge_handle gcge_handle;   /* opaque, owned by the library */

/* CSR matrix.  on_device = 0: the three arrays are host memory; 1: device
 * memory.  Either way gcge_create() copies them, so the caller may free them
 * as soon as it returns. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t *row_ptr;   /* n + 1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
  const int32_t *col_idx;   /* nnz entries in [0, n), sorted within each row */
  const double *val;        /* nnz FP64 values */
  int on_device;
} gcge_csr;

/* Options; gcge_options_default() fills the paper's defaults. */
typedef struct {
  int precision;            /* GCGE_FP64 or GCGE_MIXED                              (FP64)  */
  int cg_max_iter;          /* CG steps per GCG iteration, Section 4.1                (30)  */
  double cg_rtol;           /* CG stop at ||r|| <= cg_rtol ||r0||, Section 4.1      (1e-2)  */
  int use_shift;            /* dynamic shift theta of Section 3.2                     (1)   */
  int orth_leaf;            /* Algorithm 3 leaf width c = min(m, orth_leaf)          (16)  */
  int moving;               /* 1: moving mechanism of Section 3.3, 0: off, -1: auto (-1)  */
  int size_x;               /* 0: min(nev + 3 bs, n) (moving: max_proj_dim - 2 bs)   (0)   */
  int max_iter;             /* GCG iterations (Rayleigh-Ritz solves) before ENOTCONV (2000) */
  uint64_t seed;            /* initial block N(0,1) from splitmix64 + Box-Muller      (0)   */
  const double *initial_block; /* optional host n x size_x row-major start block (NULL) */
  double mixed_switch_tol;  /* MIXED: FP32 phase ends at this relative residual     (3e-6) */
  int verbose;              /* 1: one line per iteration on stderr                    (0)   */
  int checks;               /* 1: per iteration compare the structured Rayleigh-Ritz  (0)
                               matrix with an explicit V^T A V and V^T B V with I (slow) */
  int profile;              /* 1: time every kernel class with CUDA events           (0)   */
  int mixed_bs2;            /* MIXED: active block width of the FP64 phase; 0: blockSize (0) */
  int orth;                 /* STEP 2 orthogonaliser: GCGE_ORTH_ALG3 (RecursiveOrthSVD,
                               Algorithm 3) or GCGE_ORTH_ALG2 (modified block
                               orthogonalisation, Algorithm 2), Section 3.1        (ALG3) */
  int precond;              /* STEP 6 preconditioner (Section 2 suggests one):
                               GCGE_PRECOND_NONE or GCGE_PRECOND_JACOBI, M = |diag(A -
                               theta B)| of the shifted system, same shift       (NONE)  */
  int fp64_emulation;       /* 1: large FP64 Gram and V C products run on the bf16 tensor
                               cores from exact digit slices (gcge_gram_f64_tc); 0: the
                               FP64 kernels only                                       (1)   */
  int max_proj_dim;         /* moving mechanism (Section 3.3): largest dimension of the
                               projection subspace [X, P, W]; the X window is then
                               max_proj_dim - 2 blockSize columns. 0: 5 blockSize.
                               Must be >= 3 blockSize; ignored without moving.   (0)   */
} gcge_options;

#define GCGE_PRECOND_NONE 0
#define GCGE_PRECOND_JACOBI 1

#define GCGE_ORTH_ALG3 0      /* Algorithm 3: recursive halves, leaf M = W^T B W eigensolve */
#define GCGE_ORTH_ALG2 1      /* Algorithm 2: blocks of b = min(m/4, 200) columns, modified
                                 Gram-Schmidt inside a block, block deflation of the rest */

/* Kernel classes of the per-kernel profile in gcge_stats (profile = 1). */
#define GCGE_K_SPMM 0         /* FP32 CSR x block products (SpMM), incl. the CG SpMM + dot */
#define GCGE_K_GRAM 1         /* FP32 tall-skinny Gram X^T Y (tensor cores)               */
#define GCGE_K_VC 2           /* FP32 block update V C (tensor cores)                     */
#define GCGE_K_SYEV 3         /* dense Rayleigh-Ritz / leaf eigensolves                   */
#define GCGE_K_CGVEC 4        /* CG vector updates and reductions                         */
#define GCGE_K_OTHER 5        /* copies, residual reductions, small dense kernels         */
#define GCGE_K_SPMM64 6       /* FP64 SpMM                                                */
#define GCGE_K_GRAM64 7       /* FP64 Gram                                                */
#define GCGE_K_VC64 8         /* FP64 V C                                                 */
#define GCGE_K_GRAM64TC 9     /* FP64 Gram on the bf16 tensor cores (digit slices)        */
#define GCGE_K_VC64TC 10      /* FP64 V C on the bf16 tensor cores (digit slices)         */
#define GCGE_K_CLASSES 11

/* Per-solve statistics (times are CUDA-event milliseconds on the handle's stream). */
typedef struct {
  int iterations;           /* total GCG iterations (both phases)                     */
  int iterations_fp32;      /* of which in the FP32 phase (MIXED)                     */
  int nconv;                /* locked eigenpairs                                      */
  int64_t cg_steps;         /* total CG steps over all columns' blocks                */
  int moves;                /* moving-mechanism flushes                               */
  double ms_total;          /* gcge_solve wall time (events)                          */
  double ms_step[7];        /* time per STEP 1..6 of Algorithm 1 (index 0 unused)     */
  double ms_syev;           /* dense Rayleigh-Ritz eigensolve time (part of STEP 3)   */
  double max_orth_err;      /* largest |V^T B V - I| seen by the checks (if enabled)  */
  double max_abar_err;      /* largest |Abar - V^T A V| / max|V^T A V| (if enabled)   */
  int64_t kernel_launches;  /* kernels launched by the library during the solve       */
  /* per kernel class (GCGE_K_*), filled when options.profile = 1: summed CUDA-event
   * time of the launches, their count, and their algorithmic bytes and flops */
  double prof_ms[12];
  int64_t prof_calls[12];
  double prof_bytes[12];
  double prof_flops[12];
  int refills;              /* MIXED + moving: phase-1 vectors that refilled the FP64
                               phase's window beside W                                */
} gcge_stats;

/* ----------------------------------------------------------------- solver */

/* Fill `opt` with the defaults listed above.  Returns GCGE_EINVAL on NULL. */
int gcge_options_default(gcge_options *opt);

/* Create a solver for the smallest `nev` eigenpairs of (A, B).
 *   A      CSR, symmetric (Section 2).  Copied to the device.
 *   B      CSR, SPD, or NULL for B = I.  Copied to the device.
 *   nev    numEigen, 1 <= nev < n.
 *   block_size  blockSize (the paper's default is nev/5), 1 <= block_size <= nev.
 *   tol    relative residual ||A x - lambda B x|| / (|lambda| ||B^{1/2} x||) (Section 4).
 *   opt    NULL for defaults.
 *   stream cudaStream_t as void*, used by this call (device-resident A and B are
 *          read on it) and by every later call on this handle.
 *   out    receives the handle (NULL on failure).
 * The storage checks run on the device after the copy; the call returns when the
 * copies are complete.
 * Errors: EINVAL (bad sizes, or a malformed CSR: row_ptr not non-decreasing from 0
 * to nnz, a column outside [0, n), columns not strictly increasing within a row),
 * else ENAN (a value that is not finite), ENOMEM, ECUDA. */
int gcge_create(const gcge_csr *A, const gcge_csr *B, int nev, int block_size, double tol,
                const gcge_options *opt, void *stream, gcge_handle **out);

/* Run Algorithm 1 to convergence.  Blocks the calling thread until done.
 * Returns GCGE_OK, or ENOTCONV (partial results valid), or an error. */
int gcge_solve(gcge_handle *h);

/* Copy the converged eigenpairs out, ascending in lambda.
 *   evals  host array of nev doubles.
 *   evecs  NULL, or n x nev FP64 COLUMN-major with leading dimension ldv >= n,
 *          host memory (evecs_on_device = 0) or device memory (= 1).
 *          Eigenvectors are B-normalised (x^T B x = 1).
 *   nconv  receives the number of converged pairs (may exceed nev). */
int gcge_eigenpairs(gcge_handle *h, double *evals, double *evecs, int64_t ldv,
                    int evecs_on_device, int *nconv);

/* Statistics of the last gcge_solve. */
int gcge_stats_get(gcge_handle *h, gcge_stats *st);

/* Adjoint gradient of L = sum_i w_lambda[i] lambda_i + sum_i f_i(x_i) with respect
 * to the stored nonzeros of A (B held fixed), for the first `k` eigenpairs of the
 * last solve (not in the paper; first-order perturbation theory):
 *   dL/dA_pq = sum_i w_i x_ip x_iq - (mu_ip x_iq + x_ip mu_iq)/2,
 *   (A - lambda_i B) mu_i = (I - B x_i x_i^T) g_i,  x_i^T B mu_i = 0,
 * with g_i = d_gx[:, i] (device, n x k ROW-major, ld = ldg; NULL = no functional).
 *   w_lambda  host, k doubles (NULL = zeros).
 *   d_dA      device, nnz doubles, receives dL/dA on A's CSR pattern.
 *   adj_tol   relative tolerance of the projected CG adjoint solve (e.g. 1e-12).
 * Requires lambda_k < lambda_{k+1} (the deflated system is then SPD). */
int gcge_eig_grad(gcge_handle *h, int k, const double *w_lambda, const double *d_gx, int64_t ldg,
                  double *d_dA, double adj_tol);

/* Static text for a status code. */
const char *gcge_error_string(int status);

/* Detail of the most recent failure in this process (never NULL). */
const char *gcge_last_error_message(void);

/* Free every device and host resource of the handle (NULL is a no-op). */
void gcge_destroy(gcge_handle *h);

/* ----------------------------------------------------------------- kernels
 * The steps of the hot path, callable one by one on device buffers (used by the
 * parity tests; the solver calls the same kernels).  Each returns GCGE_EINVAL
 * on a bad size/pointer and GCGE_ECUDA on a launch failure.  Scratch memory
 * they need is allocated stream-ordered (cudaMallocAsync) and freed before
 * return. */

/* MatDotMultiVec (Section 3.4): Y = alpha * A X + beta * Y.
 * A: CSR on device (d_row_ptr n+1, d_col_idx nnz, d_val nnz); X: n x k
 * row-major (ldx), Y: n x k row-major (ldy); k >= 1.  X and Y must not overlap. */
int gcge_spmm_f64(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx,
                  const double *d_val, int k, double alpha, const double *d_X, int64_t ldx,
                  double beta, double *d_Y, int64_t ldy, void *stream);
int gcge_spmm_f32(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx,
                  const float *d_val, int k, float alpha, const float *d_X, int64_t ldx,
                  float beta, float *d_Y, int64_t ldy, void *stream);

/* MultiVecInnerProd into a strided sub-block (Section 3.4, Eq. Dense_SubMatrix):
 * C = alpha * X^T Y + beta * C, X n x m (ldx), Y n x k (ldy) row-major;
 * C m x k FP64 column-major at d_C with leading dimension ldc >= m.
 * The f32 form reads FP32 blocks (TF32 tensor cores with 3-term split
 * correction when tc != 0, else FP32 FMA) and accumulates partials in FP64. */
int gcge_gram_f64(int64_t n, int m, int k, double alpha, const double *d_X, int64_t ldx,
                  const double *d_Y, int64_t ldy, double beta, double *d_C, int64_t ldc,
                  void *stream);
int gcge_gram_f32(int64_t n, int m, int k, double alpha, const float *d_X, int64_t ldx,
                  const float *d_Y, int64_t ldy, double beta, double *d_C, int64_t ldc,
                  int tc, void *stream);

/* The X = V C update of STEPs 3/5 (and X_2 -= X_1 R of Algorithm 3):
 * Y = alpha * V C + beta * Y, V n x d row-major (ldv), C d x q FP64 column-major
 * (ldc), Y n x q row-major (ldy).  Y must not overlap V. */
int gcge_vc_f64(int64_t n, int d, int q, double alpha, const double *d_V, int64_t ldv,
                const double *d_C, int64_t ldc, double beta, double *d_Y, int64_t ldy,
                void *stream);
int gcge_vc_f32(int64_t n, int d, int q, double alpha, const float *d_V, int64_t ldv,
                const double *d_C, int64_t ldc, double beta, float *d_Y, int64_t ldy,
                int tc, void *stream);

/* The same FP64 products on the bf16 tensor cores (not in the paper: GB300 runs FP64
 * FMA at 1/64 of its FP32 rate).  Along the reduction dimension the operands are cut
 * into windows of 128 entries; each row of an operand gets one exponent per window
 * and is written as seven signed 7-bit digits (49 bits); the 28 digit-plane products
 * with the largest scales run as tcgen05 bf16 MMAs whose seven scale groups
 * accumulate exactly in FP32, and each window is summed into FP64.  The error of an
 * entry is about 2^-47 * 128 * sum over windows of max|x| max|y| (the window
 * maxima of the two operands), against about 2^-53 sqrt(n) sum |x||y| for the FP64
 * kernels.  Same arguments and layouts as gcge_gram_f64 / gcge_vc_f64; scratch
 * (about 14 bytes per operand entry, bounded per pass) is allocated
 * stream-ordered and freed before return.  n <= 2^30. */
int gcge_gram_f64_tc(int64_t n, int m, int k, double alpha, const double *d_X, int64_t ldx,
                     const double *d_Y, int64_t ldy, double beta, double *d_C, int64_t ldc,
                     void *stream);
int gcge_vc_f64_tc(int64_t n, int d, int q, double alpha, const double *d_V, int64_t ldv,
                   const double *d_C, int64_t ldc, double beta, double *d_Y, int64_t ldy,
                   void *stream);

/* Status of the tensor-core kernels (tc != 0 above, and the solver's FP32 phase):
 * synchronises `stream`, returns GCGE_ETIMEOUT if a kernel's bounded internal wait
 * ran out since the last call (that launch's output is invalid; the flag is then
 * cleared), else GCGE_OK.  Not part of the paper: the asynchronous entry points above
 * cannot return the status themselves. */
int gcge_tc_status(void *stream);

/* Dense symmetric eigensolve of STEP 3 (the paper's dsyevx role), FP64 on the
 * device by parallel cyclic Jacobi: d_A (d x d column-major, lda) is
 * overwritten; d_w receives the d eigenvalues ascending, d_Q (ldq) the
 * orthonormal eigenvectors (column j belongs to d_w[j]).  `sweeps` (host,
 * may be NULL) receives the number of Jacobi sweeps.  Synchronises the stream.
 * Returns GCGE_ETIMEOUT if a bounded grid barrier gave up. */
int gcge_syev(int d, double *d_A, int64_t lda, double *d_w, double *d_Q, int64_t ldq,
              int *sweeps, void *stream);

/* STEP 6 (Eq. compW): column-wise CG on S w_j = b_j with S = d_S (CSR, the
 * explicitly formed A - theta B), from the initial guess in d_X (n x k, ldx),
 * which is overwritten by the result; d_B is the n x k right-hand side (ldb).
 * Column j stops at ||r|| <= rtol ||r0||, after max_iter steps, or at a
 * breakdown p^T S p <= 0.  precond = GCGE_PRECOND_JACOBI runs preconditioned CG
 * with M = |diag(S)| (Section 2 suggests preconditioning STEP 6); the stop test
 * stays on the unpreconditioned ||r||.  iters (host, k ints, may be NULL)
 * receives the steps taken per column.  Synchronises the stream. */
int gcge_block_cg_f64(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx,
                      const double *d_S, int k, const double *d_B, int64_t ldb, double *d_X,
                      int64_t ldx, int max_iter, double rtol, int precond, int *iters,
                      void *stream);
int gcge_block_cg_f32(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx,
                      const float *d_S, int k, const float *d_B, int64_t ldb, float *d_X,
                      int64_t ldx, int max_iter, double rtol, int precond, int *iters,
                      void *stream);

/* STEP 2 (Section 3.1): B-orthonormalise the n x m block d_W (row-major, ldw,
 * overwritten) against the B-orthonormal block d_Q (n x q, ldq; q may be 0), then
 * by Algorithm 3 with leaf width min(m, leaf) (orth = GCGE_ORTH_ALG3) or by
 * Algorithm 2, modified block orthogonalisation with blocks of min(m/4, 200)
 * columns (orth = GCGE_ORTH_ALG2).  B is CSR on the device or all three pointers
 * NULL for B = I.  m_out (host) receives the number of columns kept (dependent
 * ones are removed and the rest compacted to the left).  Synchronises the stream. */
int gcge_borth_f64(int64_t n, const int32_t *d_Brp, const int32_t *d_Bci, const double *d_Bval,
                   const double *d_Q, int64_t ldq, int q, double *d_W, int64_t ldw, int m,
                   int leaf, int orth, int *m_out, void *stream);

/* Gram product without any device allocation (the paper has no counterpart; it
 * exists for callers that cannot allocate while they run -- e.g. their own allocator
 * has reserved the GPU's memory, or cudaMalloc/cudaFree's synchronisation is not
 * acceptable in their loop).  Same arguments and result as gcge_gram_f64, all
 * pointers device memory.  Its split-K partial sums live in one static device array
 * of GCGE_GRAM_NOALLOC_MAX_DOUBLES doubles (16 MiB) that every GPU loading the
 * library holds until exit.
 *   - m * k must be <= GCGE_GRAM_NOALLOC_MAX_DOUBLES, else GCGE_EINVAL (with a
 *     message in gcge_last_error_message()); larger m * k uses fewer row splits.
 *   - The first call on a device looks up the array's device address on that
 *     device; make that first call before any stream capture.
 *   - All calls share the one array: calls that may overlap on the GPU (different
 *     streams, concurrent threads) race and must be serialised by the caller.
 *   - Calls no cudaMalloc/cudaFree or other allocating routine. */
#define GCGE_GRAM_NOALLOC_MAX_DOUBLES (2 * 1024 * 1024)
int gcge_gram_f64_noalloc(int64_t n, int m, int k, double alpha, const double *d_X, int64_t ldx,
                          const double *d_Y, int64_t ldy, double beta, double *d_C, int64_t ldc,
                          void *stream);

/* N(0,1) block from the counter-based generator: entry (i, j) of the n x k
 * row-major block (ld) uses counter i*k + j; u1, u2 from
 * splitmix64(splitmix64(seed) + 2c) and (... + 2c + 1), z = sqrt(-2 ln u1) cos(2 pi u2). */
int gcge_random_block_f64(int64_t n, int k, uint64_t seed, double *d_X, int64_t ld, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GCGE_H */
