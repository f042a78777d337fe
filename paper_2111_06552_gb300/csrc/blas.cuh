// Tall-skinny block products and small dense helpers -- internal.
#pragma once
#include "common.cuh"

namespace gcge {

// Stream-ordered scratch arena owned by a caller (a solver handle, or one
// API call).  Buffers grow on demand; nothing is freed until release().
struct Scratch {
  void *ptr = nullptr;
  size_t bytes = 0;
  int get(size_t need, cudaStream_t st, void **out);
  void release(cudaStream_t st);
};

// C(m x k, col-major ldc) = alpha * X^T Y + beta * C, X: n x m row-major, Y: n x k
// row-major.  Split over row chunks; FP64 partials reduced in a fixed order.
// For T = float, `tc` selects the TF32 tensor-core kernel (3-term split).
template <typename T>
int gram(int64_t n, int m, int k, double alpha, const T *X, int64_t ldx, const T *Y, int64_t ldy,
         double beta, double *C, int64_t ldc, int tc, Scratch &ws, cudaStream_t st);

// The SIMT Gram kernels tile k in 32-column tiles on grid.y (at most 65535 tiles).
inline bool gram_f64_grid_ok(int m, int k) {
  (void)m;
  return (k + 31) / 32 <= 65535;
}

// Same product as gram() for FP64 blocks, with a caller-owned partial-sum workspace of
// `ws_doubles` doubles instead of an allocated one (fewer row splits when it is small).
// Returns GCGE_EINVAL when even one split (m * k doubles) does not fit.
int gram_f64_workspace(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx,
                       const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                       double *ws, int64_t ws_doubles, cudaStream_t st);

// FP64 Gram and V C on the bf16 tensor cores from exact 7-bit digit slices (oz.cu):
// same arguments and layouts as gram<double> / vc<double>.  GCGE_EINVAL when the shape
// is outside what the kernels take (n > 2^30, no tensor-map encoder).
int oz_gram(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx, const double *Y,
            int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st);
int oz_vc(int64_t n, int d, int q, double alpha, const double *V, int64_t ldv, const double *C,
          int64_t ldc, double beta, double *Y, int64_t ldy, Scratch &ws, cudaStream_t st);

// Y(n x q) = alpha * V(n x d) C(d x q col-major FP64) + beta * Y.
// `ws` (optional) holds the split operand of the tensor-core path.
template <typename T>
int vc(int64_t n, int d, int q, double alpha, const T *V, int64_t ldv, const double *C,
       int64_t ldc, double beta, T *Y, int64_t ldy, int tc, cudaStream_t st,
       Scratch *ws = nullptr);

// Error flag of the tensor-core kernels (1 once a bounded mbarrier wait ran out).
int tc_error_flag(int *host_val, cudaStream_t st);

// Small dense FP64 column-major GEMM: C = alpha op(A) op(B) + beta C.
int dgemm_small(char ta, char tb, int m, int n, int k, double alpha, const double *A, int64_t lda,
                const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                cudaStream_t st);

// Per-column sums over rows of X .* Y (row-major n x k), FP64 result in out[k] (device).
template <typename T>
int col_dots(int64_t n, int k, const T *X, int64_t ldx, const T *Y, int64_t ldy, double *out,
             Scratch &ws, cudaStream_t st);

// Residual pieces of STEP 4 for m columns: res2[j] = ||AX_j - lam_j BX_j||^2,
// xbx[j] = X_j^T BX_j (out[0:m] and out[m:2m], device FP64).  BX == nullptr means B = I (BX = X).
template <typename T>
int residual_parts(int64_t n, int m, const T *X, int64_t ldx, const T *AX, int64_t lda,
                   const T *BX, int64_t ldb, const double *lam, double *out, Scratch &ws,
                   cudaStream_t st);

// Y[:, 0:k] = X[:, 0:k] * s[j] (device scale vector, FP64), converting precision.
template <typename TI, typename TO>
int copy_cols(int64_t n, int k, const TI *X, int64_t ldx, TO *Y, int64_t ldy, const double *s,
              cudaStream_t st);

// out = a[j] * P + b[j] * Q columnwise (device coefficient vectors, may be null = 1/0).
template <typename T>
int axpby_cols(int64_t n, int k, const double *a, const T *P, int64_t ldp, const double *b,
               const T *Q, int64_t ldq, T *out, int64_t ldo, cudaStream_t st);

// Y[:, 0:k] += X[:, 0:k] (X of type TI added in the precision of Y).
template <typename TI, typename TO>
int add_cols(int64_t n, int k, const TI *X, int64_t ldx, TO *Y, int64_t ldy, cudaStream_t st);

// Gather columns: Y[:, t] = X[:, idx[t]] for t < k (device idx).
template <typename T>
int gather_cols(int64_t n, int k, const int *idx, const T *X, int64_t ldx, T *Y, int64_t ldy,
                cudaStream_t st);

// N(0,1) block from the counter-based generator (splitmix64 + Box-Muller).
template <typename T>
int random_block(int64_t n, int k, uint64_t seed, T *X, int64_t ld, cudaStream_t st);

// values of S = A - theta B on the union pattern (mapA/mapB give each union
// nonzero's position in A / B, -1 if absent; B = I is mapB == nullptr with diag flag).
template <typename T>
int shifted_values(int64_t nnz_u, const int *mapA, const double *valA, const int *mapB,
                   const double *valB, const int *is_diag, double theta, T *out,
                   cudaStream_t st);

}  // namespace gcge
