// STEP 6: column-wise CG on the explicitly shifted matrix S = A - theta B -- internal.
#pragma once
#include "blas.cuh"
#include "spmm.cuh"
#include "prof.cuh"

namespace gcge {

// Device work area of the block CG for k columns of length n.
template <typename T>
struct CgWork {
  T *r = nullptr, *p = nullptr, *q = nullptr;   // n x ld each
  int64_t ld = 0;
  double *part_a = nullptr;   // SpMM dot partials  (nbcap x k)
  double *part_b = nullptr;   // vector-kernel partials (nbcap x 2k)
  double *scal = nullptr;     // 6k: rr, r0, pq, rrn, rz, rzn
  double *rr = nullptr, *r0 = nullptr, *pq = nullptr, *rrn = nullptr;
  double *rz = nullptr, *rzn = nullptr;   // r^T M^-1 r (equal to rr without a preconditioner)
  int *flags = nullptr;       // 3k: active, iters, broke
  int *active = nullptr, *iters = nullptr, *broke = nullptr;
  unsigned *tickets = nullptr;   // last-CTA tickets of the reductions (kept at zero)
  int *h_active = nullptr;    // pinned host mirror (k)
  int kcap = 0, nbcap = 0;
  int64_t ncap = 0;
  int alloc(int64_t n, int k);
  void free_all();
};

// Run CG on S x_j = b_j for the k columns of X (row-major n x k, ldx), in place.
// If `r_init` is non-null it holds the initial residual b - S X (n x k, ldr) and B
// is not read; otherwise B (ldb) is the right-hand side and r = B - S X is formed.
// Stops per column at ||r|| <= rtol ||r0||, max_iter steps, or p^T S p <= 0.
// iters_host (k ints, may be null) receives the step counts; returns the max.
// minv (n entries, may be null): Jacobi preconditioner M^-1 = 1 / |diag(S)|; the
// recurrences then use r^T M^-1 r and the stop test the unpreconditioned ||r||.
template <typename T>
int block_cg(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, int k, const T *B,
             int64_t ldb, const T *r_init, int64_t ldr, T *X, int64_t ldx, int max_iter,
             double rtol, CgWork<T> &w, int *iters_host, int64_t *launches, cudaStream_t st,
             KProf *prof = nullptr, const T *minv = nullptr);

// minv[i] = 1 / |S_ii| (1 where the diagonal entry is absent or zero); S is CSR with
// sorted column indices.
template <typename T>
int jacobi_inverse(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, T *minv,
                   cudaStream_t st);

}  // namespace gcge
