// Dense FP64 symmetric eigensolver on the device (STEP 3's dsyevx role) -- internal.
#pragma once
#include "common.cuh"

namespace gcge {

// Work area of the mixed-precision eigensolver (FP32 cluster Jacobi + FP64 polish).
struct MpWork {
  float *V32 = nullptr, *gn = nullptr;
  double *V = nullptr, *T1 = nullptr, *T2 = nullptr, *Bm = nullptr, *lam = nullptr;
  double *dinfo = nullptr;
  int *ints = nullptr;
  double *h = nullptr;
  int *hi = nullptr;
  int dcap = 0;
  int alloc(int d);
  void free_all();
};

struct SyevWork {
  double *rot = nullptr;      // 3 * D/2 rotation parameters of one round
  double *V = nullptr;        // d x d accumulated rotations (column-major, ld = dcap)
  unsigned *sync = nullptr;   // [0]=barrier count, [1]=barrier generation, [2..4]=rotation counters
  int *flags = nullptr;       // [0]=barrier timeout, [1]=NaN seen, [2]=sweeps
  int *h_flags = nullptr;     // pinned mirror of flags
  int dcap = 0;
  int coop_grid = 0;          // co-resident CTAs for the cooperative launch
  MpWork mp;                  // mixed-precision path
  int mixed = 1;              // 1: try the mixed-precision path for d > 32
  int alloc(int d);
  void free_all();
};

// Mixed-precision eigensolve of the symmetric A (not modified); GCGE_EINVAL when it
// does not apply (size, a cluster of near-equal eigenvalues wider than 32, or no
// convergence), in which case the caller uses the FP64 Jacobi.
// off_tol: the refinement stops once the largest off-diagonal of V^T A V is below
// off_tol of its largest diagonal entry (1e-13: FP64 eigenvectors).
int syev_mixed(int d, const double *A, int64_t lda, double *w, double *Q, int64_t ldq,
               MpWork &mw, int *flags_dev, int *sweeps, cudaStream_t st,
               double off_tol = 1e-13);

// A (d x d col-major, lda) is destroyed; w[d] ascending; Q (ldq) eigenvectors.
// Synchronises the stream.  Returns GCGE_OK / GCGE_ETIMEOUT / GCGE_ENAN / GCGE_ECUDA.
// fp32_data: A was formed from FP32 blocks (entries accurate to about 1e-7): matrices
// of order <= 32 are diagonalised in FP32 arithmetic and larger ones refined to 1e-10
// instead of 1e-13; results are returned in FP64 either way.
int syev(int d, double *A, int64_t lda, double *w, double *Q, int64_t ldq, SyevWork &work,
         int *sweeps, cudaStream_t st, bool fp32_data = false);

}  // namespace gcge
