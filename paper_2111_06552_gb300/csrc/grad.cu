// Adjoint gradients of eigenvalues and eigenvector functionals (not in the paper).
#include "solver.cuh"

extern "C" int gcge_eig_grad(gcge_handle *h, int k, const double *w_lambda, const double *d_gx,
                             int64_t ldg, double *d_dA, double adj_tol) {
  (void)w_lambda; (void)d_gx; (void)ldg; (void)adj_tol;
  if (!h || k < 1 || !d_dA) return GCGE_EINVAL;
  if (!h->solved) return GCGE_ENOTREADY;
  gcge::record_message("gcge_eig_grad: not available in this build");
  return GCGE_EINVAL;
}
