// Adjoint gradients of eigenvalues and eigenvector functionals (not in the paper).
//
// For A(theta) x_i = lambda_i B x_i with B fixed and x_i^T B x_i = 1, and
// L = sum_i w_i lambda_i + sum_i f_i(x_i) with g_i = df_i/dx_i:
//   dL/dA_pq = sum_i w_i x_ip x_iq - (mu_ip x_iq + x_ip mu_iq)/2,
// where the adjoint mu_i solves (A - lambda_i B) mu_i = (I - B x_i x_i^T) g_i with
// x_i^T B mu_i = 0.  With X = [x_1 .. x_k] (the computed pairs, lambda_k < lambda_{k+1}):
//   mu_i = sum_{j != i} x_j (x_j^T g_i)/(lambda_j - lambda_i) + P z_i,
// P = I - X X^T B, and z_i from CG on the symmetric operator P^T (A - lambda_i B) P with
// right-hand side P^T g_i (SPD on the B-complement of span X).  All k columns run
// together with per-column shifts and scalars; every product is a library kernel
// (SpMM, Gram, V C, column reductions).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "solver.cuh"

namespace gcge {
namespace {

// C[j + i*ldc] = G[j + i*ldg] / (lam[j] - lam[i]) for j != i, 0 on the diagonal.
__global__ void deflation_coeff_kernel(int k, const double *__restrict__ G, int64_t ldg,
                                       const double *__restrict__ lam, double *__restrict__ C,
                                       int64_t ldc) {
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int j = t % k, i = t / k;
    C[j + (int64_t)i * ldc] = (j == i) ? 0.0 : G[j + (int64_t)i * ldg] / (lam[j] - lam[i]);
  }
}

// y[:, j] += a[j] x[:, j]
__global__ void axpy_cols_kernel(int64_t n, int k, const double *__restrict__ a,
                                 const double *__restrict__ x, int64_t ldx, double *__restrict__ y,
                                 int64_t ldy) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    y[r * ldy + j] += a[j] * x[r * ldx + j];
  }
}

// p[:, j] = r[:, j] + b[j] p[:, j]
__global__ void xpby_cols_kernel(int64_t n, int k, const double *__restrict__ r, int64_t ldr,
                                 const double *__restrict__ b, double *__restrict__ p,
                                 int64_t ldp) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / k;
    const int j = (int)(t % k);
    p[row * ldp + j] = r[row * ldr + j] + b[j] * p[row * ldp + j];
  }
}

// w = Au - lam_j Bu (per column)
__global__ void shift_combine_kernel(int64_t n, int k, const double *__restrict__ Au,
                                     const double *__restrict__ Bu, int64_t ld,
                                     const double *__restrict__ lam, double *__restrict__ w) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    w[r * ld + j] = Au[r * ld + j] - lam[j] * Bu[r * ld + j];
  }
}

// alpha_j = rr_j / pq_j on active columns (else 0); minus_alpha for the residual.
__global__ void cg_alpha_kernel(int k, const double *__restrict__ rr, const double *__restrict__ pq,
                                const int *__restrict__ active, double *__restrict__ alpha,
                                double *__restrict__ malpha) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double a = (active[j] && pq[j] > 0.0) ? rr[j] / pq[j] : 0.0;
    alpha[j] = a;
    malpha[j] = -a;
  }
}

__global__ void cg_beta_kernel(int k, double *__restrict__ rr, const double *__restrict__ rrn,
                               const double *__restrict__ r0, int *__restrict__ active,
                               double *__restrict__ beta, double tol) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    if (!active[j]) {
      beta[j] = 0.0;
      continue;
    }
    beta[j] = rrn[j] / rr[j];
    rr[j] = rrn[j];
    if (sqrt(rrn[j]) <= tol * r0[j]) active[j] = 0;
  }
}

__global__ void cg_start_kernel(int k, const double *__restrict__ rr, double *__restrict__ r0,
                                int *__restrict__ active) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    r0[j] = sqrt(rr[j]);
    active[j] = rr[j] > 0.0 ? 1 : 0;
  }
}

// dA[e] for every stored nonzero (p, q) of A.
__global__ void grad_nnz_kernel(int64_t n, const int32_t *__restrict__ rp,
                                const int32_t *__restrict__ ci, int k,
                                const double *__restrict__ X, const double *__restrict__ MU,
                                int64_t ld, const double *__restrict__ w, int has_mu,
                                double *__restrict__ out) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const double *xp = X + row * ld;
    const double *mp = MU + row * ld;
    for (int e = rp[row]; e < rp[row + 1]; ++e) {
      const int64_t q = ci[e];
      const double *xq = X + q * ld;
      const double *mq = MU + q * ld;
      double s = 0.0;
      for (int i = 0; i < k; ++i) {
        s += w[i] * xp[i] * xq[i];
        if (has_mu) s -= 0.5 * (mp[i] * xq[i] + xp[i] * mq[i]);
      }
      out[e] = s;
    }
  }
}

int egrid(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

struct GradBufs {
  std::vector<void *> ptrs;
  ~GradBufs() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  int get(T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
      record_cuda_error(e, __FILE__, __LINE__);
      return GCGE_ENOMEM;
    }
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return GCGE_OK;
  }
};

}  // namespace
}  // namespace gcge

using namespace gcge;

extern "C" int gcge_eig_grad(gcge_handle *h, int k, const double *w_lambda, const double *d_gx,
                             int64_t ldg, double *d_dA, double adj_tol) {
  if (!h || k < 1 || !d_dA || (d_gx && ldg < k)) return GCGE_EINVAL;
  if (!h->solved) return GCGE_ENOTREADY;
  if (k > (int)h->lam.size()) return GCGE_EINVAL;
  cudaStream_t st = h->st;
  const int64_t n = h->n;
  const bool bI = h->B.n == 0;
  // the k lowest computed pairs, ascending
  std::vector<int> perm(h->lam.size());
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return h->lam[a] < h->lam[b]; });
  std::vector<double> lamk(k), wv(k, 0.0);
  for (int i = 0; i < k; ++i) lamk[i] = h->lam[perm[i]];
  if (w_lambda)
    for (int i = 0; i < k; ++i) wv[i] = w_lambda[i];
  const int64_t ld = round_up(k, 4);
  GradBufs gb;
  double *X, *BX, *MU, *Z, *R, *P, *U, *AU, *BU, *Wv, *Q;
  double *d_lam, *d_w, *G1, *Cc, *Rs, *dots;
  int *idx, *active;
  const size_t nb = (size_t)n * ld;
  GCGE_CHECK(gb.get(&X, nb));
  GCGE_CHECK(gb.get(&BX, nb));
  GCGE_CHECK(gb.get(&MU, nb));
  GCGE_CHECK(gb.get(&idx, k));
  GCGE_CHECK(gb.get(&d_lam, k));
  GCGE_CHECK(gb.get(&d_w, k));
  GCGE_CHECK(gb.get(&G1, (size_t)k * k));
  GCGE_CHECK(gb.get(&Cc, (size_t)k * k));
  GCGE_CUDA(cudaMemcpyAsync(idx, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, st));
  GCGE_CUDA(cudaMemcpyAsync(d_lam, lamk.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
  GCGE_CUDA(cudaMemcpyAsync(d_w, wv.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
  GCGE_CHECK(gather_cols<double>(n, k, idx, h->store, h->ld_store, X, ld, st));
  GCGE_CUDA(cudaMemsetAsync(MU, 0, sizeof(double) * nb, st));
  Scratch ws;
  auto spA = [&](const double *x, double *y) {
    return launch_spmm<double>(n, h->A.rp, h->A.ci, h->A.v64, k, 1.0, x, ld, 0.0, y, ld, nullptr,
                               0, st);
  };
  auto spB = [&](const double *x, double *y) {
    if (bI) return copy_cols<double, double>(n, k, x, ld, y, ld, nullptr, st);
    return launch_spmm<double>(n, h->B.rp, h->B.ci, h->B.v64, k, 1.0, x, ld, 0.0, y, ld, nullptr,
                               0, st);
  };
  GCGE_CHECK(spB(X, BX));
  int status = GCGE_OK;
  if (d_gx) {
    GCGE_CHECK(gb.get(&Z, nb));
    GCGE_CHECK(gb.get(&R, nb));
    GCGE_CHECK(gb.get(&P, nb));
    GCGE_CHECK(gb.get(&U, nb));
    GCGE_CHECK(gb.get(&AU, nb));
    GCGE_CHECK(gb.get(&BU, nb));
    GCGE_CHECK(gb.get(&Wv, nb));
    GCGE_CHECK(gb.get(&Q, nb));
    GCGE_CHECK(gb.get(&Rs, (size_t)k * k));
    GCGE_CHECK(gb.get(&dots, 8 * (size_t)k));
    GCGE_CHECK(gb.get(&active, k));
    double *rr = dots, *rrn = dots + k, *pq = dots + 2 * k, *r0 = dots + 3 * k;
    double *alpha = dots + 4 * k, *malpha = dots + 5 * k, *beta = dots + 6 * k;
    // explicit part over the computed pairs: MU = X C, C_ji = (x_j^T g_i)/(lam_j - lam_i)
    GCGE_CHECK(copy_cols<double, double>(n, k, d_gx, ldg, R, ld, nullptr, st));
    GCGE_CHECK(gram<double>(n, k, k, 1.0, X, ld, R, ld, 0.0, G1, k, 0, ws, st));
    deflation_coeff_kernel<<<1, 256, 0, st>>>(k, G1, k, d_lam, Cc, k);
    GCGE_LAUNCH_CHECK();
    GCGE_CHECK(vc<double>(n, k, k, 1.0, X, ld, Cc, k, 0.0, MU, ld, 0, st));
    // r = P^T g = g - B X (X^T g)
    GCGE_CHECK(vc<double>(n, k, k, -1.0, BX, ld, G1, k, 1.0, R, ld, 0, st));
    GCGE_CUDA(cudaMemsetAsync(Z, 0, sizeof(double) * nb, st));
    GCGE_CHECK(copy_cols<double, double>(n, k, R, ld, P, ld, nullptr, st));
    GCGE_CHECK(col_dots<double>(n, k, R, ld, R, ld, rr, ws, st));
    cg_start_kernel<<<1, 256, 0, st>>>(k, rr, r0, active);
    GCGE_LAUNCH_CHECK();
    std::vector<int> hact(k);
    const int max_it = 50000;
    int it = 0;
    for (; it < max_it; ++it) {
      // u = P p
      GCGE_CHECK(spB(P, BU));
      GCGE_CHECK(gram<double>(n, k, k, 1.0, X, ld, BU, ld, 0.0, Rs, k, 0, ws, st));
      GCGE_CHECK(copy_cols<double, double>(n, k, P, ld, U, ld, nullptr, st));
      GCGE_CHECK(vc<double>(n, k, k, -1.0, X, ld, Rs, k, 1.0, U, ld, 0, st));
      // w = (A - lam B) u, q = P^T w
      GCGE_CHECK(spA(U, AU));
      GCGE_CHECK(spB(U, BU));
      shift_combine_kernel<<<egrid(n * k), 256, 0, st>>>(n, k, AU, BU, ld, d_lam, Wv);
      GCGE_LAUNCH_CHECK();
      GCGE_CHECK(gram<double>(n, k, k, 1.0, X, ld, Wv, ld, 0.0, Rs, k, 0, ws, st));
      GCGE_CHECK(copy_cols<double, double>(n, k, Wv, ld, Q, ld, nullptr, st));
      GCGE_CHECK(vc<double>(n, k, k, -1.0, BX, ld, Rs, k, 1.0, Q, ld, 0, st));
      // CG scalars and updates (per column)
      GCGE_CHECK(col_dots<double>(n, k, P, ld, Q, ld, pq, ws, st));
      cg_alpha_kernel<<<1, 256, 0, st>>>(k, rr, pq, active, alpha, malpha);
      GCGE_LAUNCH_CHECK();
      axpy_cols_kernel<<<egrid(n * k), 256, 0, st>>>(n, k, alpha, P, ld, Z, ld);
      axpy_cols_kernel<<<egrid(n * k), 256, 0, st>>>(n, k, malpha, Q, ld, R, ld);
      GCGE_LAUNCH_CHECK();
      GCGE_CHECK(col_dots<double>(n, k, R, ld, R, ld, rrn, ws, st));
      cg_beta_kernel<<<1, 256, 0, st>>>(k, rr, rrn, r0, active, beta, adj_tol);
      xpby_cols_kernel<<<egrid(n * k), 256, 0, st>>>(n, k, R, ld, beta, P, ld);
      GCGE_LAUNCH_CHECK();
      if (it % 10 == 9) {
        GCGE_CUDA(cudaMemcpyAsync(hact.data(), active, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
        GCGE_CUDA(cudaStreamSynchronize(st));
        bool any = false;
        for (int j = 0; j < k; ++j) any |= hact[j] != 0;
        if (!any) break;
      }
    }
    if (it >= max_it) status = GCGE_ENOTCONV;
    // MU += P z
    GCGE_CHECK(spB(Z, BU));
    GCGE_CHECK(gram<double>(n, k, k, 1.0, X, ld, BU, ld, 0.0, Rs, k, 0, ws, st));
    GCGE_CHECK(vc<double>(n, k, k, -1.0, X, ld, Rs, k, 1.0, Z, ld, 0, st));
    GCGE_CHECK(add_cols<double, double>(n, k, Z, ld, MU, ld, st));
  }
  grad_nnz_kernel<<<egrid(n), 256, 0, st>>>(n, h->A.rp, h->A.ci, k, X, MU, ld, d_w, d_gx ? 1 : 0,
                                            d_dA);
  GCGE_LAUNCH_CHECK();
  GCGE_CUDA(cudaStreamSynchronize(st));
  ws.release(st);
  GCGE_CUDA(cudaStreamSynchronize(st));
  return status;
}
