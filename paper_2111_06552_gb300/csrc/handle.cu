// Solver handle: gcge_create / gcge_solve / gcge_eigenpairs / gcge_stats_get / gcge_destroy.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "solver.cuh"

namespace gcge {

template <typename T>
class Engine;

// Engine is defined in solver.cu; these thin entry points instantiate it there.
int run_fp64(gcge_handle *h, const double *X0d, int64_t ld0, int *iters);
int run_mixed(gcge_handle *h, const double *X0d, int64_t ld0, int *iters, int *iters32);

namespace {

struct HostCsr {
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> val;
};

int fetch_csr(const gcge_csr *m, HostCsr &out) {
  out.n = m->n;
  out.nnz = m->nnz;
  out.rp.resize(m->n + 1);
  out.ci.resize(m->nnz);
  out.val.resize(m->nnz);
  const cudaMemcpyKind kind = m->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  GCGE_CUDA(cudaMemcpy(out.rp.data(), m->row_ptr, sizeof(int32_t) * (m->n + 1), kind));
  if (m->nnz > 0) {
    GCGE_CUDA(cudaMemcpy(out.ci.data(), m->col_idx, sizeof(int32_t) * m->nnz, kind));
    GCGE_CUDA(cudaMemcpy(out.val.data(), m->val, sizeof(double) * m->nnz, kind));
  }
  return GCGE_OK;
}

int validate(const HostCsr &m) {
  if (m.rp[0] != 0 || m.rp[m.n] != m.nnz) return GCGE_EINVAL;
  for (int64_t i = 0; i < m.n; ++i) {
    if (m.rp[i + 1] < m.rp[i]) return GCGE_EINVAL;
    for (int64_t e = m.rp[i]; e < m.rp[i + 1]; ++e) {
      const int32_t c = m.ci[e];
      if (c < 0 || c >= m.n) return GCGE_EINVAL;
      if (e > m.rp[i] && c <= m.ci[e - 1]) return GCGE_EINVAL;   // sorted, no duplicates
      if (!std::isfinite(m.val[e])) return GCGE_ENAN;
    }
  }
  return GCGE_OK;
}

int upload(const HostCsr &m, DevCsr &d, bool want32) {
  d.n = m.n;
  d.nnz = m.nnz;
  GCGE_CUDA(cudaMalloc(&d.rp, sizeof(int32_t) * (m.n + 1)));
  GCGE_CUDA(cudaMalloc(&d.ci, sizeof(int32_t) * std::max<int64_t>(m.nnz, 1)));
  GCGE_CUDA(cudaMalloc(&d.v64, sizeof(double) * std::max<int64_t>(m.nnz, 1)));
  GCGE_CUDA(cudaMemcpy(d.rp, m.rp.data(), sizeof(int32_t) * (m.n + 1), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(d.ci, m.ci.data(), sizeof(int32_t) * m.nnz, cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(d.v64, m.val.data(), sizeof(double) * m.nnz, cudaMemcpyHostToDevice));
  if (want32) {
    std::vector<float> f(m.val.begin(), m.val.end());
    GCGE_CUDA(cudaMalloc(&d.v32, sizeof(float) * std::max<int64_t>(m.nnz, 1)));
    GCGE_CUDA(cudaMemcpy(d.v32, f.data(), sizeof(float) * m.nnz, cudaMemcpyHostToDevice));
  }
  return GCGE_OK;
}

// Union pattern of A and B (or A and the diagonal when B = I) with the position of
// each union entry in A and in B (-1 when absent), for S = A - theta B.
int build_union(const HostCsr &A, const HostCsr *B, gcge_handle *h) {
  const int64_t n = A.n;
  std::vector<int32_t> rp(n + 1, 0), ci;
  std::vector<int> mA, mB, dg;
  ci.reserve(A.nnz + n);
  mA.reserve(A.nnz + n);
  mB.reserve(A.nnz + n);
  dg.reserve(A.nnz + n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t a = A.rp[i], ae = A.rp[i + 1];
    int64_t b = 0, be = 0;
    if (B) {
      b = B->rp[i];
      be = B->rp[i + 1];
    }
    bool diag_done = false;
    while (a < ae || (B ? b < be : !diag_done)) {
      const int64_t ca = a < ae ? A.ci[a] : INT64_MAX;
      int64_t cb;
      if (B)
        cb = b < be ? B->ci[b] : INT64_MAX;
      else
        cb = diag_done ? INT64_MAX : i;
      const int64_t c = std::min(ca, cb);
      ci.push_back((int32_t)c);
      mA.push_back(ca == c ? (int)a : -1);
      if (B) {
        mB.push_back(cb == c ? (int)b : -1);
        if (cb == c) ++b;
      } else {
        if (cb == c) diag_done = true;
      }
      dg.push_back(c == i ? 1 : 0);
      if (ca == c) ++a;
    }
    rp[i + 1] = (int32_t)ci.size();
  }
  h->S.n = n;
  h->S.nnz = (int64_t)ci.size();
  GCGE_CUDA(cudaMalloc(&h->S.rp, sizeof(int32_t) * (n + 1)));
  GCGE_CUDA(cudaMalloc(&h->S.ci, sizeof(int32_t) * ci.size()));
  GCGE_CUDA(cudaMalloc(&h->mapA, sizeof(int) * ci.size()));
  GCGE_CUDA(cudaMalloc(&h->isdiag, sizeof(int) * ci.size()));
  GCGE_CUDA(cudaMemcpy(h->S.rp, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->S.ci, ci.data(), sizeof(int32_t) * ci.size(), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->mapA, mA.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->isdiag, dg.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  if (B) {
    GCGE_CUDA(cudaMalloc(&h->mapB, sizeof(int) * ci.size()));
    GCGE_CUDA(cudaMemcpy(h->mapB, mB.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  }
  return GCGE_OK;
}

void free_handle(gcge_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  h->A.free_all();
  h->B.free_all();
  h->S.free_all();
  cudaFree(h->mapA);
  cudaFree(h->mapB);
  cudaFree(h->isdiag);
  cudaFree(h->store);
  h->mapA = h->mapB = h->isdiag = nullptr;
  h->store = nullptr;
}

__global__ void transpose_out_kernel(int64_t n, int k, const int *__restrict__ perm,
                                     const double *__restrict__ S, int64_t lds,
                                     double *__restrict__ out, int64_t ldo) {
  // out (n x k, column-major ldo) column t = store column perm[t]
  const int64_t tot = n * k;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < tot;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = u % n;
    const int t = (int)(u / n);
    out[r + (int64_t)t * ldo] = S[r * lds + perm[t]];
  }
}

}  // namespace
}  // namespace gcge

using namespace gcge;

extern "C" {

int gcge_options_default(gcge_options *o) {
  if (!o) return GCGE_EINVAL;
  o->precision = GCGE_FP64;
  o->cg_max_iter = 30;
  o->cg_rtol = 1e-2;
  o->use_shift = 1;
  o->orth_leaf = 16;
  o->moving = -1;
  o->size_x = 0;
  o->max_iter = 2000;
  o->seed = 0;
  o->initial_block = nullptr;
  o->mixed_switch_tol = 3e-6;
  o->mixed_bs2 = 0;
  o->verbose = 0;
  o->checks = 0;
  o->profile = 0;
  return GCGE_OK;
}

int gcge_create(const gcge_csr *A, const gcge_csr *B, int nev, int block_size, double tol,
                const gcge_options *opt, void *stream, gcge_handle **out) {
  if (!out) return GCGE_EINVAL;
  *out = nullptr;
  if (!A || A->n < 2 || A->nnz < 1 || !A->row_ptr || !A->col_idx || !A->val) return GCGE_EINVAL;
  if (nev < 1 || nev >= A->n || block_size < 1 || block_size > nev || !(tol > 0.0))
    return GCGE_EINVAL;
  if (B && (B->n != A->n || B->nnz < 1 || !B->row_ptr || !B->col_idx || !B->val))
    return GCGE_EINVAL;
  gcge_handle *h = new gcge_handle();
  if (opt)
    h->opt = *opt;
  else
    gcge_options_default(&h->opt);
  if (h->opt.cg_max_iter < 0 || h->opt.orth_leaf < 1 || h->opt.max_iter < 1 ||
      h->opt.mixed_bs2 < 0 ||
      (h->opt.precision != GCGE_FP64 && h->opt.precision != GCGE_MIXED)) {
    delete h;
    return GCGE_EINVAL;
  }
  h->st = reinterpret_cast<cudaStream_t>(stream);
  h->n = A->n;
  h->nev = nev;
  h->bs = block_size;
  h->tol = tol;
  h->moving = h->opt.moving == 1 || (h->opt.moving < 0 && nev >= 500);
  int sx = h->opt.size_x;
  if (sx <= 0) sx = h->moving ? 3 * block_size : nev + 3 * block_size;
  if (sx > A->n) sx = (int)A->n;
  if (sx < block_size || (!h->moving && sx < nev)) {
    delete h;
    return GCGE_EINVAL;
  }
  h->size_x = sx;
  const bool want32 = h->opt.precision == GCGE_MIXED;
  int s = GCGE_OK;
  {
    HostCsr ha, hb;
    s = fetch_csr(A, ha);
    if (s == GCGE_OK) s = validate(ha);
    if (s == GCGE_OK && B) s = fetch_csr(B, hb);
    if (s == GCGE_OK && B) s = validate(hb);
    if (s == GCGE_OK) s = upload(ha, h->A, want32);
    if (s == GCGE_OK && B) s = upload(hb, h->B, want32);
    if (s == GCGE_OK) s = build_union(ha, B ? &hb : nullptr, h);
  }
  if (s != GCGE_OK) {
    free_handle(h);
    delete h;
    return s;
  }
  // locked-vector store in FP64: the prefix may overshoot nev by up to size_x
  h->store_cap = nev + sx;
  h->ld_store = round_up(h->store_cap, 4);
  if (cudaMalloc(&h->store, sizeof(double) * (size_t)h->n * h->ld_store) != cudaSuccess) {
    free_handle(h);
    delete h;
    return GCGE_ENOMEM;
  }
  *out = h;
  return GCGE_OK;
}

int gcge_solve(gcge_handle *h) {
  if (!h) return GCGE_EINVAL;
  h->solved = false;
  h->stats = gcge_stats{};
  h->lam.clear();
  h->nconv = 0;
  double *X0d = nullptr;
  if (h->opt.initial_block) {
    if (cudaMalloc(&X0d, sizeof(double) * (size_t)h->n * h->size_x) != cudaSuccess)
      return GCGE_ENOMEM;
    GCGE_CUDA(cudaMemcpyAsync(X0d, h->opt.initial_block, sizeof(double) * (size_t)h->n * h->size_x,
                              cudaMemcpyHostToDevice, h->st));
  }
  const long long l0 = g_launches.load();
  auto t0 = std::chrono::steady_clock::now();
  int it = 0, it32 = 0;
  int s;
  if (h->opt.precision == GCGE_MIXED)
    s = run_mixed(h, X0d, h->size_x, &it, &it32);
  else
    s = run_fp64(h, X0d, h->size_x, &it);
  cudaStreamSynchronize(h->st);
  h->stats.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->stats.iterations = it;
  h->stats.iterations_fp32 = it32;
  h->stats.nconv = h->nconv;
  h->stats.kernel_launches = g_launches.load() - l0;
  if (X0d) cudaFree(X0d);
  if (s == GCGE_OK || s == GCGE_ENOTCONV) h->solved = true;
  return s;
}

int gcge_eigenpairs(gcge_handle *h, double *evals, double *evecs, int64_t ldv, int evecs_on_device,
                    int *nconv) {
  if (!h || !evals) return GCGE_EINVAL;
  if (!h->solved) return GCGE_ENOTREADY;
  if (evecs && ldv < h->n) return GCGE_EINVAL;
  const int nl = (int)h->lam.size();
  std::vector<int> perm(nl);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return h->lam[a] < h->lam[b]; });
  const int k = std::min(nl, h->nev);
  for (int t = 0; t < h->nev; ++t) evals[t] = t < k ? h->lam[perm[t]] : NAN;
  if (nconv) *nconv = nl;
  if (evecs && k > 0) {
    int *dperm = nullptr;
    GCGE_CUDA(cudaMalloc(&dperm, sizeof(int) * k));
    GCGE_CUDA(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, h->st));
    double *dst = evecs;
    double *tmp = nullptr;
    if (!evecs_on_device) {
      GCGE_CUDA(cudaMalloc(&tmp, sizeof(double) * (size_t)h->n * k));
      dst = tmp;
    }
    const int64_t ldo = evecs_on_device ? ldv : h->n;
    int64_t g = ((int64_t)h->n * k + 255) / 256;
    if (g > 4096) g = 4096;
    transpose_out_kernel<<<(int)g, 256, 0, h->st>>>(h->n, k, dperm, h->store, h->ld_store, dst, ldo);
    GCGE_LAUNCH_CHECK();
    if (!evecs_on_device) {
      GCGE_CUDA(cudaMemcpy2DAsync(evecs, sizeof(double) * ldv, tmp, sizeof(double) * h->n,
                                  sizeof(double) * h->n, k, cudaMemcpyDeviceToHost, h->st));
    }
    GCGE_CUDA(cudaStreamSynchronize(h->st));
    cudaFree(dperm);
    if (tmp) cudaFree(tmp);
  }
  return GCGE_OK;
}

int gcge_stats_get(gcge_handle *h, gcge_stats *st) {
  if (!h || !st) return GCGE_EINVAL;
  *st = h->stats;
  return GCGE_OK;
}

void gcge_destroy(gcge_handle *h) {
  if (!h) return;
  free_handle(h);
  delete h;
}

}  // extern "C"
