// STEP 6 of Algorithm 1 (Eq. compW): the few-step shifted inverse-power solve.
//
// All k columns advance together with per-column scalars, which equals k
// independent CG runs.  One CG step is three kernels:
//   1. q = S p with the per-column partial dots p^T q fused into the SpMM epilogue;
//   2. every CTA reduces the p^T q partials in a fixed order (so every CTA
//      derives bit-identical alpha_j), then x += alpha p, r -= alpha q and the
//      partial dots r^T r;
//   3. every CTA reduces r^T r the same way, beta_j = r^T r / (previous), p = r + beta p;
//      CTA 0 records the new r^T r, the step count and the stop flags.
// A column stops when ||r|| <= rtol ||r0||, after max_iter steps, or when
// p^T S p <= 0 (breakdown: S = A - theta B is only SPD on the complement of
// the locked vectors, Section 3.2); stopped columns take no further updates.
#include "cg.cuh"

namespace gcge {

namespace {

constexpr int kCgThreads = 256;

__device__ __forceinline__ void reduce_parts_to_smem(int k, int nparts,
                                                     const double *__restrict__ part,
                                                     double *__restrict__ s) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += part[(int64_t)b * k + j];
    s[j] = acc;
  }
  __syncthreads();
}

__global__ void cg_init_kernel(int k, int nparts, const double *__restrict__ part,
                               double *__restrict__ rr, double *__restrict__ r0,
                               int *__restrict__ active, int *__restrict__ iters,
                               int *__restrict__ broke, double rtol) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += part[(int64_t)b * k + j];
    rr[j] = acc;
    const double nr = sqrt(acc);
    r0[j] = nr;
    active[j] = (nr <= rtol * nr) ? 0 : 1;
    iters[j] = 0;
    broke[j] = 0;
  }
}

// x += alpha p, r -= alpha q, partial r^T r.  smem: alpha[k], act[k], red[256].
template <typename T>
__global__ void __launch_bounds__(kCgThreads)
cg_update_kernel(int64_t n, int k, int nparts_a, const double *__restrict__ part_a,
                 const double *__restrict__ rr, int *__restrict__ active,
                 int *__restrict__ broke, T *__restrict__ x, int64_t ldx,
                 const T *__restrict__ p, T *__restrict__ r, const T *__restrict__ q, int64_t ld,
                 double *__restrict__ part_b) {
  extern __shared__ double sm[];
  double *salpha = sm;               // k
  double *sred = sm + k;             // kCgThreads
  int *sact = (int *)(sred + kCgThreads);   // k
  reduce_parts_to_smem(k, nparts_a, part_a, salpha);   // salpha = p^T q
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double pq = salpha[j];
    int a = active[j];
    if (a && !(pq > 0.0)) {
      a = 0;
      if (blockIdx.x == 0) {
        active[j] = 0;
        broke[j] = 1;
      }
    }
    sact[j] = a;
    salpha[j] = a ? rr[j] / pq : 0.0;
  }
  __syncthreads();
  const int kc = k < kCgThreads ? k : kCgThreads;
  const int rpp = kCgThreads / kc;
  for (int j0 = 0; j0 < k; j0 += kc) {
    const int jj = threadIdx.x % kc, rr_ = threadIdx.x / kc;
    const int j = j0 + jj;
    double acc = 0.0;
    if (rr_ < rpp && j < k) {
      const T al = (T)salpha[j];
      const bool a = sact[j] != 0;
      for (int64_t row = (int64_t)blockIdx.x * rpp + rr_; row < n; row += (int64_t)gridDim.x * rpp) {
        T rv = r[row * ld + j];
        if (a) {
          x[row * ldx + j] += al * p[row * ld + j];
          rv -= al * q[row * ld + j];
          r[row * ld + j] = rv;
        }
        acc += (double)rv * (double)rv;
      }
    }
    sred[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < kc && j0 + threadIdx.x < k) {
      double s = 0.0;
      for (int t = threadIdx.x; t < rpp * kc; t += kc) s += sred[t];
      part_b[(int64_t)blockIdx.x * k + j0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// beta = rr_new / rr, p = r + beta p for the active columns (rr is read-only here;
// the commit kernel that follows records rr_new).
template <typename T>
__global__ void __launch_bounds__(kCgThreads)
cg_pupdate_kernel(int64_t n, int k, int nparts_b, const double *__restrict__ part_b,
                  const double *__restrict__ rr, const int *__restrict__ active,
                  T *__restrict__ p, const T *__restrict__ r, int64_t ld) {
  extern __shared__ double sm[];
  double *sbeta = sm;                 // k
  int *sact = (int *)(sm + k);        // k
  reduce_parts_to_smem(k, nparts_b, part_b, sbeta);   // sbeta = rr_new
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const int a = active[j];
    sact[j] = a;
    sbeta[j] = a ? sbeta[j] / rr[j] : 0.0;
  }
  __syncthreads();
  const int kc = k < kCgThreads ? k : kCgThreads;
  const int rpp = kCgThreads / kc;
  for (int j0 = 0; j0 < k; j0 += kc) {
    const int jj = threadIdx.x % kc, rr_ = threadIdx.x / kc;
    const int j = j0 + jj;
    if (rr_ < rpp && j < k && sact[j]) {
      const T be = (T)sbeta[j];
      for (int64_t row = (int64_t)blockIdx.x * rpp + rr_; row < n; row += (int64_t)gridDim.x * rpp)
        p[row * ld + j] = r[row * ld + j] + be * p[row * ld + j];
    }
  }
}

// Commit the per-column state after a step (one small kernel, so that no CTA
// of the p-update reads rr while another rewrites it).
__global__ void cg_commit_kernel(int k, int nparts_b, const double *__restrict__ part_b,
                                 double *__restrict__ rr, const double *__restrict__ r0,
                                 int *__restrict__ active, int *__restrict__ iters, double rtol) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    if (!active[j]) continue;
    double rn = 0.0;
    for (int b = 0; b < nparts_b; ++b) rn += part_b[(int64_t)b * k + j];
    rr[j] = rn;
    iters[j] += 1;
    if (sqrt(rn) <= rtol * r0[j]) active[j] = 0;
  }
}

int upd_grid(int64_t n, int k) {
  const int kc = k < kCgThreads ? k : kCgThreads;
  const int rpp = kCgThreads / kc;
  int64_t g = (n + (int64_t)rpp * 8 - 1) / ((int64_t)rpp * 8);
  const int64_t cap = (int64_t)device_sm_count() * 4;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
__global__ void residual_init_kernel(int64_t n, int k, T *__restrict__ r, int64_t ld,
                                     const T *__restrict__ B, int64_t ldb) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / k;
    const int j = (int)(t % k);
    r[row * ld + j] = B[row * ldb + j];
  }
}

}  // namespace

template <typename T>
int CgWork<T>::alloc(int64_t n, int k) {
  if (n <= ncap && k <= kcap) return GCGE_OK;
  free_all();
  ld = round_up(k, 4);
  const int nb = spmm_dot_blocks(n, k) > upd_grid(n, k) ? spmm_dot_blocks(n, k) : upd_grid(n, k);
  const size_t vb = sizeof(T) * (size_t)n * ld;
  GCGE_CUDA(cudaMalloc(&r, vb));
  GCGE_CUDA(cudaMalloc(&p, vb));
  GCGE_CUDA(cudaMalloc(&q, vb));
  GCGE_CUDA(cudaMalloc(&part_a, sizeof(double) * (size_t)nb * k));
  GCGE_CUDA(cudaMalloc(&part_b, sizeof(double) * (size_t)nb * k));
  GCGE_CUDA(cudaMalloc(&rr, sizeof(double) * k));
  GCGE_CUDA(cudaMalloc(&r0, sizeof(double) * k));
  GCGE_CUDA(cudaMalloc(&active, sizeof(int) * k));
  GCGE_CUDA(cudaMalloc(&iters, sizeof(int) * k));
  GCGE_CUDA(cudaMalloc(&broke, sizeof(int) * k));
  GCGE_CUDA(cudaMallocHost(&h_active, sizeof(int) * k));
  ncap = n;
  kcap = k;
  return GCGE_OK;
}

template <typename T>
void CgWork<T>::free_all() {
  cudaFree(r); cudaFree(p); cudaFree(q); cudaFree(part_a); cudaFree(part_b);
  cudaFree(rr); cudaFree(r0); cudaFree(active); cudaFree(iters); cudaFree(broke);
  if (h_active) cudaFreeHost(h_active);
  r = p = q = nullptr;
  part_a = part_b = rr = r0 = nullptr;
  active = iters = broke = h_active = nullptr;
  ncap = 0;
  kcap = 0;
}

template <typename T>
int block_cg(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, int k, const T *B,
             int64_t ldb, const T *r_init, int64_t ldr, T *X, int64_t ldx, int max_iter,
             double rtol, CgWork<T> &w, int *iters_host, int64_t *launches, cudaStream_t st,
             KProf *prof) {
  if (k <= 0 || n <= 0) return GCGE_OK;
  int64_t nnzS = 0;
  if (prof) {
    int32_t last = 0;
    cudaMemcpy(&last, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
    nnzS = last;
  }
  const double ts = sizeof(T), nk = (double)n * k;
  const double spmm_bytes = nnzS * (ts + 4.0) + 4.0 * (n + 1) + 2.0 * nk * ts;
  GCGE_CHECK(w.alloc(n, k));
  const int64_t ld = w.ld;
  const int nba = spmm_dot_blocks(n, k);
  const int nbb = upd_grid(n, k);
  int64_t nl = 0;
  // r = r_init, or r = B - S X
  if (r_init) {
    GCGE_CHECK(copy_cols<T, T>(n, k, r_init, ldr, w.r, ld, nullptr, st));
  } else {
    GCGE_CHECK(copy_cols<T, T>(n, k, B, ldb, w.r, ld, nullptr, st));
    GCGE_CHECK(launch_spmm<T>(n, rp, ci, S, k, T(-1), X, ldx, T(1), w.r, ld, nullptr, 0, st));
    ++nl;
  }
  ++nl;
  GCGE_CHECK(copy_cols<T, T>(n, k, w.r, ld, w.p, ld, nullptr, st));
  ++nl;
  {
    // initial r^T r: the update kernel with every column marked inactive (alpha = 0)
    // only reduces r^T r into part_b; cg_init then sets rr, r0 and the flags.
    const size_t sm = sizeof(double) * (k + kCgThreads) + sizeof(int) * k;
    GCGE_CUDA(cudaMemsetAsync(w.active, 0, sizeof(int) * k, st));
    GCGE_CUDA(cudaMemsetAsync(w.part_a, 0, sizeof(double) * (size_t)nba * k, st));
    cg_update_kernel<T><<<nbb, kCgThreads, sm, st>>>(n, k, nba, w.part_a, w.rr, w.active, w.broke,
                                                     X, ldx, w.p, w.r, w.q, ld, w.part_b);
    GCGE_LAUNCH_CHECK();
    cg_init_kernel<<<1, 256, 0, st>>>(k, nbb, w.part_b, w.rr, w.r0, w.active, w.iters, w.broke,
                                      rtol);
    GCGE_LAUNCH_CHECK();
    nl += 2;
  }
  const size_t sm_u = sizeof(double) * (k + kCgThreads) + sizeof(int) * k;
  const size_t sm_p = sizeof(double) * k + sizeof(int) * k;
  for (int it = 0; it < max_iter; ++it) {
    {
      ProfScope ps(prof, GCGE_K_SPMM, spmm_bytes, 2.0 * nnzS * k);
      GCGE_CHECK(launch_spmm<T>(n, rp, ci, S, k, T(1), w.p, ld, T(0), w.q, ld, w.part_a, nba, st));
    }
    {
      ProfScope ps(prof, GCGE_K_CGVEC, 9.0 * nk * ts, 6.0 * nk);
      cg_update_kernel<T><<<nbb, kCgThreads, sm_u, st>>>(n, k, nba, w.part_a, w.rr, w.active,
                                                         w.broke, X, ldx, w.p, w.r, w.q, ld,
                                                         w.part_b);
      GCGE_LAUNCH_CHECK();
      cg_pupdate_kernel<T><<<nbb, kCgThreads, sm_p, st>>>(n, k, nbb, w.part_b, w.rr, w.active,
                                                          w.p, w.r, ld);
      GCGE_LAUNCH_CHECK();
      cg_commit_kernel<<<1, 256, 0, st>>>(k, nbb, w.part_b, w.rr, w.r0, w.active, w.iters, rtol);
      GCGE_LAUNCH_CHECK();
    }
    nl += 4;
    // poll the stop flags every few steps (one small device->host copy)
    if ((it % 4) == 3 && it + 1 < max_iter) {
      GCGE_CUDA(cudaMemcpyAsync(w.h_active, w.active, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
      GCGE_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int j = 0; j < k; ++j) any |= (w.h_active[j] != 0);
      if (!any) break;
    }
  }
  int mx = 0;
  if (iters_host) {
    GCGE_CUDA(cudaMemcpyAsync(iters_host, w.iters, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
    GCGE_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < k; ++j) mx = iters_host[j] > mx ? iters_host[j] : mx;
  }
  if (launches) *launches += nl;
  return mx;
}

template struct CgWork<double>;
template struct CgWork<float>;
template int block_cg<double>(int64_t, const int32_t *, const int32_t *, const double *, int,
                              const double *, int64_t, const double *, int64_t, double *, int64_t,
                              int, double, CgWork<double> &, int *, int64_t *, cudaStream_t,
                              KProf *);
template int block_cg<float>(int64_t, const int32_t *, const int32_t *, const float *, int,
                             const float *, int64_t, const float *, int64_t, float *, int64_t,
                             int, double, CgWork<float> &, int *, int64_t *, cudaStream_t,
                             KProf *);

}  // namespace gcge
