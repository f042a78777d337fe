// STEP 6 of Algorithm 1 (Eq. compW): the few-step shifted inverse-power solve.
//
// All k columns advance together with per-column scalars, which equals k
// independent CG runs.  One CG step is three kernels:
//   1. q = S p, with the per-column dots p^T q fused into the SpMM epilogue
//      (summed across CTAs in a fixed order by the last CTA into pq[k]);
//   2. alpha_j = rr_j / pq_j; x += alpha p, r -= alpha q; per-column r^T r
//      (last CTA: rr_new[k], and the breakdown flags for p^T S p <= 0);
//   3. beta_j = rr_new_j / rr_j; p = r + beta p (last CTA commits rr, the step
//      counts and the stop flags ||r|| <= rtol ||r0||).
// With a Jacobi preconditioner M^-1 = 1 / |diag(S)| (per row) the same three kernels
// run preconditioned CG: z = M^-1 r is formed on the fly where it is read, alpha and
// beta use r^T z, and the stop test stays on the unpreconditioned ||r||.
// Vector kernels move 16-byte chunks when the blocks are aligned.  A stopped
// column takes no further updates.  Breakdown: S = A - theta B is only SPD on the
// complement of the locked vectors (Section 3.2), so p^T S p <= 0 stops a column.
#include "cg.cuh"

namespace gcge {

namespace {

constexpr int kCgThreads = 256;

// Column-sliced elementwise pass: thread (row slot, chunk); VEC columns per chunk.
template <int VEC>
struct Slice {
  int chunks, rows_per_block, row0, chunk;
  bool on;
  __device__ Slice(int k) {
    chunks = (k + VEC - 1) / VEC;
    const int cpb = chunks < kCgThreads ? chunks : kCgThreads;
    rows_per_block = kCgThreads / cpb;
    row0 = threadIdx.x / cpb;
    chunk = threadIdx.x % cpb;
    on = row0 < rows_per_block;
  }
};

// Per-column sums of a(row, j)^2 style reductions over a block -> part[blockIdx.x * k + j].
// A thread's own sum is kept in the block's precision (FP32 blocks: the sums only steer
// the inexact inner CG); the block and cross-CTA sums run in FP64, in a fixed order.
template <int VEC, typename A>
__device__ __forceinline__ void block_cols_to_part(const Slice<VEC> &sl, int k, const A (&acc)[VEC],
                                                   double *sred, double *part, int pstride,
                                                   int poff) {
  // sred: kCgThreads * VEC doubles laid out [row0][chunk*VEC + v] with row stride chunks*VEC
  const int w = sl.chunks * VEC;
  if (sl.on)
#pragma unroll
    for (int v = 0; v < VEC; ++v) sred[sl.row0 * w + sl.chunk * VEC + v] = (double)acc[v];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < sl.rows_per_block; ++r) s += sred[r * w + j];
    part[(int64_t)blockIdx.x * pstride + poff + j] = s;
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_vec(const T *p, T (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (VEC == 2) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = *p;
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void st_vec(T *p, const T (&v)[VEC]) {
  if constexpr (VEC == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}

// Initial sums: rr_j = r_j^T r_j, rz_j = r_j^T M^-1 r_j, and p = M^-1 r; the last CTA
// writes rr, rz, r0, active, iters, broke.
template <typename T, int VEC>
__global__ void __launch_bounds__(kCgThreads)
cg_init_kernel(int64_t n, int k, const T *__restrict__ r, T *__restrict__ p, int64_t ld,
               const T *__restrict__ minv, double *__restrict__ part,
               unsigned *__restrict__ ticket, double *__restrict__ rr, double *__restrict__ rz,
               double *__restrict__ r0, int *__restrict__ active, int *__restrict__ iters,
               int *__restrict__ broke, double rtol) {
  extern __shared__ double sm[];
  Slice<VEC> sl(k);
  T acc[VEC], accz[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = accz[v] = T(0);
  if (sl.on) {
    for (int64_t row = (int64_t)blockIdx.x * sl.rows_per_block + sl.row0; row < n;
         row += (int64_t)gridDim.x * sl.rows_per_block) {
      const int j0 = sl.chunk * VEC;
      const T mi = minv ? minv[row] : T(1);
      if (j0 + VEC <= k) {
        T rv[VEC], zv[VEC];
        ld_vec<T, VEC>(r + row * ld + j0, rv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          zv[v] = mi * rv[v];
          acc[v] += rv[v] * rv[v];
          accz[v] += rv[v] * zv[v];
        }
        st_vec<T, VEC>(p + row * ld + j0, zv);
      } else {
        for (int v = 0; v < VEC && j0 + v < k; ++v) {
          const T x = r[row * ld + j0 + v], z = mi * x;
          p[row * ld + j0 + v] = z;
          acc[v] += x * x;
          accz[v] += x * z;
        }
      }
    }
  }
  block_cols_to_part<VEC>(sl, k, acc, sm, part, 2 * k, 0);
  __syncthreads();
  block_cols_to_part<VEC>(sl, k, accz, sm, part, 2 * k, k);
  __syncthreads();
  last_cta_reduce(2 * k, part, ticket, sm, [&](int j, double s) {
    if (j < k) {
      rr[j] = s;
      const double nr = sqrt(s);
      r0[j] = nr;
      active[j] = (nr <= rtol * nr) ? 0 : 1;
      iters[j] = 0;
      broke[j] = 0;
    } else {
      rz[j - k] = s;
    }
  });
}

// alpha = rz / pq; x += alpha p, r -= alpha q; partial r^T r and r^T M^-1 r; last CTA:
// rrn, rzn and the breakdown flags.
template <typename T, int VEC>
__global__ void __launch_bounds__(kCgThreads)
cg_update_kernel(int64_t n, int k, const double *__restrict__ pq, const double *__restrict__ rz,
                 int *__restrict__ active, int *__restrict__ broke, T *__restrict__ x,
                 int64_t ldx, const T *__restrict__ p, T *__restrict__ r,
                 const T *__restrict__ q, int64_t ld, const T *__restrict__ minv,
                 double *__restrict__ part, unsigned *__restrict__ ticket,
                 double *__restrict__ rrn, double *__restrict__ rzn) {
  extern __shared__ double sm[];
  double *salpha = sm;                       // k
  double *sred = sm + k;                     // kCgThreads * VEC
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const bool a = active[j] && pq[j] > 0.0;
    salpha[j] = a ? rz[j] / pq[j] : 0.0;
  }
  __syncthreads();
  Slice<VEC> sl(k);
  T acc[VEC], accz[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = accz[v] = T(0);
  if (sl.on) {
    const int j0 = sl.chunk * VEC;
    T al[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) al[v] = (T)(j0 + v < k ? salpha[j0 + v] : 0.0);
    const bool full = j0 + VEC <= k;
#pragma unroll 2
    for (int64_t row = (int64_t)blockIdx.x * sl.rows_per_block + sl.row0; row < n;
         row += (int64_t)gridDim.x * sl.rows_per_block) {
      const T mi = minv ? minv[row] : T(1);
      if (full) {
        T xv[VEC], pv[VEC], rv[VEC], qv[VEC];
        ld_vec<T, VEC>(x + row * ldx + j0, xv);
        ld_vec<T, VEC>(p + row * ld + j0, pv);
        ld_vec<T, VEC>(r + row * ld + j0, rv);
        ld_vec<T, VEC>(q + row * ld + j0, qv);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          xv[v] += al[v] * pv[v];
          rv[v] -= al[v] * qv[v];
          acc[v] += rv[v] * rv[v];
          accz[v] += rv[v] * (mi * rv[v]);
        }
        st_vec<T, VEC>(x + row * ldx + j0, xv);
        st_vec<T, VEC>(r + row * ld + j0, rv);
      } else {
        for (int v = 0; v < VEC && j0 + v < k; ++v) {
          const int j = j0 + v;
          x[row * ldx + j] += al[v] * p[row * ld + j];
          const T rv = r[row * ld + j] - al[v] * q[row * ld + j];
          r[row * ld + j] = rv;
          acc[v] += rv * rv;
          accz[v] += rv * (mi * rv);
        }
      }
    }
  }
  block_cols_to_part<VEC>(sl, k, acc, sred, part, 2 * k, 0);
  __syncthreads();
  block_cols_to_part<VEC>(sl, k, accz, sred, part, 2 * k, k);
  __syncthreads();
  last_cta_reduce(2 * k, part, ticket, sred, [&](int j, double s) {
    if (j < k) {
      rrn[j] = s;
      if (active[j] && !(pq[j] > 0.0)) {
        active[j] = 0;
        broke[j] = 1;
      }
    } else {
      rzn[j - k] = s;
    }
  });
}

// beta = rzn / rz; p = M^-1 r + beta p for active columns; the last CTA commits rr = rrn,
// rz = rzn, the step counts and the stop flags (||r|| <= rtol ||r0||).
template <typename T, int VEC>
__global__ void __launch_bounds__(kCgThreads)
cg_pupdate_kernel(int64_t n, int k, const double *__restrict__ rrn, double *__restrict__ rr,
                  const double *__restrict__ rzn, double *__restrict__ rz,
                  const double *__restrict__ r0, int *__restrict__ active,
                  int *__restrict__ iters, T *__restrict__ p, const T *__restrict__ r, int64_t ld,
                  const T *__restrict__ minv, unsigned *__restrict__ ticket, double rtol) {
  extern __shared__ double sm[];
  double *sbeta = sm;                        // k
  int *sact = (int *)(sm + k);               // k
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const int a = active[j];
    sact[j] = a;
    sbeta[j] = a ? rzn[j] / rz[j] : 0.0;
  }
  __syncthreads();
  Slice<VEC> sl(k);
  if (sl.on) {
    const int j0 = sl.chunk * VEC;
    bool any = false;
    T be[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const bool a = j0 + v < k && sact[j0 + v];
      any |= a;
      be[v] = (T)(a ? sbeta[j0 + v] : 0.0);
    }
    const bool full = j0 + VEC <= k;
    if (any) {
      for (int64_t row = (int64_t)blockIdx.x * sl.rows_per_block + sl.row0; row < n;
           row += (int64_t)gridDim.x * sl.rows_per_block) {
        const T mi = minv ? minv[row] : T(1);
        if (full) {
          T pv[VEC], rv[VEC];
          ld_vec<T, VEC>(p + row * ld + j0, pv);
          ld_vec<T, VEC>(r + row * ld + j0, rv);
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            if (sact[j0 + v]) pv[v] = mi * rv[v] + be[v] * pv[v];
          st_vec<T, VEC>(p + row * ld + j0, pv);
        } else {
          for (int v = 0; v < VEC && j0 + v < k; ++v)
            if (sact[j0 + v])
              p[row * ld + j0 + v] = mi * r[row * ld + j0 + v] + be[v] * p[row * ld + j0 + v];
        }
      }
    }
  }
  // commit after every CTA has read rz: the last CTA to arrive does it
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    if (!active[j]) continue;
    rr[j] = rrn[j];
    rz[j] = rzn[j];
    iters[j] += 1;
    if (sqrt(rrn[j]) <= rtol * r0[j]) active[j] = 0;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// minv[i] = 1 / |S_ii| from the sorted CSR row (binary search for column i).
template <typename T>
__global__ void jacobi_inverse_kernel(int64_t n, const int32_t *__restrict__ rp,
                                      const int32_t *__restrict__ ci, const T *__restrict__ S,
                                      T *__restrict__ minv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = rp[i], hi = rp[i + 1] - 1;
    T d = T(0);
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = ci[mid];
      if (c == (int)i) {
        d = S[mid];
        break;
      }
      if (c < (int)i) lo = mid + 1;
      else hi = mid - 1;
    }
    const T a = d < T(0) ? -d : d;
    minv[i] = a > T(0) ? T(1) / a : T(1);
  }
}

int upd_grid(int64_t n, int k) {
  const int rpp = kCgThreads / (k < kCgThreads ? k : kCgThreads);
  int64_t g = (n + (int64_t)rpp * 4 - 1) / ((int64_t)rpp * 4);
  // four CTAs per SM (with two rows in flight per thread in the update): enough loads
  // in flight to stream the vectors, and few partial rows for the last CTA to sum
  const int64_t cap = (int64_t)device_sm_count() * 4;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
bool cg_aligned(const T *x, int64_t ldx, const T *r, int64_t ld) {
  constexpr int vec = 16 / sizeof(T);
  return (uintptr_t)x % 16 == 0 && (uintptr_t)r % 16 == 0 && ldx % vec == 0 && ld % vec == 0;
}

}  // namespace

template <typename T>
int CgWork<T>::alloc(int64_t n, int k) {
  if (n <= ncap && k <= kcap) return GCGE_OK;
  free_all();
  ld = round_up(k, 4);
  // both grids grow with k, so sizing for the largest k covers every later call
  int nb = spmm_dot_blocks(n, k);
  if (upd_grid(n, k) > nb) nb = upd_grid(n, k);
  const size_t vb = sizeof(T) * (size_t)n * ld;
  GCGE_CUDA(cudaMalloc(&r, vb));
  GCGE_CUDA(cudaMalloc(&p, vb));
  GCGE_CUDA(cudaMalloc(&q, vb));
  GCGE_CUDA(cudaMalloc(&part_a, sizeof(double) * (size_t)nb * k));
  GCGE_CUDA(cudaMalloc(&part_b, sizeof(double) * (size_t)nb * 2 * k));
  GCGE_CUDA(cudaMalloc(&scal, sizeof(double) * 6 * (size_t)k));
  GCGE_CUDA(cudaMalloc(&flags, sizeof(int) * 3 * (size_t)k));
  GCGE_CUDA(cudaMalloc(&tickets, sizeof(unsigned) * 4));
  GCGE_CUDA(cudaMemset(tickets, 0, sizeof(unsigned) * 4));
  GCGE_CUDA(cudaMallocHost(&h_active, sizeof(int) * k));
  rr = scal;
  r0 = scal + k;
  pq = scal + 2 * k;
  rrn = scal + 3 * k;
  rz = scal + 4 * k;
  rzn = scal + 5 * k;
  active = flags;
  iters = flags + k;
  broke = flags + 2 * k;
  ncap = n;
  kcap = k;
  nbcap = nb;
  return GCGE_OK;
}

template <typename T>
void CgWork<T>::free_all() {
  cudaFree(r); cudaFree(p); cudaFree(q); cudaFree(part_a); cudaFree(part_b);
  cudaFree(scal); cudaFree(flags); cudaFree(tickets);
  if (h_active) cudaFreeHost(h_active);
  r = p = q = nullptr;
  part_a = part_b = scal = rr = r0 = pq = rrn = rz = rzn = nullptr;
  flags = active = iters = broke = h_active = nullptr;
  tickets = nullptr;
  ncap = 0;
  kcap = 0;
}

template <typename T, int VEC>
static int cg_loop(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, int k,
                   T *X, int64_t ldx, int max_iter, double rtol, CgWork<T> &w, int64_t &nl,
                   cudaStream_t st, KProf *prof, double spmm_bytes, double nnzS,
                   const T *minv) {
  const int64_t ld = w.ld;
  const int nbb = upd_grid(n, k);
  if (nbb > w.nbcap || k > w.kcap) return GCGE_EINVAL;
  const int chunks = (k + VEC - 1) / VEC;
  const size_t sm_r = sizeof(double) * (size_t)kCgThreads * VEC + 64;   // >= blockDim doubles
  const size_t sm_u = sizeof(double) * ((size_t)k + (size_t)kCgThreads * VEC) + 64;
  const size_t sm_p = (sizeof(double) + sizeof(int)) * (size_t)k + 64;
  (void)chunks;
  const double ts = sizeof(T), nk = (double)n * k;
  {
    ProfScope ps(prof, GCGE_K_CGVEC, nk * ts, 2.0 * nk);
    cg_init_kernel<T, VEC><<<nbb, kCgThreads, sm_r, st>>>(n, k, w.r, w.p, ld, minv, w.part_b,
                                                          w.tickets + 1, w.rr, w.rz, w.r0,
                                                          w.active, w.iters, w.broke, rtol);
    GCGE_LAUNCH_CHECK();
    ++nl;
  }
  for (int it = 0; it < max_iter; ++it) {
    {
      ProfScope ps(prof, sizeof(T) == 8 ? GCGE_K_SPMM64 : GCGE_K_SPMM, spmm_bytes, 2.0 * nnzS * k);
      GCGE_CHECK(launch_spmm<T>(n, rp, ci, S, k, T(1), w.p, ld, T(0), w.q, ld, w.pq, w.nbcap, st,
                                w.part_a, w.tickets));
    }
    {
      ProfScope ps(prof, GCGE_K_CGVEC, 9.0 * nk * ts, 6.0 * nk);
      cg_update_kernel<T, VEC><<<nbb, kCgThreads, sm_u, st>>>(n, k, w.pq, w.rz, w.active, w.broke,
                                                              X, ldx, w.p, w.r, w.q, ld, minv,
                                                              w.part_b, w.tickets + 2, w.rrn,
                                                              w.rzn);
      GCGE_LAUNCH_CHECK();
      cg_pupdate_kernel<T, VEC><<<nbb, kCgThreads, sm_p, st>>>(n, k, w.rrn, w.rr, w.rzn, w.rz,
                                                               w.r0, w.active, w.iters, w.p, w.r,
                                                               ld, minv, w.tickets + 3, rtol);
      GCGE_LAUNCH_CHECK();
    }
    nl += 3;
    // poll the stop flags every few steps (one small device->host copy)
    if ((it % 5) == 4 && it + 1 < max_iter) {
      GCGE_CUDA(cudaMemcpyAsync(w.h_active, w.active, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
      GCGE_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int j = 0; j < k; ++j) any |= (w.h_active[j] != 0);
      if (!any) break;
    }
  }
  return GCGE_OK;
}

template <typename T>
int block_cg(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, int k, const T *B,
             int64_t ldb, const T *r_init, int64_t ldr, T *X, int64_t ldx, int max_iter,
             double rtol, CgWork<T> &w, int *iters_host, int64_t *launches, cudaStream_t st,
             KProf *prof, const T *minv) {
  if (k <= 0 || n <= 0) return GCGE_OK;
  GCGE_CHECK(w.alloc(n, k));
  const int64_t ld = w.ld;
  int64_t nl = 0;
  int32_t nnz_last = 0;
  if (prof) GCGE_CUDA(cudaMemcpy(&nnz_last, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost));
  const double ts = sizeof(T), nk = (double)n * k;
  const double spmm_bytes = nnz_last * (ts + 4.0) + 4.0 * (n + 1) + 2.0 * nk * ts;
  // r = r_init, or r = B - S X
  if (r_init) {
    GCGE_CHECK(copy_cols<T, T>(n, k, r_init, ldr, w.r, ld, nullptr, st));
  } else {
    GCGE_CHECK(copy_cols<T, T>(n, k, B, ldb, w.r, ld, nullptr, st));
    GCGE_CHECK(launch_spmm<T>(n, rp, ci, S, k, T(-1), X, ldx, T(1), w.r, ld, nullptr, 0, st));
    ++nl;
  }
  nl += 1;   // p = M^-1 r is written by the first kernel of the loop
  constexpr int vmax = 16 / sizeof(T);
  if (cg_aligned<T>(X, ldx, w.r, ld))
    GCGE_CHECK(cg_loop<T, vmax>(n, rp, ci, S, k, X, ldx, max_iter, rtol, w, nl, st, prof,
                                spmm_bytes, nnz_last, minv));
  else
    GCGE_CHECK(cg_loop<T, 1>(n, rp, ci, S, k, X, ldx, max_iter, rtol, w, nl, st, prof, spmm_bytes,
                             nnz_last, minv));
  int mx = 0;
  if (iters_host) {
    GCGE_CUDA(cudaMemcpyAsync(iters_host, w.iters, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
    GCGE_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < k; ++j) mx = iters_host[j] > mx ? iters_host[j] : mx;
  }
  if (launches) *launches += nl;
  return mx;
}

template <typename T>
int jacobi_inverse(int64_t n, const int32_t *rp, const int32_t *ci, const T *S, T *minv,
                   cudaStream_t st) {
  if (n <= 0) return GCGE_OK;
  int64_t g = (n + 255) / 256;
  if (g > 8 * (int64_t)device_sm_count()) g = 8 * (int64_t)device_sm_count();
  jacobi_inverse_kernel<T><<<(int)g, 256, 0, st>>>(n, rp, ci, S, minv);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template int jacobi_inverse<double>(int64_t, const int32_t *, const int32_t *, const double *,
                                   double *, cudaStream_t);
template int jacobi_inverse<float>(int64_t, const int32_t *, const int32_t *, const float *,
                                  float *, cudaStream_t);
template struct CgWork<double>;
template struct CgWork<float>;
template int block_cg<double>(int64_t, const int32_t *, const int32_t *, const double *, int,
                              const double *, int64_t, const double *, int64_t, double *, int64_t,
                              int, double, CgWork<double> &, int *, int64_t *, cudaStream_t,
                              KProf *, const double *);
template int block_cg<float>(int64_t, const int32_t *, const int32_t *, const float *, int,
                             const float *, int64_t, const float *, int64_t, float *, int64_t,
                             int, double, CgWork<float> &, int *, int64_t *, cudaStream_t,
                             KProf *, const float *);

}  // namespace gcge
