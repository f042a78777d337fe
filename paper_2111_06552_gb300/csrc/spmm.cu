// CSR x row-major multivector product, Y = alpha A X + beta Y (MatDotMultiVec, Section 3.4).
//
// Layout: X and Y are row-major n x k (ld >= k), so every nonzero a_ij of row i
// gathers the contiguous k-vector X[j, 0:k].  A group of G lanes (G = the
// smallest power of two >= k, at most a warp) owns one row at a time; lane l
// accumulates columns l, l+G, l+2G, ... in registers.  The column index and value
// of a nonzero are the same address for the whole group (one broadcast
// transaction); the gathered k-vector is one coalesced segment.  The nonzero
// loop is unrolled by four so four independent gathers are in flight per lane.
#include "spmm.cuh"

namespace gcge {

namespace {

constexpr int kSpmmThreads = 256;

template <typename T, int G, int C, bool DOT>
__global__ void __launch_bounds__(kSpmmThreads)
spmm_kernel(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
            const T *__restrict__ val, int k, T alpha, const T *__restrict__ X, int64_t ldx,
            T beta, T *__restrict__ Y, int64_t ldy, double *__restrict__ dot_out) {
  extern __shared__ double sdot[];
  if (DOT) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) sdot[j] = 0.0;
    __syncthreads();
  }
  const int lane = threadIdx.x & (G - 1);
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t ngr = ((int64_t)gridDim.x * blockDim.x) / G;
  double dacc[C];
#pragma unroll
  for (int u = 0; u < C; ++u) dacc[u] = 0.0;

  for (int64_t row = gid; row < n; row += ngr) {
    const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
    for (int j0 = 0; j0 < k; j0 += G * C) {
      T acc[C];
#pragma unroll
      for (int u = 0; u < C; ++u) acc[u] = T(0);
      const int jl = j0 + lane;
      int e = beg;
      for (; e + 3 < end; e += 4) {
        const int c0 = __ldg(ci + e), c1 = __ldg(ci + e + 1), c2 = __ldg(ci + e + 2),
                  c3 = __ldg(ci + e + 3);
        const T v0 = __ldg(val + e), v1 = __ldg(val + e + 1), v2 = __ldg(val + e + 2),
                v3 = __ldg(val + e + 3);
        const T *x0 = X + (int64_t)c0 * ldx + jl;
        const T *x1 = X + (int64_t)c1 * ldx + jl;
        const T *x2 = X + (int64_t)c2 * ldx + jl;
        const T *x3 = X + (int64_t)c3 * ldx + jl;
#pragma unroll
        for (int u = 0; u < C; ++u) {
          if (jl + u * G < k) {
            const T a0 = __ldg(x0 + u * G), a1 = __ldg(x1 + u * G), a2 = __ldg(x2 + u * G),
                    a3 = __ldg(x3 + u * G);
            acc[u] += v0 * a0;
            acc[u] += v1 * a1;
            acc[u] += v2 * a2;
            acc[u] += v3 * a3;
          }
        }
      }
      for (; e < end; ++e) {
        const int c0 = __ldg(ci + e);
        const T v0 = __ldg(val + e);
        const T *x0 = X + (int64_t)c0 * ldx + jl;
#pragma unroll
        for (int u = 0; u < C; ++u)
          if (jl + u * G < k) acc[u] += v0 * __ldg(x0 + u * G);
      }
#pragma unroll
      for (int u = 0; u < C; ++u) {
        const int j = jl + u * G;
        if (j < k) {
          T out = alpha * acc[u];
          T *yp = Y + row * ldy + j;
          if (beta != T(0)) out += beta * *yp;
          *yp = out;
          if (DOT) dacc[u] += (double)X[row * ldx + j] * (double)acc[u];
        }
      }
    }
  }
  if (DOT) {
#pragma unroll
    for (int u = 0; u < C; ++u) {
      const int j = lane + u * G;
      if (j < k && dacc[u] != 0.0) atomicAdd(&sdot[j], dacc[u]);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) dot_out[(int64_t)blockIdx.x * k + j] = sdot[j];
  }
}

template <typename T, int G, int C>
void launch_gc(int grid, int64_t n, const int32_t *rp, const int32_t *ci, const T *val, int k,
               T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *dot_out,
               cudaStream_t st) {
  if (dot_out)
    spmm_kernel<T, G, C, true><<<grid, kSpmmThreads, k * sizeof(double), st>>>(
        n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out);
  else
    spmm_kernel<T, G, C, false><<<grid, kSpmmThreads, 0, st>>>(n, rp, ci, val, k, alpha, X, ldx,
                                                                beta, Y, ldy, nullptr);
}

template <typename T, int G>
void launch_g(int C, int grid, int64_t n, const int32_t *rp, const int32_t *ci, const T *val,
              int k, T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy,
              double *dot_out, cudaStream_t st) {
  switch (C) {
    case 1: launch_gc<T, G, 1>(grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 2: launch_gc<T, G, 2>(grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 3: launch_gc<T, G, 3>(grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    default: launch_gc<T, G, 4>(grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
  }
}

int spmm_grid(int64_t n, int G) {
  const int64_t groups_per_block = kSpmmThreads / G;
  int64_t need = (n + groups_per_block - 1) / groups_per_block;
  const int64_t cap = (int64_t)device_sm_count() * 8;
  if (need > cap) need = cap;
  if (need < 1) need = 1;
  return (int)need;
}

}  // namespace

int spmm_dot_blocks(int64_t n, int k) { return spmm_grid(n, spmm_shape(k).G); }

template <typename T>
int launch_spmm(int64_t n, const int32_t *rp, const int32_t *ci, const T *val, int k, T alpha,
                const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *dot_out,
                int dot_blocks, cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  const SpmmShape s = spmm_shape(k);
  if (dot_out && k > s.G * s.C) return GCGE_EINVAL;   // dot epilogue needs one column pass
  const int grid = spmm_grid(n, s.G);
  if (dot_out && grid != dot_blocks) return GCGE_EINVAL;
  switch (s.G) {
    case 1: launch_g<T, 1>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 2: launch_g<T, 2>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 4: launch_g<T, 4>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 8: launch_g<T, 8>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    case 16: launch_g<T, 16>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
    default: launch_g<T, 32>(s.C, grid, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, dot_out, st); break;
  }
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template int launch_spmm<double>(int64_t, const int32_t *, const int32_t *, const double *, int,
                                 double, const double *, int64_t, double, double *, int64_t,
                                 double *, int, cudaStream_t);
template int launch_spmm<float>(int64_t, const int32_t *, const int32_t *, const float *, int,
                                float, const float *, int64_t, float, float *, int64_t, double *,
                                int, cudaStream_t);

}  // namespace gcge
