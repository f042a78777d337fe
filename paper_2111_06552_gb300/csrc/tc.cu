// Tensor-core (tcgen05, TF32) forms of the Gram and V C products for FP32 blocks.
//
// The dense contractions of the method on FP32 blocks run on the 5th-generation
// tensor cores: operands are staged in shared memory in the K-major core-matrix
// layout (8 rows x 16 bytes per core matrix, no swizzle), one thread issues
// tcgen05.mma (kind::tf32, M = 128) with the accumulator in tensor memory, MMA
// completion is tracked with an mbarrier (tcgen05.commit), and the epilogue reads
// the accumulator back with tcgen05.ld.  TF32 keeps 10 mantissa bits, so each FP32
// operand x is split as x = hi + lo (hi = x with the low 13 mantissa bits cleared,
// lo = x - hi exactly) and three products hi*hi + hi*lo + lo*hi are accumulated in
// FP32, which restores close to FP32 accuracy; the product is memory-bound at the
// block widths of the method, so the extra MMAs are free.
//
//   Gram  C(m x k) = X^T Y:  M = 128-row tiles of m (up to 4 in one CTA, one TMEM
//         accumulator each), N = k padded to 16, K = the rows of a split of n, staged
//         16 rows at a time (transposed into K-major order while staging), double
//         buffered; FP64 partial per split, reduced by the common FP64 reduction.
//   V C   Y(n x q) = V C:  M = 128 rows of V, N = q padded to 16 (<= 256 per CTA),
//         K = d in chunks of 16; C is FP64 and is rounded to FP32 then split.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records an error flag,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <algorithm>

#include "blas.cuh"
#include "tcgen05.cuh"

namespace gcge {

namespace {

using namespace tc;

constexpr int kTcThreads = 256;
constexpr int kKC = 16;                        // K rows per staged chunk (2 MMA k-steps)

// ------------------------------------------------------------------------- Gram
// Dynamic smem: 2 stages x [A_hi | A_lo | B_hi | B_lo], A = MT*128 rows, B = Np rows.
__global__ void __launch_bounds__(kTcThreads)
gram_tc_kernel(int64_t n, int m, int k, int MT, int Np, const float *__restrict__ X, int64_t ldx,
               const float *__restrict__ Y, int64_t ldy, int64_t rows_per_split,
               double *__restrict__ part, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tbase;
  const int arows = MT * 128;
  const uint32_t a_bytes = (uint32_t)arows * kKC * 4, b_bytes = (uint32_t)Np * kKC * 4;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  const uint32_t ncols = tmem_cols_for(MT * Np);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_split;
  int64_t r1 = r0 + rows_per_split;
  if (r1 > n) r1 = n;
  const int nchunks = (int)((r1 - r0 + kKC - 1) / kKC);
  const uint32_t idesc = idesc_tf32(128, Np);
  unsigned uses[2] = {0u, 0u};
  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    unsigned char *st = sm + (size_t)s * stage_bytes;
    if (c >= 2) {   // the MMAs that read this stage two chunks ago must be done
      ok = mbar_wait(&bar[s], (uses[s] - 1) & 1, err, nullptr);
      if (!ok) break;
    }
    const int64_t rb = r0 + (int64_t)c * kKC;
    // stage X rows [rb, rb+kKC) x arows columns, transposed to K-major (row = column of X)
    for (int t = threadIdx.x; t < kKC * arows; t += kTcThreads) {
      const int kk = t / arows, i = t % arows;
      const int64_t r = rb + kk;
      const float x = (r < r1 && i < m) ? X[r * ldx + i] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = kmaj_off(i, kk, arows);
      *reinterpret_cast<float *>(st + off) = hi;
      *reinterpret_cast<float *>(st + a_bytes + off) = lo;
    }
    for (int t = threadIdx.x; t < kKC * Np; t += kTcThreads) {
      const int kk = t / Np, j = t % Np;
      const int64_t r = rb + kk;
      const float y = (r < r1 && j < k) ? Y[r * ldy + j] : 0.f;
      float hi, lo;
      split_tf32(y, hi, lo);
      const uint32_t off = kmaj_off(j, kk, Np);
      *reinterpret_cast<float *>(st + 2 * a_bytes + off) = hi;
      *reinterpret_cast<float *>(st + 2 * a_bytes + b_bytes + off) = lo;
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t base = su32(st);
      for (int ks = 0; ks < kKC / 8; ++ks) {
        const uint32_t bh = base + 2 * a_bytes + ks * (Np / 8) * 256;
        const uint32_t bl = bh + b_bytes;
        const uint64_t dbh = smem_desc(bh, 128, 256), dbl = smem_desc(bl, 128, 256);
        for (int t = 0; t < MT; ++t) {
          const uint32_t ah = base + ks * (arows / 8) * 256 + t * 16 * 256;
          const uint32_t al = ah + a_bytes;
          const uint64_t dah = smem_desc(ah, 128, 256), dal = smem_desc(al, 128, 256);
          const uint32_t dt = tmem + t * Np;
          const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
          mma_ss(dt, dah, dbh, idesc, acc0);
          mma_ss(dt, dah, dbl, idesc, 1u);
          mma_ss(dt, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(&bar[s]);
    }
    uses[s] += 1;
    __syncthreads();
  }
  // wait for the last MMAs (both stages), bounded
  for (int s = 0; s < 2; ++s)
    if (uses[s] > 0) {
      if (!mbar_wait(&bar[s], (uses[s] - 1) & 1, err, nullptr)) ok = false;
    }
  tc_fence_after();
  if (ok && nchunks > 0 && warp < 4) {
    double *pp = part + (int64_t)blockIdx.x * m * k;
    for (int t = 0; t < MT; ++t) {
      const int i = t * 128 + warp * 32 + lane;
      for (int j0 = 0; j0 < Np; j0 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + t * Np + j0, v);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i < m && j0 + u < k) pp[(int64_t)(j0 + u) * m + i] = (double)v[u];
      }
    }
  } else if (nchunks == 0 && warp < 4) {
    double *pp = part + (int64_t)blockIdx.x * m * k;
    for (int t = 0; t < MT; ++t) {
      const int i = t * 128 + warp * 32 + lane;
      for (int j = 0; j < k; ++j)
        if (i < m) pp[(int64_t)j * m + i] = 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------- V C
// Dynamic smem: 2 stages x [A_hi | A_lo | B_hi | B_lo], A = 128 rows of V, B = Np rows.
__global__ void __launch_bounds__(kTcThreads)
vc_tc_kernel(int64_t n, int d, int q, int Np, float alpha, const float *__restrict__ V,
             int64_t ldv, const double *__restrict__ Cm, int64_t ldc, float beta,
             float *__restrict__ Yo, int64_t ldy, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tbase;
  const uint32_t a_bytes = 128u * kKC * 4, b_bytes = (uint32_t)Np * kKC * 4;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  const uint32_t ncols = tmem_cols_for(Np);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * 128;
  const int q0 = blockIdx.y * Np;
  const int qn = (q - q0) < Np ? (q - q0) : Np;
  if (warp == 0) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  const int nchunks = (d + kKC - 1) / kKC;
  const uint32_t idesc = idesc_tf32(128, Np);
  unsigned uses[2] = {0u, 0u};
  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    unsigned char *st = sm + (size_t)s * stage_bytes;
    if (c >= 2) {
      ok = mbar_wait(&bar[s], (uses[s] - 1) & 1, err, nullptr);
      if (!ok) break;
    }
    const int k0 = c * kKC;
    for (int t = threadIdx.x; t < 128 * kKC; t += kTcThreads) {
      const int i = t / kKC, kk = t % kKC;
      const int64_t r = row0 + i;
      const float x = (r < n && k0 + kk < d) ? V[r * ldv + k0 + kk] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = kmaj_off(i, kk, 128);
      *reinterpret_cast<float *>(st + off) = hi;
      *reinterpret_cast<float *>(st + a_bytes + off) = lo;
    }
    for (int t = threadIdx.x; t < Np * kKC; t += kTcThreads) {
      const int j = t / kKC, kk = t % kKC;
      const float x = (j < qn && k0 + kk < d) ? (float)Cm[(k0 + kk) + (int64_t)(q0 + j) * ldc] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = kmaj_off(j, kk, Np);
      *reinterpret_cast<float *>(st + 2 * a_bytes + off) = hi;
      *reinterpret_cast<float *>(st + 2 * a_bytes + b_bytes + off) = lo;
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t base = su32(st);
      for (int ks = 0; ks < kKC / 8; ++ks) {
        const uint32_t ah = base + ks * 16 * 256, al = ah + a_bytes;
        const uint32_t bh = base + 2 * a_bytes + ks * (Np / 8) * 256, bl = bh + b_bytes;
        const uint64_t dah = smem_desc(ah, 128, 256), dal = smem_desc(al, 128, 256);
        const uint64_t dbh = smem_desc(bh, 128, 256), dbl = smem_desc(bl, 128, 256);
        const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
        mma_ss(tmem, dah, dbh, idesc, acc0);
        mma_ss(tmem, dah, dbl, idesc, 1u);
        mma_ss(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&bar[s]);
    }
    uses[s] += 1;
    __syncthreads();
  }
  for (int s = 0; s < 2; ++s)
    if (uses[s] > 0) {
      if (!mbar_wait(&bar[s], (uses[s] - 1) & 1, err, nullptr)) ok = false;
    }
  tc_fence_after();
  if (ok && warp < 4) {
    const int64_t r = row0 + warp * 32 + lane;
    for (int j0 = 0; j0 < Np; j0 += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + j0, v);
      if (r < n) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + u;
          if (j < qn) {
            float *yp = Yo + r * ldy + q0 + j;
            float out = alpha * v[u];
            if (beta != 0.f) out += beta * *yp;
            *yp = out;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}


size_t gram_tc_smem(int MT, int Np) {
  return tmem_limited_smem(2 * (2 * (size_t)MT * 128 * kKC * 4 + 2 * (size_t)Np * kKC * 4),
                           tmem_cols_for(MT * Np));
}
size_t vc_tc_smem(int Np) {
  return tmem_limited_smem(2 * (2 * (size_t)128 * kKC * 4 + 2 * (size_t)Np * kKC * 4),
                           tmem_cols_for(Np));
}

}  // namespace

// TMA-fed kernels of tc_tma.cu (GCGE_EINVAL: not applicable, use the staged kernels)
int gram_tma(int64_t n, int m, int k, double alpha, const float *X, int64_t ldx, const float *Y,
             int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st);
int vc_tma(int64_t n, int d, int q, double alpha, const float *V, int64_t ldv, const double *C,
           int64_t ldc, double beta, float *Y, int64_t ldy, Scratch &ws, cudaStream_t st);

// reduction kernel of blas.cu
int gram_reduce_launch(int m, int k, int splits, const double *part, double alpha, double beta,
                       double *C, int64_t ldc, cudaStream_t st);

namespace tc {
int err_flag(int **p) {
  static int *dev_err = nullptr;
  if (!dev_err) {
    if (cudaMalloc(&dev_err, sizeof(int)) != cudaSuccess) return GCGE_ENOMEM;
    cudaMemset(dev_err, 0, sizeof(int));
  }
  *p = dev_err;
  return GCGE_OK;
}
}  // namespace tc

template <typename T>
int gram_tc(int64_t n, int m, int k, double alpha, const T *X, int64_t ldx, const T *Y,
            int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    return gram<T>(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, 0, ws, st);
  } else {
    if (n > 0) {   // TMA-fed kernel first (any m, k); the staged kernel takes the rest
      const int s = gram_tma(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, ws, st);
      if (s != GCGE_EINVAL) return s;
    }
    // up to 4 M-tiles of 128 and N <= 128 per launch; wider shapes are split
    const int mmax = 512, kmax = 128;
    if (m > mmax || k > kmax) {
      for (int i0 = 0; i0 < m; i0 += mmax)
        for (int j0 = 0; j0 < k; j0 += kmax) {
          const int mm = std::min(mmax, m - i0), kk = std::min(kmax, k - j0);
          GCGE_CHECK(gram_tc<T>(n, mm, kk, alpha, X + i0, ldx, Y + j0, ldy, beta,
                                C + i0 + (int64_t)j0 * ldc, ldc, ws, st));
        }
      return GCGE_OK;
    }
    const int MT = (m + 127) / 128;
    const int Np = ((k + 15) / 16) * 16;
    int *err = nullptr;
    GCGE_CHECK(tc::err_flag(&err));
    int64_t splits = 2 * (int64_t)device_sm_count();
    int64_t rps = round_up((n + splits - 1) / splits, kKC);
    if (rps < kKC) rps = kKC;
    splits = (n + rps - 1) / rps;
    if (splits < 1) splits = 1;
    double *part = nullptr;
    GCGE_CHECK(ws.get(sizeof(double) * (size_t)splits * m * k, st, (void **)&part));
    const size_t smem = gram_tc_smem(MT, Np);
    static size_t attr = 0;
    if (smem > attr) {
      GCGE_CUDA(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(smem, 48 * 1024)));
      attr = smem;
    }
    gram_tc_kernel<<<(unsigned)splits, kTcThreads, smem, st>>>(n, m, k, MT, Np, (const float *)X,
                                                               ldx, (const float *)Y, ldy, rps,
                                                               part, err);
    GCGE_LAUNCH_CHECK();
    return gram_reduce_launch(m, k, (int)splits, part, alpha, beta, C, ldc, st);
  }
}

template <typename T>
int vc_tc(int64_t n, int d, int q, double alpha, const T *V, int64_t ldv, const double *C,
          int64_t ldc, double beta, T *Y, int64_t ldy, cudaStream_t st, Scratch *ws) {
  if constexpr (sizeof(T) == 8) {
    return vc<T>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, 0, st);
  } else {
    if (d == 0) return vc<T>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, 0, st);   // Y = beta Y
    if (ws) {   // TMA-fed kernel first; the staged kernel takes what it cannot address
      const int s = vc_tma(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, *ws, st);
      if (s != GCGE_EINVAL) return s;
    }
    const int Np = std::min(256, ((q + 15) / 16) * 16);
    const int qt = (q + Np - 1) / Np;
    int *err = nullptr;
    GCGE_CHECK(tc::err_flag(&err));
    const size_t smem = vc_tc_smem(Np);
    static size_t attr = 0;
    if (smem > attr) {
      GCGE_CUDA(cudaFuncSetAttribute(vc_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)std::max<size_t>(smem, 48 * 1024)));
      attr = smem;
    }
    dim3 grid((unsigned)((n + 127) / 128), (unsigned)qt);
    vc_tc_kernel<<<grid, kTcThreads, smem, st>>>(n, d, q, Np, (float)alpha, (const float *)V, ldv,
                                                 C, ldc, (float)beta, (float *)Y, ldy, err);
    GCGE_LAUNCH_CHECK();
    return GCGE_OK;
  }
}

template int gram_tc<float>(int64_t, int, int, double, const float *, int64_t, const float *,
                            int64_t, double, double *, int64_t, Scratch &, cudaStream_t);
template int gram_tc<double>(int64_t, int, int, double, const double *, int64_t, const double *,
                             int64_t, double, double *, int64_t, Scratch &, cudaStream_t);
template int vc_tc<float>(int64_t, int, int, double, const float *, int64_t, const double *,
                          int64_t, double, float *, int64_t, cudaStream_t, Scratch *);
template int vc_tc<double>(int64_t, int, int, double, const double *, int64_t, const double *,
                           int64_t, double, double *, int64_t, cudaStream_t, Scratch *);

// Device flag set by a tensor-core kernel whose bounded mbarrier wait timed out.
// Read and clear it (a set flag is reported once).
int tc_error_flag(int *host_val, cudaStream_t st) {
  int *err = nullptr;
  GCGE_CHECK(tc::err_flag(&err));
  GCGE_CUDA(cudaMemcpyAsync(host_val, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GCGE_CUDA(cudaStreamSynchronize(st));
  if (*host_val) GCGE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  return GCGE_OK;
}

}  // namespace gcge
