// Tall-skinny block products (Gram X^T Y and update V C) and small dense helpers.
//
// Gram (MultiVecInnerProd, Section 3.4): the reduction runs over the long
// dimension n.  The grid is (m-tiles) x (k-tiles) x (row splits); each CTA
// stages a chunk of rows of both blocks in shared memory and accumulates a
// 64 x 32 output tile in registers (4 x 2 per thread), then writes one FP64
// partial per split.  A second kernel sums the partials in a fixed order and
// writes alpha * sum + beta * C straight into the strided sub-block of the
// caller's column-major matrix (Eq. Dense_SubMatrix), so no extra workspace
// of the full Rayleigh-Ritz size is needed.
//
// Update (V C): a classic smem-tiled SIMT GEMM over 64-row x 32-column output
// tiles with C staged (and, for FP32 blocks, rounded) in shared memory.
#include "blas.cuh"

namespace gcge {

int Scratch::get(size_t need, cudaStream_t st, void **out) {
  if (need > bytes) {
    if (ptr) cudaFreeAsync(ptr, st);
    ptr = nullptr;
    bytes = 0;
    size_t nb = need + need / 4 + 4096;
    cudaError_t e = cudaMallocAsync(&ptr, nb, st);
    if (e != cudaSuccess) {
      record_cuda_error(e, __FILE__, __LINE__);
      ptr = nullptr;
      return GCGE_ENOMEM;
    }
    bytes = nb;
  }
  *out = ptr;
  return GCGE_OK;
}

void Scratch::release(cudaStream_t st) {
  if (ptr) cudaFreeAsync(ptr, st);
  ptr = nullptr;
  bytes = 0;
}

namespace {

// ------------------------------------------------------------------ Gram
constexpr int GM = 64, GK = 32, GR = 32;   // tile m, tile k, rows per smem stage

template <typename T>
__global__ void __launch_bounds__(256)
gram_partial_kernel(int64_t n, int m, int k, const T *__restrict__ X, int64_t ldx,
                    const T *__restrict__ Y, int64_t ldy, int64_t rows_per_split,
                    double *__restrict__ part) {
  __shared__ T sx[GR][GM + 1];
  __shared__ T sy[GR][GK + 1];
  const int tm = blockIdx.x, tk = blockIdx.y, sp = blockIdx.z;
  const int m0 = tm * GM, k0 = tk * GK;
  const int tx = threadIdx.x & 15;   // 16 x 16 threads; thread owns rows tx*4.. of the m-tile
  const int ty = threadIdx.x >> 4;   // and columns ty*2.. of the k-tile
  const int64_t r0 = (int64_t)sp * rows_per_split;
  int64_t r1 = r0 + rows_per_split;
  if (r1 > n) r1 = n;
  T acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
  for (int64_t rb = r0; rb < r1; rb += GR) {
    // stage GR rows of X[:, m0:m0+GM] and Y[:, k0:k0+GK]
    for (int t = threadIdx.x; t < GR * GM; t += 256) {
      const int rr = t / GM, cc = t % GM;
      const int64_t r = rb + rr;
      sx[rr][cc] = (r < r1 && m0 + cc < m) ? X[r * ldx + m0 + cc] : T(0);
    }
    for (int t = threadIdx.x; t < GR * GK; t += 256) {
      const int rr = t / GK, cc = t % GK;
      const int64_t r = rb + rr;
      sy[rr][cc] = (r < r1 && k0 + cc < k) ? Y[r * ldy + k0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GR; ++rr) {
      T xv[4], yv[2];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = sx[rr][tx * 4 + a];
      yv[0] = sy[rr][ty * 2];
      yv[1] = sy[rr][ty * 2 + 1];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a][0] += xv[a] * yv[0];
        acc[a][1] += xv[a] * yv[1];
      }
    }
    __syncthreads();
  }
  // partial layout: [split][k][m] (column-major m x k per split)
  double *pp = part + (int64_t)sp * m * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = m0 + tx * 4 + a, j = k0 + ty * 2 + b;
      if (i < m && j < k) pp[(int64_t)j * m + i] = (double)acc[a][b];
    }
}

// FP64 Gram with exact-fit tiles: the FP64 units are the bound on this GPU, so the
// tile (TMx x TKx <= 64 x 32, chosen per call to cover m and k with little padding)
// gives every thread up to 8 outputs; output o = t + 256 i sits at (o % TMx, o / TMx).
template <int O>
__global__ void __launch_bounds__(256)
gram64_partial_kernel(int64_t n, int m, int k, int TMx, int TKx, const double *__restrict__ X,
                      int64_t ldx, const double *__restrict__ Y, int64_t ldy,
                      int64_t rows_per_split, double *__restrict__ part) {
  __shared__ double sx[GR][GM + 1];
  __shared__ double sy[GR][GK + 1];
  const int m0 = blockIdx.x * TMx, k0 = blockIdx.y * TKx;
  const int mt = (m - m0) < TMx ? (m - m0) : TMx;
  const int kt = (k - k0) < TKx ? (k - k0) : TKx;
  const int nout = mt * kt;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_split;
  int64_t r1 = r0 + rows_per_split;
  if (r1 > n) r1 = n;
  int om[O], ok[O];
  double acc[O];
#pragma unroll
  for (int i = 0; i < O; ++i) {
    const int o = threadIdx.x + 256 * i;
    om[i] = o < nout ? o % mt : 0;
    ok[i] = o < nout ? o / mt : 0;
    acc[i] = 0.0;
  }
  for (int64_t rb = r0; rb < r1; rb += GR) {
    for (int t = threadIdx.x; t < GR * mt; t += 256) {
      const int rr = t / mt, cc = t % mt;
      const int64_t r = rb + rr;
      sx[rr][cc] = r < r1 ? X[r * ldx + m0 + cc] : 0.0;
    }
    for (int t = threadIdx.x; t < GR * kt; t += 256) {
      const int rr = t / kt, cc = t % kt;
      const int64_t r = rb + rr;
      sy[rr][cc] = r < r1 ? Y[r * ldy + k0 + cc] : 0.0;
    }
    __syncthreads();
    // warps whose outputs all lie beyond the tile issue no FMAs (the FP64 pipe is the
    // bound, so padded outputs would cost as much as real ones)
#pragma unroll 4
    for (int rr = 0; rr < GR; ++rr) {
#pragma unroll
      for (int i = 0; i < O; ++i)
        if ((int)(threadIdx.x & ~31u) + 256 * i < nout) acc[i] += sx[rr][om[i]] * sy[rr][ok[i]];
    }
    __syncthreads();
  }
  double *pp = part + (int64_t)blockIdx.z * m * k;
#pragma unroll
  for (int i = 0; i < O; ++i) {
    const int o = threadIdx.x + 256 * i;
    if (o < nout) pp[(int64_t)(k0 + ok[i]) * m + (m0 + om[i])] = acc[i];
  }
}

void launch_gram64(dim3 grid, cudaStream_t st, int64_t n, int m, int k, int TMx, int TKx,
                   const double *X, int64_t ldx, const double *Y, int64_t ldy, int64_t rps,
                   double *part) {
  const int O = (TMx * TKx + 255) / 256;
  switch (O) {
#define GCGE_G64(o) \
    case o: gram64_partial_kernel<o><<<grid, 256, 0, st>>>(n, m, k, TMx, TKx, X, ldx, Y, ldy, rps, part); break;
    GCGE_G64(1) GCGE_G64(2) GCGE_G64(3) GCGE_G64(4) GCGE_G64(5) GCGE_G64(6) GCGE_G64(7)
    default: gram64_partial_kernel<8><<<grid, 256, 0, st>>>(n, m, k, TMx, TKx, X, ldx, Y, ldy, rps, part);
#undef GCGE_G64
  }
}

// C(i, j) = alpha sum_sp part[sp][t] + beta C(i, j), t = i + m j.  A CTA takes 32
// consecutive outputs (coalesced across the lanes) and 32 groups of splits: warp g sums
// the splits g, g + 32, ... in order, and the 32 group sums are added in group order,
// so the result is fixed for a given split count while many loads are in flight (a
// Gram with few outputs and hundreds of splits no longer waits on one serial chain).
constexpr int kRedGroups = 32;

__global__ void __launch_bounds__(32 * kRedGroups)
gram_reduce_kernel(int m, int k, int splits, const double *__restrict__ part, double alpha,
                   double beta, double *__restrict__ C, int64_t ldc) {
  __shared__ double sh[kRedGroups][33];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t mk = (int64_t)m * k;
  const int64_t t = (int64_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (t < mk)
    for (int sp = g; sp < splits; sp += kRedGroups) s += part[(int64_t)sp * mk + t];
  sh[g][lane] = s;
  __syncthreads();
  if (g == 0 && t < mk) {
    double tot = 0.0;
#pragma unroll 8
    for (int q = 0; q < kRedGroups; ++q) tot += sh[q][lane];
    const int i = (int)(t % m), j = (int)(t / m);
    double *cp = C + i + (int64_t)j * ldc;
    double out = alpha * tot;
    if (beta != 0.0) out += beta * *cp;
    *cp = out;
  }
}

int red_blocks(int64_t mk) { return (int)((mk + 31) / 32); }

// ------------------------------------------------------------------ V C
constexpr int VR = 64, VQ = 32, VD = 16;

template <typename T>
__global__ void __launch_bounds__(256)
vc_kernel(int64_t n, int d, int q, T alpha, const T *__restrict__ V, int64_t ldv,
          const double *__restrict__ C, int64_t ldc, T beta, T *__restrict__ Y, int64_t ldy) {
  __shared__ T sv[VR][VD + 1];
  __shared__ T sc[VD][VQ + 1];
  const int64_t rbase = (int64_t)blockIdx.x * VR;
  const int q0 = blockIdx.y * VQ;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // rows ty*4.., cols tx*2..
  T acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
  for (int d0 = 0; d0 < d; d0 += VD) {
    for (int t = threadIdx.x; t < VR * VD; t += 256) {
      const int rr = t / VD, cc = t % VD;
      const int64_t r = rbase + rr;
      sv[rr][cc] = (r < n && d0 + cc < d) ? V[r * ldv + d0 + cc] : T(0);
    }
    for (int t = threadIdx.x; t < VD * VQ; t += 256) {
      const int rr = t / VQ, cc = t % VQ;
      sc[rr][cc] = (d0 + rr < d && q0 + cc < q) ? (T)C[(d0 + rr) + (int64_t)(q0 + cc) * ldc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < VD; ++e) {
      T cv0 = sc[e][tx * 2], cv1 = sc[e][tx * 2 + 1];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T v = sv[ty * 4 + a][e];
        acc[a][0] += v * cv0;
        acc[a][1] += v * cv1;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = rbase + ty * 4 + a;
    if (r >= n) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = q0 + tx * 2 + b;
      if (j < q) {
        T *yp = Y + r * ldy + j;
        T out = alpha * acc[a][b];
        if (beta != T(0)) out += beta * *yp;
        *yp = out;
      }
    }
  }
}

// FP64 V C with exact-fit tiles: a CTA takes VFR rows and TQx <= 32 columns of Y
// (TQx chosen per call to cover q with little padding); output o = t + 256 i sits at
// row o / qt, column o % qt of the tile, so every lane of a live warp holds a real
// output and warps past the tile issue no FMAs.  The reduction over d runs in stages
// of VD columns of V.
constexpr int VFR = 128;

template <int O>
__global__ void __launch_bounds__(256)
vc64_fit_kernel(int64_t n, int d, int q, int TQx, double alpha, const double *__restrict__ V,
                int64_t ldv, const double *__restrict__ C, int64_t ldc, double beta,
                double *__restrict__ Y, int64_t ldy) {
  __shared__ double sv[VFR][VD + 1];
  __shared__ double sc[VD][33];
  const int64_t rbase = (int64_t)blockIdx.x * VFR;
  const int q0 = blockIdx.y * TQx;
  const int qt = (q - q0) < TQx ? (q - q0) : TQx;
  const int nout = VFR * qt;
  const int wbase = (int)(threadIdx.x & ~31u);
  int orow[O], oj[O];
  double acc[O];
#pragma unroll
  for (int i = 0; i < O; ++i) {
    const int o = threadIdx.x + 256 * i;
    orow[i] = o < nout ? o / qt : 0;
    oj[i] = o < nout ? o % qt : 0;
    acc[i] = 0.0;
  }
  for (int d0 = 0; d0 < d; d0 += VD) {
    const int dt = (d - d0) < VD ? (d - d0) : VD;
    for (int u = threadIdx.x; u < VFR * dt; u += 256) {
      const int rr = u / dt, cc = u % dt;
      const int64_t r = rbase + rr;
      sv[rr][cc] = r < n ? V[r * ldv + d0 + cc] : 0.0;
    }
    for (int u = threadIdx.x; u < dt * qt; u += 256) {
      const int rr = u / qt, cc = u % qt;
      sc[rr][cc] = C[(d0 + rr) + (int64_t)(q0 + cc) * ldc];
    }
    __syncthreads();
    for (int e = 0; e < dt; ++e) {
#pragma unroll
      for (int i = 0; i < O; ++i)
        if (wbase + 256 * i < nout) acc[i] = fma(sv[orow[i]][e], sc[e][oj[i]], acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < O; ++i) {
    const int o = threadIdx.x + 256 * i;
    const int64_t r = rbase + orow[i];
    if (o < nout && r < n) {
      double *yp = Y + r * ldy + q0 + oj[i];
      double out = alpha * acc[i];
      if (beta != 0.0) out += beta * *yp;
      *yp = out;
    }
  }
}

void launch_vc64(int64_t n, int d, int q, double alpha, const double *V, int64_t ldv,
                 const double *C, int64_t ldc, double beta, double *Y, int64_t ldy,
                 cudaStream_t st) {
  const int tq = ceil_div(q, 32);
  const int TQx = ceil_div(q, tq);
  const int O = (VFR * TQx + 255) / 256;
  dim3 grid((unsigned)ceil_div(n, VFR), (unsigned)tq);
  switch (O) {
#define GCGE_V64(o) \
    case o: vc64_fit_kernel<o><<<grid, 256, 0, st>>>(n, d, q, TQx, alpha, V, ldv, C, ldc, beta, Y, ldy); break;
    GCGE_V64(1) GCGE_V64(2) GCGE_V64(3) GCGE_V64(4) GCGE_V64(5) GCGE_V64(6) GCGE_V64(7)
    GCGE_V64(8) GCGE_V64(9) GCGE_V64(10) GCGE_V64(11) GCGE_V64(12) GCGE_V64(13) GCGE_V64(14)
    GCGE_V64(15)
    default: vc64_fit_kernel<16><<<grid, 256, 0, st>>>(n, d, q, TQx, alpha, V, ldv, C, ldc, beta, Y, ldy);
#undef GCGE_V64
  }
}

// ------------------------------------------------------------------ small FP64 GEMM
// C = alpha op(A) op(B) + beta C for the small dense FP64 products (Rayleigh-Ritz
// matrices): 8 x 8 output tiles (64 threads, one output each) so that a d x d product
// spreads over many more CTAs than SMs (the FP64 units are the limit), and the reduction
// dimension staged 64 deep so that a CTA waits on memory only every 64 FMAs.
constexpr int DT = 8, DK = 64;

__global__ void __launch_bounds__(DT * DT)
dgemm_small_kernel(int ta, int tb, int m, int n, int k, double alpha,
                   const double *__restrict__ A, int64_t lda, const double *__restrict__ B,
                   int64_t ldb, double beta, double *__restrict__ C, int64_t ldc) {
  __shared__ double sa[DT][DK + 1];   // sa[i][p] = op(A)(i0 + i, p0 + p)
  __shared__ double sb[DK][DT + 1];   // sb[p][j] = op(B)(p0 + p, j0 + j)
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * DT + tx;
  const int i0 = blockIdx.x * DT, j0 = blockIdx.y * DT;
  double acc = 0.0;
  for (int p0 = 0; p0 < k; p0 += DK) {
#pragma unroll
    for (int u = 0; u < DT * DK / (DT * DT); ++u) {
      const int e = t + u * DT * DT;        // 0 .. DT*DK-1
      {  // op(A) tile: element (i, p), consecutive threads along the contiguous index
        const int i = ta ? e / DK : e % DT, pp = ta ? e % DK : e / DT;
        const int ii = i0 + i, kp = p0 + pp;
        double v = 0.0;
        if (ii < m && kp < k) v = ta ? A[kp + (int64_t)ii * lda] : A[ii + (int64_t)kp * lda];
        sa[i][pp] = v;
      }
      {  // op(B) tile: element (p, j)
        const int j = tb ? e % DT : e / DK, pp = tb ? e / DT : e % DK;
        const int jj = j0 + j, kp = p0 + pp;
        double v = 0.0;
        if (kp < k && jj < n) v = tb ? B[jj + (int64_t)kp * ldb] : B[kp + (int64_t)jj * ldb];
        sb[pp][j] = v;
      }
    }
    __syncthreads();
#pragma unroll 16
    for (int e = 0; e < DK; ++e) acc = fma(sa[tx][e], sb[e][ty], acc);
    __syncthreads();
  }
  const int i = i0 + tx, j = j0 + ty;
  if (i < m && j < n) {
    double *cp = C + i + (int64_t)j * ldc;
    double out = alpha * acc;
    if (beta != 0.0) out += beta * *cp;
    *cp = out;
  }
}

// ------------------------------------------------------------------ column reductions
constexpr int kRedThreads = 256;

template <typename T>
__global__ void col_dots_kernel(int64_t n, int k, const T *__restrict__ X, int64_t ldx,
                                const T *__restrict__ Y, int64_t ldy, double *__restrict__ part) {
  // thread t of the block handles column (t % kc) over rows (t / kc) + s * (256 / kc)
  extern __shared__ double sred[];
  const int kc = k < kRedThreads ? k : kRedThreads;
  const int rows_per_pass = kRedThreads / kc;
  for (int j0 = 0; j0 < k; j0 += kc) {
    const int jj = threadIdx.x % kc, rr = threadIdx.x / kc;
    const int j = j0 + jj;
    double acc = 0.0;
    if (rr < rows_per_pass && j < k) {
      for (int64_t r = (int64_t)blockIdx.x * rows_per_pass + rr; r < n;
           r += (int64_t)gridDim.x * rows_per_pass)
        acc += (double)X[r * ldx + j] * (double)Y[r * ldy + j];
    }
    sred[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < kc && j0 + threadIdx.x < k) {
      double s = 0.0;
      for (int t = threadIdx.x; t < rows_per_pass * kc; t += kc) s += sred[t];
      part[(int64_t)blockIdx.x * k + j0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void residual_kernel(int64_t n, int m, const T *__restrict__ X, int64_t ldx,
                                const T *__restrict__ AX, int64_t lda, const T *__restrict__ BX,
                                int64_t ldb, const double *__restrict__ lam,
                                double *__restrict__ part) {
  extern __shared__ double sred[];
  const int kc = m < kRedThreads ? m : kRedThreads;
  const int rows_per_pass = kRedThreads / kc;
  for (int j0 = 0; j0 < m; j0 += kc) {
    const int jj = threadIdx.x % kc, rr = threadIdx.x / kc;
    const int j = j0 + jj;
    double a1 = 0.0, a2 = 0.0;
    if (rr < rows_per_pass && j < m) {
      const double l = lam[j];
      for (int64_t r = (int64_t)blockIdx.x * rows_per_pass + rr; r < n;
           r += (int64_t)gridDim.x * rows_per_pass) {
        const double x = (double)X[r * ldx + j];
        const double bx = BX ? (double)BX[r * ldb + j] : x;
        const double res = (double)AX[r * lda + j] - l * bx;
        a1 += res * res;
        a2 += x * bx;
      }
    }
    sred[threadIdx.x] = a1;
    sred[kRedThreads + threadIdx.x] = a2;
    __syncthreads();
    if (threadIdx.x < kc && j0 + threadIdx.x < m) {
      double s1 = 0.0, s2 = 0.0;
      for (int t = threadIdx.x; t < rows_per_pass * kc; t += kc) {
        s1 += sred[t];
        s2 += sred[kRedThreads + t];
      }
      part[(int64_t)blockIdx.x * 2 * m + j0 + threadIdx.x] = s1;
      part[(int64_t)blockIdx.x * 2 * m + m + j0 + threadIdx.x] = s2;
    }
    __syncthreads();
  }
}

template <typename TI, typename TO>
__global__ void copy_cols_kernel(int64_t n, int k, const TI *__restrict__ X, int64_t ldx,
                                 TO *__restrict__ Y, int64_t ldy, const double *__restrict__ s) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    double v = (double)X[r * ldx + j];
    if (s) v *= s[j];
    Y[r * ldy + j] = (TO)v;
  }
}

template <typename TI, typename TO>
__global__ void add_cols_kernel(int64_t n, int k, const TI *__restrict__ X, int64_t ldx,
                                TO *__restrict__ Y, int64_t ldy) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    Y[r * ldy + j] += (TO)X[r * ldx + j];
  }
}

template <typename T>
__global__ void axpby_cols_kernel(int64_t n, int k, const double *__restrict__ a,
                                  const T *__restrict__ P, int64_t ldp,
                                  const double *__restrict__ b, const T *__restrict__ Q,
                                  int64_t ldq, T *__restrict__ out, int64_t ldo) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    const double av = a ? a[j] : 1.0;
    const double bv = b ? b[j] : 0.0;
    double v = av * (double)P[r * ldp + j];
    if (Q) v += bv * (double)Q[r * ldq + j];
    out[r * ldo + j] = (T)v;
  }
}

template <typename T>
__global__ void gather_cols_kernel(int64_t n, int k, const int *__restrict__ idx,
                                   const T *__restrict__ X, int64_t ldx, T *__restrict__ Y,
                                   int64_t ldy) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    Y[r * ldy + j] = X[r * ldx + idx[j]];
  }
}

__device__ __forceinline__ uint64_t smix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void random_block_kernel(int64_t n, int k, uint64_t key, T *__restrict__ X,
                                    int64_t ld) {
  const int64_t tot = n * k;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = (uint64_t)t;   // = i * k + j for row-major element (i, j)
    const uint64_t a = smix(key + 2ull * c), b = smix(key + 2ull * c + 1ull);
    const double u1 = ((double)(a >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = ((double)(b >> 11) + 0.5) * 0x1.0p-53;
    const double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    const int64_t r = t / k;
    const int j = (int)(t % k);
    X[r * ld + j] = (T)z;
  }
}

template <typename T>
__global__ void shifted_values_kernel(int64_t nnz, const int *__restrict__ mapA,
                                      const double *__restrict__ valA,
                                      const int *__restrict__ mapB,
                                      const double *__restrict__ valB,
                                      const int *__restrict__ is_diag, double theta,
                                      T *__restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
    double v = mapA[t] >= 0 ? valA[mapA[t]] : 0.0;
    if (mapB) {
      if (mapB[t] >= 0) v -= theta * valB[mapB[t]];
    } else if (is_diag[t]) {
      v -= theta;
    }
    out[t] = (T)v;
  }
}

int elem_grid(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int red_grid(int64_t n) {
  int64_t g = (n + 1023) / 1024;
  const int64_t cap = (int64_t)device_sm_count() * 2;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename T>
int gram_tc(int64_t n, int m, int k, double alpha, const T *X, int64_t ldx, const T *Y,
            int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st);

int gram_reduce_launch(int m, int k, int splits, const double *part, double alpha, double beta,
                       double *C, int64_t ldc, cudaStream_t st) {
  gram_reduce_kernel<<<red_blocks((int64_t)m * k), 32 * kRedGroups, 0, st>>>(m, k, splits, part,
                                                                            alpha, beta, C, ldc);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int gram(int64_t n, int m, int k, double alpha, const T *X, int64_t ldx, const T *Y, int64_t ldy,
         double beta, double *C, int64_t ldc, int tc, Scratch &ws, cudaStream_t st) {
  if (m <= 0 || k <= 0) return GCGE_OK;
  if (tc) return gram_tc<T>(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, ws, st);
  const int tm = ceil_div(m, GM), tk = ceil_div(k, GK);
  const int64_t tiles = (int64_t)tm * tk;
  int64_t target = (int64_t)device_sm_count() * 4;
  int64_t splits = (target + tiles - 1) / tiles;
  const int64_t max_splits = (n + 4 * GR - 1) / (4 * GR);   // at least 128 rows per split
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  if (splits > 65535) splits = 65535;
  int64_t rps = (n + splits - 1) / splits;
  rps = round_up(rps, GR);
  splits = (n + rps - 1) / rps;
  if (splits < 1) splits = 1;
  double *part = nullptr;
  GCGE_CHECK(ws.get(sizeof(double) * (size_t)splits * m * k, st, (void **)&part));
  if (n > 0) {
    if (sizeof(T) == 8) {
      const int TMx = ceil_div(m, tm), TKx = ceil_div(k, tk);
      dim3 grid(tm, tk, (unsigned)splits);
      launch_gram64(grid, st, n, m, k, TMx, TKx, (const double *)X, ldx, (const double *)Y, ldy,
                    rps, part);
    } else {
      dim3 grid(tm, tk, (unsigned)splits);
      gram_partial_kernel<T><<<grid, 256, 0, st>>>(n, m, k, X, ldx, Y, ldy, rps, part);
    }
    GCGE_LAUNCH_CHECK();
  } else {
    GCGE_CUDA(cudaMemsetAsync(part, 0, sizeof(double) * m * k, st));
    splits = 1;
  }
  gram_reduce_kernel<<<red_blocks((int64_t)m * k), 32 * kRedGroups, 0, st>>>(m, k, (int)splits, part, alpha,
                                                                 beta, C, ldc);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

int gram_f64_workspace(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx,
                       const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                       double *ws, int64_t ws_doubles, cudaStream_t st) {
  if (m <= 0 || k <= 0) return GCGE_OK;
  const int64_t mk = (int64_t)m * k;
  if (mk > ws_doubles) return GCGE_EINVAL;
  const int tm = ceil_div(m, GM), tk = ceil_div(k, GK);
  const int64_t tiles = (int64_t)tm * tk;
  int64_t splits = ((int64_t)device_sm_count() * 4 + tiles - 1) / tiles;
  const int64_t max_splits = (n + 4 * GR - 1) / (4 * GR);
  if (splits > max_splits) splits = max_splits;
  if (splits > ws_doubles / mk) splits = ws_doubles / mk;
  if (splits > 65535) splits = 65535;
  if (splits < 1) splits = 1;
  int64_t rps = round_up((n + splits - 1) / splits, GR);
  if (rps < GR) rps = GR;
  splits = (n + rps - 1) / rps;
  if (splits < 1) splits = 1;
  if (n > 0) {
    dim3 grid(tm, tk, (unsigned)splits);
    gram_partial_kernel<double><<<grid, 256, 0, st>>>(n, m, k, X, ldx, Y, ldy, rps, ws);
    GCGE_LAUNCH_CHECK();
  } else {
    // nothing to reduce: the used partial block must read as zero
    GCGE_CUDA(cudaMemsetAsync(ws, 0, sizeof(double) * mk, st));
  }
  gram_reduce_kernel<<<red_blocks(mk), 32 * kRedGroups, 0, st>>>(m, k, (int)splits, ws, alpha, beta,
                                                                 C, ldc);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int vc_tc(int64_t n, int d, int q, double alpha, const T *V, int64_t ldv, const double *C,
          int64_t ldc, double beta, T *Y, int64_t ldy, cudaStream_t st, Scratch *ws);

template <typename T>
int vc(int64_t n, int d, int q, double alpha, const T *V, int64_t ldv, const double *C,
       int64_t ldc, double beta, T *Y, int64_t ldy, int tc, cudaStream_t st, Scratch *ws) {
  if (n <= 0 || q <= 0) return GCGE_OK;
  if (d < 0) return GCGE_EINVAL;   // d == 0 leaves Y = beta * Y
  if (tc) return vc_tc<T>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, st, ws);
  if (sizeof(T) == 8) {
    launch_vc64(n, d, q, alpha, (const double *)V, ldv, C, ldc, beta, (double *)Y, ldy, st);
  } else {
    dim3 grid((unsigned)ceil_div(n, VR), (unsigned)ceil_div(q, VQ));
    vc_kernel<T><<<grid, 256, 0, st>>>(n, d, q, (T)alpha, V, ldv, C, ldc, (T)beta, Y, ldy);
  }
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

int dgemm_small(char ta, char tb, int m, int n, int k, double alpha, const double *A, int64_t lda,
                const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                cudaStream_t st) {
  if (m <= 0 || n <= 0) return GCGE_OK;
  dim3 grid(ceil_div(m, DT), ceil_div(n, DT)), block(DT, DT);
  dgemm_small_kernel<<<grid, block, 0, st>>>(ta == 'T', tb == 'T', m, n, k, alpha, A, lda, B, ldb,
                                             beta, C, ldc);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int col_dots(int64_t n, int k, const T *X, int64_t ldx, const T *Y, int64_t ldy, double *out,
             Scratch &ws, cudaStream_t st) {
  if (k <= 0) return GCGE_OK;
  const int g = red_grid(n);
  double *part = nullptr;
  GCGE_CHECK(ws.get(sizeof(double) * (size_t)g * k, st, (void **)&part));
  col_dots_kernel<T><<<g, kRedThreads, kRedThreads * sizeof(double), st>>>(n, k, X, ldx, Y, ldy,
                                                                           part);
  GCGE_LAUNCH_CHECK();
  // out[j] = sum over the g partial rows (the split-K reduction of the Gram products)
  gram_reduce_kernel<<<red_blocks(k), 32 * kRedGroups, 0, st>>>(k, 1, g, part, 1.0, 0.0, out, k);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int residual_parts(int64_t n, int m, const T *X, int64_t ldx, const T *AX, int64_t lda,
                   const T *BX, int64_t ldb, const double *lam, double *out, Scratch &ws,
                   cudaStream_t st) {
  if (m <= 0) return GCGE_OK;
  const int g = red_grid(n);
  double *part = nullptr;
  GCGE_CHECK(ws.get(sizeof(double) * (size_t)g * 2 * m, st, (void **)&part));
  residual_kernel<T><<<g, kRedThreads, 2 * kRedThreads * sizeof(double), st>>>(
      n, m, X, ldx, AX, lda, BX, ldb, lam, part);
  GCGE_LAUNCH_CHECK();
  gram_reduce_kernel<<<red_blocks(2 * m), 32 * kRedGroups, 0, st>>>(2 * m, 1, g, part, 1.0, 0.0,
                                                                     out, 2 * m);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename TI, typename TO>
int copy_cols(int64_t n, int k, const TI *X, int64_t ldx, TO *Y, int64_t ldy, const double *s,
              cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  copy_cols_kernel<TI, TO><<<elem_grid(n * k), 256, 0, st>>>(n, k, X, ldx, Y, ldy, s);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int axpby_cols(int64_t n, int k, const double *a, const T *P, int64_t ldp, const double *b,
               const T *Q, int64_t ldq, T *out, int64_t ldo, cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  axpby_cols_kernel<T><<<elem_grid(n * k), 256, 0, st>>>(n, k, a, P, ldp, b, Q, ldq, out, ldo);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int gather_cols(int64_t n, int k, const int *idx, const T *X, int64_t ldx, T *Y, int64_t ldy,
                cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  gather_cols_kernel<T><<<elem_grid(n * k), 256, 0, st>>>(n, k, idx, X, ldx, Y, ldy);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

static uint64_t host_smix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
int random_block(int64_t n, int k, uint64_t seed, T *X, int64_t ld, cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  random_block_kernel<T><<<elem_grid(n * k), 256, 0, st>>>(n, k, host_smix(seed), X, ld);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template <typename T>
int shifted_values(int64_t nnz_u, const int *mapA, const double *valA, const int *mapB,
                   const double *valB, const int *is_diag, double theta, T *out,
                   cudaStream_t st) {
  if (nnz_u <= 0) return GCGE_OK;
  shifted_values_kernel<T><<<elem_grid(nnz_u), 256, 0, st>>>(nnz_u, mapA, valA, mapB, valB,
                                                             is_diag, theta, out);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

#define GCGE_INST(T)                                                                              \
  template int gram<T>(int64_t, int, int, double, const T *, int64_t, const T *, int64_t, double, \
                       double *, int64_t, int, Scratch &, cudaStream_t);                         \
  template int vc<T>(int64_t, int, int, double, const T *, int64_t, const double *, int64_t,      \
                     double, T *, int64_t, int, cudaStream_t, Scratch *);                         \
  template int col_dots<T>(int64_t, int, const T *, int64_t, const T *, int64_t, double *,       \
                           Scratch &, cudaStream_t);                                             \
  template int residual_parts<T>(int64_t, int, const T *, int64_t, const T *, int64_t,           \
                                 const T *, int64_t, const double *, double *, Scratch &,        \
                                 cudaStream_t);                                                   \
  template int axpby_cols<T>(int64_t, int, const double *, const T *, int64_t, const double *,   \
                             const T *, int64_t, T *, int64_t, cudaStream_t);                     \
  template int gather_cols<T>(int64_t, int, const int *, const T *, int64_t, T *, int64_t,       \
                              cudaStream_t);                                                      \
  template int random_block<T>(int64_t, int, uint64_t, T *, int64_t, cudaStream_t);              \
  template int shifted_values<T>(int64_t, const int *, const double *, const int *,              \
                                 const double *, const int *, double, T *, cudaStream_t);

GCGE_INST(double)
GCGE_INST(float)

template <typename TI, typename TO>
int add_cols(int64_t n, int k, const TI *X, int64_t ldx, TO *Y, int64_t ldy, cudaStream_t st) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  add_cols_kernel<TI, TO><<<elem_grid(n * k), 256, 0, st>>>(n, k, X, ldx, Y, ldy);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}
template int add_cols<float, double>(int64_t, int, const float *, int64_t, double *, int64_t,
                                     cudaStream_t);
template int add_cols<float, float>(int64_t, int, const float *, int64_t, float *, int64_t,
                                    cudaStream_t);
template int add_cols<double, double>(int64_t, int, const double *, int64_t, double *, int64_t,
                                      cudaStream_t);

template int copy_cols<double, double>(int64_t, int, const double *, int64_t, double *, int64_t,
                                       const double *, cudaStream_t);
template int copy_cols<float, float>(int64_t, int, const float *, int64_t, float *, int64_t,
                                     const double *, cudaStream_t);
template int copy_cols<float, double>(int64_t, int, const float *, int64_t, double *, int64_t,
                                      const double *, cudaStream_t);
template int copy_cols<double, float>(int64_t, int, const double *, int64_t, float *, int64_t,
                                      const double *, cudaStream_t);

}  // namespace gcge
