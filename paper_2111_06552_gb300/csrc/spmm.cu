// CSR x row-major multivector product, Y = alpha A X + beta Y (MatDotMultiVec, Section 3.4).
//
// Layout: X and Y are row-major n x k (ld >= k), so every nonzero a_ij of row i
// gathers the contiguous k-vector X[j, 0:k].  The k columns are cut into 16-byte
// chunks (4 floats or 2 doubles) when the block is 16-byte aligned, else into single
// elements.  A group of G lanes owns one row; lane l of the group holds chunks
// l, l+G, ... (at most two of them when k allows) in registers, so for the block
// widths of the method (k = 2..100) a row needs 1..16 lanes and a warp works on 2..32
// rows at once.
// This keeps the per-nonzero instruction overhead (index, value, address) shared by
// a whole row's worth of FMAs and keeps many independent gathers in flight; the
// nonzero loop is unrolled by four.
//
// The rows are dealt to the CTAs in chunks of 2 CTA steps (256 / G rows per step), in
// turn, two to four CTAs per SM: within a chunk consecutive rows of a banded (stencil /
// FEM) matrix gather mostly the same rows of X, which stay in L1 between the CTA's
// steps; across the grid all CTAs sweep the rows together, so the rows of X that are
// gathered again a grid plane later (3D stencils) are still in L2.
//
// Optional fused epilogue (used by the CG step): per column j the dot product
// sum_i X[i, j] (A X)[i, j].  Each thread accumulates its own rows in the block's
// precision (FP32 for FP32 blocks: the dot only steers the inexact inner CG); after
// the row loop the lanes holding the same columns reduce over the warp's row groups
// with shuffles (in FP64), each warp writes its own shared-memory slot, the warps'
// slots are summed in warp order into the CTA's partial row, and the last CTA to
// finish (atomic ticket) sums the partial rows in a fixed order into dot_out[0:k].
// Every sum runs in a fixed order, so the dots are bitwise reproducible for a given
// grid.
#include "spmm.cuh"

namespace gcge {

namespace {

constexpr int kSpmmThreads = 256;

template <typename T, int VEC>
struct VecT;
template <>
struct VecT<float, 4> { using type = float4; };
template <>
struct VecT<double, 2> { using type = double2; };
template <typename T>
struct VecT<T, 1> { using type = T; };

template <typename T, int VEC>
__device__ __forceinline__ void load_chunk(const T *p, T (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = __ldg(p);
  } else {
    using V = typename VecT<T, VEC>::type;
    const V t = __ldg(reinterpret_cast<const V *>(p));
    if constexpr (VEC == 4) {
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      v[0] = t.x; v[1] = t.y;
    }
  }
}

template <typename T, int VEC, int NV, bool DOT>
__global__ void __launch_bounds__(kSpmmThreads)
spmm_kernel(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
            const T *__restrict__ val, int k, int G, T alpha, const T *__restrict__ X,
            int64_t ldx, T beta, T *__restrict__ Y, int64_t ldy, double *__restrict__ part,
            double *__restrict__ dot_out, unsigned *__restrict__ ticket, int64_t chunk_rows) {
  extern __shared__ double sdot[];   // per-warp column sums (warps x k), then blockDim.x scratch
  const int nchunks = (k + VEC - 1) / VEC;
  const int full = k / VEC;                 // chunks that are complete
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);            // lane within the row group
  T dacc[DOT ? NV : 1][VEC];                // this thread's share of the fused dots
#pragma unroll
  for (int c = 0; c < (DOT ? NV : 1); ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) dacc[c][v] = T(0);
  const int64_t rows_per_step = blockDim.x / G;
  // chunks of consecutive rows dealt to the CTAs in turn: the whole grid sweeps the rows
  // together, so the rows of X that a row's neighbours (in a 3D stencil, up to a grid
  // plane away) gather again are still in L2 when they do
  for (int64_t c0 = (int64_t)blockIdx.x * chunk_rows; c0 < n; c0 += (int64_t)gridDim.x * chunk_rows) {
  const int64_t blk_end = min(n, c0 + chunk_rows);
  for (int64_t row = c0 + threadIdx.x / G; row - (threadIdx.x / G) < blk_end;
       row += rows_per_step) {
    T acc[NV][VEC];
#pragma unroll
    for (int c = 0; c < NV; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = T(0);
    const bool live = row < blk_end;
    if (live) {
      const int beg = __ldg(rp + row), end = __ldg(rp + row + 1);
      int e = beg;
      // groups of four nonzeros; the next group's indices and values are loaded before
      // this group's gathers, so their latency overlaps instead of adding up
      int cc[4], cn[4];
      T vv[4], vn[4];
      if (e + 3 < end) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cc[u] = __ldg(ci + e + u);
          vv[u] = __ldg(val + e + u);
        }
      }
      for (; e + 3 < end; e += 4) {
        const bool more = e + 7 < end;
        if (more) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            cn[u] = __ldg(ci + e + 4 + u);
            vn[u] = __ldg(val + e + 4 + u);
          }
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int ch = gl + c * G;
          if (ch < full) {
            T xv[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              load_chunk<T, VEC>(X + (int64_t)cc[u] * ldx + ch * VEC, xv[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < VEC; ++v) acc[c][v] += vv[u] * xv[u][v];
          } else if (ch < nchunks) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              for (int v = 0; v < VEC && ch * VEC + v < k; ++v)
                acc[c][v] += vv[u] * __ldg(X + (int64_t)cc[u] * ldx + ch * VEC + v);
          }
        }
        if (more) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            cc[u] = cn[u];
            vv[u] = vn[u];
          }
        }
      }
      for (; e < end; ++e) {
        const int c0 = __ldg(ci + e);
        const T v0 = __ldg(val + e);
        const T *xr = X + (int64_t)c0 * ldx;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int ch = gl + c * G;
          if (ch < full) {
            T xv[VEC];
            load_chunk<T, VEC>(xr + ch * VEC, xv);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] += v0 * xv[v];
          } else if (ch < nchunks) {
            for (int v = 0; v < VEC && ch * VEC + v < k; ++v) acc[c][v] += v0 * __ldg(xr + ch * VEC + v);
          }
        }
      }
      // epilogue: Y = alpha acc + beta Y
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        const int ch = gl + c * G;
        if (ch >= nchunks) continue;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const int j = ch * VEC + v;
          if (j < k) {
            T *yp = Y + row * ldy + j;
            T out = alpha * acc[c][v];
            if (beta != T(0)) out += beta * *yp;
            *yp = out;
          }
        }
      }
    }
    if (DOT && live) {
      // per column: X[row, j] * (A X)[row, j] into this thread's accumulators
#pragma unroll
      for (int c = 0; c < NV; ++c) {
        const int ch = gl + c * G;
        if (ch < full) {
          T xv[VEC];
          load_chunk<T, VEC>(X + row * ldx + ch * VEC, xv);
#pragma unroll
          for (int v = 0; v < VEC; ++v) dacc[c][v] += xv[v] * acc[c][v];
        } else if (ch < nchunks) {
          for (int v = 0; v < VEC && ch * VEC + v < k; ++v)
            dacc[c][v] += __ldg(X + row * ldx + ch * VEC + v) * acc[c][v];
        }
      }
    }
  }
  }
  if (DOT) {
    // reduce over the warp's row groups (fixed butterfly order), one slot per warp
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const int ch = gl + c * G;
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        double d = (double)dacc[c][v];
        for (int o = G; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const int j = ch * VEC + v;
        if (lane < G && ch < nchunks && j < k) sdot[warp * k + j] = d;
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += sdot[w * k + j];
      part[(int64_t)blockIdx.x * k + j] = t;
    }
    last_cta_reduce(k, part, ticket, sdot + nwarps * k, [&](int j, double v) { dot_out[j] = v; });
  }
}

struct Plan {
  int vec, G, nv, grid;
  int64_t chunk_rows;
};

template <typename T>
Plan plan_for(int64_t n, int k, bool aligned) {
  const int vec = aligned ? (int)(16 / sizeof(T)) : 1;
  const int chunks = (k + vec - 1) / vec;
  int G = 1;
  // FP32 blocks up to 32 columns: at most two 16-byte chunks per lane (short register
  // footprint, four CTAs per SM).  Wider FP32 blocks: one chunk per lane, so a warp (or
  // a part of one) covers a whole row: each gather is one coalesced request of the
  // row's bytes, and the warps of a CTA walk consecutive rows, whose neighbour rows of
  // X they share in L1.  FP64 blocks: up to eight chunks per lane, two CTAs per SM (the
  // FP64 pipe is the bound).
  const bool narrow = sizeof(T) == 4 && k <= 32;
  const bool wide32 = sizeof(T) == 4 && !narrow;
  const int cpl = narrow ? 2 : (wide32 ? 1 : 8);
  while ((chunks + G - 1) / G > cpl && G < 32) G <<= 1;
  int nv = (chunks + G - 1) / G;
  if (nv > 8) nv = 8;           // k > 32 * 8 * vec: the caller splits the columns
  const int64_t step = kSpmmThreads / G;   // rows per CTA step
  int64_t grid = (n + step - 1) / step;
  const int64_t cap = (int64_t)device_sm_count() * (sizeof(T) == 4 ? 4 : 2);   // row streams per SM
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  const int64_t chunk = step * 2;   // rows per chunk: 2 CTA steps
  const int64_t nchunk = (n + chunk - 1) / chunk;
  if (grid > nchunk) grid = nchunk;
  if (grid < 1) grid = 1;
  return {vec, G, nv, (int)grid, chunk};
}

template <typename T, int VEC, int NV>
void launch_v(const Plan &pl, int64_t n, const int32_t *rp, const int32_t *ci, const T *val,
              int k, T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *part,
              double *dot_out, unsigned *ticket, cudaStream_t st) {
  static bool carveout = false;   // X rows are re-read through L1: prefer L1 over shared
  if (!carveout) {
    // the fused-dot variant keeps k doubles per warp in shared memory: leave room for
    // four CTAs per SM (a zero carveout held it to one)
    cudaFuncSetAttribute(spmm_kernel<T, VEC, NV, true>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 25);
    // the fused dot keeps one k-wide slot per warp (k <= 1024: 66 KB)
    cudaFuncSetAttribute(spmm_kernel<T, VEC, NV, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (1024 * (kSpmmThreads / 32) + kSpmmThreads) * (int)sizeof(double));
    cudaFuncSetAttribute(spmm_kernel<T, VEC, NV, false>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carveout = true;
  }
  if (dot_out)
    spmm_kernel<T, VEC, NV, true><<<pl.grid, kSpmmThreads,
                                    (k * (kSpmmThreads / 32) + kSpmmThreads) * sizeof(double), st>>>(
        n, rp, ci, val, k, pl.G, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, pl.chunk_rows);
  else
    spmm_kernel<T, VEC, NV, false><<<pl.grid, kSpmmThreads, 0, st>>>(
        n, rp, ci, val, k, pl.G, alpha, X, ldx, beta, Y, ldy, nullptr, nullptr, nullptr,
        pl.chunk_rows);
}

template <typename T, int VEC>
void launch_nv(const Plan &pl, int64_t n, const int32_t *rp, const int32_t *ci, const T *val,
               int k, T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *part,
               double *dot_out, unsigned *ticket, cudaStream_t st) {
  if (pl.nv <= 2)
    launch_v<T, VEC, 2>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
  else if (pl.nv <= 4)
    launch_v<T, VEC, 4>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
  else if (pl.nv <= 6)
    launch_v<T, VEC, 6>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
  else
    launch_v<T, VEC, 8>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
}

template <typename T>
bool aligned16(const T *X, int64_t ldx, const T *Y, int64_t ldy) {
  constexpr int vec = 16 / sizeof(T);
  return ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0) && (ldx % vec == 0) &&
         (ldy % vec == 0);
}

}  // namespace

int spmm_dot_blocks(int64_t n, int k) {
  // the dot variant is launched by the CG step on 16-byte aligned blocks of either type;
  // return the larger of the two plans so a partial buffer sized by it always fits
  const Plan a = plan_for<float>(n, k, true), b = plan_for<double>(n, k, true);
  const Plan c = plan_for<float>(n, k, false), d = plan_for<double>(n, k, false);
  int g = a.grid;
  if (b.grid > g) g = b.grid;
  if (c.grid > g) g = c.grid;
  if (d.grid > g) g = d.grid;
  return g;
}

template <typename T>
int launch_spmm(int64_t n, const int32_t *rp, const int32_t *ci, const T *val, int k, T alpha,
                const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *dot_out,
                int dot_blocks, cudaStream_t st, double *part, unsigned *ticket) {
  if (n <= 0 || k <= 0) return GCGE_OK;
  constexpr int vmax = 16 / sizeof(T);
  const bool al = aligned16<T>(X, ldx, Y, ldy);
  const int maxk = 32 * 8 * (al ? vmax : 1);
  if (k > maxk) {   // very wide blocks: split the columns (no fused dot across splits)
    if (dot_out) return GCGE_EINVAL;
    for (int j0 = 0; j0 < k; j0 += maxk) {
      const int kk = (k - j0) < maxk ? (k - j0) : maxk;
      GCGE_CHECK(launch_spmm<T>(n, rp, ci, val, kk, alpha, X + j0, ldx, beta, Y + j0, ldy, nullptr,
                                0, st, nullptr, nullptr));
    }
    return GCGE_OK;
  }
  const Plan pl = plan_for<T>(n, k, al);
  if (dot_out && (pl.grid > dot_blocks || !part || !ticket)) return GCGE_EINVAL;
  if (al)
    launch_nv<T, vmax>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
  else
    launch_nv<T, 1>(pl, n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, part, dot_out, ticket, st);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

template int launch_spmm<double>(int64_t, const int32_t *, const int32_t *, const double *, int,
                                 double, const double *, int64_t, double, double *, int64_t,
                                 double *, int, cudaStream_t, double *, unsigned *);
template int launch_spmm<float>(int64_t, const int32_t *, const int32_t *, const float *, int,
                                float, const float *, int64_t, float, float *, int64_t, double *,
                                int, cudaStream_t, double *, unsigned *);

}  // namespace gcge
