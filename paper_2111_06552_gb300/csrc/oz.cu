// FP64 products on the bf16 tensor cores by exact digit slices (Ozaki-style splitting).
//
// GB300 runs FP64 FMA at 1/64 of its FP32 rate, and the FP64 phase of the solver is
// made of tall-skinny Gram products X^T Y (reduction over the n rows) and block
// updates V C (reduction over the basis width d).  Both are computed here from
// exact integer pieces on the 5th-generation tensor cores:
//
//  * Slicing.  Along the reduction dimension the operands are cut into windows of
//    128 entries.  Within a window every row of an operand gets one exponent E with
//    max|x| < 2^E; x / 2^E is rounded to 49 fraction bits and written as seven
//    signed 7-bit digits d_1..d_7 (x / 2^E = sum_p d_p 2^-7p, error <= 2^-50).  Digit p
//    is stored as the bf16 number d_p 2^-7(p-1) (exact: at most 7 significant bits),
//    one plane per digit, K-major.  The slicing works on the FP64 bit patterns with
//    integer operations only.
//  * Products.  The 28 plane pairs (i, j) with i + j <= 8 are multiplied with
//    tcgen05.mma kind::f16 (bf16 in, FP32 accumulate).  A pair contributes at the
//    scale 2^-7(i+j-2); the pairs of one scale accumulate in their own
//    tensor-memory accumulator (seven of them), where every partial sum is an
//    integer multiple of that scale below 2^24 in magnitude (128 rows x at most 7
//    pairs x 127^2), so all seven sums are exact.  The dropped pairs (i + j >= 9)
//    and the digit truncation bound the error: about 2^-47 max|x| max|y| per term
//    (window maxima), against about 2^-53 sqrt(n) Sum|x||y| for an FP64 dot
//    product of n terms.
//  * Drain.  After each window the seven accumulators are read (tcgen05.ld),
//    turned into integers and combined exactly in int64, converted once, scaled by
//    the window's 2^(E_x + E_y) and added to FP64 registers.
//
// Kernel roles (192 threads): warp 0 issues TMA copies of the seven planes of each
// operand tile per stage of 32 reduction entries (64-byte rows, 64-byte swizzle);
// warp 1 allocates tensor memory and issues the MMAs (one elected lane); warps 2-5
// own the 128 accumulator lanes (drain and epilogue).  Every mbarrier wait is
// bounded; a timeout sets the device error flag read by gcge_tc_status and the
// solver.
#include <algorithm>

#include "blas.cuh"
#include "tcgen05.cuh"

namespace gcge {

int gram_reduce_launch(int m, int k, int splits, const double *part, double alpha, double beta,
                       double *C, int64_t ldc, cudaStream_t st);

namespace {
using namespace tc;

constexpr int kDigits = 7;
constexpr int kWin = 128;                  // reduction entries per exact window
constexpr int kKS = 32;                    // reduction entries per stage (64-byte rows)
constexpr int kStPerWin = kWin / kKS;      // stages per window
constexpr int kGroups = 7;                 // accumulators: one per scale s = i + j = 0..6
constexpr int kOzThreads = 192;
constexpr int kStages = 2;
constexpr int kExpZero = -4000;            // exponent of an all-zero window row
constexpr int kMaxN = 64;                  // output columns per CTA (7 x 64 TMEM columns)

// ------------------------------------------------------------------------ slicing
// Element (i, k) of the source is src[i * si + k * sk] (zero outside I x K).  One CTA
// takes 64 rows i by one window of 128 entries k (4 threads per row, 32 entries
// each).  Planes: P[(p * Rp + i) * Kp + k] (bf16 bits), exponents E[w * Rp + i].
constexpr int kSlRows = 64;
constexpr int kSlSeg = kWin / 32;          // threads per row
constexpr int kSlThreads = 256;
static_assert(kSlRows * kSlSeg == kSlThreads, "one thread per 32 entries of a row");

__device__ __forceinline__ uint16_t digit_bf16(uint32_t d, int p, uint32_t sign) {
  if (d == 0) return 0;
  const int h = 31 - __clz(d);                          // leading bit, 0..6
  const uint32_t mant = (d << (7 - h)) & 0x7Fu;
  const uint32_t ex = (uint32_t)(h - 7 * p + 127);
  return (uint16_t)((sign << 15) | (ex << 7) | mant);
}

__global__ void __launch_bounds__(kSlThreads)
oz_slice_kernel(const double *__restrict__ src, int64_t si, int64_t sk, int I, int64_t K,
                int Rp, int64_t Kp, uint16_t *__restrict__ P, int *__restrict__ E) {
  extern __shared__ unsigned long long tile[];   // [kSlRows][kWin + 1] bit patterns
  const int i0 = blockIdx.y * kSlRows;
  const int64_t k0 = (int64_t)blockIdx.x * kWin;
  const int t = threadIdx.x;
  constexpr int LD = kWin + 1;
  if (sk == 1) {
    for (int idx = t; idx < kSlRows * kWin; idx += kSlThreads) {
      const int i = idx / kWin, k = idx % kWin;
      unsigned long long v = 0;
      if (i0 + i < I && k0 + k < K) v = __double_as_longlong(src[(int64_t)(i0 + i) * si + k0 + k]);
      tile[i * LD + k] = v;
    }
  } else {
    for (int idx = t; idx < kSlRows * kWin; idx += kSlThreads) {
      const int i = idx % kSlRows, k = idx / kSlRows;
      unsigned long long v = 0;
      if (i0 + i < I && k0 + k < K) v = __double_as_longlong(src[(int64_t)(i0 + i) * si + (k0 + k) * sk]);
      tile[i * LD + k] = v;
    }
  }
  __syncthreads();
  // a warp takes 32 consecutive rows of one 32-entry segment: conflict-free reads of
  // the tile (odd row stride) and the segment maxima combined through shared memory
  const int i = t % kSlRows, seg = t / kSlRows;
  const unsigned long long *row = tile + i * LD + seg * 32;
  unsigned long long mx = 0;
#pragma unroll 8
  for (int kk = 0; kk < 32; ++kk) mx = max(mx, row[kk] & 0x7FFFFFFFFFFFFFFFull);
  __shared__ unsigned long long smax[kSlSeg][kSlRows];
  smax[seg][i] = mx;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kSlSeg; ++q) mx = max(mx, smax[q][i]);
  const int exmax = (int)(mx >> 52);
  const int Ex = mx == 0 ? kExpZero : exmax - 1022;     // max < 2^Ex
  if (seg == 0) E[blockIdx.x * (int64_t)Rp + i0 + i] = Ex;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    unsigned long long F[16];   // |x| / 2^Ex in 49 fraction bits, 16 entries at a time
    uint32_t signs = 0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const unsigned long long u = row[16 * half + kk];
      const int ex = (int)((u >> 52) & 0x7FF);
      signs |= (uint32_t)(u >> 63) << kk;
      unsigned long long f = 0;
      if (ex != 0 && Ex != kExpZero) {
        const int sh = 1026 + Ex - ex;                      // >= 4 since |x| < 2^Ex
        const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        // rounded to nearest (no bias toward zero); the top value stays below 2^49
        f = sh < 64 ? ((mant + (1ull << (sh - 1))) >> sh) : 0ull;
        f = f > 0x1FFFFFFFFFFFFull ? 0x1FFFFFFFFFFFFull : f;
      }
      F[kk] = f;
    }
#pragma unroll
    for (int p = 0; p < kDigits; ++p) {
      uint4 *dst = reinterpret_cast<uint4 *>(P + ((int64_t)p * Rp + i0 + i) * Kp + k0 + seg * 32 +
                                             16 * half);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int k1 = 8 * q + 2 * h, k2 = k1 + 1;
          const uint32_t a = digit_bf16((uint32_t)(F[k1] >> (42 - 7 * p)) & 127u, p, (signs >> k1) & 1u);
          const uint32_t b = digit_bf16((uint32_t)(F[k2] >> (42 - 7 * p)) & 127u, p, (signs >> k2) & 1u);
          w[h] = a | (b << 16);
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// ------------------------------------------------------------------------ products
// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ double pow2(int e) {
  if (e < -1022) return 0.0;
  if (e > 1023) e = 1023;
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// D(128 x N tile) = sum over the windows [w0, w1) of A_tile B_tile^T (both K-major
// planes); out[i * so_i + j * so_j] = alpha D + beta out for i < mv, j < nv.
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const int *__restrict__ EA, int RpA, const int *__restrict__ EB, int RpB, int N,
               int nwin, int wps, int mrow0, int mvalid, int nvalid, double alpha, double beta,
               double *__restrict__ out, int64_t so_i, int64_t so_j, int64_t so_split,
               int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], dfull, dfree, done;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.y, nt = blockIdx.z;
  const int w0 = blockIdx.x * wps, w1 = min(nwin, w0 + wps);
  const int nstage = (w1 - w0) * kStPerWin;
  const uint32_t abytes = (uint32_t)kDigits * 128 * 64, bbytes = (uint32_t)kDigits * N * 64;
  const uint32_t sbytes = (abytes + bbytes + 1023u) & ~1023u;
  const uint32_t ncols = 512;
  if (warp == 1) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&dfull, 1);
    mbar_init(&dfree, 128);
    mbar_init(&done, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  volatile int *ab = &abort_flag;

  if (warp == 0) {
    if (lane == 0 && nstage > 0) {
      int issued = 0;
      for (int it = 0; it < nstage; ++it) {
        const int s = it % kStages, u = it / kStages;
        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, err, ab)) break;
        mbar_expect_tx(&full[s], abytes + bbytes);
        const int k = (w0 * kStPerWin + it) * kKS;
        tma_load_3d(sm + s * sbytes, &tmA, k, mt * 128 + mrow0, 0, &full[s]);
        tma_load_3d(sm + s * sbytes + abytes, &tmB, k, nt * N, 0, &full[s]);
        ++issued;
      }
      for (int it = max(0, issued - kStages); it < issued; ++it)
        mbar_wait(&full[it % kStages], (it / kStages) & 1, err, nullptr);
    }
  } else if (warp == 1) {
    const bool leader = elect_one();
    const uint32_t id = idesc_bf16(128, N);
    int it = 0;
    for (; it < nstage; ++it) {
      const int s = it % kStages, u = it / kStages;
      const int wl = it % kStPerWin, wi = it / kStPerWin;
      if (wl == 0 && wi > 0 &&
          !__all_sync(0xFFFFFFFFu, mbar_wait(&dfree, (wi - 1) & 1, err, ab)))
        break;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&full[s], u & 1, err, ab))) break;
      tc_fence_after();
      const uint32_t abase = su32(sm + s * sbytes), bbase = abase + abytes;
      if (leader) {
        // plane pairs (i, j), 0-based, s = i + j <= 6, into accumulator s; the first
        // pair of an accumulator overwrites it at the start of a window
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
          for (int sd = 0; sd <= 6; ++sd) {
#pragma unroll
            for (int i = 0; i <= sd; ++i) {
              const int j = sd - i;
              const uint64_t ad = smem_desc_sw64(abase + i * (128 * 64) + ks * 32);
              const uint64_t bd = smem_desc_sw64(bbase + j * (N * 64) + ks * 32);
              const uint32_t acc = (wl > 0 || ks > 0 || i > 0) ? 1u : 0u;
              mma_bf16(tmem + sd * N, ad, bd, id, acc);
            }
          }
        }
      }
      __syncwarp();
      if (leader) {
        mma_commit(&empty[s]);
        if (wl == kStPerWin - 1) mma_commit(&dfull);
      }
      __syncwarp();
    }
    if (leader) {
      mma_commit(&done);
      mbar_wait(&done, 0, err, nullptr);   // issued MMAs are complete before TMEM is freed
    }
    __syncwarp();
  } else {
    // drain / epilogue: thread = accumulator lane (row of the 128 x N tile)
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    const int ia = mt * 128 + row;                 // row of A's planes (and of D)
    double acc[kMaxN];
#pragma unroll
    for (int j = 0; j < kMaxN; ++j) acc[j] = 0.0;
    bool ok = true;
    for (int wi = 0; wi < w1 - w0 && ok; ++wi) {
      if (!mbar_wait(&dfull, wi & 1, err, ab)) { ok = false; break; }
      tc_fence_after();
      const int w = w0 + wi;
      const int ea = EA[(int64_t)w * RpA + mrow0 + ia];
      const int *eb = EB + (int64_t)w * RpB + nt * N;
      // accumulator s holds an exact multiple of 2^-7s (in units of the leading product
      // 2^(Ex + Ey - 14)); I_s = acc_s 2^7s is an integer below 2^24.  The window sum in
      // units of 2^-28: T = sum_{s<=4} I_s 2^(28-7s) + round((I_5 2^7 + I_6) / 2^14),
      // exact in int64 up to that rounding (|T| < 2^50), then one conversion and one FMA.
#pragma unroll
      for (int jb = 0; jb < kMaxN; jb += 8) {
        if (jb < N) {
          // the seven accumulators' 8 columns in one batch of loads, one wait
          uint32_t gv[kGroups][8];
#pragma unroll
          for (int sd = 0; sd < kGroups; ++sd) {
            const uint32_t ta = tmem + lane_addr + sd * N + jb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(gv[sd][0]), "=r"(gv[sd][1]), "=r"(gv[sd][2]), "=r"(gv[sd][3]),
                  "=r"(gv[sd][4]), "=r"(gv[sd][5]), "=r"(gv[sd][6]), "=r"(gv[sd][7])
                : "r"(ta));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            long long T = 0, Lw = 0;
#pragma unroll
            for (int sd = 0; sd < kGroups; ++sd) {
              const float up = __int_as_float((127 + 7 * sd) << 23);   // 2^(7 sd)
              const long long I = (long long)__float2int_rn(__uint_as_float(gv[sd][u]) * up);
              if (sd <= 4) T += I << (28 - 7 * sd);
              else if (sd == 5) Lw = I << 7;
              else T += (Lw + I + (1ll << 13)) >> 14;   // rounded, not floored
            }
            acc[jb + u] += (double)T * pow2(ea + eb[jb + u] - 42);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&dfree);
    }
    if (ok && ia < mvalid) {
      double *o = out + blockIdx.x * so_split + (int64_t)ia * so_i + (int64_t)nt * N * so_j;
#pragma unroll
      for (int j = 0; j < kMaxN; ++j) {
        if (j < N && nt * N + j < nvalid) {
          double *oj = o + (int64_t)j * so_j;
          double v = alpha * acc[j];
          if (beta != 0.0) v += beta * *oj;
          *oj = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------ host
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn oz_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 3D map of a plane set P[7][Rp][Kp] (bf16), box 32 x rows x 7, 64-byte swizzle.
bool plane_map(CUtensorMap *map, const uint16_t *P, int Rp, int64_t Kp, int rows) {
  EncodeTiledFn fn = oz_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)Rp, (cuuint64_t)kDigits};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Rp * Kp * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kKS, (cuuint32_t)rows, (cuuint32_t)kDigits};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)P, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int slice(const double *src, int64_t si, int64_t sk, int I, int64_t K, int Rp, int64_t Kp,
          uint16_t *P, int *E, cudaStream_t st) {
  const size_t smem = (size_t)kSlRows * (kWin + 1) * 8;
  static bool attr = false;
  if (!attr) {
    GCGE_CUDA(cudaFuncSetAttribute(oz_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)(Kp / kWin), (unsigned)(Rp / kSlRows));
  oz_slice_kernel<<<grid, kSlThreads, smem, st>>>(src, si, sk, I, K, Rp, Kp, P, E);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

size_t gemm_smem(int N) {
  const uint32_t sbytes = ((uint32_t)kDigits * (128 + N) * 64 + 1023u) & ~1023u;
  return (size_t)kStages * sbytes + 1024;
}

int gemm_launch(const CUtensorMap &ma, const CUtensorMap &mb, const int *EA, int RpA,
                const int *EB, int RpB, int N, int nwin, int wps, int splits, int mtiles,
                int ntiles, int mrow0, int mvalid, int nvalid, double alpha, double beta,
                double *out, int64_t so_i, int64_t so_j, int64_t so_split, cudaStream_t st) {
  int *err = nullptr;
  GCGE_CHECK(tc::err_flag(&err));
  const size_t smem = gemm_smem(N);
  static size_t attr = 0;
  if (smem > attr) {
    GCGE_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = smem;
  }
  dim3 grid((unsigned)splits, (unsigned)mtiles, (unsigned)ntiles);
  oz_gemm_kernel<<<grid, kOzThreads, smem, st>>>(ma, mb, EA, RpA, EB, RpB, N, nwin, wps, mrow0,
                                                 mvalid, nvalid, alpha, beta, out, so_i, so_j,
                                                 so_split, err);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

// Output columns per CTA and their tile count for a width of q columns.
void n_tiling(int q, int *N, int *ntiles) {
  *ntiles = (q + kMaxN - 1) / kMaxN;
  *N = (((q + *ntiles - 1) / *ntiles) + 15) / 16 * 16;
}

// Scratch layout helper: carve aligned pieces out of one workspace.
struct Carve {
  unsigned char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    off = (off + 1023) & ~(size_t)1023;
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

constexpr size_t kPlaneBudget = (size_t)4 << 30;    // bytes of digit planes per pass

}  // namespace

// C(m x k, col-major ldc) = alpha X^T Y + beta C with X n x m, Y n x k row-major FP64.
// The rows are taken in chunks and the columns of X in groups of 128-column tiles so that
// the planes of one pass stay within kPlaneBudget; every CTA adds its share of each
// chunk into its own partial block, reduced at the end in a fixed order.
int oz_gram(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx, const double *Y,
            int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st) {
  if (m <= 0 || k <= 0) return GCGE_OK;
  if (n <= 0 || n > ((int64_t)1 << 30)) return GCGE_EINVAL;
  int N = 0, ntiles = 0;
  n_tiling(k, &N, &ntiles);
  const int RpB = (int)round_up((int64_t)ntiles * N, kSlRows);   // slicing works in row tiles
  const int mtiles_all = (m + 127) / 128;
  const int mchunk = std::min(mtiles_all, 4);
  const int RpA = mchunk * 128;
  const int64_t bytes_per_row = (int64_t)kDigits * 2 * (RpA + RpB);
  int64_t nc = std::max<int64_t>(kWin, (int64_t)(kPlaneBudget / bytes_per_row) / kWin * kWin);
  nc = std::min(nc, round_up(n, kWin));
  const int nwc = (int)(nc / kWin);                 // windows per row chunk
  const int sm_count = device_sm_count();
  int splits = std::max(1, sm_count / std::max(1, mchunk * ntiles));
  splits = std::min(splits, nwc);
  const size_t bytes = (size_t)kDigits * RpB * nc * 2 + (size_t)nwc * RpB * 4 +
                       (size_t)kDigits * RpA * nc * 2 + (size_t)nwc * RpA * 4 +
                       (size_t)splits * m * k * 8 + 8 * 1024;
  void *wsp = nullptr;
  GCGE_CHECK(ws.get(bytes, st, &wsp));
  Carve cv{static_cast<unsigned char *>(wsp)};
  uint16_t *PB = cv.take<uint16_t>((size_t)kDigits * RpB * nc);
  int *EBt = cv.take<int>((size_t)nwc * RpB);
  uint16_t *PA = cv.take<uint16_t>((size_t)kDigits * RpA * nc);
  int *EAt = cv.take<int>((size_t)nwc * RpA);
  double *part = cv.take<double>((size_t)splits * m * k);
  CUtensorMap mb, ma;
  if (!plane_map(&mb, PB, RpB, nc, N) || !plane_map(&ma, PA, RpA, nc, 128)) return GCGE_EINVAL;
  for (int64_t r0 = 0; r0 < n; r0 += nc) {
    const int64_t rows = std::min(nc, n - r0);
    const int nwin = (int)((rows + kWin - 1) / kWin);
    const int wps = (nwin + splits - 1) / splits;
    const int used = (nwin + wps - 1) / wps;          // CTAs with windows; the rest add zero
    (void)used;
    // Y: rows of the B planes are the columns of Y, reduction over the rows of Y
    GCGE_CHECK(slice(Y + r0 * ldy, 1, ldy, k, rows, RpB, nc, PB, EBt, st));
    for (int t0 = 0; t0 < mtiles_all; t0 += mchunk) {
      const int tiles = std::min(mchunk, mtiles_all - t0);
      const int c0 = t0 * 128, cols = std::min(m - c0, tiles * 128);
      GCGE_CHECK(slice(X + r0 * ldx + c0, 1, ldx, cols, rows, RpA, nc, PA, EAt, st));
      // part[split][j][c0 + i] += this chunk's share (overwritten by the first chunk)
      GCGE_CHECK(gemm_launch(ma, mb, EAt, RpA, EBt, RpB, N, nwin, wps, splits, tiles, ntiles, 0,
                             cols, k, 1.0, r0 == 0 ? 0.0 : 1.0, part + c0, 1, m, (int64_t)m * k,
                             st));
    }
  }
  return gram_reduce_launch(m, k, splits, part, alpha, beta, C, ldc, st);
}

// Y(n x q) = alpha V C + beta Y with V n x d row-major, C d x q col-major, FP64.
int oz_vc(int64_t n, int d, int q, double alpha, const double *V, int64_t ldv, const double *C,
          int64_t ldc, double beta, double *Y, int64_t ldy, Scratch &ws, cudaStream_t st) {
  if (n <= 0 || q <= 0) return GCGE_OK;
  if (d <= 0 || n > ((int64_t)1 << 30)) return GCGE_EINVAL;
  const int64_t Kp = round_up(d, kWin);
  const int nwin = (int)(Kp / kWin);
  int N = 0, ntiles = 0;
  n_tiling(q, &N, &ntiles);
  const int RpB = (int)round_up((int64_t)ntiles * N, kSlRows);   // slicing works in row tiles
  const size_t per_row = (size_t)kDigits * Kp * 2;
  int64_t rchunk = (int64_t)std::max<size_t>(128, kPlaneBudget / per_row);
  rchunk = std::min<int64_t>(round_up(n, 128), (rchunk / 128) * 128);
  const int RpA = (int)rchunk;
  const size_t bytes = (size_t)kDigits * RpB * Kp * 2 + (size_t)nwin * RpB * 4 +
                       (size_t)kDigits * RpA * Kp * 2 + (size_t)nwin * RpA * 4 + 8 * 1024;
  void *wsp = nullptr;
  GCGE_CHECK(ws.get(bytes, st, &wsp));
  Carve cv{static_cast<unsigned char *>(wsp)};
  uint16_t *PB = cv.take<uint16_t>((size_t)kDigits * RpB * Kp);
  int *EBt = cv.take<int>((size_t)nwin * RpB);
  uint16_t *PA = cv.take<uint16_t>((size_t)kDigits * RpA * Kp);
  int *EAt = cv.take<int>((size_t)nwin * RpA);
  // C: rows of the B planes are the columns of C, reduction over the rows of C
  GCGE_CHECK(slice(C, ldc, 1, q, d, RpB, Kp, PB, EBt, st));
  CUtensorMap mb, ma;
  if (!plane_map(&mb, PB, RpB, Kp, N) || !plane_map(&ma, PA, RpA, Kp, 128)) return GCGE_EINVAL;
  for (int64_t r0 = 0; r0 < n; r0 += rchunk) {
    const int rows = (int)std::min<int64_t>(rchunk, n - r0);
    GCGE_CHECK(slice(V + r0 * ldv, ldv, 1, rows, d, RpA, Kp, PA, EAt, st));
    GCGE_CHECK(gemm_launch(ma, mb, EAt, RpA, EBt, RpB, N, nwin, nwin, 1, (rows + 127) / 128,
                           ntiles, 0, rows, q, alpha, beta, Y + r0 * ldy, ldy, 1, 0, st));
  }
  return GCGE_OK;
}

}  // namespace gcge
