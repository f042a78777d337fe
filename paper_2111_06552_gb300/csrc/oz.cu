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
//    is stored unscaled, as the bf16 number d_p (exact: at most 7 significant bits),
//    one plane per digit, K-major.  The slicing works on the FP64 bit patterns with
//    integer operations only.  The small operand (B: the columns of Y, or of C) is
//    sliced into planes in global memory; the large one (A: the columns of X, or the
//    rows of V) is sliced inside the product, from FP64 straight into shared memory,
//    after a pre-pass that finds its window exponents.
//  * Products.  The 28 plane pairs (i, j) with i + j <= 8 are multiplied with
//    tcgen05.mma kind::f16 (bf16 in, FP32 accumulate).  A pair contributes at the
//    scale 2^-7(i+j); the pairs of one scale accumulate in their own tensor-memory
//    accumulator (seven of them), where every partial sum is an integer below 2^24 in
//    magnitude (128 rows x at most 7 pairs x 127^2), so all seven sums are exact.
//    The digit rounding of both operands and the dropped pairs (i + j >= 9) bound the
//    error by 2^(E_x + E_y - 46) per term (at most 2^-44 max|x| max|y|, window maxima;
//    about 2^-47 on random data), against about 2^-53 sqrt(n) Sum|x||y| for an FP64
//    dot product of n terms.
//  * Drain.  After each window the seven accumulators are read (tcgen05.ld),
//    turned into integers and combined exactly in int64, converted once, scaled by
//    the window's 2^(E_x + E_y) and added to FP64 registers.
//
// Kernel roles (320 threads): warp 0 issues TMA copies of B's seven planes per stage of
// 32 reduction entries (64-byte rows, 64-byte swizzle); warp 1 allocates tensor memory
// and issues the MMAs (one elected lane); warps 2-9 slice A into the stage buffers and
// drain the accumulators (epilogue included).  Every mbarrier wait is bounded; a
// timeout sets the device error flag read by gcge_tc_status and the solver.
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
constexpr int kMaxStages = 3;
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

// Digits are stored unscaled: plane p holds the signed integer d_p (|d_p| < 128) as a
// bf16 number, exact with at most 7 significant bits.  float(d) is formed without a
// conversion instruction (2^23 + d has d in its low mantissa bits), its low 16 bits are
// zero, and the upper half of two such floats packs into one 32-bit word of two bf16.
// The sign rides in the magic constant m = (-1)^s 2^23 (bit pattern 0x4B000000 with the
// sign bit): float(m | d) - float(m) = (-1)^s (2^23 + d) - (-1)^s 2^23 = (-1)^s d, exact.
__device__ __forceinline__ uint32_t digit_magic(unsigned long long u) {
  return 0x4B000000u | ((uint32_t)(u >> 32) & 0x80000000u);
}

__device__ __forceinline__ uint32_t digit_f32(uint32_t d, uint32_t magic) {
  return __float_as_uint(__uint_as_float(magic | d) - __uint_as_float(magic));
}

__device__ __forceinline__ uint32_t pack_bf16x2(uint32_t lo_f32, uint32_t hi_f32) {
  return __byte_perm(lo_f32, hi_f32, 0x7632);
}

// Digit p (0-based, most significant first) of F < 2^49: bits [42 - 7p, 49 - 7p).
// hi = F >> 21 holds digits 0-3, lo = F mod 2^21 digits 4-6 (32-bit shifts only).
__device__ __forceinline__ uint32_t digit_of(uint32_t hi, uint32_t lo, int p) {
  return p < 4 ? (hi >> (21 - 7 * p)) & 127u : (lo >> (14 - 7 * (p - 4))) & 127u;
}

// High 32 bits of |x| (exponent field and top mantissa bits).
__device__ __forceinline__ uint32_t hi_abs(double x) {
  return (uint32_t)__double2hiint(x) & 0x7FFFFFFFu;
}

// |x| / 2^Ex rounded to nearest at 49 fraction bits (kept below 2^49) from the FP64 bit
// pattern u, for |x| < 2^Ex; zeros and subnormals give 0 (an all-zero row has only
// those).  Branch-free: the shift is clamped to [4, 63] and the zero case selected.
__device__ __forceinline__ unsigned long long frac49(unsigned long long u, int Ex) {
  const int ex = (int)((u >> 52) & 0x7FF);
  int sh = 1026 + Ex - ex;                            // >= 4 when ex != 0 (|x| < 2^Ex)
  sh = sh < 4 ? 4 : (sh > 63 ? 63 : sh);
  const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long f = (mant + (1ull << (sh - 1))) >> sh;
  f = f > 0x1FFFFFFFFFFFFull ? 0x1FFFFFFFFFFFFull : f;
  return ex == 0 ? 0ull : f;
}

// Rows i >= Iw (padding that no product tile reads) are neither sliced nor given an
// exponent.
__global__ void __launch_bounds__(kSlThreads)
oz_slice_kernel(const double *__restrict__ src, int64_t si, int64_t sk, int I, int64_t K,
                int Rp, int64_t Kp, int Iw, uint16_t *__restrict__ P, int *__restrict__ E) {
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
  uint32_t mx = 0;   // largest high word (sign cleared): its exponent field is the max
#pragma unroll 8
  for (int kk = 0; kk < 32; ++kk) mx = max(mx, (uint32_t)(row[kk] >> 32) & 0x7FFFFFFFu);
  __shared__ uint32_t smax[kSlSeg][kSlRows];
  smax[seg][i] = mx;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kSlSeg; ++q) mx = max(mx, smax[q][i]);
  const int exmax = (int)(mx >> 20);
  const int Ex = exmax == 0 ? kExpZero : exmax - 1022;     // max < 2^Ex
  if (i0 + i >= Iw) return;
  if (seg == 0) E[blockIdx.x * (int64_t)Rp + i0 + i] = Ex;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    unsigned long long F[16];   // |x| / 2^Ex in 49 fraction bits, 16 entries at a time
    uint32_t magic[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const unsigned long long u = row[16 * half + kk];
      magic[kk] = digit_magic(u);
      F[kk] = frac49(u, Ex);
    }
    uint32_t fh[16], fl[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      fh[kk] = (uint32_t)(F[kk] >> 21);
      fl[kk] = (uint32_t)F[kk] & 0x1FFFFFu;
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
          w[h] = pack_bf16x2(digit_f32(digit_of(fh[k1], fl[k1], p), magic[k1]),
                             digit_f32(digit_of(fh[k2], fl[k2], p), magic[k2]));
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// Window exponents of the operand sliced inside the product: E[w * Rp + i] = E with
// max_k |A(i, k)| < 2^E over the window k in [128 w, 128 w + 128) (kExpZero for an
// all-zero window row, and for the padding rows I <= i < Rp).  Element (i, k) is
// src[i * si + k * sk]; one thread per row and window, the same rule as the slicer.
__global__ void __launch_bounds__(256)
oz_expo_kernel(const double *__restrict__ src, int64_t si, int64_t sk, int I, int64_t K, int Rp,
               int *__restrict__ E) {
  const int64_t w = blockIdx.x;
  const int i = blockIdx.y * 256 + threadIdx.x;
  if (i >= Rp) return;
  // the largest exponent field is the largest high word (sign cleared), shifted: a
  // 32-bit integer max (a 64-bit max of the bit patterns ran on the FP64 units)
  uint32_t mx = 0;
  if (i < I) {
    const int64_t k0 = w * kWin;
    const int64_t kn = (K - k0) < kWin ? (K - k0) : kWin;
    const double *p = src + (int64_t)i * si + k0 * sk;
    if (kn == kWin) {
#pragma unroll 16
      for (int k = 0; k < kWin; ++k) mx = max(mx, hi_abs(__ldg(p + k * sk)));
    } else {
      for (int64_t k = 0; k < kn; ++k) mx = max(mx, hi_abs(__ldg(p + k * sk)));
    }
  }
  E[w * Rp + i] = (mx >> 20) == 0 ? kExpZero : (int)(mx >> 20) - 1022;
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

// ------------------------------------------------------------------------ fused product
// The same product with the A operand sliced inside the kernel: A's FP64 entries are
// read from global memory, cut into the seven digits below the window exponents EA
// (computed by a pre-pass of oz_slice_kernel) and written straight into the stage's
// plane buffers in the 64-byte-swizzle layout that the MMA descriptors expect (16-byte
// unit c of row r at unit c ^ ((r >> 1) & 3)).  A's planes never reach global memory.
// B's planes (the small operand) come by TMA as before.
//   warp 0: TMA of B's planes; warp 1: MMA issuer;
//   warps 2-9 (256 workers): slicing of A (thread = A-row, half of a 32-entry stage) and
//   the window drain (thread = accumulator lane, half of the N columns).
// A worker drains window w after slicing the first nst stages of window w + 1, so
// the slicing of the next window overlaps the MMAs of the current one.
constexpr int kFuThreads = 320;
constexpr int kFuWorkers = 256;

// NH: the most columns one worker drains (N / 2 <= NH); 16 for N <= 32 keeps the
// accumulators and the prefetched loads in registers (10 warps allow 168 per thread).
template <int NH>
__global__ void __launch_bounds__(kFuThreads, 1)
oz_fused_kernel(const __grid_constant__ CUtensorMap tmB, const double *__restrict__ A,
                int64_t a_si, int64_t a_sk, int Arows, int64_t Klen, const int *__restrict__ EA,
                int RpA, const int *__restrict__ EB, int RpB, int N, int nwin, int wps,
                int mvalid, int nvalid, double alpha, double beta, double *__restrict__ out,
                int64_t so_i, int64_t so_j, int64_t so_split, int nst, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t fullb[kMaxStages], fulla[kMaxStages], empty[kMaxStages], dfull,
      dfree, done;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.y, nt = blockIdx.z;
  const int w0 = blockIdx.x * wps, w1 = min(nwin, w0 + wps);
  const int nw = max(0, w1 - w0);
  const int nstage = nw * kStPerWin;
  const uint32_t abytes = (uint32_t)kDigits * 128 * 64, bbytes = (uint32_t)kDigits * N * 64;
  const uint32_t sbytes = (abytes + bbytes + 1023u) & ~1023u;
  const uint32_t ncols = 512;
  if (warp == 1) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&fullb[s], 1);
      mbar_init(&fulla[s], kFuWorkers);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&dfull, 1);
    mbar_init(&dfree, kFuWorkers);
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
        const int s = it % nst, u = it / nst;
        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, err, ab)) break;
        mbar_expect_tx(&fullb[s], bbytes);
        const int k = (w0 * kStPerWin + it) * kKS;
        tma_load_3d(sm + s * sbytes + abytes, &tmB, k, nt * N, 0, &fullb[s]);
        ++issued;
      }
      for (int it = max(0, issued - nst); it < issued; ++it)
        mbar_wait(&fullb[it % nst], (it / nst) & 1, err, nullptr);
    }
  } else if (warp == 1) {
    const bool leader = elect_one();
    const uint32_t id = idesc_bf16(128, N);
    for (int it = 0; it < nstage; ++it) {
      const int s = it % nst, u = it / nst;
      const int wl = it % kStPerWin, wi = it / kStPerWin;
      if (wl == 0 && wi > 0 &&
          !__all_sync(0xFFFFFFFFu, mbar_wait(&dfree, (wi - 1) & 1, err, ab)))
        break;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&fulla[s], u & 1, err, ab))) break;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&fullb[s], u & 1, err, ab))) break;
      tc_fence_after();
      const uint32_t abase = su32(sm + s * sbytes), bbase = abase + abytes;
      if (leader) {
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
    const int wt = threadIdx.x - 64;
    const int srow = wt & 127, shalf = wt >> 7;   // slicing: A-row, 16-entry half of a stage
    const int ia_s = mt * 128 + srow;
    const bool rvalid = ia_s < Arows;
    const double *arow = A + (int64_t)ia_s * a_si;
    const int q = warp & 3;                        // TMEM lane quadrant of this warp
    const int ia_d = mt * 128 + 32 * q + lane;     // drain: accumulator lane = A-row
    const int nh = N >> 1, c0 = ((warp - 2) >> 2) * nh;   // drain: this warp's column half
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    double acc[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[j] = 0.0;
    bool ok = true;
    int wd = 0;   // next window to drain
    auto drain = [&](int wdi) -> bool {
      if (!mbar_wait(&dfull, wdi & 1, err, ab)) return false;
      tc_fence_after();
      const int w = w0 + wdi;
      const int ea = EA[(int64_t)w * RpA + ia_d];
      const int *eb = EB + (int64_t)w * RpB + nt * N + c0;
      // accumulator s holds the integer I_s = sum over i + j = s of d_i d_j (|I_s| < 2^24,
      // exact in FP32), in units of 2^(Ex + Ey - 14 - 7s).  The window sum in units of
      // 2^-28 (of 2^(Ex + Ey - 14)): T = sum_{s<=4} I_s 2^(28-7s) + round((I_5 2^7 + I_6)
      // / 2^14), exact in int64 up to that rounding (|T| < 2^50).
#pragma unroll
      for (int jb = 0; jb < NH; jb += 8) {
        if (jb < nh) {
          uint32_t gv[kGroups][8];
#pragma unroll
          for (int sd = 0; sd < kGroups; ++sd) {
            const uint32_t ta = tmem + lane_addr + sd * N + c0 + jb;
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
              const long long I = (long long)__float2int_rn(__uint_as_float(gv[sd][u]));
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
      return true;
    };
    // raw FP64 bits of this thread's 16 entries of stage it; the next stage's loads are
    // issued before the current one is sliced, so their latency overlaps the work
    unsigned long long raw[16];
    auto load = [&](int it, unsigned long long (&dst)[16]) {
      const int64_t k0 = (int64_t)(w0 * kStPerWin + it) * kKS + shalf * 16;
      if (rvalid && k0 + 16 <= Klen) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
          dst[kk] = (unsigned long long)__double_as_longlong(__ldg(arow + (k0 + kk) * a_sk));
      } else {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
          dst[kk] = (rvalid && k0 + kk < Klen)
                        ? (unsigned long long)__double_as_longlong(__ldg(arow + (k0 + kk) * a_sk))
                        : 0ull;
      }
    };
    if (nstage > 0) load(0, raw);
    for (int it = 0; it < nstage && ok; ++it) {
      const int s = it % nst, u = it / nst;
      // the window before this one is drained once the first nst stages of this one are
      // sliced (slicing further would wait on MMAs that wait on that drain)
      const bool drain_now = it == (wd + 1) * kStPerWin + nst - 1;
      // cut the 16 entries into digits below this A-row's window exponent
      const int Ex = EA[(int64_t)(w0 + it / kStPerWin) * RpA + ia_s];
      uint32_t fh[16], fl[16];
      uint32_t magic[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        magic[kk] = digit_magic(raw[kk]);
        const unsigned long long F = frac49(raw[kk], Ex);
        fh[kk] = (uint32_t)(F >> 21);
        fl[kk] = (uint32_t)F & 0x1FFFFFu;
      }
      // the next stage's loads fly while this one is written (after the drain when there
      // is one, which needs the registers)
      if (!drain_now && it + 1 < nstage) load(it + 1, raw);
      if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, err, ab)) {
        ok = false;
        break;
      }
      {
        unsigned char *pa = sm + s * sbytes + srow * 64;
        const int sw = (srow >> 1) & 3;
#pragma unroll
        for (int p = 0; p < kDigits; ++p) {
#pragma unroll
          for (int cq = 0; cq < 2; ++cq) {
            uint32_t wv[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int k1 = 8 * cq + 2 * h, k2 = k1 + 1;
              wv[h] = pack_bf16x2(digit_f32(digit_of(fh[k1], fl[k1], p), magic[k1]),
                                  digit_f32(digit_of(fh[k2], fl[k2], p), magic[k2]));
            }
            const int unit = (2 * shalf + cq) ^ sw;
            *reinterpret_cast<uint4 *>(pa + p * (128 * 64) + unit * 16) =
                make_uint4(wv[0], wv[1], wv[2], wv[3]);
          }
        }
        fence_async_smem();   // generic-proxy stores -> visible to the tensor core
        mbar_arrive(&fulla[s]);
      }
      if (drain_now) {
        if (!drain(wd)) {
          ok = false;
          break;
        }
        ++wd;
        if (it + 1 < nstage) load(it + 1, raw);
      }
    }
    for (; ok && wd < nw; ++wd)
      if (!drain(wd)) ok = false;
    if (ok && ia_d < mvalid) {
      double *o = out + blockIdx.x * so_split + (int64_t)ia_d * so_i + (int64_t)(nt * N + c0) * so_j;
#pragma unroll
      for (int j = 0; j < NH; ++j) {
        if (j < nh && nt * N + c0 + j < nvalid) {
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
          int Iw, uint16_t *P, int *E, cudaStream_t st) {
  const size_t smem = (size_t)kSlRows * (kWin + 1) * 8;
  static bool attr = false;
  if (!attr) {
    GCGE_CUDA(cudaFuncSetAttribute(oz_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = true;
  }
  dim3 grid((unsigned)(Kp / kWin), (unsigned)((Iw + kSlRows - 1) / kSlRows));
  oz_slice_kernel<<<grid, kSlThreads, smem, st>>>(src, si, sk, I, K, Rp, Kp, Iw, P, E);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

int expo(const double *src, int64_t si, int64_t sk, int I, int64_t K, int Rp, int nwin, int *E,
         cudaStream_t st) {
  dim3 grid((unsigned)nwin, (unsigned)((Rp + 255) / 256));
  oz_expo_kernel<<<grid, 256, 0, st>>>(src, si, sk, I, K, Rp, E);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

// Stages of the fused product: three when they fit in shared memory (N <= 32), else two.
int fused_stages(int N) {
  const uint32_t sbytes = ((uint32_t)kDigits * (128 + N) * 64 + 1023u) & ~1023u;
  return (size_t)kMaxStages * sbytes + 1024 <= 227u * 1024 ? kMaxStages : 2;
}

size_t fused_smem(int N) {
  const uint32_t sbytes = ((uint32_t)kDigits * (128 + N) * 64 + 1023u) & ~1023u;
  return (size_t)fused_stages(N) * sbytes + 1024;
}

int fused_launch(const CUtensorMap &mb, const double *A, int64_t a_si, int64_t a_sk, int Arows,
                 int64_t Klen, const int *EA, int RpA, const int *EB, int RpB, int N, int nwin,
                 int wps, int splits, int mtiles, int ntiles, int mvalid, int nvalid, double alpha,
                 double beta, double *out, int64_t so_i, int64_t so_j, int64_t so_split,
                 cudaStream_t st) {
  int *err = nullptr;
  GCGE_CHECK(tc::err_flag(&err));
  const size_t smem = fused_smem(N);
  static size_t attr16 = 0, attr32 = 0;
  size_t &attr = N <= 32 ? attr16 : attr32;
  if (smem > attr) {
    if (N <= 32)
      GCGE_CUDA(cudaFuncSetAttribute(oz_fused_kernel<16>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
      GCGE_CUDA(cudaFuncSetAttribute(oz_fused_kernel<kMaxN / 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  dim3 grid((unsigned)splits, (unsigned)mtiles, (unsigned)ntiles);
  if (N <= 32)
    oz_fused_kernel<16><<<grid, kFuThreads, smem, st>>>(
        mb, A, a_si, a_sk, Arows, Klen, EA, RpA, EB, RpB, N, nwin, wps, mvalid, nvalid, alpha, beta,
        out, so_i, so_j, so_split, fused_stages(N), err);
  else
    oz_fused_kernel<kMaxN / 2><<<grid, kFuThreads, smem, st>>>(
        mb, A, a_si, a_sk, Arows, Klen, EA, RpA, EB, RpB, N, nwin, wps, mvalid, nvalid, alpha, beta,
        out, so_i, so_j, so_split, fused_stages(N), err);
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
  const int mtiles = (m + 127) / 128;
  const int RpA = mtiles * 128;
  // per row of X/Y: Y's planes and the two exponent tables (one entry per window)
  const int64_t bytes_per_row = (int64_t)kDigits * 2 * RpB + (4 * (int64_t)(RpA + RpB)) / kWin + 1;
  int64_t nc = std::max<int64_t>(kWin, (int64_t)(kPlaneBudget / bytes_per_row) / kWin * kWin);
  nc = std::min(nc, round_up(n, kWin));
  const int nwc = (int)(nc / kWin);                 // windows per row chunk
  const int sm_count = device_sm_count();
  int splits = std::max(1, sm_count / std::max(1, mtiles * ntiles));
  splits = std::min(splits, nwc);
  const size_t bytes = (size_t)kDigits * RpB * nc * 2 + (size_t)nwc * RpB * 4 +
                       (size_t)nwc * RpA * 4 + (size_t)splits * m * k * 8 + 8 * 1024;
  void *wsp = nullptr;
  GCGE_CHECK(ws.get(bytes, st, &wsp));
  Carve cv{static_cast<unsigned char *>(wsp)};
  uint16_t *PB = cv.take<uint16_t>((size_t)kDigits * RpB * nc);
  int *EBt = cv.take<int>((size_t)nwc * RpB);
  int *EAt = cv.take<int>((size_t)nwc * RpA);
  double *part = cv.take<double>((size_t)splits * m * k);
  CUtensorMap mb;
  if (!plane_map(&mb, PB, RpB, nc, N)) return GCGE_EINVAL;
  for (int64_t r0 = 0; r0 < n; r0 += nc) {
    const int64_t rows = std::min(nc, n - r0);
    const int nwin = (int)((rows + kWin - 1) / kWin);
    const int wps = (nwin + splits - 1) / splits;
    // Y: rows of the B planes are the columns of Y, reduction over the rows of Y
    GCGE_CHECK(slice(Y + r0 * ldy, 1, ldy, k, rows, RpB, nc, ntiles * N, PB, EBt, st));
    // X: only the window exponents; the digits are cut inside the product
    GCGE_CHECK(expo(X + r0 * ldx, 1, ldx, m, rows, RpA, nwin, EAt, st));
    // part[split][j][i] += this chunk's share (overwritten by the first chunk)
    GCGE_CHECK(fused_launch(mb, X + r0 * ldx, 1, ldx, m, rows, EAt, RpA, EBt, RpB, N, nwin, wps,
                            splits, mtiles, ntiles, m, k, 1.0, r0 == 0 ? 0.0 : 1.0, part, 1, m,
                            (int64_t)m * k, st));
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
  // the rows of V are taken in chunks only to bound the exponent table (one int per row
  // and window); V's digits are cut inside the product
  int64_t rchunk = (int64_t)std::max<size_t>(128, kPlaneBudget / ((size_t)nwin * 4));
  // a chunk's 128-row tiles are the product's grid.y (at most 65535)
  rchunk = std::min<int64_t>(rchunk, (int64_t)65535 * 128);
  rchunk = std::min<int64_t>(round_up(n, 128), (rchunk / 128) * 128);
  const int RpA = (int)rchunk;
  const size_t bytes = (size_t)kDigits * RpB * Kp * 2 + (size_t)nwin * RpB * 4 +
                       (size_t)nwin * RpA * 4 + 8 * 1024;
  void *wsp = nullptr;
  GCGE_CHECK(ws.get(bytes, st, &wsp));
  Carve cv{static_cast<unsigned char *>(wsp)};
  uint16_t *PB = cv.take<uint16_t>((size_t)kDigits * RpB * Kp);
  int *EBt = cv.take<int>((size_t)nwin * RpB);
  int *EAt = cv.take<int>((size_t)nwin * RpA);
  // C: rows of the B planes are the columns of C, reduction over the rows of C
  GCGE_CHECK(slice(C, ldc, 1, q, d, RpB, Kp, ntiles * N, PB, EBt, st));
  CUtensorMap mb;
  if (!plane_map(&mb, PB, RpB, Kp, N)) return GCGE_EINVAL;
  for (int64_t r0 = 0; r0 < n; r0 += rchunk) {
    const int rows = (int)std::min<int64_t>(rchunk, n - r0);
    GCGE_CHECK(expo(V + r0 * ldv, ldv, 1, rows, d, RpA, nwin, EAt, st));
    GCGE_CHECK(fused_launch(mb, V + r0 * ldv, ldv, 1, rows, d, EAt, RpA, EBt, RpB, N, nwin, nwin,
                            1, (rows + 127) / 128, ntiles, rows, q, alpha, beta, Y + r0 * ldy, ldy,
                            1, 0, st));
  }
  return GCGE_OK;
}

}  // namespace gcge
