// TMA-fed tcgen05 (kind::tf32, 3-term split) Gram and V C products for FP32 blocks.
//
// Both kernels are warp-specialised:
//   warp 0      one thread issues TMA tile loads into a ring of shared-memory stages;
//   warp 1      one thread issues tcgen05.mma and commits completions to mbarriers
//               (warp 1 also owns the tensor-memory allocation);
//   warps 2-5   convert: each thread owns one TMEM lane (one row of the MMA's A
//               operand); it reads its row of the staged tile, splits each FP32
//               value x into a TF32 head hi and an exact FP32 tail lo = x - hi, and
//               writes hi and lo into tensor memory with tcgen05.st, so the A operand
//               of tcgen05.mma comes from tensor memory (no shared-memory transpose);
//   (V C only) warps 6-9 drain the accumulator (tcgen05.ld) and store the result.
// The three products hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor memory.
//
//   Gram  C(m x k) = X^T Y: A = X^T (M = 128 columns of X per tile, up to 2 tiles),
//         B = Y (N = k padded to 16, <= 128), K = rows of X and Y, 32 per chunk.
//         Y is converted into the K-major core-matrix layout in shared memory.
//         FP64 partial sums per row split, reduced by the common FP64 reduction.
//   V C   Y(n x q) = alpha V C + beta Y: A = 128 rows of V, B = C (pre-split once per
//         call into hi/lo FP32 in the shared-memory layout, fetched by bulk copy),
//         K = d in chunks of 16, accumulator double-buffered in tensor memory so the
//         store of one row tile overlaps the products of the next.
//
// A block whose base address is not 16-byte aligned is addressed through a tensor
// map starting at the aligned address below it: TMA x coordinates stay multiples of
// 16 bytes and the converters index past the leading offset.  Leading dimensions must
// be multiples of 4 (16-byte rows); other shapes use the staged kernels of tc.cu.
//
// Every mbarrier wait is bounded (global timer); a timeout sets the device error flag
// and a shared abort flag so the other roles stop waiting, the MMA issuer waits
// (bounded) for its issued MMAs, the TMA issuer for its issued copies, tensor memory is
// freed, and the kernel returns.
#include <algorithm>

#include "blas.cuh"
#include "tcgen05.cuh"

namespace gcge {

int gram_reduce_launch(int m, int k, int splits, const double *part, double alpha, double beta,
                       double *C, int64_t ldc, cudaStream_t st);

namespace {
using namespace tc;

// ------------------------------------------------------------------------- Gram
constexpr int kGRows = 32;      // K rows per chunk (4 MMA k-steps of 8)
constexpr int kGXBox = 132;     // X box: 128 columns + up to 3 leading, 16-byte multiple
constexpr int kGThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 convert + epilogue
constexpr int kGConv = 256;     // converter threads
// FP32 accumulation window: the tensor memory accumulator is drained into the FP64
// partial sums every 16 chunks (512 rows; 32 chunks when Y is wider than 32 columns),
// so rounding in the FP32 accumulator stays at the level of a 512- or 1024-term sum
// however many rows one CTA covers.
constexpr int kMaxStages = 8;   // shared-memory stages (runtime count <= this)
constexpr int kMaxA = 4;        // tensor-memory A-operand stages (runtime count <= this)
constexpr uint32_t kSmemBudget = 224 * 1024;   // + alignment slack + static

struct GramSmem {
  uint32_t xraw, yraw, stage, braw, bstage, total;
  int nS, nA, abase;
};

// Tensor memory per M tile: D1 (2 Np columns: X_hi^T [Y_hi | Y_lo]) and D2 (Np columns:
// X_lo^T Y_hi); then nA A-operand stages of MT x 64 columns (32 hi + 32 lo).
// cps = CTAs per SM (1 or 2): each gets 512 / cps TMEM columns and about 1 / cps of the
// shared memory.
__host__ __device__ inline GramSmem gram_smem(int MT, int Np, int bk, int cps) {
  GramSmem L;
  const int tcols = 512 / cps;
  const uint32_t budget = cps == 1 ? kSmemBudget : 110 * 1024;
  L.xraw = 0;
  L.yraw = (uint32_t)MT * kGXBox * kGRows * 4;
  L.stage = (L.yraw + (uint32_t)bk * kGRows * 4 + 1023u) & ~1023u;
  L.abase = ((MT * 3 * Np + 31) / 32) * 32;
  L.nA = (tcols - L.abase) / (MT * 64);
  if (L.nA > kMaxA) L.nA = kMaxA;
  L.bstage = ((uint32_t)2 * Np * kGRows * 4 + 1023u) & ~1023u;   // [Y_hi; Y_lo], 2 Np rows
  int nS = (int)((budget - L.nA * L.bstage) / L.stage);
  L.nS = nS > kMaxStages ? kMaxStages : nS;
  L.braw = L.nS * L.stage;
  L.total = L.braw + L.nA * L.bstage;
  return L;
}


__global__ void __launch_bounds__(kGThreads, 1)
gram_tma_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                int64_t n, int m, int k, int ax, int ay, int MT, int Np, int bk, int cps,
                int64_t rps, double *__restrict__ part, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], afull[kMaxA],
      aempty[kMaxA], dfull, dflush, dread;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const GramSmem L = gram_smem(MT, Np, bk, cps);
  const int nS = L.nS, nA = L.nA, abase = L.abase;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * 128 * MT;
  const int MTg = min(MT, (m - i0 + 127) / 128);
  const int j0 = blockIdx.z * 128;
  const int kw = min(128, k - j0);
  const int64_t r0 = (int64_t)blockIdx.x * rps;
  const int64_t r1 = min(n, r0 + rps);
  const int nch = (int)((r1 - r0 + kGRows - 1) / kGRows);
  const int win = Np <= 32 ? 16 : 32;   // chunks per FP32 accumulation window
  const uint32_t ncols = 512 / cps;
  const uint32_t xbytes = kGXBox * kGRows * 4, ybytes = (uint32_t)bk * kGRows * 4;

  if (warp == 1) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kGConv);
    }
    for (int s = 0; s < nA; ++s) {
      mbar_init(&afull[s], kGConv);
      mbar_init(&aempty[s], 1);
    }
    mbar_init(&dfull, 1);
    mbar_init(&dflush, 1);
    mbar_init(&dread, kGConv);
    abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  volatile int *ab = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {   // TMA issuer
      int issued = 0;
      for (int c = 0; c < nch; ++c) {
        const int s = c % nS, u = c / nS;
        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1, err, ab)) break;
        mbar_expect_tx(&full[s], MTg * xbytes + ybytes);
        const int y = (int)(r0 + (int64_t)c * kGRows);
        for (int t = 0; t < MTg; ++t)
          tma_load_2d(sm + s * L.stage + L.xraw + t * xbytes, &tmX, i0 + 128 * t, y, &full[s]);
        tma_load_2d(sm + s * L.stage + L.yraw, &tmY, j0, y, &full[s]);
        ++issued;
      }
      // copies still in flight must land before the CTA exits
      for (int c = max(0, issued - nS); c < issued; ++c)
        mbar_wait(&full[c % nS], (c / nS) & 1, err, nullptr);
    }
  } else if (warp == 1) {
    // MMA issuer: the whole warp runs the loop (uniform operands), one elected lane issues
    const bool leader = elect_one();
    const uint32_t id2 = idesc_tf32(128, 2 * Np), id1 = idesc_tf32(128, Np);
    for (int c = 0; c < nch; ++c) {
      const int ts = c % nA, v = c / nA;
      const int cw = c % win, wi = c / win;
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&afull[ts], v & 1, err, ab))) break;
      // a new window overwrites the accumulator: the previous one must have been read
      if (cw == 0 && wi > 0 &&
          !__all_sync(0xFFFFFFFFu, mbar_wait(&dread, (wi - 1) & 1, err, ab)))
        break;
      tc_fence_after();
      const uint32_t bb = su32(sm + L.braw + ts * L.bstage);
#pragma unroll
      for (int ks = 0; ks < kGRows / 8; ++ks) {
        const uint64_t bd = smem_desc(bb + ks * (2 * Np / 8) * 256, 128, 256);
        for (int t = 0; t < MTg; ++t) {
          const uint32_t ah = tmem + abase + (ts * MT + t) * 64 + ks * 8, al = ah + 32;
          const uint32_t d1 = tmem + t * 3 * Np, d2 = d1 + 2 * Np;
          const uint32_t acc = (cw > 0 || ks > 0) ? 1u : 0u;
          if (leader) {
            mma_ts(d1, ah, bd, id2, acc);   // X_hi^T [Y_hi | Y_lo]
            mma_ts(d2, al, bd, id1, acc);   // X_lo^T Y_hi (first Np rows of B)
          }
        }
      }
      __syncwarp();
      if (leader) {
        mma_commit(&aempty[ts]);
        if (cw == win - 1 || c == nch - 1) mma_commit(&dflush);
      }
      __syncwarp();
    }
    if (leader) {
      mma_commit(&dfull);
      mbar_wait(&dfull, 0, err, nullptr);   // issued MMAs are done before TMEM is freed
    }
    __syncwarp();
  } else {
    // converters / epilogue: warps 2-9; thread = TMEM lane 32 q + lane, row half hs
    const int q = warp & 3, hs = (warp - 2) >> 2;
    const int ct = threadIdx.x - 64;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
      const int s = c % nS, u = c / nS, ts = c % nA, v = c / nA;
      if (!mbar_wait(&full[s], u & 1, err, ab)) { ok = false; break; }
      if (v > 0 && !mbar_wait(&aempty[ts], (v - 1) & 1, err, ab)) { ok = false; break; }
      tc_fence_after();
      const unsigned char *st = sm + s * L.stage;
      for (int t = 0; t < MTg; ++t) {
        const float *col = reinterpret_cast<const float *>(st + L.xraw + t * xbytes) + ax +
                           32 * q + lane + hs * 16 * kGXBox;
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          float h, l;
          split_tf32(col[kk * kGXBox], h, l);
          hi[kk] = __float_as_uint(h);
          lo[kk] = __float_as_uint(l);
        }
        const uint32_t a = tmem + lane_addr + abase + (ts * MT + t) * 64 + hs * 16;
        tmem_st16(a, hi);
        tmem_st16(a + 32, lo);
      }
      // Y rows of this chunk into the K-major B operand [Y_hi; Y_lo] (2 Np rows)
      const float *yr = reinterpret_cast<const float *>(st + L.yraw) + ay;
      unsigned char *bhb = sm + L.braw + ts * L.bstage;
      const int e = lane & 3, j7 = lane >> 2;
      const int items = 8 * (Np / 8);
      for (int it = ct >> 5; it < items; it += kGConv / 32) {
        const int kq = it & 7, jg = it >> 3;
        const int kk = 4 * kq + e, j = 8 * jg + j7;
        const float y = j < kw ? yr[kk * bk + j] : 0.f;
        float h, l;
        split_tf32(y, h, l);
        *reinterpret_cast<float *>(bhb + kmaj_off(j, kk, 2 * Np)) = h;
        *reinterpret_cast<float *>(bhb + kmaj_off(Np + j, kk, 2 * Np)) = l;
      }
      mbar_arrive(&empty[s]);
      tmem_st_wait();
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(&afull[ts]);
      if ((c % win) == win - 1 || c == nch - 1) {
        // drain this window's accumulator: this thread's row of every M tile, its half of
        // the columns (at most 8 groups of 8), then add into the FP64 partial sums
        const int wi = c / win;
        if (!mbar_wait(&dflush, wi & 1, err, ab)) { ok = false; break; }
        tc_fence_after();
        float acc[8][8];
        int slot = 0;
        for (int t = 0; t < MTg; ++t) {
          const uint32_t d1 = tmem + lane_addr + t * 3 * Np;
          for (int jb = hs * 8; jb < Np && slot < 8; jb += 16, ++slot) {
            float a1[8], a2[8], a3[8];
            tmem_ld8(d1 + jb, a1);
            tmem_ld8(d1 + Np + jb, a2);
            tmem_ld8(d1 + 2 * Np + jb, a3);
#pragma unroll
            for (int uu = 0; uu < 8; ++uu) acc[slot][uu] = a1[uu] + a2[uu] + a3[uu];
          }
        }
        tc_fence_before();
        mbar_arrive(&dread);
        double *pp = part + (int64_t)blockIdx.x * m * k;
        slot = 0;
        for (int t = 0; t < MTg; ++t) {
          const int i = i0 + 128 * t + 32 * q + lane;
          for (int jb = hs * 8; jb < Np && slot < 8; jb += 16, ++slot) {
#pragma unroll
            for (int uu = 0; uu < 8; ++uu) {
              const int j = jb + uu;
              if (i < m && j < kw) {
                double *pj = pp + (int64_t)(j0 + j) * m + i;
                *pj = (wi == 0 ? 0.0 : *pj) + (double)acc[slot][uu];
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------- V C
constexpr int kVK = 16;         // K (columns of V) per chunk: 2 MMA k-steps
constexpr int kVThreads = 320;  // warp 0 TMA, 1 MMA, 2-5 split, 6-9 epilogue
constexpr int kVMaxNb = 256;

// Stage: V tile (128 rows x 64 B, 64-byte swizzle; split in place to its TF32 head),
// its FP32 tail in the same layout, then C's [hi | lo] operand (K-major, Nb x 16 each).
struct VcSmem {
  uint32_t vhi, vlo, braw, stage, epi, total;
  int nS, nbal, nacc;
};

__host__ __device__ inline VcSmem vc_smem(int Nb) {
  VcSmem L;
  L.vhi = 0;
  L.vlo = 128 * kVK * 4;
  L.braw = 2 * 128 * kVK * 4;
  L.stage = (L.braw + (uint32_t)Nb * kVK * 4 * 2 + 1023u) & ~1023u;
  const uint32_t epi_bytes = 4 * 32 * 33 * 4;   // 4 warps x 32 x 33 floats
  int nS = (int)((kSmemBudget - epi_bytes) / L.stage);
  L.nS = nS > kMaxStages ? kMaxStages : nS;
  L.epi = L.nS * L.stage;
  L.total = L.epi + epi_bytes;
  L.nbal = ((Nb + 31) / 32) * 32;
  // two accumulator buffers (the store of one row tile overlaps the next); each holds
  // D1 = hi hi and D2 = the cross terms when they fit, else one accumulator for all three
  L.nacc = 4 * L.nbal <= 512 ? 2 : 1;
  return L;
}

// C (d x q col-major FP64) -> per q-group and K chunk: [hi | lo] FP32 in the K-major
// core-matrix layout of an Nb x 16 operand; K row kk of chunk c is V column
// 16 c + kk - av (zero outside [0, d)), operand row j is column q0 + j (zero past q).
__global__ void vc_split_c_kernel(int d, int q, const double *__restrict__ C, int64_t ldc, int av,
                                  int Nb, int nqg, int nch, float *__restrict__ Bs) {
  const int64_t per = (int64_t)Nb * kVK;
  const int64_t total = (int64_t)nqg * nch * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(t % kVK);
    const int j = (int)((t / kVK) % Nb);
    const int64_t blk = t / per;   // qg * nch + c
    const int c = (int)(blk % nch), qg = (int)(blk / nch);
    const int kcol = c * kVK + kk - av, col = qg * Nb + j;
    const float x = (kcol >= 0 && kcol < d && col < q) ? (float)C[kcol + (int64_t)col * ldc] : 0.f;
    float hi, lo;
    split_tf32(x, hi, lo);
    float *base = Bs + blk * 2 * per;
    const uint32_t off = kmaj_off(j, kk, Nb) / 4;
    base[off] = hi;
    base[per + off] = lo;
  }
}

__global__ void __launch_bounds__(kVThreads, 1)
vc_tma_kernel(const __grid_constant__ CUtensorMap tmV, const float *__restrict__ Bs, int64_t n,
              int d, int q, int Nb, int av, int nch, float alpha, float beta,
              float *__restrict__ Yo, int64_t ldy, int *__restrict__ err) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kMaxStages], afull[kMaxStages], empty[kMaxStages],
      dfull[2], dempty[2], fin;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const VcSmem L = vc_smem(Nb);
  const int nS = L.nS, nbal = L.nbal, nacc = L.nacc, nbuf = 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qg = blockIdx.y, q0 = qg * Nb, qn = min(Nb, q - q0);
  const int64_t ntiles = (n + 127) / 128;
  const uint32_t ncols = 512;
  const uint32_t bbytes = (uint32_t)Nb * kVK * 4 * 2;
  const uint32_t vbytes = 128 * kVK * 4;

  if (warp == 1) tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&afull[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&dfull[s], 1);
      mbar_init(&dempty[s], 128);
    }
    mbar_init(&fin, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  volatile int *ab = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {   // TMA issuer
      int64_t issued = 0;
      bool ok = true;
      int it = 0;
      for (int64_t tl = blockIdx.x; tl < ntiles && ok; tl += gridDim.x, ++it) {
        for (int c = 0; c < nch; ++c) {
          const int64_t gc = (int64_t)it * nch + c;
          const int s = (int)(gc % nS);
          const int64_t u = gc / nS;
          if (u > 0 && !mbar_wait(&empty[s], (unsigned)((u - 1) & 1), err, ab)) { ok = false; break; }
          mbar_expect_tx(&full[s], vbytes + bbytes);
          unsigned char *st = sm + s * L.stage;
          tma_load_2d(st + L.vhi, &tmV, c * kVK, (int)(tl * 128), &full[s]);
          bulk_load(st + L.braw, Bs + ((int64_t)qg * nch + c) * 2 * Nb * kVK, bbytes, &full[s]);
          ++issued;
        }
      }
      for (int64_t gc = issued > nS ? issued - nS : 0; gc < issued; ++gc)
        mbar_wait(&full[gc % nS], (unsigned)((gc / nS) & 1), err, nullptr);
    }
  } else if (warp == 1) {
    // MMA issuer: the whole warp runs the loop (uniform operands), one elected lane issues
    const bool leader = elect_one();
    const uint32_t idesc = idesc_tf32(128, Nb);
    int it = 0;
    bool ok = true;
    for (int64_t tl = blockIdx.x; tl < ntiles && ok; tl += gridDim.x, ++it) {
      const int db = it % nbuf, w = it / nbuf;
      if (w > 0 && !__all_sync(0xFFFFFFFFu, mbar_wait(&dempty[db], (w - 1) & 1, err, ab))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d1 = tmem + db * nacc * nbal, d2 = d1 + (nacc - 1) * nbal;
      for (int c = 0; c < nch; ++c) {
        const int64_t gc = (int64_t)it * nch + c;
        const int s = (int)(gc % nS);
        const unsigned u = (unsigned)((gc / nS) & 1);
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(&afull[s], u, err, ab))) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = su32(sm + s * L.stage);
#pragma unroll
        for (int ks = 0; ks < kVK / 8; ++ks) {
          const uint64_t ah = smem_desc_sw64(st + L.vhi + ks * 32);
          const uint64_t al = smem_desc_sw64(st + L.vlo + ks * 32);
          const uint64_t bh = smem_desc(st + L.braw + ks * (Nb / 8) * 256, 128, 256);
          const uint64_t bl = smem_desc(st + L.braw + Nb * kVK * 4 + ks * (Nb / 8) * 256, 128, 256);
          const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
          if (leader) {
            mma_ss(d1, ah, bh, idesc, acc);   // hi hi
            mma_ss(d2, ah, bl, idesc, nacc == 2 ? acc : 1u);   // hi lo
            mma_ss(d2, al, bh, idesc, 1u);    // lo hi
          }
        }
        __syncwarp();
        if (leader) mma_commit(&empty[s]);
        __syncwarp();
      }
      if (ok && leader) mma_commit(&dfull[db]);
      __syncwarp();
    }
    // all issued MMAs complete before tensor memory is released
    if (leader) {
      mma_commit(&fin);
      mbar_wait(&fin, 0, err, nullptr);
    }
    __syncwarp();
  } else if (warp < 6) {
    // split: V tile -> TF32 head (in place) and FP32 tail, same swizzled layout
    const int ct = threadIdx.x - 64;
    bool ok = true;
    int it = 0;
    for (int64_t tl = blockIdx.x; tl < ntiles && ok; tl += gridDim.x, ++it) {
      for (int c = 0; c < nch; ++c) {
        const int64_t gc = (int64_t)it * nch + c;
        const int s = (int)(gc % nS);
        const int64_t u = gc / nS;
        if (!mbar_wait(&full[s], (unsigned)(u & 1), err, ab)) { ok = false; break; }
        unsigned char *st = sm + s * L.stage;
        float4 *vh = reinterpret_cast<float4 *>(st + L.vhi);
        float4 *vl = reinterpret_cast<float4 *>(st + L.vlo);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int idx = ct + 128 * f;            // 16-byte unit: row idx / 4, slot idx % 4
          const int r = idx >> 2, c4 = (idx & 3) ^ ((r >> 1) & 3);
          float4 x = vh[idx];
          float xv[4] = {x.x, x.y, x.z, x.w}, hv[4], lv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float val = (c * kVK + 4 * c4 + e - av) >= 0 ? xv[e] : 0.f;
            split_tf32(val, hv[e], lv[e]);
          }
          vh[idx] = make_float4(hv[0], hv[1], hv[2], hv[3]);
          vl[idx] = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
        fence_async_smem();
        mbar_arrive(&afull[s]);
      }
    }
  } else {
    // epilogue: drain [D1 + D2] of one row tile (overlapping the next when double-buffered)
    const int qq = warp & 3;
    const uint32_t lane_addr = (uint32_t)(32 * qq) << 16;
    float *stg = reinterpret_cast<float *>(sm + L.epi) + (warp - 6) * 32 * 33;
    int it = 0;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, ++it) {
      const int db = it % nbuf, w = it / nbuf;
      if (!mbar_wait(&dfull[db], w & 1, err, ab)) break;
      tc_fence_after();
      const uint32_t d1 = tmem + lane_addr + db * nacc * nbal, d2 = d1 + nbal;
      const int64_t row0 = tl * 128 + 32 * qq;
      for (int jb = 0; jb < qn; jb += 32) {
        for (int h = 0; h < 2; ++h) {
          if (jb + 16 * h < Nb) {
            float v1[16], v2[16];
            tmem_ld16(d1 + jb + 16 * h, v1);
            if (nacc == 2) {
              tmem_ld16(d2 + jb + 16 * h, v2);
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) v1[jj] += v2[jj];
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) stg[lane * 33 + 16 * h + jj] = v1[jj];
          }
        }
        __syncwarp();
        const int j = jb + lane;
        for (int rr = 0; rr < 32; ++rr) {
          const int64_t rowg = row0 + rr;
          if (rowg < n && j < qn) {
            float *yp = Yo + rowg * ldy + q0 + j;
            float out = alpha * stg[rr * 33 + lane];
            if (beta != 0.f) out += beta * *yp;
            *yp = out;
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      mbar_arrive(&dempty[db]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

// Tensor map of a row-major FP32 block (rows x cols, ld elements per row) whose first
// element may sit `*shift` elements past a 16-byte boundary: the map starts at that
// boundary and spans cols + shift columns.  false when TMA cannot address the block.
bool fp32_block_map(CUtensorMap *map, const float *p, int64_t rows, int64_t cols, int64_t ld,
                    int box_x, int box_y, CUtensorMapSwizzle swz, int *shift) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (ld % 4) != 0 || rows <= 0 || cols <= 0) return false;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if (a % 4) return false;
  const int sh = (int)((a & 15u) / 4);
  const cuuint64_t dims[2] = {(cuuint64_t)(cols + sh), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(a - 4u * sh), dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  *shift = sh;
  return r == CUDA_SUCCESS;
}

int occupancy(const void *kernel, int threads, size_t smem) {
  static const void *ck[8] = {};
  static size_t cs[8] = {};
  static int co[8] = {};
  static int dev[8] = {};
  int cur = 0;
  cudaGetDevice(&cur);
  for (int i = 0; i < 8; ++i)
    if (ck[i] == kernel && cs[i] == smem && dev[i] == cur) return co[i];
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  occ = std::max(occ, 1);
  static int next = 0;
  ck[next] = kernel;
  cs[next] = smem;
  co[next] = occ;
  dev[next] = cur;
  next = (next + 1) % 8;
  return occ;
}

}  // namespace

// GCGE_EINVAL: shape or alignment outside what the TMA kernels take (caller falls back).
int gram_tma(int64_t n, int m, int k, double alpha, const float *X, int64_t ldx, const float *Y,
             int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st) {
  if (n <= 0 || m <= 0 || k <= 0 || n > INT32_MAX - 64) return GCGE_EINVAL;
  const int kmax = std::min(k, 128);
  const int Np = ((kmax + 15) / 16) * 16;
  // two 128-column tiles of X per CTA when the accumulators leave room for two A stages
  const int MT = (Np <= 32 && m > 128) ? 2 : 1;
  const int cps = 1;
  CUtensorMap mx, my;
  int ax = 0, ay = 0;
  if (!fp32_block_map(&mx, X, n, m, ldx, kGXBox, kGRows, CU_TENSOR_MAP_SWIZZLE_NONE, &ax))
    return GCGE_EINVAL;
  const int bk0 = ((kmax + 3 + 3) / 4) * 4;   // room for any leading shift of Y
  if (!fp32_block_map(&my, Y, n, k, ldy, bk0, kGRows, CU_TENSOR_MAP_SWIZZLE_NONE, &ay))
    return GCGE_EINVAL;
  const int bk = bk0;
  int *err = nullptr;
  GCGE_CHECK(tc::err_flag(&err));
  const GramSmem L = gram_smem(MT, Np, bk, cps);
  if (L.nS < 2 || L.nA < 2) return GCGE_EINVAL;
  const size_t smem = tmem_limited_smem((size_t)L.total + 1024, 512 / cps);
  if (smem > 227 * 1024) return GCGE_EINVAL;
  static size_t attr = 0;
  if (smem > attr) {
    GCGE_CUDA(cudaFuncSetAttribute(gram_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = smem;
  }
  const int mg = (m + 128 * MT - 1) / (128 * MT), kg = (k + 127) / 128;
  const int occ = occupancy((const void *)gram_tma_kernel, kGThreads, smem);
  int64_t splits = std::max<int64_t>(1, (int64_t)occ * device_sm_count() / (mg * kg));
  int64_t rps = round_up((n + splits - 1) / splits, kGRows);
  splits = (n + rps - 1) / rps;
  if (splits > 65535) return GCGE_EINVAL;
  double *part = nullptr;
  GCGE_CHECK(ws.get(sizeof(double) * (size_t)splits * m * k, st, (void **)&part));
  dim3 grid((unsigned)splits, (unsigned)mg, (unsigned)kg);
  gram_tma_kernel<<<grid, kGThreads, smem, st>>>(mx, my, n, m, k, ax, ay, MT, Np, bk, cps, rps,
                                                 part, err);
  GCGE_LAUNCH_CHECK();
  return gram_reduce_launch(m, k, (int)splits, part, alpha, beta, C, ldc, st);
}

int vc_tma(int64_t n, int d, int q, double alpha, const float *V, int64_t ldv, const double *C,
           int64_t ldc, double beta, float *Y, int64_t ldy, Scratch &ws, cudaStream_t st) {
  if (n <= 0 || d <= 0 || q <= 0 || n > INT32_MAX - 256) return GCGE_EINVAL;
  CUtensorMap mv;
  int av = 0;
  if (!fp32_block_map(&mv, V, n, d, ldv, kVK, 128, CU_TENSOR_MAP_SWIZZLE_64B, &av))
    return GCGE_EINVAL;
  const int nqg = (q + kVMaxNb - 1) / kVMaxNb;
  const int Nb = (((q + nqg - 1) / nqg + 15) / 16) * 16;
  const int nch = (d + av + kVK - 1) / kVK;
  int *err = nullptr;
  GCGE_CHECK(tc::err_flag(&err));
  // C split once per call: nqg x nch blocks of [hi | lo] (Nb x 16 FP32 each)
  const size_t bs_floats = (size_t)nqg * nch * 2 * Nb * kVK;
  float *Bs = nullptr;
  GCGE_CHECK(ws.get(sizeof(float) * bs_floats, st, (void **)&Bs));
  {
    const int64_t total = (int64_t)nqg * nch * Nb * kVK;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 4 * device_sm_count());
    vc_split_c_kernel<<<grid, 256, 0, st>>>(d, q, C, ldc, av, Nb, nqg, nch, Bs);
    GCGE_LAUNCH_CHECK();
  }
  const VcSmem L = vc_smem(Nb);
  if (L.nS < 2) return GCGE_EINVAL;
  const size_t smem = tmem_limited_smem((size_t)L.total + 1024, 512);
  if (smem > 227 * 1024) return GCGE_EINVAL;
  static size_t attr = 0;
  if (smem > attr) {
    GCGE_CUDA(cudaFuncSetAttribute(vc_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr = smem;
  }
  const int64_t ntiles = (n + 127) / 128;
  const int occ = occupancy((const void *)vc_tma_kernel, kVThreads, smem);
  const int64_t gx = std::max<int64_t>(
      1, std::min<int64_t>(ntiles, (int64_t)occ * device_sm_count() / nqg));
  dim3 grid((unsigned)gx, (unsigned)nqg);
  vc_tma_kernel<<<grid, kVThreads, smem, st>>>(mv, Bs, n, d, q, Nb, av, nch, (float)alpha,
                                              (float)beta, Y, ldy, err);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

}  // namespace gcge
