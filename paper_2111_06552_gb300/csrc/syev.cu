// Parallel cyclic Jacobi for the dense symmetric Rayleigh-Ritz matrix (FP64).
//
// The paper solves the small problem of STEP 3 with LAPACK's dsyevx on the CPU
// (Section 3.2) and splits it over MPI processes.  Here it runs on the GPU in
// FP64 as two-sided Jacobi with the round-robin ("circle") ordering: in every
// round the d indices form d/2 disjoint pairs, so the d/2 rotations of a round
// commute and are applied together, A <- J^T A J and V <- V J.  A sweep is d-1
// rounds and visits every pair once.  One round is two phases separated by a
// grid barrier: (A) each pair's rotation from a_pp, a_qq, a_pq (Rutishauser's
// stable formulas); (B) every 2x2 block (row pair, column pair) of A and every
// (row, pair) of V is updated by exactly one thread, in place.  Sweeps stop when
// a whole sweep finds every |a_pq| <= 1e-15 sqrt(|a_pp a_qq|) (or below an
// absolute floor), which gives eigenvalues to high relative accuracy for the
// definite matrices met here.
//
// The whole solve is ONE cooperative launch (all CTAs co-resident).  The grid
// barrier is a counter/generation pair in global memory; every wait is bounded
// and a timeout sets a flag, after which all CTAs leave and the host reports
// GCGE_ETIMEOUT.  Odd d is padded with a dummy index that never rotates.
#include "syev.cuh"

namespace gcge {

namespace {

constexpr int kSyevThreads = 256;
constexpr long long kSpinLimit = 1ll << 24;   // ~ seconds with the back-off below

__device__ __forceinline__ bool grid_barrier(unsigned *sync, int *flags, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = sync + 1;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(sync, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(sync, 0u);
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > kSpinLimit || *((volatile int *)flags) != 0) {
          atomicExch(flags, 1);
          break;
        }
        if (spins > 64) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int *)flags) == 0;
}

// Pair k of round r for D (even) indices: the circle method with D-1 fixed.
__device__ __forceinline__ void round_pair(int D, int r, int k, int &p, int &q) {
  const int m = D - 1;
  int a, b;
  if (k == 0) {
    a = m;
    b = r;
  } else {
    a = (r + k) % m;
    b = (r - k + m) % m;
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// One grid barrier per round: every CTA derives the round's d/2 rotations itself
// (into shared memory) from the diagonal and pair entries, then the grid updates the
// 2x2 blocks of A and the rows of V.  Entries written by other CTAs are read with
// L1-bypassing loads (__ldcg) after the barrier.
constexpr int kMaxPairs = 512;   // d <= 1024

__global__ void __launch_bounds__(kSyevThreads)
jacobi_kernel(int d, int D, double *__restrict__ A, int64_t lda, double *__restrict__ V,
              int64_t ldv, double *__restrict__ rot_unused, unsigned *__restrict__ sync,
              int *__restrict__ flags, int max_sweeps) {
  (void)rot_unused;
  __shared__ double rot[kMaxPairs][3];
  __shared__ int local_cnt;
  const int P = D / 2;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const unsigned nb = gridDim.x;
  for (int64_t u = gt; u < (int64_t)d * d; u += gs) {
    const int i = (int)(u % d), j = (int)(u / d);
    __stcg(V + i + (int64_t)j * ldv, (i == j) ? 1.0 : 0.0);
  }
  if (gt == 0) {
    sync[2] = 0;
    sync[3] = 0;
    sync[4] = 0;
  }
  if (!grid_barrier(sync, flags, nb)) return;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    unsigned *cnt = sync + 2 + (sweep % 3);
    if (gt == 0) sync[2 + ((sweep + 1) % 3)] = 0;
    if (threadIdx.x == 0) local_cnt = 0;
    __syncthreads();
    for (int r = 0; r < D - 1; ++r) {
      // rotations of this round (identical in every CTA)
      for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int p, q;
        round_pair(D, r, k, p, q);
        double c = 1.0, s = 0.0, t = 0.0;
        if (q < d) {
          const double app = __ldcg(A + p + (int64_t)p * lda), aqq = __ldcg(A + q + (int64_t)q * lda);
          const double apq = __ldcg(A + p + (int64_t)q * lda);
          if (apq != apq || app != app || aqq != aqq) flags[1] = 1;
          const double thr = 1e-15 * sqrt(fabs(app) * fabs(aqq));
          if (fabs(apq) > thr && fabs(apq) > 1e-300) {
            const double th = (aqq - app) / (2.0 * apq);
            t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            c = rsqrt(1.0 + t * t);
            s = t * c;
            if (blockIdx.x == 0) atomicAdd(&local_cnt, 1);
          }
        }
        rot[k][0] = c;
        rot[k][1] = s;
        rot[k][2] = t;
      }
      __syncthreads();
      const int64_t nblk = (int64_t)P * P;
      for (int64_t u = gt; u < nblk + (int64_t)d * P; u += gs) {
        if (u < nblk) {
          const int kr = (int)(u % P), kc = (int)(u / P);
          const double s1 = rot[kr][1], s2 = rot[kc][1];
          if (s1 == 0.0 && s2 == 0.0) continue;
          int pr, qr, pc, qc;
          round_pair(D, r, kr, pr, qr);
          round_pair(D, r, kc, pc, qc);
          if (kr == kc) {   // diagonal block of an active rotation: exact update
            const double t = rot[kr][2];
            const double apq = __ldcg(A + pr + (int64_t)qr * lda);
            __stcg(A + pr + (int64_t)pr * lda, __ldcg(A + pr + (int64_t)pr * lda) - t * apq);
            __stcg(A + qr + (int64_t)qr * lda, __ldcg(A + qr + (int64_t)qr * lda) + t * apq);
            __stcg(A + pr + (int64_t)qr * lda, 0.0);
            __stcg(A + qr + (int64_t)pr * lda, 0.0);
            continue;
          }
          const double c1 = rot[kr][0], c2 = rot[kc][0];
          const bool vqr = qr < d, vqc = qc < d;
          double *ap = A + pr + (int64_t)pc * lda;
          const double a = __ldcg(ap);
          const double b = vqc ? __ldcg(A + pr + (int64_t)qc * lda) : 0.0;
          const double e = vqr ? __ldcg(A + qr + (int64_t)pc * lda) : 0.0;
          const double f = (vqr && vqc) ? __ldcg(A + qr + (int64_t)qc * lda) : 0.0;
          const double a1 = c1 * a - s1 * e, b1 = c1 * b - s1 * f;
          const double e1 = s1 * a + c1 * e, f1 = s1 * b + c1 * f;
          __stcg(ap, c2 * a1 - s2 * b1);
          if (vqc) __stcg(A + pr + (int64_t)qc * lda, s2 * a1 + c2 * b1);
          if (vqr) __stcg(A + qr + (int64_t)pc * lda, c2 * e1 - s2 * f1);
          if (vqr && vqc) __stcg(A + qr + (int64_t)qc * lda, s2 * e1 + c2 * f1);
        } else {
          const int64_t v = u - nblk;
          const int k = (int)(v % P), i = (int)(v / P);
          const double s = rot[k][1];
          if (s == 0.0) continue;
          const double c = rot[k][0];
          int p, q;
          round_pair(D, r, k, p, q);
          double *vp = V + i + (int64_t)p * ldv;
          double *vq = V + i + (int64_t)q * ldv;
          const double x = __ldcg(vp), y = __ldcg(vq);
          __stcg(vp, c * x - s * y);
          __stcg(vq, s * x + c * y);
        }
      }
      if (r == D - 2 && blockIdx.x == 0 && threadIdx.x == 0 && local_cnt) atomicAdd(cnt, 1u);
      if (!grid_barrier(sync, flags, nb)) return;
    }
    const unsigned done = *((volatile unsigned *)cnt);
    if (done == 0) {
      ++sweep;
      break;
    }
  }
  if (gt == 0) flags[2] = sweep;
}

// Small matrices (d <= kSmallD): the whole Jacobi in one CTA with A and V in shared
// memory and __syncthreads() between the two phases of a round.  R is the arithmetic:
// FP64, or FP32 for matrices formed from FP32 data (the Algorithm 3 leaves of the FP32
// phase, whose drop and repeat tests are at FP32 level): on GB300 a round of FP64
// rotations waits on the FP64 units of one SM (two lanes per clock).
constexpr int kSmallD = 32;

template <typename R>
__global__ void __launch_bounds__(256)
jacobi_small_kernel(int d, int D, double *__restrict__ A, int64_t lda, double *__restrict__ Vout,
                    int64_t ldv, int *__restrict__ flags, int max_sweeps) {
  constexpr R kRel = sizeof(R) == 8 ? R(1e-15) : R(1e-6);     // rotation threshold
  constexpr R kTiny = sizeof(R) == 8 ? R(1e-300) : R(1e-30);
  __shared__ R sA[kSmallD][kSmallD + 1];
  __shared__ R sV[kSmallD][kSmallD + 1];
  __shared__ R rot[kSmallD / 2][3];
  __shared__ int cnt;
  const int P = D / 2;
  for (int u = threadIdx.x; u < d * d; u += blockDim.x) {
    const int i = u % d, j = u / d;
    sA[i][j] = (R)A[i + (int64_t)j * lda];
    sV[i][j] = (i == j) ? R(1) : R(0);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int r = 0; r < D - 1; ++r) {
      for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int p, q;
        round_pair(D, r, k, p, q);
        R c = R(1), s = R(0), t = R(0);
        if (q < d) {
          const R app = sA[p][p], aqq = sA[q][q], apq = sA[p][q];
          if (apq != apq || app != app || aqq != aqq) flags[1] = 1;
          const R thr = kRel * sqrt(fabs(app) * fabs(aqq));
          if (fabs(apq) > thr && fabs(apq) > kTiny) {
            const R th = (aqq - app) / (R(2) * apq);
            t = (th >= R(0) ? R(1) : R(-1)) / (fabs(th) + sqrt(R(1) + th * th));
            c = R(1) / sqrt(R(1) + t * t);
            s = t * c;
            atomicAdd(&cnt, 1);
          }
        }
        rot[k][0] = c;
        rot[k][1] = s;
        rot[k][2] = t;
      }
      __syncthreads();
      const int nblk = P * P;
      for (int u = threadIdx.x; u < nblk + d * P; u += blockDim.x) {
        if (u < nblk) {
          const int kr = u % P, kc = u / P;
          const R s1 = rot[kr][1], s2 = rot[kc][1];
          if (s1 == R(0) && s2 == R(0)) continue;
          int pr, qr, pc, qc;
          round_pair(D, r, kr, pr, qr);
          round_pair(D, r, kc, pc, qc);
          if (kr == kc) {
            const R t = rot[kr][2];
            const R apq = sA[pr][qr];
            sA[pr][pr] -= t * apq;
            sA[qr][qr] += t * apq;
            sA[pr][qr] = R(0);
            sA[qr][pr] = R(0);
            continue;
          }
          const R c1 = rot[kr][0], c2 = rot[kc][0];
          const bool vqr = qr < d, vqc = qc < d;
          const R a = sA[pr][pc];
          const R b = vqc ? sA[pr][qc] : R(0);
          const R e = vqr ? sA[qr][pc] : R(0);
          const R f = (vqr && vqc) ? sA[qr][qc] : R(0);
          const R a1 = c1 * a - s1 * e, b1 = c1 * b - s1 * f;
          const R e1 = s1 * a + c1 * e, f1 = s1 * b + c1 * f;
          sA[pr][pc] = c2 * a1 - s2 * b1;
          if (vqc) sA[pr][qc] = s2 * a1 + c2 * b1;
          if (vqr) sA[qr][pc] = c2 * e1 - s2 * f1;
          if (vqr && vqc) sA[qr][qc] = s2 * e1 + c2 * f1;
        } else {
          const int v = u - nblk;
          const int k = v % P, i = v / P;
          const R s = rot[k][1];
          if (s == R(0)) continue;
          const R c = rot[k][0];
          int p, q;
          round_pair(D, r, k, p, q);
          const R x = sV[i][p], y = sV[i][q];
          sV[i][p] = c * x - s * y;
          sV[i][q] = s * x + c * y;
        }
      }
      __syncthreads();
    }
    if (cnt == 0) {
      ++sweep;
      break;
    }
    __syncthreads();
  }
  for (int u = threadIdx.x; u < d * d; u += blockDim.x) {
    const int i = u % d, j = u / d;
    A[i + (int64_t)j * lda] = (double)sA[i][j];
    Vout[i + (int64_t)j * ldv] = (double)sV[i][j];
  }
  if (threadIdx.x == 0) flags[2] = sweep;
}

// Ascending order by rank; ties keep the original index order.
__global__ void sort_eig_kernel(int d, const double *__restrict__ A, int64_t lda,
                                const double *__restrict__ V, int64_t ldv, double *__restrict__ w,
                                double *__restrict__ Q, int64_t ldq, int *__restrict__ flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
    const double li = A[i + (int64_t)i * lda];
    if (li != li) flags[1] = 1;
    int rank = 0;
    for (int j = 0; j < d; ++j) {
      const double lj = A[j + (int64_t)j * lda];
      rank += (lj < li) || (lj == li && j < i);
    }
    w[rank] = li;
    for (int r = 0; r < d; ++r) Q[r + (int64_t)rank * ldq] = V[r + (int64_t)i * ldv];
  }
}

}  // namespace

int SyevWork::alloc(int d) {
  if (d <= dcap) return GCGE_OK;
  free_all();
  const int D = d + (d & 1);
  GCGE_CUDA(cudaMalloc(&rot, sizeof(double) * 3 * (D / 2 + 1)));
  GCGE_CUDA(cudaMalloc(&V, sizeof(double) * (size_t)d * d));
  GCGE_CUDA(cudaMalloc(&sync, sizeof(unsigned) * 8));
  GCGE_CUDA(cudaMalloc(&flags, sizeof(int) * 4));
  GCGE_CUDA(cudaMallocHost(&h_flags, sizeof(int) * 4));
  int per_sm = 0;
  GCGE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, kSyevThreads, 0));
  coop_grid = per_sm * device_sm_count();
  dcap = d;
  return GCGE_OK;
}

void SyevWork::free_all() {
  mp.free_all();
  cudaFree(rot);
  cudaFree(V);
  cudaFree(sync);
  cudaFree(flags);
  if (h_flags) cudaFreeHost(h_flags);
  rot = V = nullptr;
  sync = nullptr;
  flags = h_flags = nullptr;
  dcap = 0;
}

int syev(int d, double *A, int64_t lda, double *w, double *Q, int64_t ldq, SyevWork &work,
         int *sweeps, cudaStream_t st, bool fp32_data) {
  if (d <= 0) return GCGE_OK;
  GCGE_CHECK(work.alloc(d));
  const int D = d + (d & 1);
  const int P = D / 2;
  if (d > 2 * kMaxPairs) return GCGE_EINVAL;
  const int64_t items = (int64_t)P * P + (int64_t)d * P;
  int grid = (int)((items + kSyevThreads - 1) / kSyevThreads);
  if (grid > device_sm_count()) grid = device_sm_count();
  if (d <= 48) grid = 1;                    // small leaves: one CTA, barrier = local
  if (grid > work.coop_grid) grid = work.coop_grid;
  if (grid < 1) grid = 1;
  GCGE_CUDA(cudaMemsetAsync(work.sync, 0, sizeof(unsigned) * 8, st));
  GCGE_CUDA(cudaMemsetAsync(work.flags, 0, sizeof(int) * 4, st));
  if (work.mixed && d > kSmallD) {
    const int s = syev_mixed(d, A, lda, w, Q, ldq, work.mp, work.flags, sweeps, st,
                             fp32_data ? 1e-10 : 1e-13);
    if (s == GCGE_OK) {
      GCGE_CUDA(cudaStreamSynchronize(st));
      return GCGE_OK;
    }
    if (s != GCGE_EINVAL) return s;
    GCGE_CUDA(cudaMemsetAsync(work.flags, 0, sizeof(int) * 4, st));   // fall back to FP64 Jacobi
  }
  int max_sweeps = 60;
  double *Vw = work.V;
  int64_t ldv = d;
  if (d <= kSmallD) {
    if (fp32_data)
      jacobi_small_kernel<float><<<1, 256, 0, st>>>(d, D, A, lda, Vw, ldv, work.flags, max_sweeps);
    else
      jacobi_small_kernel<double><<<1, 256, 0, st>>>(d, D, A, lda, Vw, ldv, work.flags, max_sweeps);
    GCGE_LAUNCH_CHECK();
  } else {
    void *args[] = {&d, (void *)&D, &A, &lda, &Vw, &ldv, &work.rot, &work.sync, &work.flags,
                    &max_sweeps};
    GCGE_CUDA(cudaLaunchCooperativeKernel((void *)jacobi_kernel, dim3(grid), dim3(kSyevThreads),
                                          args, 0, st));
  }
  sort_eig_kernel<<<ceil_div(d, 128), 128, 0, st>>>(d, A, lda, Vw, ldv, w, Q, ldq, work.flags);
  GCGE_LAUNCH_CHECK();
  GCGE_CUDA(cudaMemcpyAsync(work.h_flags, work.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  GCGE_CUDA(cudaStreamSynchronize(st));
  if (sweeps) *sweeps = work.h_flags[2];
  if (work.h_flags[0]) return GCGE_ETIMEOUT;
  if (work.h_flags[1]) return GCGE_ENAN;
  return GCGE_OK;
}

}  // namespace gcge
