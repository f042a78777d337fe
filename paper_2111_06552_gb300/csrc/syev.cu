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

__global__ void __launch_bounds__(kSyevThreads)
jacobi_kernel(int d, int D, double *__restrict__ A, int64_t lda, double *__restrict__ V,
              int64_t ldv, double *__restrict__ rot, unsigned *__restrict__ sync,
              int *__restrict__ flags, int max_sweeps) {
  const int P = D / 2;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const unsigned nb = gridDim.x;
  for (int64_t u = gt; u < (int64_t)d * d; u += gs) {
    const int i = (int)(u % d), j = (int)(u / d);
    V[i + (int64_t)j * ldv] = (i == j) ? 1.0 : 0.0;
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
    for (int r = 0; r < D - 1; ++r) {
      // phase A: rotation of every pair of this round
      for (int64_t k = gt; k < P; k += gs) {
        int p, q;
        round_pair(D, r, (int)k, p, q);
        double c = 1.0, s = 0.0, t = 0.0;
        if (q < d) {
          const double app = A[p + (int64_t)p * lda], aqq = A[q + (int64_t)q * lda];
          const double apq = A[p + (int64_t)q * lda];
          if (apq != apq || app != app || aqq != aqq) flags[1] = 1;
          const double thr = 1e-15 * sqrt(fabs(app) * fabs(aqq));
          if (fabs(apq) > thr && fabs(apq) > 1e-300) {
            const double th = (aqq - app) / (2.0 * apq);
            t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            atomicAdd(cnt, 1u);
          }
        }
        rot[3 * k] = c;
        rot[3 * k + 1] = s;
        rot[3 * k + 2] = t;
      }
      if (!grid_barrier(sync, flags, nb)) return;
      // phase B: 2x2 blocks of A, then rows of V
      const int64_t nblk = (int64_t)P * P;
      for (int64_t u = gt; u < nblk + (int64_t)d * P; u += gs) {
        if (u < nblk) {
          const int kr = (int)(u % P), kc = (int)(u / P);
          const double s1 = rot[3 * kr + 1], s2 = rot[3 * kc + 1];
          if (s1 == 0.0 && s2 == 0.0) continue;
          int pr, qr, pc, qc;
          round_pair(D, r, kr, pr, qr);
          round_pair(D, r, kc, pc, qc);
          if (kr == kc) {   // diagonal block of an active rotation: exact update
            const double t = rot[3 * kr + 2];
            const double apq = A[pr + (int64_t)qr * lda];
            A[pr + (int64_t)pr * lda] -= t * apq;
            A[qr + (int64_t)qr * lda] += t * apq;
            A[pr + (int64_t)qr * lda] = 0.0;
            A[qr + (int64_t)pr * lda] = 0.0;
            continue;
          }
          const double c1 = rot[3 * kr], c2 = rot[3 * kc];
          const bool vqr = qr < d, vqc = qc < d;
          double *ap = A + pr + (int64_t)pc * lda;
          const double a = *ap;
          const double b = vqc ? A[pr + (int64_t)qc * lda] : 0.0;
          const double e = vqr ? A[qr + (int64_t)pc * lda] : 0.0;
          const double f = (vqr && vqc) ? A[qr + (int64_t)qc * lda] : 0.0;
          const double a1 = c1 * a - s1 * e, b1 = c1 * b - s1 * f;
          const double e1 = s1 * a + c1 * e, f1 = s1 * b + c1 * f;
          *ap = c2 * a1 - s2 * b1;
          if (vqc) A[pr + (int64_t)qc * lda] = s2 * a1 + c2 * b1;
          if (vqr) A[qr + (int64_t)pc * lda] = c2 * e1 - s2 * f1;
          if (vqr && vqc) A[qr + (int64_t)qc * lda] = s2 * e1 + c2 * f1;
        } else {
          const int64_t v = u - nblk;
          const int k = (int)(v % P), i = (int)(v / P);
          const double s = rot[3 * k + 1];
          if (s == 0.0) continue;
          const double c = rot[3 * k];
          int p, q;
          round_pair(D, r, k, p, q);
          double *vp = V + i + (int64_t)p * ldv;
          double *vq = V + i + (int64_t)q * ldv;
          const double x = *vp, y = *vq;
          *vp = c * x - s * y;
          *vq = s * x + c * y;
        }
      }
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
         int *sweeps, cudaStream_t st) {
  if (d <= 0) return GCGE_OK;
  GCGE_CHECK(work.alloc(d));
  const int D = d + (d & 1);
  const int P = D / 2;
  const int64_t items = (int64_t)P * P + (int64_t)d * P;
  int grid = (int)((items + kSyevThreads - 1) / kSyevThreads);
  if (d <= 48) grid = 1;                    // small leaves: one CTA, barrier = local
  if (grid > work.coop_grid) grid = work.coop_grid;
  if (grid < 1) grid = 1;
  GCGE_CUDA(cudaMemsetAsync(work.sync, 0, sizeof(unsigned) * 8, st));
  GCGE_CUDA(cudaMemsetAsync(work.flags, 0, sizeof(int) * 4, st));
  int max_sweeps = 60;
  double *Vw = work.V;
  int64_t ldv = d;
  void *args[] = {&d, (void *)&D, &A, &lda, &Vw, &ldv, &work.rot, &work.sync, &work.flags,
                  &max_sweeps};
  GCGE_CUDA(cudaLaunchCooperativeKernel((void *)jacobi_kernel, dim3(grid), dim3(kSyevThreads),
                                        args, 0, st));
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
