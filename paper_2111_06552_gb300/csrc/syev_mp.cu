// Mixed-precision dense symmetric eigensolver for the Rayleigh-Ritz matrix (STEP 3).
//
// FP64 throughput on GB300 is ~1/64 of FP32, and a two-sided FP64 Jacobi needs d-1
// grid-wide rounds per sweep, so it is bound by latency and the FP64 units.  Here the
// eigenvectors are first found in FP32 on chip and then polished in FP64:
//
// 1. FP32 one-sided (Hestenes) block Jacobi in one thread-block cluster of C CTAs.
//    G = Abar + sigma I with sigma from the Gershgorin bound, so G is positive
//    semidefinite and the vectors that make G's columns orthogonal are eigenvectors
//    of Abar.  The 2C blocks of b columns (of G and of the accumulated V) live in
//    shared memory, two per CTA.  A sweep is 2C-1 steps of the round-robin
//    tournament on blocks: in each step every CTA orthogonalises all column pairs
//    between its two blocks (one warp per pair, b disjoint pairs at a time), then the
//    blocks move one position around the circle by two pulls over distributed shared
//    memory with cluster barriers.  Each block's internal pairs are done in the first
//    step of a sweep, so a sweep visits every pair once.
// 2. FP64 polish with dense FP64 products on all SMs: V <- V (3I - V^T V)/2
//    (Newton-Schulz), B = V^T Abar V, lambda_i = B_ii.  Pairs in different eigenvalue
//    clusters are corrected to first order, E_ij = B_ij / (lambda_j - lambda_i); each
//    cluster (gaps below 100 x the largest off-diagonal of B) is diagonalised exactly
//    by a small FP64 Jacobi, V <- V (I + E) Q_clusters.  Repeated until the
//    off-diagonal part of B is at rounding level; eigenvalues are the final Rayleigh
//    quotients.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "blas.cuh"
#include "syev.cuh"

namespace cg = cooperative_groups;

namespace gcge {

namespace {

struct OjPlan {
  int C, b, dp, threads;
  size_t smem;
};

// Cluster size C (power of two, 1..16) and block width b such that three buffers of
// (G, V) blocks of b columns x dp rows fit in shared memory.  b <= 16 is preferred: a
// round of rotations streams its columns through shared memory, so spreading the blocks
// over more CTAs (SMs) shortens a round; b <= 32 when 16 CTAs are not enough.
bool oj_plan(int d, OjPlan &pl) {
  const int dp = ((d + 127) / 128) * 128;   // a lane takes 4 consecutive rows per 128
  for (int bmax : {16, 32}) {
    for (int C = 1; C <= 16; C <<= 1) {
      const int b = (d + 2 * C - 1) / (2 * C);
      if (b > bmax) continue;
      const size_t smem = sizeof(float) * 6 * (size_t)b * dp;
      if (smem > 200 * 1024) continue;
      const int bi = b + (b & 1);
      pl = {C, b, dp, 32 * std::max(b, bi), smem};
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ void rr_pair(int B, int r, int k, int &p, int &q) {
  const int m = B - 1;
  int a, c;
  if (k == 0) {
    a = m;
    c = r;
  } else {
    a = (r + k) % m;
    c = (r - k + m) % m;
  }
  p = a < c ? a : c;
  q = a < c ? c : a;
}

// One-sided rotation of the column pair (x, y) of G and V by one warp; a lane takes rows
// 4 lane + 128 i .. + 3 (16-byte shared-memory accesses; dp is a multiple of 128).
__device__ __forceinline__ bool oj_rotate(float *gx, float *gy, float *vx, float *vy, int dp,
                                          int lane, float tol) {
  float4 *gx4 = reinterpret_cast<float4 *>(gx), *gy4 = reinterpret_cast<float4 *>(gy);
  float4 *vx4 = reinterpret_cast<float4 *>(vx), *vy4 = reinterpret_cast<float4 *>(vy);
  const int nq = dp >> 7;
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i = 0; i < nq; ++i) {
    const float4 x = gx4[lane + 32 * i], y = gy4[lane + 32 * i];
    al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
    be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
    ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (al == 0.f || be == 0.f || !(fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return false;
  // tan of the rotation angle, the smaller root (fast reciprocal and square root: the
  // rotation only has to be orthogonal to FP32 level, the FP64 stage refines it)
  const float ze = __fdividef(be - al, 2.f * ga);
  const float h = fmaf(ze, ze, 1.f);
  const float t = __fdividef(ze >= 0.f ? 1.f : -1.f, fabsf(ze) + h * rsqrtf(h));
  const float c = rsqrtf(fmaf(t, t, 1.f));
  const float s = c * t;
  for (int i = 0; i < nq; ++i) {
    const int r = lane + 32 * i;
    const float4 x = gx4[r], y = gy4[r], u = vx4[r], w = vy4[r];
    gx4[r] = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
    gy4[r] = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
    vx4[r] = make_float4(c * u.x - s * w.x, c * u.y - s * w.y, c * u.z - s * w.z, c * u.w - s * w.w);
    vy4[r] = make_float4(s * u.x + c * w.x, s * u.y + c * w.y, s * u.z + c * w.z, s * u.w + c * w.w);
  }
  return true;
}

__global__ void oj_cluster_kernel(int d, int b, int dp, const double *__restrict__ A, int64_t lda,
                                  const double *__restrict__ gersh, float *__restrict__ Vout,
                                  int64_t ldv,
                                  float *__restrict__ gnorm, int *__restrict__ flags,
                                  int max_sweeps) {
  extern __shared__ float4 smem4[];
  float *smem = reinterpret_cast<float *>(smem4);
  __shared__ int role[2];      // buffer index (0..2) holding this CTA's top / bottom block
  __shared__ int blk[2];       // global block id of top / bottom
  __shared__ unsigned cnt[2];  // cluster rotation counters (rank 0), by sweep parity
  __shared__ unsigned local;
  __shared__ int stop;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nthr = blockDim.x;
  const size_t bufsz = (size_t)2 * b * dp;   // floats per buffer (G block then V block)
  auto G = [&](int buf, int col) { return smem + buf * bufsz + (size_t)col * dp; };
  auto V = [&](int buf, int col) { return smem + buf * bufsz + (size_t)(b + col) * dp; };
  if (threadIdx.x == 0) {
    role[0] = 0;
    role[1] = 1;
    blk[0] = rank;
    blk[1] = 2 * C - 1 - rank;
    cnt[0] = cnt[1] = 0u;
    stop = 0;
  }
  __syncthreads();
  // sigma: make G = A + sigma I positive semidefinite (Gershgorin lower bound)
  const double sigma = gersh[0] < 0.0 ? -gersh[0] : 0.0;
  for (int s = 0; s < 2; ++s) {
    const int j0 = blk[s] * b;
    for (int u = threadIdx.x; u < b * dp; u += nthr) {
      const int col = u / dp, r = u % dp;
      const int j = j0 + col;
      float g = 0.f, v = 0.f;
      if (j < d && r < d) {
        g = (float)(A[r + (int64_t)j * lda] + (r == j ? sigma : 0.0));
        v = (r == j) ? 1.f : 0.f;
      }
      G(role[s], col)[r] = g;
      V(role[s], col)[r] = v;
    }
  }
  cl.sync();
  const float tol = 1e-6f;
  const int bi = b + (b & 1);
  const int nf4 = (int)(bufsz / 4);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) local = 0u;
    __syncthreads();
    for (int step = 0; step < 2 * C - 1; ++step) {
      if (step == 0) {   // pairs inside each of the two blocks
        for (int r = 0; r < bi - 1; ++r) {
          if (warp < bi) {
            const int s = warp < bi / 2 ? 0 : 1;
            const int k = warp - s * (bi / 2);
            int p, q;
            rr_pair(bi, r, k, p, q);
            if (q < b && oj_rotate(G(role[s], p), G(role[s], q), V(role[s], p), V(role[s], q), dp,
                                   lane, tol) && lane == 0)
              atomicAdd(&local, 1u);
          }
          __syncthreads();
        }
      }
      for (int r = 0; r < b; ++r) {   // pairs between the two blocks
        if (warp < b) {
          const int q = (warp + r) % b;
          if (oj_rotate(G(role[0], warp), G(role[1], q), V(role[0], warp), V(role[1], q), dp, lane,
                        tol) && lane == 0)
            atomicAdd(&local, 1u);
        }
        __syncthreads();
      }
      if (C > 1 && step < 2 * C - 2) {
        // Circle method with position 0 fixed: CTA c holds positions c (top) and
        // 2C-1-c (bottom); new[i] = old[i-1] for i >= 2, new[1] = old[2C-1].
        cl.sync();
        const int freeb = 3 - role[0] - role[1];
        int t_blk = blk[0], b_buf = role[1], b_blk = blk[1];
        // phase 1: the new top block, pulled into the free buffer
        if (rank >= 1) {
          const int src = rank == 1 ? 0 : rank - 1;
          const int which = rank == 1 ? 1 : 0;
          const int sbuf = cl.map_shared_rank(role, src)[which];
          t_blk = cl.map_shared_rank(blk, src)[which];
          const float4 *sp = reinterpret_cast<const float4 *>(cl.map_shared_rank(smem, src) + sbuf * bufsz);
          float4 *dp4 = reinterpret_cast<float4 *>(smem + freeb * bufsz);
          for (int u = threadIdx.x; u < nf4; u += nthr) dp4[u] = sp[u];
        }
        cl.sync();
        // phase 2: the new bottom block (rank C-1 takes its own old top without a copy)
        if (rank == C - 1) {
          b_buf = role[0];
          b_blk = blk[0];
        } else {
          const int src = rank + 1;
          const int sbuf = cl.map_shared_rank(role, src)[1];
          b_blk = cl.map_shared_rank(blk, src)[1];
          b_buf = rank == 0 ? role[1] : role[0];
          const float4 *sp = reinterpret_cast<const float4 *>(cl.map_shared_rank(smem, src) + sbuf * bufsz);
          float4 *dp4 = reinterpret_cast<float4 *>(smem + b_buf * bufsz);
          for (int u = threadIdx.x; u < nf4; u += nthr) dp4[u] = sp[u];
        }
        cl.sync();
        if (threadIdx.x == 0) {
          if (rank >= 1) {
            role[0] = freeb;
            blk[0] = t_blk;
          }
          role[1] = b_buf;
          blk[1] = b_blk;
        }
        __syncthreads();
      }
    }
    // convergence: rotations over the whole cluster in this sweep
    unsigned *c0 = cl.map_shared_rank(&cnt[sweep & 1], 0);
    if (threadIdx.x == 0 && local) atomicAdd(c0, local);
    cl.sync();
    if (threadIdx.x == 0) stop = (*c0 == 0u) ? 1 : 0;
    __syncthreads();
    const bool done = stop != 0;
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) cnt[(sweep + 1) & 1] = 0u;
    if (done) {
      ++sweep;
      break;
    }
  }
  // output: V columns and G column norms (= eigenvalue + sigma for a PSD G)
  for (int s = 0; s < 2; ++s) {
    const int j0 = blk[s] * b;
    for (int col = warp; col < b; col += nthr / 32) {
      const int j = j0 + col;
      if (j >= d) continue;
      const float *g = G(role[s], col);
      const float *v = V(role[s], col);
      float nn = 0.f;
      for (int r = lane; r < dp; r += 32) nn = fmaf(g[r], g[r], nn);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      if (lane == 0) gnorm[j] = sqrtf(nn);
      for (int r = lane; r < d; r += 32) Vout[r + (int64_t)j * ldv] = v[r];
    }
  }
  if (rank == 0 && threadIdx.x == 0) flags[2] = sweep;
  cl.sync();
}

// Gershgorin lower bound min_i (a_ii - sum_{j != i} |a_ij|) -> out[0] (single CTA).
__global__ void gershgorin_kernel(int d, const double *__restrict__ A, int64_t lda,
                                  double *__restrict__ out) {
  __shared__ double red[256];
  double mn = 1e300;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    int j = 0;
    for (; j + 4 <= d; j += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) s4[u] += fabs(A[i + (int64_t)(j + u) * lda]);
    }
    for (; j < d; ++j) s4[0] += fabs(A[i + (int64_t)j * lda]);
    const double aii = A[i + (int64_t)i * lda];
    const double s = (s4[0] + s4[1]) + (s4[2] + s4[3]) - fabs(aii);
    mn = fmin(mn, aii - s);
  }
  red[threadIdx.x] = mn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// V64[:, t] = V32[:, perm[t]] with perm the ascending order of (gnorm - sigma).
__global__ void sort_convert_kernel(int d, const float *__restrict__ V32, int64_t ld32,
                                    const float *__restrict__ gn, double *__restrict__ V64,
                                    int64_t ld64) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
    const float li = gn[i];
    int rank = 0;
    for (int j = 0; j < d; ++j) rank += (gn[j] < li) || (gn[j] == li && j < i);
    for (int r = 0; r < d; ++r) V64[r + (int64_t)rank * ld64] = (double)V32[r + (int64_t)i * ld32];
  }
}

// M <- 1.5 I - 0.5 M (Newton-Schulz factor), d x d.
__global__ void ns_factor_kernel(int d, double *__restrict__ M, int64_t ld) {
  const int64_t tot = (int64_t)d * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    const double v = M[i + (int64_t)j * ld];
    M[i + (int64_t)j * ld] = (i == j ? 1.5 : 0.0) - 0.5 * v;
  }
}

constexpr int kMaxCluster = 32;
constexpr int kMaxAnalyze = 1024;   // largest d of this method (16 CTAs x 2 blocks x 32)

// Analysis of B (single CTA): lam = diag(B), the largest off-diagonal, clusters of the
// sorted lam with gaps <= 100 * max_off.  Outputs: cid[d] cluster id per column,
// clist (column indices grouped by cluster), cstart[ncl+1], info[0] = ncl,
// info[1] = largest cluster, dinfo[0] = max_off, dinfo[1] = max |lam|.
__global__ void analyze_kernel(int d, const double *__restrict__ B, int64_t ldb,
                               double *__restrict__ lam, int *__restrict__ order,
                               int *__restrict__ cid, int *__restrict__ clist,
                               int *__restrict__ cstart, int *__restrict__ info,
                               double *__restrict__ dinfo) {
  __shared__ double red[1024];
  __shared__ double slam[kMaxAnalyze];
  __shared__ int sord[kMaxAnalyze];
  __shared__ double s_off;
  double mx = 0.0, ml = 0.0;
  for (int64_t t = threadIdx.x; t < (int64_t)d * d; t += blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    const double v = B[i + (int64_t)j * ldb];
    if (i != j)
      mx = fmax(mx, fabs(v));
    else
      ml = fmax(ml, fabs(v));
  }
  for (int pass = 0; pass < 2; ++pass) {
    red[threadIdx.x] = pass == 0 ? mx : ml;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) dinfo[pass] = red[0];
    if (threadIdx.x == 0 && pass == 0) s_off = red[0];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double v = B[i + (int64_t)i * ldb];
    lam[i] = v;
    slam[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double li = slam[i];
    int rank = 0;
    for (int j = 0; j < d; ++j) rank += (slam[j] < li) || (slam[j] == li && j < i);
    order[rank] = i;
    sord[rank] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double thr = 100.0 * s_off;
    int ncl = 0, big = 0, start = 0;
    double prev = slam[sord[0]];
    for (int t = 0; t < d; ++t) {
      const int o = sord[t];
      const double cur = slam[o];
      if (t > 0 && cur - prev > thr) {
        cstart[ncl] = start;
        big = max(big, t - start);
        ++ncl;
        start = t;
      }
      prev = cur;
      cid[o] = ncl;
      clist[t] = o;
    }
    cstart[ncl] = start;
    big = max(big, d - start);
    ++ncl;
    cstart[ncl] = d;
    info[0] = ncl;
    info[1] = big;
  }
}

// M = (I + E) with E_ij = B_ij / (lam_j - lam_i) between clusters, 0 inside a cluster.
__global__ void first_order_kernel(int d, const double *__restrict__ B, int64_t ldb,
                                   const double *__restrict__ lam, const int *__restrict__ cid,
                                   double *__restrict__ M, int64_t ldm) {
  const int64_t tot = (int64_t)d * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    double v = (i == j) ? 1.0 : 0.0;
    if (i != j && cid[i] != cid[j]) v = B[i + (int64_t)j * ldb] / (lam[j] - lam[i]);
    M[i + (int64_t)j * ldm] = v;
  }
}

// Q (d x d, identity outside clusters) gets the exact eigenvectors of every cluster
// block B[c, c] (one CTA per cluster, FP64 Jacobi in shared memory, size <= 32).
__global__ void __launch_bounds__(256)
cluster_eig_kernel(int d, const double *__restrict__ B, int64_t ldb,
                   const int *__restrict__ clist, const int *__restrict__ cstart,
                   double *__restrict__ Q, int64_t ldq) {
  __shared__ double sA[kMaxCluster][kMaxCluster + 1];
  __shared__ double sV[kMaxCluster][kMaxCluster + 1];
  __shared__ double rot[kMaxCluster / 2][3];
  __shared__ int cnt;
  const int c = blockIdx.x;
  const int s0 = cstart[c], m = cstart[c + 1] - s0;
  if (m <= 1) {
    if (m == 1 && threadIdx.x == 0) {
      const int i = clist[s0];
      Q[i + (int64_t)i * ldq] = 1.0;
    }
    return;
  }
  const int D = m + (m & 1), P = D / 2;
  for (int u = threadIdx.x; u < m * m; u += blockDim.x) {
    const int a = u % m, bb = u / m;
    sA[a][bb] = B[clist[s0 + a] + (int64_t)clist[s0 + bb] * ldb];
    sV[a][bb] = a == bb ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int r = 0; r < D - 1; ++r) {
      for (int k = threadIdx.x; k < P; k += blockDim.x) {
        int p, q;
        rr_pair(D, r, k, p, q);
        double cc = 1.0, ss = 0.0, tt = 0.0;
        if (q < m) {
          const double app = sA[p][p], aqq = sA[q][q], apq = sA[p][q];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app) * fabs(aqq)) && fabs(apq) > 1e-300) {
            const double th = (aqq - app) / (2.0 * apq);
            tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            cc = rsqrt(1.0 + tt * tt);
            ss = tt * cc;
            atomicAdd(&cnt, 1);
          }
        }
        rot[k][0] = cc;
        rot[k][1] = ss;
        rot[k][2] = tt;
      }
      __syncthreads();
      for (int u = threadIdx.x; u < P * P + m * P; u += blockDim.x) {
        if (u < P * P) {
          const int kr = u % P, kc = u / P;
          const double s1 = rot[kr][1], s2 = rot[kc][1];
          if (s1 == 0.0 && s2 == 0.0) continue;
          int pr, qr, pc, qc;
          rr_pair(D, r, kr, pr, qr);
          rr_pair(D, r, kc, pc, qc);
          if (kr == kc) {
            const double tt = rot[kr][2], apq = sA[pr][qr];
            sA[pr][pr] -= tt * apq;
            sA[qr][qr] += tt * apq;
            sA[pr][qr] = sA[qr][pr] = 0.0;
            continue;
          }
          const double c1 = rot[kr][0], c2 = rot[kc][0];
          const bool vqr = qr < m, vqc = qc < m;
          const double a = sA[pr][pc];
          const double bb = vqc ? sA[pr][qc] : 0.0;
          const double e = vqr ? sA[qr][pc] : 0.0;
          const double f = (vqr && vqc) ? sA[qr][qc] : 0.0;
          const double a1 = c1 * a - s1 * e, b1 = c1 * bb - s1 * f;
          const double e1 = s1 * a + c1 * e, f1 = s1 * bb + c1 * f;
          sA[pr][pc] = c2 * a1 - s2 * b1;
          if (vqc) sA[pr][qc] = s2 * a1 + c2 * b1;
          if (vqr) sA[qr][pc] = c2 * e1 - s2 * f1;
          if (vqr && vqc) sA[qr][qc] = s2 * e1 + c2 * f1;
        } else {
          const int v = u - P * P;
          const int k = v % P, i = v / P;
          const double ss = rot[k][1];
          if (ss == 0.0) continue;
          const double cc = rot[k][0];
          int p, q;
          rr_pair(D, r, k, p, q);
          const double x = sV[i][p], y = sV[i][q];
          sV[i][p] = cc * x - ss * y;
          sV[i][q] = ss * x + cc * y;
        }
      }
      __syncthreads();
    }
    const bool done = cnt == 0;
    __syncthreads();
    if (done) break;
  }
  for (int u = threadIdx.x; u < m * m; u += blockDim.x) {
    const int a = u % m, bb = u / m;
    Q[clist[s0 + a] + (int64_t)clist[s0 + bb] * ldq] = sV[a][bb];
  }
}

__global__ void set_identity_kernel(int d, double *__restrict__ M, int64_t ld) {
  const int64_t tot = (int64_t)d * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    M[i + (int64_t)j * ld] = i == j ? 1.0 : 0.0;
  }
}

__global__ void symmetrize_full_kernel(int d, double *__restrict__ A, int64_t lda) {
  const int64_t tot = (int64_t)d * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    if (i < j) {
      const double v = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
      A[i + (int64_t)j * lda] = v;
      A[j + (int64_t)i * lda] = v;
    }
  }
}

// w[t] = lam[order[t]], Q[:, t] = V[:, order[t]].
__global__ void finish_kernel(int d, const double *__restrict__ lam, const int *__restrict__ order,
                              const double *__restrict__ V, int64_t ldv, double *__restrict__ w,
                              double *__restrict__ Q, int64_t ldq) {
  const int64_t tot = (int64_t)d * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % d), c = (int)(t / d);
    const int src = order[c];
    Q[r + (int64_t)c * ldq] = V[r + (int64_t)src * ldv];
    if (r == 0) w[c] = lam[src];
  }
}

int gridfor(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  if (g > 2048) g = 2048;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int MpWork::alloc(int d) {
  if (d <= dcap) return GCGE_OK;
  free_all();
  const size_t dd = (size_t)d * d;
  GCGE_CUDA(cudaMalloc(&V32, sizeof(float) * dd));
  GCGE_CUDA(cudaMalloc(&gn, sizeof(float) * d));
  GCGE_CUDA(cudaMalloc(&V, sizeof(double) * dd));
  GCGE_CUDA(cudaMalloc(&T1, sizeof(double) * dd));
  GCGE_CUDA(cudaMalloc(&T2, sizeof(double) * dd));
  GCGE_CUDA(cudaMalloc(&Bm, sizeof(double) * dd));
  GCGE_CUDA(cudaMalloc(&lam, sizeof(double) * d));
  GCGE_CUDA(cudaMalloc(&ints, sizeof(int) * (4 * (size_t)d + 16)));
  GCGE_CUDA(cudaMalloc(&dinfo, sizeof(double) * 8));
  GCGE_CUDA(cudaMallocHost(&h, sizeof(double) * 8));
  GCGE_CUDA(cudaMallocHost(&hi, sizeof(int) * 8));
  dcap = d;
  return GCGE_OK;
}

void MpWork::free_all() {
  cudaFree(V32); cudaFree(gn); cudaFree(V); cudaFree(T1); cudaFree(T2); cudaFree(Bm);
  cudaFree(lam); cudaFree(ints); cudaFree(dinfo);
  if (h) cudaFreeHost(h);
  if (hi) cudaFreeHost(hi);
  V32 = nullptr; gn = nullptr; V = T1 = T2 = Bm = lam = dinfo = nullptr; ints = nullptr;
  h = nullptr; hi = nullptr; dcap = 0;
}

// Returns GCGE_OK, or GCGE_EINVAL when this method does not apply (then the caller
// falls back to the FP64 Jacobi); A is not modified.
int syev_mixed(int d, const double *A, int64_t lda, double *w, double *Q, int64_t ldq,
               MpWork &mw, int *flags_dev, int *sweeps, cudaStream_t st, double off_tol) {
  OjPlan pl;
  if (d < 2 || !oj_plan(d, pl)) return GCGE_EINVAL;
  GCGE_CHECK(mw.alloc(d));
  // sigma: make G = A + sigma I positive semidefinite
  if (d > kMaxAnalyze) return GCGE_EINVAL;
  gershgorin_kernel<<<1, 256, 0, st>>>(d, A, lda, mw.dinfo + 4);   // read by the FP32 stage
  GCGE_LAUNCH_CHECK();
  // 1. FP32 one-sided block Jacobi in one cluster
  static bool attr_set = false;
  if (!attr_set) {
    GCGE_CUDA(cudaFuncSetAttribute(oj_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
    GCGE_CUDA(cudaFuncSetAttribute(oj_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_set = true;
  }
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.C);
    cfg.blockDim = dim3(pl.threads);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = pl.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int64_t ld32 = d;
    int ms = 40;
    const double *gersh = mw.dinfo + 4;
    cudaError_t e = cudaLaunchKernelEx(&cfg, oj_cluster_kernel, d, pl.b, pl.dp, A, lda, gersh,
                                       mw.V32, ld32, mw.gn, flags_dev, ms);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return GCGE_EINVAL;
    }
  }
  sort_convert_kernel<<<gridfor(d), 256, 0, st>>>(d, mw.V32, d, mw.gn, mw.V, d);
  GCGE_LAUNCH_CHECK();
  // 2. FP64 polish
  int *order = mw.ints, *cid = mw.ints + d, *clist = mw.ints + 2 * d, *cstart = mw.ints + 3 * d;
  int *info = mw.ints + 4 * d + 4;   // cstart holds up to d + 1 entries
  const int64_t ld = d;
  bool converged = false;
  double prev_off = 1e300;
  int it = 0;
  for (; it < 8; ++it) {
    for (int ns = 0; ns < (it == 0 ? 2 : 1); ++ns) {   // V <- V (3I - V^T V) / 2
      GCGE_CHECK(dgemm_small('T', 'N', d, d, d, 1.0, mw.V, ld, mw.V, ld, 0.0, mw.T1, ld, st));
      ns_factor_kernel<<<gridfor((int64_t)d * d), 256, 0, st>>>(d, mw.T1, ld);
      GCGE_LAUNCH_CHECK();
      GCGE_CHECK(dgemm_small('N', 'N', d, d, d, 1.0, mw.V, ld, mw.T1, ld, 0.0, mw.T2, ld, st));
      std::swap(mw.V, mw.T2);
    }
    GCGE_CHECK(dgemm_small('N', 'N', d, d, d, 1.0, A, lda, mw.V, ld, 0.0, mw.T1, ld, st));
    GCGE_CHECK(dgemm_small('T', 'N', d, d, d, 1.0, mw.V, ld, mw.T1, ld, 0.0, mw.Bm, ld, st));
    symmetrize_full_kernel<<<gridfor((int64_t)d * d), 256, 0, st>>>(d, mw.Bm, ld);
    GCGE_LAUNCH_CHECK();
    analyze_kernel<<<1, 1024, 0, st>>>(d, mw.Bm, ld, mw.lam, order, cid, clist, cstart, info,
                                       mw.dinfo);
    GCGE_LAUNCH_CHECK();
    GCGE_CUDA(cudaMemcpyAsync(mw.h, mw.dinfo, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    GCGE_CUDA(cudaMemcpyAsync(mw.hi, info, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    GCGE_CUDA(cudaStreamSynchronize(st));
    const double off = mw.h[0], nrm = mw.h[1];
    // done at 1e-13 of the norm, or once the off-diagonal stops shrinking near the
    // rounding level of the FP64 products (about d eps of the norm)
    if (off <= off_tol * nrm || (off <= 1e-11 * nrm && off > 0.25 * prev_off)) {
      converged = true;
      break;
    }
    prev_off = off;
    if (mw.hi[1] > kMaxCluster) return GCGE_EINVAL;   // a cluster too large for this method
    // M = (I + E) Q_clusters, V <- V M
    first_order_kernel<<<gridfor((int64_t)d * d), 256, 0, st>>>(d, mw.Bm, ld, mw.lam, cid, mw.T1, ld);
    GCGE_LAUNCH_CHECK();
    set_identity_kernel<<<gridfor((int64_t)d * d), 256, 0, st>>>(d, mw.T2, ld);
    GCGE_LAUNCH_CHECK();
    cluster_eig_kernel<<<mw.hi[0], 256, 0, st>>>(d, mw.Bm, ld, clist, cstart, mw.T2, ld);
    GCGE_LAUNCH_CHECK();
    GCGE_CHECK(dgemm_small('N', 'N', d, d, d, 1.0, mw.T1, ld, mw.T2, ld, 0.0, mw.Bm, ld, st));
    GCGE_CHECK(dgemm_small('N', 'N', d, d, d, 1.0, mw.V, ld, mw.Bm, ld, 0.0, mw.T1, ld, st));
    std::swap(mw.V, mw.T1);
  }
  if (!converged) return GCGE_EINVAL;
  finish_kernel<<<gridfor((int64_t)d * d), 256, 0, st>>>(d, mw.lam, order, mw.V, ld, w, Q, ldq);
  GCGE_LAUNCH_CHECK();
  if (sweeps) *sweeps = it;
  return GCGE_OK;
}

}  // namespace gcge
