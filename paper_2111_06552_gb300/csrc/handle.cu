// Solver handle: gcge_create / gcge_solve / gcge_eigenpairs / gcge_stats_get / gcge_destroy.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "solver.cuh"

namespace gcge {

template <typename T>
class Engine;

// Engine is defined in solver.cu; these thin entry points instantiate it there.
int run_fp64(gcge_handle *h, const double *X0d, int64_t ld0, int *iters);
int run_mixed(gcge_handle *h, const double *X0d, int64_t ld0, int *iters, int *iters32);

namespace {

// ---------------------------------------------------------------- matrix intake
// The caller's CSR arrays go to the device as they are; the checks, the FP32 copy
// of the values and the union pattern of S = A - theta B are formed there.

// Grid for the one-pass intake kernels (rows or entries, grid-stride).
int intake_grid(int64_t tot) {
  const int64_t cap = (int64_t)device_sm_count() * 8;
  int64_t g = (tot + 255) / 256;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// Storage checks of one CSR matrix, one thread per row.  flags[0]: malformed
// pattern (row_ptr not a non-decreasing path from 0 to nnz, a column outside
// [0, n), columns not strictly increasing in a row); flags[1]: a value that is
// not finite; *nodiag: some row does not store its diagonal entry.  Every read
// stays inside row_ptr[0..n] and, for a row whose bounds pass, inside [0, nnz).
__global__ void inspect_csr_kernel(int64_t n, int64_t nnz, const int32_t *__restrict__ rp,
                                   const int32_t *__restrict__ ci, const double *__restrict__ val,
                                   int *flags, int *nodiag) {
  bool bad = false, nonfin = false, missing = false;
  if (blockIdx.x == 0 && threadIdx.x == 0) bad = rp[0] != 0 || (int64_t)rp[n] != nnz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = rp[i], r1 = rp[i + 1];
    if (r0 < 0 || r1 < r0 || r1 > nnz) {
      bad = true;
      continue;
    }
    bool diag = false;
    int64_t prev = -1;
    for (int64_t e = r0; e < r1; ++e) {
      const int64_t c = ci[e];
      if (c < 0 || c >= n || c <= prev) bad = true;
      prev = c;
      diag = diag || c == i;
      if (!isfinite(val[e])) nonfin = true;
    }
    missing = missing || !diag;
  }
  // every thread of the block reaches this point: warp votes, then one atomic per warp
  const unsigned m = 0xffffffffu;
  const bool any_bad = __any_sync(m, bad), any_nf = __any_sync(m, nonfin),
             any_miss = __any_sync(m, missing);
  if ((threadIdx.x & 31) == 0) {
    if (any_bad) atomicOr(&flags[0], 1);
    if (any_nf) atomicOr(&flags[1], 1);
    if (any_miss) atomicOr(nodiag, 1);
  }
}

// *differ = 1 when the two patterns (same n, same nnz) are not identical.
__global__ void same_pattern_kernel(int64_t n, int64_t nnz, const int32_t *__restrict__ rpA,
                                    const int32_t *__restrict__ ciA,
                                    const int32_t *__restrict__ rpB,
                                    const int32_t *__restrict__ ciB, int *differ) {
  bool d = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t u = t0; u <= n; u += stride) d = d || rpA[u] != rpB[u];
  for (int64_t u = t0; u < nnz; u += stride) d = d || ciA[u] != ciB[u];
  if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(differ, 1);
}

__global__ void values_to_f32_kernel(int64_t nnz, const double *__restrict__ v,
                                     float *__restrict__ f) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nnz;
       u += (int64_t)gridDim.x * blockDim.x)
    f[u] = (float)v[u];
}

// Union pattern equal to A's own (B has A's pattern, or B = I and A stores every
// diagonal entry): entry e of S is entry e of A (and of B).  Runs after the checks
// passed, so row_ptr is a valid non-decreasing path inside [0, nnz].
__global__ void identity_maps_kernel(int64_t n, const int32_t *__restrict__ rp,
                                     const int32_t *__restrict__ ci, int *__restrict__ mapA,
                                     int *__restrict__ mapB, int *__restrict__ isdiag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      mapA[e] = (int)e;
      if (mapB) mapB[e] = (int)e;
      isdiag[e] = ci[e] == i ? 1 : 0;
    }
  }
}

// Copy the caller's arrays into the handle's device memory (host or device source).
int upload(const gcge_csr *m, DevCsr &d, cudaStream_t st) {
  d.n = m->n;
  d.nnz = m->nnz;
  const cudaMemcpyKind kind = m->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GCGE_CUDA(cudaMalloc(&d.rp, sizeof(int32_t) * (m->n + 1)));
  GCGE_CUDA(cudaMalloc(&d.ci, sizeof(int32_t) * std::max<int64_t>(m->nnz, 1)));
  GCGE_CUDA(cudaMalloc(&d.v64, sizeof(double) * std::max<int64_t>(m->nnz, 1)));
  GCGE_CUDA(cudaMemcpyAsync(d.rp, m->row_ptr, sizeof(int32_t) * (m->n + 1), kind, st));
  GCGE_CUDA(cudaMemcpyAsync(d.ci, m->col_idx, sizeof(int32_t) * m->nnz, kind, st));
  GCGE_CUDA(cudaMemcpyAsync(d.v64, m->val, sizeof(double) * m->nnz, kind, st));
  return GCGE_OK;
}

int make_f32(DevCsr &d, cudaStream_t st) {
  GCGE_CUDA(cudaMalloc(&d.v32, sizeof(float) * std::max<int64_t>(d.nnz, 1)));
  values_to_f32_kernel<<<intake_grid(d.nnz), 256, 0, st>>>(d.nnz, d.v64, d.v32);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

// Row pointers and columns of a caller's matrix on the host: its own arrays when
// they are host memory, else a copy.
struct HostPattern {
  int64_t n = 0, nnz = 0;
  const int32_t *rp = nullptr, *ci = nullptr;
  std::vector<int32_t> rp_copy, ci_copy;
};

int host_pattern(const gcge_csr *m, HostPattern &p) {
  p.n = m->n;
  p.nnz = m->nnz;
  if (!m->on_device) {
    p.rp = m->row_ptr;
    p.ci = m->col_idx;
    return GCGE_OK;
  }
  p.rp_copy.resize(m->n + 1);
  p.ci_copy.resize(m->nnz);
  GCGE_CUDA(cudaMemcpy(p.rp_copy.data(), m->row_ptr, sizeof(int32_t) * (m->n + 1),
                       cudaMemcpyDeviceToHost));
  GCGE_CUDA(cudaMemcpy(p.ci_copy.data(), m->col_idx, sizeof(int32_t) * m->nnz,
                       cudaMemcpyDeviceToHost));
  p.rp = p.rp_copy.data();
  p.ci = p.ci_copy.data();
  return GCGE_OK;
}

// General union pattern of A and B (or A and the diagonal when B = I) with the
// position of each union entry in A and in B (-1 when absent), for S = A - theta B.
// Used when the union is not A's own pattern.
int build_union(const HostPattern &A, const HostPattern *B, gcge_handle *h) {
  const int64_t n = A.n;
  std::vector<int32_t> rp(n + 1, 0), ci;
  std::vector<int> mA, mB, dg;
  ci.reserve(A.nnz + n);
  mA.reserve(A.nnz + n);
  mB.reserve(A.nnz + n);
  dg.reserve(A.nnz + n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t a = A.rp[i], ae = A.rp[i + 1];
    int64_t b = 0, be = 0;
    if (B) {
      b = B->rp[i];
      be = B->rp[i + 1];
    }
    bool diag_done = false;
    while (a < ae || (B ? b < be : !diag_done)) {
      const int64_t ca = a < ae ? A.ci[a] : INT64_MAX;
      int64_t cb;
      if (B)
        cb = b < be ? B->ci[b] : INT64_MAX;
      else
        cb = diag_done ? INT64_MAX : i;
      const int64_t c = std::min(ca, cb);
      ci.push_back((int32_t)c);
      mA.push_back(ca == c ? (int)a : -1);
      if (B) {
        mB.push_back(cb == c ? (int)b : -1);
        if (cb == c) ++b;
      } else {
        if (cb == c) diag_done = true;
      }
      dg.push_back(c == i ? 1 : 0);
      if (ca == c) ++a;
    }
    rp[i + 1] = (int32_t)ci.size();
  }
  h->S.n = n;
  h->S.nnz = (int64_t)ci.size();
  GCGE_CUDA(cudaMalloc(&h->S.rp, sizeof(int32_t) * (n + 1)));
  GCGE_CUDA(cudaMalloc(&h->S.ci, sizeof(int32_t) * ci.size()));
  GCGE_CUDA(cudaMalloc(&h->mapA, sizeof(int) * ci.size()));
  GCGE_CUDA(cudaMalloc(&h->isdiag, sizeof(int) * ci.size()));
  GCGE_CUDA(cudaMemcpy(h->S.rp, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->S.ci, ci.data(), sizeof(int32_t) * ci.size(), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->mapA, mA.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  GCGE_CUDA(cudaMemcpy(h->isdiag, dg.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  if (B) {
    GCGE_CUDA(cudaMalloc(&h->mapB, sizeof(int) * ci.size()));
    GCGE_CUDA(cudaMemcpy(h->mapB, mB.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  }
  return GCGE_OK;
}

// The union is A's own pattern: S shares A's row pointers and columns (copied).
int identity_union(gcge_handle *h, bool withB) {
  const int64_t n = h->A.n, nnz = h->A.nnz;
  h->S.n = n;
  h->S.nnz = nnz;
  const size_t e = (size_t)std::max<int64_t>(nnz, 1);
  GCGE_CUDA(cudaMalloc(&h->S.rp, sizeof(int32_t) * (n + 1)));
  GCGE_CUDA(cudaMalloc(&h->S.ci, sizeof(int32_t) * e));
  GCGE_CUDA(cudaMalloc(&h->mapA, sizeof(int) * e));
  GCGE_CUDA(cudaMalloc(&h->isdiag, sizeof(int) * e));
  if (withB) GCGE_CUDA(cudaMalloc(&h->mapB, sizeof(int) * e));
  GCGE_CUDA(cudaMemcpyAsync(h->S.rp, h->A.rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice,
                            h->st));
  GCGE_CUDA(cudaMemcpyAsync(h->S.ci, h->A.ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice,
                            h->st));
  identity_maps_kernel<<<intake_grid(n), 256, 0, h->st>>>(n, h->A.rp, h->A.ci, h->mapA,
                                                          withB ? h->mapB : nullptr, h->isdiag);
  GCGE_LAUNCH_CHECK();
  return GCGE_OK;
}

struct DevFlags {
  int *p = nullptr;
  ~DevFlags() {
    if (p) cudaFree(p);
  }
};

// Upload, check and prepare A and B: EINVAL for a malformed pattern, else ENAN for
// a non-finite value.  Returns after the device copies are complete, so the
// caller may free its arrays.
int intake(const gcge_csr *A, const gcge_csr *B, bool want32, gcge_handle *h) {
  GCGE_CHECK(upload(A, h->A, h->st));
  if (B) GCGE_CHECK(upload(B, h->B, h->st));
  // flags: 0 malformed, 1 non-finite, 2 A lacks a diagonal entry, 3 (B's, unused),
  // 4 patterns of A and B differ
  DevFlags f;
  GCGE_CUDA(cudaMalloc(&f.p, 8 * sizeof(int)));
  GCGE_CUDA(cudaMemsetAsync(f.p, 0, 8 * sizeof(int), h->st));
  inspect_csr_kernel<<<intake_grid(A->n), 256, 0, h->st>>>(A->n, A->nnz, h->A.rp, h->A.ci,
                                                           h->A.v64, f.p, f.p + 2);
  GCGE_LAUNCH_CHECK();
  const bool same_size = B && B->nnz == A->nnz;
  if (B) {
    inspect_csr_kernel<<<intake_grid(B->n), 256, 0, h->st>>>(B->n, B->nnz, h->B.rp, h->B.ci,
                                                             h->B.v64, f.p, f.p + 3);
    GCGE_LAUNCH_CHECK();
    if (same_size) {
      same_pattern_kernel<<<intake_grid(A->nnz + A->n + 1), 256, 0, h->st>>>(
          A->n, A->nnz, h->A.rp, h->A.ci, h->B.rp, h->B.ci, f.p + 4);
      GCGE_LAUNCH_CHECK();
    }
  }
  int hf[8];
  GCGE_CUDA(cudaMemcpyAsync(hf, f.p, sizeof(hf), cudaMemcpyDeviceToHost, h->st));
  GCGE_CUDA(cudaStreamSynchronize(h->st));
  if (hf[0]) return GCGE_EINVAL;
  if (hf[1]) return GCGE_ENAN;
  if (want32) {
    GCGE_CHECK(make_f32(h->A, h->st));
    if (B) GCGE_CHECK(make_f32(h->B, h->st));
  }
  const bool own = B ? (same_size && !hf[4]) : !hf[2];
  if (own) {
    GCGE_CHECK(identity_union(h, B != nullptr));
  } else {
    HostPattern pa, pb;
    GCGE_CHECK(host_pattern(A, pa));
    if (B) GCGE_CHECK(host_pattern(B, pb));
    GCGE_CHECK(build_union(pa, B ? &pb : nullptr, h));
  }
  GCGE_CUDA(cudaStreamSynchronize(h->st));
  return GCGE_OK;
}

void free_handle(gcge_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  h->A.free_all();
  h->B.free_all();
  h->S.free_all();
  cudaFree(h->mapA);
  cudaFree(h->mapB);
  cudaFree(h->isdiag);
  cudaFree(h->store);
  h->mapA = h->mapB = h->isdiag = nullptr;
  h->store = nullptr;
}

// Two pinned staging buffers and their events, released (after the stream has
// drained) on every exit path.
struct Staging {
  double *buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t st = nullptr;
  ~Staging() {
    if (buf[0] || buf[1]) cudaStreamSynchronize(st);
    for (int b = 0; b < 2; ++b) {
      if (buf[b]) cudaFreeHost(buf[b]);
      if (ev[b]) cudaEventDestroy(ev[b]);
    }
  }
};

// Device n x k (leading dimension n) to host (leading dimension ldv) in pieces of
// at most 8 MB through two pinned buffers: the GPU fills one while the CPU copies
// the other into the destination.  The CPU thus writes the caller's pages itself;
// a direct copy into pageable memory that was never touched runs about a hundred
// times slower than into touched pages.
int copy_out_staged(double *dst, int64_t ldv, const double *src, int64_t n, int k,
                    cudaStream_t st) {
  int64_t rows = n, cols = k;
  if (ldv == n) {            // contiguous destination: one flat array
    rows = n * k;
    cols = 1;
  }
  const int64_t piece = std::min<int64_t>(rows, (int64_t)1 << 20);   // doubles
  Staging sg;
  sg.st = st;
  // GCGE_NO_PINNED_STAGING=1 takes the direct-copy branch below as if no pinned
  // memory could be allocated (used by the tests of that branch)
  static const bool no_pinned = [] {
    const char *e = std::getenv("GCGE_NO_PINNED_STAGING");
    return e && e[0] == '1';
  }();
  for (int b = 0; b < 2; ++b) {
    if (no_pinned ||
        cudaHostAlloc(reinterpret_cast<void **>(&sg.buf[b]), sizeof(double) * piece,
                      cudaHostAllocDefault) != cudaSuccess) {
      // no pinned memory to stage through: one direct copy
      (void)cudaGetLastError();
      sg.buf[b] = nullptr;
      GCGE_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ldv, src, sizeof(double) * n,
                                  sizeof(double) * n, k, cudaMemcpyDeviceToHost, st));
      GCGE_CUDA(cudaStreamSynchronize(st));
      return GCGE_OK;
    }
    GCGE_CUDA(cudaEventCreateWithFlags(&sg.ev[b], cudaEventDisableTiming));
  }
  int64_t pc = 0, pr = 0, plen = 0;    // the piece in flight before this one
  int64_t p = 0;
  for (int64_t c = 0; c < cols; ++c) {
    for (int64_t r0 = 0; r0 < rows; r0 += piece) {
      const int64_t len = std::min(piece, rows - r0);
      const int b = (int)(p & 1);
      GCGE_CUDA(cudaMemcpyAsync(sg.buf[b], src + c * n + r0, sizeof(double) * len,
                                cudaMemcpyDeviceToHost, st));
      GCGE_CUDA(cudaEventRecord(sg.ev[b], st));
      if (p > 0) {
        GCGE_CUDA(cudaEventSynchronize(sg.ev[b ^ 1]));
        std::memcpy(dst + pc * ldv + pr, sg.buf[b ^ 1], sizeof(double) * plen);
      }
      pc = c;
      pr = r0;
      plen = len;
      ++p;
    }
  }
  if (p > 0) {
    const int b = (int)((p - 1) & 1);
    GCGE_CUDA(cudaEventSynchronize(sg.ev[b]));
    std::memcpy(dst + pc * ldv + pr, sg.buf[b], sizeof(double) * plen);
  }
  return GCGE_OK;
}

__global__ void transpose_out_kernel(int64_t n, int k, const int *__restrict__ perm,
                                     const double *__restrict__ S, int64_t lds,
                                     double *__restrict__ out, int64_t ldo) {
  // out (n x k, column-major ldo) column t = store column perm[t]
  const int64_t tot = n * k;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < tot;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = u % n;
    const int t = (int)(u / n);
    out[r + (int64_t)t * ldo] = S[r * lds + perm[t]];
  }
}

}  // namespace
}  // namespace gcge

using namespace gcge;

extern "C" {

int gcge_options_default(gcge_options *o) {
  if (!o) return GCGE_EINVAL;
  o->precision = GCGE_FP64;
  o->cg_max_iter = 30;
  o->cg_rtol = 1e-2;
  o->use_shift = 1;
  o->orth_leaf = 16;
  o->moving = -1;
  o->size_x = 0;
  o->max_iter = 2000;
  o->seed = 0;
  o->initial_block = nullptr;
  o->mixed_switch_tol = 3e-6;
  o->mixed_bs2 = 0;
  o->verbose = 0;
  o->checks = 0;
  o->profile = 0;
  o->orth = GCGE_ORTH_ALG3;
  o->precond = GCGE_PRECOND_NONE;
  o->fp64_emulation = 1;
  o->max_proj_dim = 0;
  return GCGE_OK;
}

int gcge_create(const gcge_csr *A, const gcge_csr *B, int nev, int block_size, double tol,
                const gcge_options *opt, void *stream, gcge_handle **out) {
  if (!out) return GCGE_EINVAL;
  *out = nullptr;
  if (!A || A->n < 2 || A->nnz < 1 || !A->row_ptr || !A->col_idx || !A->val) return GCGE_EINVAL;
  if (nev < 1 || nev >= A->n || block_size < 1 || block_size > nev || !(tol > 0.0))
    return GCGE_EINVAL;
  if (B && (B->n != A->n || B->nnz < 1 || !B->row_ptr || !B->col_idx || !B->val))
    return GCGE_EINVAL;
  gcge_handle *h = new gcge_handle();
  if (opt)
    h->opt = *opt;
  else
    gcge_options_default(&h->opt);
  if (h->opt.cg_max_iter < 0 || h->opt.orth_leaf < 1 || h->opt.max_iter < 1 ||
      h->opt.mixed_bs2 < 0 || h->opt.max_proj_dim < 0 ||
      (h->opt.orth != GCGE_ORTH_ALG3 && h->opt.orth != GCGE_ORTH_ALG2) ||
      (h->opt.precond != GCGE_PRECOND_NONE && h->opt.precond != GCGE_PRECOND_JACOBI) ||
      (h->opt.precision != GCGE_FP64 && h->opt.precision != GCGE_MIXED)) {
    delete h;
    return GCGE_EINVAL;
  }
  h->st = reinterpret_cast<cudaStream_t>(stream);
  h->n = A->n;
  h->nev = nev;
  h->bs = block_size;
  h->tol = tol;
  h->moving = h->opt.moving == 1 || (h->opt.moving < 0 && nev >= 500);
  int sx = h->opt.size_x;
  if (h->moving && h->opt.max_proj_dim > 0) {
    // maxProjDim bounds [X, P, W]: the X window takes what P and W (bs each) leave
    if (h->opt.max_proj_dim < 3 * block_size ||
        (sx > 0 && sx != h->opt.max_proj_dim - 2 * block_size)) {
      record_message("max_proj_dim must be >= 3 blockSize and agree with size_x");
      delete h;
      return GCGE_EINVAL;
    }
    sx = h->opt.max_proj_dim - 2 * block_size;
  }
  if (sx <= 0) sx = h->moving ? 3 * block_size : nev + 3 * block_size;
  if (sx > A->n) sx = (int)A->n;
  if (sx < block_size || (!h->moving && sx < nev)) {
    delete h;
    return GCGE_EINVAL;
  }
  h->size_x = sx;
  const bool want32 = h->opt.precision == GCGE_MIXED;
  int s = intake(A, B, want32, h);
  if (s != GCGE_OK) {
    free_handle(h);
    delete h;
    return s;
  }
  // locked-vector store in FP64: the prefix may overshoot nev by up to size_x
  h->store_cap = nev + sx;
  h->ld_store = round_up(h->store_cap, 4);
  if (cudaMalloc(&h->store, sizeof(double) * (size_t)h->n * h->ld_store) != cudaSuccess) {
    free_handle(h);
    delete h;
    return GCGE_ENOMEM;
  }
  *out = h;
  return GCGE_OK;
}

int gcge_solve(gcge_handle *h) {
  if (!h) return GCGE_EINVAL;
  h->solved = false;
  h->stats = gcge_stats{};
  h->lam.clear();
  h->nconv = 0;
  double *X0d = nullptr;
  if (h->opt.initial_block) {
    if (cudaMalloc(&X0d, sizeof(double) * (size_t)h->n * h->size_x) != cudaSuccess)
      return GCGE_ENOMEM;
    GCGE_CUDA(cudaMemcpyAsync(X0d, h->opt.initial_block, sizeof(double) * (size_t)h->n * h->size_x,
                              cudaMemcpyHostToDevice, h->st));
  }
  const long long l0 = g_launches.load();
  auto t0 = std::chrono::steady_clock::now();
  int it = 0, it32 = 0;
  int s;
  if (h->opt.precision == GCGE_MIXED)
    s = run_mixed(h, X0d, h->size_x, &it, &it32);
  else
    s = run_fp64(h, X0d, h->size_x, &it);
  cudaStreamSynchronize(h->st);
  h->stats.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->stats.iterations = it;
  h->stats.iterations_fp32 = it32;
  h->stats.nconv = h->nconv;
  h->stats.kernel_launches = g_launches.load() - l0;
  if (X0d) cudaFree(X0d);
  if (s == GCGE_OK || s == GCGE_ENOTCONV) h->solved = true;
  return s;
}

int gcge_eigenpairs(gcge_handle *h, double *evals, double *evecs, int64_t ldv, int evecs_on_device,
                    int *nconv) {
  if (!h || !evals) return GCGE_EINVAL;
  if (!h->solved) return GCGE_ENOTREADY;
  if (evecs && ldv < h->n) return GCGE_EINVAL;
  const int nl = (int)h->lam.size();
  std::vector<int> perm(nl);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return h->lam[a] < h->lam[b]; });
  const int k = std::min(nl, h->nev);
  for (int t = 0; t < h->nev; ++t) evals[t] = t < k ? h->lam[perm[t]] : NAN;
  if (nconv) *nconv = nl;
  if (evecs && k > 0) {
    // device temporaries, freed on every exit path once the stream has drained
    struct Temps {
      int *dperm = nullptr;
      double *tmp = nullptr;
      cudaStream_t st = nullptr;
      ~Temps() {
        if (dperm || tmp) cudaStreamSynchronize(st);
        if (dperm) cudaFree(dperm);
        if (tmp) cudaFree(tmp);
      }
    } t;
    t.st = h->st;
    GCGE_CUDA(cudaMalloc(&t.dperm, sizeof(int) * k));
    GCGE_CUDA(cudaMemcpyAsync(t.dperm, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, h->st));
    double *dst = evecs;
    if (!evecs_on_device) {
      GCGE_CUDA(cudaMalloc(&t.tmp, sizeof(double) * (size_t)h->n * k));
      dst = t.tmp;
    }
    const int64_t ldo = evecs_on_device ? ldv : h->n;
    int64_t g = ((int64_t)h->n * k + 255) / 256;
    if (g > 4096) g = 4096;
    transpose_out_kernel<<<(int)g, 256, 0, h->st>>>(h->n, k, t.dperm, h->store, h->ld_store, dst,
                                                    ldo);
    GCGE_LAUNCH_CHECK();
    GCGE_CUDA(cudaStreamSynchronize(h->st));
    if (!evecs_on_device) GCGE_CHECK(copy_out_staged(evecs, ldv, t.tmp, h->n, k, h->st));
  }
  return GCGE_OK;
}

int gcge_stats_get(gcge_handle *h, gcge_stats *st) {
  if (!h || !st) return GCGE_EINVAL;
  *st = h->stats;
  return GCGE_OK;
}

void gcge_destroy(gcge_handle *h) {
  if (!h) return;
  free_handle(h);
  delete h;
}

}  // extern "C"
