// C ABI wrappers of the individual hot-path steps, error reporting, device queries.
#include <atomic>
#include <mutex>
#include <string>

#include "blas.cuh"
#include "cg.cuh"
#include "spmm.cuh"
#include "syev.cuh"
#include "solver.cuh"

namespace gcge {

static std::mutex g_err_mu;
static std::string g_err_msg = "no error";
std::atomic<long long> g_launches{0};

void record_cuda_error(cudaError_t e, const char *file, int line) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) at %s:%d", (int)e, cudaGetErrorString(e), file, line);
  g_err_msg = buf;
}

void record_message(const char *msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err_msg = msg;
}

int device_sm_count() {
  static int cached = -1;
  if (cached > 0) return cached;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    cached = sms;
  else
    cached = kNumSMs;
  return cached;
}

}  // namespace gcge

using namespace gcge;

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool bad_ptr(const void *p) { return p == nullptr; }

}  // namespace

extern "C" {

const char *gcge_error_string(int status) {
  switch (status) {
    case GCGE_OK: return "success";
    case GCGE_EINVAL: return "invalid argument";
    case GCGE_ENOMEM: return "device allocation failed";
    case GCGE_ECUDA: return "CUDA runtime or launch failure";
    case GCGE_ENOTCONV: return "not converged within max_iter (partial results valid)";
    case GCGE_EBREAKDOWN: return "orthogonalisation lost the whole block";
    case GCGE_ETIMEOUT: return "a bounded device-side wait timed out";
    case GCGE_ENAN: return "NaN or Inf in a Gram or Rayleigh-Ritz matrix";
    case GCGE_ENOTREADY: return "no successful solve on this handle yet";
    default: return "unknown status";
  }
}

const char *gcge_last_error_message(void) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err_msg;
  return copy.c_str();
}

int gcge_spmm_f64(int64_t n, const int32_t *rp, const int32_t *ci, const double *val, int k,
                  double alpha, const double *X, int64_t ldx, double beta, double *Y, int64_t ldy,
                  void *stream) {
  if (n < 0 || k < 1 || ldx < k || ldy < k) return GCGE_EINVAL;
  if (n > 0 && (bad_ptr(rp) || bad_ptr(X) || bad_ptr(Y))) return GCGE_EINVAL;
  g_launches += 1;
  return launch_spmm<double>(n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, nullptr, 0,
                             as_stream(stream));
}

int gcge_spmm_f32(int64_t n, const int32_t *rp, const int32_t *ci, const float *val, int k,
                  float alpha, const float *X, int64_t ldx, float beta, float *Y, int64_t ldy,
                  void *stream) {
  if (n < 0 || k < 1 || ldx < k || ldy < k) return GCGE_EINVAL;
  if (n > 0 && (bad_ptr(rp) || bad_ptr(X) || bad_ptr(Y))) return GCGE_EINVAL;
  g_launches += 1;
  return launch_spmm<float>(n, rp, ci, val, k, alpha, X, ldx, beta, Y, ldy, nullptr, 0,
                            as_stream(stream));
}

int gcge_gram_f64(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx,
                  const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                  void *stream) {
  if (n < 0 || m < 0 || k < 0 || ldx < m || ldy < k || ldc < m) return GCGE_EINVAL;
  if (m == 0 || k == 0) return GCGE_OK;
  if (bad_ptr(C) || (n > 0 && (bad_ptr(X) || bad_ptr(Y)))) return GCGE_EINVAL;
  if (!gram_f64_grid_ok(m, k)) {
    record_message("gcge_gram_f64: k needs more than 65535 column tiles");
    return GCGE_EINVAL;
  }
  Scratch ws;
  cudaStream_t st = as_stream(stream);
  g_launches += 2;
  int s = gram<double>(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, 0, ws, st);
  ws.release(st);
  return s;
}

int gcge_gram_f32(int64_t n, int m, int k, double alpha, const float *X, int64_t ldx,
                  const float *Y, int64_t ldy, double beta, double *C, int64_t ldc, int tc,
                  void *stream) {
  if (n < 0 || m < 0 || k < 0 || ldx < m || ldy < k || ldc < m) return GCGE_EINVAL;
  if (m == 0 || k == 0) return GCGE_OK;
  if (bad_ptr(C) || (n > 0 && (bad_ptr(X) || bad_ptr(Y)))) return GCGE_EINVAL;
  Scratch ws;
  cudaStream_t st = as_stream(stream);
  g_launches += 2;
  int s = gram<float>(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, tc, ws, st);
  ws.release(st);
  return s;
}

int gcge_vc_f64(int64_t n, int d, int q, double alpha, const double *V, int64_t ldv,
                const double *C, int64_t ldc, double beta, double *Y, int64_t ldy, void *stream) {
  if (n < 0 || d < 0 || q < 0 || ldv < d || ldc < d || ldy < q) return GCGE_EINVAL;
  if (q == 0 || n == 0) return GCGE_OK;
  if (bad_ptr(Y) || (d > 0 && (bad_ptr(V) || bad_ptr(C)))) return GCGE_EINVAL;
  g_launches += 1;
  return vc<double>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, 0, as_stream(stream));
}

int gcge_gram_f64_tc(int64_t n, int m, int k, double alpha, const double *X, int64_t ldx,
                     const double *Y, int64_t ldy, double beta, double *C, int64_t ldc,
                     void *stream) {
  if (n < 0 || m < 0 || k < 0 || ldx < m || ldy < k || ldc < m) return GCGE_EINVAL;
  if (m == 0 || k == 0) return GCGE_OK;
  if (bad_ptr(C) || (n > 0 && (bad_ptr(X) || bad_ptr(Y)))) return GCGE_EINVAL;
  cudaStream_t st = as_stream(stream);
  if (n == 0) return gcge_gram_f64(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, stream);
  Scratch ws;
  g_launches += 4;
  const int s = oz_gram(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, ws, st);
  ws.release(st);
  if (s == GCGE_EINVAL) record_message("gcge_gram_f64_tc: shape outside the emulated kernel");
  return s;
}

int gcge_vc_f64_tc(int64_t n, int d, int q, double alpha, const double *V, int64_t ldv,
                   const double *C, int64_t ldc, double beta, double *Y, int64_t ldy,
                   void *stream) {
  if (n < 0 || d < 0 || q < 0 || ldv < d || ldc < d || ldy < q) return GCGE_EINVAL;
  if (q == 0 || n == 0) return GCGE_OK;
  if (bad_ptr(Y) || (d > 0 && (bad_ptr(V) || bad_ptr(C)))) return GCGE_EINVAL;
  if (d == 0) return gcge_vc_f64(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, stream);
  cudaStream_t st = as_stream(stream);
  Scratch ws;
  g_launches += 3;
  const int s = oz_vc(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, ws, st);
  ws.release(st);
  if (s == GCGE_EINVAL) record_message("gcge_vc_f64_tc: shape outside the emulated kernel");
  return s;
}

int gcge_vc_f32(int64_t n, int d, int q, double alpha, const float *V, int64_t ldv,
                const double *C, int64_t ldc, double beta, float *Y, int64_t ldy, int tc,
                void *stream) {
  if (n < 0 || d < 0 || q < 0 || ldv < d || ldc < d || ldy < q) return GCGE_EINVAL;
  if (q == 0 || n == 0) return GCGE_OK;
  if (bad_ptr(Y) || (d > 0 && (bad_ptr(V) || bad_ptr(C)))) return GCGE_EINVAL;
  g_launches += tc ? 2 : 1;
  Scratch ws;
  cudaStream_t st = as_stream(stream);
  int s = vc<float>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, tc, st, &ws);
  ws.release(st);
  return s;
}

int gcge_syev(int d, double *A, int64_t lda, double *w, double *Q, int64_t ldq, int *sweeps,
              void *stream) {
  if (d < 0 || lda < d || ldq < d) return GCGE_EINVAL;
  if (d == 0) return GCGE_OK;
  if (bad_ptr(A) || bad_ptr(w) || bad_ptr(Q)) return GCGE_EINVAL;
  SyevWork work;
  g_launches += 2;
  int s = syev(d, A, lda, w, Q, ldq, work, sweeps, as_stream(stream));
  work.free_all();
  return s;
}

int gcge_block_cg_f64(int64_t n, const int32_t *rp, const int32_t *ci, const double *S, int k,
                      const double *B, int64_t ldb, double *X, int64_t ldx, int max_iter,
                      double rtol, int precond, int *iters, void *stream) {
  if (n < 1 || k < 1 || ldb < k || ldx < k || max_iter < 0) return GCGE_EINVAL;
  if (precond != GCGE_PRECOND_NONE && precond != GCGE_PRECOND_JACOBI) return GCGE_EINVAL;
  if (bad_ptr(rp) || bad_ptr(ci) || bad_ptr(S) || bad_ptr(B) || bad_ptr(X)) return GCGE_EINVAL;
  CgWork<double> w;
  int64_t nl = 0;
  cudaStream_t st = as_stream(stream);
  double *minv = nullptr;
  if (precond == GCGE_PRECOND_JACOBI) {
    GCGE_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&minv), sizeof(double) * (size_t)n, st));
    const int sj = jacobi_inverse<double>(n, rp, ci, S, minv, st);
    if (sj != GCGE_OK) {
      cudaFreeAsync(minv, st);
      return sj;
    }
  }
  int s = block_cg<double>(n, rp, ci, S, k, B, ldb, nullptr, 0, X, ldx, max_iter, rtol, w, iters,
                        &nl, st, nullptr, minv);
  if (minv) cudaFreeAsync(minv, st);
  g_launches += nl;
  cudaStreamSynchronize(as_stream(stream));
  w.free_all();
  return s < 0 ? s : GCGE_OK;
}

int gcge_block_cg_f32(int64_t n, const int32_t *rp, const int32_t *ci, const float *S, int k,
                      const float *B, int64_t ldb, float *X, int64_t ldx, int max_iter,
                      double rtol, int precond, int *iters, void *stream) {
  if (n < 1 || k < 1 || ldb < k || ldx < k || max_iter < 0) return GCGE_EINVAL;
  if (precond != GCGE_PRECOND_NONE && precond != GCGE_PRECOND_JACOBI) return GCGE_EINVAL;
  if (bad_ptr(rp) || bad_ptr(ci) || bad_ptr(S) || bad_ptr(B) || bad_ptr(X)) return GCGE_EINVAL;
  CgWork<float> w;
  int64_t nl = 0;
  cudaStream_t st = as_stream(stream);
  float *minv = nullptr;
  if (precond == GCGE_PRECOND_JACOBI) {
    GCGE_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&minv), sizeof(float) * (size_t)n, st));
    const int sj = jacobi_inverse<float>(n, rp, ci, S, minv, st);
    if (sj != GCGE_OK) {
      cudaFreeAsync(minv, st);
      return sj;
    }
  }
  int s = block_cg<float>(n, rp, ci, S, k, B, ldb, nullptr, 0, X, ldx, max_iter, rtol, w, iters,
                        &nl, st, nullptr, minv);
  if (minv) cudaFreeAsync(minv, st);
  g_launches += nl;
  cudaStreamSynchronize(as_stream(stream));
  w.free_all();
  return s < 0 ? s : GCGE_OK;
}

int gcge_borth_f64(int64_t n, const int32_t *Brp, const int32_t *Bci, const double *Bval,
                   const double *Q, int64_t ldq, int q, double *W, int64_t ldw, int m, int leaf,
                   int orth, int *m_out, void *stream) {
  if (n < 1 || m < 0 || q < 0 || ldw < m || (q > 0 && (ldq < q || bad_ptr(Q))) || leaf < 1)
    return GCGE_EINVAL;
  if (orth != GCGE_ORTH_ALG3 && orth != GCGE_ORTH_ALG2) return GCGE_EINVAL;
  if (m > 0 && bad_ptr(W)) return GCGE_EINVAL;
  const bool hasB = Brp != nullptr;
  if (hasB && (bad_ptr(Bci) || bad_ptr(Bval))) return GCGE_EINVAL;
  return borth_standalone(n, Brp, Bci, Bval, Q, ldq, q, W, ldw, m, leaf, orth, m_out,
                          as_stream(stream));
}

int gcge_tc_status(void *stream) {
  int flag = 0;
  GCGE_CHECK(tc_error_flag(&flag, as_stream(stream)));
  if (flag) {
    record_message("a tensor-core kernel's bounded wait ran out; its output is invalid");
    return GCGE_ETIMEOUT;
  }
  return GCGE_OK;
}

int gcge_random_block_f64(int64_t n, int k, uint64_t seed, double *X, int64_t ld, void *stream) {
  if (n < 0 || k < 0 || ld < k) return GCGE_EINVAL;
  if (n > 0 && k > 0 && bad_ptr(X)) return GCGE_EINVAL;
  g_launches += 1;
  return random_block<double>(n, k, seed, X, ld, as_stream(stream));
}

}  // extern "C"
