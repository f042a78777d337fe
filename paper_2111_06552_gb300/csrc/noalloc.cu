// gcge_gram_f64_noalloc: the FP64 Gram product with library-owned static scratch.
//
// Who needs this: callers that must not allocate device memory while they run,
// for example an application whose own allocator has already reserved nearly all
// of HBM (a cudaMalloc here could fail or fragment its pool), or a latency-critical
// loop that cannot afford cudaMalloc/cudaFree (they may synchronise the device and
// take allocator locks).  gcge_gram_f64 needs a split-K partial-sum buffer and
// obtains it with cudaMallocAsync; this variant uses a fixed array in device memory
// that is part of the library image instead, so it allocates nothing.
//
// The array g_gram_scratch below is a file-scope __device__ array of
// GCGE_GRAM_NOALLOC_MAX_DOUBLES doubles (16 MiB).  Every GPU on which the library is
// loaded holds it until the process exits.  In host code its name is only a
// host-side stand-in: the device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <mutex>

#include "blas.cuh"

namespace gcge {
void record_message(const char *msg);
}

namespace {

static __device__ __align__(256) double g_gram_scratch[GCGE_GRAM_NOALLOC_MAX_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the first
// call on that device, which therefore must not happen during stream capture).
int scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    gcge::record_cuda_error(e, __FILE__, __LINE__);
    return GCGE_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    gcge::record_message("gcge_gram_f64_noalloc: device index beyond the 64 devices it serves");
    return GCGE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess || p == nullptr) {
      gcge::record_cuda_error(e, __FILE__, __LINE__);
      return GCGE_ECUDA;
    }
    g_addr[dev] = static_cast<double *>(p);
  }
  *out = g_addr[dev];
  return GCGE_OK;
}

}  // namespace

extern "C" int gcge_gram_f64_noalloc(int64_t n, int m, int k, double alpha, const double *X,
                                     int64_t ldx, const double *Y, int64_t ldy, double beta,
                                     double *C, int64_t ldc, void *stream) {
  if (n < 0 || m < 0 || k < 0 || ldx < m || ldy < k || ldc < m) return GCGE_EINVAL;
  if (m == 0 || k == 0) return GCGE_OK;
  if (!C || (n > 0 && (!X || !Y))) return GCGE_EINVAL;
  if ((int64_t)m * k > (int64_t)GCGE_GRAM_NOALLOC_MAX_DOUBLES) {
    gcge::record_message(
        "gcge_gram_f64_noalloc: m * k exceeds GCGE_GRAM_NOALLOC_MAX_DOUBLES (static scratch)");
    return GCGE_EINVAL;
  }
  if (!gcge::gram_f64_grid_ok(m, k)) {
    gcge::record_message("gcge_gram_f64_noalloc: k needs more than 65535 column tiles");
    return GCGE_EINVAL;
  }
  double *ws = nullptr;
  const int s = scratch_address(&ws);
  if (s != GCGE_OK) return s;
  return gcge::gram_f64_workspace(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, ws,
                                  (int64_t)GCGE_GRAM_NOALLOC_MAX_DOUBLES,
                                  reinterpret_cast<cudaStream_t>(stream));
}
