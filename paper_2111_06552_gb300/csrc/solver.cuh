// Solver handle and host driver of Algorithm 1 -- internal.
#pragma once
#include <atomic>
#include <vector>

#include "blas.cuh"
#include "cg.cuh"
#include "spmm.cuh"
#include "syev.cuh"

namespace gcge {

extern std::atomic<long long> g_launches;
void record_message(const char *msg);

// A CSR matrix resident on the device in FP64 and (when needed) FP32.
struct DevCsr {
  int64_t n = 0, nnz = 0;
  int32_t *rp = nullptr, *ci = nullptr;
  double *v64 = nullptr;
  float *v32 = nullptr;
  void free_all();
};

template <typename T>
inline const T *csr_vals(const DevCsr &m);
template <>
inline const double *csr_vals<double>(const DevCsr &m) { return m.v64; }
template <>
inline const float *csr_vals<float>(const DevCsr &m) { return m.v32; }

// B-orthonormalisation of a block through the C ABI (standalone buffers).
int borth_standalone(int64_t n, const int32_t *Brp, const int32_t *Bci, const double *Bval,
                     const double *Q, int64_t ldq, int q, double *W, int64_t ldw, int m, int leaf,
                     int orth, int *m_out, cudaStream_t st);

}  // namespace gcge

struct gcge_handle {
  cudaStream_t st = nullptr;
  int64_t n = 0;
  int nev = 0, bs = 0;
  double tol = 1e-8;
  gcge_options opt{};
  bool moving = false;
  int size_x = 0;
  gcge::DevCsr A, B;       // B.n == 0 means B = I
  // union pattern of A and B for the explicitly shifted S = A - theta B
  gcge::DevCsr S;
  int *mapA = nullptr, *mapB = nullptr, *isdiag = nullptr;
  double theta64 = -1.0, theta32 = -1.0;
  bool s64_valid = false, s32_valid = false;
  // results (FP64)
  double *store = nullptr;     // n x ld_store row-major, locked eigenvectors
  int64_t ld_store = 0;
  int store_cap = 0;
  std::vector<double> lam;     // locked eigenvalues in lock order
  int nconv = 0;
  bool solved = false;
  gcge_stats stats{};
  double max_abar_err = 0.0;
};
