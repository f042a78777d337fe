// Tensor-core forms of the Gram and V C products for FP32 blocks.
#include "blas.cuh"

namespace gcge {

template <typename T>
int gram_tc(int64_t n, int m, int k, double alpha, const T *X, int64_t ldx, const T *Y,
            int64_t ldy, double beta, double *C, int64_t ldc, Scratch &ws, cudaStream_t st) {
  return gram<T>(n, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, 0, ws, st);
}

template <typename T>
int vc_tc(int64_t n, int d, int q, double alpha, const T *V, int64_t ldv, const double *C,
          int64_t ldc, double beta, T *Y, int64_t ldy, cudaStream_t st) {
  return vc<T>(n, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, 0, st);
}

template int gram_tc<float>(int64_t, int, int, double, const float *, int64_t, const float *,
                            int64_t, double, double *, int64_t, Scratch &, cudaStream_t);
template int gram_tc<double>(int64_t, int, int, double, const double *, int64_t, const double *,
                             int64_t, double, double *, int64_t, Scratch &, cudaStream_t);
template int vc_tc<float>(int64_t, int, int, double, const float *, int64_t, const double *,
                          int64_t, double, float *, int64_t, cudaStream_t);
template int vc_tc<double>(int64_t, int, int, double, const double *, int64_t, const double *,
                           int64_t, double, double *, int64_t, cudaStream_t);

}  // namespace gcge
