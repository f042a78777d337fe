// CSR x row-major multivector products (MatDotMultiVec of Section 3.4) -- internal.
#pragma once
#include "common.cuh"

namespace gcge {

// Per-row group width: the smallest power of two >= k, capped at 32 lanes;
// each lane owns columns lane, lane + G, lane + 2G, ... (C of them).
struct SpmmShape {
  int G;   // lanes per row
  int C;   // columns per lane per pass
};

inline SpmmShape spmm_shape(int k) {
  int G = 1;
  while (G < k && G < 32) G <<= 1;
  int C = (k + G - 1) / G;
  if (C > 4) C = 4;   // wider blocks loop over column passes
  return {G, C};
}

// Y = alpha * A X + beta * Y.  When `dot_out` is non-null the kernel also
// accumulates, per column j, sum_i X[i, j] * (A X)[i, j] into
// dot_out[blockIdx.x * k + j] (one partial per block, FP64).
template <typename T>
int launch_spmm(int64_t n, const int32_t *rp, const int32_t *ci, const T *val, int k, T alpha,
                const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *dot_out,
                int dot_blocks, cudaStream_t st);

// Number of blocks launch_spmm uses when dot partials are requested (so the
// caller can size and reduce the partial buffer).
int spmm_dot_blocks(int64_t n, int k);

}  // namespace gcge
