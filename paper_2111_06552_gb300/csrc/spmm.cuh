// CSR x row-major multivector products (MatDotMultiVec of Section 3.4) -- internal.
#pragma once
#include "common.cuh"

namespace gcge {

// Y = alpha * A X + beta * Y.  When `dot_out` is non-null the kernel also forms, per
// column j, sum_i X[i, j] * (A X)[i, j] into dot_out[j] (FP64): each CTA writes a
// partial row of `part` (at least dot_blocks x k doubles) and the last CTA, chosen by
// the atomic `ticket` (a zeroed unsigned, left zeroed), sums them in order.  Every sum
// runs in a fixed order, so the dots are bitwise reproducible for a given grid.
template <typename T>
int launch_spmm(int64_t n, const int32_t *rp, const int32_t *ci, const T *val, int k, T alpha,
                const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, double *dot_out,
                int dot_blocks, cudaStream_t st, double *part = nullptr,
                unsigned *ticket = nullptr);

// Upper bound on the CTAs launch_spmm uses for n rows and k columns (partial sizing).
int spmm_dot_blocks(int64_t n, int k);

}  // namespace gcge
