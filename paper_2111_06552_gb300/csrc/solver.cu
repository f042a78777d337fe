// Host driver of the GCG iteration (Algorithm 1) on device-resident data.
//
// Everything of length n lives on the GPU; the host only reads back small
// scalars that steer the iteration (residual norms, kept-column counts,
// deflation sizes) and launches the kernels.  Per GCG iteration:
//
//   STEP 3  AW = A W; one Gram [X_a, P, W]^T (A W) written straight into the
//           last columns of the Rayleigh-Ritz matrix; the rest of Abar comes
//           from its structure, Eq. (struct_bar_A_new): Lambda on the X block,
//           alpha_0 = p^T Abar_old p^ on the P block, zero X-P coupling; FP64
//           Jacobi eigensolve on the device; X_new = V_a x^.
//   STEP 4  relative residuals of X_new's columns in order (chunks of 2 bs);
//           the converged prefix moves to the locked store (internal locking).
//   STEP 5  p~ from the Ritz block (Eq. CP_tilde), L2-orthogonalised against it
//           (Eq. Equality_Cpx) in small FP64 kernels; P_new = V_a p^.
//   STEP 6  theta = largest locked eigenvalue; S = A - theta B formed on the
//           union pattern; column-wise CG on S W = B X_n (Lambda_n - theta).
//   STEP 2  W deflated against [locked store, X_a, P] and Algorithm 3.
//   Moving  (Section 3.3) window of 3 bs X columns; after 2 bs locks all d Ritz
//           vectors are taken, the locked ones flushed, P = W = [].
//
// Storage: V[2] are n x ldV row-major double buffers holding [X_a | P | W]
// at a column offset; the next iteration's block is written into the other
// buffer and the two are swapped.  The locked vectors live in `store`.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "prof.cuh"
#include "solver.cuh"

namespace gcge {

void DevCsr::free_all() {
  cudaFree(rp);
  cudaFree(ci);
  cudaFree(v64);
  cudaFree(v32);
  rp = ci = nullptr;
  v64 = nullptr;
  v32 = nullptr;
  n = nnz = 0;
}

namespace {

// ------------------------------------------------------------------ small device kernels
// Keep the eigenpairs of a leaf Gram with lam > max(rel * max(lam), thr) (ascending order)
// and form C[:, t] = Q[:, idx_t] / sqrt(lam_t); out_i[0] = kept count,
// out_d[0] = max |lam_kept - 1|.  The relative part follows the rounding level of the
// computed Gram; the absolute floor catches a block whose columns all collapsed.
__global__ void leaf_coeffs_kernel(int len, const double *__restrict__ lam,
                                   const double *__restrict__ Q, int64_t ldq, double thr,
                                   double rel, double *__restrict__ C, int64_t ldc,
                                   int *__restrict__ out_i, double *__restrict__ out_d) {
  __shared__ int idx[1024];
  __shared__ int r;
  if (threadIdx.x == 0) {
    double lmax = 0.0;
    for (int i = 0; i < len; ++i) lmax = fmax(lmax, lam[i]);
    const double cut = fmax(rel * lmax, thr);
    int cnt = 0;
    double mx = 0.0;
    for (int i = 0; i < len; ++i) {
      if (lam[i] > cut) {
        idx[cnt++] = i;
        mx = fmax(mx, fabs(lam[i] - 1.0));
      }
    }
    r = cnt;
    out_i[0] = cnt;
    out_d[0] = mx;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < len * r; t += blockDim.x) {
    const int row = t % len, col = t / len;
    const int i = idx[col];
    C[row + (int64_t)col * ldc] = Q[row + (int64_t)i * ldq] / sqrt(lam[i]);
  }
}

// out = max_ij |R_ij| / sqrt(s2_j) (R col-major q x m; s2 = squared column B-norms).
__global__ void max_rel_kernel(int q, int m, const double *__restrict__ R, int64_t ldr,
                               const double *__restrict__ s2, double *__restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int64_t t = threadIdx.x; t < (int64_t)q * m; t += blockDim.x) {
    const int i = (int)(t % q), j = (int)(t / q);
    const double sj = fmax(sqrt(fmax(s2[j], 0.0)), 1e-300);
    mx = fmax(mx, fabs(R[i + (int64_t)j * ldr]) / sj);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// From squared norms s2[m]: keep columns with sqrt(s2) > thr; idx/scale lists; out count.
__global__ void keep_norms_kernel(int m, const double *__restrict__ s2, double thr,
                                  int *__restrict__ idx, double *__restrict__ scale,
                                  int *__restrict__ out_i) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < m; ++j) {
      const double s = sqrt(fmax(s2[j], 0.0));
      if (s > thr) {
        idx[cnt] = j;
        scale[cnt] = 1.0 / s;
        ++cnt;
      }
    }
    out_i[0] = cnt;
  }
}

template <typename T>
__global__ void gather_scale_kernel(int64_t n, int k, const int *__restrict__ idx,
                                    const double *__restrict__ sc, const T *__restrict__ X,
                                    int64_t ldx, T *__restrict__ Y, int64_t ldy) {
  const int64_t tot = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int j = (int)(t % k);
    Y[r * ldy + j] = (T)((double)X[r * ldx + idx[j]] * sc[j]);
  }
}

// x *= s (and bx *= s when bx is a separate column): one column of a row-major block.
template <typename T>
__global__ void scale_col_kernel(int64_t n, T *__restrict__ x, T *__restrict__ bx, int64_t ld,
                                 double s) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    x[r * ld] = (T)((double)x[r * ld] * s);
    if (bx) bx[r * ld] = (T)((double)bx[r * ld] * s);
  }
}

// Abar assembly from its structure (left part and mirror of the Gram block).
// Abar is d x d col-major (lda); columns [kp, d) hold G = V_a^T (A W) already.
__global__ void assemble_abar_kernel(int d, int kx, int np, const double *__restrict__ lam,
                                     const double *__restrict__ a0, int64_t lda0,
                                     double *__restrict__ Abar, int64_t lda) {
  const int kp = kx + np;
  const int64_t tot = (int64_t)d * kp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    double v;
    if (i < kp) {
      if (i < kx || j < kx)
        v = (i == j && i < kx) ? lam[i] : 0.0;
      else
        v = a0[(i - kx) + (int64_t)(j - kx) * lda0];
    } else {
      v = Abar[j + (int64_t)i * lda];   // mirror of the Gram block
    }
    Abar[i + (int64_t)j * lda] = v;
  }
}

// Symmetrise the square block [o, d) x [o, d): (a_ij + a_ji)/2.
__global__ void symmetrize_kernel(int d, int o, double *__restrict__ A, int64_t lda) {
  const int m = d - o;
  const int64_t tot = (int64_t)m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % m) + o, j = (int)(t / m) + o;
    if (i < j) {
      const double v = 0.5 * (A[i + (int64_t)j * lda] + A[j + (int64_t)i * lda]);
      A[i + (int64_t)j * lda] = v;
      A[j + (int64_t)i * lda] = v;
    }
  }
}

// dst (m x k, ldd) = src (m x k, lds) with rows [0, zr) set to zero (col-major).
__global__ void copy_zero_rows_kernel(int m, int k, const double *__restrict__ src, int64_t lds,
                                      int zr, double *__restrict__ dst, int64_t ldd) {
  const int64_t tot = (int64_t)m * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    dst[i + (int64_t)j * ldd] = i < zr ? 0.0 : src[i + (int64_t)j * lds];
  }
}

__global__ void copy_small_kernel(int m, int k, const double *__restrict__ src, int64_t lds,
                                  double *__restrict__ dst, int64_t ldd) {
  const int64_t tot = (int64_t)m * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    dst[i + (int64_t)j * ldd] = src[i + (int64_t)j * lds];
  }
}

// max_ij |A - B| over d x d (col-major), single block.
__global__ void max_diff_kernel(int d, const double *__restrict__ A, int64_t lda,
                                const double *__restrict__ B, int64_t ldb, int ident,
                                double *__restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0, nm = 0.0;
  for (int64_t t = threadIdx.x; t < (int64_t)d * d; t += blockDim.x) {
    const int i = (int)(t % d), j = (int)(t / d);
    const double a = A[i + (int64_t)j * lda];
    const double b = ident ? (i == j ? 1.0 : 0.0) : B[i + (int64_t)j * ldb];
    mx = fmax(mx, fabs(a - b));
    nm = fmax(nm, fabs(b));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
  __syncthreads();
  red[threadIdx.x] = nm;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[1] = red[0];
}

int small_grid(int64_t tot) {
  int64_t g = (tot + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------------ thresholds
// The paper's "small enough" / "close to zero" tests (Sections 3.1, 3.2) with the
// readings taken: relative deflation size, drop level after unit B-norm scaling,
// leaf repeat until max|Lambda - 1| small, P-construction drop.
struct Thresholds {
  double defl_tol, drop_tol, leaf_tol, leaf_drop, inner_tol, p_drop, leaf_rel;
  int defl_max, leaf_max, inner_max;
};

template <typename T>
Thresholds thresholds();
template <>
Thresholds thresholds<double>() {
  return {1e-12, 1e-13, 1e-12, 1e-20, 1e-12, 1e-10, 1e-14, 3, 3, 3};
}
template <>
Thresholds thresholds<float>() {
  return {1e-5, 1e-4, 1e-5, 1e-8, 1e-5, 1e-5, 1e-6, 3, 3, 3};
}

struct QPart {
  const void *ptr;
  int64_t ld;
  int cols;
};

// Per-step event timer.
struct StepTimer {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double ms = 0.0;
  bool open = false;
  void init() {
    if (!ev[0]) {
      cudaEventCreate(&ev[0]);
      cudaEventCreate(&ev[1]);
    }
  }
  void destroy() {
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    ev[0] = ev[1] = nullptr;
  }
};

}  // namespace

// ====================================================================== engine
template <typename T>
class Engine {
 public:
  Engine(gcge_handle *h, double tol, int max_iter) : h_(h), tol_(tol), max_iter_(max_iter) {
    th_ = thresholds<T>();
    st_ = h->st;
    bI_ = (h->B.n == 0);
  }
  ~Engine() { free_all(); }

  int setup(int size_x, int nev, int store_cap, int bs = 0);
  // Start block: device FP64 (X0d) or FP32 (X0f) n x size_x; both null = generator.
  int run(const double *X0d, int64_t ld0, const float *X0f, int64_t ld0f);
  // STEP 2 on a caller block (the C ABI's standalone orthogonalisation).
  int borth_api(double *W, int64_t ldw, int m, const double *Q, int64_t ldq, int q, int *m_out);

  int iterations() const { return it_; }
  int nlock() const { return nlock_; }
  const T *store() const { return store_; }
  int64_t ld_store() const { return ldS_; }
  const std::vector<double> &locked_lam() const { return lam_lock_; }
  const T *xa() const { return V_[cur_] + off_; }   // unlocked Ritz block of the last iteration
  int64_t ldv() const { return ldV_; }
  int kx() const { return kx_; }
  bool converged() const { return done_; }

  int64_t cg_steps = 0;
  int moves = 0;
  int refills = 0;                 // reservoir vectors that joined the basis beside W
  double ms_step[7] = {0, 0, 0, 0, 0, 0, 0};
  double ms_syev = 0.0;
  double max_orth = 0.0, max_abar = 0.0;
  bool checks = false;
  bool stagnated = false;
  int stagnation_limit = 0;   // > 0: stop after this many iterations without a new lock
                              // or progress of the first unconverged column (a 10% gain
                              // on its best residual, or a falling Ritz value)
  KProf *prof = nullptr;      // per-kernel-class event profile (null: off)
  bool cg_fp32 = false;       // FP64 engine: run the inner CG in FP32 on the FP64 residual
  bool use_p = true;          // build P (STEP 5); the refinement phase may go without it
  bool allow_move = true;     // moving mechanism when the handle asks for it
  // Reservoir of start vectors (FP32, n x nres, ascending): the X window is filled from
  // its first columns and, as pairs lock, refilled from the next ones, which enter the
  // iteration beside W (so their rows of Abar come from the Gram product).
  // set before setup() when a reservoir will be given: W then holds up to
  // max(sizeX, 2 blockSize) columns and A W is sized for that
  bool reservoir_planned = false;
  // FP64 engine: keep the locked vectors in the handle's store (no second n x nev copy)
  bool share_store = false;
  void set_reservoir(const float *Z, int64_t ldz, int nz) {
    res_ = reservoir_planned ? Z : nullptr;
    ldres_ = ldz;
    nres_ = nz;
  }

 private:
  gcge_handle *h_;
  double tol_;
  int max_iter_;
  Thresholds th_;
  cudaStream_t st_;
  bool bI_;
  int64_t n_ = 0;
  int nev_ = 0, bs_ = 0, sizeX_ = 0, dmax_ = 0;
  // n-sized buffers (row-major)
  T *V_[2] = {nullptr, nullptr};   // [X_a | P | W] double buffer, ldV_
  int64_t ldV_ = 0;
  int cur_ = 0;
  T *store_ = nullptr;             // locked vectors, ldS_
  bool store_shared_ = false;      // store_ is the handle's FP64 store (not freed here)
  int64_t ldS_ = 0;
  int store_cap_ = 0;
  T *AW_ = nullptr;                // A W, ldAW_ (W may hold reservoir vectors beside blockSize)
  int64_t ldAW_ = 0;
  T *R0_ = nullptr;                // CG initial residual, ldB_
  int64_t ldB_ = 0;
  T *BWb_ = nullptr, *TMP_ = nullptr, *TMP2_ = nullptr;   // ldW_
  int64_t ldW_ = 0;
  T *AXc_ = nullptr, *BXc_ = nullptr;                     // residual chunks, ldC_
  int64_t ldC_ = 0;
  T *Sval_ = nullptr;              // values of S = A - theta B on the union pattern
  double theta_cur_ = -1.0;
  // small FP64 device buffers
  double *Abar_ = nullptr, *Asave_ = nullptr, *Qe_ = nullptr;   // dmax x dmax
  double *ph_ = nullptr, *t1_ = nullptr, *t2_ = nullptr;        // dmax x dmax scratch
  double *theta_ = nullptr, *lam_ = nullptr;                    // dmax
  double *a0_ = nullptr;                                        // bs x bs (ld bs)
  double *Rg_ = nullptr;                                        // Gram results, ldR_ x ldW_
  int64_t ldR_ = 0;
  int kLeaf = 64;                                               // leaf / small Gram capacity (ld)
  double *Ms_ = nullptr, *Ml_ = nullptr, *Mq_ = nullptr, *Mc_ = nullptr;
  double *d_norm2_ = nullptr, *d_scale_ = nullptr;              // ldW_
  double *d_res_ = nullptr;                                     // 2 ldC_
  double *d_crit_ = nullptr;                                    // 4
  double *d_lamn_ = nullptr, *d_m1_ = nullptr;                  // ldB_
  int *d_idx_ = nullptr;                                        // ldW_
  int *d_cnt_ = nullptr;                                        // 4
  double *h_d_ = nullptr;                                       // pinned, 2 ldC_ + 8
  int *h_i_ = nullptr;                                          // pinned, ldB_ + 8
  Scratch ws_;
  SyevWork sw_;
  CgWork<T> cg_;
  CgWork<float> cg32_;
  float *Sval32_ = nullptr, *R032_ = nullptr, *D32_ = nullptr;   // FP32 inner-CG buffers
  T *Minv_ = nullptr;              // Jacobi preconditioner 1 / |diag(S)| (option precond)
  float *Minv32_ = nullptr;
  double theta32_cur_ = -1.0;
  // iteration state
  int off_ = 0, kx_ = 0, np_ = 0, nw_ = 0, nb_old_ = 0, lw_ = 0;
  int nlock_ = 0, it_ = 0;
  int kgrow_ = 0;                  // extra Ritz vectors the next RR keeps (window refill)
  double first_res_ = 0.0;         // residual of the first unconverged column (STEP 4)
  const float *res_ = nullptr;
  int64_t ldres_ = 0;
  int nres_ = 0, res_next_ = 0;
  bool done_ = false;
  std::vector<double> lam_lock_, lam_h_;
  StepTimer tm_;

  int alloc_dev(void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      record_cuda_error(e, __FILE__, __LINE__);
      *p = nullptr;
      return GCGE_ENOMEM;
    }
    return GCGE_OK;
  }
  void free_all();
  int sync() {
    GCGE_CUDA(cudaStreamSynchronize(st_));
    return GCGE_OK;
  }
  int read_d(const double *d, double *hst, int cnt) {
    GCGE_CUDA(cudaMemcpyAsync(hst, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st_));
    return sync();
  }
  int read_i(const int *d, int *hst, int cnt) {
    GCGE_CUDA(cudaMemcpyAsync(hst, d, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st_));
    return sync();
  }
  double spmm_bytes(const DevCsr &M, int k) const {
    return M.nnz * (sizeof(T) + 4.0) + 4.0 * (M.n + 1) + 2.0 * (double)n_ * k * sizeof(T);
  }
  int spA(const T *X, int64_t ldx, int k, T *Y, int64_t ldy) {
    g_launches += 1;
    ProfScope ps(prof, cls(GCGE_K_SPMM), spmm_bytes(h_->A, k), 2.0 * h_->A.nnz * k);
    return launch_spmm<T>(n_, h_->A.rp, h_->A.ci, csr_vals<T>(h_->A), k, T(1), X, ldx, T(0), Y,
                          ldy, nullptr, 0, st_);
  }
  int spB(const T *X, int64_t ldx, int k, T *Y, int64_t ldy) {
    g_launches += 1;
    if (bI_) return copyT(k, X, ldx, Y, ldy);
    ProfScope ps(prof, cls(GCGE_K_SPMM), spmm_bytes(h_->B, k), 2.0 * h_->B.nnz * k);
    return launch_spmm<T>(n_, h_->B.rp, h_->B.ci, csr_vals<T>(h_->B), k, T(1), X, ldx, T(0), Y,
                          ldy, nullptr, 0, st_);
  }
  int use_tc() const;
  // profile class of an FP32 kernel kind, or its FP64 counterpart in the FP64 engine
  static int cls(int c) {
    if (sizeof(T) == 4) return c;
    return c == GCGE_K_SPMM ? GCGE_K_SPMM64 : c == GCGE_K_GRAM ? GCGE_K_GRAM64 : GCGE_K_VC64;
  }
  // FP64 products of at least this size run on the bf16 tensor cores from exact digit
  // slices (oz.cu); smaller ones cost less in the FP64 kernels than their slicing.  A V C
  // product pads its reduction width d to a 128-entry window, so it needs d >= 32.
  bool emulate(int64_t a, int64_t b) const {
    return sizeof(T) == 8 && h_->opt.fp64_emulation && n_ >= 16384 && a * b >= 512 && a >= 8 &&
           b >= 8;
  }
  int gramT(int m, int k, double alpha, const T *X, int64_t ldx, const T *Y, int64_t ldy,
            double beta, double *C, int64_t ldc) {
    if (emulate(m, k)) {
      g_launches += 5;
      ProfScope ps(prof, GCGE_K_GRAM64TC, (double)n_ * (m + k) * sizeof(T), 2.0 * n_ * m * k);
      return oz_gram(n_, m, k, alpha, (const double *)X, ldx, (const double *)Y, ldy, beta, C,
                     ldc, ws_, st_);
    }
    g_launches += 2;
    ProfScope ps(prof, cls(GCGE_K_GRAM), (double)n_ * (m + k) * sizeof(T), 2.0 * n_ * m * k);
    return gram<T>(n_, m, k, alpha, X, ldx, Y, ldy, beta, C, ldc, use_tc(), ws_, st_);
  }
  int vcT(int d, int q, double alpha, const T *V, int64_t ldv, const double *C, int64_t ldc,
          double beta, T *Y, int64_t ldy) {
    const double vbytes = (double)n_ * (d + (beta != 0.0 ? 2 : 1) * q) * sizeof(T);
    if (d >= 32 && emulate(d, q)) {
      g_launches += 3;
      ProfScope ps(prof, GCGE_K_VC64TC, vbytes, 2.0 * n_ * d * q);
      return oz_vc(n_, d, q, alpha, (const double *)V, ldv, C, ldc, beta, (double *)Y, ldy, ws_,
                   st_);
    }
    g_launches += 1;
    ProfScope ps(prof, cls(GCGE_K_VC), vbytes, 2.0 * n_ * d * q);
    // reduction widths up to 32 (Algorithm 3 leaves, short deflations) stream faster
    // through the SIMT kernel than through the tensor-core pipeline
    return vc<T>(n_, d, q, alpha, V, ldv, C, ldc, beta, Y, ldy, use_tc() && d > 32, st_, &ws_);
  }
  int copyT(int k, const T *X, int64_t ldx, T *Y, int64_t ldy) {
    g_launches += 1;
    ProfScope ps(prof, GCGE_K_OTHER, 2.0 * n_ * k * sizeof(T), 0.0);
    return copy_cols<T, T>(n_, k, X, ldx, Y, ldy, nullptr, st_);
  }
  // fp32: a matrix of order <= 32 formed from FP32 blocks, diagonalised in FP32
  int syev_small(int d, double *A, int64_t lda, double *w, double *Q, int64_t ldq,
                 bool fp32 = false) {
    // (the Algorithm 3 leaves are of order <= 16: fp32 selects FP32 rotations)
    g_launches += 2;
    ProfScope ps(prof, GCGE_K_SYEV, 0.0, 0.0);
    return syev(d, A, lda, w, Q, ldq, sw_, nullptr, st_, fp32);
  }
  int borth(T *W, int m, const QPart *parts, int nparts, int *m_out);
  int normalize_drop(T *W, T *BW, int64_t ld, int m, double thr, int *m_out);
  int rec(T *W, T *BW, int64_t ld, int len, int c, int *out);
  int leaf(T *W, T *BW, int64_t ld, int len, int *out);
  int alg2(T *W, T *BW, int64_t ld, int m, int *out);
  int mgs_block(T *W, T *BW, int64_t ld, int m, int *out);
  int rayleigh_ritz(bool first, int d);
  int convergence(const T *X, int *c_out, int *chunk_start, int *chunk_len);
  int build_p(int d, int c, int bsn, int *np_out);
  int shifted_cg(const T *Xn, int64_t ldx, int bsn, const T *AXn, int64_t lda, const T *BXn,
                 int64_t ldb, double theta, T *Wout, int64_t ldw);
  void tic() { cudaEventRecord(tm_.ev[0], st_); }
  void toc(int step) {
    cudaEventRecord(tm_.ev[1], st_);
    cudaEventSynchronize(tm_.ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm_.ev[0], tm_.ev[1]);
    ms_step[step] += ms;
  }
};

template <>
int Engine<double>::use_tc() const { return 0; }
template <>
int Engine<float>::use_tc() const { return 1; }

template <typename T>
void Engine<T>::free_all() {
  if (st_) cudaStreamSynchronize(st_);
  if (store_shared_) store_ = nullptr;
  void *ptrs[] = {Sval32_, R032_, D32_, Minv_, Minv32_,
                  V_[0], V_[1], store_, AW_,   R0_,  BWb_,    TMP_,    TMP2_,  AXc_,  BXc_,
                  Sval_, Abar_, Asave_, Qe_,   ph_,  t1_,     t2_,     theta_, lam_,  a0_,
                  Rg_,   Ms_,   Ml_,    Mq_,   Mc_,  d_norm2_, d_scale_, d_res_, d_crit_,
                  d_lamn_, d_m1_, d_idx_, d_cnt_};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  V_[0] = V_[1] = store_ = AW_ = R0_ = BWb_ = TMP_ = TMP2_ = AXc_ = BXc_ = Sval_ = nullptr;
  Abar_ = Asave_ = Qe_ = ph_ = t1_ = t2_ = theta_ = lam_ = a0_ = Rg_ = nullptr;
  Ms_ = Ml_ = Mq_ = Mc_ = d_norm2_ = d_scale_ = d_res_ = d_crit_ = d_lamn_ = d_m1_ = nullptr;
  d_idx_ = d_cnt_ = nullptr;
  Sval32_ = R032_ = D32_ = nullptr;
  Minv_ = nullptr;
  Minv32_ = nullptr;
  cg32_.free_all();
  if (h_d_) cudaFreeHost(h_d_);
  if (h_i_) cudaFreeHost(h_i_);
  h_d_ = nullptr;
  h_i_ = nullptr;
  ws_.release(st_);
  sw_.free_all();
  cg_.free_all();
  tm_.destroy();
}

template <typename T>
int Engine<T>::setup(int size_x, int nev, int store_cap, int bs) {
  n_ = h_->n;
  nev_ = nev;
  bs_ = bs > 0 ? bs : h_->bs;
  sizeX_ = size_x;
  dmax_ = sizeX_ + 2 * bs_;
  ldV_ = round_up(dmax_, 4);
  store_cap_ = std::max(store_cap, 1);
  ldS_ = round_up(store_cap_, 4);
  ldB_ = round_up(bs_, 4);
  ldAW_ = reservoir_planned ? round_up(std::max(sizeX_, 2 * bs_), 4) : ldB_;
  ldW_ = round_up(std::max(sizeX_, 2 * bs_), 4);
  ldC_ = round_up(2 * bs_, 4);
  ldR_ = ldS_ + ldV_;
  const size_t ts = sizeof(T);
  const size_t n = (size_t)n_;
  GCGE_CHECK(alloc_dev((void **)&V_[0], ts * n * ldV_));
  GCGE_CHECK(alloc_dev((void **)&V_[1], ts * n * ldV_));
  if (sizeof(T) == 8 && share_store && h_->store && h_->ld_store == ldS_ &&
      h_->store_cap >= store_cap_) {
    store_ = reinterpret_cast<T *>(h_->store);   // the FP64 engine locks straight into it
    store_shared_ = true;
  } else {
    GCGE_CHECK(alloc_dev((void **)&store_, ts * n * ldS_));
  }
  GCGE_CHECK(alloc_dev((void **)&AW_, ts * n * ldAW_));
  GCGE_CHECK(alloc_dev((void **)&R0_, ts * n * ldB_));
  GCGE_CHECK(alloc_dev((void **)&BWb_, ts * n * ldW_));
  GCGE_CHECK(alloc_dev((void **)&TMP_, ts * n * ldW_));
  GCGE_CHECK(alloc_dev((void **)&TMP2_, ts * n * ldW_));
  GCGE_CHECK(alloc_dev((void **)&AXc_, ts * n * ldC_));
  GCGE_CHECK(alloc_dev((void **)&BXc_, ts * n * ldC_));
  GCGE_CHECK(alloc_dev((void **)&Sval_, ts * (size_t)h_->S.nnz));
  const size_t dd = (size_t)dmax_ * dmax_;
  GCGE_CHECK(alloc_dev((void **)&Abar_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&Asave_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&Qe_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&ph_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&t1_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&t2_, sizeof(double) * dd));
  GCGE_CHECK(alloc_dev((void **)&theta_, sizeof(double) * dmax_));
  GCGE_CHECK(alloc_dev((void **)&lam_, sizeof(double) * dmax_));
  GCGE_CHECK(alloc_dev((void **)&a0_, sizeof(double) * (size_t)bs_ * bs_));
  GCGE_CHECK(alloc_dev((void **)&Rg_, sizeof(double) * (size_t)ldR_ * ldW_));
  kLeaf = std::max(64, std::max(bs_, std::min(h_->opt.orth_leaf, 1024)));
  GCGE_CHECK(alloc_dev((void **)&Ms_, sizeof(double) * kLeaf * kLeaf));
  GCGE_CHECK(alloc_dev((void **)&Ml_, sizeof(double) * kLeaf));
  GCGE_CHECK(alloc_dev((void **)&Mq_, sizeof(double) * kLeaf * kLeaf));
  GCGE_CHECK(alloc_dev((void **)&Mc_, sizeof(double) * kLeaf * kLeaf));
  GCGE_CHECK(alloc_dev((void **)&d_norm2_, sizeof(double) * ldW_));
  GCGE_CHECK(alloc_dev((void **)&d_scale_, sizeof(double) * ldW_));
  GCGE_CHECK(alloc_dev((void **)&d_res_, sizeof(double) * 2 * ldC_));
  GCGE_CHECK(alloc_dev((void **)&d_crit_, sizeof(double) * 4));
  GCGE_CHECK(alloc_dev((void **)&d_lamn_, sizeof(double) * ldB_));
  GCGE_CHECK(alloc_dev((void **)&d_m1_, sizeof(double) * ldB_));
  GCGE_CHECK(alloc_dev((void **)&d_idx_, sizeof(int) * ldW_));
  GCGE_CHECK(alloc_dev((void **)&d_cnt_, sizeof(int) * 4));
  GCGE_CUDA(cudaMallocHost(&h_d_, sizeof(double) * (2 * ldC_ + 8)));
  GCGE_CUDA(cudaMallocHost(&h_i_, sizeof(int) * (ldB_ + 8)));
  GCGE_CHECK(sw_.alloc(std::max(dmax_, kLeaf)));
  if (h_->opt.precond == GCGE_PRECOND_JACOBI) {
    if (cg_fp32 && sizeof(T) == 8)
      GCGE_CHECK(alloc_dev((void **)&Minv32_, sizeof(float) * n));
    else
      GCGE_CHECK(alloc_dev((void **)&Minv_, ts * n));
  }
  if (cg_fp32 && sizeof(T) == 8) {
    GCGE_CHECK(alloc_dev((void **)&Sval32_, sizeof(float) * (size_t)h_->S.nnz));
    GCGE_CHECK(alloc_dev((void **)&R032_, sizeof(float) * n * ldB_));
    GCGE_CHECK(alloc_dev((void **)&D32_, sizeof(float) * n * ldB_));
    GCGE_CHECK(cg32_.alloc(n_, bs_));
  } else {
    GCGE_CHECK(cg_.alloc(n_, bs_));
  }
  tm_.init();
  std::vector<double> m1(ldB_, -1.0);
  GCGE_CUDA(cudaMemcpyAsync(d_m1_, m1.data(), sizeof(double) * ldB_, cudaMemcpyHostToDevice, st_));
  return sync();
}

// ---------------------------------------------------------------- orthogonalisation
// Scale columns to unit B-norm and drop those with B-norm <= thr (compacting left).
template <typename T>
int Engine<T>::normalize_drop(T *W, T *BW, int64_t ld, int m, double thr, int *m_out) {
  if (m == 0) {
    *m_out = 0;
    return GCGE_OK;
  }
  g_launches += 3;
  GCGE_CHECK(col_dots<T>(n_, m, W, ld, BW, ld, d_norm2_, ws_, st_));
  keep_norms_kernel<<<1, 32, 0, st_>>>(m, d_norm2_, thr, d_idx_, d_scale_, d_cnt_);
  GCGE_LAUNCH_CHECK();
  GCGE_CHECK(read_i(d_cnt_, h_i_, 1));
  const int r = h_i_[0];
  if (r > 0) {
    g_launches += 1;
    gather_scale_kernel<T><<<small_grid(n_ * r), 256, 0, st_>>>(n_, r, d_idx_, d_scale_, W, ld,
                                                                TMP_, ldW_);
    GCGE_LAUNCH_CHECK();
    GCGE_CHECK(copyT(r, TMP_, ldW_, W, ld));
    if (!bI_) {
      g_launches += 1;
      gather_scale_kernel<T><<<small_grid(n_ * r), 256, 0, st_>>>(n_, r, d_idx_, d_scale_, BW,
                                                                  ld, TMP_, ldW_);
      GCGE_LAUNCH_CHECK();
      GCGE_CHECK(copyT(r, TMP_, ldW_, BW, ld));
    }
  }
  *m_out = r;
  return GCGE_OK;
}

// Leaf of Algorithm 3: M = W^T B W = Q Lambda Q^T, W <- W Q Lambda^{-1/2}, repeated
// until Lambda ~ I; eigenvalues <= leaf_drop mark dependent directions (removed).
template <typename T>
int Engine<T>::leaf(T *W, T *BW, int64_t ld, int len, int *out) {
  for (int rep = 0; rep < th_.leaf_max && len > 0; ++rep) {
    GCGE_CHECK(gramT(len, len, 1.0, W, ld, BW, ld, 0.0, Ms_, kLeaf));
    symmetrize_kernel<<<1, 256, 0, st_>>>(len, 0, Ms_, kLeaf);
    GCGE_LAUNCH_CHECK();
    // the FP32 engine's leaf Gram comes from FP32 blocks and its drop and repeat tests
    // are at FP32 level: FP32 rotations suffice
    GCGE_CHECK(syev_small(len, Ms_, kLeaf, Ml_, Mq_, kLeaf, sizeof(T) == 4));
    leaf_coeffs_kernel<<<1, 256, 0, st_>>>(len, Ml_, Mq_, kLeaf, th_.leaf_drop, th_.leaf_rel, Mc_,
                                           kLeaf, d_cnt_, d_crit_);
    GCGE_LAUNCH_CHECK();
    g_launches += 2;
    GCGE_CUDA(cudaMemcpyAsync(h_i_, d_cnt_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    GCGE_CHECK(read_d(d_crit_, h_d_, 1));
    const int r = h_i_[0];
    const double dev = h_d_[0];
    if (r > 0) {
      GCGE_CHECK(vcT(len, r, 1.0, W, ld, Mc_, kLeaf, 0.0, TMP_, ldW_));
      GCGE_CHECK(copyT(r, TMP_, ldW_, W, ld));
      if (!bI_) {
        GCGE_CHECK(vcT(len, r, 1.0, BW, ld, Mc_, kLeaf, 0.0, TMP_, ldW_));
        GCGE_CHECK(copyT(r, TMP_, ldW_, BW, ld));
      }
    }
    len = r;
    if (r > 0 && dev <= th_.leaf_tol) break;
  }
  *out = len;
  return GCGE_OK;
}

// Algorithm 3 (RecursiveOrthSVD) on columns [0, len) of W (BW alongside); the kept
// columns end up compacted at [0, *out).
template <typename T>
int Engine<T>::rec(T *W, T *BW, int64_t ld, int len, int c, int *out) {
  if (len == 0) {
    *out = 0;
    return GCGE_OK;
  }
  if (len <= c) return leaf(W, BW, ld, len, out);
  const int h = len / 2;
  int L = 0;
  GCGE_CHECK(rec(W, BW, ld, h, c, &L));
  T *WR = W + h;
  T *BWR = BW + h;
  const int Rl = len - h;
  if (L > 0) {
    for (int rep = 0; rep < th_.inner_max; ++rep) {
      // R = (B X_left)^T X_right, X_right -= X_left R, repeated until R is small
      GCGE_CHECK(gramT(L, Rl, 1.0, BW, ld, WR, ld, 0.0, Rg_, ldR_));
      g_launches += 3;
      GCGE_CHECK(col_dots<T>(n_, Rl, WR, ld, BWR, ld, d_norm2_, ws_, st_));
      max_rel_kernel<<<1, 256, 0, st_>>>(L, Rl, Rg_, ldR_, d_norm2_, d_crit_);
      GCGE_LAUNCH_CHECK();
      GCGE_CHECK(vcT(L, Rl, -1.0, W, ld, Rg_, ldR_, 1.0, WR, ld));
      if (!bI_) GCGE_CHECK(vcT(L, Rl, -1.0, BW, ld, Rg_, ldR_, 1.0, BWR, ld));
      GCGE_CHECK(read_d(d_crit_, h_d_, 1));
      if (h_d_[0] <= th_.inner_tol) break;
    }
  }
  int R = 0;
  GCGE_CHECK(rec(WR, BWR, ld, Rl, c, &R));
  if (R > 0 && L < h) {   // close the gap left by dropped columns
    GCGE_CHECK(copyT(R, WR, ld, TMP_, ldW_));
    GCGE_CHECK(copyT(R, TMP_, ldW_, W + L, ld));
    if (!bI_) {
      GCGE_CHECK(copyT(R, BWR, ld, TMP_, ldW_));
      GCGE_CHECK(copyT(R, TMP_, ldW_, BW + L, ld));
    }
  }
  *out = L + R;
  return GCGE_OK;
}

// STEP 2 for a block W (n x m at ld = ldW_, in place): unit B-norm columns, deflation
// against the B-orthonormal parts (repeated while relatively large), drop of dependent
// columns, then Algorithm 3.  BW lives in BWb_ (or is W itself when B = I).
template <typename T>
int Engine<T>::borth(T *W, int m, const QPart *parts, int nparts, int *m_out) {
  const int64_t ld = ldW_;
  T *BW = bI_ ? W : BWb_;
  if (m == 0) {
    *m_out = 0;
    return GCGE_OK;
  }
  if (!bI_) GCGE_CHECK(spB(W, ld, m, BW, ld));
  int mm = 0;
  GCGE_CHECK(normalize_drop(W, BW, ld, m, 1e-300, &mm));
  m = mm;
  int qtot = 0;
  for (int p = 0; p < nparts; ++p) qtot += parts[p].cols;
  if (qtot > 0 && m > 0) {
    for (int pass = 0; pass < th_.defl_max; ++pass) {
      int row = 0;
      for (int p = 0; p < nparts; ++p) {
        if (parts[p].cols == 0) continue;
        GCGE_CHECK(gramT(parts[p].cols, m, 1.0, (const T *)parts[p].ptr, parts[p].ld, BW, ld, 0.0,
                         Rg_ + row, ldR_));
        row += parts[p].cols;
      }
      g_launches += 3;
      GCGE_CHECK(col_dots<T>(n_, m, W, ld, BW, ld, d_norm2_, ws_, st_));
      max_rel_kernel<<<1, 256, 0, st_>>>(qtot, m, Rg_, ldR_, d_norm2_, d_crit_);
      GCGE_LAUNCH_CHECK();
      row = 0;
      for (int p = 0; p < nparts; ++p) {
        if (parts[p].cols == 0) continue;
        GCGE_CHECK(vcT(parts[p].cols, m, -1.0, (const T *)parts[p].ptr, parts[p].ld, Rg_ + row,
                       ldR_, 1.0, W, ld));
        row += parts[p].cols;
      }
      if (!bI_) GCGE_CHECK(spB(W, ld, m, BW, ld));
      GCGE_CHECK(read_d(d_crit_, h_d_, 1));
      if (h_d_[0] <= th_.defl_tol) break;
    }
    GCGE_CHECK(normalize_drop(W, BW, ld, m, th_.drop_tol, &mm));
    m = mm;
  }
  int out = 0;
  if (h_->opt.orth == GCGE_ORTH_ALG2) {
    GCGE_CHECK(alg2(W, BW, ld, m, &out));
  } else {
    const int c = std::max(1, std::min(std::min(m, h_->opt.orth_leaf), std::min(kLeaf, 1024)));
    GCGE_CHECK(rec(W, BW, ld, m, c, &out));
  }
  *m_out = out;
  return GCGE_OK;
}

// Modified Gram-Schmidt inside one block of Algorithm 2, in the B inner product:
// column j is scaled to unit B-norm and removed from the later columns of the block
// at once.  A column whose B-norm fell to drop_tol (the block's columns started
// Algorithm 2 at unit B-norm) is dependent: the block's rearmost column takes its
// place (Section 3.1).  The pass repeats while the block's Gram differs from I by
// more than leaf_tol.  Each column costs a global reduction read by the host, as
// the paper counts for this method.
template <typename T>
int Engine<T>::mgs_block(T *W, T *BW, int64_t ld, int m, int *out) {
  int mm = m;
  for (int pass = 0; pass < th_.leaf_max && mm > 0; ++pass) {
    int j = 0;
    while (j < mm) {
      g_launches += 2;
      GCGE_CHECK(col_dots<T>(n_, 1, W + j, ld, BW + j, ld, d_norm2_, ws_, st_));
      GCGE_CHECK(read_d(d_norm2_, h_d_, 1));
      const double s = std::sqrt(std::max(h_d_[0], 0.0));
      if (!(s > th_.drop_tol)) {
        if (j < mm - 1) {
          GCGE_CHECK(copyT(1, W + mm - 1, ld, W + j, ld));
          if (!bI_) GCGE_CHECK(copyT(1, BW + mm - 1, ld, BW + j, ld));
        }
        --mm;
        continue;
      }
      g_launches += 1;
      scale_col_kernel<T><<<small_grid(n_), 256, 0, st_>>>(n_, W + j, bI_ ? nullptr : BW + j, ld,
                                                          1.0 / s);
      GCGE_LAUNCH_CHECK();
      const int q = mm - j - 1;
      if (q > 0) {   // r = (B x_j)^T X_later; X_later -= x_j r (and B X_later alike)
        GCGE_CHECK(gramT(1, q, 1.0, BW + j, ld, W + j + 1, ld, 0.0, Rg_, ldR_));
        GCGE_CHECK(vcT(1, q, -1.0, W + j, ld, Rg_, ldR_, 1.0, W + j + 1, ld));
        if (!bI_) GCGE_CHECK(vcT(1, q, -1.0, BW + j, ld, Rg_, ldR_, 1.0, BW + j + 1, ld));
      }
      ++j;
    }
    if (mm == 0) break;
    GCGE_CHECK(gramT(mm, mm, 1.0, W, ld, BW, ld, 0.0, t1_, dmax_));
    g_launches += 1;
    max_diff_kernel<<<1, 256, 0, st_>>>(mm, t1_, dmax_, nullptr, 0, 1, d_crit_);
    GCGE_LAUNCH_CHECK();
    GCGE_CHECK(read_d(d_crit_, h_d_, 1));
    if (h_d_[0] <= th_.leaf_tol) break;
  }
  *out = mm;
  return GCGE_OK;
}

// Algorithm 2 (modified block orthogonalisation, Section 3.1) on columns [0, m) of W
// (BW alongside), after the deflation against [X_c, X, P]: blocks of
// b = min(m/4, 200) columns; each block by modified Gram-Schmidt, then every later
// column deflated against it (R = (B X_k)^T X_later, X_later -= X_k R, repeated
// while R is relatively large).  Kept columns end up compacted at [0, *out).
template <typename T>
int Engine<T>::alg2(T *W, T *BW, int64_t ld, int m, int *out) {
  const int b = std::max(1, std::min(m / 4, 200));
  int pos = 0, mm = m;
  while (pos < mm) {
    const int bk = std::min(b, mm - pos);
    int r = 0;
    GCGE_CHECK(mgs_block(W + pos, BW + pos, ld, bk, &r));
    const int later0 = pos + bk, nlater = mm - later0;
    if (r < bk && nlater > 0) {   // dropped columns: the later ones move left
      GCGE_CHECK(copyT(nlater, W + later0, ld, TMP_, ldW_));
      GCGE_CHECK(copyT(nlater, TMP_, ldW_, W + pos + r, ld));
      if (!bI_) {
        GCGE_CHECK(copyT(nlater, BW + later0, ld, TMP_, ldW_));
        GCGE_CHECK(copyT(nlater, TMP_, ldW_, BW + pos + r, ld));
      }
    }
    mm -= bk - r;
    const int rs = pos + r, nr = mm - rs;
    if (r > 0 && nr > 0) {
      for (int rep = 0; rep < th_.inner_max; ++rep) {
        GCGE_CHECK(gramT(r, nr, 1.0, BW + pos, ld, W + rs, ld, 0.0, Rg_, ldR_));
        g_launches += 3;
        GCGE_CHECK(col_dots<T>(n_, nr, W + rs, ld, BW + rs, ld, d_norm2_, ws_, st_));
        max_rel_kernel<<<1, 256, 0, st_>>>(r, nr, Rg_, ldR_, d_norm2_, d_crit_);
        GCGE_LAUNCH_CHECK();
        GCGE_CHECK(vcT(r, nr, -1.0, W + pos, ld, Rg_, ldR_, 1.0, W + rs, ld));
        if (!bI_) GCGE_CHECK(vcT(r, nr, -1.0, BW + pos, ld, Rg_, ldR_, 1.0, BW + rs, ld));
        GCGE_CHECK(read_d(d_crit_, h_d_, 1));
        if (h_d_[0] <= th_.inner_tol) break;
      }
    }
    pos += r;
  }
  *out = mm;
  return GCGE_OK;
}

template <typename T>
int Engine<T>::borth_api(double *W, int64_t ldw, int m, const double *Q, int64_t ldq, int q,
                         int *m_out) {
  GCGE_CHECK(copy_cols<double, T>(n_, m, W, ldw, TMP2_, ldW_, nullptr, st_));
  QPart part{Q, ldq, q};
  int out = 0;
  GCGE_CHECK(borth(TMP2_, m, &part, Q ? 1 : 0, &out));
  if (out > 0) GCGE_CHECK(copy_cols<T, double>(n_, out, TMP2_, ldW_, W, ldw, nullptr, st_));
  *m_out = out;
  return sync();
}

// ---------------------------------------------------------------- STEP 3
template <typename T>
int Engine<T>::rayleigh_ritz(bool first, int d) {
  T *Va = V_[cur_] + off_;
  const int64_t lda = dmax_;
  T *scratchV = V_[1 - cur_];   // free until X_new is written there
  if (first) {
    // full Abar = V_a^T (A V_a)
    GCGE_CHECK(spA(Va, ldV_, d, scratchV, ldV_));
    GCGE_CHECK(gramT(d, d, 1.0, Va, ldV_, scratchV, ldV_, 0.0, Abar_, lda));
    symmetrize_kernel<<<small_grid((int64_t)d * d), 256, 0, st_>>>(d, 0, Abar_, lda);
    GCGE_LAUNCH_CHECK();
    g_launches += 1;
  } else {
    // structure of Eq. (struct_bar_A_new): only [X_a, P, W]^T (A W) is a large product
    const int kp = kx_ + np_;
    T *W = Va + kp;
    if (nw_ > ldAW_) {
      record_message("W is wider than its A W buffer");
      return GCGE_EINVAL;
    }
    GCGE_CHECK(spA(W, ldV_, nw_, AW_, ldAW_));
    GCGE_CHECK(gramT(d, nw_, 1.0, Va, ldV_, AW_, ldAW_, 0.0, Abar_ + (int64_t)kp * lda, lda));
    assemble_abar_kernel<<<small_grid((int64_t)d * kp), 256, 0, st_>>>(d, kx_, np_, lam_, a0_, bs_,
                                                                       Abar_, lda);
    GCGE_LAUNCH_CHECK();
    symmetrize_kernel<<<small_grid((int64_t)nw_ * nw_), 256, 0, st_>>>(d, kp, Abar_, lda);
    GCGE_LAUNCH_CHECK();
    g_launches += 2;
    if (checks) {   // the shortcut against the explicit V_a^T A V_a
      GCGE_CHECK(spA(Va, ldV_, d, scratchV, ldV_));
      GCGE_CHECK(gramT(d, d, 1.0, Va, ldV_, scratchV, ldV_, 0.0, t1_, lda));
      max_diff_kernel<<<1, 256, 0, st_>>>(d, Abar_, lda, t1_, lda, 0, d_crit_);
      GCGE_CHECK(read_d(d_crit_, h_d_, 2));
      max_abar = std::max(max_abar, h_d_[0] / std::max(h_d_[1], 1e-300));
    }
  }
  if (checks) {   // V_a^T B V_a = I
    GCGE_CHECK(spB(Va, ldV_, d, scratchV, ldV_));
    GCGE_CHECK(gramT(d, d, 1.0, Va, ldV_, scratchV, ldV_, 0.0, t1_, lda));
    max_diff_kernel<<<1, 256, 0, st_>>>(d, t1_, lda, nullptr, 0, 1, d_crit_);
    GCGE_CHECK(read_d(d_crit_, h_d_, 2));
    max_orth = std::max(max_orth, h_d_[0]);
  }
  copy_small_kernel<<<small_grid((int64_t)d * d), 256, 0, st_>>>(d, d, Abar_, lda, Asave_, lda);
  GCGE_LAUNCH_CHECK();
  g_launches += 3;
  auto t0 = std::chrono::steady_clock::now();
  int s;
  {
    ProfScope ps(prof, GCGE_K_SYEV, 0.0, 0.0);
    // the FP32 engine's Abar comes from FP32 products: refining its eigenvectors beyond
    // 1e-10 buys nothing
    s = syev(d, Abar_, lda, theta_, Qe_, lda, sw_, nullptr, st_, sizeof(T) == 4);
  }
  ms_syev += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

// ---------------------------------------------------------------- STEP 4
// X (kx_ columns, ldV_) checked in chunks of 2 bs; returns the converged prefix and the
// chunk [start, start + len) whose A X and B X are left in AXc_ / BXc_.
template <typename T>
int Engine<T>::convergence(const T *X, int *c_out, int *chunk_start, int *chunk_len) {
  const int chunk = (int)std::min<int64_t>(2 * bs_, ldC_);
  int c = 0, start = 0, m = 0, held = 0;   // held: first column of the chunk in AXc_
  while (start < kx_) {
    m = std::min(chunk, kx_ - start);
    held = start;
    GCGE_CHECK(spA(X + start, ldV_, m, AXc_, ldC_));
    if (!bI_) GCGE_CHECK(spB(X + start, ldV_, m, BXc_, ldC_));
    g_launches += 2;
    GCGE_CHECK(residual_parts<T>(n_, m, X + start, ldV_, AXc_, ldC_, bI_ ? nullptr : BXc_, ldC_,
                                 theta_ + start, d_res_, ws_, st_));
    GCGE_CHECK(read_d(d_res_, h_d_, 2 * m));
    bool stop = false;
    while (c < start + m) {
      const int j = c - start;
      const double lam = lam_h_[c];
      const double r = std::sqrt(std::max(h_d_[j], 0.0)) /
                       (std::fabs(lam) * std::sqrt(std::max(h_d_[m + j], 1e-300)));
      if (!(r < tol_)) {
        first_res_ = r;
        stop = true;
        break;
      }
      ++c;
    }
    if (stop) break;
    start += m;
  }
  *c_out = c;
  *chunk_start = held;
  *chunk_len = m;
  return GCGE_OK;
}

// ---------------------------------------------------------------- STEP 5 (small dense)
template <typename T>
int Engine<T>::build_p(int d, int c, int bsn, int *np_out) {
  const int64_t ld = dmax_;
  const int kx = kx_;
  // p~ = x^[:, c:c+bsn] with the rows of the previous active block zeroed (Eq. CP_tilde)
  copy_zero_rows_kernel<<<small_grid((int64_t)d * bsn), 256, 0, st_>>>(
      d, bsn, Qe_ + (int64_t)c * ld, ld, nb_old_, ph_, ld);
  GCGE_LAUNCH_CHECK();
  g_launches += 1;
  int r = bsn;
  for (int round = 0; round < 2 && r > 0; ++round) {
    for (int pj = 0; pj < 2; ++pj) {   // p~ -= x^ (x^T p~), twice
      GCGE_CHECK(dgemm_small('T', 'N', kx, r, d, 1.0, Qe_, ld, ph_, ld, 0.0, t1_, ld, st_));
      GCGE_CHECK(dgemm_small('N', 'N', d, r, kx, -1.0, Qe_, ld, t1_, ld, 1.0, ph_, ld, st_));
      g_launches += 2;
    }
    if (r > kLeaf) return GCGE_EINVAL;
    GCGE_CHECK(dgemm_small('T', 'N', r, r, d, 1.0, ph_, ld, ph_, ld, 0.0, Ms_, kLeaf, st_));
    symmetrize_kernel<<<1, 256, 0, st_>>>(r, 0, Ms_, kLeaf);
    GCGE_LAUNCH_CHECK();
    GCGE_CHECK(syev_small(r, Ms_, kLeaf, Ml_, Mq_, kLeaf));
    leaf_coeffs_kernel<<<1, 256, 0, st_>>>(r, Ml_, Mq_, kLeaf, th_.p_drop * th_.p_drop,
                                           th_.leaf_rel, Mc_, kLeaf, d_cnt_, d_crit_);
    GCGE_LAUNCH_CHECK();
    g_launches += 3;
    GCGE_CHECK(read_i(d_cnt_, h_i_, 1));
    const int r2 = h_i_[0];
    if (r2 > 0) {
      GCGE_CHECK(dgemm_small('N', 'N', d, r2, r, 1.0, ph_, ld, Mc_, kLeaf, 0.0, t2_, ld, st_));
      copy_small_kernel<<<small_grid((int64_t)d * r2), 256, 0, st_>>>(d, r2, t2_, ld, ph_, ld);
      GCGE_LAUNCH_CHECK();
      g_launches += 2;
    }
    r = r2;
  }
  if (r > 0) {   // alpha_0 = p^T Abar p^  (Eq. Equality_pp)
    GCGE_CHECK(dgemm_small('N', 'N', d, r, d, 1.0, Asave_, ld, ph_, ld, 0.0, t2_, ld, st_));
    GCGE_CHECK(dgemm_small('T', 'N', r, r, d, 1.0, ph_, ld, t2_, ld, 0.0, a0_, bs_, st_));
    symmetrize_kernel<<<1, 256, 0, st_>>>(r, 0, a0_, bs_);
    GCGE_LAUNCH_CHECK();
    g_launches += 3;
  }
  *np_out = r;
  return GCGE_OK;
}

// ---------------------------------------------------------------- STEP 6
template <typename T>
int Engine<T>::shifted_cg(const T *Xn, int64_t ldx, int bsn, const T *AXn, int64_t lda,
                          const T *BXn, int64_t ldb, double theta, T *Wout, int64_t ldw) {
  if (theta != theta_cur_) {   // S = A - theta B on the union pattern
    g_launches += 1;
    GCGE_CHECK(shifted_values<T>(h_->S.nnz, h_->mapA, h_->A.v64, bI_ ? nullptr : h_->mapB,
                                 bI_ ? nullptr : h_->B.v64, h_->isdiag, theta, Sval_, st_));
    if (Minv_) {
      g_launches += 1;
      GCGE_CHECK(jacobi_inverse<T>(n_, h_->S.rp, h_->S.ci, Sval_, Minv_, st_));
    }
    theta_cur_ = theta;
  }
  // initial guess x = X_n; initial residual r0 = (lambda - theta) B x - S x = lambda B x - A x
  GCGE_CHECK(copyT(bsn, Xn, ldx, Wout, ldw));
  g_launches += 1;
  GCGE_CHECK(axpby_cols<T>(n_, bsn, d_lamn_, BXn, ldb, d_m1_, AXn, lda, R0_, ldB_, st_));
  int64_t nl = 0;
  int mx;
  if (cg_fp32 && sizeof(T) == 8) {
    // inexact inner solve in FP32: S delta = r0 from delta = 0, then W = X_n + delta (FP64)
    if (theta != theta32_cur_) {
      g_launches += 1;
      GCGE_CHECK(shifted_values<float>(h_->S.nnz, h_->mapA, h_->A.v64, bI_ ? nullptr : h_->mapB,
                                       bI_ ? nullptr : h_->B.v64, h_->isdiag, theta, Sval32_,
                                       st_));
      if (Minv32_) {
        g_launches += 1;
        GCGE_CHECK(jacobi_inverse<float>(n_, h_->S.rp, h_->S.ci, Sval32_, Minv32_, st_));
      }
      theta32_cur_ = theta;
    }
    g_launches += 2;
    GCGE_CHECK(copy_cols<T, float>(n_, bsn, R0_, ldB_, R032_, ldB_, nullptr, st_));
    GCGE_CUDA(cudaMemsetAsync(D32_, 0, sizeof(float) * (size_t)n_ * ldB_, st_));
    mx = block_cg<float>(n_, h_->S.rp, h_->S.ci, Sval32_, bsn, nullptr, 0, R032_, ldB_, D32_,
                         ldB_, h_->opt.cg_max_iter, h_->opt.cg_rtol, cg32_, h_i_, &nl, st_, prof,
                         Minv32_);
    if (mx >= 0) {
      g_launches += 1;
      GCGE_CHECK(add_cols<float, T>(n_, bsn, D32_, ldB_, Wout, ldw, st_));
    }
  } else {
    mx = block_cg<T>(n_, h_->S.rp, h_->S.ci, Sval_, bsn, nullptr, 0, R0_, ldB_, Wout, ldw,
                     h_->opt.cg_max_iter, h_->opt.cg_rtol, cg_, h_i_, &nl, st_, prof, Minv_);
  }
  g_launches += nl;
  if (mx < 0) return mx;
  cg_steps += mx;
  return GCGE_OK;
}

// ---------------------------------------------------------------- the iteration
template <typename T>
int Engine<T>::run(const double *X0d, int64_t ld0, const float *X0f, int64_t ld0f) {
  cur_ = 0;
  off_ = 0;
  // ---- STEP 1: the start block, orthonormalised by Algorithm 3 (STEP 2 with P = W = [])
  tic();
  g_launches += 1;
  if (X0d)
    GCGE_CHECK(copy_cols<double, T>(n_, sizeX_, X0d, ld0, TMP2_, ldW_, nullptr, st_));
  else if (X0f)
    GCGE_CHECK(copy_cols<float, T>(n_, sizeX_, X0f, ld0f, TMP2_, ldW_, nullptr, st_));
  else
    GCGE_CHECK(random_block<T>(n_, sizeX_, h_->opt.seed, TMP2_, ldW_, st_));
  int m0 = 0;
  GCGE_CHECK(borth(TMP2_, sizeX_, nullptr, 0, &m0));
  if (m0 < sizeX_) {
    record_message("initial block is rank deficient");
    return GCGE_EBREAKDOWN;
  }
  GCGE_CHECK(copyT(sizeX_, TMP2_, ldW_, V_[cur_], ldV_));
  toc(1);
  kx_ = sizeX_;
  kgrow_ = 0;
  res_next_ = (res_ && X0f == res_) ? sizeX_ : 0;
  np_ = nw_ = 0;
  nb_old_ = 0;
  lw_ = 0;
  nlock_ = 0;
  it_ = 0;
  done_ = false;
  lam_lock_.clear();
  bool first = true;
  int since_lock = 0;            // iterations without a new lock and without progress
  int no_lock = 0;               // iterations without a new lock at all
  double best_res = 1e300;       // best residual of the first unconverged column
  double prev_lam = 1e300;       // its Ritz value in the previous iteration
  while (true) {
    ++it_;
    const int d = kx_ + np_ + nw_;
    const int nxt = 1 - cur_;
    T *Va = V_[cur_] + off_;
    // ---- STEP 3: Rayleigh-Ritz, X_new = V_a x^ into the other buffer
    tic();
    GCGE_CHECK(rayleigh_ritz(first, d));
    lam_h_.resize(d);
    GCGE_CHECK(read_d(theta_, lam_h_.data(), d));
    if (kgrow_ > 0) {   // reservoir vectors joined last iteration: the window grows back
      kx_ = std::min(kx_ + kgrow_, d);
      kgrow_ = 0;
    }
    GCGE_CHECK(vcT(d, kx_, 1.0, Va, ldV_, Qe_, dmax_, 0.0, V_[nxt], ldV_));
    toc(3);
    // ---- STEP 4: convergence, prefix locking into the store
    tic();
    int c = 0, cs = 0, cl = 0;
    first_res_ = 0.0;
    GCGE_CHECK(convergence(V_[nxt], &c, &cs, &cl));
    // with a reservoir the window is refilled from it; the moving mechanism takes over
    // once it is used up
    // (Section 3.3 moves after 2 blockSize new locks; the window is also moved when all
    // of its unlocked vectors converged, which would otherwise leave X empty)
    const bool reservoir_left = res_ && res_next_ < nres_;
    const bool move = allow_move && !reservoir_left && h_->moving && nlock_ + c < nev_ &&
                      ((lw_ + c) >= 2 * bs_ || c == kx_);
    if (c > 0) {
      if (nlock_ + c > store_cap_) {
        record_message("locked-vector store overflow");
        return GCGE_EINVAL;
      }
      GCGE_CHECK(copyT(c, V_[nxt], ldV_, store_ + nlock_, ldS_));
      for (int j = 0; j < c; ++j) lam_lock_.push_back(lam_h_[j]);
      nlock_ += c;
      since_lock = 0;
      no_lock = 0;
      best_res = 1e300;
      prev_lam = 1e300;
    } else {
      ++no_lock;
      // progress: the residual of the first unconverged column gains 10% on its best, or
      // its Ritz value still falls (the start block is far from the eigenvector)
      const double lam_first = (size_t)c < lam_h_.size() ? lam_h_[c] : 0.0;
      const bool falling = lam_first < prev_lam - 1e-6 * std::fabs(lam_first);
      if (first_res_ < 0.9 * best_res || falling) {
        best_res = std::min(best_res, first_res_);
        since_lock = 0;
      } else {
        ++since_lock;
      }
      prev_lam = lam_first;
    }
    toc(4);
    if (h_->opt.verbose)
      fprintf(stderr, "[gcge] it %4d d %4d nconv %5d first-unlocked %.12e theta %.6e%s\n", it_, d,
              nlock_, (size_t)c < lam_h_.size() ? lam_h_[c] : 0.0, theta_cur_, move ? " move" : "");
    // FP32 rounding can keep a Ritz value drifting below the eigenvalue, which reads as
    // progress: the phase also ends after 4 x stagnation_limit iterations without a lock
    const bool stalled = stagnation_limit > 0 &&
                         (since_lock >= stagnation_limit || no_lock >= 4 * stagnation_limit);
    const bool stop = nlock_ >= nev_ || it_ >= max_iter_ || stalled;
    if (stop) {
      done_ = nlock_ >= nev_;
      stagnated = !done_ && stalled;
      cur_ = nxt;
      off_ = c;
      kx_ -= c;
      break;
    }
    int xoff = c;        // column of the new unlocked X block in V[nxt]
    int kxn = kx_ - c;
    int npn = 0;
    tic();
    if (move) {
      // moving mechanism: all Ritz vectors of Abar, P and W folded into X; the window
      // keeps the lowest min(3 bs, d - c) unlocked ones at offset 0
      kxn = std::min(sizeX_, d - c);
      GCGE_CHECK(vcT(d, kxn, 1.0, Va, ldV_, Qe_ + (int64_t)c * dmax_, dmax_, 0.0, V_[nxt], ldV_));
      xoff = 0;
      lw_ = 0;
      ++moves;
    } else {
      lw_ += c;
    }
    const int bsn = std::min(std::min(bs_, nev_ - nlock_), kxn);
    // ---- STEP 5: P from the Ritz block (none right after a move or the first RR)
    if (use_p && !move && !first && nb_old_ > 0 && bsn > 0) {
      GCGE_CHECK(build_p(d, c, bsn, &npn));
      if (npn > 0) GCGE_CHECK(vcT(d, npn, 1.0, Va, ldV_, ph_, dmax_, 0.0, V_[nxt] + kx_, ldV_));
    }
    toc(5);
    // Ritz values of the new X block (device copy for the next Abar)
    GCGE_CUDA(cudaMemcpyAsync(lam_, lam_h_.data() + c, sizeof(double) * kxn,
                              cudaMemcpyHostToDevice, st_));
    GCGE_CUDA(cudaMemcpyAsync(d_lamn_, lam_h_.data() + c, sizeof(double) * bsn,
                              cudaMemcpyHostToDevice, st_));
    // ---- STEP 6: W from the shifted CG on the active block
    tic();
    double theta = 0.0;
    if (h_->opt.use_shift && !lam_lock_.empty())
      theta = *std::max_element(lam_lock_.begin(), lam_lock_.end());
    const T *Xn = V_[nxt] + xoff;
    const T *AXn = AXc_, *BXn = BXc_;
    int64_t ldbx = ldC_;
    if (c >= cs && c + bsn <= cs + cl) {
      AXn = AXc_ + (c - cs);
      BXn = BXc_ + (c - cs);
    } else {
      GCGE_CHECK(spA(Xn, ldV_, bsn, AXc_, ldC_));
      if (!bI_) GCGE_CHECK(spB(Xn, ldV_, bsn, BXc_, ldC_));
    }
    if (bI_) {
      BXn = Xn;
      ldbx = ldV_;
    }
    GCGE_CHECK(shifted_cg(Xn, ldV_, bsn, AXn, ldC_, BXn, ldbx, theta, TMP2_, ldW_));
    toc(6);
    // ---- STEP 2: W against [store, X_a, P], then Algorithm 3
    tic();
    int rres = 0;   // reservoir vectors that refill the window, orthogonalised with W
    if (res_ && res_next_ < nres_ && kxn < sizeX_) {
      rres = std::min(nres_ - res_next_, sizeX_ - kxn);
      rres = std::min(rres, (int)ldW_ - bsn);
      if (xoff > 0 && xoff + kxn + npn + bsn + rres > dmax_) {
        // the columns in front of X_a were locked (they are in the store): move
        // [X_a, P] to column 0 so that the refill fits behind W
        GCGE_CHECK(copyT(kxn, V_[nxt] + xoff, ldV_, TMP_, ldW_));
        GCGE_CHECK(copyT(kxn, TMP_, ldW_, V_[nxt], ldV_));
        if (npn > 0) {
          GCGE_CHECK(copyT(npn, V_[nxt] + xoff + kxn, ldV_, TMP_, ldW_));
          GCGE_CHECK(copyT(npn, TMP_, ldW_, V_[nxt] + kxn, ldV_));
        }
        xoff = 0;
      }
      // the next basis [X_a, P, W] starts at column xoff of V[nxt] and must end by dmax_
      rres = std::min(rres, dmax_ - (xoff + kxn + npn + bsn));
      rres = std::max(rres, 0);
      if (rres > 0) {
        g_launches += 1;
        GCGE_CHECK(copy_cols<float, T>(n_, rres, res_ + res_next_, ldres_, TMP2_ + bsn, ldW_,
                                       nullptr, st_));
        res_next_ += rres;
        refills += rres;
      }
    }
    QPart parts[2] = {{store_, ldS_, nlock_}, {V_[nxt] + xoff, ldV_, kxn + npn}};
    int nwn = 0;
    GCGE_CHECK(borth(TMP2_, bsn + rres, parts, 2, &nwn));
    kgrow_ = rres;
    if (xoff + kxn + npn + nwn > dmax_) {   // the next basis must fit the row width of V
      record_message("basis [X_a, P, W] wider than the basis buffer");
      return GCGE_EINVAL;
    }
    if (nwn > 0) GCGE_CHECK(copyT(nwn, TMP2_, ldW_, V_[nxt] + xoff + kxn + npn, ldV_));
    toc(2);
    if (prof) prof->harvest();
    if (kxn + npn + nwn == 0) {
      if (stagnation_limit > 0) {   // FP32 phase: the FP64 phase restarts from the store
        stagnated = true;
        kx_ = 0;
        break;
      }
      record_message("the search window holds no vector to iterate on");
      return GCGE_EBREAKDOWN;
    }
    cur_ = nxt;
    off_ = xoff;
    kx_ = kxn;
    np_ = npn;
    nw_ = nwn;
    nb_old_ = bsn;
    first = false;
  }
  return done_ ? GCGE_OK : GCGE_ENOTCONV;
}

template class Engine<double>;
template class Engine<float>;

// ---------------------------------------------------------------- standalone B-orth
int borth_standalone(int64_t n, const int32_t *Brp, const int32_t *Bci, const double *Bval,
                     const double *Q, int64_t ldq, int q, double *W, int64_t ldw, int m, int leaf,
                     int orth, int *m_out, cudaStream_t st) {
  gcge_handle h;
  h.st = st;
  h.n = n;
  h.bs = 1;
  gcge_options_default(&h.opt);
  h.opt.orth_leaf = leaf;
  h.opt.orth = orth;
  if (Brp) {
    h.B.n = n;
    h.B.rp = const_cast<int32_t *>(Brp);
    h.B.ci = const_cast<int32_t *>(Bci);
    h.B.v64 = const_cast<double *>(Bval);
  }
  int s = GCGE_OK;
  {
    Engine<double> e(&h, 1e-8, 1);
    s = e.setup(std::max(m, 1), 1, 1);
    if (s == GCGE_OK) s = e.borth_api(W, ldw, m, q > 0 ? Q : nullptr, ldq, q, m_out);
  }
  // the caller owns B's arrays
  h.B.rp = nullptr;
  h.B.ci = nullptr;
  h.B.v64 = nullptr;
  h.B.n = 0;
  return s;
}

}  // namespace gcge

namespace gcge {

namespace {
template <typename T>
void add_stats(gcge_handle *h, const Engine<T> &e) {
  for (int i = 0; i < 7; ++i) h->stats.ms_step[i] += e.ms_step[i];
  h->stats.ms_syev += e.ms_syev;
  h->stats.cg_steps += e.cg_steps;
  h->stats.moves += e.moves;
  h->stats.refills += e.refills;
  h->stats.max_orth_err = std::max(h->stats.max_orth_err, e.max_orth);
  h->stats.max_abar_err = std::max(h->stats.max_abar_err, e.max_abar);
  if (e.prof) {
    e.prof->harvest();
    for (int c = 0; c < GCGE_K_CLASSES; ++c) {
      h->stats.prof_ms[c] += e.prof->ms[c];
      h->stats.prof_calls[c] += e.prof->calls[c];
      h->stats.prof_bytes[c] += e.prof->bytes[c];
      h->stats.prof_flops[c] += e.prof->flops[c];
      e.prof->ms[c] = e.prof->bytes[c] = e.prof->flops[c] = 0.0;
      e.prof->calls[c] = 0;
    }
  }
}

template <typename T>
int export_store(gcge_handle *h, const Engine<T> &e) {
  const int k = std::min(e.nlock(), h->store_cap);
  if (k > 0 && (const void *)e.store() != (const void *)h->store)
    GCGE_CHECK(copy_cols<T, double>(h->n, k, e.store(), e.ld_store(), h->store, h->ld_store,
                                    nullptr, h->st));
  h->lam.assign(e.locked_lam().begin(), e.locked_lam().begin() + k);
  h->nconv = k;
  GCGE_CUDA(cudaStreamSynchronize(h->st));
  return GCGE_OK;
}
}  // namespace

// Plain FP64 path: every step in FP64.
int run_fp64(gcge_handle *h, const double *X0d, int64_t ld0, int *iters) {
  Engine<double> e(h, h->tol, h->opt.max_iter);
  e.checks = h->opt.checks != 0;
  e.share_store = true;
  KProf prof;
  prof.st = h->st;
  if (h->opt.profile) e.prof = &prof;
  GCGE_CHECK(e.setup(h->size_x, h->nev, h->store_cap));
  const int s = e.run(X0d, ld0, nullptr, 0);
  *iters = e.iterations();
  add_stats(h, e);
  if (s != GCGE_OK && s != GCGE_ENOTCONV) return s;
  int tc_err = 0;   // a tensor-core kernel whose bounded wait ran out leaves a flag
  GCGE_CHECK(tc_error_flag(&tc_err, h->st));
  if (tc_err) return GCGE_ETIMEOUT;
  GCGE_CHECK(export_store(h, e));
  return s;
}

// Mixed path: phase 1 runs the whole iteration on FP32 blocks (TF32 tensor-core
// Gram/update products, FP64 small dense work) until every wanted pair reaches
// mixed_switch_tol or no pair locks for 10 iterations; phase 2 restarts the FP64
// iteration from phase 1's vectors (locked ones first) to the requested tol.
int run_mixed(gcge_handle *h, const double *X0d, int64_t ld0, int *iters, int *iters32) {
  const int sx = h->size_x;
  KProf prof;
  prof.st = h->st;
  float *Z = nullptr;   // phase-1 vectors, ascending: locked store, then the unlocked window
  int nz = 0;
  const int64_t ldz = round_up(h->store_cap, 4);
  int it1 = 0;
  bool p1_all = false;   // phase 1 locked every wanted pair
  {
    Engine<float> e1(h, std::max(h->opt.mixed_switch_tol, h->tol), h->opt.max_iter);
    e1.stagnation_limit = 10;
    e1.checks = h->opt.checks != 0;
    if (h->opt.profile) e1.prof = &prof;
    GCGE_CHECK(e1.setup(sx, h->nev, h->store_cap));
    const int s1 = e1.run(X0d, ld0, nullptr, 0);
    if (s1 != GCGE_OK && s1 != GCGE_ENOTCONV) return s1;
    int tc_err = 0;   // a tensor-core kernel whose bounded wait ran out leaves a flag
    GCGE_CHECK(tc_error_flag(&tc_err, h->st));
    if (tc_err) return GCGE_ETIMEOUT;
    it1 = e1.iterations();
    p1_all = e1.nlock() >= h->nev;
    add_stats(h, e1);
    const int take_s = std::min(e1.nlock(), h->store_cap);
    const int take_x = std::min(e1.kx(), h->store_cap - take_s);
    nz = std::max(take_s + take_x, sx);
    GCGE_CUDA(cudaMalloc(&Z, sizeof(float) * (size_t)h->n * ldz));
    if (take_s > 0)
      GCGE_CHECK(copy_cols<float, float>(h->n, take_s, e1.store(), e1.ld_store(), Z, ldz, nullptr,
                                         h->st));
    if (take_x > 0)
      GCGE_CHECK(copy_cols<float, float>(h->n, take_x, e1.xa(), e1.ldv(), Z + take_s, ldz,
                                         nullptr, h->st));
    if (take_s + take_x < nz)
      GCGE_CHECK(random_block<float>(h->n, nz - take_s - take_x, h->opt.seed + 1,
                                     Z + take_s + take_x, ldz, h->st));
    GCGE_CUDA(cudaStreamSynchronize(h->st));
  }
  *iters32 = it1;
  int s;
  {
    // phase 2: FP64 iteration started from the phase-1 vectors (active block blockSize
    // unless mixed_bs2 says otherwise); with the moving mechanism the window of size_x
    // is refilled from the phase-1 vectors as pairs lock.  The inexact inner CG runs
    // in FP32 on the FP64 residual.
    int bs2 = std::min(h->bs, sx);
    if (h->opt.mixed_bs2 > 0) bs2 = std::min(h->opt.mixed_bs2, sx);
    Engine<double> e2(h, h->tol, std::max(1, h->opt.max_iter - it1));
    e2.checks = h->opt.checks != 0;
    e2.cg_fp32 = true;
    // when phase 1 reached the switch tolerance on every pair, phase 2 is a short
    // refinement and P does not pay for itself; otherwise it is a full FP64 solve
    // and P (STEP 5) is built as in the plain path
    e2.use_p = h->moving || !p1_all;
    if (h->opt.profile) e2.prof = &prof;
    e2.reservoir_planned = true;
    e2.share_store = true;
    s = e2.setup(sx, h->nev, h->store_cap, bs2);
    if (s == GCGE_OK) {
      e2.set_reservoir(Z, ldz, nz);
      s = e2.run(nullptr, 0, Z, ldz);
    }
    *iters = it1 + e2.iterations();
    add_stats(h, e2);
    if (s == GCGE_OK || s == GCGE_ENOTCONV) {
      int tc_err = 0;
      const int s3 = tc_error_flag(&tc_err, h->st);
      if (s3 != GCGE_OK) s = s3;
      else if (tc_err) s = GCGE_ETIMEOUT;
    }
    if (s == GCGE_OK || s == GCGE_ENOTCONV) {
      const int s2 = export_store(h, e2);
      if (s2 != GCGE_OK) s = s2;
    }
  }
  cudaFree(Z);
  return s;
}

}  // namespace gcge
