// OLS kernels (Section 4.1 and Examples 3.1-3.3 of arXiv 1403.6968).
//
// beta* = (X^T X)^{-1} X^T Y.  Replacing the rows R of X by X'_R changes
// Z = X^T X by dZ = X'_R^T X'_R - X_R^T X_R = U C U^T with U = [X'_R^T, X_R^T]
// (n x 2k) and C = diag(I_k, -I_k); W = Z^{-1} then follows from block
// Woodbury (the rank-2k form of the paper's two Sherman-Morrison steps):
//   G = W U,  M = C^{-1} + U^T G (2k x 2k, FP64),  W' = W - G M^{-1} G^T.
// The view passes (products G = W U, beta = W' X^T Y; update W += G Wu^T)
// run in the shared pass kernels; this file holds the small pieces: row
// gather/scatter, the FP64 core inverse, Wu = -G M^{-1}, the X^T Y update and
// the re-evaluation helpers.
#include <cuda_runtime.h>

#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {

// dst[t * ts + j * js] = X[rows[t] * ldx + j]
template <typename T>
__global__ void gather_rows_kernel(const T* X, int64_t ldx, const int64_t* rows, int k, int n,
                                   T* dst, int64_t ts, int64_t js) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * n) return;
  int t, j;
  split_index(idx, n, t, j);
  dst[t * ts + j * js] = X[rows[t] * ldx + j];
}

// X[rows[t] * ldx + j] = src[t * ts + j]
template <typename T>
__global__ void scatter_rows_kernel(T* X, int64_t ldx, const int64_t* rows, int k, int n,
                                    const T* src, int64_t ts) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * n) return;
  int t, j;
  split_index(idx, n, t, j);
  X[rows[t] * ldx + j] = src[t * ts + j];
}

// Minv = (diag(c) + S)^{-1} for the kk x kk FP64 matrix S (row-major) with
// c = (+1 x kpos, -1 x (kk - kpos)); Gauss-Jordan with partial pivoting in one
// CTA.  A pivot below 1e-13 * max|entry| latches kStatusSingular.
__global__ void core_inverse_kernel(const double* S, int kk, int kpos, double* Minv,
                                    unsigned* status) {
  extern __shared__ double a[];  // kk x 2kk augmented [M | I]
  __shared__ int piv;
  __shared__ double scale;
  const int w = 2 * kk;
  for (int e = threadIdx.x; e < kk * w; e += blockDim.x) {
    const int i = e / w, j = e % w;
    double v;
    if (j < kk) v = S[i * kk + j] + (i == j ? (i < kpos ? 1.0 : -1.0) : 0.0);
    else v = (j - kk == i) ? 1.0 : 0.0;
    a[e] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < kk; ++i)
      for (int j = 0; j < kk; ++j) m = fmax(m, fabs(a[i * w + j]));
    scale = m;
  }
  __syncthreads();
  bool singular = false;
  for (int col = 0; col < kk; ++col) {
    if (threadIdx.x == 0) {
      int best = col;
      double bv = fabs(a[col * w + col]);
      for (int i = col + 1; i < kk; ++i) {
        const double v = fabs(a[i * w + col]);
        if (v > bv) { bv = v; best = i; }
      }
      piv = best;
      if (!(bv > 1e-13 * scale)) atomicOr(status, kStatusSingular);
    }
    __syncthreads();
    const int pr = piv;
    if (!(fabs(a[pr * w + col]) > 1e-13 * scale)) singular = true;
    if (pr != col) {
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = a[col * w + j];
        a[col * w + j] = a[pr * w + j];
        a[pr * w + j] = t;
      }
    }
    __syncthreads();
    const double d = a[col * w + col];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) a[col * w + j] /= d;
    __syncthreads();
    for (int e = threadIdx.x; e < kk * w; e += blockDim.x) {
      const int i = e / w, j = e % w;
      if (i != col) {
        const double f = a[i * w + col];
        if (j != col) a[e] -= f * a[col * w + j];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kk; i += blockDim.x)
      if (i != col) a[i * w + col] = 0.0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
    const int i = e / kk, j = e % kk;
    Minv[e] = singular ? 0.0 : a[i * w + kk + j];
  }
}

// Wu(:, c) = - sum_c' G(:, c') Minv(c', c)   (FP64 accumulation)
template <typename T>
__global__ void wu_kernel(const T* G, int64_t fs, int n, int kk, const double* Minv, T* Wu) {
  extern __shared__ double ms[];
  for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) ms[e] = Minv[e];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int c = 0; c < kk; ++c) {
    double acc = 0.0;
    for (int c2 = 0; c2 < kk; ++c2) acc = fma((double)G[(int64_t)c2 * fs + j], ms[c2 * kk + c], acc);
    Wu[(int64_t)c * fs + j] = (T)(-acc);
  }
}

// X^T Y += (X'_R - X_R)^T Y_R.  U holds X'_R^T in columns [0, k) and X_R^T in
// [k, 2k); Yr is k x p row-major.  Updates the row-major view (ld) and the
// column-major mirror (fs).
template <typename T>
__global__ void xty_update_kernel(T* xty, int64_t ld, T* xtyc, int64_t fs, const T* U, int n,
                                  int p, int k, const T* Yr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * p) return;
  int j, c;
  split_index(idx, p, j, c);
  double acc = (double)xty[(int64_t)j * ld + c];
  for (int t = 0; t < k; ++t) {
    const double d = (double)U[(int64_t)t * fs + j] - (double)U[(int64_t)(k + t) * fs + j];
    acc = fma(d, (double)Yr[(int64_t)t * p + c], acc);
  }
  xty[(int64_t)j * ld + c] = (T)acc;
  xtyc[(int64_t)c * fs + j] = (T)acc;
}

// dst (double, row-major rows x cols, ldd) = (double) src (T, lds)
template <typename T>
__global__ void to_double_kernel(const T* src, int64_t lds, double* dst, int64_t ldd, int rows,
                                 int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int i, j;
  split_index(idx, cols, i, j);
  dst[(int64_t)i * ldd + j] = (double)src[(int64_t)i * lds + j];
}

// dst (T, row-major n x n) from the lower triangle of a column-major FP64
// symmetric matrix; optionally also the full FP64 symmetric copy.
template <typename T>
__global__ void sym_lower_to_full_kernel(const double* Lcm, int64_t ldl, int n, T* dst,
                                         int64_t ldd, double* full, int64_t ldf) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int i, j;
  split_index(idx, n, i, j);
  const int r = i > j ? i : j, c = i > j ? j : i;  // lower: row >= col
  const double v = Lcm[(int64_t)c * ldl + r];       // column-major (r, c)
  dst[(int64_t)i * ldd + j] = (T)v;
  if (full) full[(int64_t)i * ldf + j] = v;
}

// dst (T, ldd) = (T) src (double, lds); also optional column-major mirror
template <typename T>
__global__ void from_double_kernel(const double* src, int64_t lds, T* dst, int64_t ldd, int rows,
                                   int cols, T* cm, int64_t cfs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int i, j;
  split_index(idx, cols, i, j);
  const T v = (T)src[(int64_t)i * lds + j];
  dst[(int64_t)i * ldd + j] = v;
  if (cm) cm[(int64_t)j * cfs + i] = v;
}

static unsigned blocks_for(int64_t tot) { return (unsigned)((tot + kThreads - 1) / kThreads); }

template <typename T>
cudaError_t launch_gather_rows(const T* X, int64_t ldx, const int64_t* rows, int k, int n, T* dst,
                               int64_t ts, int64_t js, cudaStream_t s) {
  if ((int64_t)k * n == 0) return cudaSuccess;
  gather_rows_kernel<T><<<blocks_for((int64_t)k * n), kThreads, 0, s>>>(X, ldx, rows, k, n, dst,
                                                                        ts, js);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_rows(T* X, int64_t ldx, const int64_t* rows, int k, int n,
                                const T* src, int64_t ts, cudaStream_t s) {
  if ((int64_t)k * n == 0) return cudaSuccess;
  scatter_rows_kernel<T><<<blocks_for((int64_t)k * n), kThreads, 0, s>>>(X, ldx, rows, k, n, src,
                                                                         ts);
  return cudaGetLastError();
}

cudaError_t launch_core_inverse(const double* S, int kk, int kpos, double* Minv, unsigned* status,
                                cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)kk * 2 * kk;
  core_inverse_kernel<<<1, kThreads, smem, s>>>(S, kk, kpos, Minv, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wu(const T* G, int64_t fs, int n, int kk, const double* Minv, T* Wu,
                      cudaStream_t s) {
  wu_kernel<T><<<blocks_for(n), kThreads, sizeof(double) * kk * kk, s>>>(G, fs, n, kk, Minv, Wu);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xty_update(T* xty, int64_t ld, T* xtyc, int64_t fs, const T* U, int n, int p,
                              int k, const T* Yr, cudaStream_t s) {
  xty_update_kernel<T><<<blocks_for((int64_t)n * p), kThreads, 0, s>>>(xty, ld, xtyc, fs, U, n, p,
                                                                       k, Yr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_double(const T* src, int64_t lds, double* dst, int64_t ldd, int rows,
                             int cols, cudaStream_t s) {
  if ((int64_t)rows * cols == 0) return cudaSuccess;
  to_double_kernel<T><<<blocks_for((int64_t)rows * cols), kThreads, 0, s>>>(src, lds, dst, ldd,
                                                                           rows, cols);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sym_lower_to_full(const double* Lcm, int64_t ldl, int n, T* dst, int64_t ldd,
                                     double* full, int64_t ldf, cudaStream_t s) {
  sym_lower_to_full_kernel<T><<<blocks_for((int64_t)n * n), kThreads, 0, s>>>(Lcm, ldl, n, dst,
                                                                              ldd, full, ldf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_from_double(const double* src, int64_t lds, T* dst, int64_t ldd, int rows,
                               int cols, T* cm, int64_t cfs, cudaStream_t s) {
  from_double_kernel<T><<<blocks_for((int64_t)rows * cols), kThreads, 0, s>>>(src, lds, dst, ldd,
                                                                              rows, cols, cm, cfs);
  return cudaGetLastError();
}

#define LV_OLS_INST(T)                                                                           \
  template cudaError_t launch_gather_rows<T>(const T*, int64_t, const int64_t*, int, int, T*,     \
                                             int64_t, int64_t, cudaStream_t);                    \
  template cudaError_t launch_scatter_rows<T>(T*, int64_t, const int64_t*, int, int, const T*,    \
                                              int64_t, cudaStream_t);                            \
  template cudaError_t launch_wu<T>(const T*, int64_t, int, int, const double*, T*, cudaStream_t); \
  template cudaError_t launch_xty_update<T>(T*, int64_t, T*, int64_t, const T*, int, int, int,    \
                                            const T*, cudaStream_t);                             \
  template cudaError_t launch_to_double<T>(const T*, int64_t, double*, int64_t, int, int,         \
                                           cudaStream_t);                                        \
  template cudaError_t launch_sym_lower_to_full<T>(const double*, int64_t, int, T*, int64_t,      \
                                                   double*, int64_t, cudaStream_t);              \
  template cudaError_t launch_from_double<T>(const double*, int64_t, T*, int64_t, int, int, T*,   \
                                             int64_t, cudaStream_t);
LV_OLS_INST(float)
LV_OLS_INST(double)

}  // namespace lv
