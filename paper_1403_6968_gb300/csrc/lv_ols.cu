// OLS kernels (Section 4.1 and Examples 3.1-3.3 of arXiv 1403.6968).
//
// beta* = (X^T X)^{-1} X^T Y.  Replacing the rows R of X by X'_R changes
// Z = X^T X by dZ = X'_R^T X'_R - X_R^T X_R = U C U^T with U = [X'_R^T, X_R^T]
// (n x 2k) and C = diag(I_k, -I_k); W = Z^{-1} then follows from block
// Woodbury (the rank-2k form of the paper's two Sherman-Morrison steps):
//   G = W U,  M = C^{-1} + U^T G (2k x 2k, FP64),  W' = W - G M^{-1} G^T.
// beta' = W' C' with C' = X^T Y + D^T Y_R (D = X'_R - X_R) is refreshed from
// factors only, with no pass over W:
//   W C' = beta + W D^T Y_R = beta + (G_1 - G_2) Y_R   (G_1, G_2: the halves of G)
//   W' C' = W C' + G (Wu^T C'),  Wu = -G M^{-1},
// i.e. the delta rule of a product applied to beta = W (X^T Y).
// The view passes (G = W U; W += G Wu^T) run in the shared pass kernels;
// this file holds the small pieces: row gather/scatter, the FP64 core
// inverse, Wu, the X^T Y and beta updates and the re-evaluation helpers.
#include <cuda_runtime.h>

#include "lv_device.cuh"
#include "lv_internal.h"
#include "lv_ols.h"

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

// Minv = (diag(c) + S)^{-1} for the kk x kk FP64 matrix S (row-major, kk <=
// 64) with c = (+1 x kpos, -1 x (kk - kpos)): Gauss-Jordan elimination with
// partial pivoting on the augmented [M | I] in one CTA of 32 x 16 threads.
// Each column step reads one copy of the augmented matrix and writes the
// other: warp 0 picks the pivot (largest magnitude in the column, the first
// row on ties) and scales the pivot row; then every thread writes its
// elements of the next copy with the pivot row swapped into place.  Two
// barriers per column; the FP64 work (about 1.5 kk^3 FMAs) is spread over
// all 512 threads.  A pivot at or below 1e-13 * max|M| latches
// kStatusSingular and the result is zero.
constexpr int kInvTx = 32, kInvTy = 16;

size_t core_inverse_smem(int kk) { return sizeof(double) * ((size_t)4 * kk * kk + 3 * kk); }

__global__ void __launch_bounds__(kInvTx * kInvTy)
    core_inverse_kernel(const double* S, int kk, int kpos, double* Minv, unsigned* status) {
  extern __shared__ double inv_sm[];
  const int w = 2 * kk;
  double* cur = inv_sm;           // kk x w
  double* nxt = cur + kk * w;     // kk x w
  double* prow = nxt + kk * w;    // w: the pivot row divided by the pivot
  double* fcol = prow + w;        // kk: column col before the step
  __shared__ double wmax[kInvTy];
  __shared__ int s_piv, s_sing;
  const int tx = threadIdx.x, ty = threadIdx.y;
  double m = 0.0;
  for (int i = ty; i < kk; i += kInvTy)
    for (int j = tx; j < w; j += kInvTx) {
      double v;
      if (j < kk) {
        v = S[i * kk + j] + (i == j ? (i < kpos ? 1.0 : -1.0) : 0.0);
        m = fmax(m, fabs(v));
      } else {
        v = (j - kk == i) ? 1.0 : 0.0;
      }
      cur[i * w + j] = v;
    }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (tx == 0) wmax[ty] = m;
  if (tx == 0 && ty == 0) s_sing = 0;
  __syncthreads();
  double scale = 0.0;
  for (int t = 0; t < kInvTy; ++t) scale = fmax(scale, wmax[t]);
  const double tiny = 1e-13 * scale;
  for (int col = 0; col < kk; ++col) {
    if (ty == 0) {
      double bv = -1.0;
      int bi = kk;
      for (int i = col + tx; i < kk; i += kInvTx) {
        const double v = fabs(cur[i * w + col]);
        if (v > bv) { bv = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (bi >= kk) bi = col;  // the column is all NaN
      if (!(bv > tiny) && tx == 0) {
        s_sing = 1;
        atomicOr(status, kStatusSingular);
      }
      const double r = 1.0 / cur[bi * w + col];
      for (int j = tx; j < w; j += kInvTx) prow[j] = cur[bi * w + j] * r;
      for (int i = tx; i < kk; i += kInvTx) fcol[i] = cur[i * w + col];
      if (tx == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    for (int i = ty; i < kk; i += kInvTy) {
      const int src = (i == col) ? piv : (i == piv ? col : i);  // rows col and piv swap
      const double f = fcol[src];
      const double* a = cur + src * w;
      double* o = nxt + i * w;
      for (int j = tx; j < w; j += kInvTx) {
        double v;
        if (i == col) v = (j == col) ? 1.0 : prow[j];
        else if (j == col) v = 0.0;
        else if (j < col) v = a[j];  // finished columns: prow[j] is 0 there
        else v = fma(-f, prow[j], a[j]);
        o[j] = v;
      }
    }
    __syncthreads();
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  const bool singular = s_sing != 0;
  for (int i = ty; i < kk; i += kInvTy)
    for (int j = tx; j < kk; j += kInvTx) Minv[i * kk + j] = singular ? 0.0 : cur[i * w + kk + j];
}

// Double-float arithmetic (a value is hi + lo, two FP32 numbers, about 48
// significant bits): the core inverse of FP32 programs runs on GB300's FP32
// pipe, 64 times as wide as its FP64 pipe.  Products are exact by FMA
// (p = a b, e = fma(a, b, -p)), sums by Knuth's TwoSum; the intrinsics keep
// the compiler from contracting or reassociating any step.
struct df2 {
  float hi, lo;
};
__device__ __forceinline__ df2 df_make(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_double(df2 x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ df2 df_sum(df2 a, df2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df2 df_prod(df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
// a - f b
__device__ __forceinline__ df2 df_fms(df2 a, df2 f, df2 b) {
  const df2 q = df_prod(f, b);
  return df_sum(a, {-q.hi, -q.lo});
}
// 1 / a: an FP32 reciprocal refined by two Newton steps x += x (1 - a x)
__device__ __forceinline__ df2 df_recip(df2 a) {
  df2 x = {__frcp_rn(a.hi), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df2 ax = df_prod(a, x);
    const df2 e = df_sum({1.f, 0.f}, {-ax.hi, -ax.lo});
    x = df_sum(x, df_prod(x, e));
  }
  return x;
}

// The same Gauss-Jordan elimination as core_inverse_kernel in double-float
// arithmetic (FP32 programs): M and the result are FP64 at the interface.
__global__ void __launch_bounds__(kInvTx * kInvTy)
    core_inverse_df_kernel(const double* S, int kk, int kpos, double* Minv, unsigned* status) {
  extern __shared__ double inv_sm[];
  const int w = 2 * kk;
  df2* cur = reinterpret_cast<df2*>(inv_sm);  // kk x w
  df2* nxt = cur + kk * w;                    // kk x w
  df2* prow = nxt + kk * w;                   // w: the pivot row divided by the pivot
  df2* fcol = prow + w;                       // kk: column col before the step
  __shared__ float wmax[kInvTy];
  __shared__ int s_piv, s_sing;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float m = 0.f;
  for (int i = ty; i < kk; i += kInvTy)
    for (int j = tx; j < w; j += kInvTx) {
      df2 v;
      if (j < kk) {
        v = df_make(S[i * kk + j] + (i == j ? (i < kpos ? 1.0 : -1.0) : 0.0));
        m = fmaxf(m, fabsf(v.hi));
      } else {
        v = {(j - kk == i) ? 1.f : 0.f, 0.f};
      }
      cur[i * w + j] = v;
    }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (tx == 0) wmax[ty] = m;
  if (tx == 0 && ty == 0) s_sing = 0;
  __syncthreads();
  float scale = 0.f;
  for (int t = 0; t < kInvTy; ++t) scale = fmaxf(scale, wmax[t]);
  const float tiny = 1e-13f * scale;
  for (int col = 0; col < kk; ++col) {
    if (ty == 0) {
      float bv = -1.f;
      int bi = kk;
      for (int i = col + tx; i < kk; i += kInvTx) {
        const float v = fabsf(cur[i * w + col].hi);
        if (v > bv) { bv = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (bi >= kk) bi = col;  // the column is all NaN
      if (!(bv > tiny) && tx == 0) {
        s_sing = 1;
        atomicOr(status, kStatusSingular);
      }
      const df2 r = df_recip(cur[bi * w + col]);
      for (int j = tx; j < w; j += kInvTx) prow[j] = df_prod(cur[bi * w + j], r);
      for (int i = tx; i < kk; i += kInvTx) fcol[i] = cur[i * w + col];
      if (tx == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    for (int i = ty; i < kk; i += kInvTy) {
      const int src = (i == col) ? piv : (i == piv ? col : i);  // rows col and piv swap
      const df2 f = fcol[src];
      const df2* a = cur + src * w;
      df2* o = nxt + i * w;
      for (int j = tx; j < w; j += kInvTx) {
        df2 v;
        if (i == col) v = (j == col) ? df2{1.f, 0.f} : prow[j];
        else if (j == col) v = {0.f, 0.f};
        else if (j < col) v = a[j];  // finished columns: prow[j] is 0 there
        else v = df_fms(a[j], f, prow[j]);
        o[j] = v;
      }
    }
    __syncthreads();
    df2* t = cur;
    cur = nxt;
    nxt = t;
  }
  const bool singular = s_sing != 0;
  for (int i = ty; i < kk; i += kInvTy)
    for (int j = tx; j < kk; j += kInvTx)
      Minv[i * kk + j] = singular ? 0.0 : df_double(cur[i * w + kk + j]);
}

// Wu(:, c) = - sum_c' G(:, c') Minv(c', c) in FP64; a thread computes two
// columns c = 2 blockIdx.y, 2 blockIdx.y + 1 of one row j (kk is even).
template <typename T>
__global__ void wu_kernel(const T* G, int64_t fs, int n, int kk, const double* Minv, T* Wu) {
  __shared__ double ms[64][2];
  const int c = 2 * blockIdx.y;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    ms[e][0] = Minv[e * kk + c];
    ms[e][1] = Minv[e * kk + c + 1];
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a0 = 0.0, a1 = 0.0;
  for (int c2 = 0; c2 < kk; ++c2) {
    const double g = (double)G[(int64_t)c2 * fs + j];
    a0 = fma(g, ms[c2][0], a0);
    a1 = fma(g, ms[c2][1], a1);
  }
  Wu[(int64_t)c * fs + j] = (T)(-a0);
  Wu[(int64_t)(c + 1) * fs + j] = (T)(-a1);
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

// H(c2, c) = sum_j Wu(j, c2) C(j, c) for column-major Wu (n x kk) and C
// (n x p), column stride fs; one CTA per entry (blockIdx.x = c * kk + c2),
// per-thread partial sums in T, combined in FP64 in a fixed order.  H is
// kk x p row-major.
template <typename T>
__global__ void __launch_bounds__(256) wtc_kernel(const T* Wu, const T* Cc, int64_t fs, int n,
                                                  int kk, int p, T* H) {
  __shared__ double part[8];
  const int c2 = blockIdx.x % kk, c = blockIdx.x / kk;
  const T* a = Wu + (int64_t)c2 * fs;
  const T* b = Cc + (int64_t)c * fs;
  T acc = 0;
  for (int j = threadIdx.x; j < n; j += 256) acc += a[j] * b[j];
  double d = (double)acc;
#pragma unroll
  for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += part[i];
    H[c2 * p + c] = (T)t;
  }
}

// beta(j, c) += sum_t (G(j, t) - G(j, k + t)) Y_R(t, c) + sum_c2 G(j, c2) H(c2, c)
// (the factored beta refresh above); G column-major (fs), Y_R k x p and H
// 2k x p row-major, beta row-major (ld).
template <typename T>
__global__ void beta_update_kernel(T* beta, int64_t ld, const T* G, int64_t fs, int n, int p,
                                   int k, const T* Yr, const T* H) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * p) return;
  int j, c;
  split_index(idx, p, j, c);
  T acc = 0;
  for (int t = 0; t < k; ++t)
    acc += (G[(int64_t)t * fs + j] - G[(int64_t)(k + t) * fs + j]) * Yr[t * p + c];
  for (int c2 = 0; c2 < 2 * k; ++c2) acc += G[(int64_t)c2 * fs + j] * H[c2 * p + c];
  beta[(int64_t)j * ld + c] += acc;
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
                                cudaStream_t s, bool double_float) {
  if (kk < 1 || kk > 64) return cudaErrorInvalidValue;
  static const cudaError_t configured =
      cudaFuncSetAttribute(core_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)core_inverse_smem(64));
  if (configured != cudaSuccess) return configured;
  static const cudaError_t configured_df =
      cudaFuncSetAttribute(core_inverse_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)core_inverse_smem(64));
  if (configured_df != cudaSuccess) return configured_df;
  if (double_float)
    core_inverse_df_kernel<<<1, dim3(kInvTx, kInvTy), core_inverse_smem(kk), s>>>(S, kk, kpos,
                                                                                Minv, status);
  else
    core_inverse_kernel<<<1, dim3(kInvTx, kInvTy), core_inverse_smem(kk), s>>>(S, kk, kpos, Minv,
                                                                             status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wu(const T* G, int64_t fs, int n, int kk, const double* Minv, T* Wu,
                      cudaStream_t s) {
  if (kk < 2 || kk > 64 || (kk & 1)) return cudaErrorInvalidValue;
  wu_kernel<T><<<dim3(blocks_for(n), kk / 2), kThreads, 0, s>>>(G, fs, n, kk, Minv, Wu);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_beta_update(T* beta, int64_t ld, const T* G, const T* Wu, const T* Cc,
                               int64_t fs, int n, int p, int k, const T* Yr, T* H,
                               cudaStream_t s) {
  wtc_kernel<T><<<(unsigned)(2 * k * p), 256, 0, s>>>(Wu, Cc, fs, n, 2 * k, p, H);
  beta_update_kernel<T><<<blocks_for((int64_t)n * p), kThreads, 0, s>>>(beta, ld, G, fs, n, p, k,
                                                                        Yr, H);
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
  template cudaError_t launch_beta_update<T>(T*, int64_t, const T*, const T*, const T*, int64_t,  \
                                             int, int, int, const T*, T*, cudaStream_t);         \
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
