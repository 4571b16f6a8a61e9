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

// ---------------------------------------------------------------------------
// FP32 programs: the core inverse in double-float on the FP32 pipe (one CTA
// of kCoreThreads threads), M = C^{-1} + S with S = U^T W U given as FP32
// pairs and C = diag(I, -I).
//
// Newton-Schulz first.  M stays close to C^{-1} = C (the replaced rows'
// leverages x^T W x are about n / m), so X_{j+1} = X_j + X_j R_j with
// R_j = I - M X_j and X_0 = C converges quadratically: R_{j+1} = R_j^2, hence
// ||R_{j+1}||_F <= ||R_j||_F^2 (Frobenius norm, submultiplicative) and the
// iteration converges iff ||R_0||_F < 1.  Every step is two kk x kk products
// whose entries are independent dot products (each thread takes a 2 x 2 tile
// of entries), not kk barrier-separated pivot steps.  The steps run in FP32
// on M rounded to FP32 until their rounding floor (a step that no longer
// squares the norm, or a norm below 1e-6).  One residual R = I - M X of that
// FP32 iterate is then taken in double-float against the unrounded M and
// rounded to FP32 (|R| ~ 1e-6, so FP32 keeps it to ~1e-13 absolute), and the
// result is X + X R: the product X R in FP32 (its rounding error is ~1e-13
// of X), the sum as a double-float pair.  Since the new residual is R^2 plus
// that rounding, a double-float residual below kNsFinish gives an inverse
// with a residual near 1e-11 or better.
//
// Otherwise -- ||R_0|| >= 1, an FP32 floor above 1e-3, a double-float
// residual at or above kNsFinish, or non-finite values: a core far from C,
// ill-conditioned or singular -- the same CTA runs Gauss-Jordan elimination
// with partial pivoting in double-float (as core_inverse_kernel does in FP64),
// which also latches kStatusSingular for a singular core.
// ---------------------------------------------------------------------------
constexpr int kCoreThreads = kInvTx * kInvTy;  // 512
constexpr int kNsMaxIter = 12;
constexpr float kNsFinish = 1e-5f;

__host__ __device__ inline int ns_ld(int kk) { return kk + 2; }  // padded row stride (even)

size_t core_df_smem(int kk) {
  const size_t ld = (size_t)ns_ld(kk);
  const size_t ns = (size_t)kk * ld * (sizeof(df2) + 4 * sizeof(float));  // Md, Mf, Xa, Xb, Rf
  const size_t gj = sizeof(df2) * ((size_t)4 * kk * kk + 3 * kk);
  return ns > gj ? ns : gj;
}

// acc += x y for df2 x and float y: the exact product of the high parts by
// FMA, the low part's product in FP32; the high sum by TwoSum, the errors
// collected in acc.lo (renormalised by the caller)
__device__ __forceinline__ void df_acc(df2& acc, df2 x, float y) {
  const float p = __fmul_rn(x.hi, y);
  const float e = __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -p));
  const float t = __fadd_rn(acc.hi, p);
  const float z = __fsub_rn(t, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
  acc.hi = t;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ df2 df_norm(df2 a) {
  const float h = __fadd_rn(a.hi, a.lo);
  return {h, __fsub_rn(a.lo, __fsub_rn(h, a.hi))};
}

// sum over the CTA of the per-thread values v, in a fixed order; every
// thread returns the same total
__device__ __forceinline__ float cta_sum(float v, float* wsum) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // earlier readers of wsum are done
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kCoreThreads / 32; ++w) t += wsum[w];
  return t;
}

// Gauss-Jordan elimination with partial pivoting in double-float on the
// augmented [M | I]: each column step reads one copy and writes the other;
// warp 0 picks the pivot (largest magnitude, first row on ties) and scales the
// pivot row.  A pivot at or below 1e-13 max|M| latches kStatusSingular and
// the result is zero.  (tx, ty) in [0, kInvTx) x [0, kInvTy).
__device__ void gauss_jordan_df(const float2* S, int kk, int kpos, float2* Minv, unsigned* status,
                                df2* sm, int tx, int ty) {
  const int w = 2 * kk;
  df2* cur = sm;               // kk x w
  df2* nxt = cur + kk * w;     // kk x w
  df2* prow = nxt + kk * w;    // w: the pivot row divided by the pivot
  df2* fcol = prow + w;        // kk: column col before the step
  __shared__ float wmax[kInvTy];
  __shared__ int s_piv, s_sing;
  float m = 0.f;
  for (int i = ty; i < kk; i += kInvTy)
    for (int j = tx; j < w; j += kInvTx) {
      df2 v;
      if (j < kk) {
        const float2 sv = S[i * kk + j];
        v = {sv.x, sv.y};
        if (i == j) v = df_sum(v, {i < kpos ? 1.f : -1.f, 0.f});
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
    for (int j = tx; j < kk; j += kInvTx) {
      const df2 v = cur[i * w + kk + j];
      Minv[i * kk + j] = singular ? make_float2(0.f, 0.f) : make_float2(v.hi, v.lo);
    }
}

// O = D + sgn A B over 2 x 2 tiles (FP32; A, B, O with row stride ld; D the
// identity if ident, else A itself when addA).  Returns this thread's sum of
// squares of the O entries it wrote.
__device__ __forceinline__ float ns_product(const float* A, const float* B, float* O, int kk,
                                            int ld, float sgn, bool ident, const float* Dsrc) {
  const int h = kk / 2;
  float m = 0.f;
  for (int tile = threadIdx.x; tile < h * h; tile += kCoreThreads) {
    const int i0 = 2 * (tile / h), j0 = 2 * (tile % h);
    float a00, a01, a10, a11;
    if (ident) {
      a00 = (i0 == j0) ? 1.f : 0.f;
      a01 = 0.f;
      a10 = 0.f;
      a11 = a00;
    } else {
      const float2 d0 = *reinterpret_cast<const float2*>(Dsrc + i0 * ld + j0);
      const float2 d1 = *reinterpret_cast<const float2*>(Dsrc + (i0 + 1) * ld + j0);
      a00 = d0.x; a01 = d0.y; a10 = d1.x; a11 = d1.y;
    }
    const float* a0 = A + i0 * ld;
    const float* a1 = a0 + ld;
#pragma unroll 4
    for (int t = 0; t < kk; ++t) {
      const float2 bv = *reinterpret_cast<const float2*>(B + t * ld + j0);
      const float x0 = sgn * a0[t], x1 = sgn * a1[t];
      a00 = fmaf(x0, bv.x, a00);
      a01 = fmaf(x0, bv.y, a01);
      a10 = fmaf(x1, bv.x, a10);
      a11 = fmaf(x1, bv.y, a11);
    }
    *reinterpret_cast<float2*>(O + i0 * ld + j0) = make_float2(a00, a01);
    *reinterpret_cast<float2*>(O + (i0 + 1) * ld + j0) = make_float2(a10, a11);
    m = fmaf(a00, a00, fmaf(a01, a01, fmaf(a10, a10, fmaf(a11, a11, m))));
  }
  return m;
}

__global__ void __launch_bounds__(kCoreThreads)
    core_inverse_df_kernel(const float2* S, int kk, int kpos, float2* Minv, unsigned* status) {
  extern __shared__ __align__(16) unsigned char core_sm[];
  __shared__ float wsum[kCoreThreads / 32];
  const int tid = threadIdx.x;
  const int ld = ns_ld(kk);
  const int e2 = kk * kk;
  df2* Md = reinterpret_cast<df2*>(core_sm);  // kk x ld
  float* Mf = reinterpret_cast<float*>(Md + kk * ld);
  float* Xa = Mf + kk * ld;
  float* Xb = Xa + kk * ld;
  float* Rf = Xb + kk * ld;
  for (int e = tid; e < e2; e += kCoreThreads) {
    const int i = e / kk, j = e % kk;
    const float2 sv = S[e];
    df2 v = {sv.x, sv.y};
    float c = 0.f;
    if (i == j) {
      c = i < kpos ? 1.f : -1.f;
      v = df_sum(v, {c, 0.f});
    }
    Md[i * ld + j] = v;
    Mf[i * ld + j] = v.hi;
    Xa[i * ld + j] = c;
  }
  __syncthreads();
  float* Xc = Xa;
  float* Xn = Xb;
  bool to_df = false;
  if ((kk & 1) == 0) {
    float prev = -1.f;
    for (int it = 0; it < kNsMaxIter; ++it) {
      // R = I - M X (FP32); every thread reaches the same decision
      const float r = sqrtf(cta_sum(ns_product(Mf, Xc, Rf, kk, ld, -1.f, true, nullptr), wsum));
      if (!(r < 1.f)) break;  // diverges (or NaN): Gauss-Jordan
      if (r < 1e-6f || (prev >= 0.f && r > 2.f * prev * prev)) {
        to_df = r < 1e-3f;  // the FP32 floor: finish in double-float
        break;
      }
      prev = r;
      // X' = X + X R into the other buffer
      ns_product(Xc, Rf, Xn, kk, ld, 1.f, false, Xc);
      __syncthreads();
      float* t = Xc;
      Xc = Xn;
      Xn = t;
    }
  }
  if (to_df) {
    // R = I - M X with M in double-float, rounded to FP32
    const int h = kk / 2;
    float m = 0.f;
    __syncthreads();  // the FP32 residual's readers are done
    for (int tile = tid; tile < h * h; tile += kCoreThreads) {
      const int i0 = 2 * (tile / h), j0 = 2 * (tile % h);
      df2 a00 = {(i0 == j0) ? 1.f : 0.f, 0.f}, a01 = {0.f, 0.f}, a10 = {0.f, 0.f}, a11 = a00;
      const df2* m0 = Md + i0 * ld;
      const df2* m1 = m0 + ld;
      for (int t = 0; t < kk; ++t) {
        const float2 bv = *reinterpret_cast<const float2*>(Xc + t * ld + j0);
        const df2 x0 = {-m0[t].hi, -m0[t].lo}, x1 = {-m1[t].hi, -m1[t].lo};
        df_acc(a00, x0, bv.x);
        df_acc(a01, x0, bv.y);
        df_acc(a10, x1, bv.x);
        df_acc(a11, x1, bv.y);
      }
      const float r00 = __fadd_rn(a00.hi, a00.lo), r01 = __fadd_rn(a01.hi, a01.lo);
      const float r10 = __fadd_rn(a10.hi, a10.lo), r11 = __fadd_rn(a11.hi, a11.lo);
      *reinterpret_cast<float2*>(Rf + i0 * ld + j0) = make_float2(r00, r01);
      *reinterpret_cast<float2*>(Rf + (i0 + 1) * ld + j0) = make_float2(r10, r11);
      m = fmaf(r00, r00, fmaf(r01, r01, fmaf(r10, r10, fmaf(r11, r11, m))));
    }
    const float r = sqrtf(cta_sum(m, wsum));
    if (r < kNsFinish) {
      // Minv = X + X R: X R in FP32, the sum as a pair
      for (int tile = tid; tile < h * h; tile += kCoreThreads) {
        const int i0 = 2 * (tile / h), j0 = 2 * (tile % h);
        float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
        const float* x0 = Xc + i0 * ld;
        const float* x1 = x0 + ld;
#pragma unroll 4
        for (int t = 0; t < kk; ++t) {
          const float2 bv = *reinterpret_cast<const float2*>(Rf + t * ld + j0);
          a00 = fmaf(x0[t], bv.x, a00);
          a01 = fmaf(x0[t], bv.y, a01);
          a10 = fmaf(x1[t], bv.x, a10);
          a11 = fmaf(x1[t], bv.y, a11);
        }
        const df2 o00 = df_sum({x0[j0], 0.f}, {a00, 0.f}), o01 = df_sum({x0[j0 + 1], 0.f}, {a01, 0.f});
        const df2 o10 = df_sum({x1[j0], 0.f}, {a10, 0.f}), o11 = df_sum({x1[j0 + 1], 0.f}, {a11, 0.f});
        Minv[i0 * kk + j0] = make_float2(o00.hi, o00.lo);
        Minv[i0 * kk + j0 + 1] = make_float2(o01.hi, o01.lo);
        Minv[(i0 + 1) * kk + j0] = make_float2(o10.hi, o10.lo);
        Minv[(i0 + 1) * kk + j0 + 1] = make_float2(o11.hi, o11.lo);
      }
      return;
    }
  }
  __syncthreads();  // the Newton-Schulz buffers are done with: the same memory
  gauss_jordan_df(S, kk, kpos, Minv, status, reinterpret_cast<df2*>(core_sm), tid % kInvTx,
                  tid / kInvTx);
}

// Wu(:, c) = - sum_c' G(:, c') Minv(c', c), FP64 views and core; a thread
// computes two columns c = 2 blockIdx.y, 2 blockIdx.y + 1 of one row j (kk
// is even).
__global__ void wu_f64_kernel(const double* G, int64_t fs, int n, int kk, const double* Minv,
                              double* Wu) {
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
    const double g = G[(int64_t)c2 * fs + j];
    a0 = fma(g, ms[c2][0], a0);
    a1 = fma(g, ms[c2][1], a1);
  }
  Wu[(int64_t)c * fs + j] = -a0;
  Wu[(int64_t)(c + 1) * fs + j] = -a1;
}

// The same for FP32 views with the double-float core: each product of an
// FP32 G entry and a core pair is accumulated as a pair (df_acc) and the sum
// is rounded once to FP32.  A thread computes four columns c = 4 blockIdx.y
// .. + 3 of one row j (kk is even; a trailing pair is masked).
constexpr int kWuCols = 4;
__global__ void wu_df_kernel(const float* G, int64_t fs, int n, int kk, const float2* Minv,
                             float* Wu) {
  __shared__ df2 ms[64][kWuCols];
  const int c0 = kWuCols * blockIdx.y;
  for (int e = threadIdx.x; e < kk * kWuCols; e += blockDim.x) {
    const int r = e / kWuCols, q = e % kWuCols;
    const float2 v = (c0 + q < kk) ? Minv[r * kk + c0 + q] : make_float2(0.f, 0.f);
    ms[r][q] = {-v.x, -v.y};
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  df2 acc[kWuCols];
#pragma unroll
  for (int q = 0; q < kWuCols; ++q) acc[q] = {0.f, 0.f};
  for (int c2 = 0; c2 < kk; ++c2) {
    const float g = G[(int64_t)c2 * fs + j];
#pragma unroll
    for (int q = 0; q < kWuCols; ++q) df_acc(acc[q], ms[c2][q], g);
  }
#pragma unroll
  for (int q = 0; q < kWuCols; ++q)
    if (c0 + q < kk) Wu[(int64_t)(c0 + q) * fs + j] = __fadd_rn(acc[q].hi, acc[q].lo);
}

// X^T Y += (X'_R - X_R)^T Y_R.  U holds X'_R^T in columns [0, k) and X_R^T in
// [k, 2k); Yr is k x p row-major.  Updates the row-major view (ld) and the
// column-major mirror (fs).  FP64 views: FP64 sums.
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

// FP32 views: the same sum in double-float (the old value, then the exact
// products x'_t y_t and -x_t y_t accumulated as pairs), rounded once.  A
// thread takes kRowCols columns c0 .. of one row j, so the factor entries are
// loaded once per row and the loads of U are coalesced over j.
constexpr int kRowCols = 4;
__global__ void xty_update_df_kernel(float* xty, float* xtyl, int64_t ld, float* xtyc, int64_t fs,
                                     const float* U, int n, int p, int k, const float* Yr) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * kRowCols;
  if (j >= n) return;
  df2 acc[kRowCols];
#pragma unroll
  for (int q = 0; q < kRowCols; ++q) {
    const bool ok = c0 + q < p;
    acc[q] = {ok ? xty[(int64_t)j * ld + c0 + q] : 0.f,
              ok && xtyl ? xtyl[(int64_t)j * ld + c0 + q] : 0.f};
  }
  for (int t = 0; t < k; ++t) {
    const float xn = U[(int64_t)t * fs + j], xo = U[(int64_t)(k + t) * fs + j];
#pragma unroll
    for (int q = 0; q < kRowCols; ++q) {
      const float y = c0 + q < p ? Yr[(int64_t)t * p + c0 + q] : 0.f;
      df_acc(acc[q], {xn, 0.f}, y);
      df_acc(acc[q], {-xo, 0.f}, y);
    }
  }
#pragma unroll
  for (int q = 0; q < kRowCols; ++q)
    if (c0 + q < p) {
      const df2 v = df_norm(acc[q]);
      xty[(int64_t)j * ld + c0 + q] = v.hi;
      xtyc[(int64_t)(c0 + q) * fs + j] = v.hi;
      if (xtyl) xtyl[(int64_t)j * ld + c0 + q] = v.lo;  // the pair's low half, if kept
    }
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
// 2k x p row-major, beta row-major (ld).  A thread takes kRowCols columns c0
// .. of one row j: the two G entries of each t are loaded once (coalesced
// over j) and serve both sums; Y_R and H are read from shared memory.
template <typename T>
__global__ void beta_update_kernel(T* beta, int64_t ld, const T* G, int64_t fs, int n, int p,
                                   int k, const T* Yr, const T* H) {
  extern __shared__ __align__(16) unsigned char beta_sm[];
  T* Ys = reinterpret_cast<T*>(beta_sm);  // k x kRowCols
  T* Hs = Ys + k * kRowCols;              // 2k x kRowCols
  const int c0 = blockIdx.y * kRowCols;
  for (int e = threadIdx.x; e < 3 * k * kRowCols; e += blockDim.x) {
    const int r = e / kRowCols, q = e % kRowCols;
    const bool ok = c0 + q < p;
    if (r < k) Ys[e] = ok ? Yr[(int64_t)r * p + c0 + q] : T(0);
    else Hs[e - k * kRowCols] = ok ? H[(int64_t)(r - k) * p + c0 + q] : T(0);
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  T acc[kRowCols] = {};
  for (int t = 0; t < k; ++t) {
    const T g1 = G[(int64_t)t * fs + j], g2 = G[(int64_t)(k + t) * fs + j];
    const T d = g1 - g2;
#pragma unroll
    for (int q = 0; q < kRowCols; ++q) {
      acc[q] += d * Ys[t * kRowCols + q];
      acc[q] += g1 * Hs[t * kRowCols + q];
      acc[q] += g2 * Hs[(k + t) * kRowCols + q];
    }
  }
#pragma unroll
  for (int q = 0; q < kRowCols; ++q)
    if (c0 + q < p) beta[(int64_t)j * ld + c0 + q] += acc[q];
}

// ---------------------------------------------------------------------------
// Newton-Schulz residual correction of FP32 OLS programs: Z = X^T X kept as
// double-float pairs (Zh + Zl, row-major, rows and columns padded to ldz with
// zeros).
// ---------------------------------------------------------------------------

// (Zh, Zl)(i, j) = the pair of L(max(i, j), min(i, j)), L the lower triangle of
// the FP64 X^T X (column-major, ldl) that re-evaluation computes.
__global__ void z_from_lower_kernel(const double* L, int64_t ldl, int n, float* Zh, float* Zl,
                                    int64_t ldz) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  const int r = i > j ? i : j, c = i > j ? j : i;
  const double v = L[r + (int64_t)c * ldl];
  const float h = __double2float_rn(v);
  Zh[(int64_t)i * ldz + j] = h;
  Zl[(int64_t)i * ldz + j] = __double2float_rn(v - (double)h);
}

// Z += Hp Hp^T - Hm Hm^T for the history of replaced rows (Hp: the new rows
// X'_R^T, Hm: the old rows X_R^T of every row block since the last flush, cnt
// columns each, column stride fs, zero past row n): each product of two FP32
// entries is exact as a pair and is accumulated onto the pair (Zh, Zl)
// (df_acc), so Z stays the FP64-grade sum of exact products.  Z is symmetric
// and kept whole: a CTA takes one 64 x 64 tile on or below the diagonal and
// writes it and its mirror image (a diagonal tile is symmetric by itself:
// entries (i, j) and (j, i) take the same products in the same order).  A
// thread holds 4 x 4 entries; the history passes through shared memory 32
// columns at a time.  ldz is a multiple of 64 (whole tiles lie inside).
constexpr int kZTile = 64, kZK = 32;
__global__ void __launch_bounds__(256, 1)
    z_flush_kernel(float* Zh, float* Zl, int64_t ldz, const float* Hp, const float* Hm,
                   int64_t fs, int cnt) {
  __shared__ __align__(16) float Si[kZK][kZTile];
  __shared__ __align__(16) float Sj[kZK][kZTile];
  // blockIdx.x -> (bi, bj), bj <= bi, row-wise over the lower triangle
  int bi = (int)((sqrtf(8.f * blockIdx.x + 1.f) - 1.f) * 0.5f);
  while ((bi + 1) * (bi + 2) / 2 <= (int)blockIdx.x) ++bi;
  while (bi * (bi + 1) / 2 > (int)blockIdx.x) --bi;
  const int bj = (int)blockIdx.x - bi * (bi + 1) / 2;
  const int i0 = bi * kZTile, j0 = bj * kZTile;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  df2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t o = (int64_t)(i0 + 4 * ty + a) * ldz + j0 + 4 * tx;
    const float4 h = *reinterpret_cast<const float4*>(Zh + o);
    const float4 l = *reinterpret_cast<const float4*>(Zl + o);
    acc[a][0] = {h.x, l.x};
    acc[a][1] = {h.y, l.y};
    acc[a][2] = {h.z, l.z};
    acc[a][3] = {h.w, l.w};
  }
  for (int side = 0; side < 2; ++side) {
    const float* H = side ? Hm : Hp;
    const float sg = side ? -1.f : 1.f;
    for (int t0 = 0; t0 < cnt; t0 += kZK) {
      const int nt = min(kZK, cnt - t0);
      __syncthreads();  // the previous chunk's readers are done
      for (int e = threadIdx.x; e < nt * kZTile; e += blockDim.x) {
        const int t = e / kZTile, r = e % kZTile;
        Si[t][r] = H[(int64_t)(t0 + t) * fs + i0 + r];
        Sj[t][r] = H[(int64_t)(t0 + t) * fs + j0 + r];
      }
      __syncthreads();
      for (int t = 0; t < nt; ++t) {
        const float4 ui = *reinterpret_cast<const float4*>(&Si[t][4 * ty]);
        const float4 uj = *reinterpret_cast<const float4*>(&Sj[t][4 * tx]);
        const float av[4] = {sg * ui.x, sg * ui.y, sg * ui.z, sg * ui.w};
        const float bv[4] = {uj.x, uj.y, uj.z, uj.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) df_acc(acc[a][b], {av[a], 0.f}, bv[b]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = df_norm(acc[a][b]);
  const df2(&v)[4][4] = acc;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t o = (int64_t)(i0 + 4 * ty + a) * ldz + j0 + 4 * tx;
    *reinterpret_cast<float4*>(Zh + o) = make_float4(v[a][0].hi, v[a][1].hi, v[a][2].hi, v[a][3].hi);
    *reinterpret_cast<float4*>(Zl + o) = make_float4(v[a][0].lo, v[a][1].lo, v[a][2].lo, v[a][3].lo);
  }
  if (bi != bj) {  // the mirror tile (j0.., i0..)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t o = (int64_t)(j0 + 4 * tx + b) * ldz + i0 + 4 * ty;
      *reinterpret_cast<float4*>(Zh + o) =
          make_float4(v[0][b].hi, v[1][b].hi, v[2][b].hi, v[3][b].hi);
      *reinterpret_cast<float4*>(Zl + o) =
          make_float4(v[0][b].lo, v[1][b].lo, v[2][b].lo, v[3][b].lo);
    }
  }
}

// R = D - Z B for n x n Z (pairs), B n x nb (FP32, row-major ldb) and D the
// identity (Dh null) or the pairs (Dh + Dl, row-major ldd), rounded to FP32
// (ldr): every product of a Z pair and a B entry accumulated as a pair
// (df_acc), so the residual, a difference of nearly equal numbers, keeps ~44
// bits of the sums.  64 x 64 output tiles, K steps of 16 through shared
// memory (Z tile stored K-major), a thread 4 x 4 outputs.
constexpr int kRsTile = 64, kRsK = 16;
__global__ void __launch_bounds__(256)
    ns_residual_kernel(const float* Zh, const float* Zl, int64_t ldz, const float* B, int64_t ldb,
                       int nb, const float* Dh, const float* Dl, int64_t ldd, float* R,
                       int64_t ldr, int n) {
  __shared__ __align__(16) float Ah[kRsK][kRsTile + 4];
  __shared__ __align__(16) float Al[kRsK][kRsTile + 4];
  __shared__ __align__(16) float Bs[kRsK][kRsTile + 4];
  const int i0 = blockIdx.y * kRsTile, j0 = blockIdx.x * kRsTile;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  df2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = {0.f, 0.f};
  for (int k0 = 0; k0 < n; k0 += kRsK) {
    for (int e = threadIdx.x; e < kRsTile * kRsK; e += blockDim.x) {
      const int r = e / kRsK, c = e % kRsK;  // Z(i0 + r, k0 + c)
      const bool ok = i0 + r < n && k0 + c < n;
      const int64_t o = (int64_t)(i0 + r) * ldz + k0 + c;
      Ah[c][r] = ok ? Zh[o] : 0.f;
      Al[c][r] = ok ? Zl[o] : 0.f;
      const int rb = e / kRsTile, cb = e % kRsTile;  // B(k0 + rb, j0 + cb)
      Bs[rb][cb] = (k0 + rb < n && j0 + cb < nb) ? B[(int64_t)(k0 + rb) * ldb + j0 + cb] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < kRsK; ++t) {
      const float4 h = *reinterpret_cast<const float4*>(&Ah[t][4 * ty]);
      const float4 l = *reinterpret_cast<const float4*>(&Al[t][4 * ty]);
      const float4 w = *reinterpret_cast<const float4*>(&Bs[t][4 * tx]);
      const df2 zv[4] = {{h.x, l.x}, {h.y, l.y}, {h.z, l.z}, {h.w, l.w}};
      const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_acc(acc[a][b], zv[a], wv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + 4 * ty + a;
    if (i >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + 4 * tx + b;
      if (j >= nb) continue;
      const df2 d = Dh ? df2{Dh[(int64_t)i * ldd + j], Dl[(int64_t)i * ldd + j]}
                       : df2{i == j ? 1.f : 0.f, 0.f};
      const df2 v = df_sum(d, {-acc[a][b].hi, -acc[a][b].lo});
      R[(int64_t)i * ldr + j] = __fadd_rn(v.hi, v.lo);
    }
  }
}

// lo(i, j) = src(i, j) - (double)(float)src(i, j), rounded to FP32 (src
// row-major FP64, lds): the low halves of a matrix whose FP32 rounding is
// stored elsewhere.
__global__ void low_half_kernel(const double* src, int64_t lds, float* lo, int64_t ldl, int rows,
                                int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  const int i = (int)(idx / cols), j = (int)(idx % cols);
  const double v = src[(int64_t)i * lds + j];
  lo[(int64_t)i * ldl + j] = __double2float_rn(v - (double)__double2float_rn(v));
}

cudaError_t launch_low_half(const double* src, int64_t lds, float* lo, int64_t ldl, int rows,
                            int cols, cudaStream_t s) {
  const int64_t tot = (int64_t)rows * cols;
  if (tot == 0) return cudaSuccess;
  low_half_kernel<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(src, lds, lo,
                                                                                 ldl, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_z_from_lower(const double* L, int64_t ldl, int n, float* Zh, float* Zl,
                                int64_t ldz, cudaStream_t s) {
  const int64_t tot = (int64_t)n * n;
  z_from_lower_kernel<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(L, ldl, n,
                                                                                     Zh, Zl, ldz);
  return cudaGetLastError();
}

cudaError_t launch_z_flush(float* Zh, float* Zl, int64_t ldz, const float* Hp, const float* Hm,
                           int64_t fs, int n, int cnt, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  if (cnt < 0 || ldz % kZTile || fs < ldz) return cudaErrorInvalidValue;
  const int64_t g = (n + kZTile - 1) / kZTile;
  z_flush_kernel<<<(unsigned)(g * (g + 1) / 2), 256, 0, s>>>(Zh, Zl, ldz, Hp, Hm, fs, cnt);
  return cudaGetLastError();
}

cudaError_t launch_ns_residual(const float* Zh, const float* Zl, int64_t ldz, const float* B,
                               int64_t ldb, int nb, const float* Dh, const float* Dl, int64_t ldd,
                               float* R, int64_t ldr, int n, cudaStream_t s) {
  if (nb < 1 || (Dh == nullptr) != (Dl == nullptr)) return cudaErrorInvalidValue;
  const unsigned gy = (unsigned)((n + kRsTile - 1) / kRsTile);
  const unsigned gx = (unsigned)((nb + kRsTile - 1) / kRsTile);
  ns_residual_kernel<<<dim3(gx, gy), 256, 0, s>>>(Zh, Zl, ldz, B, ldb, nb, Dh, Dl, ldd, R, ldr, n);
  return cudaGetLastError();
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
  if (kk < 1 || kk > 64) return cudaErrorInvalidValue;
  static const cudaError_t configured =
      cudaFuncSetAttribute(core_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)core_inverse_smem(64));
  if (configured != cudaSuccess) return configured;
  core_inverse_kernel<<<1, dim3(kInvTx, kInvTy), core_inverse_smem(kk), s>>>(S, kk, kpos, Minv,
                                                                           status);
  return cudaGetLastError();
}

cudaError_t launch_core_inverse_df(const float2* S, int kk, int kpos, float2* Minv,
                                   unsigned* status, cudaStream_t s) {
  if (kk < 1 || kk > 64) return cudaErrorInvalidValue;
  static const cudaError_t configured =
      cudaFuncSetAttribute(core_inverse_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)core_df_smem(64));
  if (configured != cudaSuccess) return configured;
  core_inverse_df_kernel<<<1, kCoreThreads, core_df_smem(kk), s>>>(S, kk, kpos, Minv, status);
  return cudaGetLastError();
}

cudaError_t launch_wu(const double* G, int64_t fs, int n, int kk, const double* Minv, double* Wu,
                      cudaStream_t s) {
  if (kk < 2 || kk > 64 || (kk & 1)) return cudaErrorInvalidValue;
  wu_f64_kernel<<<dim3(blocks_for(n), kk / 2), kThreads, 0, s>>>(G, fs, n, kk, Minv, Wu);
  return cudaGetLastError();
}

cudaError_t launch_wu(const float* G, int64_t fs, int n, int kk, const float2* Minv, float* Wu,
                      cudaStream_t s) {
  if (kk < 2 || kk > 64 || (kk & 1)) return cudaErrorInvalidValue;
  wu_df_kernel<<<dim3(blocks_for(n), (kk + kWuCols - 1) / kWuCols), kThreads, 0, s>>>(G, fs, n,
                                                                                      kk, Minv, Wu);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_beta_update(T* beta, int64_t ld, const T* G, const T* Wu, const T* Cc,
                               int64_t fs, int n, int p, int k, const T* Yr, T* H,
                               cudaStream_t s) {
  wtc_kernel<T><<<(unsigned)(2 * k * p), 256, 0, s>>>(Wu, Cc, fs, n, 2 * k, p, H);
  beta_update_kernel<T>
      <<<dim3(blocks_for(n), (p + kRowCols - 1) / kRowCols), kThreads,
         sizeof(T) * 3 * k * kRowCols, s>>>(beta, ld, G, fs, n, p, k, Yr, H);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xty_update(T* xty, int64_t ld, T* xtyc, int64_t fs, const T* U, int n, int p,
                              int k, const T* Yr, cudaStream_t s, T* xtyl) {
  if constexpr (sizeof(T) == 4)
    xty_update_df_kernel<<<dim3(blocks_for(n), (p + kRowCols - 1) / kRowCols), kThreads, 0, s>>>(
        xty, xtyl, ld, xtyc, fs, U, n, p, k, Yr);
  else
    xty_update_kernel<T><<<blocks_for((int64_t)n * p), kThreads, 0, s>>>(xty, ld, xtyc, fs, U, n,
                                                                         p, k, Yr);
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
  template cudaError_t launch_beta_update<T>(T*, int64_t, const T*, const T*, const T*, int64_t,  \
                                             int, int, int, const T*, T*, cudaStream_t);         \
  template cudaError_t launch_xty_update<T>(T*, int64_t, T*, int64_t, const T*, int, int, int,    \
                                            const T*, cudaStream_t, T*);                         \
  template cudaError_t launch_to_double<T>(const T*, int64_t, double*, int64_t, int, int,         \
                                           cudaStream_t);                                        \
  template cudaError_t launch_sym_lower_to_full<T>(const double*, int64_t, int, T*, int64_t,      \
                                                   double*, int64_t, cudaStream_t);              \
  template cudaError_t launch_from_double<T>(const double*, int64_t, T*, int64_t, int, int, T*,   \
                                             int64_t, cudaStream_t);
LV_OLS_INST(float)
LV_OLS_INST(double)

}  // namespace lv
