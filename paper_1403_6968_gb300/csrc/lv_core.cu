// Factor cores and factor assembly of the exponential model (Appendix A of
// arXiv 1403.6968) and small helpers (ingest, layout changes).
//
//   C_h     = V_h^T U_h                       (r_h x r_h, FP64)
//   U_{2h}  = [U_h, P_h U_h + U_h C_h]         (right block written here)
//   V_{2h}  = [P_h^T V_h, V_h]                 (left block written here)
//
// P_h U_h and P_h^T V_h arrive as per-block partial sums from the view pass;
// they are summed here in a fixed order so every run gives identical bits.
#include <cuda_runtime.h>

#include <type_traits>

#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {

constexpr int kGramRows = 32;   // rows staged per tile
constexpr int kGramMaxR = 64;
constexpr int kGramPerThread = kGramMaxR * kGramMaxR / kThreads;  // 16

// Blocks of the factor-core kernels: one 32-row tile per block up to 320
// blocks (>= 2 per SM), more tiles per block beyond.
int gram_grid(int n) {
  int g = (n + kGramRows - 1) / kGramRows;
  if (g > 320) g = 320;
  if (g < 1) g = 1;
  return g;
}

// FP64 programs: C = V^T U (r x r, row-major, FP64).  Block b sums rows of its
// chunk; the last block to finish (ticket) adds the block partials in index
// order.
__global__ void __launch_bounds__(kThreads) gram_f64_kernel(const double* __restrict__ V,
                                                            const double* __restrict__ U,
                                                            int64_t fs, int n, int r,
                                                            double* Cpart, unsigned* ticket,
                                                            double* C, unsigned* status) {
  __shared__ double Vs[kGramRows][kGramMaxR + 1];
  __shared__ double Us[kGramRows][kGramMaxR + 1];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int chunk = (n + G - 1) / G;
  const int r0 = blockIdx.x * chunk;
  const int r1 = min(n, r0 + chunk);
  const int ne = r * r;
  double acc[kGramPerThread];
#pragma unroll
  for (int i = 0; i < kGramPerThread; ++i) acc[i] = 0.0;
  for (int t0 = r0; t0 < r1; t0 += kGramRows) {
    const int nr = min(kGramRows, r1 - t0);
    for (int idx = tid; idx < kGramRows * r; idx += kThreads) {
      const int c = idx / kGramRows;
      const int j = idx % kGramRows;
      const bool ok = j < nr;
      Vs[j][c] = ok ? V[(int64_t)c * fs + t0 + j] : 0.0;
      Us[j][c] = ok ? U[(int64_t)c * fs + t0 + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kGramPerThread; ++i) {
      const int e = tid + i * kThreads;
      if (e < ne) {
        const int c1 = e / r, c2 = e % r;
        double a = acc[i];
        for (int j = 0; j < nr; ++j) a = fma(Vs[j][c1], Us[j][c2], a);
        acc[i] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kGramPerThread; ++i) {
    const int e = tid + i * kThreads;
    if (e < ne) Cpart[(int64_t)blockIdx.x * ne + e] = acc[i];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket, 1u) == (unsigned)(G - 1));
  __syncthreads();
  if (last) {
    __threadfence();
    for (int e = tid; e < ne; e += kThreads) {
      double sum = 0.0;
      for (int b = 0; b < G; ++b) sum += Cpart[(int64_t)b * ne + e];
      if (!isfinite(sum)) atomicOr(status, kStatusNonFinite);
      C[e] = sum;
    }
    if (tid == 0) *ticket = 0u;
  }
}

// Double-float accumulation (hi + lo, each FP32): the exact product of two
// floats is p + pe with pe = fma(v, u, -p); hi absorbs it by Knuth's TwoSum
// and lo collects the rounding errors, so the sum carries about 44 bits.
// Rounded intrinsics keep the compiler from contracting the error terms.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x, float xe) {
  const float t = __fadd_rn(hi, x);
  const float z = __fsub_rn(t, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(x, z));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(err, xe));
}

// FP32 programs: per-block partials of C = V^T U in double-float.  GB300's
// FP64 pipe is narrow, so the FP64-grade sums use FP32 arithmetic; every
// block of 256 threads takes one 32-row tile per step.
__global__ void __launch_bounds__(kThreads) gram_df_kernel(const float* __restrict__ V,
                                                           const float* __restrict__ U,
                                                           int64_t fs, int n, int r,
                                                           float2* Cpart) {
  __shared__ float Vs[kGramRows][kGramMaxR + 1];
  __shared__ float Us[kGramRows][kGramMaxR + 1];
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int ne = r * r;
  float hi[kGramPerThread], lo[kGramPerThread];
#pragma unroll
  for (int i = 0; i < kGramPerThread; ++i) hi[i] = lo[i] = 0.f;
  for (int t0 = blockIdx.x * kGramRows; t0 < n; t0 += G * kGramRows) {
    const int nr = min(kGramRows, n - t0);
    for (int idx = tid; idx < kGramRows * r; idx += kThreads) {
      const int c = idx / kGramRows;
      const int j = idx % kGramRows;
      const bool ok = j < nr;
      Vs[j][c] = ok ? V[(int64_t)c * fs + t0 + j] : 0.f;
      Us[j][c] = ok ? U[(int64_t)c * fs + t0 + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kGramPerThread; ++i) {
      const int e = tid + i * kThreads;
      if (e < ne) {
        const int c1 = e / r, c2 = e % r;
        float h = hi[i], l = lo[i];
        for (int j = 0; j < nr; ++j) {
          const float v = Vs[j][c1], u = Us[j][c2];
          const float p = __fmul_rn(v, u);
          df_add(h, l, p, __fmaf_rn(v, u, -p));
        }
        hi[i] = h;
        lo[i] = l;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < kGramPerThread; ++i) {
    const int e = tid + i * kThreads;
    if (e < ne) Cpart[(int64_t)blockIdx.x * ne + e] = make_float2(hi[i], lo[i]);
  }
}

// One warp per core entry: lane l adds the partials of blocks l, l + 32, ...
// in order, then a fixed butterfly combines the lanes (lane 0's sum is kept).
__global__ void gram_reduce_kernel(const float2* __restrict__ Cpart, int G, int ne, double* C,
                                   unsigned* status, float2* Cdf) {
  const int e = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= ne) return;  // warp-uniform
  float h = 0.f, l = 0.f;
  for (int b = lane; b < G; b += 32) {
    const float2 x = Cpart[(int64_t)b * ne + e];
    df_add(h, l, x.x, x.y);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
  if (lane == 0) {
    const double sum = (double)h + (double)l;
    if (!isfinite(sum)) atomicOr(status, kStatusNonFinite);
    C[e] = sum;
    if (Cdf) {  // the same sum as a normalised FP32 pair
      const float hh = __fadd_rn(h, l);
      Cdf[e] = make_float2(hh, __fsub_rn(l, __fsub_rn(hh, h)));
    }
  }
}

template <typename T>
cudaError_t launch_gram(const T* V, const T* U, int64_t fs, int n, int r, double* Cpart,
                        unsigned* ticket, double* C, unsigned* status, cudaStream_t s,
                        float2* Cdf) {
  if (r < 1 || r > kGramMaxR) return cudaErrorInvalidValue;
  const int G = gram_grid(n);
  if constexpr (std::is_same<T, float>::value) {
    float2* part = reinterpret_cast<float2*>(Cpart);
    gram_df_kernel<<<G, kThreads, 0, s>>>(V, U, fs, n, r, part);
    const int ne = r * r;
    const int warps_per_block = kThreads / 32;
    gram_reduce_kernel<<<(ne + warps_per_block - 1) / warps_per_block, kThreads, 0, s>>>(
        part, G, ne, C, status, Cdf);
  } else {
    gram_f64_kernel<<<G, kThreads, 0, s>>>(V, U, fs, n, r, Cpart, ticket, C, status);
  }
  return cudaGetLastError();
}

// Assembly of the next level's factor columns, for factor column c and row j:
//   X'(j,c) = sum_s Xpart[s](j,c) + sum_c2 U_h(j,c2) C_h(c2,c),
//   Y(j,c)  = sum_q Ypart[q](j,c),
// with C_h = V_h^T U_h the sum of the nC FP64 partial blocks.  Everything
// read here was written by the kernels just before, so the time is load
// latency, not bandwidth: a CTA takes 32 rows of one column c and its 8 warps
// split the strips s, the row ranges q and the columns c2 (warp w takes those
// congruent to w mod 8), so every thread issues a handful of independent
// loads at once.  The C_h column is summed by groups of 8 lanes over the
// blocks (same split) and a fixed butterfly; the warp partials are added in
// warp order.  All orders are fixed, so the results are reproducible.  The
// sums are in the view type except C_h (FP64, rounded once): FP64 arithmetic
// is slow on this part and buys nothing, the partials themselves being sums
// in the view type.
constexpr int kAsmWarps = kThreads / 32;

// sum over i = w, w + kAsmWarps, ... < count of src[i * stride], in increasing i
template <typename T, typename A>
__device__ __forceinline__ A strided_sum(const T* src, int64_t stride, int count, int w) {
  A acc = A(0);
  constexpr int kU = 4;
  for (int i0 = w; i0 < count; i0 += kU * kAsmWarps) {
    T v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kAsmWarps;
      v[u] = (i < count) ? src[(int64_t)i * stride] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) acc += (A)v[u];
  }
  return acc;
}

// sum over all i < count of src[i * stride], in increasing i (chunks of 8
// independent loads)
template <typename T>
__device__ __forceinline__ T strided_sum_all(const T* src, int64_t stride, int count) {
  T acc = T(0);
  for (int i0 = 0; i0 < count; i0 += 8) {
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (i0 + i < count) ? src[(int64_t)(i0 + i) * stride] : T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += v[i];
  }
  return acc;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) assemble_kernel(const AssembleParams a) {
  __shared__ T Cc[kMaxAsmR];                 // column c of C_h (rounded to T)
  __shared__ T red[3][kAsmWarps][32];        // per-warp partials: X, U_h C_h, Y
  griddep_wait();  // everything read here comes from the kernels before
  griddep_launch_dependents();
  const int rh = a.r_h;
  const int c = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + lane;
  const bool valid = j < a.n;
  const int jj = valid ? j : 0;
  const T* Xp = static_cast<const T*>(a.Xpart);
  const T* Yp = static_cast<const T*>(a.Ypart);
  const T* Uh = static_cast<const T*>(a.Uh);
  // C_h(c2, c): lane group g = threadIdx.x / 8 takes c2 = g, g + 32, ...;
  // its 8 lanes split the blocks (the loop bound is the same for a whole
  // warp, so every lane reaches the shuffles)
  const int ne = rh * rh;
  for (int c2b = warp * 4; c2b < rh; c2b += kThreads / 8) {
    const int c2 = c2b + (lane >> 3);
    double sum = (c2 < rh) ? strided_sum<double, double>(a.C + (int64_t)c2 * rh + c, ne, a.nC,
                                                         lane & 7)
                           : 0.0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((lane & 7) == 0 && c2 < rh) {
      Cc[c2] = (T)sum;
      // every CTA sums the same core: the first one reports a non-finite entry
      if (a.status && blockIdx.x == 0 && !isfinite(sum)) atomicOr(a.status, kStatusNonFinite);
    }
  }
  // this warp's share of the strips, row ranges and columns of U_h
  T x = strided_sum<T, T>(Xp + (int64_t)c * a.part_cs + jj, a.xp_s, a.gC, warp);
  T y = Yp ? strided_sum<T, T>(Yp + (int64_t)c * a.part_cs + jj, a.yp_q, a.gR, warp) : T(0);
  T u[kMaxAsmR / kAsmWarps];
#pragma unroll
  for (int i = 0; i < kMaxAsmR / kAsmWarps; ++i) {
    const int c2 = warp + i * kAsmWarps;
    u[i] = (c2 < rh) ? Uh[(int64_t)c2 * a.fs + jj] : T(0);
  }
  __syncthreads();  // Cc complete
  T uc = T(0);
#pragma unroll
  for (int i = 0; i < kMaxAsmR / kAsmWarps; ++i) {
    const int c2 = warp + i * kAsmWarps;
    if (c2 < rh) uc = fma(u[i], Cc[c2], uc);
  }
  red[0][warp][lane] = x;
  red[1][warp][lane] = uc;
  red[2][warp][lane] = y;
  __syncthreads();
  if (warp != 0 || !valid) return;
  T xs = T(0), us = T(0), ys = T(0);
#pragma unroll
  for (int w = 0; w < kAsmWarps; ++w) {
    xs += red[0][w][lane];
    us += red[1][w][lane];
    ys += red[2][w][lane];
  }
  static_cast<T*>(a.Unew)[(int64_t)c * a.fs + j] = xs + us;
  if (Yp) static_cast<T*>(a.Ynew)[(int64_t)c * a.fs + j] = ys;
}

// The same assembly for wide blocks (r_out >= 8): there are enough outputs
// to fill the GPU with one thread per (j, c), which then sums all partials
// itself (CTA = 256 rows of one column; the C_h column is summed once per
// CTA).  Same fixed orders as above within a thread's sums.
template <typename T>
__global__ void __launch_bounds__(kThreads) assemble_wide_kernel(const AssembleParams a) {
  __shared__ T Cc[kMaxAsmR];
  griddep_wait();
  griddep_launch_dependents();
  const int rh = a.r_h;
  const int c = blockIdx.y;
  const int j = blockIdx.x * kThreads + threadIdx.x;
  const bool valid = j < a.n;
  const int jj = valid ? j : 0;
  const T* Xp = static_cast<const T*>(a.Xpart);
  const T* Yp = static_cast<const T*>(a.Ypart);
  const T* Uh = static_cast<const T*>(a.Uh);
  const int ne = rh * rh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c2b = warp * 4; c2b < rh; c2b += kThreads / 8) {
    const int c2 = c2b + (lane >> 3);
    double sum = (c2 < rh) ? strided_sum<double, double>(a.C + (int64_t)c2 * rh + c, ne, a.nC,
                                                         lane & 7)
                           : 0.0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((lane & 7) == 0 && c2 < rh) {
      Cc[c2] = (T)sum;
      // every CTA sums the same core: the first one reports a non-finite entry
      if (a.status && blockIdx.x == 0 && !isfinite(sum)) atomicOr(a.status, kStatusNonFinite);
    }
  }
  T x = strided_sum_all<T>(Xp + (int64_t)c * a.part_cs + jj, a.xp_s, a.gC);
  T y = Yp ? strided_sum_all<T>(Yp + (int64_t)c * a.part_cs + jj, a.yp_q, a.gR) : T(0);
  __syncthreads();
  if (!valid) return;
  T uc = T(0);
  for (int c0 = 0; c0 < rh; c0 += 8) {
    T u[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) u[i] = (c0 + i < rh) ? Uh[(int64_t)(c0 + i) * a.fs + j] : T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c0 + i < rh) uc = fma(u[i], Cc[c0 + i], uc);
  }
  static_cast<T*>(a.Unew)[(int64_t)c * a.fs + j] = x + uc;
  if (Yp) static_cast<T*>(a.Ynew)[(int64_t)c * a.fs + j] = y;
}

template <typename T>
cudaError_t launch_assemble(const AssembleParams& a, cudaStream_t s) {
  if (a.r_h > kMaxAsmR) return cudaErrorInvalidValue;
  const int ro = a.r_out > 0 ? a.r_out : a.r_h;
  cudaError_t e;
  if (ro >= 8) {
    const dim3 grid((unsigned)((a.n + kThreads - 1) / kThreads), (unsigned)ro);
    e = launch_pdl(assemble_wide_kernel<T>, grid, kThreads, 0, s, a);
  } else {
    const dim3 grid((unsigned)((a.n + 31) / 32), (unsigned)ro);
    e = launch_pdl(assemble_kernel<T>, grid, kThreads, 0, s, a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

constexpr int kChunk = 16;  // independent loads issued together

// W = V K^T for the block-upper-triangular K of identity blocks (width r_in):
// block b of W is the sum of blocks b .. nblk-1 of V, added from the last
// block down in the element type.  One thread per (row, column in block).
template <typename T>
__global__ void suffix_sums_kernel(const T* __restrict__ V, T* __restrict__ W, int64_t fs, int n,
                                   int width, int r_in) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * r_in) return;
  int c, j;
  split_index(idx, n, c, j);
  const int nblk = width / r_in;
  // the blocks are read in chunks of independent loads (V and W do not
  // overlap), then summed from the last block down
  T acc = T(0);
  for (int b1 = nblk; b1 > 0; b1 -= kChunk) {
    T v[kChunk];
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int b = b1 - 1 - i;
      v[i] = (b >= 0) ? V[(int64_t)(b * r_in + c) * fs + j] : T(0);
    }
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int b = b1 - 1 - i;
      if (b >= 0) {
        acc += v[i];
        W[(int64_t)(b * r_in + c) * fs + j] = acc;
      }
    }
  }
}

template <typename T>
cudaError_t launch_suffix_sums(const T* V, T* W, int64_t fs, int n, int width, int r_in,
                               cudaStream_t s) {
  const int64_t tot = (int64_t)n * r_in;
  suffix_sums_kernel<T><<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      V, W, fs, n, width, r_in);
  return cudaGetLastError();
}

template <typename T>
__global__ void rm_to_cm_kernel(const T* src, int64_t ld, T* dst, int64_t fs, int rows, int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int c, j;
  split_index(idx, rows, c, j);
  dst[(int64_t)c * fs + j] = src[(int64_t)j * ld + c];
}

template <typename T>
cudaError_t launch_rm_to_cm(const T* src, int64_t ld, T* dst, int64_t fs, int rows, int cols,
                            cudaStream_t s) {
  const int64_t tot = (int64_t)rows * cols;
  if (tot == 0) return cudaSuccess;
  rm_to_cm_kernel<T><<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      src, ld, dst, fs, rows, cols);
  return cudaGetLastError();
}

template <typename T>
__global__ void unit_column_kernel(T* dst, int n, int row) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = (j == row) ? T(1) : T(0);
}

template <typename T>
cudaError_t launch_unit_column(T* dst, int n, int row, cudaStream_t s) {
  unit_column_kernel<T><<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(dst, n, row);
  return cudaGetLastError();
}

template <typename T>
__global__ void sum_partials_kernel(const T* part, int blocks, int64_t bs, int64_t cs, int n,
                                    int r, T* out, int64_t ocs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * r) return;
  int c, j;
  split_index(idx, n, c, j);
  double acc = 0.0;
  for (int b = 0; b < blocks; ++b) acc += (double)part[(int64_t)b * bs + (int64_t)c * cs + j];
  out[(int64_t)c * ocs + j] = (T)acc;
}

// FP32 partials: a cascaded sum in FP32 pairs (each addition's rounding
// error, exact by TwoSum, is carried in a second accumulator), so the total
// is FP32-rounded from a ~48-bit sum without GB300's narrow FP64 pipe (some
// passes leave a few dozen partials per entry).
__global__ void sum_partials_f32_kernel(const float* part, int blocks, int64_t bs, int64_t cs,
                                        int n, int r, float* out, int64_t ocs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * r) return;
  int c, j;
  split_index(idx, n, c, j);
  float hi = 0.f, lo = 0.f;
  auto add = [&](float x) {
    const float t = __fadd_rn(hi, x);
    const float bb = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
    hi = t;
  };
  const float* src = part + (int64_t)c * cs + j;
  int b = 0;
  for (; b + 8 <= blocks; b += 8) {  // eight loads in flight, added in order
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = src[(int64_t)(b + i) * bs];
#pragma unroll
    for (int i = 0; i < 8; ++i) add(x[i]);
  }
  for (; b < blocks; ++b) add(src[(int64_t)b * bs]);
  out[(int64_t)c * ocs + j] = __fadd_rn(hi, lo);
}

template <typename T>
cudaError_t launch_sum_partials(const T* part, int blocks, int64_t block_stride, int64_t cs, int n,
                                int r, T* out, int64_t out_cs, cudaStream_t s) {
  const int64_t tot = (int64_t)n * r;
  if (tot == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((tot + kThreads - 1) / kThreads);
  if constexpr (sizeof(T) == 4)
    sum_partials_f32_kernel<<<grid, kThreads, 0, s>>>(part, blocks, block_stride, cs, n, r, out,
                                                      out_cs);
  else
    sum_partials_kernel<T><<<grid, kThreads, 0, s>>>(part, blocks, block_stride, cs, n, r, out,
                                                      out_cs);
  return cudaGetLastError();
}

template <typename T>
__global__ void axpy_rows_kernel(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                                 int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int i, c;
  split_index(idx, cols, i, c);
  y[(int64_t)i * ldy + c] += alpha * x[(int64_t)i * ldx + c];
}

template <typename T>
cudaError_t launch_axpy_rows(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                             int cols, cudaStream_t s) {
  const int64_t tot = (int64_t)rows * cols;
  if (tot == 0) return cudaSuccess;
  axpy_rows_kernel<T><<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      y, ldy, x, ldx, alpha, rows, cols);
  return cudaGetLastError();
}

template <typename T>
__global__ void scale_copy_kernel(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                                  int cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int i, c;
  split_index(idx, cols, i, c);
  y[(int64_t)i * ldy + c] = alpha * x[(int64_t)i * ldx + c];
}

template <typename T>
cudaError_t launch_scale_copy(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                              int cols, cudaStream_t s) {
  const int64_t tot = (int64_t)rows * cols;
  if (tot == 0) return cudaSuccess;
  scale_copy_kernel<T><<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      y, ldy, x, ldx, alpha, rows, cols);
  return cudaGetLastError();
}

// Diagnostic of the bounded waits: one thread waits on an mbarrier that no
// thread or copy ever completes; the wait gives up after limit_ns, latches
// the timeout bit in *status exactly as a view pass does, and reports how
// long it waited.  Nothing faults and the context stays usable.
__global__ void bounded_wait_probe_kernel(uint64_t limit_ns, unsigned* status,
                                          unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    const bool done = mbar_wait_bounded(&bar, 0, status, limit_ns);
    *waited_ns = done ? 0ull : (unsigned long long)(global_ns() - t0);
  }
}

cudaError_t launch_bounded_wait_probe(uint64_t limit_ns, unsigned* status,
                                      unsigned long long* waited_ns, cudaStream_t s) {
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(limit_ns, status, waited_ns);
  return cudaGetLastError();
}

// T panel update of the linear iteration model, all views in one launch:
// T_i += [K_0 .. K_{i-1}] [M blocks]^T for i = 1..k, i.e.
//   T_i(j, q) = Tp[j ldT + i p + q] += sum_{t < i r} K[t fs + j] M[((k - i) r + t) ldm + q]
// (App. B, linear model: view i takes the first i Krylov blocks and the i
// newest M blocks).  A CTA takes 16 rows j and 64 columns q of every view;
// the 16 x k r Krylov rows and the k r x 64 slice of M are staged in shared
// memory once for all k views.  A thread owns 4 adjacent columns of one row
// (one broadcast K load and one 128-bit M load per 4 FMAs) and loads the T
// entries of 8 views at once before it updates them.  Sums over t in
// increasing order, in T.
constexpr int kPanelRows = 16, kPanelQ = 64;

template <typename T>
__global__ void __launch_bounds__(256)
    panel_update_kernel(T* Tp, int64_t ldT, const T* K, int64_t fs, const T* M, int64_t ldm,
                        int n, int p, int k, int r) {
  extern __shared__ __align__(16) unsigned char panel_sm[];
  const int KR = k * r;
  T* Ks = reinterpret_cast<T*>(panel_sm);  // [kPanelRows][KR]
  T* Ms = Ks + kPanelRows * KR;            // [KR][kPanelQ]
  const int j0 = blockIdx.x * kPanelRows, q0 = blockIdx.y * kPanelQ;
  for (int e = threadIdx.x; e < kPanelRows * KR; e += blockDim.x) {
    const int jr = e % kPanelRows, t = e / kPanelRows;  // coalesced down a Krylov column
    Ks[jr * KR + t] = (j0 + jr < n) ? K[(int64_t)t * fs + j0 + jr] : T(0);
  }
  for (int e = threadIdx.x; e < KR * kPanelQ; e += blockDim.x) {
    const int q = e % kPanelQ, t = e / kPanelQ;
    Ms[t * kPanelQ + q] = (q0 + q < p) ? M[(int64_t)t * ldm + q0 + q] : T(0);
  }
  __syncthreads();
  const int jr = threadIdx.x / 16, qa = 4 * (threadIdx.x % 16);
  const int j = j0 + jr;
  if (j >= n || q0 + qa >= p) return;
  const int nq = (p - q0 - qa) < 4 ? p - q0 - qa : 4;  // columns of this thread in the view
  const T* kr = Ks + jr * KR;
  T* trow = Tp + (int64_t)j * ldT + q0 + qa;
  constexpr int VB = 8;  // views per group: their T loads are in flight together
  for (int i0 = 1; i0 <= k; i0 += VB) {
    T tv[VB][4];
#pragma unroll
    for (int v = 0; v < VB; ++v)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (i0 + v <= k && c < nq) tv[v][c] = trow[(int64_t)(i0 + v) * p + c];
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      const int i = i0 + v;
      if (i > k) break;
      const T* mi = Ms + (k - i) * r * kPanelQ + qa;
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      for (int t = 0; t < i * r; ++t) {
        const T kv = kr[t];
        const T* mt = mi + t * kPanelQ;
        a0 += kv * mt[0];
        a1 += kv * mt[1];
        a2 += kv * mt[2];
        a3 += kv * mt[3];
      }
      const T av[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < nq) trow[(int64_t)i * p + c] = tv[v][c] + av[c];
    }
  }
}

// M_i = T_i^T V of the linear iteration model, all views in one pass over
// the T panel (App. B: V_{i+1} = [T_i^T V_1, V_i]): for i < k, c < r, q < p,
//   M[((k - 1 - i) r + c) ldm + q] = sum_j Tp[j ldT + i p + q] V[c fs + j],
// as partial sums over blocks of ``rows`` rows (part[b][col][q], column
// stride p) that launch_sum_partials adds in block order.  A thread owns
// column q of one view (4 views per CTA, grid z over the views); V's rows of
// the block are staged in shared memory (r <= 8).
template <typename T>
__global__ void __launch_bounds__(256)
    panel_tv_kernel(const T* Tp, int64_t ldT, const T* V, int64_t fs, T* part, int n, int p,
                    int k, int r, int rows) {
  extern __shared__ __align__(16) unsigned char tv_sm[];
  T* Vs = reinterpret_cast<T*>(tv_sm);  // [rows][8]
  const int j0 = blockIdx.x * rows, q0 = blockIdx.y * 64;
  for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
    const int jr = e % rows, c = e / rows;
    Vs[jr * 8 + c] = (j0 + jr < n) ? V[(int64_t)c * fs + j0 + jr] : T(0);
  }
  __syncthreads();
  const int q = q0 + (int)(threadIdx.x % 64);
  const int i = (int)blockIdx.z * 4 + (int)(threadIdx.x / 64);
  if (q >= p || i >= k) return;
  const int nr = (n - j0 < rows) ? n - j0 : rows;
  T* pb = part + (int64_t)blockIdx.x * k * r * p;
  {
    T acc[8] = {};
    const T* tcol = Tp + (int64_t)j0 * ldT + (int64_t)i * p + q;
#pragma unroll 8
    for (int jr = 0; jr < nr; ++jr) {
      const T t = tcol[(int64_t)jr * ldT];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] += t * Vs[jr * 8 + c];
    }
    for (int c = 0; c < r; ++c) pb[((int64_t)(k - 1 - i) * r + c) * p + q] = acc[c];
  }
}

// blocks of about n / 128 rows (at least 64, at most 768, so that V's staged
// rows stay within 48 KB of shared memory in FP64)
int panel_tv_blocks(int n) {
  int rows = (n + 127) / 128;
  rows = rows < 64 ? 64 : (rows + 7) / 8 * 8;
  if (rows > 768) rows = 768;
  return (n + rows - 1) / rows;
}

template <typename T>
cudaError_t launch_panel_tv(const T* Tp, int64_t ldT, const T* V, int64_t fs, T* part, T* M,
                            int64_t ldm, int n, int p, int k, int r, cudaStream_t s) {
  if (r < 1 || r > 8 || k < 1 || p < 1) return cudaErrorInvalidValue;
  const int nb = panel_tv_blocks(n);
  const int rows = (n + nb - 1) / nb;
  const dim3 grid((unsigned)nb, (unsigned)((p + 63) / 64), (unsigned)((k + 3) / 4));
  panel_tv_kernel<T><<<grid, 256, sizeof(T) * (size_t)rows * 8, s>>>(Tp, ldT, V, fs, part, n, p,
                                                                     k, r, rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_partials<T>(part, nb, (int64_t)k * r * p, p, p, k * r, M, ldm, s);
}

// largest dynamic shared memory a block of this device may opt in to
static int smem_optin_max() {
  static const int v = [] {
    int dev = 0, b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      return 49152;
    }
    return b;
  }();
  return v;
}

bool panel_update_fits(int k, int r, size_t elem_bytes) {
  return elem_bytes * (size_t)(kPanelRows + kPanelQ) * (size_t)k * (size_t)r <=
         (size_t)smem_optin_max();
}

template <typename T>
cudaError_t launch_panel_update(T* Tp, int64_t ldT, const T* K, int64_t fs, const T* M,
                                int64_t ldm, int n, int p, int k, int r, cudaStream_t s) {
  if (n <= 0 || p <= 0 || k < 1 || r < 1) return cudaSuccess;
  if (!panel_update_fits(k, r, sizeof(T))) return cudaErrorInvalidValue;
  const size_t smem = sizeof(T) * (size_t)(kPanelRows + kPanelQ) * k * r;
  if (smem > 49152) {  // opt in once, to the device's limit
    static const cudaError_t configured = cudaFuncSetAttribute(
        panel_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
    if (configured != cudaSuccess) return configured;
  }
  const dim3 grid((unsigned)((n + kPanelRows - 1) / kPanelRows),
                  (unsigned)((p + kPanelQ - 1) / kPanelQ));
  panel_update_kernel<T><<<grid, 256, smem, s>>>(Tp, ldT, K, fs, M, ldm, n, p, k, r);
  return cudaGetLastError();
}

#define LV_INST(T)                                                                              \
  template cudaError_t launch_gram<T>(const T*, const T*, int64_t, int, int, double*, unsigned*, \
                                      double*, unsigned*, cudaStream_t, float2*);               \
  template cudaError_t launch_assemble<T>(const AssembleParams&, cudaStream_t);                  \
  template cudaError_t launch_suffix_sums<T>(const T*, T*, int64_t, int, int, int, cudaStream_t); \
  template cudaError_t launch_rm_to_cm<T>(const T*, int64_t, T*, int64_t, int, int,               \
                                          cudaStream_t);                                        \
  template cudaError_t launch_unit_column<T>(T*, int, int, cudaStream_t);                        \
  template cudaError_t launch_sum_partials<T>(const T*, int, int64_t, int64_t, int, int, T*,      \
                                              int64_t, cudaStream_t);                           \
  template cudaError_t launch_axpy_rows<T>(T*, int64_t, const T*, int64_t, T, int, int,           \
                                           cudaStream_t);                                       \
  template cudaError_t launch_scale_copy<T>(T*, int64_t, const T*, int64_t, T, int, int,          \
                                            cudaStream_t);                                      \
  template cudaError_t launch_panel_update<T>(T*, int64_t, const T*, int64_t, const T*, int64_t, \
                                              int, int, int, int, cudaStream_t);                \
  template cudaError_t launch_panel_tv<T>(const T*, int64_t, const T*, int64_t, T*, T*, int64_t, \
                                          int, int, int, int, cudaStream_t);
LV_INST(float)
LV_INST(double)

}  // namespace lv
