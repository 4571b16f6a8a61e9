// View passes of the exponential model (Appendix A of arXiv 1403.6968).
//
// One pass streams a maintained n x n view P (row-major) through shared
// memory exactly once and, from that single read, produces
//   X = P Xf      (row sums: P_h U_h, the right block of U_{2h})
//   Y = P^T Yf    (column sums: P_h^T V_h, the left block of V_{2h})
// on the view *before* the update, and writes P + Uu Wu^T back in place
// (the "+=" statements of Example 3.8).  The update-only pass does the last
// part alone (final P_k += U_k V_k^T and the sums views).
//
// Layout / schedule (GB300, sm_103a):
//  * The grid tiles P into gC column strips x gR row ranges; one CTA owns one
//    (strip, row range) block and walks down it in batches of kBatch rows.
//  * A single thread feeds a kStages-deep ring of shared-memory stages with
//    2-D TMA box loads (cp.async.bulk.tensor, 1 KB x kBatch rows per box),
//    completing on one mbarrier per stage; every wait is bounded.
//  * Each thread owns a fixed group of adjacent columns (one 16-byte vector)
//    for the whole CTA: the Xf and Wu rows of those columns live in
//    registers, and the column sums Y accumulate in registers across all rows.
//  * Row sums X are reduced across the CTA through a shared-memory buffer
//    (one warp per row of the batch, conflict-free, fixed order) and written
//    as per-strip partials; column sums are written as per-row-range
//    partials.  A separate assembly kernel sums the partials in fixed order,
//    so results are bitwise reproducible run to run.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {

template <typename T>
__host__ __device__ constexpr int box_cols() {
  return kBoxBytes / (int)sizeof(T);
}

// ---------------------------------------------------------------------------
// Fused products (+ optional update) pass.  Two row groups of 128 threads;
// thread (rg, tc) owns columns strip0 + tc*COLS .. +COLS-1 and processes rows
// rg, rg+2, ... of every batch.
// ---------------------------------------------------------------------------
template <typename T, int R, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
    fused_pass_kernel(const __grid_constant__ CUtensorMap tmap, const PassParams p) {
  constexpr int COLS = Vec<T>::N;  // one 16-byte vector per thread and row
  constexpr int STRIP = 128 * COLS;
  constexpr int BOXC = box_cols<T>();
  constexpr int NB = STRIP / BOXC;
  constexpr int STAGE_ELEMS = kBatch * STRIP;
  constexpr bool DO_X = (MODE & 1) != 0;
  constexpr bool DO_Y = (MODE & 2) != 0;
  constexpr bool DO_U = (MODE & 4) != 0;
  static_assert(NB * BOXC == STRIP, "strip must be whole boxes");
  static_assert(32 % R == 0 && R <= 32, "R must divide a warp");
  // row-sum pieces are stored [batch row][factor column][thread] with a
  // column stride of 128 + 32/R words: stores (consecutive threads) and the
  // reduction reads (R columns x 32/R threads per warp) are both conflict-free
  constexpr int XS = 128 + 32 / R;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * kStages * STAGE_ELEMS);
  T* Us = reinterpret_cast<T*>(full + kStages);  // [kBatch][R] update-left rows
  T* Vs = Us + kBatch * R;                        // [kBatch][R] Y-factor rows
  T* Xbuf = Vs + kBatch * R;                      // [kBatch][R][XS] row-sum pieces
  double* Csh = reinterpret_cast<double*>(Xbuf + kBatch * R * XS);  // [R*R] factor-core sums

  const int tid = threadIdx.x;
  const int rg = tid >> 7;
  const int tc = tid & 127;
  const int s = blockIdx.x % p.gC;
  const int q = blockIdx.x / p.gC;
  const int n = p.n;
  const int r = p.r;
  const int rb = q * p.rows_per_cta;
  const int re = min(n, rb + p.rows_per_cta);
  if (rb >= re) return;
  const int strip0 = s * STRIP;
  const int col0 = strip0 + tc * COLS;
  const int nbatch = (re - rb + kBatch - 1) / kBatch;
  const T* Xf = static_cast<const T*>(p.Xf);
  const T* Yf = static_cast<const T*>(p.Yf);
  const T* Uu = static_cast<const T*>(p.Uu);
  const T* Wu = static_cast<const T*>(p.Wu);
  T* P = static_cast<T*>(p.P);

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // launched with programmatic stream serialisation: everything below may
  // read what the kernel before wrote
  griddep_wait();
  griddep_launch_dependents();

  // boxes of this strip that lie inside the matrix
  int nbox = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) nbox += (strip0 + b * BOXC < n) ? 1 : 0;
  const uint32_t stage_bytes = (uint32_t)(nbox * kBatch * BOXC * sizeof(T));

  auto issue = [&](int b) {
    const int st = b % kStages;
    T* dst = stages + st * STAGE_ELEMS;
    mbar_arrive_expect_tx(&full[st], stage_bytes);
#pragma unroll
    for (int bx = 0; bx < NB; ++bx) {
      if (strip0 + bx * BOXC < n)
        tma_load_2d(dst + bx * kBatch * BOXC, &tmap, strip0 + bx * BOXC, rb + b * kBatch,
                    &full[st]);
    }
  };
  if (tid == 0) {
    for (int b = 0; b < kStages && b < nbatch; ++b) issue(b);
  }

  // per-thread column-side factors
  T ucol[COLS][R];
  T vcol[COLS][R];
  T yacc[COLS][R];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int col = col0 + k;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const bool ok = (c < r) && (col < n);
      ucol[k][c] = (DO_X && ok) ? Xf[(int64_t)c * p.fs + col] : T(0);
      vcol[k][c] = (DO_U && ok) ? Wu[(int64_t)c * p.fs + col] : T(0);
      yacc[k][c] = T(0);
    }
  }
  const int box = (tc * COLS) / BOXC;
  const int inbox = (tc * COLS) % BOXC;
  const bool vec_ok = (col0 + COLS <= n);
  // C = V^T U over this CTA's rows (FP64): every CTA holds exactly those rows
  // of both factors in shared memory; the r*r entries are dealt out over the
  // gC column strips (entry e goes to strip e % gC), so the FP64 work is
  // spread evenly and each entry of the [gR][r*r] partials is written once
  const int ecore = s + tid * p.gC;
  const bool do_core = DO_U && DO_Y && (p.Cpart != nullptr) && (ecore < r * r);
  if (do_core) Csh[tid] = 0.0;  // read back only by the same thread

  int issued = min(kStages, nbatch);
  for (int b = 0; b < nbatch; ++b) {
    const int st = b % kStages;
    const uint32_t parity = (uint32_t)((b / kStages) & 1);
    const int row0 = rb + b * kBatch;
    const int nb = min(kBatch, re - row0);
    // stage the row-side factor entries of this batch
    for (int idx = tid; idx < kBatch * R; idx += kThreads) {
      const int c = idx / kBatch;
      const int j = idx % kBatch;
      const bool ok = (j < nb) && (c < r);
      if (DO_U) Us[j * R + c] = ok ? Uu[(int64_t)c * p.fs + row0 + j] : T(0);
      if (DO_Y) Vs[j * R + c] = ok ? Yf[(int64_t)c * p.fs + row0 + j] : T(0);
    }
    const bool ok = mbar_wait_bounded(&full[st], parity, p.status);
    if (__syncthreads_or(!ok)) {
      // lost transaction: drain what is still in flight (bounded) and leave
      if (tid == 0) {
        for (int bb = b + 1; bb < issued; ++bb)
          mbar_wait_bounded(&full[bb % kStages], (uint32_t)((bb / kStages) & 1), nullptr);
      }
      return;
    }
    if (do_core) {
      const int c1 = ecore / r, c2 = ecore % r;
      double acc = Csh[tid];
#pragma unroll
      for (int j = 0; j < kBatch; ++j)
        acc = fma((double)Vs[j * R + c1], (double)Us[j * R + c2], acc);
      Csh[tid] = acc;
    }
    const T* sp = stages + st * STAGE_ELEMS + box * kBatch * BOXC + inbox;
#pragma unroll
    for (int jj = 0; jj < kBatch / 2; ++jj) {
      const int j = rg + 2 * jj;
      T xp[R];
#pragma unroll
      for (int c = 0; c < R; ++c) xp[c] = T(0);
      if (j < nb) {
        T pv[COLS];
        const typename Vec<T>::type v4 =
            *reinterpret_cast<const typename Vec<T>::type*>(sp + j * BOXC);
        const T* pe = reinterpret_cast<const T*>(&v4);
#pragma unroll
        for (int k = 0; k < COLS; ++k) pv[k] = (col0 + k < n) ? pe[k] : T(0);
        if (DO_Y) {
          T vr[R];
#pragma unroll
          for (int c = 0; c < R; ++c) vr[c] = Vs[j * R + c];
#pragma unroll
          for (int k = 0; k < COLS; ++k)
#pragma unroll
            for (int c = 0; c < R; ++c) yacc[k][c] = fma(pv[k], vr[c], yacc[k][c]);
        }
        if (DO_X) {
#pragma unroll
          for (int k = 0; k < COLS; ++k)
#pragma unroll
            for (int c = 0; c < R; ++c) xp[c] = fma(pv[k], ucol[k][c], xp[c]);
        }
        if (DO_U) {
          T ur[R];
#pragma unroll
          for (int c = 0; c < R; ++c) ur[c] = Us[j * R + c];
          T pn[COLS];
#pragma unroll
          for (int k = 0; k < COLS; ++k) {
            T acc = pv[k];
#pragma unroll
            for (int c = 0; c < R; ++c) acc = fma(ur[c], vcol[k][c], acc);
            pn[k] = acc;
          }
          T* dst = P + (int64_t)(row0 + j) * p.ldp + col0;
          if (vec_ok) {
            typename Vec<T>::type o;
            T* oe = reinterpret_cast<T*>(&o);
#pragma unroll
            for (int k = 0; k < COLS; ++k) oe[k] = pn[k];
            *reinterpret_cast<typename Vec<T>::type*>(dst) = o;
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k)
              if (col0 + k < n) dst[k] = pn[k];
          }
        }
      }
      if (DO_X) {
#pragma unroll
        for (int c = 0; c < R; ++c) Xbuf[(j * R + c) * XS + tc] = xp[c];
      }
    }
    __syncthreads();  // stage consumed, Xbuf complete
    if (tid == 0 && b + kStages < nbatch) {
      fence_proxy_async();
      issue(b + kStages);
      ++issued;
    }
    if (DO_X) {
      // warp w reduces the row-sum pieces of batch row w (fixed order)
      const int w = tid >> 5;
      const int lane = tid & 31;
      constexpr int L = 32 / R;
      const int c = lane % R;
      const int ts = lane / R;
      T sum = T(0);
#pragma unroll 4
      for (int t = ts; t < 128; t += L) sum += Xbuf[(w * R + c) * XS + t];
#pragma unroll
      for (int off = R; off < 32; off <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
      if (ts == 0 && w < nb && c < r) {
        T* xo = static_cast<T*>(p.Xpart);
        xo[(int64_t)s * p.xp_s + (int64_t)c * p.part_cs + row0 + w] = sum;
      }
    }
    // the next iteration's __syncthreads_or orders Xbuf / Us / Vs reuse
  }

  if (do_core) p.Cpart[(int64_t)q * r * r + ecore] = Csh[tid];
  if (DO_Y) {
    __syncthreads();
    T* yc = Xbuf;  // reuse: COLS * R * 128 <= kBatch * R * XS, layout [k][c][tc]
    if (rg == 1) {
#pragma unroll
      for (int k = 0; k < COLS; ++k)
#pragma unroll
        for (int c = 0; c < R; ++c) yc[(k * R + c) * 128 + tc] = yacc[k][c];
    }
    __syncthreads();
    if (rg == 0 && col0 < n) {
      T* yo = static_cast<T*>(p.Ypart) + (int64_t)q * p.yp_q;
#pragma unroll
      for (int c = 0; c < R; ++c) {
        if (c >= r) break;
        T vals[COLS];
#pragma unroll
        for (int k = 0; k < COLS; ++k) vals[k] = yacc[k][c] + yc[(k * R + c) * 128 + tc];
        T* dst = yo + (int64_t)c * p.part_cs + col0;
        if (vec_ok) {
          typename Vec<T>::type o;
          T* oe = reinterpret_cast<T*>(&o);
#pragma unroll
          for (int k = 0; k < COLS; ++k) oe[k] = vals[k];
          *reinterpret_cast<typename Vec<T>::type*>(dst) = o;
        } else {
#pragma unroll
          for (int k = 0; k < COLS; ++k)
            if (col0 + k < n) dst[k] = vals[k];
        }
      }
    }
  }
}

// w[:, c] += w[:, c + RI] from the last column down: block suffix sums
template <typename T, int R, int COLS, int RI>
__device__ __forceinline__ void suffix_blocks(T (&w)[COLS][R]) {
  if constexpr (RI < R) {
#pragma unroll
    for (int c = R - 1 - RI; c >= 0; --c)
#pragma unroll
      for (int k = 0; k < COLS; ++k) w[k][c] += w[k][c + RI];
  }
}

// ---------------------------------------------------------------------------
// Update-only pass: P += Uu Wu^T with R up to 64.  One row group of 256
// threads; thread t owns columns strip0 + t*COLS .. +COLS-1.
// ---------------------------------------------------------------------------
template <typename T, int R, int COLS>
__global__ void __launch_bounds__(kThreads, 2)
    update_pass_kernel(const __grid_constant__ CUtensorMap tmap, const PassParams p) {
  constexpr int STRIP = kThreads * COLS;
  constexpr int BOXC = box_cols<T>();
  constexpr int NB = STRIP / BOXC;
  constexpr int STAGE_ELEMS = kBatch * STRIP;
  static_assert(NB * BOXC == STRIP, "strip must be whole boxes");

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * kStages * STAGE_ELEMS);
  T* Us = reinterpret_cast<T*>(full + kStages);  // [kBatch][R]

  const int tid = threadIdx.x;
  const int s = blockIdx.x % p.gC;
  const int q = blockIdx.x / p.gC;
  const int n = p.n;
  const int r = p.r;
  const int rb = q * p.rows_per_cta;
  const int re = min(n, rb + p.rows_per_cta);
  if (rb >= re) return;
  const int strip0 = s * STRIP;
  const int col0 = strip0 + tid * COLS;
  const int nbatch = (re - rb + kBatch - 1) / kBatch;
  const T* Uu = static_cast<const T*>(p.Uu);
  const T* Wu = static_cast<const T*>(p.Wu);
  T* P = static_cast<T*>(p.P);

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // launched with programmatic stream serialisation: everything below may
  // read what the kernel before wrote
  griddep_wait();
  griddep_launch_dependents();
  int nbox = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) nbox += (strip0 + b * BOXC < n) ? 1 : 0;
  const uint32_t stage_bytes = (uint32_t)(nbox * kBatch * BOXC * sizeof(T));
  auto issue = [&](int b) {
    const int st = b % kStages;
    T* dst = stages + st * STAGE_ELEMS;
    mbar_arrive_expect_tx(&full[st], stage_bytes);
#pragma unroll
    for (int bx = 0; bx < NB; ++bx) {
      if (strip0 + bx * BOXC < n)
        tma_load_2d(dst + bx * kBatch * BOXC, &tmap, strip0 + bx * BOXC, rb + b * kBatch,
                    &full[st]);
    }
  };
  if (tid == 0) {
    for (int b = 0; b < kStages && b < nbatch; ++b) issue(b);
  }

  T wcol[COLS][R];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int col = col0 + k;
#pragma unroll
    for (int c = 0; c < R; ++c)
      wcol[k][c] = (c < r && col < n) ? Wu[(int64_t)c * p.fs + col] : T(0);
  }
  // sums views: S'_h += U_h (V_h K_h^T)^T, K_h block upper triangular of
  // identities, i.e. the column-side factor is the suffix block sums of V_h
  switch (p.suffix_rin) {
    case 0: break;
    case 1: suffix_blocks<T, R, COLS, 1>(wcol); break;
    case 2: suffix_blocks<T, R, COLS, 2>(wcol); break;
    case 3: suffix_blocks<T, R, COLS, 3>(wcol); break;
    case 4: suffix_blocks<T, R, COLS, 4>(wcol); break;
    case 5: suffix_blocks<T, R, COLS, 5>(wcol); break;
    case 6: suffix_blocks<T, R, COLS, 6>(wcol); break;
    case 7: suffix_blocks<T, R, COLS, 7>(wcol); break;
    case 8: suffix_blocks<T, R, COLS, 8>(wcol); break;
    default: break;  // host rejects larger block widths
  }
  const int box = (tid * COLS) / BOXC;
  const int inbox = (tid * COLS) % BOXC;
  const bool vec_ok = (col0 + COLS <= n);
  const bool any_col = (col0 < n);

  int issued = min(kStages, nbatch);
  for (int b = 0; b < nbatch; ++b) {
    const int st = b % kStages;
    const uint32_t parity = (uint32_t)((b / kStages) & 1);
    const int row0 = rb + b * kBatch;
    const int nb = min(kBatch, re - row0);
    for (int idx = tid; idx < kBatch * R; idx += kThreads) {
      const int c = idx / kBatch;
      const int j = idx % kBatch;
      Us[j * R + c] = (j < nb && c < r) ? Uu[(int64_t)c * p.fs + row0 + j] : T(0);
    }
    const bool ok = mbar_wait_bounded(&full[st], parity, p.status);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        for (int bb = b + 1; bb < issued; ++bb)
          mbar_wait_bounded(&full[bb % kStages], (uint32_t)((bb / kStages) & 1), nullptr);
      }
      return;
    }
    const T* sp = stages + st * STAGE_ELEMS + box * kBatch * BOXC + inbox;
    if (any_col) {
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        if (j < nb) {
          T pv[COLS];
#pragma unroll
          for (int k = 0; k < COLS; ++k) pv[k] = sp[j * BOXC + k];
#pragma unroll
          for (int c = 0; c < R; ++c) {
            const T u = Us[j * R + c];
#pragma unroll
            for (int k = 0; k < COLS; ++k) pv[k] = fma(u, wcol[k][c], pv[k]);
          }
          T* dst = P + (int64_t)(row0 + j) * p.ldp + col0;
          if (vec_ok) {
            if constexpr (COLS * sizeof(T) == 16) {
              typename Vec<T>::type o;
              T* oe = reinterpret_cast<T*>(&o);
#pragma unroll
              for (int k = 0; k < COLS; ++k) oe[k] = pv[k];
              *reinterpret_cast<typename Vec<T>::type*>(dst) = o;
            } else if constexpr (COLS == 2 && sizeof(T) == 4) {
              *reinterpret_cast<float2*>(dst) = make_float2(pv[0], pv[1]);
            } else {
#pragma unroll
              for (int k = 0; k < COLS; ++k) dst[k] = pv[k];
            }
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k)
              if (col0 + k < n) dst[k] = pv[k];
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && b + kStages < nbatch) {
      fence_proxy_async();
      issue(b + kStages);
      ++issued;
    }
  }
}

#include "lv_pass_ws.cuh"

// ---------------------------------------------------------------------------
// Host side: geometry, tensor maps and launchers.
// ---------------------------------------------------------------------------
static int round_up(int a, int b) { return (a + b - 1) / b * b; }

static PassGeom geom_for_strip(int strip, int n, int num_sms) {
  PassGeom g;
  g.strip = strip;
  g.gC = (n + strip - 1) / strip;
  const int target = 2 * num_sms;  // two resident CTAs per SM, one wave
  int gR = target / g.gC;
  const int max_gR = (n + kBatch - 1) / kBatch;
  if (gR > max_gR) gR = max_gR;
  if (gR < 1) gR = 1;
  g.rows_per_cta = round_up((n + gR - 1) / gR, kBatch);
  g.gR = (n + g.rows_per_cta - 1) / g.rows_per_cta;
  return g;
}

PassGeom fused_geom(int elem_bytes, int n, int num_sms) {
  return geom_for_strip(128 * (16 / elem_bytes), n, num_sms);
}

static int update_cols(int elem_bytes, int R) {
  if (elem_bytes == 4) return R <= 32 ? 2 : 1;
  return R <= 16 ? 2 : 1;
}

PassGeom update_geom(int elem_bytes, int R, int n, int num_sms) {
  return geom_for_strip(kThreads * update_cols(elem_bytes, R), n, num_sms);
}

bool make_tmap(CUtensorMap* out, const void* base, int elem_bytes, int64_t cols, int64_t rows,
               int64_t ld) {
  // looked up once (thread-safe static initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)(kBoxBytes / elem_bytes), (cuuint32_t)kBatch};
  cuuint32_t estr[2] = {1, 1};
  CUresult rc = encode(out, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                       2, const_cast<void*>(base), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return rc == CUDA_SUCCESS;
}

template <typename T, int R, int MODE>
static cudaError_t launch_fused_t(const PassParams& p, const CUtensorMap& tm, cudaStream_t s) {
  constexpr int COLS = Vec<T>::N;
  constexpr int STRIP = 128 * COLS;
  // FP32 runs the decoupled-ring variant (lv_pass_ws.cuh)
  constexpr bool kWs = std::is_same<T, float>::value;
  const size_t smem =
      kWs ? sizeof(T) * kStagesWs * kBatch * STRIP + sizeof(uint64_t) * (2 * kStagesWs + 2) +
                kStagesWs * kBatch * R *
                    (((MODE & 4) ? sizeof(float) : 0) + ((MODE & 2) ? sizeof(float) : 0) +
                     ((MODE & 1) ? 4 * sizeof(float) : 0)) +
                (((MODE & 6) == 6) ? sizeof(double) * kThreads : 0)
          : sizeof(T) * kStages * kBatch * STRIP + sizeof(uint64_t) * kStages +
                sizeof(T) * (2 * kBatch * R + kBatch * R * (128 + 32 / R)) +
                sizeof(double) * R * R;
  using Kfn = void (*)(const CUtensorMap, const PassParams);
  Kfn kfn;
  if constexpr (kWs) {
    // the TMA write-back variant exists for the non-split update modes only
    constexpr bool kTs = (MODE & 4) != 0 && R <= 4;
    static const cudaError_t configured_ts =
        cudaFuncSetAttribute(fused_ws_kernel<R, MODE, kTs>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static const cudaError_t configured =
        cudaFuncSetAttribute(fused_ws_kernel<R, MODE, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured_ts != cudaSuccess) return configured_ts;
    if (configured != cudaSuccess) return configured;
    kfn = p.tma_store ? fused_ws_kernel<R, MODE, kTs> : fused_ws_kernel<R, MODE, false>;
  } else {
    kfn = fused_pass_kernel<T, R, MODE>;
    // set once per kernel instance (thread-safe static initialisation)
    static const cudaError_t configured =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured != cudaSuccess) return configured;
  }
  const cudaError_t e = launch_pdl(kfn, p.gC * p.gR, kThreads, smem, s, tm, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t fused_by_r(const PassParams& p, const CUtensorMap& tm, int R,
                              cudaStream_t s) {
  if (R <= 1) return launch_fused_t<T, 1, MODE>(p, tm, s);
  if (R <= 2) return launch_fused_t<T, 2, MODE>(p, tm, s);
  if (R <= 4) return launch_fused_t<T, 4, MODE>(p, tm, s);
  if (R <= 8) return launch_fused_t<T, 8, MODE>(p, tm, s);
  if constexpr (std::is_same<T, float>::value && (MODE & 4) == 0)
    if (R <= kMaxProductR) return launch_fused_t<T, kMaxProductR, MODE>(p, tm, s);
  if constexpr (std::is_same<T, float>::value && MODE == kModeY)
    if (R <= kMaxColSumR) return launch_fused_t<T, kMaxColSumR, MODE>(p, tm, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_fused(const PassParams& p, const CUtensorMap& tm, int R, int mode,
                         cudaStream_t s) {
  switch (mode) {
    case kModeXYU: return fused_by_r<T, kModeXYU>(p, tm, R, s);
    case kModeXY: return fused_by_r<T, kModeXY>(p, tm, R, s);
    case kModeXU: return fused_by_r<T, kModeXU>(p, tm, R, s);
    case kModeX: return fused_by_r<T, kModeX>(p, tm, R, s);
    case kModeY:
      if constexpr (std::is_same<T, float>::value) return fused_by_r<T, kModeY>(p, tm, R, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int R, int COLS>
static cudaError_t launch_update_t(const PassParams& p, const CUtensorMap& tm, cudaStream_t s,
                                   bool programmatic) {
  constexpr int STRIP = kThreads * COLS;
  constexpr bool kWs = std::is_same<T, float>::value;
  const size_t smem =
      kWs ? sizeof(T) * kStagesWs * kBatch * STRIP + sizeof(uint64_t) * (2 * kStagesWs + 2) +
                sizeof(float) * kStagesWs * kBatch * R
          : sizeof(T) * kStages * kBatch * STRIP + sizeof(uint64_t) * kStages +
                sizeof(T) * kBatch * R;
  using Kfn = void (*)(const CUtensorMap, const PassParams);
  Kfn kfn;
  if constexpr (kWs) {
    // set once per kernel instance (thread-safe static initialisation)
    static const cudaError_t configured_ts = cudaFuncSetAttribute(
        update_ws_kernel<R, COLS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static const cudaError_t configured = cudaFuncSetAttribute(
        update_ws_kernel<R, COLS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured_ts != cudaSuccess) return configured_ts;
    if (configured != cudaSuccess) return configured;
    kfn = p.tma_store ? update_ws_kernel<R, COLS, true> : update_ws_kernel<R, COLS, false>;
  } else {
    kfn = update_pass_kernel<T, R, COLS>;
    static const cudaError_t configured =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured != cudaSuccess) return configured;
  }
  if (!programmatic) {
    kfn<<<p.gC * p.gR, kThreads, smem, s>>>(tm, p);
    return cudaGetLastError();
  }
  const cudaError_t e = launch_pdl(kfn, p.gC * p.gR, kThreads, smem, s, tm, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <>
cudaError_t launch_update<float>(const PassParams& p, const CUtensorMap& tm, int R,
                                 cudaStream_t s, bool programmatic) {
  if (R <= 1) return launch_update_t<float, 1, 2>(p, tm, s, programmatic);
  if (R <= 2) return launch_update_t<float, 2, 2>(p, tm, s, programmatic);
  if (R <= 4) return launch_update_t<float, 4, 2>(p, tm, s, programmatic);
  if (R <= 8) return launch_update_t<float, 8, 2>(p, tm, s, programmatic);
  if (R <= 16) return launch_update_t<float, 16, 2>(p, tm, s, programmatic);
  if (R <= 32) return launch_update_t<float, 32, 2>(p, tm, s, programmatic);
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_update<double>(const PassParams& p, const CUtensorMap& tm, int R,
                                  cudaStream_t s, bool programmatic) {
  if (R <= 1) return launch_update_t<double, 1, 2>(p, tm, s, programmatic);
  if (R <= 2) return launch_update_t<double, 2, 2>(p, tm, s, programmatic);
  if (R <= 4) return launch_update_t<double, 4, 2>(p, tm, s, programmatic);
  if (R <= 8) return launch_update_t<double, 8, 2>(p, tm, s, programmatic);
  if (R <= 16) return launch_update_t<double, 16, 2>(p, tm, s, programmatic);
  if (R <= 32) return launch_update_t<double, 32, 1>(p, tm, s, programmatic);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_fused<float>(const PassParams&, const CUtensorMap&, int, int,
                                         cudaStream_t);
template cudaError_t launch_fused<double>(const PassParams&, const CUtensorMap&, int, int,
                                          cudaStream_t);

}  // namespace lv
