// The library's own dense contractions: the n^3 squarings and sums of the
// re-evaluation strategy (Section 4.2.2, "Re-evaluation"; Table 1), the
// products of the reverse pass (the adjoint chain through the squarings, the
// G_i = A^T G_{i+1} products and dA = [G_1 .. G_k][T_0 .. T_{k-1}]^T), the
// iteration's n x n x p products (T_i = A T_{i-1} + B, the hybrid strategy's
// D_i = A D_{i-1}) and the small factor products of the general form.
//
//  * tc_gemm_kernel<BN> (FP32): D = A_s B_s^T (+ beta C) on tcgen05 in split
//    TF32.  Every FP32 operand value x is split as x = hi + lo with hi = x
//    rounded to nearest TF32 and lo = x - hi (exact in FP32) rounded to nearest
//    TF32 in turn (so the tensor cores' handling of the low mantissa bits does
//    not matter and the split carries no one-sided bias);
//    A B^T ~= hi(A) hi(B)^T + lo(A) hi(B)^T + hi(A) lo(B)^T (the dropped
//    lo lo^T term is ~2^-22 relative): near-FP32 accuracy, where one TF32
//    product alone gives ~5e-4.  The operands are split
//    beforehand by split_rows_kernel into K-major rows [hi(x) | lo(x)] (which
//    also transposes where the product needs the other operand layout).
//    Tiles of 128 x BN outputs (BN = 256, 128 or 64), K chunks of 32 values
//    (one 128-byte swizzle atom); a persistent grid of one CTA per SM walks the
//    tiles in groups of 8 row blocks (the A and B chunks a wave reads stay in
//    L2).  Per CTA: warp 0 streams A and B chunks with TMA into an S-stage ring,
//    one thread of warp 1 issues 12 MMAs per chunk (3 products x 4 K steps of
//    8) into one of two BN-column FP32 accumulators in tensor memory, and the
//    epilogue warps read the other accumulator back (tcgen05.ld).  The tensor
//    cores accumulate with round-toward-zero, a bias that grows with the number
//    of accumulation steps (measured 7.9e-6 relative at K = 1000, ~6e-5 at
//    K = 8192 if the whole K were accumulated in tensor memory), so the MMAs
//    accumulate only segments of kSegChunks chunks into a fresh accumulator
//    (each chunk's two small correction products first, while the accumulator
//    is small), and the epilogue warps add each segment's result into FP32
//    registers (round to nearest), 128 columns per thread (8 epilogue warps
//    for 256-column tiles, 4 otherwise); after the tile's last segment they
//    add beta C and store D.
//    Every wait is bounded; an expired wait latches LINVIEW_ETIMEOUT and the
//    CTA drains its copies and MMAs and frees its tensor memory.
//  * gemm_simt_kernel<T>: C = alpha op(A) op(B) + beta C with arbitrary
//    strides on the CUDA cores (64 x 64 tiles, 4 x 4 outputs per thread), with
//    a deterministic split of long inner dimensions (partials summed in a
//    fixed order by a second kernel): the FP64 programs' products (GB300 has
//    no fast FP64 tensor path) and the small FP32 factor products.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {

namespace {

constexpr int kGBM = 128;       // tile rows (MMA M)
constexpr int kGroupM = 8;      // row blocks per raster group
#ifndef LV_GEMM_SEG_CHUNKS
#define LV_GEMM_SEG_CHUNKS 1
#endif
// K chunks of 32 accumulated in tensor memory per segment (compile-time tuning)
constexpr int kSegChunks = LV_GEMM_SEG_CHUNKS;

template <int BN>
struct GShape {
  static constexpr uint32_t AHalf = kGBM * 128;           // one half (hi or lo) of an A chunk
  static constexpr uint32_t BHalf = BN * 128;
  static constexpr uint32_t StageBytes = 2 * AHalf + 2 * BHalf;
  static constexpr int S = BN == 256 ? 2 : (BN == 128 ? 3 : 4);
  static constexpr uint32_t OffBar = S * StageBytes;
  static constexpr uint32_t SmemBytes = OffBar + 256 + 1024;  // + alignment slack
  static constexpr uint32_t TmemCols = 2 * BN;                // two accumulators
  static constexpr int CW = BN < 128 ? BN : 128;              // columns per epilogue thread
  static constexpr int NE = 4 * (BN / CW);                    // epilogue warps
  static constexpr int Threads = 64 + 32 * NE;
  // instruction descriptor: D F32, A/B TF32, both K-major, N = BN, M = 128
  static constexpr uint32_t Idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kGBM >> 4) << 24);
};
static_assert(GShape<256>::SmemBytes <= 232448 && GShape<128>::SmemBytes <= 232448 &&
                  GShape<64>::SmemBytes <= 232448,
              "shared memory per CTA");

struct GBars {
  uint64_t full[4], empty[4];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(GBars) <= 256, "barrier block");

// shared-memory descriptor of a K-major operand in 128-byte swizzled rows,
// 8-row groups 1024 bytes apart (the layout TMA writes with SWIZZLE_128B)
__device__ __forceinline__ uint64_t g_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1u << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;                   // descriptor version
  d |= (uint64_t)2u << 61;                   // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void g_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                      uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void g_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void g_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void g_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void g_tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void g_tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ bool g_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                       unsigned* status) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity, status)) return true;
  *abort_flag = 1;
  return false;
}

// tile t of the raster: groups of kGroupM row blocks, column blocks within
__device__ __forceinline__ void g_tile(long long t, int mt, int nt, int& mb, int& nb) {
  const long long per_group = (long long)kGroupM * nt;
  const int group = (int)(t / per_group);
  const int first = group * kGroupM;
  const int gm = (mt - first < kGroupM) ? (mt - first) : kGroupM;
  const int rem = (int)(t - (long long)group * per_group);
  mb = first + rem % gm;
  nb = rem / gm;
}

// D (M x N, row-major, ldd) = alpha A_s B_s^T + beta C over inner length K (nk
// chunks of 32); A_s / B_s: split rows [hi | lo] of length 2 kp (tensor maps
// tmA: box 32 x 128, tmB: box 32 x BN, both 128-byte swizzle).
template <int BN>
__global__ void __launch_bounds__(GShape<BN>::Threads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int M, int N, int nk, int kp, float* __restrict__ D, int64_t ldd,
                   const float* __restrict__ C, int64_t ldc, float alpha, float beta, int vec_ok,
                   int ksplit, float* __restrict__ work, unsigned* status) {
  using Sh = GShape<BN>;
  constexpr int S = Sh::S, CW = Sh::CW, NE = Sh::NE;
  extern __shared__ __align__(1024) unsigned char g_smem_raw[];
  const uint32_t raw = smem_u32(g_smem_raw);
  unsigned char* base = g_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  GBars* bars = reinterpret_cast<GBars*>(base + Sh::OffBar);
  volatile int* abort_flag = &bars->abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int mt = (M + kGBM - 1) / kGBM;
  const int nt = (N + BN - 1) / BN;
  // work items: (tile, K part); a split K (ksplit > 1) sends each part's
  // product to work[part] and a second kernel sums the parts in order
  const long long tiles = (long long)mt * nt;
  const long long T = tiles * ksplit;

  if (tid == 0) {
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    for (int i = 0; i < S; ++i) {
      mbar_init(&bars->full[i], 1);
      mbar_init(&bars->empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->acc_full[i], 1);
      mbar_init(&bars->acc_empty[i], NE);  // one arrival per epilogue warp
    }
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(Sh::TmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  g_fence_before();
  __syncthreads();
  g_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long g = 0;
      for (long long t = blockIdx.x; t < T && !*abort_flag; t += gridDim.x) {
        int mb, nb;
        g_tile(t % tiles, mt, nt, mb, nb);
        const int ks = (int)(t / tiles);
        const int kb = (int)((long long)nk * ks / ksplit), ke = (int)((long long)nk * (ks + 1) / ksplit);
        for (int kc = kb; kc < ke; ++kc, ++g) {
          const int st = (int)(g % S);
          const long long use = g / S;
          if (use >= 1 && !g_wait(&bars->empty[st], (uint32_t)((use - 1) & 1), abort_flag, status))
            break;
          unsigned char* sb = base + st * Sh::StageBytes;
          mbar_arrive_expect_tx(&bars->full[st], Sh::StageBytes);
          tma_load_2d(sb, &tmA, kc * 32, mb * kGBM, &bars->full[st]);
          tma_load_2d(sb + Sh::AHalf, &tmA, kp + kc * 32, mb * kGBM, &bars->full[st]);
          tma_load_2d(sb + 2 * Sh::AHalf, &tmB, kc * 32, nb * BN, &bars->full[st]);
          tma_load_2d(sb + 2 * Sh::AHalf + Sh::BHalf, &tmB, kp + kc * 32, nb * BN,
                      &bars->full[st]);
        }
      }
      if (*abort_flag) {
        // the stages loaded last may still be in flight: wait (bounded) for them
        const long long first = g > S ? g - S : 0;
        for (long long j = first; j < g; ++j)
          mbar_wait_bounded(&bars->full[j % S], (uint32_t)((j / S) & 1), nullptr);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long g = 0, gs = 0;  // chunks and segments consumed
      bool ok = true;
      for (long long t = blockIdx.x; t < T && ok && !*abort_flag; t += gridDim.x) {
        const int ks = (int)(t / tiles);
        const int kb = (int)((long long)nk * ks / ksplit), ke = (int)((long long)nk * (ks + 1) / ksplit);
        const int nseg = (ke - kb + kSegChunks - 1) / kSegChunks;
        for (int sg = 0; sg < nseg && ok; ++sg, ++gs) {
          const int buf = (int)(gs & 1);
          const long long ause = gs >> 1;
          if (ause >= 1 &&
              !g_wait(&bars->acc_empty[buf], (uint32_t)((ause - 1) & 1), abort_flag, status)) {
            ok = false;
            break;
          }
          g_fence_after();
          const uint32_t d = tmem + buf * BN;
          const int kc0 = kb + sg * kSegChunks;
          const int kc1 = kc0 + kSegChunks < ke ? kc0 + kSegChunks : ke;
          for (int kc = kc0; kc < kc1; ++kc, ++g) {
            const int st = (int)(g % S);
            if (!g_wait(&bars->full[st], (uint32_t)((g / S) & 1), abort_flag, status)) {
              ok = false;
              break;
            }
            g_fence_after();
            const uint32_t a_hi = smem_u32(base + st * Sh::StageBytes);
            const uint32_t a_lo = a_hi + Sh::AHalf;
            const uint32_t b_hi = a_hi + 2 * Sh::AHalf;
            const uint32_t b_lo = b_hi + Sh::BHalf;
            // lo(A) hi(B), hi(A) lo(B), then hi(A) hi(B)
            const uint32_t pa[3] = {a_lo, a_hi, a_hi};
            const uint32_t pb[3] = {b_hi, b_lo, b_hi};
            const bool first = kc == kc0;
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)  // K = 8 per MMA: 32 bytes of a 128-byte row
                g_mma(d, g_desc(pa[pr] + kk * 32), g_desc(pb[pr] + kk * 32), Sh::Idesc,
                      (!first || pr != 0 || kk != 0) ? 1u : 0u);
            }
            g_commit(&bars->empty[st]);
          }
          if (!ok) break;
          g_commit(&bars->acc_full[buf]);
        }
      }
      // every MMA issued has completed before the tensor memory is freed
      g_commit(&bars->drain);
      mbar_wait_bounded(&bars->drain, 0, status);
    }
  } else {
    // ---------------- epilogue (warps 2 .. 2 + NE - 1) ----------------
    const int ew = warp - 2;
    const int quarter = warp & 3;     // tensor-memory lanes 32*quarter .. +31
    const int cpart = ew >> 2;        // column part: columns cpart*CW .. +CW-1
    const int row = quarter * 32 + lane;
    long long gs = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < T && ok; t += gridDim.x) {
      int mb, nb;
      g_tile(t % tiles, mt, nt, mb, nb);
      const int ks = (int)(t / tiles);
      const int kb = (int)((long long)nk * ks / ksplit), ke = (int)((long long)nk * (ks + 1) / ksplit);
      const int nseg = (ke - kb + kSegChunks - 1) / kSegChunks;
      float acc[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) acc[c] = 0.f;
      for (int sg = 0; sg < nseg; ++sg, ++gs) {
        const int buf = (int)(gs & 1);
        const bool w = g_wait(&bars->acc_full[buf], (uint32_t)((gs >> 1) & 1), abort_flag, status);
        if (!__all_sync(0xffffffffu, w)) {  // tcgen05.ld is warp-collective
          ok = false;
          break;
        }
        g_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + buf * BN + cpart * CW;
#pragma unroll
        for (int q = 0; q < CW / 16; ++q) {
          float v[16];
          g_tmem_ld16(ta + q * 16, v);
          g_tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[q * 16 + e] += v[e];
        }
        g_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);  // the accumulator is free
      }
      if (!ok) break;
      const int grow = mb * kGBM + row;
      const int gc0 = nb * BN + cpart * CW;
      if (ksplit > 1) {  // this K part's product, to be summed by gemm_parts_kernel
        if (grow < M && gc0 < N) {
          float* wrow = work + ((int64_t)ks * M + grow) * N + gc0;
#pragma unroll
          for (int j = 0; j < CW; ++j)
            if (gc0 + j < N) wrow[j] = acc[j];
        }
      } else if (grow < M && gc0 < N) {
        float* drow = D + (int64_t)grow * ldd + gc0;
        const float* crow = (C && beta != 0.f) ? C + (int64_t)grow * ldc + gc0 : nullptr;
        if (vec_ok && gc0 + CW <= N) {
#pragma unroll
          for (int j = 0; j < CW / 4; ++j) {
            float4 o = make_float4(alpha * acc[4 * j], alpha * acc[4 * j + 1],
                                   alpha * acc[4 * j + 2], alpha * acc[4 * j + 3]);
            if (crow) {
              const float4 c = *reinterpret_cast<const float4*>(crow + 4 * j);
              o.x += beta * c.x;
              o.y += beta * c.y;
              o.z += beta * c.z;
              o.w += beta * c.w;
            }
            *reinterpret_cast<float4*>(drow + 4 * j) = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            if (gc0 + j < N) drow[j] = alpha * acc[j] + (crow ? beta * crow[j] : 0.f);
          }
        }
      }
    }
  }
  g_fence_before();
  __syncthreads();
  if (warp == 1) {
    g_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::TmemCols)
                 : "memory");
  }
}

// Split rows: element (i, k) of the source, X[i * rs + k * cs] (i < rows,
// k < K), goes to dst row i as hi at column k and lo at column kp + k (kp =
// rup(K, 32)); columns K .. kp - 1 of both halves are zero.  32 x 32 tiles
// through shared memory, read along whichever source index has unit stride.
__global__ void __launch_bounds__(256) split_rows_kernel(const float* __restrict__ X, int64_t rs,
                                                         int64_t cs, int rows, int K, int kp,
                                                         float* __restrict__ dst, int64_t ldd) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
  const bool k_fast = cs == 1;
  for (int j = ty; j < 32; j += 8) {
    const int il = k_fast ? j : tx, kl = k_fast ? tx : j;
    const int i = i0 + il, k = k0 + kl;
    tile[il][kl] = (i < rows && k < K) ? X[(int64_t)i * rs + (int64_t)k * cs] : 0.f;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int i = i0 + j, k = k0 + tx;
    if (i >= rows || k >= kp) continue;
    const float x = tile[j][tx];
    // round to nearest TF32 (ties away from zero): add half of the dropped
    // 13-bit field, then clear it; x - hi is exact
    const float hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    const float r = x - hi;
    float* d = dst + (int64_t)i * ldd;
    d[k] = hi;
    d[kp + k] = __uint_as_float((__float_as_uint(r) + 0x1000u) & 0xFFFFE000u);
  }
}

// ---------------------------------------------------------------- CUDA-core GEMM
constexpr int kSB = 64;   // tile
constexpr int kSK = 16;   // inner chunk

// One tile of C (or of a split's partial) of product z / splits of a batch:
// acc = sum over k in [k0, k1) of A(m, k) B(k, n) with A(m, k) = A[m * a_rs +
// k * a_cs], B(k, n) = B[k * b_rs + n * b_cs], the operands of batch entry b
// at A + b * a_bs, B + b * b_bs, C + b * c_bs (strides may be negative).
// splits == 1: C(m, n) = alpha acc + beta C(m, n) (C(m, n) at C[m * c_rs +
// n * c_cs]); else the partial goes to work[b][split][m][n].
template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int M, int N, int K, int kchunk, int splits,
                                                        T alpha, const T* __restrict__ A,
                                                        int64_t a_rs, int64_t a_cs, int64_t a_bs,
                                                        const T* __restrict__ B, int64_t b_rs,
                                                        int64_t b_cs, int64_t b_bs, T beta, T* C,
                                                        int64_t c_rs, int64_t c_cs, int64_t c_bs,
                                                        T* work) {
  __shared__ T As[kSK][kSB + 1];
  __shared__ T Bs[kSK][kSB + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * kSB, n0 = blockIdx.x * kSB;
  const int bz = blockIdx.z / splits, split = blockIdx.z % splits;
  A += (int64_t)bz * a_bs;
  B += (int64_t)bz * b_bs;
  const int kbeg = split * kchunk;
  const int kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const bool a_kfast = a_cs == 1;
  const bool b_nfast = b_cs == 1;
  for (int k0 = kbeg; k0 < kend; k0 += kSK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l;  // 0 .. 1023 = 64 x 16
      int mm, kk;
      if (a_kfast) {
        kk = e & 15;
        mm = e >> 4;
      } else {
        mm = e & 63;
        kk = e >> 6;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < kend) ? A[(int64_t)gm * a_rs + (int64_t)gk * a_cs] : T(0);
      int nn, kb;
      if (b_nfast) {
        nn = e & 63;
        kb = e >> 6;
      } else {
        kb = e & 15;
        nn = e >> 4;
      }
      const int gn = n0 + nn, gkb = k0 + kb;
      Bs[kb][nn] = (gn < N && gkb < kend) ? B[(int64_t)gkb * b_rs + (int64_t)gn * b_cs] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kSK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  T* Cb = C + (int64_t)bz * c_bs;
  T* wb = work ? work + ((int64_t)bz * splits + split) * M * N : nullptr;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int m = m0 + ty + 16 * x;
    if (m >= M) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int n = n0 + tx + 16 * y;
      if (n >= N) continue;
      if (wb) {
        wb[(int64_t)m * N + n] = acc[x][y];
      } else {
        T* c = Cb + (int64_t)m * c_rs + (int64_t)n * c_cs;
        *c = beta == T(0) ? alpha * acc[x][y] : alpha * acc[x][y] + beta * *c;
      }
    }
  }
}

// C(m, n) of batch entry b = alpha sum_s work[b][s][m][n] + beta C(m, n): one
// warp per output, lanes over the splits, then a fixed shuffle tree
// (deterministic).
template <typename T>
__global__ void gemm_reduce_kernel(int M, int N, int splits, int batch, T alpha,
                                   const T* __restrict__ work, T beta, T* C, int64_t c_rs,
                                   int64_t c_cs, int64_t c_bs) {
  const int lane = threadIdx.x & 31;
  const int64_t mn = (int64_t)M * N;
  const int64_t total = mn * batch;
  const int64_t wpb = blockDim.x / 32;
  for (int64_t o = blockIdx.x * wpb + (threadIdx.x >> 5); o < total; o += (int64_t)gridDim.x * wpb) {
    const int b = (int)(o / mn);
    const int64_t e = o - (int64_t)b * mn;
    const T* w = work + (int64_t)b * splits * mn + e;
    T s = T(0);
    for (int q = lane; q < splits; q += 32) s += w[(int64_t)q * mn];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
      T* c = C + (int64_t)b * c_bs + (int64_t)m * c_rs + (int64_t)n * c_cs;
      *c = beta == T(0) ? alpha * s : alpha * s + beta * *c;
    }
  }
}

// D = alpha sum_q work[q] + beta C (the K parts of a split product, summed in order)
__global__ void gemm_parts_kernel(int M, int N, int parts, const float* __restrict__ work,
                                  float alpha, float beta, const float* C, int64_t ldc, float* D,
                                  int64_t ldd) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float acc = work[e];
    for (int q = 1; q < parts; ++q) acc += work[(int64_t)q * total + e];
    const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
    float o = alpha * acc;
    if (C && beta != 0.f) o += beta * C[(int64_t)m * ldc + n];
    D[(int64_t)m * ldd + n] = o;
  }
}

template <int BN>
cudaError_t launch_tc_gemm_t(const CUtensorMap& tmA, const CUtensorMap& tmB, int M, int N, int nk,
                             int kp, float* D, int64_t ldd, const float* C, int64_t ldc,
                             float alpha, float beta, int vec_ok, int num_sms, float* work,
                             int64_t work_floats, unsigned* status, cudaStream_t s) {
  using Sh = GShape<BN>;
  static const cudaError_t configured = cudaFuncSetAttribute(
      tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SmemBytes);
  if (configured != cudaSuccess) return configured;
  const long long tiles = (long long)((M + kGBM - 1) / kGBM) * ((N + BN - 1) / BN);
  // too few tiles to fill the SMs: split K (each part at least 16 chunks of 32)
  int ksplit = 1;
  if (work) {
    while (tiles * (ksplit + 1) <= num_sms && nk / (ksplit + 1) >= 16 &&
           (int64_t)(ksplit + 1) * M * N <= work_floats)
      ++ksplit;
  }
  const long long T = tiles * ksplit;
  const int grid = (int)(T < num_sms ? T : num_sms);
  tc_gemm_kernel<BN><<<grid, Sh::Threads, Sh::SmemBytes, s>>>(
      tmA, tmB, M, N, nk, kp, D, ldd, C, ldc, alpha, beta, vec_ok, ksplit, work, status);
  if (ksplit == 1) return cudaGetLastError();
  const int64_t total = (int64_t)M * N;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  gemm_parts_kernel<<<blocks, 256, 0, s>>>(M, N, ksplit, work, alpha, beta, C, ldc, D, ldd);
  return cudaGetLastError();
}

}  // namespace

int64_t tc_split_ld(int64_t K) { return 2 * ((K + 31) / 32 * 32); }

cudaError_t launch_split_rows(const float* X, int64_t rs, int64_t cs, int rows, int K, float* dst,
                              int64_t ldd, cudaStream_t s) {
  if (rows <= 0 || K <= 0) return cudaSuccess;
  const int kp = (K + 31) / 32 * 32;
  if (ldd < 2 * kp) return cudaErrorInvalidValue;
  dim3 grid(kp / 32, (rows + 31) / 32);
  split_rows_kernel<<<grid, 256, 0, s>>>(X, rs, cs, rows, K, kp, dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const float* As, const float* Bs, int M, int N, int K, float* D,
                           int64_t ldd, const float* C, int64_t ldc, float alpha, float beta,
                           int num_sms, unsigned* status, cudaStream_t s, float* work,
                           int64_t work_floats) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  const int64_t ld = tc_split_ld(K);
  const int kp = (int)(ld / 2);
  const int nk = kp / 32;
  // the split buffers are TMA sources: 16-byte aligned bases (rows are 128-byte multiples)
  if ((reinterpret_cast<uintptr_t>(As) | reinterpret_cast<uintptr_t>(Bs)) & 15)
    return cudaErrorInvalidValue;
  const int BN = N >= 192 ? 256 : (N > 64 ? 128 : 64);
  CUtensorMap tmA, tmB;
  if (!make_tmap_sw128(&tmA, As, ld, M, ld, kGBM) || !make_tmap_sw128(&tmB, Bs, ld, N, ld, BN))
    return cudaErrorInvalidValue;
  const bool c_used = C != nullptr && beta != 0.f;
  const int vec_ok = (ldd % 4 == 0) && (reinterpret_cast<uintptr_t>(D) % 16 == 0) &&
                     (!c_used || (ldc % 4 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0));
  if (BN == 256)
    return launch_tc_gemm_t<256>(tmA, tmB, M, N, nk, kp, D, ldd, C, ldc, alpha, beta, vec_ok,
                                 num_sms, work, work_floats, status, s);
  if (BN == 128)
    return launch_tc_gemm_t<128>(tmA, tmB, M, N, nk, kp, D, ldd, C, ldc, alpha, beta, vec_ok,
                                 num_sms, work, work_floats, status, s);
  return launch_tc_gemm_t<64>(tmA, tmB, M, N, nk, kp, D, ldd, C, ldc, alpha, beta, vec_ok,
                              num_sms, work, work_floats, status, s);
}

static int gemm_simt_splits(int M, int N, int K, int batch, int num_sms, int64_t work_elems) {
  const int64_t tiles = (int64_t)((M + kSB - 1) / kSB) * ((N + kSB - 1) / kSB) * batch;
  int splits = 1;
  // split long inner dimensions until about two waves of CTAs are running
  while (tiles * splits < 2 * num_sms && K / (splits * 2) >= 8 * kSK &&
         (int64_t)(splits * 2) * M * N * batch <= work_elems)
    splits *= 2;
  return splits;
}

template <typename T>
cudaError_t launch_gemm_simt(int M, int N, int K, T alpha, const T* A, int64_t a_rs, int64_t a_cs,
                             const T* B, int64_t b_rs, int64_t b_cs, T beta, T* C, int64_t c_rs,
                             int64_t c_cs, T* work, int64_t work_elems, int num_sms,
                             cudaStream_t s, int batch, int64_t a_bs, int64_t b_bs,
                             int64_t c_bs) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (K <= 0) return cudaErrorInvalidValue;
  const int splits = work ? gemm_simt_splits(M, N, K, batch, num_sms, work_elems) : 1;
  const int kchunk = ((K + splits - 1) / splits + kSK - 1) / kSK * kSK;
  dim3 grid((N + kSB - 1) / kSB, (M + kSB - 1) / kSB, splits * batch);
  gemm_simt_kernel<T><<<grid, 256, 0, s>>>(M, N, K, kchunk, splits, alpha, A, a_rs, a_cs, a_bs, B,
                                           b_rs, b_cs, b_bs, beta, C, c_rs, c_cs, c_bs,
                                           splits > 1 ? work : nullptr);
  if (splits == 1) return cudaGetLastError();
  const int64_t outs = (int64_t)M * N * batch;
  const int blocks = (int)((outs + 7) / 8 < 4096 ? (outs + 7) / 8 : 4096);
  gemm_reduce_kernel<T><<<blocks, 256, 0, s>>>(M, N, splits, batch, alpha, work, beta, C, c_rs,
                                               c_cs, c_bs);
  return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<float>(int, int, int, float, const float*, int64_t, int64_t,
                                             const float*, int64_t, int64_t, float, float*,
                                             int64_t, int64_t, float*, int64_t, int, cudaStream_t,
                                             int, int64_t, int64_t, int64_t);
template cudaError_t launch_gemm_simt<double>(int, int, int, double, const double*, int64_t,
                                              int64_t, const double*, int64_t, int64_t, double,
                                              double*, int64_t, int64_t, double*, int64_t, int,
                                              cudaStream_t, int, int64_t, int64_t, int64_t);

}  // namespace lv
