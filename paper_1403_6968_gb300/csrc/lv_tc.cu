// Tensor-core update pass (tcgen05, sm_103a): P += U W^T for a factor block
// of 17..64 columns, the in-place rank-r refresh of a view (App. A, the
// "P_h += U_h V_h^T" step; the final P_k update) once r is past what the
// shared-memory broadcasts of the CUDA-core pass sustain at HBM speed.
//
// Arithmetic: split TF32 ("3xTF32").  Each FP32 factor value x is split as
// x = hi + lo with hi = x with the low 13 mantissa bits cleared (exact in
// TF32) and lo = x - hi (exact in FP32), and
//   U W^T ~= hi(U) hi(W)^T + lo(U) hi(W)^T + hi(U) lo(W)^T
// accumulated in FP32 in tensor memory: about 2^-22 relative error per
// product, i.e. FP32 accuracy for the delta.  A_cat = [hi(U) | lo(U)] and
// B_cat = [hi(W) | lo(W)] are row-major n x 128 (hi in columns 0..63, lo in
// 64..127, zero padded past r); the three products are one MMA chain over
// the K-chunk pairs (hi, hi), (lo, hi), (hi, lo).
//
// Two shapes, chosen by the block width r, both 224 KB of shared memory:
//   RP = 32: tiles of 128 rows x 64 columns of P, A block 32 KB, B tile
//            16 KB (double buffered), 5 P stages of 32 KB;
//   RP = 64: tiles of 128 rows x 64 columns, A block 64 KB, B tile 32 KB
//            (double buffered), 3 P stages of 32 KB.
// A persistent grid (one CTA per SM) walks the tiles row-block by
// row-block; per CTA:
//   warp 0     TMA producer: A block (reloaded when the row block changes),
//              B tile and P tile;
//   warp 1     allocates 2 x BN TMEM columns (two FP32 accumulators) and
//              issues the MMAs from one thread;
//   warps 2-5  epilogue: TMEM -> registers, + P (shared, 128B-swizzled),
//              back to shared memory, TMA store (by one thread once the four
//              warps have arrived on an mbarrier; a stage is released when
//              its store has been read out, one store in flight).
// Every mbarrier wait is bounded; an expired wait latches LINVIEW_ETIMEOUT,
// aborts the CTA's loops, drains the copies in flight and frees the TMEM.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {

namespace {

constexpr int kBM = 128;                 // tile rows (MMA M)
constexpr int kSplitCols = 128;          // columns of A_cat / B_cat: hi 0..63, lo 64..127
constexpr int kTcThreads = 192;
constexpr int kStoresInFlight = 1;       // TMA stores not yet read out

// Shape of one variant: RP factor columns (padded), BN tile columns.
template <int RP>
struct TcShape {
  static constexpr int BN = 64;                        // tile columns (MMA N)
  static constexpr int H = RP / 32;                    // 128-byte K chunks per half
  static constexpr int KC = 2 * H;                     // chunks: hi 0..H-1, lo H..2H-1
  static constexpr uint32_t ABytes = KC * kBM * 128;   // A block
  static constexpr uint32_t BBytes = KC * BN * 128;    // B tile (one buffer)
  static constexpr int PBoxes = BN / 32;               // 32-column boxes per P tile
  static constexpr uint32_t PBytes = PBoxes * kBM * 128;
  static constexpr int PS = RP == 32 ? 5 : 3;          // P tile stages
  static constexpr uint32_t TmemCols = 2 * BN;         // two accumulators
  static constexpr uint32_t OffA = 0;
  static constexpr uint32_t OffB = OffA + ABytes;      // 2 buffers
  static constexpr uint32_t OffP = OffB + 2 * BBytes;  // PS buffers
  static constexpr uint32_t OffBar = OffP + PS * PBytes;
  static constexpr uint32_t SmemBytes = OffBar + 512 + 1024;  // + alignment slack
  // instruction descriptor: D F32, A/B TF32, both K-major, N = BN, M = 128
  static constexpr uint32_t Idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  // column of A_cat / B_cat where K chunk kc starts
  static __host__ __device__ constexpr int chunk_x(int kc) { return (kc / H) * 64 + (kc % H) * 32; }
};
constexpr int kMaxPS = 8;
static_assert(TcShape<32>::SmemBytes <= 232448 && TcShape<64>::SmemBytes <= 232448,
              "shared memory per CTA");

// shared-memory matrix descriptor: K-major operand in 128-byte swizzled rows,
// 8-row groups 1024 bytes apart (the layout TMA writes with SWIZZLE_128B)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);         // start address
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1u << 46;                          // descriptor version
  d |= (uint64_t)2u << 61;                          // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
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

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcBars {
  uint64_t a_full;
  uint64_t b_full[2], b_empty[2];
  uint64_t p_full[kMaxPS], p_empty[kMaxPS];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t ep_done[kMaxPS];  // the 4 epilogue warps have written their rows of a P tile
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(TcBars) <= 512, "barrier block");

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        unsigned* status) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity, status)) return true;
  *abort_flag = 1;
  return false;
}

// P (n x n, row-major, tensor map tmP: box 32 x 128, 128B swizzle) +=
// A_cat B_cat^T with A_cat, B_cat n x 128 row-major (tmA: box 32 x 128,
// tmB: box 32 x 32, both 128B swizzle); RP = 32 reads K chunks (hi 0..31,
// lo 64..95), RP = 64 reads all four.
template <int RP>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_update_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, float* P, int64_t ldp, int n,
                     unsigned* status) {
  using Sh = TcShape<RP>;
  constexpr int BN = Sh::BN, KC = Sh::KC, H = Sh::H, PS = Sh::PS;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  const uint32_t raw = smem_u32(tc_smem_raw);
  unsigned char* base = tc_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  TcBars* bars = reinterpret_cast<TcBars*>(base + Sh::OffBar);
  volatile int* abort_flag = &bars->abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  const int nrb = (n + kBM - 1) / kBM;
  const int ncb = (n + BN - 1) / BN;
  const long long T = (long long)nrb * ncb;
  const long long t0 = T * blockIdx.x / gridDim.x;
  const long long t1 = T * (blockIdx.x + 1) / gridDim.x;
  const int ntile = (int)(t1 - t0);

  if (tid == 0) {
    prefetch_tmap(&tmP);
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
    mbar_init(&bars->a_full, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->b_full[i], 1);
      mbar_init(&bars->b_empty[i], 1);
      mbar_init(&bars->acc_full[i], 1);
      mbar_init(&bars->acc_empty[i], 4);  // one arrival per epilogue warp
    }
    for (int i = 0; i < PS; ++i) {
      mbar_init(&bars->p_full[i], 1);
      mbar_init(&bars->p_empty[i], 1);
      mbar_init(&bars->ep_done[i], 4);
    }
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {  // TMEM: two BN-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(Sh::TmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int cur_rb = -1;
      int b_issued = 0, p_issued = 0, a_issued = 0;  // loads issued (for the abort drain)
      for (int i = 0; i < ntile && !*abort_flag; ++i) {
        const long long t = t0 + i;
        const int rb = (int)(t / ncb), cb = (int)(t % ncb);
        const int buf = i & 1, use = i >> 1;
        if (rb != cur_rb) {
          // the MMAs of the previous tile read the old A block
          if (i > 0 && !tc_wait(&bars->acc_full[(i - 1) & 1], ((i - 1) >> 1) & 1, abort_flag,
                                status))
            break;
          fence_proxy_async();
          mbar_arrive_expect_tx(&bars->a_full, Sh::ABytes);
          for (int kc = 0; kc < KC; ++kc)
            tma_load_2d(base + Sh::OffA + kc * kBM * 128, &tmA, Sh::chunk_x(kc), rb * kBM,
                        &bars->a_full);
          ++a_issued;
          cur_rb = rb;
        }
        if (use >= 1 && !tc_wait(&bars->b_empty[buf], (use - 1) & 1, abort_flag, status)) break;
        mbar_arrive_expect_tx(&bars->b_full[buf], Sh::BBytes);
        for (int kc = 0; kc < KC; ++kc)
          for (int sb = 0; sb < BN / 32; ++sb)  // 32-row boxes
            tma_load_2d(base + Sh::OffB + buf * Sh::BBytes + (kc * BN + sb * 32) * 128, &tmB,
                        Sh::chunk_x(kc), cb * BN + sb * 32, &bars->b_full[buf]);
        ++b_issued;
        const int ps = i % PS, puse = i / PS;
        if (puse >= 1 && !tc_wait(&bars->p_empty[ps], (puse - 1) & 1, abort_flag, status)) break;
        mbar_arrive_expect_tx(&bars->p_full[ps], Sh::PBytes);
        for (int h = 0; h < Sh::PBoxes; ++h)
          tma_load_2d(base + Sh::OffP + ps * Sh::PBytes + h * kBM * 128, &tmP, cb * BN + 32 * h,
                      rb * kBM, &bars->p_full[ps]);
        ++p_issued;
      }
      if (*abort_flag) {
        // wait (bounded) until every load issued has landed before the CTA exits
        for (int j = 0; j < a_issued; ++j) mbar_wait_bounded(&bars->a_full, j & 1, nullptr);
        for (int j = 0; j < b_issued; ++j)
          mbar_wait_bounded(&bars->b_full[j & 1], (j >> 1) & 1, nullptr);
        for (int j = 0; j < p_issued; ++j)
          mbar_wait_bounded(&bars->p_full[j % PS], (j / PS) & 1, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int cur_rb = -1, a_loads = 0, issued = 0;
      for (int i = 0; i < ntile && !*abort_flag; ++i) {
        const long long t = t0 + i;
        const int rb = (int)(t / ncb);
        const int buf = i & 1, use = i >> 1;
        if (rb != cur_rb) {
          if (!tc_wait(&bars->a_full, a_loads & 1, abort_flag, status)) break;
          ++a_loads;
          cur_rb = rb;
        }
        if (!tc_wait(&bars->b_full[buf], use & 1, abort_flag, status)) break;
        if (use >= 1 && !tc_wait(&bars->acc_empty[buf], (use - 1) & 1, abort_flag, status)) break;
        tc_fence_after();
        const uint32_t d = tmem + buf * BN;
        const uint32_t a0 = smem_u32(base + Sh::OffA);
        const uint32_t b0 = smem_u32(base + Sh::OffB + buf * Sh::BBytes);
        // (A half, B half): hi*hi, lo*hi, hi*lo; each over the H chunks of a half
        constexpr int kPairA[3] = {0, 1, 0};
        constexpr int kPairB[3] = {0, 0, 1};
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
#pragma unroll
          for (int hk = 0; hk < H; ++hk) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // K = 8 per MMA: 32 bytes of a 128-byte row
              const uint64_t ad = sw128_desc(a0 + (kPairA[pr] * H + hk) * kBM * 128 + kk * 32);
              const uint64_t bd = sw128_desc(b0 + (kPairB[pr] * H + hk) * BN * 128 + kk * 32);
              tc_mma(d, ad, bd, Sh::Idesc, (pr | hk | kk) != 0 ? 1u : 0u);
            }
          }
        }
        tc_commit(&bars->b_empty[buf]);
        tc_commit(&bars->acc_full[buf]);
        issued = i + 1;
      }
      if (*abort_flag && issued > 0) {
        // the MMAs issued must finish before the TMEM is freed
        const int j = issued - 1;
        mbar_wait_bounded(&bars->acc_full[j & 1], (j >> 1) & 1, nullptr);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;        // tile row of this thread
    const bool leader = (warp == 2 && lane == 0);
    // A TMA store writes whole 16-byte chunks at the right edge of the
    // tensor; when n % 4 != 0 the last tile column is stored element by
    // element instead, so that no column >= n (caller padding) is written.
    const bool ragged = (n & 3) != 0;
    for (int i = 0; i < ntile; ++i) {
      const long long t = t0 + i;
      const int rb = (int)(t / ncb), cb = (int)(t % ncb);
      const int buf = i & 1, use = i >> 1;
      const int ps = i % PS, puse = i / PS;
      bool ok = tc_wait(&bars->acc_full[buf], use & 1, abort_flag, status) &&
                tc_wait(&bars->p_full[ps], puse & 1, abort_flag, status);
      // the TMEM loads below are warp-collective: the warp leaves together
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      float acc[BN];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + buf * BN;
#pragma unroll
      for (int q = 0; q < BN / 16; ++q) {
        float v[16];
        tmem_ld16(ta + q * 16, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[q * 16 + e] = v[e];
      }
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
      // P tile: BN / 32 boxes of 32 columns, rows of 128 bytes, 16-byte chunk
      // j of row r stored at chunk j ^ (r % 8)
      unsigned char* pt = base + Sh::OffP + ps * Sh::PBytes;
      const bool direct = ragged && cb == ncb - 1;
      const int grow = rb * kBM + row;
#pragma unroll
      for (int h = 0; h < Sh::PBoxes; ++h) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4* q = reinterpret_cast<float4*>(pt + h * kBM * 128 + row * 128 +
                                                ((j ^ (row & 7)) << 4));
          float4 pv = *q;
          const int c = h * 32 + j * 4;
          pv.x += acc[c];
          pv.y += acc[c + 1];
          pv.z += acc[c + 2];
          pv.w += acc[c + 3];
          if (!direct) {
            *q = pv;
          } else if (grow < n) {
            const int gc = cb * BN + c;
            float* dst = P + (int64_t)grow * ldp + gc;
            if (gc + 0 < n) dst[0] = pv.x;
            if (gc + 1 < n) dst[1] = pv.y;
            if (gc + 2 < n) dst[2] = pv.z;
            if (gc + 3 < n) dst[3] = pv.w;
          }
        }
      }
      // make the rows visible to the TMA store (async proxy); the leader
      // stores once all four warps have arrived (a bounded wait, no
      // unbounded named barrier)
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->ep_done[ps]);
      bool stop = false;
      if (leader) {
        if (tc_wait(&bars->ep_done[ps], puse & 1, abort_flag, status)) {
          if (!direct) {
            for (int h = 0; h < Sh::PBoxes; ++h)
              tma_store_2d(&tmP, pt + h * kBM * 128, cb * BN + 32 * h, rb * kBM);
          }
          bulk_commit();  // one group per tile (empty for a ragged edge tile)
          // the store group of tile i - kStoresInFlight has read its stage
          bulk_wait_read<kStoresInFlight>();
          if (i >= kStoresInFlight) mbar_arrive(&bars->p_empty[(i - kStoresInFlight) % PS]);
        } else {
          stop = true;
        }
      }
      if (__any_sync(0xffffffffu, stop)) break;  // warp-uniform exit
    }
    if (leader) bulk_wait0();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::TmemCols)
                 : "memory");
  }
}

// A_cat = [hi(U) | lo(U)], B_cat = [hi(W) | lo(W)] (n x 128, row-major: hi in
// columns 0..63, lo in 64..127) from column-major U, W (column stride fs,
// r <= 64 columns); the first ``half`` columns of each half are written (32
// or 64: the columns the variant reads), zero past r.  A block of 256
// threads transposes 32 rows through shared memory: reads run down the
// factor columns, writes along the rows.
__global__ void __launch_bounds__(256) tc_split_kernel(const float* __restrict__ U,
                                                       const float* __restrict__ W, int64_t fs,
                                                       int n, int r, int half,
                                                       float* __restrict__ Acat,
                                                       float* __restrict__ Bcat) {
  __shared__ float su[64][33], sw[64][33];
  const int row0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
  for (int c = ty; c < half; c += 8) {
    const int i = row0 + tx;
    const bool ok = c < r && i < n;
    su[c][tx] = ok ? U[(int64_t)c * fs + i] : 0.f;
    sw[c][tx] = ok ? W[(int64_t)c * fs + i] : 0.f;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int i = row0 + j;
    if (i >= n) break;
    float* a = Acat + (int64_t)i * kSplitCols;
    float* b = Bcat + (int64_t)i * kSplitCols;
    for (int c = tx; c < half; c += 32) {
      const float u = su[c][j], w = sw[c][j];
      const float uh = __uint_as_float(__float_as_uint(u) & 0xFFFFE000u);
      const float wh = __uint_as_float(__float_as_uint(w) & 0xFFFFE000u);
      a[c] = uh;
      a[64 + c] = u - uh;
      b[c] = wh;
      b[64 + c] = w - wh;
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core products passes: X = P U (rows of P, TR = false) and Y = P^T V
// (columns of P, TR = true) for a factor block of up to RP (32 or 64)
// columns -- App. A's P_h U_h and P_h^T V_h once the block is too wide for
// the CUDA-core pass (a 16-column products pass is issue bound there).
//
// Arithmetic: split TF32 as in the update pass, with both operands split.
// The factor is pre-split as [hi | lo] rows (hi rounded to nearest TF32).
// P is split on the fly in shared memory: the tensor pipe reads a TF32
// operand from the top 19 bits of each 32-bit word, so the loaded FP32 box
// itself is hi(P) = P truncated to TF32 (X; the transposing split of Y
// writes it out explicitly), and lo(P) = P - hi(P) is exact in FP32.  Per K
// chunk of 32 the products hi*[hi | lo] (one MMA of width 2 RP) and lo*hi go
// into one TMEM accumulator, and the epilogue warps add each chunk's
// accumulator into FP32 registers (round to nearest): the tensor pipe
// truncates its own accumulations, which over K = n would bias the sums.
//
// Operands, all K-major with 128-byte swizzle (the layout TMA writes):
//   X: A = P rows (the loaded 128 x 32 box of P; lo beside it),
//      B = U^T (RP factor columns x 32 of K);
//   Y: A = P^T (the loaded 32 x 128 slab of P transposed by the split warps
//      into 128 x 32 hi and lo tiles), B = V^T.
// Work: the output tiles' K chunks in one tile-major sequence, cut into one
// contiguous range per CTA (one CTA per SM); a tile's chunks are shared by a
// few CTAs, whose sums land in consecutive partials of the output (Xpart /
// Ypart layout: partial stride ps, column stride cs), summed by the
// assembly.  Warps: 0 TMA producer, 1 TMEM allocation and
// MMA issue, 2-5 split, 6-9 epilogue.  The pass is bound by shared-memory
// traffic (the TMA writes, the split, and the tensor pipe reading each A
// tile three times), not by HBM.  Every mbarrier wait is bounded: an expired
// wait latches LINVIEW_ETIMEOUT, stops the CTA's loops, drains the copies and
// MMAs in flight and frees the TMEM.
constexpr int kTpThreads = 320;
constexpr int kTpMaxStages = 5;

template <bool TR, int RP>
struct TpShape {
  static constexpr uint32_t PBytes = kBM * 128;            // 128 x 32 FP32 (X) / 4 boxes 32 x 32 (Y)
  static constexpr uint32_t HiBytes = TR ? kBM * 128 : 0;  // Y: transposed hi (X: the loaded box)
  static constexpr uint32_t LoBytes = kBM * 128;
  static constexpr uint32_t BBytes = 2 * RP * 128;         // factor chunk: hi rows, then lo rows
  static constexpr uint32_t StageBytes = PBytes + HiBytes + LoBytes + BBytes;
  static constexpr int S = (int)((221184u / StageBytes) < (uint32_t)kTpMaxStages
                                     ? (221184u / StageBytes) : (uint32_t)kTpMaxStages);
  static constexpr uint32_t OffBar = S * StageBytes;
  static constexpr uint32_t SmemBytes = OffBar + 512 + 1024;
  // a chunk accumulator holds hi(A) [hi(B) | lo(B)] in 2 RP columns (with
  // lo(A) hi(B) added to the first RP); two of them
  static constexpr uint32_t TmemCols = 4 * RP;
  static constexpr uint32_t IdescW = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(2 * RP >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  static constexpr uint32_t IdescN = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(RP >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
};
static_assert(TpShape<false, 64>::SmemBytes <= 232448 && TpShape<true, 64>::SmemBytes <= 232448,
              "shared memory per CTA");
static_assert(TpShape<true, 64>::S >= 3 && TpShape<false, 64>::S >= 4, "pipeline depth");

struct TpBars {
  uint64_t full[kTpMaxStages], split[kTpMaxStages], empty[kTpMaxStages];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem_base;
  int abort;
};
static_assert(sizeof(TpBars) <= 512, "barrier block");

__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float tf32_trunc(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

// byte offset of 16-byte chunk ``chunk`` of row ``row`` in a tile of 128-byte
// rows with 128-byte swizzle: the chunk sits at chunk ^ (row % 8)
__device__ __forceinline__ uint32_t sw128_off(int row, int chunk) {
  return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}

template <bool TR, int RP>
__global__ void __launch_bounds__(kTpThreads, 1)
    tc_products_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmF,
                       float* out, int64_t ps, int64_t cs, int n, int r_out, int parts,
                       unsigned* status) {
  using Sh = TpShape<TR, RP>;
  constexpr int S = Sh::S;
  extern __shared__ __align__(1024) unsigned char tp_smem_raw[];
  const uint32_t raw = smem_u32(tp_smem_raw);
  unsigned char* base = tp_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  TpBars* bars = reinterpret_cast<TpBars*>(base + Sh::OffBar);
  volatile int* abort_flag = &bars->abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  // Work: the C = ot_n x nkb chunks (output tile ot, K chunk kb of 32),
  // tile-major, cut into gridDim.x contiguous ranges; a CTA's range splits
  // into segments, one per output tile it touches.  The CTAs touching tile
  // ot are b_lo(ot) .. : a segment's sums go to partial b - b_lo(ot) (< parts),
  // and the CTA that ends a tile zero-fills the partials past its own.
  const int ot_n = (n + kBM - 1) / kBM;  // output tiles
  const int nkb = (n + 31) / 32;          // K chunks of 32
  const long long C = (long long)ot_n * nkb;
  const long long G = gridDim.x;
  const long long c0 = C * blockIdx.x / G;
  const long long c1 = C * (blockIdx.x + 1) / G;
  // first CTA whose range holds chunk x: the largest b with C b / G <= x
  auto cta_of = [&](long long x) { return (int)(((x + 1) * G + C - 1) / C - 1); };
  // segment of the chunk range starting at chunk c: tile, K range, slot
  auto segment = [&](long long c, int& ot, int& kb0, int& kb1, int& part) {
    ot = (int)(c / nkb);
    kb0 = (int)(c % nkb);
    const long long tile_end = (long long)(ot + 1) * nkb;
    kb1 = (int)((c1 < tile_end ? c1 : tile_end) - (long long)ot * nkb);
    part = (int)blockIdx.x - cta_of((long long)ot * nkb);
  };

  if (tid == 0) {
    prefetch_tmap(&tmP);
    prefetch_tmap(&tmF);
    for (int i = 0; i < S; ++i) {
      mbar_init(&bars->full[i], 1);
      mbar_init(&bars->split[i], 4);  // one arrival per split warp
      mbar_init(&bars->empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->acc_full[i], 1);
      mbar_init(&bars->acc_empty[i], 4);  // one arrival per epilogue warp
    }
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
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long g = 0, issued = 0;
      for (long long c = c0; c < c1 && !*abort_flag;) {
        int ot, part, kb0, kb1;
        segment(c, ot, kb0, kb1, part);
        c += kb1 - kb0;
        for (int kb = kb0; kb < kb1 && !*abort_flag; ++kb, ++g) {
          const int st = (int)(g % S);
          const long long use = g / S;
          if (use >= 1 && !tc_wait(&bars->empty[st], (uint32_t)((use - 1) & 1), abort_flag, status))
            break;
          unsigned char* sb = base + st * Sh::StageBytes;
          fence_proxy_async();
          mbar_arrive_expect_tx(&bars->full[st], Sh::PBytes + Sh::BBytes);
          if constexpr (!TR) {
            tma_load_2d(sb, &tmP, kb * 32, ot * kBM, &bars->full[st]);
          } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
              tma_load_2d(sb + b * 4096, &tmP, ot * kBM + 32 * b, kb * 32, &bars->full[st]);
          }
          unsigned char* bb = sb + Sh::PBytes + Sh::HiBytes + Sh::LoBytes;
          tma_load_2d(bb, &tmF, kb * 32, 0, &bars->full[st]);
          tma_load_2d(bb + RP * 128, &tmF, kb * 32, 64, &bars->full[st]);
          issued = g + 1;
        }
      }
      if (*abort_flag)  // the loads issued land before the CTA exits (bounded)
        for (long long j = (issued > S ? issued - S : 0); j < issued; ++j)
          mbar_wait_bounded(&bars->full[j % S], (uint32_t)((j / S) & 1), nullptr);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long g = 0, issued = 0;
      for (long long c = c0; c < c1 && !*abort_flag;) {
        int ot, part, kb0, kb1;
        segment(c, ot, kb0, kb1, part);
        c += kb1 - kb0;
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int st = (int)(g % S);
          const long long use = g / S;
          const int buf = (int)(g & 1);
          const long long bu = g >> 1;
          if (!tc_wait(&bars->split[st], (uint32_t)(use & 1), abort_flag, status)) break;
          if (bu >= 1 && !tc_wait(&bars->acc_empty[buf], (uint32_t)((bu - 1) & 1), abort_flag, status))
            break;
          tc_fence_after();
          const uint32_t d = tmem + buf * (2 * RP);
          const uint32_t s0 = smem_u32(base + st * Sh::StageBytes);
          const uint32_t a_hi = TR ? s0 + Sh::PBytes : s0;
          const uint32_t a_lo = s0 + Sh::PBytes + Sh::HiBytes;
          const uint32_t b_hi = a_lo + Sh::LoBytes;  // 2 RP rows: hi(B), then lo(B)
          // per K step of 8 (32 bytes of each 128-byte row): hi(A) [hi(B) |
          // lo(B)] over 2 RP columns, then lo(A) hi(B) into the first RP: the
          // three products of the split in two MMAs, the wider one filling
          // the tensor pipe better than three of width RP
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            tc_mma(d, sw128_desc(a_hi + kk * 32), sw128_desc(b_hi + kk * 32), Sh::IdescW,
                   kk != 0 ? 1u : 0u);
            tc_mma(d, sw128_desc(a_lo + kk * 32), sw128_desc(b_hi + kk * 32), Sh::IdescN, 1u);
          }
          tc_commit(&bars->empty[st]);
          tc_commit(&bars->acc_full[buf]);
          issued = g + 1;
        }
      }
      if (*abort_flag && issued > 0) {
        const long long j = issued - 1;  // the MMAs issued finish before the TMEM is freed
        mbar_wait_bounded(&bars->acc_full[j & 1], (uint32_t)((j >> 1) & 1), nullptr);
      }
    }
  } else if (warp < 6) {
    // ---------------- split (warps 2..5, 128 threads) ----------------
    const int st_tid = tid - 64;
    long long g = 0;
    bool ok = true;
    for (long long c = c0; c < c1 && ok;) {
      int ot, part, kb0, kb1;
      segment(c, ot, kb0, kb1, part);
      c += kb1 - kb0;
      for (int kb = kb0; kb < kb1; ++kb, ++g) {
        const int st = (int)(g % S);
        const long long use = g / S;
        ok = tc_wait(&bars->full[st], (uint32_t)(use & 1), abort_flag, status);
        if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
        unsigned char* sb = base + st * Sh::StageBytes;
        if constexpr (!TR) {
          // the loaded box is hi(P) as the tensor pipe reads it; lo beside it
          // (same swizzled offsets)
          const float4* pv = reinterpret_cast<const float4*>(sb);
          float4* lv = reinterpret_cast<float4*>(sb + Sh::PBytes);
#pragma unroll
          for (int q = 0; q < (int)(Sh::PBytes / 16) / 128; ++q) {
            const int f = st_tid + q * 128;
            const float4 x = pv[f];
            lv[f] = make_float4(x.x - tf32_trunc(x.x), x.y - tf32_trunc(x.y),
                                x.z - tf32_trunc(x.z), x.w - tf32_trunc(x.w));
          }
        } else {
          // slab rows i (32) x columns j (128, 4 boxes of 32) -> hi/lo tiles of
          // 128 rows j x 32 i; a thread moves 4 x 4 blocks (4 i, 4 j): the 8
          // threads of a group take distinct (i-block, j-block mod 8) pairs,
          // which fall in distinct 16-byte chunks on both sides
          unsigned char* hi = sb + Sh::PBytes;
          unsigned char* lo = hi + Sh::HiBytes;
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const int grp = (st_tid >> 3) + 16 * it;  // 0..31
            const int k8 = st_tid & 7;
            const int ib = k8;                                       // rows 4 ib .. 4 ib + 3
            const int jb = 8 * (grp & 3) + ((k8 + (grp >> 2)) & 7);  // columns 4 jb .. + 3
            const int box = jb >> 3, jc = jb & 7;
            float x[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const float4 v = *reinterpret_cast<const float4*>(sb + box * 4096 +
                                                                sw128_off(4 * ib + a, jc));
              x[a][0] = v.x; x[a][1] = v.y; x[a][2] = v.z; x[a][3] = v.w;
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int j = 4 * jb + b;
              float4 h, l2;
              h.x = tf32_rn(x[0][b]); l2.x = x[0][b] - h.x;
              h.y = tf32_rn(x[1][b]); l2.y = x[1][b] - h.y;
              h.z = tf32_rn(x[2][b]); l2.z = x[2][b] - h.z;
              h.w = tf32_rn(x[3][b]); l2.w = x[3][b] - h.w;
              *reinterpret_cast<float4*>(hi + sw128_off(j, ib)) = h;
              *reinterpret_cast<float4*>(lo + sw128_off(j, ib)) = l2;
            }
          }
        }
        fence_proxy_async();  // generic-proxy writes, read next by the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->split[st]);
      }
    }
  } else {
    // ---------------- epilogue (warps 6..9) ----------------
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. + 31
    const int row = quarter * 32 + lane;
    long long g = 0;
    bool ok = true;
    for (long long c = c0; c < c1 && ok;) {
      int ot, part, kb0, kb1;
      segment(c, ot, kb0, kb1, part);
      c += kb1 - kb0;
      float acc[RP];
#pragma unroll
      for (int c = 0; c < RP; ++c) acc[c] = 0.f;
      for (int kb = kb0; kb < kb1; ++kb, ++g) {
        const int buf = (int)(g & 1);
        const long long bu = g >> 1;
        ok = tc_wait(&bars->acc_full[buf], (uint32_t)(bu & 1), abort_flag, status);
        if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (2 * RP);
#pragma unroll
        for (int q = 0; q < RP / 16; ++q) {
          float v[16], w[16];
          tmem_ld16(ta + q * 16, v);       // hi hi + lo hi
          tmem_ld16(ta + RP + q * 16, w);  // hi lo
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[q * 16 + e] += w[e] + v[e];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
      }
      if (!ok) break;
      const int orow = ot * kBM + row;
      if (orow < n) {
        float* o = out + (int64_t)part * ps + orow;
#pragma unroll
        for (int q = 0; q < RP; ++q)
          if (q < r_out) o[(int64_t)q * cs] = acc[q];
        if (kb1 == nkb)  // this CTA ends the tile: the partials past its own are zero
          for (int pz = part + 1; pz < parts; ++pz)
            for (int q = 0; q < r_out; ++q) out[(int64_t)pz * ps + (int64_t)q * cs + orow] = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Sh::TmemCols)
                 : "memory");
  }
}

// Factor split for the products passes: F (128 rows x fs) row c = hi(Fin
// column c) for c < r, 0 for r <= c < rp; row 64 + c = the low part.  Fin is
// column-major (column stride fs), n rows.
__global__ void tp_split_kernel(const float* __restrict__ Fin, int64_t fs, int n, int r, int rp,
                                float* __restrict__ F) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rp * n) return;
  const int c = (int)(idx / n), i = (int)(idx % n);
  const float x = c < r ? Fin[(int64_t)c * fs + i] : 0.f;
  const float h = tf32_rn(x);
  F[(int64_t)c * fs + i] = h;
  F[(int64_t)(64 + c) * fs + i] = x - h;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

}  // namespace

bool make_tmap_sw128(CUtensorMap* out, const void* base, int64_t cols, int64_t rows, int64_t ld,
                     int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn();
  if (!encode) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t tc_split_floats(int64_t n) { return 2 * n * kSplitCols; }

template <int RP>
static cudaError_t launch_tc_t(const CUtensorMap& tmP, const CUtensorMap& tmA,
                               const CUtensorMap& tmB, float* P, int64_t ldp, int n, int num_sms,
                               unsigned* status, cudaStream_t s) {
  using Sh = TcShape<RP>;
  static const cudaError_t configured = cudaFuncSetAttribute(
      tc_update_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SmemBytes);
  if (configured != cudaSuccess) return configured;
  const long long T = (long long)((n + kBM - 1) / kBM) * ((n + Sh::BN - 1) / Sh::BN);
  const int grid = (int)(T < num_sms ? T : num_sms);
  tc_update_kernel<RP><<<grid, kTcThreads, Sh::SmemBytes, s>>>(tmP, tmA, tmB, P, ldp, n, status);
  return cudaGetLastError();
}

cudaError_t launch_tc_update(const CUtensorMap& tmP, const CUtensorMap& tmA,
                             const CUtensorMap& tmB, float* P, int64_t ldp, float* Acat,
                             float* Bcat, const float* U, const float* W, int64_t fs, int n, int r,
                             int num_sms, unsigned* status, cudaStream_t s) {
  if (r < 1 || r > kMaxTcR) return cudaErrorInvalidValue;
  const int half = r <= 32 ? 32 : 64;
  tc_split_kernel<<<(n + 31) / 32, 256, 0, s>>>(U, W, fs, n, r, half, Acat, Bcat);
  if (half == 32) return launch_tc_t<32>(tmP, tmA, tmB, P, ldp, n, num_sms, status, s);
  return launch_tc_t<64>(tmP, tmA, tmB, P, ldp, n, num_sms, status, s);
}

// CTAs of a products pass over an n x n view: one per SM, but at most
// kTpMaxParts - 1 per output tile and no more than the chunks
static long long tp_grid(int n, int num_sms) {
  const long long ot = (n + kBM - 1) / kBM, chunks = ot * ((n + 31) / 32);
  long long g = num_sms;
  if (g > ot * (kTpMaxParts - 1)) g = ot * (kTpMaxParts - 1);
  if (g > chunks) g = chunks;
  return g < 1 ? 1 : g;
}

// partial sets: a tile's chunks span at most ceil(G / ot) + 1 CTAs
int tp_parts(int n, int num_sms) {
  const long long ot = (n + kBM - 1) / kBM;
  const long long g = tp_grid(n, num_sms);
  return (int)((g + ot - 1) / ot + 1);
}

template <bool TR, int RP>
static cudaError_t launch_tp_t(const CUtensorMap& tmP, const CUtensorMap& tmF, float* out,
                               int64_t ps, int64_t cs, int n, int r_out, int parts, int num_sms,
                               unsigned* status, cudaStream_t s) {
  using Sh = TpShape<TR, RP>;
  static const cudaError_t configured = cudaFuncSetAttribute(
      tc_products_kernel<TR, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SmemBytes);
  if (configured != cudaSuccess) return configured;
  const int grid = (int)tp_grid(n, num_sms);
  tc_products_kernel<TR, RP><<<grid, kTpThreads, Sh::SmemBytes, s>>>(tmP, tmF, out, ps, cs, n,
                                                                     r_out, parts, status);
  return cudaGetLastError();
}

cudaError_t launch_tc_products(bool transpose, const float* P, int64_t ldp, const float* F,
                               int64_t fs, float* Fsplit, int n, int r, float* out, int64_t ps,
                               int64_t cs, int parts, int num_sms, unsigned* status,
                               cudaStream_t s) {
  if (r < 1 || r > kMaxTcR || parts != tp_parts(n, num_sms) || fs % 64 || fs < n)
    return cudaErrorInvalidValue;
  const int rp = r <= 32 ? 32 : 64;
  const int64_t tot = (int64_t)rp * n;
  tp_split_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(F, fs, n, r, rp, Fsplit);
  CUtensorMap tmP, tmF;
  // P: boxes of 32 columns x 128 rows (X) or 32 x 32 (Y); F: 32 columns of
  // K x rp factor rows (hi at row 0, lo at row 64)
  if (!make_tmap_sw128(&tmP, P, n, n, ldp, transpose ? 32 : 128) ||
      !make_tmap_sw128(&tmF, Fsplit, n, 128, fs, rp))
    return cudaErrorInvalidValue;
  if (transpose)
    return rp == 32 ? launch_tp_t<true, 32>(tmP, tmF, out, ps, cs, n, r, parts, num_sms, status, s)
                    : launch_tp_t<true, 64>(tmP, tmF, out, ps, cs, n, r, parts, num_sms, status, s);
  return rp == 32 ? launch_tp_t<false, 32>(tmP, tmF, out, ps, cs, n, r, parts, num_sms, status, s)
                  : launch_tp_t<false, 64>(tmP, tmF, out, ps, cs, n, r, parts, num_sms, status, s);
}

}  // namespace lv
