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

}  // namespace lv
