// FP32 view passes with a decoupled stage ring (included by lv_pass.cu).
//
// Same arithmetic and ownership as fused_pass_kernel / update_pass_kernel
// (every lane performs the same multiply-adds in the same order, with packed
// FP32x2 FMAs), but no CTA-wide barrier per batch:
//  * each stage of the ring has a "full" mbarrier (TMA bytes of the view tile
//    + the asynchronous copies of the batch's factor rows) and an "empty"
//    mbarrier that every warp arrives on once it has finished with the stage;
//  * warp 0 alone waits for "empty", combines the per-warp row sums of the
//    batch (fused pass), starts the cp.async copies of the factor rows of the
//    batch kStages ahead (tracked by "full" through
//    cp.async.mbarrier.arrive.noinc, so no warp waits for their latency) and
//    re-issues the TMA loads; the other warps run up to kStages-1 batches
//    ahead;
//  * the row sums P U are reduced inside each warp by a fixed butterfly
//    (shuffle reduce-scatter), so only R values per warp and row cross warps.
// Every wait is bounded; the first expired wait sets a CTA-wide abort flag
// that makes all later waits return at once, so a lost transaction ends the
// kernel with LINVIEW_ETIMEOUT latched instead of a hang.
// (Included inside namespace lv after update_pass_kernel and suffix_blocks.)

// Row sums P U: each of V = MC x MG values (MC factor columns x MG rows) is
// summed over the 32 lanes of a warp by a fixed butterfly (reduce-scatter):
// each level sends half of the remaining values to the partner lane and keeps
// the other half, then plain xor-sums finish (V - 1 + 5 - log2(V) shuffles
// for all V values).
// Reduce-scatter of MC x MG values (slot c * MG + g) in which the first
// log2(MC) levels need no lane selects: there each lane keeps the first half
// of its slots and adds its partner's second half, which works because lane
// L stores value (c, g) at slot ((c ^ cmask) * MG + g), cmask =
// scatter_mask<MC * MG>(L) / MG (so partners hold each other's halves).  The
// log2(MG) levels after them keep the half the lane's own bit selects.  On
// return, lanes with lane % (32 / (MC * MG)) == 0 hold the total of value
// (cmask, scatter_mask<MC * MG>(L) % MG).
template <int V>
__device__ __forceinline__ int scatter_mask(int lane) {
  constexpr int m = V >= 32 ? 5 : V >= 16 ? 4 : V >= 8 ? 3 : V >= 4 ? 2 : V >= 2 ? 1 : 0;
  return (lane >> (5 - m)) & (V - 1);
}

template <int MC, int MG>
__device__ __forceinline__ float mixed_levels(const float (&in)[MC * MG], int lane, int o) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int M = MC * MG;
  if constexpr (M == 1) {
    float v = in[0];
#pragma unroll
    for (int oo = o; oo >= 1; oo >>= 1) v += __shfl_xor_sync(FULL, v, oo);
    return v;
  } else if constexpr (MC > 1) {
    float out[M / 2];
#pragma unroll
    for (int i = 0; i < M / 2; ++i) out[i] = in[i] + __shfl_xor_sync(FULL, in[i + M / 2], o);
    return mixed_levels<MC / 2, MG>(out, lane, o >> 1);
  } else {
    const bool up = (lane & o) != 0;
    float out[M / 2];
#pragma unroll
    for (int i = 0; i < M / 2; ++i)
      out[i] = (up ? in[i + M / 2] : in[i]) + __shfl_xor_sync(FULL, up ? in[i] : in[i + M / 2], o);
    return mixed_levels<1, MG / 2>(out, lane, o >> 1);
  }
}

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned* status) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity, status)) return true;
  *abort_flag = 1;
  return false;
}

// One row of the in-place rank-R update p_k + sum_c u_c W(col_k, c) for the
// COLS columns of a thread.  R >= 2: the staged row u (16-byte aligned) is
// read once and the FMAs are paired over factor columns, (u_c, u_c+1) *
// (W(col_k, c), W(col_k, c+1)), summed in increasing c from the first packed
// product (no accumulator to set up) and finished as p_k + (even + odd): a
// fixed order, so results are reproducible.  R = 1: one FMA per entry, two
// columns per packed FMA.
template <int R, int COLS>
__device__ __forceinline__ void rank_update_row(const float* u, const float (&pv)[COLS],
                                                const float2 (&wp)[COLS][R >= 2 ? R / 2 : 1],
                                                float (&out)[COLS]) {
  if constexpr (R == 1) {
    const float2 uu = make_float2(u[0], u[0]);
#pragma unroll
    for (int m = 0; m < COLS / 2; ++m) {
      const float2 t = __ffma2_rn(uu, wp[m][0], make_float2(pv[2 * m], pv[2 * m + 1]));
      out[2 * m] = t.x;
      out[2 * m + 1] = t.y;
    }
  } else {
    float2 uu[R / 2];
    if constexpr (R >= 4) {
      const float4* u4 = reinterpret_cast<const float4*>(u);
#pragma unroll
      for (int c4 = 0; c4 < R / 4; ++c4) {
        const float4 t = u4[c4];
        uu[2 * c4] = make_float2(t.x, t.y);
        uu[2 * c4 + 1] = make_float2(t.z, t.w);
      }
    } else {
      uu[0] = *reinterpret_cast<const float2*>(u);
    }
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
      float2 acc = __fmul2_rn(uu[0], wp[k][0]);
#pragma unroll
      for (int c2 = 1; c2 < R / 2; ++c2) acc = __ffma2_rn(uu[c2], wp[k][c2], acc);
      out[k] = pv[k] + (acc.x + acc.y);
    }
  }
}

// ---------------------------------------------------------------------------
// Fused products (+ update) pass, FP32, R in {1, 2, 4, 8}; products only
// (no update) also R = 16.
// Thread (rg = warp / 4, tc = tid % 128) owns columns strip0 + 4 tc .. +3.
//  R <= 4: row group rg takes rows rg, rg+2, rg+4, rg+6 of every batch (all
//          R factor columns); every element is read and updated by one
//          thread, so updated tiles can leave by TMA store;
//  R >= 8 (SPLIT): row group rg takes the products P U and P^T V of factor
//          columns rg R/2 .. rg R/2 + R/2 - 1 on all 8 rows of the batch, and
//          the in-place update of rows 4 rg .. 4 rg + 3; this halves the
//          column factors each thread keeps in registers (R = 4 fits without:
//          89 us instead of 93 at n = 8192, with the TMA store).
// ---------------------------------------------------------------------------
template <int R, int MODE, bool TS>
__global__ void __launch_bounds__(kThreads, 2)
    fused_ws_kernel(const __grid_constant__ CUtensorMap tmap, const PassParams p) {
  using T = float;
  constexpr int COLS = 4;
  constexpr int STRIP = 128 * COLS;
  constexpr int BOXC = kBoxBytes / 4;
  constexpr int NB = STRIP / BOXC;
  constexpr int STAGE_ELEMS = kBatch * STRIP;
  constexpr bool DO_X = (MODE & 1) != 0;
  constexpr bool DO_Y = (MODE & 2) != 0;
  constexpr bool DO_U = (MODE & 4) != 0;
  constexpr bool PACK = R >= 2;
  constexpr int R2 = PACK ? R / 2 : 1;
  constexpr bool SPLIT = R >= 8;
  constexpr int RH = SPLIT ? R / 2 : R;          // factor columns of the products per group
  constexpr int RH2 = PACK ? RH / 2 : 1;         // ... as packed pairs
  constexpr int ROWS = SPLIT ? kBatch : kBatch / 2;  // batch rows a thread visits
  // rows whose products are reduced by one butterfly (G * RH values)
  constexpr int G = SPLIT ? (16 / RH < 4 ? 16 / RH : 4) : (R <= 4 ? ROWS : 1);
  constexpr int S = kStagesWs;
  static_assert(ROWS % G == 0 && G * RH <= 32, "butterfly grouping");
  // Without SPLIT every view element is read and updated by one thread, so
  // the updated rows go back into the stage and leave by TMA store (TS: the
  // tensor map's rows end on 16-byte units); with SPLIT both row groups read
  // every row, and each thread stores its own.
  constexpr bool TSTORE = TS && DO_U && !SPLIT;

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * S * STAGE_ELEMS);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  // 16-byte aligned so that four u or v values load as one 128-bit word;
  // regions a mode does not use take no space
  T* Us = reinterpret_cast<T*>(empty + S + 2);   // [S][kBatch][R] (DO_U)
  T* Vs = Us + (DO_U ? S * kBatch * R : 0);      // [S][kBatch][R] (DO_Y)
  T* Xw = Vs + (DO_Y ? S * kBatch * R : 0);      // [S][kBatch][4][R] warp sums (DO_X)
  double* Csh = reinterpret_cast<double*>(Xw + (DO_X ? S * kBatch * 4 * R : 0));  // [kThreads] core sums (DO_U && DO_Y)

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int rg = warp >> 2;
  const int wq = warp & 3;
  const int tc = tid & 127;
  const int cb = SPLIT ? rg * RH : 0;  // first factor column of this group's products
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
  // first row of batch b: a reversed pass walks the CTA's row range from its
  // last batch up to its first
  const bool rev = p.reverse != 0;
  auto batch_row = [&](int b) { return rb + (rev ? nbatch - 1 - b : b) * kBatch; };
  const T* Xf = static_cast<const T*>(p.Xf);
  const T* Yf = static_cast<const T*>(p.Yf);
  const T* Uu = static_cast<const T*>(p.Uu);
  const T* Wu = static_cast<const T*>(p.Wu);
  T* P = static_cast<T*>(p.P);
  constexpr bool STAGE_ROWS = DO_U || DO_Y;

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], STAGE_ROWS ? 33 : 1);  // expect_tx arrive (+ 32 cp.async arrivals)
      mbar_init(&empty[i], kThreads / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  // boxes of the strip that lie wholly past column n are never loaded: zero
  // them once, so that every row of a stage can be read without masks (the
  // loaded boxes read zeros past the view: TMA fills rows and columns outside
  // the tensor map with zeros, and a program's own views keep zero padding)
#pragma unroll
  for (int bx = 0; bx < NB; ++bx)
    if (strip0 + bx * BOXC >= n)
      for (int i = tid; i < S * kBatch * BOXC; i += kThreads)
        stages[(i / (kBatch * BOXC)) * STAGE_ELEMS + bx * kBatch * BOXC + i % (kBatch * BOXC)] = 0.f;
  __syncthreads();
  int nbox = 0;
#pragma unroll
  for (int bx = 0; bx < NB; ++bx) nbox += (strip0 + bx * BOXC < n) ? 1 : 0;
  const uint32_t stage_bytes = (uint32_t)(nbox * kBatch * BOXC * sizeof(T));

  // warp 0: start batch b in stage b % S (factor rows by cp.async, tile by TMA)
  auto produce_rows = [&](int b) {
    const int st = b % S;
    const int row0 = batch_row(b);
    const int nb = min(kBatch, re - row0);
    if constexpr (STAGE_ROWS) {
      // consecutive lanes take consecutive factor columns of a row: the shared
      // memory writes then fall in distinct banks (the reads are L2 hits)
      for (int idx = lane; idx < kBatch * R; idx += 32) {
        const int j = idx / R;
        const int c = idx % R;
        const bool ok = (j < nb) && (c < r);
        const int64_t g = ok ? (int64_t)c * p.fs + row0 + j : 0;
        if constexpr (DO_U) cp_async4(Us + (st * kBatch + j) * R + c, Uu + g, ok);
        if constexpr (DO_Y) cp_async4(Vs + (st * kBatch + j) * R + c, Yf + g, ok);
      }
      cp_async_arrive_noinc(&full[st]);
    }
  };
  auto produce_tile = [&](int b) {
    const int st = b % S;
    const int row0 = batch_row(b);
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&full[st], stage_bytes);
#pragma unroll
      for (int bx = 0; bx < NB; ++bx) {
        if (strip0 + bx * BOXC < n)
          tma_load_2d(stages + st * STAGE_ELEMS + bx * kBatch * BOXC, &tmap, strip0 + bx * BOXC,
                      row0, &full[st]);
      }
    }
  };
  auto produce = [&](int b) {
    produce_rows(b);
    produce_tile(b);
  };
  int issued = 0;
  // The view is not written by the kernels launched just before this one, so
  // its first tiles are requested before waiting on them; the factors and the
  // partial-sum buffers are (programmatic dependent launch).
  if (warp == 0)
    for (int b = 0; b < S && b < nbatch; ++b) produce_tile(b);
  griddep_wait();
  griddep_launch_dependents();
  if (warp == 0) {
    for (int b = 0; b < S && b < nbatch; ++b) produce_rows(b);
    issued = min(S, nbatch);
  }

  // Lane layout of the row products P U: this lane keeps the product of
  // (factor column c, row-in-group g) at slot (c ^ cmask) * G + g, so that
  // the butterfly's column levels need no lane selects (mixed_levels).
  const int vmask = scatter_mask<G * RH>(lane);
  const int cmask = vmask / G, rmask = vmask % G;
  // column-side factors for this thread's 4 columns (X slots permuted by cmask)
  float2 ucol2[COLS][RH2];  // PACK: (U(col_k, cb+(2c2^cmask)), U(col_k, cb+((2c2+1)^cmask)))
  float2 yacc2[COLS][RH2];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int col = col0 + k;
#pragma unroll
    for (int c2 = 0; c2 < RH2; ++c2) {
      const int c = cb + ((PACK ? 2 * c2 : 0) ^ cmask);
      const int cn = cb + ((PACK ? 2 * c2 + 1 : 0) ^ cmask);
      const bool ok0 = DO_X && (c < r) && (col < n);
      const bool ok1 = DO_X && PACK && (cn < r) && (col < n);
      ucol2[k][c2] = make_float2(ok0 ? Xf[(int64_t)c * p.fs + col] : 0.f,
                                 ok1 ? Xf[(int64_t)cn * p.fs + col] : 0.f);
      yacc2[k][c2] = make_float2(0.f, 0.f);
    }
  }
  // R >= 2: wp[k][c2] = (W(col_k, 2 c2), W(col_k, 2 c2 + 1)), paired over
  // factor columns; R = 1: wp[m][0] = (W(col_2m, 0), W(col_2m+1, 0))
  float2 wp[COLS][R2];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
#pragma unroll
    for (int c2 = 0; c2 < R2; ++c2) {
      // (column, factor column) of the two entries of wp[k][c2]
      const int ca = PACK ? col0 + k : col0 + 2 * k, fa = PACK ? 2 * c2 : 0;
      const int cb2 = PACK ? ca : ca + 1, fb = PACK ? fa + 1 : 0;
      const bool use = DO_U && (PACK || k < 2);
      wp[k][c2] = make_float2(use && fa < r && ca < n ? Wu[(int64_t)fa * p.fs + ca] : 0.f,
                              use && fb < r && cb2 < n ? Wu[(int64_t)fb * p.fs + cb2] : 0.f);
    }
  }
  const int box = (tc * COLS) / BOXC;
  const int inbox = (tc * COLS) % BOXC;
  const bool vec_ok = (col0 + COLS <= n);
  // the same for the whole warp (a vote, so the compiler sees a uniform
  // branch); only the warps at the right edge of the view take the other path
  const bool warp_vec = __all_sync(0xffffffffu, vec_ok);
  // factor core C = V^T U over this CTA's rows (FP64).  The CTA owns the
  // entries e = s + i * gC; each entry is split over LPE threads, thread li
  // taking batch rows li, li + LPE, ..., so every thread does at most
  // kBatch / LPE independent FP64 FMAs per batch (no dependent chain, which
  // on this part would make its warp the slowest).  Threads are taken from
  // the end of the CTA so warp 0, which refills the ring, stays free.
  const int ncore = (r * r > s) ? (r * r - s + p.gC - 1) / p.gC : 0;  // entries owned
  const int LPE = ncore * kBatch <= kThreads ? kBatch : kBatch / 2;
  const int cslot = kThreads - 1 - tid;
  const int centry = cslot / LPE;
  const int cli = cslot % LPE;
  const int ecore = s + centry * p.gC;
  const bool do_core = DO_U && DO_Y && (p.Cpart != nullptr) && (centry < ncore);
  if (do_core) Csh[cslot] = 0.0;  // one slot per thread (kept out of registers)
  int waited = 0;  // batches whose "full" phase this thread has seen complete
  // batch row of the jj-th row this thread visits
  auto row_of = [&](int jj) { return SPLIT ? ((jj + 4 * rg) & (kBatch - 1)) : rg + 2 * jj; };

  for (int b = 0; b < nbatch; ++b) {
    const int st = b % S;
    const uint32_t parity = (uint32_t)((b / S) & 1);
    const int row0 = batch_row(b);
    const int nb = min(kBatch, re - row0);
    const bool full_batch = nb == kBatch;  // the same for the whole CTA
    if (wait_or_abort(&full[st], parity, abort_flag, p.status)) {
      waited = b + 1;
      const T* Ust = Us + st * kBatch * R;
      const T* Vst = Vs + st * kBatch * R;
      if (do_core) {
        const int c1 = ecore / r, c2 = ecore % r;
        double acc = Csh[cslot];
        for (int j = cli; j < kBatch; j += LPE)
          acc = fma((double)Vst[j * R + c1], (double)Ust[j * R + c2], acc);
        Csh[cslot] = acc;
      }
      T* sp = stages + st * STAGE_ELEMS + box * kBatch * BOXC + inbox;
      float xg[RH * G];  // products of the current group of rows
      auto do_row = [&](int j, int g, bool upd) {
          const float4 v4 = *reinterpret_cast<const float4*>(sp + j * BOXC);
          const float pvs[COLS] = {v4.x, v4.y, v4.z, v4.w};
          if constexpr (PACK) {
            const float2 pd[COLS] = {make_float2(v4.x, v4.x), make_float2(v4.y, v4.y),
                                     make_float2(v4.z, v4.z), make_float2(v4.w, v4.w)};
            if constexpr (DO_Y) {
              float2 vv[RH2];
              if constexpr (RH >= 4) {
                const float4* vr4 = reinterpret_cast<const float4*>(Vst + j * R + cb);
#pragma unroll
                for (int c4 = 0; c4 < RH / 4; ++c4) {
                  const float4 t = vr4[c4];
                  vv[2 * c4] = make_float2(t.x, t.y);
                  vv[2 * c4 + 1] = make_float2(t.z, t.w);
                }
              } else {
                vv[0] = *reinterpret_cast<const float2*>(Vst + j * R + cb);
              }
#pragma unroll
              for (int c2 = 0; c2 < RH2; ++c2)
#pragma unroll
                for (int k = 0; k < COLS; ++k) yacc2[k][c2] = __ffma2_rn(pd[k], vv[c2], yacc2[k][c2]);
            }
            if constexpr (DO_X) {
              float2 x2[RH2];
#pragma unroll
              for (int c2 = 0; c2 < RH2; ++c2) x2[c2] = make_float2(0.f, 0.f);
#pragma unroll
              for (int k = 0; k < COLS; ++k)
#pragma unroll
                for (int c2 = 0; c2 < RH2; ++c2) x2[c2] = __ffma2_rn(pd[k], ucol2[k][c2], x2[c2]);
#pragma unroll
              for (int c2 = 0; c2 < RH2; ++c2) {
                xg[(2 * c2) * G + g] = x2[c2].x;
                xg[(2 * c2 + 1) * G + g] = x2[c2].y;
              }
            }
          } else {
            if constexpr (DO_Y) {
              const float v = Vst[j * R];
#pragma unroll
              for (int k = 0; k < COLS; ++k) yacc2[k][0].x = fmaf(pvs[k], v, yacc2[k][0].x);
            }
            if constexpr (DO_X) {
              float x = 0.f;
#pragma unroll
              for (int k = 0; k < COLS; ++k) x = fmaf(pvs[k], ucol2[k][0].x, x);
              xg[g] = x;
            }
          }
          if constexpr (DO_U) {
            if (upd && (TSTORE || full_batch || j < nb)) {
              float o[COLS];
              rank_update_row<R, COLS>(Ust + j * R, pvs, wp, o);
              if constexpr (TSTORE) {
                *reinterpret_cast<float4*>(sp + j * BOXC) = make_float4(o[0], o[1], o[2], o[3]);
              } else {
                T* dst = P + (int64_t)(row0 + j) * p.ldp + col0;
                if (warp_vec || vec_ok) {
                  *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                  for (int k = 0; k < COLS; ++k)
                    if (col0 + k < n) dst[k] = o[k];
                }
              }
            }
          }
      };
      auto finish_group = [&](int jj) {  // after the last row of a group: one butterfly
        if constexpr (DO_X) {
          if ((jj % G) == G - 1) {
            const float tot = mixed_levels<RH, G>(xg, lane, 16);  // value (cmask, rmask)
            const int jr = row_of(jj - (G - 1) + rmask);
            if ((lane % (32 / (G * RH))) == 0)
              Xw[((st * kBatch + jr) * 4 + wq) * R + cb + cmask] = tot;
          }
        }
      };
      // whether the row visited at step jj is one this thread updates: its
      // own half of the batch (SPLIT: the first four rows it visits)
      auto updates_row = [&](int jj) { return SPLIT ? jj < kBatch / 2 : true; };
      // rows past the view (a partial last batch) read zeros from the stage
      // and the factor rows, so they add nothing to the products and need no
      // guard (only their stores are skipped); R = 16 keeps one per row, which
      // stops the compiler from interleaving rows past the register budget
#pragma unroll
      for (int jj = 0; jj < ROWS; ++jj) {
        if (R < 16 || row_of(jj) < nb) {
          do_row(row_of(jj), jj % G, updates_row(jj));
        } else if constexpr (DO_X) {
#pragma unroll
          for (int c = 0; c < RH; ++c) xg[c * G + jj % G] = 0.f;
        }
        finish_group(jj);
      }
      if constexpr (TSTORE) fence_proxy_async();  // rows written back, before the TMA store
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if (warp == 0) {
      // all warps are done with batch b: store it (TSTORE), fold its row
      // sums, refill a stage
      if (wait_or_abort(&empty[st], parity, abort_flag, p.status)) {
        if constexpr (TSTORE) {
          if (lane == 0) {
#pragma unroll
            for (int bx = 0; bx < NB; ++bx)
              if (strip0 + bx * BOXC < n)
                tma_store_2d(&tmap, stages + st * STAGE_ELEMS + bx * kBatch * BOXC,
                             strip0 + bx * BOXC, row0);
            bulk_commit();
          }
        }
        if constexpr (DO_X) {
          T* xo = static_cast<T*>(p.Xpart) + (int64_t)s * p.xp_s;
          for (int idx = lane; idx < kBatch * R; idx += 32) {
            const int j = idx / R, c = idx % R;
            if (j < nb && c < r) {
              const T* w4 = Xw + ((st * kBatch + j) * 4) * R + c;
              xo[(int64_t)c * p.part_cs + row0 + j] = ((w4[0] + w4[R]) + w4[2 * R]) + w4[3 * R];
            }
          }
        }
        if constexpr (TSTORE) {
          // the stage of batch b - 1, whose store has been read out, takes
          // batch b - 1 + S
          if (b >= 1 && b - 1 + S < nbatch) {
            if (lane == 0) bulk_wait_read<1>();
            __syncwarp();
            produce(b - 1 + S);
            ++issued;
          }
        } else if (b + S < nbatch) {
          __syncwarp();
          produce(b + S);
          ++issued;
        }
      }
    }
  }
  if (warp == 0) {
    // stores complete before the ring is reused below or the CTA exits
    if (TSTORE && lane == 0) bulk_wait0();
    // on an abort, wait (bounded) for the copies issued but never waited on
    if (*abort_flag)
      for (int bb = waited; bb < issued; ++bb)
        mbar_wait_bounded(&full[bb % S], (uint32_t)((bb / S) & 1), nullptr);
  }
  if (DO_U && DO_Y && p.Cpart != nullptr) {
    __syncthreads();
    if (do_core && cli == 0) {  // fixed-order sum of the entry's LPE partials
      double sum = 0.0;
      for (int i = 0; i < LPE; ++i) sum += Csh[centry * LPE + i];
      p.Cpart[(int64_t)q * r * r + ecore] = sum;
    }
  }
  if constexpr (DO_Y) {
    T* yo = static_cast<T*>(p.Ypart) + (int64_t)q * p.yp_q;
    if constexpr (SPLIT) {
      // each group holds whole column sums of its own factor columns
      __syncthreads();
      if (col0 < n && !*abort_flag) {
#pragma unroll
        for (int c2 = 0; c2 < RH2; ++c2) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = cb + 2 * c2 + h;
            if (c >= r) break;
            const float vals[COLS] = {h ? yacc2[0][c2].y : yacc2[0][c2].x,
                                      h ? yacc2[1][c2].y : yacc2[1][c2].x,
                                      h ? yacc2[2][c2].y : yacc2[2][c2].x,
                                      h ? yacc2[3][c2].y : yacc2[3][c2].x};
            T* dst = yo + (int64_t)c * p.part_cs + col0;
            if (vec_ok) {
              *reinterpret_cast<float4*>(dst) = make_float4(vals[0], vals[1], vals[2], vals[3]);
            } else {
#pragma unroll
              for (int k = 0; k < COLS; ++k)
                if (col0 + k < n) dst[k] = vals[k];
            }
          }
        }
      }
    } else {
      __syncthreads();
      T* yc = stages;  // [k][c][tc], reusing the ring
      if (rg == 1) {
#pragma unroll
        for (int k = 0; k < COLS; ++k)
#pragma unroll
          for (int c2 = 0; c2 < R2; ++c2) {
            yc[(k * R + (PACK ? 2 * c2 : 0)) * 128 + tc] = yacc2[k][c2].x;
            if (PACK) yc[(k * R + 2 * c2 + 1) * 128 + tc] = yacc2[k][c2].y;
          }
      }
      __syncthreads();
      if (rg == 0 && col0 < n && !*abort_flag) {
#pragma unroll
        for (int c = 0; c < R; ++c) {
          if (c >= r) break;
          float vals[COLS];
#pragma unroll
          for (int k = 0; k < COLS; ++k) {
            const float mine = (c & 1) ? yacc2[k][c / 2].y : yacc2[k][c / 2].x;
            vals[k] = mine + yc[(k * R + c) * 128 + tc];
          }
          T* dst = yo + (int64_t)c * p.part_cs + col0;
          if (vec_ok) {
            *reinterpret_cast<float4*>(dst) = make_float4(vals[0], vals[1], vals[2], vals[3]);
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k)
              if (col0 + k < n) dst[k] = vals[k];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Update-only pass, FP32.  COLS = 4: two row groups of 128 threads, thread
// (rg, tc) owns columns strip0 + 4 tc .. +3 and rows rg, rg+2, ... of each
// batch (each broadcast U row is read by 4 warps); COLS = 2: one group of 256
// threads owning 2 columns each (R <= 32); COLS = 1: one column each (R = 64,
// whose column factor fills 64 registers per column).
// ---------------------------------------------------------------------------
template <int R, int COLS, bool TS>
__global__ void __launch_bounds__(kThreads, 2)
    update_ws_kernel(const __grid_constant__ CUtensorMap tmap, const PassParams p) {
  using T = float;
  constexpr int GROUPS = COLS == 4 ? 2 : 1;
  constexpr int GT = kThreads / GROUPS;  // threads per row group
  constexpr int STRIP = GT * COLS;
  constexpr int BOXC = kBoxBytes / 4;
  constexpr int NB = STRIP / BOXC;
  constexpr int STAGE_ELEMS = kBatch * STRIP;
  constexpr int S = kStagesWs;
  static_assert(NB * BOXC == STRIP, "strip must be whole boxes");

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T* stages = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(T) * S * STAGE_ELEMS);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  T* Us = reinterpret_cast<T*>(empty + S + 2);  // [S][kBatch][R], 16-byte aligned

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int rg = GROUPS == 2 ? (tid / GT) : 0;
  const int tc = tid % GT;
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
  const bool rev = p.reverse != 0;  // as in the fused pass
  auto batch_row = [&](int b) { return rb + (rev ? nbatch - 1 - b : b) * kBatch; };
  const T* Uu = static_cast<const T*>(p.Uu);
  const T* Wu = static_cast<const T*>(p.Wu);
  T* P = static_cast<T*>(p.P);

  if (tid == 0) {
    prefetch_tmap(&tmap);
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 33);
      mbar_init(&empty[i], kThreads / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  int nbox = 0;
#pragma unroll
  for (int bx = 0; bx < NB; ++bx) nbox += (strip0 + bx * BOXC < n) ? 1 : 0;
  const uint32_t stage_bytes = (uint32_t)(nbox * kBatch * BOXC * sizeof(T));
  auto produce_rows = [&](int b) {
    const int st = b % S;
    const int row0 = batch_row(b);
    const int nb = min(kBatch, re - row0);
    for (int idx = lane; idx < kBatch * R; idx += 32) {  // lanes over columns (see above)
      const int j = idx / R;
      const int c = idx % R;
      const bool ok = (j < nb) && (c < r);
      const int64_t g = ok ? (int64_t)c * p.fs + row0 + j : 0;
      cp_async4(Us + (st * kBatch + j) * R + c, Uu + g, ok);
    }
    cp_async_arrive_noinc(&full[st]);
  };
  auto produce_tile = [&](int b) {
    const int st = b % S;
    const int row0 = batch_row(b);
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&full[st], stage_bytes);
#pragma unroll
      for (int bx = 0; bx < NB; ++bx) {
        if (strip0 + bx * BOXC < n)
          tma_load_2d(stages + st * STAGE_ELEMS + bx * kBatch * BOXC, &tmap, strip0 + bx * BOXC,
                      row0, &full[st]);
      }
    }
  };
  auto produce = [&](int b) {
    produce_rows(b);
    produce_tile(b);
  };
  int issued = 0;
  // first tiles of the view before waiting on the previous kernel (see the
  // fused pass; a block of a wide update that follows another block on the
  // same view is launched without programmatic serialisation, so its
  // predecessor has completed); the factor rows after
  if (warp == 0)
    for (int b = 0; b < S && b < nbatch; ++b) produce_tile(b);
  griddep_wait();
  griddep_launch_dependents();
  if (warp == 0) {
    for (int b = 0; b < S && b < nbatch; ++b) produce_rows(b);
    issued = min(S, nbatch);
  }

  T wcol[COLS][R];
#pragma unroll
  for (int k = 0; k < COLS; ++k) {
    const int col = col0 + k;
#pragma unroll
    for (int c = 0; c < R; ++c)
      wcol[k][c] = (c < r && col < n) ? Wu[(int64_t)c * p.fs + col] : 0.f;
  }
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
    default: break;
  }
  // column factor in the layout of rank_update_row
  constexpr int R2 = R >= 2 ? R / 2 : 1;
  float2 wp[COLS][R2];
#pragma unroll
  for (int k = 0; k < COLS; ++k)
#pragma unroll
    for (int c2 = 0; c2 < R2; ++c2)
      wp[k][c2] = R >= 2 ? make_float2(wcol[k][2 * c2], wcol[k][2 * c2 + 1])
                         : make_float2(k < COLS / 2 ? wcol[2 * k][0] : 0.f,
                                       k < COLS / 2 ? wcol[2 * k + 1][0] : 0.f);
  const int box = (tc * COLS) / BOXC;
  const int inbox = (tc * COLS) % BOXC;
  const bool vec_ok = (col0 + COLS <= n);
  const bool any_col = (col0 < n);
  int waited = 0;

  for (int b = 0; b < nbatch; ++b) {
    const int st = b % S;
    const uint32_t parity = (uint32_t)((b / S) & 1);
    const int row0 = batch_row(b);
    const int nb = min(kBatch, re - row0);
    const bool ready = wait_or_abort(&full[st], parity, abort_flag, p.status);
    if (ready) waited = b + 1;
    if (ready && any_col) {
      T* sp = stages + st * STAGE_ELEMS + box * kBatch * BOXC + inbox;
      const T* Ust = Us + st * kBatch * R;
      // TS: the updated row goes back to its place in the stage, which warp 0
      // then stores with TMA (rows and columns past the view are clipped)
      auto row = [&](int j) {
          float pv[COLS];
          if constexpr (COLS == 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(sp + j * BOXC);
            pv[0] = v4.x; pv[1] = v4.y; pv[2] = v4.z; pv[3] = v4.w;
          } else if constexpr (COLS == 2) {
            const float2 v2 = *reinterpret_cast<const float2*>(sp + j * BOXC);
            pv[0] = v2.x; pv[1] = v2.y;
          } else {
            pv[0] = sp[j * BOXC];
          }
          float o[COLS];
          rank_update_row<R, COLS>(Ust + j * R, pv, wp, o);
          T* dst = TS ? sp + j * BOXC : P + (int64_t)(row0 + j) * p.ldp + col0;
          if (TS || vec_ok) {
            if constexpr (COLS == 4)
              *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            else if constexpr (COLS == 2)
              *reinterpret_cast<float2*>(dst) = make_float2(o[0], o[1]);
            else
              dst[0] = o[0];
          } else {
#pragma unroll
            for (int k = 0; k < COLS; ++k)
              if (col0 + k < n) dst[k] = o[k];
          }
      };
      if (nb == kBatch) {  // full batch: no per-row guards, rows interleave
#pragma unroll
        for (int jj = 0; jj < kBatch / GROUPS; ++jj) row(rg + GROUPS * jj);
      } else {
#pragma unroll
        for (int jj = 0; jj < kBatch / GROUPS; ++jj)
          if (rg + GROUPS * jj < nb) row(rg + GROUPS * jj);
      }
      if constexpr (TS) fence_proxy_async();  // rows written back, before the TMA store
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if (warp == 0) {
      if (wait_or_abort(&empty[st], parity, abort_flag, p.status)) {
        if constexpr (TS) {
          // all warps have written batch b back: store it; the stage of
          // batch b - 1, whose store has been read out, takes batch b - 1 + S
          if (lane == 0) {
#pragma unroll
            for (int bx = 0; bx < NB; ++bx)
              if (strip0 + bx * BOXC < n)
                tma_store_2d(&tmap, stages + st * STAGE_ELEMS + bx * kBatch * BOXC,
                             strip0 + bx * BOXC, row0);
            bulk_commit();
          }
          if (b >= 1 && b - 1 + S < nbatch) {
            if (lane == 0) bulk_wait_read<1>();
            __syncwarp();
            produce(b - 1 + S);
            ++issued;
          }
        } else if (b + S < nbatch) {
          __syncwarp();
          produce(b + S);
          ++issued;
        }
      }
    }
  }
  if (warp == 0) {
    if (TS && lane == 0) bulk_wait0();  // stores complete before the shared memory goes away
    if (*abort_flag)  // on an abort, wait (bounded) for the copies never waited on
      for (int bb = waited; bb < issued; ++bb)
        mbar_wait_bounded(&full[bb % S], (uint32_t)((bb / S) & 1), nullptr);
  }
}
