// Internal declarations shared by the LINVIEW translation units (kernels and
// the C-ABI/engine).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lv {

// Launch ``k`` with programmatic stream serialisation (the kernel calls
// griddep_wait() before it reads what earlier kernels of the stream wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, unsigned block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

constexpr int kThreads = 256;   // threads per pass CTA
constexpr int kBatch = 8;       // rows per pipeline stage = TMA box height = warps per CTA
constexpr int kStages = 4;      // TMA ring depth (generic passes)
constexpr int kStagesWs = 6;    // TMA ring depth of the decoupled-ring FP32 passes
constexpr int kBoxBytes = 1024; // bytes per TMA box row (256 floats / 128 doubles)
constexpr int kMaxAsmR = 64;    // widest factor block U_h of one assembly (= the widest Gram block)
constexpr int kMaxFusedR = 8;   // widest factor block of the fused products pass
constexpr int kMaxProductR = 16;  // widest factor block of an FP32 products-only pass
constexpr int kMaxUpdateR = 32;   // widest factor block of one update pass (shared-memory
                                  // broadcasts of the factor rows bound wider blocks)

// Pass modes: which of X = P Xf, Y = P^T Yf and P += Uu Wu^T a launch does.
enum PassMode : int { kModeXYU = 7, kModeXY = 3, kModeXU = 5, kModeX = 1, kModeY = 2 };
constexpr int kMaxColSumR = 32;  // widest factor block of an FP32 column-sums-only pass (Y)

// Everything a view pass needs.  Factors are column-major with column
// stride ``fs`` (elements); the partial-sum arrays are [block][column][row]
// with column stride ``part_cs`` and block strides ``xp_s`` / ``yp_q``.
struct PassParams {
  void* P;            // view, row-major
  int64_t ldp;        // leading dimension of P (elements)
  int n;              // P is n x n
  const void* Xf;     // X factor (n x r) or null
  const void* Yf;     // Y factor (n x r) or null
  const void* Uu;     // update left factor (n x r) or null
  const void* Wu;     // update right factor (n x r) or null
  int64_t fs;         // factor column stride
  int r;              // valid factor columns (<= template width)
  void* Xpart;        // [gC][r][part_cs] row-sum partials (pre-offset to the column block)
  void* Ypart;        // [gR][r][part_cs] column-sum partials
  int64_t part_cs;
  int64_t xp_s;
  int64_t yp_q;
  int gC, gR;         // column strips x row ranges; grid = gC * gR
  int rows_per_cta;   // multiple of kBatch
  unsigned* status;   // device status word
  double* Cpart;      // fused XYU pass: per-row-range V^T U partials [gR][r*r] (or null)
  int suffix_rin;     // update pass: >0 applies block suffix sums (block width) to Wu
  int tma_store;      // FP32 passes may store updated tiles with TMA: the tensor map's
                      // row extent is a multiple of 16 bytes (a TMA store writes whole
                      // 16-byte units, so a row ending inside one would overwrite the
                      // elements past the view, e.g. a caller's padding)
  int reverse;        // FP32 passes: each CTA visits its row batches last to first.
                      // Alternating it over consecutive passes on one view makes a
                      // pass start on the rows the previous one read last, which are
                      // still in L2 (the FP64 pass ignores it)
};

// Host: grid geometry for a pass over an n x n view.
struct PassGeom {
  int strip, gC, gR, rows_per_cta;
};
PassGeom fused_geom(int elem_bytes, int n, int num_sms);
PassGeom update_geom(int elem_bytes, int R, int n, int num_sms);

// Host: 2-D tensor map over a row-major matrix (rows x cols, ld elements),
// box = (kBoxBytes / elem_bytes) columns x kBatch rows.
bool make_tmap(CUtensorMap* out, const void* base, int elem_bytes, int64_t cols, int64_t rows,
               int64_t ld);

// Host: FP32 tensor map with 32-column x box_rows boxes and 128-byte swizzle
// (operand and tile layout of the tensor-core update pass).
bool make_tmap_sw128(CUtensorMap* out, const void* base, int64_t cols, int64_t rows, int64_t ld,
                     int box_rows);
// Floats of the split-factor scratch of the tensor-core update pass (A_cat
// then B_cat, n x 128 each).
int64_t tc_split_floats(int64_t n);
constexpr int kMaxTcR = 64;  // widest factor block of one tensor-core update pass
constexpr int kTpMaxParts = 8;  // K parts (partial sums) of a tensor-core products pass
// Tensor-core products pass (FP32, 1 <= r <= 64): transpose = false: the
// partial sums of X = P F over column ranges of P; true: of Y = P^T F over
// row ranges; ``parts`` = tp_parts(n, num_sms) partial sets, every one
// written.  Partial q, factor column c, output row i lands at
// out[q ps + c cs + i].  F column-major (column stride fs, a multiple of 64,
// >= n); Fsplit is scratch of 128 x fs floats (the split factor).
cudaError_t launch_tc_products(bool transpose, const float* P, int64_t ldp, const float* F,
                               int64_t fs, float* Fsplit, int n, int r, float* out, int64_t ps,
                               int64_t cs, int parts, int num_sms, unsigned* status,
                               cudaStream_t s);
// partial sets the products pass writes for an n x n view (<= kTpMaxParts)
int tp_parts(int n, int num_sms);
// Tensor-core update pass P += U W^T (FP32 view, 17 <= r <= 64 factor
// columns, split TF32): splits U, W into the scratch, then one persistent
// launch over 128 x 64 tiles.  tmP:
// make_tmap_sw128 over the view P (box rows 128, row stride ldp); tmA / tmB:
// over A_cat (128 columns, box rows 128) / B_cat (128 columns, box rows 32).
cudaError_t launch_tc_update(const CUtensorMap& tmP, const CUtensorMap& tmA,
                             const CUtensorMap& tmB, float* P, int64_t ldp, float* Acat,
                             float* Bcat, const float* U, const float* W, int64_t fs, int n, int r,
                             int num_sms, unsigned* status, cudaStream_t s);

// Own dense GEMMs (lv_gemm.cu).
// Split-TF32 operand rows: rows x tc_split_ld(K) floats, row i = [hi | lo]
// (each half rup(K, 32) long, zero past K).
int64_t tc_split_ld(int64_t K);
// Split the rows of op(X) (element (i, k) at X[i * rs + k * cs], rs or cs == 1)
// into dst (ldd >= tc_split_ld(K)).
cudaError_t launch_split_rows(const float* X, int64_t rs, int64_t cs, int rows, int K, float* dst,
                              int64_t ldd, cudaStream_t s);
// D (M x N, row-major, ldd) = alpha A_s B_s^T + beta C on the tensor cores
// (split TF32, FP32 accumulation), A_s / B_s split rows of inner length K
// (16-byte aligned).  C may alias D (beta == 0 ignores it).  ``work``
// (work_floats floats, may be null): room for the K parts of a product with
// too few tiles to fill the SMs (split K, parts summed in a fixed order).
cudaError_t launch_tc_gemm(const float* As, const float* Bs, int M, int N, int K, float* D,
                           int64_t ldd, const float* C, int64_t ldc, float alpha, float beta,
                           int num_sms, unsigned* status, cudaStream_t s, float* work = nullptr,
                           int64_t work_floats = 0);
// C (M x N) = alpha A B + beta C on the CUDA cores, A(m, k) = A[m a_rs + k a_cs],
// B(k, n) = B[k b_rs + n b_cs], C(m, n) = C[m c_rs + n c_cs]; long inner
// dimensions are split over ``work`` (work_elems elements, may be null) and
// the partials summed in a fixed order.  ``batch`` products at once: entry b
// reads A + b a_bs, B + b b_bs and writes C + b c_bs (strides may be negative).
template <typename T>
cudaError_t launch_gemm_simt(int M, int N, int K, T alpha, const T* A, int64_t a_rs, int64_t a_cs,
                             const T* B, int64_t b_rs, int64_t b_cs, T beta, T* C, int64_t c_rs,
                             int64_t c_cs, T* work, int64_t work_elems, int num_sms,
                             cudaStream_t s, int batch = 1, int64_t a_bs = 0, int64_t b_bs = 0,
                             int64_t c_bs = 0);

// Launchers (return cudaGetLastError()).  R is the runtime factor width,
// bucketed internally to a compiled width.  The passes are launched with
// programmatic stream serialisation, and the FP32 passes request their first
// view tiles before waiting on the kernel before them: that kernel must not
// write the view.  An update launched right after another pass that wrote
// the same view (the second block of a wide update) takes programmatic =
// false: a plain launch, which starts only once that kernel has completed.
template <typename T>
cudaError_t launch_fused(const PassParams& p, const CUtensorMap& tm, int R, int mode,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_update(const PassParams& p, const CUtensorMap& tm, int R, cudaStream_t s,
                          bool programmatic = true);

// Factor cores and assembly (lv_core.cu).
// C (r x r, FP64, row-major) = V^T U over n rows; deterministic two-level
// reduction using Cpart (grid x r*r doubles) and a ticket counter.  FP32
// programs may also take C as double-float pairs (Cdf, r x r float2).
template <typename T>
cudaError_t launch_gram(const T* V, const T* U, int64_t fs, int n, int r, double* Cpart,
                        unsigned* ticket, double* C, unsigned* status, cudaStream_t s,
                        float2* Cdf = nullptr);
int gram_grid(int n);

struct AssembleParams {
  int n, r_h;             // rows, current factor width
  int r_out;              // columns of X_h / Y_h to assemble (0 = r_h)
  int64_t fs;             // arena column stride
  const void* Xpart; int gC; int64_t xp_s;   // row-sum partials of P_h U_h
  const void* Ypart; int gR; int64_t yp_q;   // column-sum partials of P_h^T V_h (or null)
  int64_t part_cs;
  const double* C;        // r_h x r_h = V_h^T U_h, summed over nC partial blocks (the first
                          // r_out columns are used)
  int nC;                 // number of [r_h*r_h] partial blocks in C (1 = already reduced)
  const void* Uh;         // U_h (n x r_h)
  void* Unew;             // destination of X_h + U_h C_h (n x r_h), = U arena + r_h columns
  void* Ynew;             // destination of Y_h (n x r_h), = V arena left of V_h
  unsigned* status;       // device status word: a non-finite C_h entry latches
                          // kStatusNonFinite (or null)
};
template <typename T>
cudaError_t launch_assemble(const AssembleParams& a, cudaStream_t s);

// One bounded wait that always expires (diagnostic; see lv_core.cu).
cudaError_t launch_bounded_wait_probe(uint64_t limit_ns, unsigned* status,
                                      unsigned long long* waited_ns, cudaStream_t s);

// Suffix block sums: W[:, a-block] = sum_{b >= a} V[:, b-block] (blocks of r_in).
template <typename T>
cudaError_t launch_suffix_sums(const T* V, T* W, int64_t fs, int n, int width, int r_in,
                               cudaStream_t s);

// Copy a row-major user matrix (rows x cols, ld) into column-major storage
// (column stride fs) -- factor ingest.
template <typename T>
cudaError_t launch_rm_to_cm(const T* src, int64_t ld, T* dst, int64_t fs, int rows, int cols,
                            cudaStream_t s);
// e_row as one column (column-major, n rows).
template <typename T>
cudaError_t launch_unit_column(T* dst, int n, int row, cudaStream_t s);

// Sum of column-major partial blocks: out[c][j] = sum_b part[b][c][j].
template <typename T>
cudaError_t launch_sum_partials(const T* part, int blocks, int64_t block_stride, int64_t cs,
                                int n, int r, T* out, int64_t out_cs, cudaStream_t s);

// Elementwise helpers.
template <typename T>
cudaError_t launch_axpy_rows(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                             int cols, cudaStream_t s);  // y += alpha x (row-major blocks)
template <typename T>
cudaError_t launch_scale_copy(T* y, int64_t ldy, const T* x, int64_t ldx, T alpha, int rows,
                              int cols, cudaStream_t s);  // y = alpha x
// Linear-model T panel update, all k views in one launch: T_i(j, q) =
// Tp[j ldT + i p + q] += sum_{t < i r} K[t fs + j] M[((k - i) r + t) ldm + q]
// (one launch for all views; its shared memory, (16 + 64) k r elements, must fit
// the device's opt-in limit: panel_update_fits)
template <typename T>
cudaError_t launch_panel_update(T* Tp, int64_t ldT, const T* K, int64_t fs, const T* M,
                                int64_t ldm, int n, int p, int k, int r, cudaStream_t s);
bool panel_update_fits(int k, int r, size_t elem_bytes);
// M[((k - 1 - i) r + c) ldm + q] = sum_j Tp[j ldT + i p + q] V[c fs + j] for
// i < k, c < r <= 8, q < p, through panel_tv_blocks(n) partial sets in
// ``part`` (panel_tv_blocks(n) x k r p elements)
int panel_tv_blocks(int n);
template <typename T>
cudaError_t launch_panel_tv(const T* Tp, int64_t ldT, const T* V, int64_t fs, T* part, T* M,
                            int64_t ldm, int n, int p, int k, int r, cudaStream_t s);

// OLS pieces (lv_ols.cu).
template <typename T>
cudaError_t launch_gather_rows(const T* X, int64_t ldx, const int64_t* rows, int k, int n, T* dst,
                               int64_t ts, int64_t js, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter_rows(T* X, int64_t ldx, const int64_t* rows, int k, int n,
                                const T* src, int64_t ts, cudaStream_t s);
// Minv = (diag(+1 x kpos, -1 x (kk - kpos)) + S)^{-1}, kk <= 64: FP64
// programs in FP64 (S and Minv kk x kk doubles); FP32 programs in
// double-float on the FP32 pipe (S and Minv kk x kk float2 pairs).
cudaError_t launch_core_inverse(const double* S, int kk, int kpos, double* Minv, unsigned* status,
                                cudaStream_t s);
cudaError_t launch_core_inverse_df(const float2* S, int kk, int kpos, float2* Minv,
                                   unsigned* status, cudaStream_t s);
// Wu = -G Minv (FP64 core for double views, double-float core for float views)
cudaError_t launch_wu(const double* G, int64_t fs, int n, int kk, const double* Minv, double* Wu,
                      cudaStream_t s);
cudaError_t launch_wu(const float* G, int64_t fs, int n, int kk, const float2* Minv, float* Wu,
                      cudaStream_t s);
// Newton-Schulz correction of FP32 OLS programs: Z = X^T X as double-float
// pairs (Zh, Zl; n x n, row-major ldz, a multiple of 64 with zero padding)
cudaError_t launch_z_from_lower(const double* L, int64_t ldl, int n, float* Zh, float* Zl,
                                int64_t ldz, cudaStream_t s);
// Z += Hp Hp^T - Hm Hm^T (cnt history columns each, column stride fs >= ldz)
cudaError_t launch_z_flush(float* Zh, float* Zl, int64_t ldz, const float* Hp, const float* Hm,
                           int64_t fs, int n, int cnt, cudaStream_t s);
// R = D - Z B (B n x nb; D the identity if Dh is null, else the pairs Dh + Dl;
// double-float sums, rounded to FP32)
cudaError_t launch_ns_residual(const float* Zh, const float* Zl, int64_t ldz, const float* B,
                               int64_t ldb, int nb, const float* Dh, const float* Dl, int64_t ldd,
                               float* R, int64_t ldr, int n, cudaStream_t s);
// lo = src - (float)src, rounded to FP32 (src FP64 row-major)
cudaError_t launch_low_half(const double* src, int64_t lds, float* lo, int64_t ldl, int rows,
                            int cols, cudaStream_t s);
template <typename T>
cudaError_t launch_xty_update(T* xty, int64_t ld, T* xtyc, int64_t fs, const T* U, int n, int p,
                              int k, const T* Yr, cudaStream_t s,
                              T* xtyl = nullptr);
template <typename T>
cudaError_t launch_to_double(const T* src, int64_t lds, double* dst, int64_t ldd, int rows,
                             int cols, cudaStream_t s);
template <typename T>
cudaError_t launch_sym_lower_to_full(const double* Lcm, int64_t ldl, int n, T* dst, int64_t ldd,
                                     double* full, int64_t ldf, cudaStream_t s);
template <typename T>
cudaError_t launch_from_double(const double* src, int64_t lds, T* dst, int64_t ldd, int rows,
                               int cols, T* cm, int64_t cfs, cudaStream_t s);

}  // namespace lv
