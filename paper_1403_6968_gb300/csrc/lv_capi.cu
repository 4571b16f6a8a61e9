// C ABI and program engine of the GB300 LINVIEW library (arXiv 1403.6968).
//
// A program owns its views (materialised in HBM, row-major, leading
// dimension padded to a multiple of 256 elements and rows to a multiple of
// kBatch so that every TMA box of a view pass lies inside the allocation),
// the factor arenas of the exponential model (column-major n x R_cap: U
// grows left to right, V grows right to left so that V_{2h} = [Y_h, V_h]
// stays contiguous and pairs column by column with U_{2h} = [U_h, X'_h]),
// the partial-sum buffers of the view passes and a device status word.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/linview.h"
#include "lv_device.cuh"
#include "lv_internal.h"
#include "lv_ols.h"

using namespace lv;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static linview_status fail(linview_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

namespace lv {
// error setter for the other translation units of the ABI
linview_status lv_set_error(linview_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

// A pointer that kernels will read or write must be device (or managed)
// memory of ``device``: a host pointer handed over as device memory, or
// memory of another GPU, would be an invalid device access, so it is EINVAL
// here instead (a host-side query; null pointers are the caller's check).
linview_status check_dev_ptr(const void* ptr, int device, const char* name) {
  if (!ptr) return LINVIEW_OK;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return lv_set_error(LINVIEW_EINVAL, "%s is not device memory", name);
  }
  if (a.type == cudaMemoryTypeManaged) return LINVIEW_OK;
  if (a.type != cudaMemoryTypeDevice || a.device != device)
    return lv_set_error(LINVIEW_EINVAL, "%s is not device memory of device %d", name, device);
  return LINVIEW_OK;
}
}  // namespace lv

#define LV_CUDA(expr)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(LINVIEW_EDEVICE, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define LV_BLAS(expr)                                                                     \
  do {                                                                                    \
    cublasStatus_t e_ = (expr);                                                           \
    if (e_ != CUBLAS_STATUS_SUCCESS)                                                      \
      return fail(LINVIEW_EDEVICE, "%s failed: cublas status %d (%s:%d)", #expr, (int)e_, \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define LV_TRY(expr)                        \
  do {                                      \
    linview_status s_ = (expr);             \
    if (s_ != LINVIEW_OK) return s_;        \
  } while (0)

static int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// split-K partials of the CUDA-core GEMM, per program
constexpr size_t kGemmWorkBytes = size_t(4) << 20;

// ---------------------------------------------------------------------------
// program
// ---------------------------------------------------------------------------
struct View {
  void* ptr = nullptr;
  int64_t rows = 0, cols = 0, ld = 0;
  bool square = false;  // has a tensor map for view passes
  bool tma_store = false;  // tmap's row extent is a multiple of 16 bytes
  CUtensorMap tmap;
  CUtensorMap tmap_tc;  // FP32: 32 x 128 boxes, 128B swizzle (tensor-core update pass)
};

struct linview_program {
  linview_program_desc d = {};
  int elem = 4;
  int device = 0;
  int sms = 148;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;  // (pointer, bytes) of every device allocation
  int64_t bytes = 0;  // sum of the device allocations in allocs
  std::vector<View> views;
  int L = 0;    // log2 k for powers
  int npv = 0;  // power programs: number of power views (the sums views follow)
  // factor arenas
  void* Uar = nullptr;
  void* Var = nullptr;
  void* Wsum = nullptr;  // explicit V_h K_h^T for sums programs with wide factors
  // tensor-core update pass: split factors A_cat, B_cat (n x 64 each) and their maps
  float* tcA = nullptr;
  float* tcB = nullptr;
  CUtensorMap tmA, tmB;
  // a second set for the sums updates on the side stream (wide sums only)
  float* tpF = nullptr;  // split factor of the tensor-core products pass (128 x fs floats)
  int xslots = 0, yslots = 0;  // partial sets Xpart / Ypart hold
  int pc_x = 0, pc_y = 0;      // partial sets the last products pass wrote
  float* tcA2 = nullptr;
  float* tcB2 = nullptr;
  CUtensorMap tmA2, tmB2;
  int64_t fs = 0;
  int Rcap = 0;
  // partial sums of the view passes
  void* Xpart = nullptr;
  void* Ypart = nullptr;
  int64_t part_cs = 0, xp_s = 0, yp_q = 0;
  double* Cpart = nullptr;
  unsigned* ticket = nullptr;
  double* C = nullptr;
  unsigned* status = nullptr;
  // host -> device staging for host-side update factors
  void* stage = nullptr;
  size_t stage_bytes = 0;
  int64_t updates = 0;
  // iteration
  void* Tpanel = nullptr;
  int64_t ldT = 0;
  void* Bm = nullptr;
  int64_t ldB = 0;
  void* Kar = nullptr;  // Krylov blocks K_0..K_{k-1}, column-major n x k r_max
  void* V1 = nullptr;   // input right factor, column-major n x r_max
  void* Mr = nullptr;   // T_i^T V blocks in reverse order, p x k r_max
  void* TVpart = nullptr;  // row-block partial sums of those products
  int64_t tv_cap = 0;      // columns x p the partial sets hold (k r p <= tv_cap)
  void* Gpanel = nullptr;
  void* Dh = nullptr;   // hybrid strategy: dense deltas D_{i-1}, D_i (2 x n x p, ld ldD)
  int64_t ldD = 0;
  // exponential model of the iteration: factors of dT_h (ping-pong), the
  // suffix sums W^_h and the small product X_h^T V_h
  void* Xar[2] = {nullptr, nullptr};  // n x r_max k, column-major (fs)
  void* Yar[2] = {nullptr, nullptr};  // p x r_max k, column-major (ld p)
  void* What = nullptr;               // n x Rcap, column-major (fs)
  void* XtV = nullptr;                // (r_max k) x Rcap
  int ie_s = 0, ie_Ls = 0, ie_NT = 0;  // skip step s (k/2 for EXP), log2 s, number of T views
  void* Tfull = nullptr;  // T_0 .. T_k recomputed for the adjoint (exponential / skip)
  int64_t ldTf = 0;
  int64_t ldG = 0;
  // power adjoint work
  void* Gw0 = nullptr;
  void* Gw1 = nullptr;
  // own GEMMs: split-K partials of the CUDA-core GEMM (program-owned, so that
  // captured propagations can use it) and, for the hybrid strategy (FP32),
  // persistent split operands of the tensor-core GEMM
  void* gwork = nullptr;
  int64_t gwork_elems = 0;
  float* hyA = nullptr;  // split rows of the old A (n x tc_split_ld(n))
  float* hyB = nullptr;  // split rows of D_{i-1}^T (p x tc_split_ld(n))
  // OLS: X (m x n), Y (m x p) on the device; views W, beta, X^T Y, X
  void* Xd = nullptr;
  int64_t ldX = 0;
  void* Yd = nullptr;
  int64_t ldY = 0;
  void* XtYc = nullptr;   // column-major mirror of X^T Y (n x p, fs)
  void* Gf = nullptr;     // G = W U, column-major n x 2k
  void* Wuf = nullptr;    // -G M^{-1}, column-major n x 2k
  void* Hols = nullptr;   // Wu^T C', 2k x p (the factored beta refresh)
  void* Yr = nullptr;     // Y rows of the block, k x p
  int64_t* rows_d = nullptr;
  double* Minv = nullptr;
  void* Cdf = nullptr;  // OLS FP32: the Woodbury core as double-float pairs
  float* Zh = nullptr;  // OLS with Newton-Schulz correction: Z = X^T X as pairs (Zh + Zl)
  float* Zl = nullptr;
  int64_t ldz = 0;
  float* XtYl = nullptr;  // ... and the low halves of X^T Y (layout of the X^T Y view)
  float* Hp = nullptr;    // ... the replaced rows since Z was last brought up to date:
  float* Hm = nullptr;    //     new rows (Hp) and old rows (Hm), columns of stride fs
  int hcap = 0, hcnt = 0;
  // OLS re-evaluation scratch (FP64)
  double* Z64 = nullptr;
  double* X64 = nullptr;
  double* Y64 = nullptr;
  double* XtY64 = nullptr;
  double* W64 = nullptr;
  double* B64 = nullptr;
  double* solver_work = nullptr;
  int solver_lwork = 0;
  int* solver_info = nullptr;
  int64_t ols_chunk = 0;
  // CUDA graphs of the per-update propagation (powers/sums), one per rank,
  // replayed on a program-owned stream joined to the caller's stream
  bool use_graphs = true;
  cudaStream_t gstream = nullptr;
  // side stream of a propagation: the sums-view updates run there, forked
  // from the main stream after the factors they read and joined at the end
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork_ev = nullptr, side_join_ev = nullptr;
  bool side_pending = false;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  struct Rec {
    cudaEvent_t e0, e1;
    int kind;
    double bytes;
  };
  struct GraphEntry {
    int r;
    cudaGraphExec_t exec;
    int64_t launches;
    // instrumented copies (profiling): event-record nodes around each view
    // pass; recs hold the events of the copy's last replay
    bool instrumented = false;
    std::vector<Rec> recs;
    bool replayed = false;  // replayed since the last linview_reset_stats
  };
  std::vector<GraphEntry> graphs;
  std::vector<int> prof_rr;  // round-robin position over the instrumented copies, per rank
  // profiling
  bool prof = false;
  bool capturing_prof = false;       // capturing an instrumented graph copy
  std::vector<Rec>* capture_recs = nullptr;
  std::vector<cudaEvent_t> ev_pool;  // events of eager records (freed by reset)
  std::vector<cudaEvent_t> gev_pool; // events owned by instrumented graphs
  std::vector<Rec> ev_recs;
  int64_t all_launches = 0;
};

// Every device allocation of a program is rounded up to kAllocAlign bytes
// (the caching allocators' granule), so that the program's byte count equals
// what an allocator behind the callbacks hands out.
constexpr int64_t kAllocAlign = 512;
static int64_t alloc_bytes(int64_t b) { return rup(b > 0 ? b : 1, kAllocAlign); }

// A program's device memory: from the caller's allocator when the
// descriptor supplies one (e.g. PyTorch's caching allocator), else
// cudaMalloc.  Zero-filled in stream order on s.
static linview_status dalloc(linview_program* p, size_t bytes_in, void** out, cudaStream_t s) {
  const size_t bytes = (size_t)alloc_bytes((int64_t)bytes_in);
  void* ptr = nullptr;
  if (p->d.alloc) {
    ptr = p->d.alloc(bytes, static_cast<void*>(s), p->d.alloc_ctx);
    if (!ptr) return fail(LINVIEW_ENOMEM, "the caller's allocator returned NULL for %zu bytes", bytes);
    if (reinterpret_cast<uintptr_t>(ptr) % 256 != 0) {
      if (p->d.free) p->d.free(ptr, bytes, static_cast<void*>(s), p->d.alloc_ctx);
      return fail(LINVIEW_EINVAL, "the caller's allocator returned memory not 256-byte aligned");
    }
  } else {
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(LINVIEW_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  p->allocs.push_back({ptr, bytes});
  p->bytes += (int64_t)bytes;
  LV_CUDA(cudaMemsetAsync(ptr, 0, bytes, s));
  *out = ptr;
  return LINVIEW_OK;
}

// partial factor cores: one 64 x 64 block per gram CTA, or one r_h^2 <= 64
// block per row range of a fused pass (>= 2 CTAs per SM on any current part)
static size_t cpart_bytes(int64_t n) {
  const int sms_guess = 2 * 256;
  const size_t cp = (size_t)64 * 64 * gram_grid((int)n);
  const size_t cf = (size_t)64 * sms_guess;
  return sizeof(double) * (cp > cf ? cp : cf);
}

static int64_t square_view_bytes(int64_t n, int elem) {
  return rup(n, kBatch) * rup(n, 256) * elem;
}

static linview_status add_square_view(linview_program* p, int64_t n, cudaStream_t s) {
  View v;
  v.rows = n;
  v.cols = n;
  v.ld = rup(n, 256);
  const int64_t rows_pad = rup(n, kBatch);
  LV_TRY(dalloc(p, (size_t)square_view_bytes(n, p->elem), &v.ptr, s));
  v.square = true;
  v.tma_store = (v.ld * p->elem) % 16 == 0;
  if (!make_tmap(&v.tmap, v.ptr, p->elem, v.ld, rows_pad, v.ld))
    return fail(LINVIEW_EDEVICE, "cuTensorMapEncodeTiled failed for an %lld x %lld view",
                (long long)n, (long long)n);
  if (p->elem == 4 && !make_tmap_sw128(&v.tmap_tc, v.ptr, n, n, v.ld, 128))
    return fail(LINVIEW_EDEVICE, "cuTensorMapEncodeTiled (swizzled) failed for an %lld x %lld view",
                (long long)n, (long long)n);
  p->views.push_back(v);
  return LINVIEW_OK;
}

static linview_status add_rect_view(linview_program* p, void* ptr, int64_t rows, int64_t cols,
                                    int64_t ld) {
  View v;
  v.ptr = ptr;
  v.rows = rows;
  v.cols = cols;
  v.ld = ld;
  p->views.push_back(v);
  return LINVIEW_OK;
}

static linview_status copy_in(void* dst, int64_t ldd, const void* src, int64_t lds, int64_t rows,
                              int64_t cols, int elem, int on_device, cudaStream_t s) {
  if (rows == 0 || cols == 0) return LINVIEW_OK;
  LV_CUDA(cudaMemcpy2DAsync(dst, ldd * elem, src, lds * elem, cols * elem, rows,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return LINVIEW_OK;
}

static linview_status ensure_stage(linview_program* p, size_t bytes, cudaStream_t s) {
  if (p->stage_bytes >= bytes) return LINVIEW_OK;
  void* np = nullptr;
  LV_TRY(dalloc(p, bytes, &np, s));
  p->stage = np;
  p->stage_bytes = bytes;
  return LINVIEW_OK;
}

// ---------------------------------------------------------------------------
// profiling of view passes
// ---------------------------------------------------------------------------
// An event for a profiling record.  While an instrumented graph copy is
// captured the event belongs to the graph (an external event-record node
// that records on every replay); otherwise it is an eager record.
static cudaEvent_t prof_event(linview_program* p) {
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  (p->capturing_prof ? p->gev_pool : p->ev_pool).push_back(e);
  return e;
}

static void prof_record(linview_program* p, cudaEvent_t e, cudaStream_t s) {
  if (p->capturing_prof)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

struct ProfScope {
  linview_program* p;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  int kind = 0;
  double bytes = 0.0;
  // kind 1 = fused pass, 2 = update pass (timed when profiling); kind 0 =
  // other kernels (only counted)
  ProfScope(linview_program* p_, cudaStream_t s_, double bytes_, int kind_ = 0)
      : p(p_), s(s_), kind(kind_), bytes(bytes_) {
    p->all_launches++;
    if (!p->prof || kind == 0) return;
    e0 = prof_event(p);
    if (e0) prof_record(p, e0, s);
  }
  ~ProfScope() {
    if (!p->prof || !e0) return;
    cudaEvent_t e1 = prof_event(p);
    if (!e1) return;
    prof_record(p, e1, s);
    (p->capturing_prof ? *p->capture_recs : p->ev_recs).push_back({e0, e1, kind, bytes});
  }
};

// ---------------------------------------------------------------------------
// view passes
// ---------------------------------------------------------------------------

// X = P Xf, Y = P^T Yf (either may be skipped by mode), optional P += Uu Wu^T,
// for a factor block of width r <= kMaxFusedR; partials land at column offset 0
// of the given partial arrays.
template <typename T>
static linview_status run_fused(linview_program* p, const View& v, int mode, int r, const T* Xf,
                                const T* Yf, const T* Uu, const T* Wu, void* Xpart, void* Ypart,
                                cudaStream_t s, double* Cpart = nullptr,
                                bool reverse = false) {
  const PassGeom g = fused_geom(sizeof(T), (int)v.rows, p->sms);
  PassParams pp{};
  pp.P = v.ptr;
  pp.ldp = v.ld;
  pp.n = (int)v.rows;
  pp.Xf = Xf;
  pp.Yf = Yf;
  pp.Uu = Uu;
  pp.Wu = Wu;
  pp.fs = p->fs;
  pp.r = r;
  pp.Xpart = Xpart;
  pp.Ypart = Ypart;
  pp.part_cs = p->part_cs;
  pp.xp_s = p->xp_s;
  pp.yp_q = p->yp_q;
  pp.gC = g.gC;
  pp.gR = g.gR;
  pp.rows_per_cta = g.rows_per_cta;
  pp.status = p->status;
  pp.Cpart = Cpart;
  pp.tma_store = v.tma_store ? 1 : 0;
  pp.reverse = reverse ? 1 : 0;
  const double nn = (double)v.rows * (double)v.rows * sizeof(T);
  ProfScope ps(p, s, (mode & 4) ? 2.0 * nn : nn, 1);
  LV_CUDA((launch_fused<T>(pp, v.tmap, r, mode, s)));
  return LINVIEW_OK;
}

// A view pass that follows another one over the same view (same row ranges
// per CTA) runs in the opposite row order (reverse), so that it starts on the
// rows that are still in L2; blocks of one update alternate in the same way.
template <typename T>
static linview_status run_update(linview_program* p, const View& v, const T* Uu, const T* Wu,
                                 int r, cudaStream_t s, int suffix_rin = 0, int tcset = 0,
                                 bool reverse = false) {
  constexpr int MU = kMaxUpdateR;
  // split-factor scratch of the tensor-core pass (set 1: the side stream's)
  float* tA = tcset ? p->tcA2 : p->tcA;
  float* tB = tcset ? p->tcB2 : p->tcB;
  const CUtensorMap& mA = tcset ? p->tmA2 : p->tmA;
  const CUtensorMap& mB = tcset ? p->tmB2 : p->tmB;
  for (int c0 = 0; c0 < r;) {
    int w = (r - c0 < MU) ? (r - c0) : MU;
    if constexpr (sizeof(T) == 4) {
      // blocks wider than the CUDA-core pass sustains go to the tensor cores,
      // up to kMaxTcR columns per pass
      if (tA && r - c0 > kMaxProductR && suffix_rin == 0) {
        w = (r - c0 < kMaxTcR) ? (r - c0) : kMaxTcR;
        ProfScope ps(p, s, 2.0 * (double)v.rows * (double)v.rows * sizeof(T), 2);
        LV_CUDA(launch_tc_update(v.tmap_tc, mA, mB, static_cast<float*>(v.ptr), v.ld, tA, tB,
                                 reinterpret_cast<const float*>(Uu) + (int64_t)c0 * p->fs,
                                 reinterpret_cast<const float*>(Wu) + (int64_t)c0 * p->fs, p->fs,
                                 (int)v.rows, w, p->sms, p->status, s));
        p->all_launches++;  // the split kernel
        c0 += w;
        reverse = !reverse;
        continue;
      }
    }
    const PassGeom g = update_geom(sizeof(T), w, (int)v.rows, p->sms);
    PassParams pp{};
    pp.P = v.ptr;
    pp.ldp = v.ld;
    pp.n = (int)v.rows;
    pp.Uu = Uu + (int64_t)c0 * p->fs;
    pp.Wu = Wu + (int64_t)c0 * p->fs;
    pp.fs = p->fs;
    pp.r = w;
    pp.gC = g.gC;
    pp.gR = g.gR;
    pp.rows_per_cta = g.rows_per_cta;
    pp.status = p->status;
    pp.suffix_rin = suffix_rin;  // host guarantees a single chunk when set
    pp.tma_store = v.tma_store ? 1 : 0;
    pp.reverse = reverse ? 1 : 0;
    ProfScope ps(p, s, 2.0 * (double)v.rows * (double)v.rows * sizeof(T), 2);
    // a block after the first follows a pass that wrote this view
    LV_CUDA((launch_update<T>(pp, v.tmap, w, s, /*programmatic=*/c0 == 0)));
    c0 += w;
    reverse = !reverse;
  }
  return LINVIEW_OK;
}

// Products X = P Xf, Y = P^T Yf for any width r (chunks of kMaxProductR in
// FP32, kMaxFusedR in FP64) into
// the program's partial buffers (column block c0 at column offset c0), then
// (if Uu) the in-place update.  Fused in one pass when r <= kMaxFusedR.
// next_reverse (if given) receives the row order for a further pass over the
// view (the opposite of the last CUDA-core products pass).
template <typename T>
static linview_status run_products_update(linview_program* p, const View& v, int r, const T* Xf,
                                          const T* Yf, const T* Uu, const T* Wu, cudaStream_t s,
                                          double* Cpart = nullptr, bool allow_tc = false,
                                          bool* next_reverse = nullptr) {
  if (next_reverse) *next_reverse = false;
  const bool want_y = (Yf != nullptr);
  const PassGeom g = fused_geom(sizeof(T), (int)v.rows, p->sms);
  p->pc_x = g.gC;
  p->pc_y = g.gR;
  if (r <= kMaxFusedR) {
    const int mode = kModeX | (want_y ? 2 : 0) | (Uu ? 4 : 0);  // XYU, XY, XU or X
    if (next_reverse) *next_reverse = true;
    return run_fused<T>(p, v, mode, r, Xf, Yf, Uu, Wu, p->Xpart, p->Ypart, s,
                        mode == kModeXYU ? Cpart : nullptr);
  }
  if constexpr (sizeof(T) == 4) {
    // blocks wider than the CUDA-core products pass sustains: X = P U and
    // Y = P^T V on the tensor cores, one read of P each, K split in ``parts``
    const int n = (int)v.rows;
    const int parts = tp_parts(n, p->sms);  // partial sets the pass writes
    if (allow_tc && p->tpF && v.square && r > kMaxProductR && parts <= p->xslots &&
        (!want_y || parts <= p->yslots) && (v.ld * 4) % 16 == 0 && p->fs % 64 == 0) {
      const double nn = (double)n * (double)n * sizeof(float);
      for (int c0 = 0; c0 < r; c0 += kMaxTcR) {
        const int w = (r - c0 < kMaxTcR) ? (r - c0) : kMaxTcR;
        {
          ProfScope ps(p, s, nn, 1);
          LV_CUDA(launch_tc_products(false, static_cast<const float*>(v.ptr), v.ld,
                                     reinterpret_cast<const float*>(Xf) + (int64_t)c0 * p->fs,
                                     p->fs, p->tpF, n, w,
                                     static_cast<float*>(p->Xpart) + (int64_t)c0 * p->part_cs,
                                     p->xp_s, p->part_cs, parts, p->sms, p->status, s));
          p->all_launches++;  // the split kernel
        }
        if (want_y) {
          ProfScope ps(p, s, nn, 1);
          LV_CUDA(launch_tc_products(true, static_cast<const float*>(v.ptr), v.ld,
                                     reinterpret_cast<const float*>(Yf) + (int64_t)c0 * p->fs,
                                     p->fs, p->tpF, n, w,
                                     static_cast<float*>(p->Ypart) + (int64_t)c0 * p->part_cs,
                                     p->yp_q, p->part_cs, parts, p->sms, p->status, s));
          p->all_launches++;
        }
      }
      p->pc_x = p->pc_y = parts;
      if (Uu) LV_TRY(run_update<T>(p, v, Uu, Wu, r, s));
      return LINVIEW_OK;
    }
  }
  constexpr int MW = sizeof(T) == 4 ? kMaxProductR : kMaxFusedR;  // products-only width
  bool rev = false;  // consecutive passes over the view alternate their row order
  for (int c0 = 0; c0 < r; c0 += MW) {
    const int w = (r - c0 < MW) ? (r - c0) : MW;
    T* xp = static_cast<T*>(p->Xpart) + (int64_t)c0 * p->part_cs;
    T* yp = static_cast<T*>(p->Ypart) + (int64_t)c0 * p->part_cs;
    LV_TRY(run_fused<T>(p, v, want_y ? kModeXY : kModeX, w, Xf + (int64_t)c0 * p->fs,
                        want_y ? Yf + (int64_t)c0 * p->fs : nullptr, nullptr, nullptr, xp, yp, s,
                        nullptr, rev));
    rev = !rev;
  }
  if (next_reverse) *next_reverse = rev;
  if (Uu) LV_TRY(run_update<T>(p, v, Uu, Wu, r, s, 0, 0, rev));
  return LINVIEW_OK;
}

// ---------------------------------------------------------------------------
// GEMM helper: row-major C = alpha op(A) op(B) + beta C  (M x N, inner K)
// ---------------------------------------------------------------------------
static linview_status gemm_cm(linview_program* p, bool ta, bool tb, int64_t M, int64_t N,
                              int64_t K, double alpha, const void* A, int64_t lda, const void* B,
                              int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t s,
                              int mode) {
  LV_BLAS(cublasSetStream(p->blas, s));
  p->all_launches++;
  const cublasOperation_t oa = ta ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasOperation_t ob = tb ? CUBLAS_OP_T : CUBLAS_OP_N;
  if (p->elem == 8) {
    LV_BLAS(cublasDgemm(p->blas, oa, ob, (int)M, (int)N, (int)K, &alpha,
                        static_cast<const double*>(A), (int)lda, static_cast<const double*>(B),
                        (int)ldb, &beta, static_cast<double*>(C), (int)ldc));
    return LINVIEW_OK;
  }
  const float af = (float)alpha, bf = (float)beta;
  cublasComputeType_t ct = CUBLAS_COMPUTE_32F_PEDANTIC;
  if (mode == LINVIEW_REEVAL_TF32) ct = CUBLAS_COMPUTE_32F_FAST_TF32;
  if (mode == LINVIEW_REEVAL_BF16X9) ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  LV_BLAS(cublasGemmEx(p->blas, oa, ob, (int)M, (int)N, (int)K, &af, A, CUDA_R_32F, (int)lda, B,
                       CUDA_R_32F, (int)ldb, &bf, C, CUDA_R_32F, (int)ldc, ct,
                       CUBLAS_GEMM_DEFAULT));
  return LINVIEW_OK;
}

// Row-major C = alpha op(A) op(B) + beta C (M x N, inner K): the column-major
// view of a row-major buffer is its transpose, so swap the operands.
static linview_status gemm_rm(linview_program* p, bool ta, bool tb, int64_t M, int64_t N,
                              int64_t K, double alpha, const void* A, int64_t lda, const void* B,
                              int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t s,
                              int mode) {
  return gemm_cm(p, tb, ta, N, M, K, alpha, B, ldb, A, lda, beta, C, ldc, s, mode);
}

// accurate arithmetic for the internal small GEMMs of the incremental path
static int exact_mode(const linview_program* p) {
  return p->elem == 8 ? LINVIEW_REEVAL_FP64 : LINVIEW_REEVAL_FP32;
}

// the program's re-evaluation arithmetic: the library's own GEMM (split-TF32
// tensor cores for FP32, FP64 CUDA cores for FP64) unless a library
// comparison mode was selected
static int reeval_mode(const linview_program* p) {
  int m = p->d.reeval_mode;
  if (m == LINVIEW_REEVAL_DEFAULT) m = (p->elem == 8) ? LINVIEW_REEVAL_FP64 : LINVIEW_REEVAL_TC3;
  return m;
}

// ---------------------------------------------------------------------------
// own GEMMs (lv_gemm.cu): the dense contractions of re-evaluation, of the
// reverse pass and of the general form
// ---------------------------------------------------------------------------
// Rows of an operand: element (i, k) at X[i * rs + k * cs].
struct Opnd {
  const void* p;
  int64_t rs, cs;
};
static Opnd rows_of(const void* X, int64_t ld) { return {X, ld, 1}; }  // rows of row-major X
static Opnd cols_of(const void* X, int64_t ld) { return {X, 1, ld}; }  // rows of X^T

// The library's stream-ordered pool for the temporary memory of calls whose
// program has no allocator callbacks, one per device.  It keeps up to
// kPoolKeepBytes of freed memory mapped (the default pool returns everything
// at each synchronisation, so a call that needs a large temporary, e.g. the
// split operands of an n = 8192 product, would map it again every time).
constexpr uint64_t kPoolKeepBytes = uint64_t(4) << 30;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {nullptr};

static cudaError_t library_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

// Temporary device memory of one call, returned in stream order at the end
// of that call (through the caller's allocator when the program has one,
// else from the library's pool).
static linview_status talloc(linview_program* p, size_t bytes_in, void** out, cudaStream_t s) {
  const size_t bytes = (size_t)alloc_bytes((int64_t)bytes_in);
  void* ptr = nullptr;
  if (p->d.alloc) {
    ptr = p->d.alloc(bytes, static_cast<void*>(s), p->d.alloc_ctx);
    if (!ptr) return fail(LINVIEW_ENOMEM, "the caller's allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&ptr, bytes, pool, s);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(LINVIEW_ENOMEM, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
  }
  *out = ptr;
  return LINVIEW_OK;
}
static void tfree(linview_program* p, void* ptr, size_t bytes_in, cudaStream_t s) {
  if (!ptr) return;
  const size_t bytes = (size_t)alloc_bytes((int64_t)bytes_in);
  if (p->d.free)
    p->d.free(ptr, bytes, static_cast<void*>(s), p->d.alloc_ctx);
  else
    cudaFreeAsync(ptr, s);
}

// Split-operand scratch of the tensor-core GEMM: rows of A_s, then of B_s,
// then room for the K parts of a split product.
constexpr int64_t kTcWorkFloats = int64_t(4) << 20;  // 16 MB
struct TcScratch {
  float* a = nullptr;
  float* b = nullptr;
  float* work = nullptr;
  int64_t a_rows = 0, b_rows = 0, K = 0;
  void* block = nullptr;  // temporary block owned by this scratch (null: borrowed)
  size_t bytes = 0;
  linview_program* p = nullptr;
  cudaStream_t s = nullptr;
  ~TcScratch() {
    if (block) tfree(p, block, bytes, s);
  }
};

// Temporary split scratch for products with up to a_rows x K and b_rows x K
// operands (FP32 programs; FP64 programs take the CUDA-core path and get none).
static linview_status tc_scratch(linview_program* p, TcScratch* sc, int64_t a_rows, int64_t b_rows,
                                 int64_t K, cudaStream_t s) {
  if (p->elem != 4 || a_rows < 128) return LINVIEW_OK;  // such products run on the CUDA cores
  const int64_t ld = tc_split_ld(K);
  const size_t abytes = (size_t)alloc_bytes(a_rows * ld * 4);
  const size_t bbytes = (size_t)alloc_bytes(b_rows * ld * 4);
  const size_t bytes = abytes + bbytes + (size_t)kTcWorkFloats * 4;
  void* blk = nullptr;
  LV_TRY(talloc(p, bytes, &blk, s));
  sc->block = blk;
  sc->bytes = bytes;
  sc->p = p;
  sc->s = s;
  sc->a = static_cast<float*>(blk);
  sc->b = reinterpret_cast<float*>(static_cast<char*>(blk) + abytes);
  sc->work = reinterpret_cast<float*>(static_cast<char*>(blk) + abytes + bbytes);
  sc->a_rows = a_rows;
  sc->b_rows = b_rows;
  sc->K = K;
  return LINVIEW_OK;
}

// Products that go to the tensor cores (FP32, dense enough to fill tiles);
// the rest run on the CUDA cores.
static bool tc_eligible(const linview_program* p, const TcScratch* sc, int64_t M, int64_t N,
                        int64_t K) {
  return p->elem == 4 && sc && sc->a && M >= 128 && N >= 8 && K >= 128 && M <= sc->a_rows &&
         N <= sc->b_rows && K <= sc->K;
}

// D (M x N, row-major, ldd) = alpha sum_k a(m, k) b(n, k) + beta C (C row-major,
// ldc; may be D; beta == 0 ignores it), with a = rows of op(A) (M x K) and b =
// rows of op(B)^T (N x K).  FP32 with scratch: split TF32 on the tensor cores
// (a_ready / b_ready: the scratch already holds that operand's split rows);
// otherwise the CUDA-core GEMM in the program's arithmetic.
static linview_status gemm_ab(linview_program* p, int64_t M, int64_t N, int64_t K, double alpha,
                              Opnd a, Opnd b, double beta, const void* C, int64_t ldc, void* D,
                              int64_t ldd, cudaStream_t s, TcScratch* sc = nullptr,
                              bool a_ready = false, bool b_ready = false) {
  if (M <= 0 || N <= 0) return LINVIEW_OK;
  const int e = p->elem;
  if (tc_eligible(p, sc, M, N, K)) {
    const int64_t ld = tc_split_ld(K);
    if (!a_ready) {
      LV_CUDA(launch_split_rows(static_cast<const float*>(a.p), a.rs, a.cs, (int)M, (int)K, sc->a,
                                ld, s));
      p->all_launches++;
    }
    if (!b_ready) {
      LV_CUDA(launch_split_rows(static_cast<const float*>(b.p), b.rs, b.cs, (int)N, (int)K, sc->b,
                                ld, s));
      p->all_launches++;
    }
    LV_CUDA(launch_tc_gemm(sc->a, sc->b, (int)M, (int)N, (int)K, static_cast<float*>(D), ldd,
                           static_cast<const float*>(C), ldc, (float)alpha, (float)beta, p->sms,
                           p->status, s, sc->work, sc->work ? kTcWorkFloats : 0));
    p->all_launches++;
    return LINVIEW_OK;
  }
  if (beta != 0.0 && C != D)
    LV_CUDA(cudaMemcpy2DAsync(D, ldd * e, C, ldc * e, N * e, M, cudaMemcpyDeviceToDevice, s));
  // B(k, n) = b(n, k): k stride b.cs, n stride b.rs
  if (e == 4)
    LV_CUDA(launch_gemm_simt<float>((int)M, (int)N, (int)K, (float)alpha,
                                    static_cast<const float*>(a.p), a.rs, a.cs,
                                    static_cast<const float*>(b.p), b.cs, b.rs, (float)beta,
                                    static_cast<float*>(D), ldd, 1, static_cast<float*>(p->gwork),
                                    p->gwork_elems, p->sms, s));
  else
    LV_CUDA(launch_gemm_simt<double>((int)M, (int)N, (int)K, alpha, static_cast<const double*>(a.p),
                                     a.rs, a.cs, static_cast<const double*>(b.p), b.cs, b.rs, beta,
                                     static_cast<double*>(D), ldd, 1,
                                     static_cast<double*>(p->gwork), p->gwork_elems, p->sms, s));
  p->all_launches += 2;
  return LINVIEW_OK;
}

// Column-major products of the factor arenas, C (M x N, column stride ldc) =
// alpha op(A) op(B) + beta C with A, B column-major (lda, ldb): the CUDA-core
// GEMM with the program's split-K partials (small products of the general
// form, captured into the propagation graphs).
// (batch > 1: ``batch`` such products, entry b at A + b a_bs, B + b b_bs,
// C + b c_bs elements, strides possibly negative, in one launch)
static linview_status gemm_cm_own(linview_program* p, bool ta, bool tb, int64_t M, int64_t N,
                                  int64_t K, double alpha, const void* A, int64_t lda,
                                  const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                                  cudaStream_t s, int batch = 1, int64_t a_bs = 0,
                                  int64_t b_bs = 0, int64_t c_bs = 0) {
  if (M <= 0 || N <= 0) return LINVIEW_OK;
  // column-major X(i, j) = X[i + j ld]; op(A)(m, k), op(B)(k, n)
  const int64_t a_rs = ta ? lda : 1, a_cs = ta ? 1 : lda;
  const int64_t b_rs = tb ? ldb : 1, b_cs = tb ? 1 : ldb;
  if (p->elem == 4)
    LV_CUDA(launch_gemm_simt<float>((int)M, (int)N, (int)K, (float)alpha,
                                    static_cast<const float*>(A), a_rs, a_cs,
                                    static_cast<const float*>(B), b_rs, b_cs, (float)beta,
                                    static_cast<float*>(C), 1, ldc, static_cast<float*>(p->gwork),
                                    p->gwork_elems, p->sms, s, batch, a_bs, b_bs, c_bs));
  else
    LV_CUDA(launch_gemm_simt<double>((int)M, (int)N, (int)K, alpha, static_cast<const double*>(A),
                                     a_rs, a_cs, static_cast<const double*>(B), b_rs, b_cs, beta,
                                     static_cast<double*>(C), 1, ldc,
                                     static_cast<double*>(p->gwork), p->gwork_elems, p->sms, s,
                                     batch, a_bs, b_bs, c_bs));
  p->all_launches += 2;
  return LINVIEW_OK;
}

// Narrow products of a square view with a row-major panel, out (n x nc,
// row-major) = op(view) X (+ add; add may be out) with op = identity or transpose, nc <=
// kMaxFusedR: one products pass over the view (memory-bound, the view's own
// arithmetic) instead of a GEMM whose tiles a few columns cannot fill.  X is
// staged column-major in the GEMM work buffer, the pass's partial sums are
// reduced there, and the result is transposed back into ``out``.  Returns
// false (nothing enqueued) when the shapes do not fit this path.
template <typename T>
static bool view_panel_fits(const linview_program* p, const View& v, int nc) {
  const int64_t fs = rup(v.rows, 64);
  return v.square && nc >= 1 && nc <= kMaxFusedR && p->xp_s >= (int64_t)nc * p->part_cs &&
         p->yp_q >= (int64_t)nc * p->part_cs && p->part_cs >= v.rows && p->gwork &&
         3 * fs * nc <= p->gwork_elems;
}

template <typename T>
static linview_status view_panel_product(linview_program* p, const View& v, bool transpose,
                                         const T* X, int64_t ldx, int nc, const T* add,
                                         int64_t ldadd, T* out, int64_t ldo, cudaStream_t s) {
  const int n = (int)v.rows;
  const int64_t fs = rup(n, 64);
  T* xcm = static_cast<T*>(p->gwork);
  T* ocm = xcm + fs * nc;
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  const int64_t fs_prog = p->fs;
  p->fs = fs;  // the staged factor's column stride
  LV_CUDA(launch_rm_to_cm<T>(X, ldx, xcm, fs, n, nc, s));
  const linview_status st =
      run_fused<T>(p, v, transpose ? kModeXY : kModeX, nc, xcm, transpose ? xcm : nullptr,
                   nullptr, nullptr, p->Xpart, p->Ypart, s);
  p->fs = fs_prog;
  LV_TRY(st);
  if (transpose)
    LV_CUDA(launch_sum_partials<T>(static_cast<const T*>(p->Ypart), g.gR, p->yp_q, p->part_cs, n,
                                   nc, ocm, fs, s));
  else
    LV_CUDA(launch_sum_partials<T>(static_cast<const T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n,
                                   nc, ocm, fs, s));
  // column-major n x nc -> row-major: the transpose of an nc x n row-major block
  if (add && add == out) {  // out += op(view) X: transpose into the scratch, then add
    T* rm = ocm + fs * nc;  // row-major n x nc, ld nc
    LV_CUDA(launch_rm_to_cm<T>(ocm, fs, rm, nc, nc, n, s));
    LV_CUDA(launch_axpy_rows<T>(out, ldo, rm, nc, T(1), n, nc, s));
  } else {
    LV_CUDA(launch_rm_to_cm<T>(ocm, fs, out, ldo, nc, n, s));
    if (add) LV_CUDA(launch_axpy_rows<T>(out, ldo, add, ldadd, T(1), n, nc, s));
  }
  p->all_launches += add ? 4 : 3;
  return LINVIEW_OK;
}

// Comparison modes of the re-evaluation: library GEMMs, selected explicitly.
static bool library_mode(int mode) {
  return mode == LINVIEW_REEVAL_FP32 || mode == LINVIEW_REEVAL_TF32 ||
         mode == LINVIEW_REEVAL_BF16X9;
}

// ---------------------------------------------------------------------------
// powers and sums of powers
// ---------------------------------------------------------------------------
static bool is_pow2(int k) { return k >= 1 && (k & (k - 1)) == 0; }
static int ilog2(int k) {
  int l = 0;
  while ((1 << l) < k) ++l;
  return l;
}
static bool is_linear(const linview_program* p) { return p->d.model == LINVIEW_MODEL_LINEAR; }

// Shape rules of the linear and skip-s models (the exponential model's are
// checked where it is built).
static linview_status check_power_model(const linview_program_desc& d) {
  if (d.model == LINVIEW_MODEL_LINEAR || d.model == LINVIEW_MODEL_SKIP) {
    if (d.k < 2) return fail(LINVIEW_EINVAL, "k=%d must be >= 2", d.k);
    if (d.r_max < 1 || (int64_t)d.r_max * d.k > 64)
      return fail(LINVIEW_EUNSUPPORTED, "linear and skip models: r_max*k=%lld must be <= 64",
                  (long long)d.r_max * d.k);
  }
  if (d.model == LINVIEW_MODEL_SKIP) {
    if (!is_pow2(d.skip) || d.k % d.skip != 0 || d.k < 2 * d.skip)
      return fail(LINVIEW_EINVAL, "skip s=%d: s must be a power of two and k=%d a multiple >= 2s",
                  d.skip, d.k);
  } else if (d.skip != 0) {
    return fail(LINVIEW_EINVAL, "skip must be 0 unless model is LINVIEW_MODEL_SKIP");
  }
  return LINVIEW_OK;
}
static bool has_sums(const linview_program* p) {
  if (p->d.model != LINVIEW_MODEL_EXP) return p->d.kind == LINVIEW_POWER_SUM;
  return p->d.kind == LINVIEW_POWER_SUM && p->L >= 1;
}
static View& pview(linview_program* p, int l) { return p->views[l]; }
// S'_h for the power view of index l >= 1 (h = 2^l, or the skip view l)
static View& sview(linview_program* p, int l) { return p->views[p->npv + l - 1]; }

// Linear model (Section 3.3): P_i = P_{i-1} A, i = 2..k (views i-1), and
// S'_k = P_1 + ... + P_k (view k) for sums programs.
static linview_status linear_reeval(linview_program* p, cudaStream_t s) {
  const int64_t n = p->d.n;
  const int k = p->d.k;
  const int mode = reeval_mode(p);
  View& a = p->views[0];
  TcScratch sc;
  if (!library_mode(mode)) LV_TRY(tc_scratch(p, &sc, n, n, n, s));
  for (int i = 2; i <= k; ++i) {
    View& prev = p->views[i - 2];
    View& c = p->views[i - 1];
    if (library_mode(mode))
      LV_TRY(gemm_rm(p, false, false, n, n, n, 1.0, prev.ptr, prev.ld, a.ptr, a.ld, 0.0, c.ptr,
                     c.ld, s, mode));
    else  // A^T's rows are split once
      LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(prev.ptr, prev.ld), cols_of(a.ptr, a.ld), 0.0,
                     nullptr, 0, c.ptr, c.ld, s, &sc, false, i > 2));
  }
  if (has_sums(p)) {
    View& sv = p->views[k];
    LV_CUDA(cudaMemcpy2DAsync(sv.ptr, sv.ld * p->elem, a.ptr, a.ld * p->elem, n * p->elem, n,
                              cudaMemcpyDeviceToDevice, s));
    for (int i = 2; i <= k; ++i) {
      View& pi = p->views[i - 1];
      if (p->elem == 4)
        LV_CUDA(launch_axpy_rows<float>(static_cast<float*>(sv.ptr), sv.ld,
                                        static_cast<const float*>(pi.ptr), pi.ld, 1.0f, (int)n,
                                        (int)n, s));
      else
        LV_CUDA(launch_axpy_rows<double>(static_cast<double*>(sv.ptr), sv.ld,
                                         static_cast<const double*>(pi.ptr), pi.ld, 1.0, (int)n,
                                         (int)n, s));
      p->all_launches++;
    }
  }
  return LINVIEW_OK;
}

// Skip-s model: squarings up to P_s (views 0..log2 s), then P_{is} =
// P_s P_{(i-1)s} (views log2(s) + i - 1, i = 2..k/s).
static linview_status skip_reeval(linview_program* p, cudaStream_t s) {
  const int64_t n = p->d.n;
  const int mode = reeval_mode(p);
  const bool lib = library_mode(mode);
  const int Ls = ilog2(p->d.skip);
  TcScratch sc;
  if (!lib) LV_TRY(tc_scratch(p, &sc, n, n, n, s));
  // out = pm prev (+ add)
  auto prod = [&](View& pm, View& prev, View* add, View& out, bool a_ready) -> linview_status {
    if (lib) {
      if (add)
        LV_CUDA(cudaMemcpy2DAsync(out.ptr, out.ld * p->elem, add->ptr, add->ld * p->elem,
                                  n * p->elem, n, cudaMemcpyDeviceToDevice, s));
      return gemm_rm(p, false, false, n, n, n, 1.0, pm.ptr, pm.ld, prev.ptr, prev.ld,
                     add ? 1.0 : 0.0, out.ptr, out.ld, s, mode);
    }
    return gemm_ab(p, n, n, n, 1.0, rows_of(pm.ptr, pm.ld), cols_of(prev.ptr, prev.ld),
                   add ? 1.0 : 0.0, add ? add->ptr : nullptr, add ? add->ld : 0, out.ptr, out.ld,
                   s, &sc, a_ready, false);
  };
  for (int l = 0; l < Ls; ++l) LV_TRY(prod(pview(p, l), pview(p, l), nullptr, pview(p, l + 1), false));
  View& ps = pview(p, Ls);
  for (int i = 2; i <= p->d.k / p->d.skip; ++i)  // P_s's rows are split once
    LV_TRY(prod(ps, pview(p, Ls + i - 2), nullptr, pview(p, Ls + i - 1), i > 2));
  if (has_sums(p)) {
    // S'_{2h} = P_h S'_h + S'_h up to s (S'_1 = A), then S'_i = P_s S'_{i-s} + S'_s
    for (int l = 0; l < Ls; ++l) {
      View& sh = (l == 0) ? pview(p, 0) : sview(p, l);
      LV_TRY(prod(pview(p, l), sh, &sh, sview(p, l + 1), false));
    }
    View& ss = (Ls == 0) ? pview(p, 0) : sview(p, Ls);
    for (int i = 2; i <= p->d.k / p->d.skip; ++i) {
      View& prev = (Ls + i - 2 == 0) ? pview(p, 0) : sview(p, Ls + i - 2);
      LV_TRY(prod(ps, prev, &ss, sview(p, Ls + i - 1), false));
    }
  }
  return LINVIEW_OK;
}

static linview_status powers_reeval(linview_program* p, cudaStream_t s) {
  if (is_linear(p)) return linear_reeval(p, s);
  if (p->d.model == LINVIEW_MODEL_SKIP) return skip_reeval(p, s);
  const int64_t n = p->d.n;
  const int mode = reeval_mode(p);
  if (library_mode(mode)) {  // comparison: library GEMMs
    for (int l = 0; l < p->L; ++l) {
      View& a = pview(p, l);
      View& c = pview(p, l + 1);
      LV_TRY(gemm_rm(p, false, false, n, n, n, 1.0, a.ptr, a.ld, a.ptr, a.ld, 0.0, c.ptr, c.ld, s,
                     mode));
    }
    if (has_sums(p)) {
      for (int l = 0; l < p->L; ++l) {
        View& ph = pview(p, l);
        View& sh = (l == 0) ? pview(p, 0) : sview(p, l);
        View& s2 = sview(p, l + 1);
        LV_CUDA(cudaMemcpy2DAsync(s2.ptr, s2.ld * p->elem, sh.ptr, sh.ld * p->elem, n * p->elem,
                                  n, cudaMemcpyDeviceToDevice, s));
        LV_TRY(gemm_rm(p, false, false, n, n, n, 1.0, ph.ptr, ph.ld, sh.ptr, sh.ld, 1.0, s2.ptr,
                       s2.ld, s, mode));
      }
    }
    return LINVIEW_OK;
  }
  // own GEMM, level by level: P_2h = P_h P_h, then S'_2h = P_h S'_h + S'_h with
  // P_h's split rows reused (Table 1, exponential model)
  TcScratch sc;
  LV_TRY(tc_scratch(p, &sc, n, n, n, s));
  const bool sums = has_sums(p);
  for (int l = 0; l < p->L; ++l) {
    View& ph = pview(p, l);
    View& c = pview(p, l + 1);
    LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(ph.ptr, ph.ld), cols_of(ph.ptr, ph.ld), 0.0, nullptr,
                   0, c.ptr, c.ld, s, &sc));
    if (sums) {
      View& sh = (l == 0) ? pview(p, 0) : sview(p, l);
      View& s2 = sview(p, l + 1);
      LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(ph.ptr, ph.ld), cols_of(sh.ptr, sh.ld), 1.0, sh.ptr,
                     sh.ld, s2.ptr, s2.ld, s, &sc, /*a_ready=*/true));
    }
  }
  return LINVIEW_OK;
}

// sums programs apply their block-triangular core inside one update pass
// when the whole factor fits one pass; wider factors get an explicit
// suffix-sum factor (see sums_update)
static bool powers_wide_sums(const linview_program_desc& d) {
  const int64_t mu = kMaxUpdateR;
  return d.kind == LINVIEW_POWER_SUM && ((int64_t)d.r_max * d.k > mu || d.r_max > 8);
}

// Views of a power program: exponential model P_{2^j} (j = 0..log2 k) and,
// with sums, S'_{2^j} (j >= 1); linear model P_1..P_k and, with sums, S'_k;
// skip-s model P_{2^j} (j = 0..log2 s) then P_{2s}, ..., P_k and, with sums,
// S'_h for the same h > 1.
static int powers_num_views(const linview_program_desc& d) {
  const bool sums = d.kind == LINVIEW_POWER_SUM;
  if (d.model == LINVIEW_MODEL_LINEAR) return d.k + (sums ? 1 : 0);
  if (d.model == LINVIEW_MODEL_SKIP) {
    const int np = ilog2(d.skip) + d.k / d.skip;
    return np + (sums ? np - 1 : 0);
  }
  const int L = ilog2(d.k);
  return L + 1 + (sums ? L : 0);
}

// FP32 power programs whose update blocks can be wider than kMaxProductR
// refresh those blocks on the tensor cores.
static bool powers_uses_tc(const linview_program_desc& d) {
  return d.precision == LINVIEW_F32 && (int64_t)d.r_max * d.k > kMaxProductR;
}
// exponential-model products of width r_h = r h, h <= k / 2, wider than the
// CUDA-core products pass: the tensor-core products pass
static bool powers_uses_tp(const linview_program_desc& d) {
  return d.precision == LINVIEW_F32 && d.model == LINVIEW_MODEL_EXP &&
         (int64_t)d.r_max * (d.k / 2) > kMaxProductR;
}

// Device bytes powers_create allocates (with the buffers every program has),
// in the same order; linview_estimate_device_bytes reports it.
static int64_t powers_device_bytes(const linview_program_desc& d, int sms) {
  const int elem = d.precision == LINVIEW_F64 ? 8 : 4;
  const int64_t n = d.n;
  int64_t b = alloc_bytes((int64_t)sizeof(unsigned) * 4) +
              alloc_bytes((int64_t)sizeof(double) * 64 * 64) + alloc_bytes((int64_t)cpart_bytes(n)) +
              alloc_bytes((int64_t)kGemmWorkBytes);
  b += powers_num_views(d) * alloc_bytes(square_view_bytes(n, elem));
  const int64_t Rcap = (int64_t)d.r_max * d.k;
  const int64_t fs = rup(n, 64);
  b += (powers_wide_sums(d) ? 3 : 2) * alloc_bytes(fs * Rcap * elem);
  const PassGeom g = fused_geom(elem, (int)n, sms);
  const int64_t half = Rcap / 2 > 0 ? Rcap / 2 : 1;
  const bool tp = powers_uses_tp(d);
  const int64_t xs = tp && g.gC < kTpMaxParts ? kTpMaxParts : g.gC;
  const int64_t ys = tp && g.gR < kTpMaxParts ? kTpMaxParts : g.gR;
  b += alloc_bytes(xs * half * fs * elem) + alloc_bytes(ys * half * fs * elem);
  b += alloc_bytes(2 * n * d.r_max * elem);
  if (powers_uses_tc(d)) b += alloc_bytes(tc_split_floats(n) * 4) * (powers_wide_sums(d) ? 2 : 1);
  if (tp) b += alloc_bytes(128 * fs * 4);
  return b;
}

static linview_status powers_create(linview_program* p, const void* const* inputs,
                                    const int64_t* lds, int on_dev, cudaStream_t s) {
  const int64_t n = p->d.n;
  const int k = p->d.k;
  LV_TRY(check_power_model(p->d));
  if (p->d.model != LINVIEW_MODEL_EXP) {
    // the Krylov-type levels use square factor cores of width < r_max * k
  } else {
    if (!is_pow2(k)) return fail(LINVIEW_EINVAL, "k=%d must be a power of two", k);
    if ((int64_t)p->d.r_max * k > 128)
      return fail(LINVIEW_EUNSUPPORTED,
                  "r_max*k=%lld exceeds 128 (factor cores are at most 64x64)",
                  (long long)p->d.r_max * k);
  }
  p->L = ilog2(k);
  const bool wide_sums = powers_wide_sums(p->d);
  if (lds[0] < n) return fail(LINVIEW_ESHAPE, "ld of A (%lld) < n", (long long)lds[0]);
  const int nviews = powers_num_views(p->d);
  for (int l = 0; l < nviews; ++l) LV_TRY(add_square_view(p, n, s));
  p->npv = p->d.model == LINVIEW_MODEL_EXP      ? p->L + 1
           : p->d.model == LINVIEW_MODEL_SKIP ? ilog2(p->d.skip) + k / p->d.skip
                                              : k;
  LV_TRY(copy_in(pview(p, 0).ptr, pview(p, 0).ld, inputs[0], lds[0], n, n, p->elem, on_dev, s));
  p->Rcap = p->d.r_max * k;
  p->fs = rup(n, 64);
  const size_t fbytes = (size_t)p->fs * p->Rcap * p->elem;
  LV_TRY(dalloc(p, fbytes, &p->Uar, s));
  LV_TRY(dalloc(p, fbytes, &p->Var, s));
  if (wide_sums) LV_TRY(dalloc(p, fbytes, &p->Wsum, s));
  const PassGeom g = fused_geom(p->elem, (int)n, p->sms);
  const int half = (p->Rcap / 2 > 0) ? p->Rcap / 2 : 1;
  p->part_cs = p->fs;
  p->xp_s = (int64_t)half * p->part_cs;
  p->yp_q = (int64_t)half * p->part_cs;
  // levels wider than the CUDA-core products pass go to the tensor cores,
  // whose K parts need their own partial sets
  const bool tp = powers_uses_tp(p->d);
  p->xslots = tp && g.gC < kTpMaxParts ? kTpMaxParts : g.gC;
  p->yslots = tp && g.gR < kTpMaxParts ? kTpMaxParts : g.gR;
  LV_TRY(dalloc(p, (size_t)p->xslots * p->xp_s * p->elem, &p->Xpart, s));
  LV_TRY(dalloc(p, (size_t)p->yslots * p->yp_q * p->elem, &p->Ypart, s));
  if (tp) {
    void* t = nullptr;
    LV_TRY(dalloc(p, sizeof(float) * 128 * p->fs, &t, s));
    p->tpF = static_cast<float*>(t);
  }
  // host-side update factors are staged here (allocated now so that an
  // update never allocates)
  LV_TRY(ensure_stage(p, (size_t)2 * n * p->d.r_max * p->elem, s));
  if (powers_uses_tc(p->d)) {
    void* tc = nullptr;
    LV_TRY(dalloc(p, (size_t)tc_split_floats(n) * sizeof(float), &tc, s));
    p->tcA = static_cast<float*>(tc);
    p->tcB = p->tcA + tc_split_floats(n) / 2;
    if (!make_tmap_sw128(&p->tmA, p->tcA, 128, n, 128, 128) ||
        !make_tmap_sw128(&p->tmB, p->tcB, 128, n, 128, 32))
      return fail(LINVIEW_EDEVICE, "cuTensorMapEncodeTiled failed for the split factors");
    if (wide_sums) {  // the sums updates on the side stream have their own
      void* tc2 = nullptr;
      LV_TRY(dalloc(p, (size_t)tc_split_floats(n) * sizeof(float), &tc2, s));
      p->tcA2 = static_cast<float*>(tc2);
      p->tcB2 = p->tcA2 + tc_split_floats(n) / 2;
      if (!make_tmap_sw128(&p->tmA2, p->tcA2, 128, n, 128, 128) ||
          !make_tmap_sw128(&p->tmB2, p->tcB2, 128, n, 128, 32))
        return fail(LINVIEW_EDEVICE, "cuTensorMapEncodeTiled failed for the split factors");
    }
  }
  return powers_reeval(p, s);
}

// S'_h += U_h (V_h K_h^T)^T, K_h block upper triangular of identities: the
// update pass takes the suffix block sums of V_h itself when the factor fits
// one pass, else they are formed first (one thread per row).
template <typename T>
static linview_status sums_update_on(linview_program* p, View& sv, const T* U, const T* Vh, int rh,
                                     int r, cudaStream_t s, int tcset) {
  if (!p->Wsum) return run_update<T>(p, sv, U, Vh, rh, s, r);
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_suffix_sums<T>(Vh, static_cast<T*>(p->Wsum), p->fs, (int)p->d.n, rh, r, s));
  }
  return run_update<T>(p, sv, U, static_cast<const T*>(p->Wsum), rh, s, 0, tcset);
}

// A sums view is written by nothing else during a propagation and its update
// reads only factor columns that are final once enqueued, so it runs on the
// program's side stream, forked from s here (everything enqueued on s so far
// happens before it) and joined by side_join at the end of the propagation.
// The view passes of the two streams then fill each other's ramps and tails,
// and an HBM-bound sums pass can use the bandwidth a compute-bound level pass
// leaves idle.  (Inside a graph capture the fork and join become edges.)
static linview_status side_fork(linview_program* p, cudaStream_t s, cudaStream_t* out) {
  if (!p->side) {
    LV_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    LV_CUDA(cudaEventCreateWithFlags(&p->side_fork_ev, cudaEventDisableTiming));
    LV_CUDA(cudaEventCreateWithFlags(&p->side_join_ev, cudaEventDisableTiming));
  }
  LV_CUDA(cudaEventRecord(p->side_fork_ev, s));
  LV_CUDA(cudaStreamWaitEvent(p->side, p->side_fork_ev, 0));
  p->side_pending = true;
  *out = p->side;
  return LINVIEW_OK;
}

static linview_status side_join(linview_program* p, cudaStream_t s) {
  if (!p->side_pending) return LINVIEW_OK;
  p->side_pending = false;
  LV_CUDA(cudaEventRecord(p->side_join_ev, p->side));
  LV_CUDA(cudaStreamWaitEvent(s, p->side_join_ev, 0));
  return LINVIEW_OK;
}

template <typename T>
static linview_status sums_update(linview_program* p, View& sv, const T* U, const T* Vh, int rh,
                                  int r, cudaStream_t s) {
  // profiling times each view pass alone: no overlap
  if (p->prof) return sums_update_on<T>(p, sv, U, Vh, rh, r, s, 0);
  cudaStream_t side = nullptr;
  LV_TRY(side_fork(p, s, &side));
  return sums_update_on<T>(p, sv, U, Vh, rh, r, side, 1);
}

// Exponential-model levels l = 0 .. nlev-1 (h = 2^l, Appendix A): the level
// pass on P_h (P_h U_h, P_h^T V_h from the old view, P_h += U_h V_h^T; for
// r_h <= kMaxFusedR the same pass yields the partials of C_h = V_h^T U_h),
// the sums view S'_h (h >= 2) when ``sums``, and the assembly of
// U_{2h} = [U_h, P_h U_h + U_h C_h], V_{2h} = [P_h^T V_h, V_h].
template <typename T>
static linview_status exp_levels(linview_program* p, int r, int nlev, bool sums, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t fs = p->fs;
  T* U = static_cast<T*>(p->Uar);
  T* V = static_cast<T*>(p->Var);
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  for (int l = 0; l < nlev; ++l) {
    const int rh = r << l;
    T* Vh = V + (int64_t)(p->Rcap - rh) * fs;
    const bool fused = rh <= kMaxFusedR;
    if (!fused) {
      ProfScope ps(p, s, 0.0);
      LV_CUDA((launch_gram<T>(Vh, U, fs, n, rh, p->Cpart, p->ticket, p->C, p->status, s)));
    }
    // sums: S'_h += U_h (V_h K_h^T)^T, the suffix block sums taken in the pass
    // (side stream, concurrent with the level pass)
    if (sums && l >= 1) LV_TRY(sums_update<T>(p, sview(p, l), U, Vh, rh, r, s));
    LV_TRY(run_products_update<T>(p, pview(p, l), rh, U, Vh, U, Vh, s,
                                  fused ? p->Cpart : nullptr, /*allow_tc=*/true));
    AssembleParams a{};
    a.status = p->status;
    a.n = n;
    a.r_h = rh;
    a.fs = fs;
    a.Xpart = p->Xpart;
    a.gC = p->pc_x;
    a.xp_s = p->xp_s;
    a.Ypart = p->Ypart;
    a.gR = p->pc_y;
    a.yp_q = p->yp_q;
    a.part_cs = p->part_cs;
    a.C = fused ? p->Cpart : p->C;
    a.nC = fused ? g.gR : 1;
    a.Uh = U;
    a.Unew = U + (int64_t)rh * fs;
    a.Ynew = V + (int64_t)(p->Rcap - 2 * rh) * fs;
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_assemble<T>(a, s));
  }
  return LINVIEW_OK;
}

// Linear-type levels on a base block of width bw (Appendix A).  Linear model:
// base (U_1, V_1), Q_j = P_j;  skip-s model: base (U_s, V_s) from the
// exponential levels, Q_j = P_{js}.  With Q' the refreshed views,
//   U_{j+1} = [U_base, Q_1' U_j]   = [U_base, Q_1' U_base, ..., Q_j' U_base],
//   V_{j+1} = [Q_j^T V_base, V_j]  (old Q),  Q_j += U_j V_j^T,
// since Q_1'^j = Q_j'.  Only the newest blocks are new at each step (Krylov
// reuse): the pass over the old Q_j yields Y = Q_j^T V_base and X = Q_j U_base,
// and Q_j' U_base = X + U_j (V_j^T U_base); the view is refreshed after its
// products.  U grows from the left of the arena, V from the right, block i of
// U_j pairing with block i of V_j.  Views: Q_j = views[view0 + j - 1]; the
// last one, views[view0 + nsteps], gets only its refresh.
template <typename T>
static linview_status krylov_levels(linview_program* p, int bw, int nsteps, int view0,
                                    int sums_r, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t fs = p->fs;
  T* U = static_cast<T*>(p->Uar);
  T* V = static_cast<T*>(p->Var);
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  const T* Vb = V + (int64_t)(p->Rcap - bw) * fs;
  for (int j = 1; j <= nsteps; ++j) {
    const int rh = j * bw;
    T* Vj = V + (int64_t)(p->Rcap - rh) * fs;
    View& Q = p->views[view0 + j - 1];
    {  // C = V_j^T U_j (its first bw columns are V_j^T U_base)
      ProfScope ps(p, s, 0.0);
      LV_CUDA((launch_gram<T>(Vj, U, fs, n, rh, p->Cpart, p->ticket, p->C, p->status, s)));
    }
    bool rev = false;
    LV_TRY(run_products_update<T>(p, Q, bw, U, Vb, nullptr, nullptr, s, nullptr, false, &rev));
    LV_TRY(run_update<T>(p, Q, U, Vj, rh, s, 0, 0, rev));
    // skip model with sums: U_j, V_j are Krylov bases of width j bw, so
    // dS'_h = U_j (V_j K^T)^T as in the exponential model
    // (S'_1 is A itself: no sums view for power index 0)
    if (sums_r > 0 && view0 + j - 1 >= 1)
      LV_TRY(sums_update<T>(p, sview(p, view0 + j - 1), U, Vj, rh, sums_r, s));
    AssembleParams a{};
    a.status = p->status;
    a.n = n;
    a.r_h = rh;
    a.r_out = bw;
    a.fs = fs;
    a.Xpart = p->Xpart;
    a.gC = g.gC;
    a.xp_s = p->xp_s;
    a.Ypart = p->Ypart;
    a.gR = g.gR;
    a.yp_q = p->yp_q;
    a.part_cs = p->part_cs;
    a.C = p->C;
    a.nC = 1;
    a.Uh = U;
    a.Unew = U + (int64_t)rh * fs;
    a.Ynew = V + (int64_t)(p->Rcap - rh - bw) * fs;
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_assemble<T>(a, s));
  }
  const int rk = (nsteps + 1) * bw;
  T* Vk = V + (int64_t)(p->Rcap - rk) * fs;
  LV_TRY(run_update<T>(p, p->views[view0 + nsteps], U, Vk, rk, s));
  if (sums_r > 0) LV_TRY(sums_update<T>(p, sview(p, view0 + nsteps), U, Vk, rk, sums_r, s));
  return LINVIEW_OK;
}

template <typename T>
static linview_status powers_propagate_levels(linview_program* p, int r, cudaStream_t s) {
  T* U = static_cast<T*>(p->Uar);
  T* V = static_cast<T*>(p->Var);
  const int k = p->d.k;
  if (p->d.model == LINVIEW_MODEL_LINEAR) {
    LV_TRY(krylov_levels<T>(p, r, k - 1, 0, 0, s));
    // S'_k = sum_i P_i: dS'_k = U_k K V_k^T (suffix block sums, as for the
    // exponential model's sums)
    if (has_sums(p)) {
      const int rk = k * r;
      LV_TRY(sums_update<T>(p, p->views[k], U, V + (int64_t)(p->Rcap - rk) * p->fs, rk, r, s));
    }
    return LINVIEW_OK;
  }
  if (p->d.model == LINVIEW_MODEL_SKIP) {
    const int sk = p->d.skip, Ls = ilog2(sk);
    const bool sums = has_sums(p);
    LV_TRY(exp_levels<T>(p, r, Ls, sums, s));
    return krylov_levels<T>(p, sk * r, k / sk - 1, Ls, sums ? r : 0, s);
  }
  const bool sums = has_sums(p);
  LV_TRY(exp_levels<T>(p, r, p->L, sums, s));
  const int rk = r << p->L;
  T* Vk = V + (int64_t)(p->Rcap - rk) * p->fs;
  if (sums) LV_TRY(sums_update<T>(p, sview(p, p->L), U, Vk, rk, r, s));
  LV_TRY(run_update<T>(p, pview(p, p->L), U, Vk, rk, s));
  return LINVIEW_OK;
}

template <typename T>
static linview_status powers_propagate(linview_program* p, int r, cudaStream_t s) {
  const linview_status st = powers_propagate_levels<T>(p, r, s);
  const linview_status sj = side_join(p, s);  // also after an error, to close the fork
  return st != LINVIEW_OK ? st : sj;
}

// ---------------------------------------------------------------------------
// general form T_{i+1} = A T_i + B (Appendix B, linear model)
// ---------------------------------------------------------------------------

static linview_status iter_reeval(linview_program* p, cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  const int k = p->d.k;
  const int mode = reeval_mode(p);
  View& a = p->views[0];
  char* T = static_cast<char*>(p->Tpanel);
  TcScratch sc;
  if (!library_mode(mode) && !(p->elem == 4 && view_panel_fits<float>(p, a, (int)pp)))
    LV_TRY(tc_scratch(p, &sc, n, pp, n, s));
  for (int i = 1; i <= k; ++i) {
    void* ti = T + (size_t)i * pp * p->elem;
    void* tp = T + (size_t)(i - 1) * pp * p->elem;
    if (library_mode(mode)) {
      LV_CUDA(cudaMemcpy2DAsync(ti, p->ldT * p->elem, p->Bm, p->ldB * p->elem, pp * p->elem, n,
                                cudaMemcpyDeviceToDevice, s));
      LV_TRY(gemm_rm(p, false, false, n, pp, n, 1.0, a.ptr, a.ld, tp, p->ldT, 1.0, ti, p->ldT, s,
                     mode));
    } else if (p->elem == 4 && view_panel_fits<float>(p, a, (int)pp)) {
      // a few columns: one products pass over A per step
      LV_TRY(view_panel_product<float>(p, a, false, static_cast<const float*>(tp), p->ldT,
                                       (int)pp, static_cast<const float*>(p->Bm), p->ldB,
                                       static_cast<float*>(ti), p->ldT, s));
    } else {  // T_i = A T_{i-1} + B, A's rows split once
      LV_TRY(gemm_ab(p, n, pp, n, 1.0, rows_of(a.ptr, a.ld), cols_of(tp, p->ldT), 1.0, p->Bm,
                     p->ldB, ti, p->ldT, s, &sc, i > 1));
    }
  }
  return LINVIEW_OK;
}

// exponential or skip model of an iteration program
static bool iter_exp(const linview_program* p) {
  return p->d.kind == LINVIEW_ITERATION &&
         (p->d.model == LINVIEW_MODEL_EXP || p->d.model == LINVIEW_MODEL_SKIP);
}
static linview_status iter_sk_create(linview_program* p, const void* const* inputs,
                                     const int64_t* lds, int on_dev, cudaStream_t s);

constexpr int64_t kTvCap = 16384;  // k r p of the one-pass M_i products

static linview_status iter_create(linview_program* p, const void* const* inputs,
                                  const int64_t* lds, int on_dev, cudaStream_t s) {
  if (iter_exp(p)) return iter_sk_create(p, inputs, lds, on_dev, s);
  const int64_t n = p->d.n, pp = p->d.p;
  const int k = p->d.k;
  if (pp < 1) return fail(LINVIEW_EINVAL, "p must be >= 1");
  if (k < 1) return fail(LINVIEW_EINVAL, "k must be >= 1");
  if (p->d.r_max > kMaxFusedR)
    return fail(LINVIEW_EUNSUPPORTED, "iteration programs accept rank <= %d", kMaxFusedR);
  if (lds[0] < n || lds[1] < pp || lds[2] < pp) return fail(LINVIEW_ESHAPE, "bad leading dims");
  LV_TRY(add_square_view(p, n, s));
  p->ldT = rup((int64_t)(k + 1) * pp, 64);
  LV_TRY(dalloc(p, (size_t)n * p->ldT * p->elem, &p->Tpanel, s));
  p->ldB = rup(pp, 64);
  LV_TRY(dalloc(p, (size_t)n * p->ldB * p->elem, &p->Bm, s));
  for (int i = 1; i <= k; ++i)
    LV_TRY(add_rect_view(p, static_cast<char*>(p->Tpanel) + (size_t)i * pp * p->elem, n, pp,
                         p->ldT));
  LV_TRY(add_rect_view(p, p->Bm, n, pp, p->ldB));
  LV_TRY(add_rect_view(p, p->Tpanel, n, pp, p->ldT));
  LV_TRY(copy_in(p->views[0].ptr, p->views[0].ld, inputs[0], lds[0], n, n, p->elem, on_dev, s));
  LV_TRY(copy_in(p->Bm, p->ldB, inputs[1], lds[1], n, pp, p->elem, on_dev, s));
  LV_TRY(copy_in(p->Tpanel, p->ldT, inputs[2], lds[2], n, pp, p->elem, on_dev, s));
  p->fs = rup(n, 64);
  p->Rcap = p->d.r_max * k;
  LV_TRY(dalloc(p, (size_t)p->fs * p->Rcap * p->elem, &p->Kar, s));
  LV_TRY(dalloc(p, (size_t)p->fs * p->d.r_max * p->elem, &p->V1, s));
  LV_TRY(dalloc(p, (size_t)pp * p->Rcap * p->elem, &p->Mr, s));
  // partial sets of M_i = T_i^T V for all views (one pass over the T panel),
  // when small: k r_max p <= 16384 per row block
  if ((int64_t)p->Rcap * pp <= kTvCap) {
    p->tv_cap = (int64_t)p->Rcap * pp;
    LV_TRY(dalloc(p, (size_t)panel_tv_blocks((int)n) * p->tv_cap * p->elem, &p->TVpart, s));
  }
  const PassGeom g = fused_geom(p->elem, (int)n, p->sms);
  p->part_cs = p->fs;
  p->xp_s = (int64_t)kMaxFusedR * p->part_cs;
  p->yp_q = p->xp_s;
  LV_TRY(dalloc(p, (size_t)g.gC * p->xp_s * p->elem, &p->Xpart, s));
  LV_TRY(dalloc(p, (size_t)g.gR * p->yp_q * p->elem, &p->Ypart, s));
  if (p->d.strategy == LINVIEW_STRATEGY_HYBRID) {
    p->ldD = rup(pp, 64);
    LV_TRY(dalloc(p, (size_t)2 * n * p->ldD * p->elem, &p->Dh, s));
    if (p->elem == 4 && n >= 128 && pp > kMaxFusedR) {  // products A D_{i-1} on the tensor cores
      void* t = nullptr;
      LV_TRY(dalloc(p, (size_t)n * tc_split_ld(n) * 4, &t, s));
      p->hyA = static_cast<float*>(t);
      LV_TRY(dalloc(p, (size_t)pp * tc_split_ld(n) * 4, &t, s));
      p->hyB = static_cast<float*>(t);
    }
  }
  return iter_reeval(p, s);
}

// Appendix B: U_1 = U, V_1 = T_0^T V, U_i = [U, A U_{i-1} + U (V^T U_{i-1})],
// V_i = [T_{i-1}^T V, V_{i-1}], dT_i = U_i V_i^T.  U_i's blocks are the
// Krylov blocks K_a = A'^a U (A' = A + U V^T); each step adds only the
// newest block, K_1 = A K_0 + K_0 (V^T K_0) from the old A in the pass that
// also writes A', and K_a = A' K_{a-1} afterwards.
// T_i += [K_0 .. K_{i-1}] [M_{i-1} .. M_0]^T for i = 1 .. k on the T panel
// (App. B, linear model; M blocks stored newest first, p x r each, or all
// equal to V_b when same_m): one launch of the panel kernel, else (its
// staged blocks past the device's shared memory) one GEMM per view,
// column-major T_i^T (p x n) += Mc (p x i r) Kc^T.
template <typename T>
static linview_status panel_update(linview_program* p, char* Tp, const T* K, const T* M, int k,
                                   int r, bool same_m, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int64_t fs = p->fs;
  if (panel_update_fits(k, r, sizeof(T))) {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_panel_update<T>(reinterpret_cast<T*>(Tp), p->ldT, K, fs, M, pp, n, (int)pp, k,
                                   r, s));
    return LINVIEW_OK;
  }
  for (int i = 1; i <= k; ++i) {
    void* ti = Tp + (size_t)i * pp * sizeof(T);
    const T* mc = same_m ? M : M + (int64_t)(k - i) * r * pp;
    LV_TRY(gemm_cm_own(p, false, true, pp, n, (int64_t)i * r, 1.0, mc, pp, K, fs, 1.0, ti, p->ldT,
                       s));
  }
  return LINVIEW_OK;
}

template <typename T>
static linview_status iter_propagate(linview_program* p, int r, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int k = p->d.k;
  const int64_t fs = p->fs;
  T* K = static_cast<T*>(p->Kar);
  T* V1 = static_cast<T*>(p->V1);
  T* M = static_cast<T*>(p->Mr);
  char* Tp = static_cast<char*>(p->Tpanel);
  View& a = p->views[0];
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  // M_i = T_i^T V (old T_i), stored at block k-1-i so that [M_{i-1} .. M_0]
  // is one contiguous p x (i r) slab: one pass over the T panel (partials
  // per row block) when its partial sets fit, else one batched GEMM launch
  // (column-major view: T_i is p x n (ld ldT) at panel block i, V is n x r (ld fs))
  if (p->TVpart && (int64_t)k * r * pp <= p->tv_cap) {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_panel_tv<T>(reinterpret_cast<const T*>(Tp), p->ldT, V1, fs,
                               static_cast<T*>(p->TVpart), M, pp, n, (int)pp, k, r, s));
    p->all_launches++;  // the partial sums
  } else {
    LV_TRY(gemm_cm_own(p, false, false, pp, r, n, 1.0, Tp, p->ldT, V1, fs, 0.0,
                       M + (int64_t)(k - 1) * r * pp, pp, s, k, pp, 0, -(int64_t)r * pp));
  }
  if (k >= 2) {
    {
      ProfScope ps(p, s, 0.0);
      LV_CUDA((launch_gram<T>(V1, K, fs, n, r, p->Cpart, p->ticket, p->C, p->status, s)));
    }
    // X = A K_0 on the old A, A += K_0 V^T in the same pass
    LV_TRY(run_fused<T>(p, a, kModeXU, r, K, nullptr, K, V1, p->Xpart, p->Ypart, s));
    AssembleParams as{};
    as.status = p->status;
    as.n = n;
    as.r_h = r;
    as.fs = fs;
    as.Xpart = p->Xpart;
    as.gC = g.gC;
    as.xp_s = p->xp_s;
    as.part_cs = p->part_cs;
    as.C = p->C;
    as.nC = 1;
    as.Uh = K;
    as.Unew = K + (int64_t)r * fs;
    {
      ProfScope ps(p, s, 0.0);
      LV_CUDA(launch_assemble<T>(as, s));
    }
    // the k - 1 passes over A alternate their row order (j = 1 was forward)
    for (int j = 2; j < k; ++j) {
      LV_TRY(run_fused<T>(p, a, kModeX, r, K + (int64_t)(j - 1) * r * fs, nullptr, nullptr,
                          nullptr, p->Xpart, p->Ypart, s, nullptr, j % 2 == 0));
      ProfScope ps(p, s, 0.0);
      LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n, r,
                                     K + (int64_t)j * r * fs, fs, s));
    }
  } else {
    LV_TRY(run_update<T>(p, a, K, V1, r, s));
  }
  // T_i += [K_0 .. K_{i-1}] [M_{i-1} .. M_0]^T for every i: one launch, or
  // one GEMM per view when the panel kernel's staged blocks do not fit
  LV_TRY(panel_update<T>(p, Tp, K, M, k, r, false, s));
  return LINVIEW_OK;
}

// Updates to B, dB = U_b V_b^T with A unchanged (U_b in Krylov block K_0,
// V_b in the first block of M): dT_i = A dT_{i-1} + dB gives
// dT_i = [K_0 .. K_{i-1}] [V_b .. V_b]^T with K_a = A^a U_b, so the k-1
// products with A are the only passes over the view, and every M block is
// V_b.  B itself is refreshed as well.
template <typename T>
static linview_status iter_propagate_b(linview_program* p, int rb, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int k = p->d.k;
  const int64_t fs = p->fs;
  T* K = static_cast<T*>(p->Kar);
  T* M = static_cast<T*>(p->Mr);
  char* Tp = static_cast<char*>(p->Tpanel);
  View& a = p->views[0];
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  for (int i = 1; i < k; ++i)
    LV_CUDA(cudaMemcpyAsync(M + (int64_t)i * rb * pp, M, sizeof(T) * rb * pp,
                            cudaMemcpyDeviceToDevice, s));
  for (int j = 1; j < k; ++j) {
    LV_TRY(run_fused<T>(p, a, kModeX, rb, K + (int64_t)(j - 1) * rb * fs, nullptr, nullptr,
                        nullptr, p->Xpart, p->Ypart, s, nullptr, j % 2 == 0));
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n, rb,
                                   K + (int64_t)j * rb * fs, fs, s));
  }
  // T_i += [K_0 .. K_{i-1}] [V_b .. V_b]^T for every i (every M block is V_b)
  LV_TRY(panel_update<T>(p, Tp, K, M, k, rb, true, s));
  // B += U_b V_b^T (column-major B^T, p x n)
  LV_TRY(gemm_cm_own(p, false, true, pp, n, rb, 1.0, M, pp, K, fs, 1.0, p->Bm, p->ldB, s));
  return LINVIEW_OK;
}

// Hybrid strategy (Sec. 4.3; App. B, hybrid linear model): the change of
// every iteration is kept as one dense n x p matrix D_i instead of factors.
// For dA = U V^T (U in Krylov block K_0, V in V1; A is the old matrix until
// the last step):
//   D_1 = U (V^T T_0),   D_i = A D_{i-1} + U (V^T (T_{i-1} + D_{i-1})),
// the paper's three terms U V^T T_{i-1} + A D_{i-1} + U V^T D_{i-1} with the
// two products by V^T taken once on the refreshed T'_{i-1} = T_{i-1} +
// D_{i-1}; then A += U V^T.  For dB = U_b V_b^T (U_b in K_0, V_b in the first
// block of M; A unchanged):  D_1 = U_b V_b^T,  D_i = A D_{i-1} + U_b V_b^T,
// and B += U_b V_b^T.  Each step is one n x n x p product with A (the own
// split-TF32 GEMM, or one products pass over A when p is a few columns), the
// rank-r term and T_i += D_i.  Column-major views:
// T_i^T, D_i^T are p x n (ld ldT, ldD), A's row-major storage is A^T.
template <typename T>
static linview_status iter_propagate_hybrid(linview_program* p, int r, bool b_update,
                                            cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  const int k = p->d.k;
  const int64_t fs = p->fs;
  const T* K = static_cast<const T*>(p->Kar);
  const T* V1 = static_cast<const T*>(p->V1);
  T* W = static_cast<T*>(p->Mr);  // p x r: (V^T T'_{i-1})^T, or V_b for dB
  char* Tp = static_cast<char*>(p->Tpanel);
  T* D[2] = {static_cast<T*>(p->Dh), static_cast<T*>(p->Dh) + n * p->ldD};
  const View& a = p->views[0];
  // FP32: D_i = A D_{i-1} on the tensor cores, the old A's split rows taken
  // once per propagation into the program's persistent split buffers
  TcScratch hy;
  if (p->hyA) {
    hy.a = p->hyA;
    hy.b = p->hyB;
    hy.a_rows = n;
    hy.b_rows = pp;
    hy.K = n;
  }
  bool a_split = false;
  for (int i = 1; i <= k; ++i) {
    T* dc = D[i & 1];
    const T* dp = D[(i - 1) & 1];
    T* ti = reinterpret_cast<T*>(Tp + (size_t)i * pp * sizeof(T));
    const T* tprev = reinterpret_cast<const T*>(Tp + (size_t)(i - 1) * pp * sizeof(T));
    if (!b_update)  // W^T = T'_{i-1}^T V (T'_{i-1} is already refreshed)
      LV_TRY(gemm_cm_own(p, false, false, pp, r, n, 1.0, tprev, p->ldT, V1, fs, 0.0, W, pp, s));
    double beta = 0.0;
    if (i >= 2) {  // D_i = A D_{i-1}
      if (sizeof(T) == 4 && view_panel_fits<T>(p, a, (int)pp)) {  // a few columns
        LV_TRY(view_panel_product<T>(p, a, false, dp, p->ldD, (int)pp, nullptr, 0, dc, p->ldD, s));
      } else {
        LV_TRY(gemm_ab(p, n, pp, n, 1.0, rows_of(a.ptr, a.ld), cols_of(dp, p->ldD), 0.0, nullptr,
                       0, dc, p->ldD, s, p->hyA ? &hy : nullptr, a_split));
        a_split = true;
      }
      beta = 1.0;
    }
    // D_i^T += W U^T  (the rank-r term)
    LV_TRY(gemm_cm_own(p, false, true, pp, n, r, 1.0, W, pp, K, fs, beta, dc, p->ldD, s));
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_axpy_rows<T>(ti, p->ldT, dc, p->ldD, T(1), (int)n, (int)pp, s));
  }
  if (b_update)  // B += U_b V_b^T (column-major B^T, p x n)
    LV_TRY(gemm_cm_own(p, false, true, pp, n, r, 1.0, W, pp, K, fs, 1.0, p->Bm, p->ldB, s));
  else
    LV_TRY(run_update<T>(p, a, K, V1, r, s));
  return LINVIEW_OK;
}

// ---------------------------------------------------------------------------
// general form, exponential and skip-s models (Section 3.3; Appendix B).  The
// skip-s model (s a power of two, k a multiple of s, k >= 2s) keeps
//   T_1, T_2, T_4, .., T_s  by the exponential rule T_2h = P_h T_h + S_h B,
//   T_2s, T_3s, .., T_k     by T_i = P_s T_{i-s} + S_s B,
// with the auxiliary views P_h = A^h and S'_h = A + .. + A^h (h = 2, .., s;
// P_1 = S'_1 = A) and S_h = I + S'_h - P_h; the exponential model is the
// skip model with s = k/2 (T_1, T_2, .., T_k at powers of two).
// View ids: 0 = A, 1 + j = the j-th T view (j = 0..NT-1, NT = log2(s) + k/s),
// NT + 1 = B, NT + 2 = T_0, NT + 2 + l = P_{2^l} (l = 1..log2 s),
// NT + 2 + log2(s) + l = S'_{2^l} (l = 1..log2 s).
// ---------------------------------------------------------------------------
static View& ie_T(linview_program* p, int j) { return p->views[1 + j]; }
static View& ie_P(linview_program* p, int l) {
  return l == 0 ? p->views[0] : p->views[p->ie_NT + 2 + l];
}
static View& ie_S(linview_program* p, int l) {  // S'_{2^l}; S'_1 = A
  return l == 0 ? p->views[0] : p->views[p->ie_NT + 2 + p->ie_Ls + l];
}

// t2 = B + P (th - B) + S' B  (= P th + S B with S = I + S' - P)
static linview_status iter_sk_next(linview_program* p, const View& th, View& t2, const View& ph,
                                   const View& sh, cudaStream_t s, TcScratch* sc) {
  const int64_t n = p->d.n, pp = p->d.p;
  const int mode = reeval_mode(p), e = p->elem;
  const View& b = p->views[p->ie_NT + 1];
  LV_CUDA(cudaMemcpy2DAsync(p->Dh, p->ldD * e, th.ptr, th.ld * e, pp * e, n,
                            cudaMemcpyDeviceToDevice, s));
  if (e == 4)
    LV_CUDA(launch_axpy_rows<float>(static_cast<float*>(p->Dh), p->ldD,
                                    static_cast<const float*>(b.ptr), b.ld, -1.f, (int)n, (int)pp,
                                    s));
  else
    LV_CUDA(launch_axpy_rows<double>(static_cast<double*>(p->Dh), p->ldD,
                                     static_cast<const double*>(b.ptr), b.ld, -1.0, (int)n,
                                     (int)pp, s));
  if (library_mode(mode)) {
    LV_CUDA(cudaMemcpy2DAsync(t2.ptr, t2.ld * e, b.ptr, b.ld * e, pp * e, n,
                              cudaMemcpyDeviceToDevice, s));
    LV_TRY(gemm_rm(p, false, false, n, pp, n, 1.0, ph.ptr, ph.ld, p->Dh, p->ldD, 1.0, t2.ptr,
                   t2.ld, s, mode));
    return gemm_rm(p, false, false, n, pp, n, 1.0, sh.ptr, sh.ld, b.ptr, b.ld, 1.0, t2.ptr, t2.ld,
                   s, mode);
  }
  if (e == 4 && view_panel_fits<float>(p, ph, (int)pp)) {  // a few columns: products passes
    LV_TRY(view_panel_product<float>(p, ph, false, static_cast<const float*>(p->Dh), p->ldD,
                                     (int)pp, static_cast<const float*>(b.ptr), b.ld,
                                     static_cast<float*>(t2.ptr), t2.ld, s));
    return view_panel_product<float>(p, sh, false, static_cast<const float*>(b.ptr), b.ld, (int)pp,
                                     static_cast<const float*>(t2.ptr), t2.ld,
                                     static_cast<float*>(t2.ptr), t2.ld, s);
  }
  LV_TRY(gemm_ab(p, n, pp, n, 1.0, rows_of(ph.ptr, ph.ld), cols_of(p->Dh, p->ldD), 1.0, b.ptr,
                 b.ld, t2.ptr, t2.ld, s, sc));
  return gemm_ab(p, n, pp, n, 1.0, rows_of(sh.ptr, sh.ld), cols_of(b.ptr, b.ld), 1.0, t2.ptr,
                 t2.ld, t2.ptr, t2.ld, s, sc);
}

static linview_status iter_sk_reeval(linview_program* p, cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  const int Ls = p->ie_Ls, mode = reeval_mode(p), e = p->elem;
  const bool lib = library_mode(mode);
  View& a = p->views[0];
  TcScratch sc;
  if (!lib) LV_TRY(tc_scratch(p, &sc, n, n, n, s));
  for (int l = 1; l <= Ls; ++l) {  // P_2h = P_h P_h, S'_2h = S'_h + P_h S'_h
    View& ph = ie_P(p, l - 1);
    const View& sh = ie_S(p, l - 1);
    View& p2 = ie_P(p, l);
    View& s2 = ie_S(p, l);
    if (lib) {
      LV_TRY(gemm_rm(p, false, false, n, n, n, 1.0, ph.ptr, ph.ld, ph.ptr, ph.ld, 0.0, p2.ptr,
                     p2.ld, s, mode));
      LV_CUDA(cudaMemcpy2DAsync(s2.ptr, s2.ld * e, sh.ptr, sh.ld * e, n * e, n,
                                cudaMemcpyDeviceToDevice, s));
      LV_TRY(gemm_rm(p, false, false, n, n, n, 1.0, ph.ptr, ph.ld, sh.ptr, sh.ld, 1.0, s2.ptr,
                     s2.ld, s, mode));
    } else {
      LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(ph.ptr, ph.ld), cols_of(ph.ptr, ph.ld), 0.0,
                     nullptr, 0, p2.ptr, p2.ld, s, &sc));
      LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(ph.ptr, ph.ld), cols_of(sh.ptr, sh.ld), 1.0,
                     sh.ptr, sh.ld, s2.ptr, s2.ld, s, &sc, /*a_ready=*/true));
    }
  }
  const View& b = p->views[p->ie_NT + 1];
  const View& t0 = p->views[p->ie_NT + 2];
  View& t1 = ie_T(p, 0);  // T_1 = A T_0 + B
  if (lib) {
    LV_CUDA(cudaMemcpy2DAsync(t1.ptr, t1.ld * e, b.ptr, b.ld * e, pp * e, n,
                              cudaMemcpyDeviceToDevice, s));
    LV_TRY(gemm_rm(p, false, false, n, pp, n, 1.0, a.ptr, a.ld, t0.ptr, t0.ld, 1.0, t1.ptr,
                   t1.ld, s, mode));
  } else if (e == 4 && view_panel_fits<float>(p, a, (int)pp)) {
    LV_TRY(view_panel_product<float>(p, a, false, static_cast<const float*>(t0.ptr), t0.ld,
                                     (int)pp, static_cast<const float*>(b.ptr), b.ld,
                                     static_cast<float*>(t1.ptr), t1.ld, s));
  } else {
    LV_TRY(gemm_ab(p, n, pp, n, 1.0, rows_of(a.ptr, a.ld), cols_of(t0.ptr, t0.ld), 1.0, b.ptr,
                   b.ld, t1.ptr, t1.ld, s, &sc));
  }
  for (int l = 0; l < Ls; ++l)  // T_2h from T_h, h = 2^l
    LV_TRY(iter_sk_next(p, ie_T(p, l), ie_T(p, l + 1), ie_P(p, l), ie_S(p, l), s, &sc));
  for (int j = Ls + 1; j < p->ie_NT; ++j)  // T_i from T_{i-s}
    LV_TRY(iter_sk_next(p, ie_T(p, j - 1), ie_T(p, j), ie_P(p, Ls), ie_S(p, Ls), s, &sc));
  return LINVIEW_OK;
}

static linview_status iter_sk_create(linview_program* p, const void* const* inputs,
                                     const int64_t* lds, int on_dev, cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  const int k = p->d.k;
  if (pp < 1) return fail(LINVIEW_EINVAL, "p must be >= 1");
  int sk = 0;
  if (p->d.model == LINVIEW_MODEL_EXP) {
    if (k < 2 || !is_pow2(k))
      return fail(LINVIEW_EINVAL, "the exponential model needs k a power of two >= 2 (k=%d)", k);
    sk = k / 2;
  } else {
    sk = p->d.skip;
    if (!is_pow2(sk) || k % sk != 0 || k < 2 * sk)
      return fail(LINVIEW_EINVAL,
                  "the skip model needs s a power of two, k a multiple of s, k >= 2s (k=%d s=%d)",
                  k, sk);
  }
  if ((int64_t)p->d.r_max * k > 128)
    return fail(LINVIEW_EUNSUPPORTED, "r_max*k=%lld exceeds 128", (long long)p->d.r_max * k);
  if (p->d.strategy != LINVIEW_STRATEGY_FACTORED)
    return fail(LINVIEW_EINVAL, "the exponential and skip models take the factored strategy");
  if (lds[0] < n || lds[1] < pp || lds[2] < pp) return fail(LINVIEW_ESHAPE, "bad leading dims");
  p->ie_s = sk;
  p->ie_Ls = ilog2(sk);
  p->ie_NT = p->ie_Ls + k / sk;
  const int NT = p->ie_NT, Ls = p->ie_Ls;
  LV_TRY(add_square_view(p, n, s));  // A = P_1
  p->ldT = rup((int64_t)(NT + 1) * pp, 64);
  LV_TRY(dalloc(p, (size_t)n * p->ldT * p->elem, &p->Tpanel, s));
  p->ldB = rup(pp, 64);
  LV_TRY(dalloc(p, (size_t)n * p->ldB * p->elem, &p->Bm, s));
  char* tp = static_cast<char*>(p->Tpanel);
  for (int j = 0; j < NT; ++j)  // the j-th T view in panel block j + 1
    LV_TRY(add_rect_view(p, tp + (size_t)(j + 1) * pp * p->elem, n, pp, p->ldT));
  LV_TRY(add_rect_view(p, p->Bm, n, pp, p->ldB));
  LV_TRY(add_rect_view(p, p->Tpanel, n, pp, p->ldT));  // T_0 in block 0
  for (int l = 1; l <= Ls; ++l) LV_TRY(add_square_view(p, n, s));  // P_2 .. P_s
  for (int l = 1; l <= Ls; ++l) LV_TRY(add_square_view(p, n, s));  // S'_2 .. S'_s
  LV_TRY(copy_in(p->views[0].ptr, p->views[0].ld, inputs[0], lds[0], n, n, p->elem, on_dev, s));
  LV_TRY(copy_in(p->Bm, p->ldB, inputs[1], lds[1], n, pp, p->elem, on_dev, s));
  LV_TRY(copy_in(p->Tpanel, p->ldT, inputs[2], lds[2], n, pp, p->elem, on_dev, s));
  p->fs = rup(n, 64);
  p->Rcap = p->d.r_max * sk;  // U_h, V_h up to h = s
  const int64_t ck = (int64_t)p->d.r_max * k;  // width of the factors of dT_k
  const size_t fb = (size_t)p->fs * p->Rcap * p->elem;
  LV_TRY(dalloc(p, fb, &p->Uar, s));
  LV_TRY(dalloc(p, fb, &p->Var, s));
  LV_TRY(dalloc(p, fb, &p->What, s));
  for (int i = 0; i < 2; ++i) {
    LV_TRY(dalloc(p, (size_t)p->fs * ck * p->elem, &p->Xar[i], s));
    LV_TRY(dalloc(p, (size_t)pp * ck * p->elem, &p->Yar[i], s));
  }
  LV_TRY(dalloc(p, (size_t)ck * p->Rcap * p->elem, &p->XtV, s));
  LV_TRY(dalloc(p, (size_t)pp * p->d.r_max * p->elem, &p->Mr, s));  // V_b of an update to B
  const PassGeom g = fused_geom(p->elem, (int)n, p->sms);
  p->part_cs = p->fs;
  p->xp_s = ck * p->part_cs;  // widest products block: P_s X_{k-s}
  p->yp_q = (int64_t)p->Rcap * p->part_cs;
  LV_TRY(dalloc(p, (size_t)g.gC * p->xp_s * p->elem, &p->Xpart, s));
  LV_TRY(dalloc(p, (size_t)g.gR * p->yp_q * p->elem, &p->Ypart, s));
  p->ldD = rup(pp, 64);
  LV_TRY(dalloc(p, (size_t)n * p->ldD * p->elem, &p->Dh, s));
  LV_TRY(ensure_stage(p, (size_t)2 * n * p->d.r_max * p->elem, s));
  return iter_sk_reeval(p, s);
}

// Incremental exponential / skip model for dA = U_1 V_1^T (U_1 in the U
// arena, V_1 at the right end of the V arena).  The powers part is Appendix
// A's exponential model up to P_s (and S'_h by the suffix block sums W^_h of
// V_h).  The factors of dT_i = X_i Y_i^T follow Appendix B's rule
//   U_i = [Q_h, P_h U_j + Q_h (R_h^T U_j), Z_h],  V_i = [T_j^T R_h, V_j, B^T W_h]
// (i = 2h, j = h in the exponential part; h = s, j = i - s in the skip part)
// with Q_h = U_h, R_h = V_h and dS_h = Z_h W_h^T = U_h (W^_h - V_h)^T
// (S_h = I + S'_h - P_h), so the Q_h and Z_h blocks, both U_h, merge:
//   X_i = [U_h, P_h X_j],
//   Y_i = [T_j^T V_h + Y_j (X_j^T V_h) + B^T (W^_h - V_h), Y_j],
// X_1 = U_1, Y_1 = T_0^T V_1.  Each step takes the small products from the
// old T_j, then T_j += X_j Y_j^T, and one products pass over the old P_h for
// P_h X_j.  The exponential part runs App. A's level pass on P_h (h < s)
// after its step; P_s, used by every skip step, is refreshed after them.
template <typename T>
static linview_status iter_sk_step(linview_program* p, int cur, View& tj, const View& ph, int rh,
                                   int c, const T* Vh, bool with_b, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int64_t fs = p->fs;
  const int mode = exact_mode(p);
  const View& b = p->views[p->ie_NT + 1];
  T* Xc = static_cast<T*>(p->Xar[cur]);
  T* Yc = static_cast<T*>(p->Yar[cur]);
  T* Xn = static_cast<T*>(p->Xar[cur ^ 1]);
  T* Yn = static_cast<T*>(p->Yar[cur ^ 1]);
  T* XtV = static_cast<T*>(p->XtV);
  // first block of Y_i (column-major p x rh): T_j^T V_h + Y_j (X_j^T V_h)
  LV_TRY(gemm_cm_own(p, false, false, pp, rh, n, 1.0, tj.ptr, tj.ld, Vh, fs, 0.0, Yn, pp, s));
  LV_TRY(gemm_cm_own(p, true, false, c, rh, n, 1.0, Xc, fs, Vh, fs, 0.0, XtV, c, s));
  LV_TRY(gemm_cm_own(p, false, false, pp, rh, c, 1.0, Yc, pp, XtV, c, 1.0, Yn, pp, s));
  if (with_b) {  // + B^T (W^_h - V_h) (W^_h in the What arena; dS_1 = 0)
    LV_TRY(gemm_cm_own(p, false, false, pp, rh, n, 1.0, b.ptr, b.ld, p->What, fs, 1.0, Yn, pp, s));
    LV_TRY(gemm_cm_own(p, false, false, pp, rh, n, -1.0, b.ptr, b.ld, Vh, fs, 1.0, Yn, pp, s));
  }
  LV_CUDA(cudaMemcpyAsync(Yn + (int64_t)rh * pp, Yc, sizeof(T) * pp * c, cudaMemcpyDeviceToDevice,
                          s));
  // T_j += X_j Y_j^T  (column-major T_j^T, p x n)
  LV_TRY(gemm_cm_own(p, false, true, pp, n, c, 1.0, Yc, pp, Xc, fs, 1.0, tj.ptr, tj.ld, s));
  // X_i = [U_h, P_h X_j] from the old P_h
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  LV_TRY(run_products_update<T>(p, ph, c, Xc, nullptr, nullptr, nullptr, s));
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n, c,
                                   Xn + (int64_t)rh * fs, fs, s));
  }
  LV_CUDA(cudaMemcpyAsync(Xn, p->Uar, sizeof(T) * fs * rh, cudaMemcpyDeviceToDevice, s));
  return LINVIEW_OK;
}

template <typename T>
static linview_status iter_sk_propagate(linview_program* p, int r, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int k = p->d.k, sk = p->ie_s, Ls = p->ie_Ls, NT = p->ie_NT;
  const int64_t fs = p->fs;
  T* U = static_cast<T*>(p->Uar);
  T* V = static_cast<T*>(p->Var);
  T* Wh = static_cast<T*>(p->What);
  const View& t0 = p->views[NT + 2];
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  int cur = 0;
  // X_1 = U_1, Y_1 = T_0^T V_1
  LV_CUDA(cudaMemcpyAsync(p->Xar[0], U, sizeof(T) * fs * r, cudaMemcpyDeviceToDevice, s));
  LV_TRY(gemm_cm_own(p, false, false, pp, r, n, 1.0, t0.ptr, t0.ld, V + (int64_t)(p->Rcap - r) * fs,
                 fs, 0.0, p->Yar[0], pp, s));
  for (int l = 0; l < Ls; ++l) {  // exponential part: T_2h from T_h, h = 2^l < s
    const int rh = r << l;
    T* Vh = V + (int64_t)(p->Rcap - rh) * fs;
    if (l >= 1) {
      ProfScope ps(p, s, 0.0);
      LV_CUDA(launch_suffix_sums<T>(Vh, Wh, fs, n, rh, r, s));
    }
    View& ph = ie_P(p, l);
    LV_TRY(iter_sk_step<T>(p, cur, ie_T(p, l), ph, rh, rh, Vh, l >= 1, s));
    cur ^= 1;
    // App. A's level pass on P_h, the update of S'_h, the assembly of U_2h, V_2h
    const bool fused = rh <= kMaxFusedR;
    if (!fused) {
      ProfScope ps(p, s, 0.0);
      LV_CUDA((launch_gram<T>(Vh, U, fs, n, rh, p->Cpart, p->ticket, p->C, p->status, s)));
    }
    LV_TRY(run_products_update<T>(p, ph, rh, U, Vh, U, Vh, s, fused ? p->Cpart : nullptr));
    if (l >= 1) LV_TRY(run_update<T>(p, ie_S(p, l), U, Wh, rh, s));  // dS'_h = U_h W^_h^T
    AssembleParams a{};
    a.status = p->status;
    a.n = n;
    a.r_h = rh;
    a.fs = fs;
    a.Xpart = p->Xpart;
    a.gC = g.gC;
    a.xp_s = p->xp_s;
    a.Ypart = p->Ypart;
    a.gR = g.gR;
    a.yp_q = p->yp_q;
    a.part_cs = p->part_cs;
    a.C = fused ? p->Cpart : p->C;
    a.nC = fused ? g.gR : 1;
    a.Uh = U;
    a.Unew = U + (int64_t)rh * fs;
    a.Ynew = V + (int64_t)(p->Rcap - 2 * rh) * fs;
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_assemble<T>(a, s));
  }
  // skip part: T_i from T_{i-s} with the old P_s, i = 2s, .., k
  const int rs = r * sk;
  T* Vs = V + (int64_t)(p->Rcap - rs) * fs;
  if (Ls >= 1) {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_suffix_sums<T>(Vs, Wh, fs, n, rs, r, s));
  }
  for (int j = Ls + 1; j < NT; ++j) {
    const int c = (j - Ls) * rs;  // width of the factors of T_{i-s}
    LV_TRY(iter_sk_step<T>(p, cur, ie_T(p, j - 1), ie_P(p, Ls), rs, c, Vs, Ls >= 1, s));
    cur ^= 1;
  }
  // T_k += X_k Y_k^T, then P_s and S'_s
  View& tk = ie_T(p, NT - 1);
  LV_TRY(gemm_cm_own(p, false, true, pp, n, (int64_t)r * k, 1.0, p->Yar[cur], pp, p->Xar[cur], fs,
                 1.0, tk.ptr, tk.ld, s));
  LV_TRY(run_update<T>(p, ie_P(p, Ls), U, Vs, rs, s));
  if (Ls >= 1) LV_TRY(run_update<T>(p, ie_S(p, Ls), U, Wh, rs, s));
  return LINVIEW_OK;
}

// Updates to B, dB = U_b V_b^T (U_b in the U arena, V_b in Mr, p x rb) with
// A unchanged, so P_h and S_h are unchanged (derived from the recurrences;
// the paper omits changes in B, Section 4.3.2):
//   dT_1 = dB,  dT_i = P dT_j + S dB  (P, S = P_h, S_h with j = h, i = 2h in
//   the exponential part; P_s, S_s with j = i - s in the skip part), i.e.
//   X_1 = U_b, Y_1 = V_b,  X_i = [P X_j, S U_b],  Y_i = [Y_j, V_b],
// with S U_b = U_b + S' U_b - P U_b (S_1 = I).  Each step: T_j += X_j Y_j^T,
// one products pass over P with [X_j | U_b] and, for S' != A, one over S'
// with U_b; B += U_b V_b^T at the end.
template <typename T>
static linview_status iter_sk_step_b(linview_program* p, int cur, int c, int rb, View& tj,
                                     const View& ph, const View* sh, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int64_t fs = p->fs;
  const int mode = exact_mode(p);
  const T* Ub = static_cast<const T*>(p->Uar);
  const T* Vb = static_cast<const T*>(p->Mr);
  T* Xc = static_cast<T*>(p->Xar[cur]);
  T* Yc = static_cast<T*>(p->Yar[cur]);
  T* Xn = static_cast<T*>(p->Xar[cur ^ 1]);
  T* Yn = static_cast<T*>(p->Yar[cur ^ 1]);
  T* tmp = static_cast<T*>(p->What);
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  // T_j += X_j Y_j^T
  LV_TRY(gemm_cm_own(p, false, true, pp, n, c, 1.0, Yc, pp, Xc, fs, 1.0, tj.ptr, tj.ld, s));
  // [P X_j | P U_b] in one products pass over P
  LV_CUDA(cudaMemcpyAsync(Xc + (int64_t)c * fs, Ub, sizeof(T) * fs * rb, cudaMemcpyDeviceToDevice,
                          s));
  LV_TRY(run_products_update<T>(p, ph, c + rb, Xc, nullptr, nullptr, nullptr, s));
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n,
                                   c + rb, Xn, fs, s));
  }
  // second block S U_b = U_b + S' U_b - P U_b  (U_b when S = I)
  T* blk = Xn + (int64_t)c * fs;  // column-major n x rb, seen as rb rows of n (ld fs)
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_scale_copy<T>(blk, fs, blk, fs, T(sh ? -1 : 0), rb, n, s));
    LV_CUDA(launch_axpy_rows<T>(blk, fs, Ub, fs, T(1), rb, n, s));
  }
  if (sh) {
    LV_TRY(run_products_update<T>(p, *sh, rb, Ub, nullptr, nullptr, nullptr, s));
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n, rb,
                                   tmp, fs, s));
    LV_CUDA(launch_axpy_rows<T>(blk, fs, tmp, fs, T(1), rb, n, s));
  }
  // Y_i = [Y_j, V_b]
  LV_CUDA(cudaMemcpyAsync(Yn, Yc, sizeof(T) * pp * c, cudaMemcpyDeviceToDevice, s));
  LV_CUDA(cudaMemcpyAsync(Yn + (int64_t)c * pp, Vb, sizeof(T) * pp * rb, cudaMemcpyDeviceToDevice,
                          s));
  return LINVIEW_OK;
}

template <typename T>
static linview_status iter_sk_propagate_b(linview_program* p, int rb, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int64_t pp = p->d.p;
  const int Ls = p->ie_Ls, NT = p->ie_NT;
  const int64_t fs = p->fs;
  LV_CUDA(cudaMemcpyAsync(p->Xar[0], p->Uar, sizeof(T) * fs * rb, cudaMemcpyDeviceToDevice, s));
  LV_CUDA(cudaMemcpyAsync(p->Yar[0], p->Mr, sizeof(T) * pp * rb, cudaMemcpyDeviceToDevice, s));
  int cur = 0, c = rb;
  for (int j = 1; j < NT; ++j) {  // the j-th T view from the (j-1)-th
    const int l = j <= Ls ? j - 1 : Ls;  // P_{2^l}, S'_{2^l} (S_1 = I)
    LV_TRY(iter_sk_step_b<T>(p, cur, c, rb, ie_T(p, j - 1), ie_P(p, l),
                             l >= 1 ? &ie_S(p, l) : nullptr, s));
    cur ^= 1;
    c += rb;
  }
  View& tk = ie_T(p, NT - 1);
  LV_TRY(gemm_cm_own(p, false, true, pp, n, c, 1.0, p->Yar[cur], pp, p->Xar[cur], fs, 1.0, tk.ptr,
                 tk.ld, s));
  // B += U_b V_b^T (column-major B^T, p x n)
  LV_TRY(gemm_cm_own(p, false, true, pp, n, rb, 1.0, p->Mr, pp, p->Uar, fs, 1.0, p->Bm, p->ldB, s));
  return LINVIEW_OK;
}

// ---------------------------------------------------------------------------
// OLS (Section 4.1): views W = (X^T X)^{-1}, beta = W X^T Y, X^T Y, X
// ---------------------------------------------------------------------------
#define LV_SOLVER(expr)                                                                      \
  do {                                                                                       \
    cusolverStatus_t e_ = (expr);                                                            \
    if (e_ != CUSOLVER_STATUS_SUCCESS)                                                       \
      return fail(LINVIEW_EDEVICE, "%s failed: cusolver status %d", #expr, (int)e_);         \
  } while (0)

enum { kOlsW = 0, kOlsBeta = 1, kOlsXtY = 2, kOlsX = 3 };
// replaced rows held per side before they are folded into Z (Newton-Schulz
// correction); a row block has at most 32 rows
constexpr int kOlsHistory = 512;

// Re-evaluation: Z = X^T X and X^T Y accumulated in FP64 over row chunks
// (DSYRK / DGEMM), W = Z^{-1} by Cholesky (potrf + potri), beta = W X^T Y in
// FP64, rounded once to the view type.
template <typename T>
static linview_status ols_reeval_t(linview_program* p, cudaStream_t s) {
  const int64_t m = p->d.m, n = p->d.n, pp = p->d.p;
  const int64_t ch = p->ols_chunk;
  if (!p->Z64) {
    void* t;
    LV_TRY(dalloc(p, sizeof(double) * n * n, &t, s)); p->Z64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(double) * n * n, &t, s)); p->W64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(double) * ch * n, &t, s)); p->X64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(double) * ch * pp, &t, s)); p->Y64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(double) * n * pp, &t, s)); p->XtY64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(double) * n * pp, &t, s)); p->B64 = static_cast<double*>(t);
    LV_TRY(dalloc(p, sizeof(int) * 4, &t, s)); p->solver_info = static_cast<int*>(t);
  }
  if (!p->solver && cusolverDnCreate(&p->solver) != CUSOLVER_STATUS_SUCCESS)
    return fail(LINVIEW_EDEVICE, "cusolverDnCreate failed");
  LV_BLAS(cublasSetStream(p->blas, s));
  LV_SOLVER(cusolverDnSetStream(p->solver, s));
  const double one = 1.0, zero = 0.0;
  const T* X = static_cast<const T*>(p->Xd);
  const T* Y = static_cast<const T*>(p->Yd);
  for (int64_t r0 = 0; r0 < m; r0 += ch) {
    const int64_t mc = (m - r0 < ch) ? (m - r0) : ch;
    LV_CUDA(launch_to_double<T>(X + r0 * p->ldX, p->ldX, p->X64, n, (int)mc, (int)n, s));
    LV_CUDA(launch_to_double<T>(Y + r0 * p->ldY, p->ldY, p->Y64, pp, (int)mc, (int)pp, s));
    // column-major view: X_c is n x mc (ld n); Z += X_c X_c^T (lower)
    LV_BLAS(cublasDsyrk(p->blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)n, (int)mc, &one,
                        p->X64, (int)n, r0 ? &one : &zero, p->Z64, (int)n));
    // (X^T Y)^T (p x n) += Y_c^T-view (p x mc) * X_c-view^T (mc x n)
    LV_BLAS(cublasDgemm(p->blas, CUBLAS_OP_N, CUBLAS_OP_T, (int)pp, (int)n, (int)mc, &one,
                        p->Y64, (int)pp, p->X64, (int)n, r0 ? &one : &zero, p->XtY64, (int)pp));
    p->all_launches += 4;
  }
  if (p->Zh) {  // Z = X^T X as pairs, before the factorisation overwrites it
    LV_CUDA(launch_z_from_lower(p->Z64, n, (int)n, p->Zh, p->Zl, p->ldz, s));
    p->hcnt = 0;  // the history is in this Z already
  }
  if (!p->solver_work) {
    int l1 = 0, l2 = 0;
    LV_SOLVER(cusolverDnDpotrf_bufferSize(p->solver, CUBLAS_FILL_MODE_LOWER, (int)n, p->Z64,
                                          (int)n, &l1));
    LV_SOLVER(cusolverDnDpotri_bufferSize(p->solver, CUBLAS_FILL_MODE_LOWER, (int)n, p->Z64,
                                          (int)n, &l2));
    p->solver_lwork = l1 > l2 ? l1 : l2;
    void* t;
    LV_TRY(dalloc(p, sizeof(double) * (size_t)p->solver_lwork, &t, s));
    p->solver_work = static_cast<double*>(t);
  }
  LV_SOLVER(cusolverDnDpotrf(p->solver, CUBLAS_FILL_MODE_LOWER, (int)n, p->Z64, (int)n,
                             p->solver_work, p->solver_lwork, p->solver_info));
  LV_SOLVER(cusolverDnDpotri(p->solver, CUBLAS_FILL_MODE_LOWER, (int)n, p->Z64, (int)n,
                             p->solver_work, p->solver_lwork, p->solver_info + 1));
  View& w = p->views[kOlsW];
  LV_CUDA(launch_sym_lower_to_full<T>(p->Z64, n, (int)n, static_cast<T*>(w.ptr), w.ld, p->W64, n,
                                      s));
  // beta^T (p x n) = (X^T Y)^T (p x n) * W (symmetric)
  LV_BLAS(cublasDgemm(p->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)pp, (int)n, (int)n, &one, p->XtY64,
                      (int)pp, p->W64, (int)n, &zero, p->B64, (int)pp));
  View& xty = p->views[kOlsXtY];
  View& beta = p->views[kOlsBeta];
  LV_CUDA(launch_from_double<T>(p->XtY64, pp, static_cast<T*>(xty.ptr), xty.ld, (int)n, (int)pp,
                                static_cast<T*>(p->XtYc), p->fs, s));
  LV_CUDA(launch_from_double<T>(p->B64, pp, static_cast<T*>(beta.ptr), beta.ld, (int)n, (int)pp,
                                static_cast<T*>(nullptr), 0, s));
  if (p->XtYl) LV_CUDA(launch_low_half(p->XtY64, pp, p->XtYl, xty.ld, (int)n, (int)pp, s));
  p->all_launches += 6;
  int info[2] = {0, 0};
  LV_CUDA(cudaMemcpyAsync(info, p->solver_info, sizeof(info), cudaMemcpyDeviceToHost, s));
  LV_CUDA(cudaStreamSynchronize(s));
  if (info[0] != 0 || info[1] != 0)
    return fail(LINVIEW_ESINGULAR, "X^T X is not positive definite (potrf/potri info %d/%d)",
                info[0], info[1]);
  return LINVIEW_OK;
}

static linview_status ols_create(linview_program* p, const void* const* inputs,
                                 const int64_t* lds, int on_dev, cudaStream_t s) {
  const int64_t m = p->d.m, n = p->d.n, pp = p->d.p;
  const int kmax = p->d.k;
  if (m < n || pp < 1 || kmax < 1) return fail(LINVIEW_EINVAL, "OLS needs m >= n, p >= 1, k >= 1");
  if (2 * kmax > 64) return fail(LINVIEW_EUNSUPPORTED, "row blocks are limited to k <= 32");
  if (lds[0] < n || lds[1] < pp) return fail(LINVIEW_ESHAPE, "bad leading dims");
  p->fs = rup(n, 64);
  LV_TRY(add_square_view(p, n, s));                     // W
  const int64_t ldp = rup(pp, 4);
  void* t;
  LV_TRY(dalloc(p, (size_t)n * ldp * p->elem, &t, s));   // beta
  LV_TRY(add_rect_view(p, t, n, pp, ldp));
  LV_TRY(dalloc(p, (size_t)n * ldp * p->elem, &t, s));   // X^T Y
  LV_TRY(add_rect_view(p, t, n, pp, ldp));
  p->ldX = rup(n, 64);
  LV_TRY(dalloc(p, (size_t)m * p->ldX * p->elem, &p->Xd, s));
  LV_TRY(add_rect_view(p, p->Xd, m, n, p->ldX));
  p->ldY = ldp;
  LV_TRY(dalloc(p, (size_t)m * p->ldY * p->elem, &p->Yd, s));
  LV_TRY(copy_in(p->Xd, p->ldX, inputs[0], lds[0], m, n, p->elem, on_dev, s));
  LV_TRY(copy_in(p->Yd, p->ldY, inputs[1], lds[1], m, pp, p->elem, on_dev, s));
  const int kk = 2 * kmax;
  LV_TRY(dalloc(p, (size_t)p->fs * pp * p->elem, &p->XtYc, s));
  LV_TRY(dalloc(p, (size_t)p->fs * kk * p->elem, &p->Uar, s));
  LV_TRY(dalloc(p, (size_t)p->fs * kk * p->elem, &p->Gf, s));
  LV_TRY(dalloc(p, (size_t)p->fs * kk * p->elem, &p->Wuf, s));
  LV_TRY(dalloc(p, (size_t)kk * pp * p->elem, &p->Hols, s));
  LV_TRY(dalloc(p, (size_t)kmax * pp * p->elem, &p->Yr, s));
  LV_TRY(dalloc(p, sizeof(int64_t) * kmax, &t, s));
  p->rows_d = static_cast<int64_t*>(t);
  LV_TRY(dalloc(p, sizeof(double) * kk * kk, &t, s));  // (FP32: kk x kk float2 pairs)
  p->Minv = static_cast<double*>(t);
  if (p->d.correction == LINVIEW_CORRECT_NEWTON) {  // Z = X^T X as pairs, zero padding
    p->ldz = rup(n, 64);
    LV_TRY(dalloc(p, sizeof(float) * p->ldz * p->ldz, &t, s));
    p->Zh = static_cast<float*>(t);
    LV_TRY(dalloc(p, sizeof(float) * p->ldz * p->ldz, &t, s));
    p->Zl = static_cast<float*>(t);
    LV_TRY(dalloc(p, sizeof(float) * n * ldp, &t, s));
    p->XtYl = static_cast<float*>(t);
    p->hcap = kOlsHistory;
    LV_TRY(dalloc(p, sizeof(float) * p->fs * p->hcap, &t, s));
    p->Hp = static_cast<float*>(t);
    LV_TRY(dalloc(p, sizeof(float) * p->fs * p->hcap, &t, s));
    p->Hm = static_cast<float*>(t);
  }
  if (p->elem == 4) LV_TRY(dalloc(p, sizeof(float2) * kk * kk, &p->Cdf, s));
  const PassGeom g = fused_geom(p->elem, (int)n, p->sms);
  p->part_cs = p->fs;
  const int64_t width = (kk > pp) ? kk : pp;
  p->xp_s = rup(width, kMaxFusedR) * p->part_cs;
  LV_TRY(dalloc(p, (size_t)g.gC * p->xp_s * p->elem, &p->Xpart, s));
  // FP32: G = W U by column sums, up to kMaxColSumR columns per pass, one
  // partial per row block
  const int64_t ycols = p->elem == 4 ? rup(kk < kMaxColSumR ? kk : kMaxColSumR, kMaxFusedR)
                                     : kMaxFusedR;
  p->yp_q = ycols * p->part_cs;
  LV_TRY(dalloc(p, (size_t)g.gR * p->yp_q * p->elem, &p->Ypart, s));
  if (p->elem == 4 && kk > kMaxProductR) {
    // split factors of the tensor-core update pass W += G Wu^T
    void* tc = nullptr;
    LV_TRY(dalloc(p, (size_t)tc_split_floats(n) * sizeof(float), &tc, s));
    p->tcA = static_cast<float*>(tc);
    p->tcB = p->tcA + tc_split_floats(n) / 2;
    if (!make_tmap_sw128(&p->tmA, p->tcA, 128, n, 128, 128) ||
        !make_tmap_sw128(&p->tmB, p->tcB, 128, n, 128, 32))
      return fail(LINVIEW_EDEVICE, "cuTensorMapEncodeTiled failed for the split factors");
  }
  p->ols_chunk = m < 8192 ? m : 8192;
  return p->elem == 4 ? ols_reeval_t<float>(p, s) : ols_reeval_t<double>(p, s);
}

// Row-block replacement by block Woodbury (see lv_ols.cu for the algebra).
// The launches of a row-block update once the new rows are in U's first kr
// columns and the row indices in rows_d: they depend only on kr (all
// pointers are the program's own), so they replay as a CUDA graph per kr.
template <typename T>
static linview_status ols_propagate_t(linview_program* p, int kr, cudaStream_t s) {
  const int n = (int)p->d.n;
  const int pp = (int)p->d.p;
  const int64_t fs = p->fs;
  const int kk = 2 * kr;
  T* U = static_cast<T*>(p->Uar);
  T* G = static_cast<T*>(p->Gf);
  T* Wu = static_cast<T*>(p->Wuf);
  View& w = p->views[kOlsW];
  const PassGeom g = fused_geom(sizeof(T), n, p->sms);
  // U = [X'_R^T, X_R^T]: the old rows become the kr columns after the new ones
  LV_CUDA(launch_gather_rows<T>(static_cast<const T*>(p->Xd), p->ldX, p->rows_d, kr, n,
                                U + (int64_t)kr * fs, fs, 1, s));
  LV_CUDA(launch_gather_rows<T>(static_cast<const T*>(p->Yd), p->ldY, p->rows_d, kr, pp,
                                static_cast<T*>(p->Yr), pp, 1, s));
  p->all_launches += 2;
  // X's rows and X^T Y read only U and Y_R: a side stream, next to the
  // Woodbury passes and the core, joined before the beta refresh that reads
  // the new X^T Y
  {
    cudaStream_t side = nullptr;
    LV_TRY(side_fork(p, s, &side));
    LV_CUDA(launch_scatter_rows<T>(static_cast<T*>(p->Xd), p->ldX, p->rows_d, kr, n, U, fs,
                                   side));
    View& xty0 = p->views[kOlsXtY];
    T* xtyl = nullptr;
    if constexpr (sizeof(T) == 4) xtyl = p->XtYl;
    LV_CUDA(launch_xty_update<T>(static_cast<T*>(xty0.ptr), xty0.ld, static_cast<T*>(p->XtYc),
                                 fs, U, n, pp, kr, static_cast<const T*>(p->Yr), side, xtyl));
    p->all_launches += 2;
  }
  if constexpr (sizeof(T) == 4) {
    // G = W U = W^T U (W is symmetric): column sums of a pass over W, which
    // need no cross-lane reductions, up to 32 columns per read of W
    for (int c0 = 0; c0 < kk; c0 += kMaxColSumR) {
      const int wd = (kk - c0 < kMaxColSumR) ? kk - c0 : kMaxColSumR;
      LV_TRY(run_fused<T>(p, w, kModeY, wd, nullptr, U + (int64_t)c0 * fs, nullptr, nullptr,
                          p->Xpart, p->Ypart, s));
      ProfScope ps(p, s, 0.0);
      LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Ypart), g.gR, p->yp_q, p->part_cs, n, wd,
                                     G + (int64_t)c0 * fs, fs, s));
    }
  } else {
    // G = W U (row sums, one read of W per 8 columns)
    LV_TRY(run_products_update<T>(p, w, kk, U, nullptr, nullptr, nullptr, s));
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_sum_partials<T>(static_cast<T*>(p->Xpart), g.gC, p->xp_s, p->part_cs, n, kk, G,
                                   fs, s));
  }
  // M = C^{-1} + U^T G (FP64), its inverse, Wu = -G M^{-1}
  // (FP32 programs: the core and its inverse as double-float pairs)
  float2* Cdf = sizeof(T) == 4 ? reinterpret_cast<float2*>(p->Cdf) : nullptr;
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA((launch_gram<T>(U, G, fs, n, kk, p->Cpart, p->ticket, p->C, p->status, s, Cdf)));
  }
  {
    ProfScope ps(p, s, 0.0);
    if constexpr (sizeof(T) == 4)
      LV_CUDA(launch_core_inverse_df(Cdf, kk, kr, reinterpret_cast<float2*>(p->Minv), p->status,
                                     s));
    else
      LV_CUDA(launch_core_inverse(p->C, kk, kr, p->Minv, p->status, s));
  }
  {
    ProfScope ps(p, s, 0.0);
    if constexpr (sizeof(T) == 4)
      LV_CUDA(launch_wu(G, fs, n, kk, reinterpret_cast<const float2*>(p->Minv), Wu, s));
    else
      LV_CUDA(launch_wu(G, fs, n, kk, p->Minv, Wu, s));
  }
  // W' = W + G Wu^T = W - G M^{-1} G^T
  LV_TRY(run_update<T>(p, w, G, Wu, kk, s));
  LV_TRY(side_join(p, s));  // the new X rows and X^T Y
  // beta' = beta + (G_1 - G_2) Y_R + G (Wu^T C'): from the factors, no pass over W
  View& beta = p->views[kOlsBeta];
  {
    ProfScope ps(p, s, 0.0);
    LV_CUDA(launch_beta_update<T>(static_cast<T*>(beta.ptr), beta.ld, G, Wu,
                                  static_cast<const T*>(p->XtYc), fs, n, pp, kr,
                                  static_cast<const T*>(p->Yr), static_cast<T*>(p->Hols), s));
  }
  p->all_launches += 2;
  return LINVIEW_OK;
}

// Z += X'_R^T X'_R - X_R^T X_R for the Newton-Schulz correction, deferred:
// the block's new and old rows (U's two halves) join the history, which is
// folded into Z when full and before a correction.
static linview_status ols_history_push(linview_program* p, int kr, cudaStream_t s) {
  if (!p->Zh) return LINVIEW_OK;
  const int64_t fs = p->fs;
  const float* U = static_cast<const float*>(p->Uar);
  if (p->hcnt + kr > p->hcap) {
    LV_CUDA(launch_z_flush(p->Zh, p->Zl, p->ldz, p->Hp, p->Hm, fs, (int)p->d.n, p->hcnt, s));
    p->all_launches++;
    p->hcnt = 0;
  }
  LV_CUDA(cudaMemcpyAsync(p->Hp + (int64_t)p->hcnt * fs, U, sizeof(float) * fs * kr,
                          cudaMemcpyDeviceToDevice, s));
  LV_CUDA(cudaMemcpyAsync(p->Hm + (int64_t)p->hcnt * fs, U + (int64_t)kr * fs,
                          sizeof(float) * fs * kr, cudaMemcpyDeviceToDevice, s));
  p->hcnt += kr;
  return LINVIEW_OK;
}

// Newton-Schulz correction of an FP32 OLS program: R = I - Z W (double-float),
// W <- W + W R (split-TF32 GEMM; W R is small, so its FP32-level error is far
// below W's rounding); then one step of iterative refinement of beta against
// the normal equations, r = X^T Y - Z beta (double-float, X^T Y as pairs),
// beta <- beta + W r.  (beta = W X^T Y from the corrected W would lose about
// kappa(Z) u to cancellation in the product.)
static linview_status ols_newton_correct(linview_program* p, cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  View& w = p->views[kOlsW];
  View& beta = p->views[kOlsBeta];
  View& xty = p->views[kOlsXtY];
  const int64_t ldr = rup(n, 64);
  const size_t rbytes = (size_t)alloc_bytes(n * ldr * (int64_t)sizeof(float));
  void* blk = nullptr;
  LV_TRY(talloc(p, 2 * rbytes, &blk, s));
  float* R = static_cast<float*>(blk);
  float* Tw = reinterpret_cast<float*>(static_cast<char*>(blk) + rbytes);
  float* W = static_cast<float*>(w.ptr);
  linview_status st = LINVIEW_OK;
  auto dev = [&](cudaError_t e, const char* what) {
    p->all_launches++;
    if (e != cudaSuccess && st == LINVIEW_OK)
      st = fail(LINVIEW_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
  };
  {
    TcScratch sc;
    st = tc_scratch(p, &sc, n, n > pp ? n : pp, n, s);
    if (st == LINVIEW_OK) {  // Z up to date
      dev(launch_z_flush(p->Zh, p->Zl, p->ldz, p->Hp, p->Hm, p->fs, (int)n, p->hcnt, s),
          "history flush");
      if (st == LINVIEW_OK) p->hcnt = 0;
    }
    if (st == LINVIEW_OK)  // R = I - Z W
      dev(launch_ns_residual(p->Zh, p->Zl, p->ldz, W, w.ld, (int)n, nullptr, nullptr, 0, R, ldr,
                             (int)n, s),
          "Newton-Schulz residual");
    if (st == LINVIEW_OK)  // Tw = W + W R
      st = gemm_ab(p, n, n, n, 1.0, rows_of(W, w.ld), cols_of(R, ldr), 1.0, W, w.ld, Tw, ldr, s,
                   &sc);
    if (st == LINVIEW_OK &&
        cudaMemcpy2DAsync(W, w.ld * sizeof(float), Tw, ldr * sizeof(float), n * sizeof(float), n,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      st = fail(LINVIEW_EDEVICE, "copy of the corrected W failed");
    if (st == LINVIEW_OK)  // r = X^T Y - Z beta (n x p, in R)
      dev(launch_ns_residual(p->Zh, p->Zl, p->ldz, static_cast<const float*>(beta.ptr), beta.ld,
                             (int)pp, static_cast<const float*>(xty.ptr), p->XtYl, xty.ld, R,
                             beta.ld, (int)n, s),
          "normal-equation residual");
    if (st == LINVIEW_OK)  // beta += W r
      st = gemm_ab(p, n, pp, n, 1.0, rows_of(W, w.ld), cols_of(R, beta.ld), 1.0, beta.ptr, beta.ld,
                   beta.ptr, beta.ld, s, &sc);
  }
  tfree(p, blk, 2 * rbytes, s);
  return st;
}

static linview_status correct_now(linview_program* p, cudaStream_t s) {
  if (p->d.kind == LINVIEW_OLS && p->d.correction == LINVIEW_CORRECT_NEWTON)
    return ols_newton_correct(p, s);
  return linview_reeval(p, s);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* linview_last_error(void) { return g_err.c_str(); }

linview_status linview_create_program(const linview_program_desc* desc, const void* const* inputs,
                                      const int64_t* lds, int inputs_on_device, void* stream,
                                      linview_program** out) {
  if (!desc || !inputs || !lds || !out) return fail(LINVIEW_EINVAL, "null argument");
  *out = nullptr;
  if (desc->precision != LINVIEW_F32 && desc->precision != LINVIEW_F64)
    return fail(LINVIEW_EINVAL, "bad precision %d", desc->precision);
  if (desc->n < 1 || desc->n > (1 << 20)) return fail(LINVIEW_EINVAL, "bad n=%lld", (long long)desc->n);
  if (desc->r_max < 1) return fail(LINVIEW_EINVAL, "r_max must be >= 1");
  if (desc->correction_period < 0) return fail(LINVIEW_EINVAL, "correction_period < 0");
  if ((desc->alloc == nullptr) != (desc->free == nullptr))
    return fail(LINVIEW_EINVAL, "alloc and free must both be given or both be NULL");
  if (desc->correction != LINVIEW_CORRECT_REEVAL && desc->correction != LINVIEW_CORRECT_NEWTON)
    return fail(LINVIEW_EINVAL, "bad correction %d", desc->correction);
  if (desc->correction == LINVIEW_CORRECT_NEWTON &&
      !(desc->kind == LINVIEW_OLS && desc->precision == LINVIEW_F32))
    return fail(LINVIEW_EUNSUPPORTED, "Newton-Schulz correction is built for FP32 OLS programs");
  if (desc->model != LINVIEW_MODEL_EXP &&
      !(desc->model == LINVIEW_MODEL_LINEAR &&
        (desc->kind == LINVIEW_POWER || desc->kind == LINVIEW_POWER_SUM ||
         desc->kind == LINVIEW_ITERATION)) &&
      !(desc->model == LINVIEW_MODEL_SKIP &&
        (desc->kind == LINVIEW_POWER || desc->kind == LINVIEW_POWER_SUM ||
         desc->kind == LINVIEW_ITERATION)))
    return fail(LINVIEW_EINVAL, "model %d is not available for kind %d", desc->model, desc->kind);
  if (desc->strategy != LINVIEW_STRATEGY_FACTORED &&
      !(desc->strategy == LINVIEW_STRATEGY_HYBRID && desc->kind == LINVIEW_ITERATION))
    return fail(LINVIEW_EINVAL, "strategy %d is not available for kind %d", desc->strategy,
                desc->kind);
  int ninputs = 0;
  switch (desc->kind) {
    case LINVIEW_POWER:
    case LINVIEW_POWER_SUM: ninputs = 1; break;
    case LINVIEW_ITERATION: ninputs = 3; break;
    case LINVIEW_OLS: ninputs = 2; break;
    default: return fail(LINVIEW_EINVAL, "bad kind %d", desc->kind);
  }
  for (int i = 0; i < ninputs; ++i)
    if (!inputs[i]) return fail(LINVIEW_EINVAL, "input %d is null", i);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    (void)cudaGetLastError();
    return fail(LINVIEW_EDEVICE, "no CUDA device");
  }
  if (inputs_on_device) {
    int cur = 0;
    cudaGetDevice(&cur);
    for (int i = 0; i < ninputs; ++i) LV_TRY(check_dev_ptr(inputs[i], cur, "an input"));
  }
  linview_program* p = new linview_program();
  p->d = *desc;
  p->elem = desc->precision == LINVIEW_F64 ? 8 : 4;
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  linview_status st = LINVIEW_OK;
  if (cublasCreate(&p->blas) != CUBLAS_STATUS_SUCCESS) {
    st = fail(LINVIEW_EDEVICE, "cublasCreate failed");
  }
  if (st == LINVIEW_OK) {
    void* tmp = nullptr;
    st = dalloc(p, sizeof(unsigned) * 4, &tmp, s);
    p->status = static_cast<unsigned*>(tmp);
    p->ticket = p->status + 1;
  }
  if (st == LINVIEW_OK) {
    void* tmp = nullptr;
    st = dalloc(p, sizeof(double) * 64 * 64, &tmp, s);
    p->C = static_cast<double*>(tmp);
  }
  if (st == LINVIEW_OK) {
    void* tmp = nullptr;
    st = dalloc(p, cpart_bytes(desc->n), &tmp, s);
    p->Cpart = static_cast<double*>(tmp);
  }
  if (st == LINVIEW_OK) {  // split-K partials of the CUDA-core GEMM
    void* tmp = nullptr;
    st = dalloc(p, kGemmWorkBytes, &tmp, s);
    p->gwork = tmp;
    p->gwork_elems = (int64_t)kGemmWorkBytes / p->elem;
  }
  if (st == LINVIEW_OK) {
    switch (desc->kind) {
      case LINVIEW_POWER:
      case LINVIEW_POWER_SUM: st = powers_create(p, inputs, lds, inputs_on_device, s); break;
      case LINVIEW_ITERATION: st = iter_create(p, inputs, lds, inputs_on_device, s); break;
      case LINVIEW_OLS: st = ols_create(p, inputs, lds, inputs_on_device, s); break;
      default: st = fail(LINVIEW_EUNSUPPORTED, "program kind %d not built", desc->kind);
    }
  }
  if (st != LINVIEW_OK) {
    std::string keep = g_err;
    cudaStreamSynchronize(s);
    linview_destroy(p);
    g_err = keep;
    return st;
  }
  *out = p;
  return LINVIEW_OK;
}

void linview_destroy(linview_program* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (auto& a : p->allocs) {
    if (p->d.free)
      p->d.free(a.first, a.second, nullptr, p->d.alloc_ctx);
    else if (!p->d.alloc)
      cudaFree(a.first);
  }
  for (auto& ge : p->graphs) cudaGraphExecDestroy(ge.exec);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : p->gev_pool) cudaEventDestroy(e);
  if (p->gev_in) cudaEventDestroy(p->gev_in);
  if (p->gev_out) cudaEventDestroy(p->gev_out);
  if (p->gstream) cudaStreamDestroy(p->gstream);
  if (p->side_fork_ev) cudaEventDestroy(p->side_fork_ev);
  if (p->side_join_ev) cudaEventDestroy(p->side_join_ev);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->blas) cublasDestroy(p->blas);
  if (p->solver) cusolverDnDestroy(p->solver);
  delete p;
}

linview_status linview_program_device_bytes(const linview_program* p, int64_t* bytes) {
  if (!p || !bytes) return fail(LINVIEW_EINVAL, "null argument");
  *bytes = p->bytes;
  return LINVIEW_OK;
}

linview_status linview_estimate_device_bytes(const linview_program_desc* d, int64_t* bytes) {
  if (!d || !bytes) return fail(LINVIEW_EINVAL, "null argument");
  if (d->kind != LINVIEW_POWER && d->kind != LINVIEW_POWER_SUM)
    return fail(LINVIEW_EUNSUPPORTED, "estimate only for power programs");
  if (d->precision != LINVIEW_F32 && d->precision != LINVIEW_F64)
    return fail(LINVIEW_EINVAL, "bad precision %d", d->precision);
  if (d->n < 1 || d->n > (1 << 20)) return fail(LINVIEW_EINVAL, "bad n=%lld", (long long)d->n);
  if (d->model == LINVIEW_MODEL_LINEAR || d->model == LINVIEW_MODEL_SKIP) {
    LV_TRY(check_power_model(*d));
  } else if (d->model == LINVIEW_MODEL_EXP) {
    if (!is_pow2(d->k)) return fail(LINVIEW_EINVAL, "k=%d must be a power of two", d->k);
    if (d->r_max < 1 || (int64_t)d->r_max * d->k > 128)
      return fail(LINVIEW_EUNSUPPORTED, "r_max*k must be in 1..128");
  } else {
    return fail(LINVIEW_EINVAL, "bad model %d", d->model);
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LINVIEW_EDEVICE, "no CUDA device");
  }
  *bytes = powers_device_bytes(*d, sms);
  return LINVIEW_OK;
}

int linview_num_views(const linview_program* p) { return p ? (int)p->views.size() : 0; }

linview_status linview_view_shape(const linview_program* p, int id, int64_t* rows, int64_t* cols) {
  if (!p || !rows || !cols) return fail(LINVIEW_EINVAL, "null argument");
  if (id < 0 || id >= (int)p->views.size()) return fail(LINVIEW_EINVAL, "bad view id %d", id);
  *rows = p->views[id].rows;
  *cols = p->views[id].cols;
  return LINVIEW_OK;
}

linview_status linview_view_device_ptr(const linview_program* p, int id, void** ptr, int64_t* ld) {
  if (!p || !ptr || !ld) return fail(LINVIEW_EINVAL, "null argument");
  if (id < 0 || id >= (int)p->views.size()) return fail(LINVIEW_EINVAL, "bad view id %d", id);
  *ptr = p->views[id].ptr;
  *ld = p->views[id].ld;
  return LINVIEW_OK;
}

linview_status linview_read_view(const linview_program* p, int id, void* dst, int64_t ld,
                                 int dst_on_device, void* stream) {
  if (!p || !dst) return fail(LINVIEW_EINVAL, "null argument");
  if (id < 0 || id >= (int)p->views.size()) return fail(LINVIEW_EINVAL, "bad view id %d", id);
  if (dst_on_device < LINVIEW_DST_HOST || dst_on_device > LINVIEW_DST_HOST_ASYNC)
    return fail(LINVIEW_EINVAL, "bad destination %d", dst_on_device);
  const View& v = p->views[id];
  if (ld < v.cols) return fail(LINVIEW_ESHAPE, "ld %lld < cols %lld", (long long)ld, (long long)v.cols);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LV_CUDA(cudaSetDevice(p->device));
  const bool dev = dst_on_device == LINVIEW_DST_DEVICE;
  if (dev) LV_TRY(check_dev_ptr(dst, p->device, "dst"));
  LV_CUDA(cudaMemcpy2DAsync(dst, ld * p->elem, v.ptr, v.ld * p->elem, v.cols * p->elem, v.rows,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (dst_on_device == LINVIEW_DST_HOST) LV_CUDA(cudaStreamSynchronize(s));
  return LINVIEW_OK;
}

linview_status linview_read_view_rows(const linview_program* p, int id, int64_t row0,
                                      int64_t nrows, void* dst, int64_t ld, int dst_on_device,
                                      void* stream) {
  if (!p || !dst) return fail(LINVIEW_EINVAL, "null argument");
  if (id < 0 || id >= (int)p->views.size()) return fail(LINVIEW_EINVAL, "bad view id %d", id);
  if (dst_on_device < LINVIEW_DST_HOST || dst_on_device > LINVIEW_DST_HOST_ASYNC)
    return fail(LINVIEW_EINVAL, "bad destination %d", dst_on_device);
  const View& v = p->views[id];
  if (row0 < 0 || nrows < 0 || row0 + nrows > v.rows)
    return fail(LINVIEW_EINVAL, "rows [%lld, %lld) outside the view", (long long)row0,
                (long long)(row0 + nrows));
  if (ld < v.cols) return fail(LINVIEW_ESHAPE, "ld < cols");
  if (dst_on_device == LINVIEW_DST_DEVICE) LV_TRY(check_dev_ptr(dst, p->device, "dst"));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LV_CUDA(cudaSetDevice(p->device));
  if (nrows > 0)
    LV_CUDA(cudaMemcpy2DAsync(dst, ld * p->elem,
                              static_cast<const char*>(v.ptr) + (size_t)row0 * v.ld * p->elem,
                              v.ld * p->elem, v.cols * p->elem, nrows,
                              dst_on_device == LINVIEW_DST_DEVICE ? cudaMemcpyDeviceToDevice
                                                                  : cudaMemcpyDeviceToHost,
                              s));
  if (dst_on_device == LINVIEW_DST_HOST) LV_CUDA(cudaStreamSynchronize(s));
  return LINVIEW_OK;
}

linview_status linview_reeval(linview_program* p, void* stream) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (p->d.kind) {
    case LINVIEW_POWER:
    case LINVIEW_POWER_SUM: return powers_reeval(p, s);
    case LINVIEW_ITERATION: return iter_exp(p) ? iter_sk_reeval(p, s) : iter_reeval(p, s);
    case LINVIEW_OLS: return p->elem == 4 ? ols_reeval_t<float>(p, s) : ols_reeval_t<double>(p, s);
    default: return fail(LINVIEW_EUNSUPPORTED, "reeval for kind %d", p->d.kind);
  }
}

linview_status linview_correct(linview_program* p, void* stream) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  LV_CUDA(cudaSetDevice(p->device));
  return correct_now(p, static_cast<cudaStream_t>(stream));
}

linview_status linview_set_reeval_mode(linview_program* p, int mode) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  if (mode < LINVIEW_REEVAL_DEFAULT || mode > LINVIEW_REEVAL_TC3)
    return fail(LINVIEW_EINVAL, "bad reeval mode %d", mode);
  if (p->elem == 8 && mode != LINVIEW_REEVAL_DEFAULT && mode != LINVIEW_REEVAL_FP64)
    return fail(LINVIEW_EINVAL, "FP64 programs re-evaluate in FP64");
  if (p->elem == 4 && mode == LINVIEW_REEVAL_FP64)
    return fail(LINVIEW_EINVAL, "FP32 programs cannot re-evaluate in FP64 storage");
  p->d.reeval_mode = mode;
  return LINVIEW_OK;
}

static linview_status after_update(linview_program* p, cudaStream_t s) {
  p->updates++;
  if (p->d.correction_period > 0 && p->updates % p->d.correction_period == 0)
    return correct_now(p, s);
  return LINVIEW_OK;
}

// Powers/sums: the launches after ingest depend only on the rank (all
// pointers are the program's own), so they are captured once per rank into
// a CUDA graph and replayed.  With profiling on, kProfCopies instrumented
// copies per rank (an event pair around every view pass) are captured at the
// first call and replayed round-robin, so that the passes are timed inside
// the same graph replays the caller times.
constexpr int kProfCopies = 16;

// Graph keys: the update rank r; updates to B of an iteration program use
// kKeyB + r.
constexpr int kKeyB = 1024;

// The launches of one update after its factors are in place, on stream s.
static linview_status propagate_eager(linview_program* p, int key, cudaStream_t s) {
  if (p->d.kind == LINVIEW_OLS) {
    const linview_status st = p->elem == 4 ? ols_propagate_t<float>(p, key, s)
                                           : ols_propagate_t<double>(p, key, s);
    const linview_status sj = side_join(p, s);  // also after an error, to close the fork
    LV_TRY(st);
    return sj;
  }
  if (p->d.kind == LINVIEW_ITERATION) {
    if (iter_exp(p)) {
      if (key >= kKeyB)
        return p->elem == 4 ? iter_sk_propagate_b<float>(p, key - kKeyB, s)
                            : iter_sk_propagate_b<double>(p, key - kKeyB, s);
      return p->elem == 4 ? iter_sk_propagate<float>(p, key, s)
                          : iter_sk_propagate<double>(p, key, s);
    }
    if (p->d.strategy == LINVIEW_STRATEGY_HYBRID) {
      const bool bu = key >= kKeyB;
      const int r = bu ? key - kKeyB : key;
      return p->elem == 4 ? iter_propagate_hybrid<float>(p, r, bu, s)
                          : iter_propagate_hybrid<double>(p, r, bu, s);
    }
    if (key >= kKeyB)
      return p->elem == 4 ? iter_propagate_b<float>(p, key - kKeyB, s)
                          : iter_propagate_b<double>(p, key - kKeyB, s);
    return p->elem == 4 ? iter_propagate<float>(p, key, s) : iter_propagate<double>(p, key, s);
  }
  return p->elem == 4 ? powers_propagate<float>(p, key, s) : powers_propagate<double>(p, key, s);
}

static linview_status capture_graph(linview_program* p, int r, bool inst,
                                    linview_program::GraphEntry* out) {
  const int64_t before = p->all_launches;
  out->r = r;
  out->instrumented = inst;
  p->capturing_prof = inst;
  p->capture_recs = inst ? &out->recs : nullptr;
  const bool prof_was = p->prof;
  p->prof = inst;
  LV_CUDA(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
  linview_status st = propagate_eager(p, r, p->gstream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(p->gstream, &graph);
  p->capturing_prof = false;
  p->capture_recs = nullptr;
  p->prof = prof_was;
  const int64_t launches = p->all_launches - before;
  p->all_launches = before;
  if (st != LINVIEW_OK) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();  // do not leave the capture error to later calls
    return st;
  }
  if (ec != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(LINVIEW_EDEVICE, "graph capture failed: %s", cudaGetErrorString(ec));
  }
  const cudaError_t ei = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess)
    return fail(LINVIEW_EDEVICE, "graph instantiate failed: %s", cudaGetErrorString(ei));
  out->launches = launches;
  return LINVIEW_OK;
}

// The graphs of key r (captured on first use), indices into p->graphs.
static linview_status graphs_for(linview_program* p, int r, bool inst, std::vector<size_t>* idx) {
  if (!p->gstream) {
    LV_CUDA(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    LV_CUDA(cudaEventCreateWithFlags(&p->gev_in, cudaEventDisableTiming));
    LV_CUDA(cudaEventCreateWithFlags(&p->gev_out, cudaEventDisableTiming));
  }
  idx->clear();
  for (size_t i = 0; i < p->graphs.size(); ++i)
    if (p->graphs[i].r == r && p->graphs[i].instrumented == inst) idx->push_back(i);
  if (idx->empty()) {
    const int copies = inst ? kProfCopies : 1;
    for (int c = 0; c < copies; ++c) {
      linview_program::GraphEntry ge;
      LV_TRY(capture_graph(p, r, inst, &ge));
      p->graphs.push_back(std::move(ge));
      idx->push_back(p->graphs.size() - 1);
    }
  }
  return LINVIEW_OK;
}

static linview_status graph_propagate(linview_program* p, int r, cudaStream_t s) {
  const bool inst = p->prof;
  std::vector<size_t> idx;
  LV_TRY(graphs_for(p, r, inst, &idx));
  size_t pick = idx[0];
  if (inst) {
    if ((int)p->prof_rr.size() <= r) p->prof_rr.resize(r + 1, 0);
    pick = idx[p->prof_rr[r]++ % idx.size()];
  }
  linview_program::GraphEntry& ge = p->graphs[pick];
  LV_CUDA(cudaEventRecord(p->gev_in, s));
  LV_CUDA(cudaStreamWaitEvent(p->gstream, p->gev_in, 0));
  LV_CUDA(cudaGraphLaunch(ge.exec, p->gstream));
  LV_CUDA(cudaEventRecord(p->gev_out, p->gstream));
  LV_CUDA(cudaStreamWaitEvent(s, p->gev_out, 0));
  ge.replayed = true;
  p->all_launches += ge.launches;
  return LINVIEW_OK;
}

// Powers, sums and iterations: the launches after ingest depend only on the
// key (all pointers are the program's own), so they replay as CUDA graphs.
static linview_status propagate(linview_program* p, int key, cudaStream_t s) {
  switch (p->d.kind) {
    case LINVIEW_POWER:
    case LINVIEW_POWER_SUM:
    case LINVIEW_ITERATION:
    case LINVIEW_OLS:
      if (p->use_graphs) return graph_propagate(p, key, s);
      return propagate_eager(p, key, s);
    default: return fail(LINVIEW_EUNSUPPORTED, "updates for kind %d", p->d.kind);
  }
}

// column-major destinations of the input factors
static void* u_dst(linview_program* p) {
  return (p->d.kind == LINVIEW_ITERATION && !iter_exp(p)) ? p->Kar : p->Uar;
}
static void* v_dst(linview_program* p, int r) {
  if (p->d.kind == LINVIEW_ITERATION && !iter_exp(p)) return p->V1;
  return static_cast<char*>(p->Var) + (size_t)(p->Rcap - r) * p->fs * p->elem;
}

// dB = U V^T for an iteration program: U (n x rank) into Krylov block K_0, V
// (p x rank) into the first M block, then the propagation above.
static linview_status apply_b_delta(linview_program* p, int r, const void* U, int64_t ldu,
                                    const void* V, int64_t ldv, int on_device, cudaStream_t s) {
  const int64_t n = p->d.n, pp = p->d.p;
  const void* u = U;
  const void* v = V;
  if (!on_device) {
    LV_TRY(ensure_stage(p, (size_t)(n + pp) * r * p->elem, s));
    char* st = static_cast<char*>(p->stage);
    LV_TRY(copy_in(st, r, U, ldu, n, r, p->elem, 0, s));
    LV_TRY(copy_in(st + (size_t)n * r * p->elem, r, V, ldv, pp, r, p->elem, 0, s));
    u = st;
    v = st + (size_t)n * r * p->elem;
    ldu = r;
    ldv = r;
  }
  // U_b into Krylov block K_0 (linear model) or the U arena (exponential and
  // skip models); V_b into M (p x rank)
  void* ub_dst = iter_exp(p) ? p->Uar : p->Kar;
  if (p->elem == 4) {
    LV_CUDA(launch_rm_to_cm<float>(static_cast<const float*>(u), ldu, static_cast<float*>(ub_dst),
                                   p->fs, (int)n, r, s));
    LV_CUDA(launch_rm_to_cm<float>(static_cast<const float*>(v), ldv, static_cast<float*>(p->Mr),
                                   pp, (int)pp, r, s));
  } else {
    LV_CUDA(launch_rm_to_cm<double>(static_cast<const double*>(u), ldu,
                                    static_cast<double*>(ub_dst), p->fs, (int)n, r, s));
    LV_CUDA(launch_rm_to_cm<double>(static_cast<const double*>(v), ldv,
                                    static_cast<double*>(p->Mr), pp, (int)pp, r, s));
  }
  p->all_launches += 2;
  LV_TRY(propagate(p, kKeyB + r, s));
  return after_update(p, s);
}

linview_status linview_apply_delta(linview_program* p, int input_id, int64_t rank, const void* U,
                                   int64_t ldu, const void* V, int64_t ldv, int on_device,
                                   void* stream) {
  if (!p || !U || !V) return fail(LINVIEW_EINVAL, "null argument");
  if (p->d.kind == LINVIEW_OLS) return fail(LINVIEW_EINVAL, "OLS takes linview_apply_row_block");
  const bool b_update = p->d.kind == LINVIEW_ITERATION && input_id == 1;
  if (input_id != 0 && !b_update)
    return fail(LINVIEW_EUNSUPPORTED, "input %d has no trigger for this program", input_id);
  if (rank < 1) return fail(LINVIEW_EINVAL, "rank must be >= 1");
  if (rank > p->d.r_max) return fail(LINVIEW_ERANK, "rank %lld > r_max %d", (long long)rank, p->d.r_max);
  if (ldu < rank || ldv < rank) return fail(LINVIEW_ESHAPE, "ldu/ldv < rank");
  if (on_device) {
    LV_TRY(check_dev_ptr(U, p->device, "U"));
    LV_TRY(check_dev_ptr(V, p->device, "V"));
  }
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b_update) return apply_b_delta(p, (int)rank, U, ldu, V, ldv, on_device, s);
  const int64_t n = p->d.n;
  const int r = (int)rank;
  const void* u = U;
  const void* v = V;
  if (!on_device) {
    LV_TRY(ensure_stage(p, (size_t)2 * n * r * p->elem, s));
    char* st = static_cast<char*>(p->stage);
    LV_TRY(copy_in(st, r, U, ldu, n, r, p->elem, 0, s));
    LV_TRY(copy_in(st + (size_t)n * r * p->elem, r, V, ldv, n, r, p->elem, 0, s));
    u = st;
    v = st + (size_t)n * r * p->elem;
    ldu = r;
    ldv = r;
  }
  if (p->elem == 4) {
    LV_CUDA(launch_rm_to_cm<float>(static_cast<const float*>(u), ldu, static_cast<float*>(u_dst(p)),
                                   p->fs, (int)n, r, s));
    LV_CUDA(launch_rm_to_cm<float>(static_cast<const float*>(v), ldv,
                                   static_cast<float*>(v_dst(p, r)), p->fs, (int)n, r, s));
  } else {
    LV_CUDA(launch_rm_to_cm<double>(static_cast<const double*>(u), ldu,
                                    static_cast<double*>(u_dst(p)), p->fs, (int)n, r, s));
    LV_CUDA(launch_rm_to_cm<double>(static_cast<const double*>(v), ldv,
                                    static_cast<double*>(v_dst(p, r)), p->fs, (int)n, r, s));
  }
  p->all_launches += 2;
  LV_TRY(propagate(p, r, s));
  return after_update(p, s);
}

linview_status linview_apply_row_delta(linview_program* p, int input_id, int64_t row,
                                       const void* v, int on_device, void* stream) {
  if (!p || !v) return fail(LINVIEW_EINVAL, "null argument");
  if (p->d.kind == LINVIEW_OLS) return fail(LINVIEW_EINVAL, "OLS takes linview_apply_row_block");
  if (input_id != 0) return fail(LINVIEW_EUNSUPPORTED, "only input 0 (A) has a trigger");
  const int64_t n = p->d.n;
  if (row < 0 || row >= n) return fail(LINVIEW_EINVAL, "row %lld out of range", (long long)row);
  if (on_device) LV_TRY(check_dev_ptr(v, p->device, "v"));
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LV_CUDA(cudaMemcpyAsync(v_dst(p, 1), v, n * p->elem,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (p->elem == 4) {
    LV_CUDA(launch_unit_column<float>(static_cast<float*>(u_dst(p)), (int)n, (int)row, s));
  } else {
    LV_CUDA(launch_unit_column<double>(static_cast<double*>(u_dst(p)), (int)n, (int)row, s));
  }
  p->all_launches += 1;
  LV_TRY(propagate(p, 1, s));
  return after_update(p, s);
}

linview_status linview_apply_row_block(linview_program* p, int64_t kr, const int64_t* rows,
                                       const void* new_rows, int64_t ld, int on_device,
                                       void* stream) {
  if (!p || !rows || !new_rows) return fail(LINVIEW_EINVAL, "null argument");
  if (p->d.kind != LINVIEW_OLS) return fail(LINVIEW_EINVAL, "not an OLS program");
  if (kr < 1 || kr > p->d.k)
    return fail(LINVIEW_ESHAPE, "row block of %lld rows (program takes 1..%d)", (long long)kr,
                p->d.k);
  const int64_t n = p->d.n, m = p->d.m;
  if (ld < n) return fail(LINVIEW_ESHAPE, "ld < n");
  for (int64_t i = 0; i < kr; ++i) {
    if (rows[i] < 0 || rows[i] >= m) return fail(LINVIEW_EINVAL, "row index out of range");
    for (int64_t j = 0; j < i; ++j)
      if (rows[j] == rows[i]) return fail(LINVIEW_EINVAL, "row indices must be distinct");
  }
  if (on_device) LV_TRY(check_dev_ptr(new_rows, p->device, "new_rows"));
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // stage: the row indices, and the new rows as U's first kr columns
  LV_CUDA(cudaMemcpyAsync(p->rows_d, rows, sizeof(int64_t) * kr, cudaMemcpyHostToDevice, s));
  LV_CUDA(cudaMemcpy2DAsync(p->Uar, p->fs * p->elem, new_rows, ld * p->elem, (size_t)n * p->elem,
                            kr, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  LV_TRY(propagate(p, (int)kr, s));
  LV_TRY(ols_history_push(p, (int)kr, s));
  return after_update(p, s);
}

linview_status linview_prepare_updates(linview_program* p, int32_t max_rank, void* stream) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  if (max_rank < 1 || max_rank > p->d.r_max)
    return fail(LINVIEW_ERANK, "max_rank must be in 1..r_max (%d)", p->d.r_max);
  (void)stream;  // capture only: nothing is queued
  if (!p->use_graphs || p->d.kind == LINVIEW_OLS) return LINVIEW_OK;
  LV_CUDA(cudaSetDevice(p->device));
  std::vector<size_t> idx;
  for (int r = 1; r <= max_rank; ++r) LV_TRY(graphs_for(p, r, p->prof, &idx));
  return LINVIEW_OK;
}

linview_status linview_sync(linview_program* p, void* stream) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  LV_CUDA(cudaSetDevice(p->device));
  LV_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned st = 0;
  LV_CUDA(cudaMemcpy(&st, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) LV_CUDA(cudaMemset(p->status, 0, sizeof(unsigned)));
  if (st & kStatusTimeout) return fail(LINVIEW_ETIMEOUT, "a bounded device wait expired");
  if (st & kStatusSingular) return fail(LINVIEW_ESINGULAR, "Woodbury core is singular");
  if (st & kStatusNonFinite) return fail(LINVIEW_ENONFINITE, "non-finite factor core");
  return LINVIEW_OK;
}

linview_status linview_check_bounded_wait(int64_t limit_ns, void* stream, int64_t* waited_ns) {
  if (!waited_ns) return fail(LINVIEW_EINVAL, "null argument");
  *waited_ns = 0;
  if (limit_ns < 1000000 || limit_ns > 10000000000ll)
    return fail(LINVIEW_EINVAL, "limit_ns must be in [1e6, 1e10]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* buf = nullptr;
  LV_CUDA(cudaMalloc(&buf, 16));
  unsigned* status = static_cast<unsigned*>(buf);
  auto* waited = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 8);
  cudaError_t e = cudaMemsetAsync(buf, 0, 16, s);
  if (e == cudaSuccess) e = launch_bounded_wait_probe((uint64_t)limit_ns, status, waited, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  unsigned st = 0;
  unsigned long long w = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&w, waited, sizeof(w), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(LINVIEW_EDEVICE, "bounded-wait probe: %s", cudaGetErrorString(e));
  *waited_ns = (int64_t)w;
  if (st & kStatusTimeout) return fail(LINVIEW_ETIMEOUT, "the probe's bounded wait expired");
  return LINVIEW_OK;
}

// ---------------------------------------------------------------- adjoints
// Reverse pass of T_i = A T_{i-1} + B, i = 1..k, from the seed G_k = dL/dT_k
// (Gk, or 2 T_k when Gk is NULL: L = ||T_k||_F^2).
static linview_status adjoint_iteration(linview_program* p, const void* Gk, int64_t ldg, void* dA,
                                        int64_t ld_dA, void* dB, int64_t ld_dB, void* dT0,
                                        int64_t ld_dT0, void* stream) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  if (p->d.kind != LINVIEW_ITERATION) return fail(LINVIEW_EINVAL, "not an iteration program");
  const int64_t n = p->d.n, pp = p->d.p;
  const int k = p->d.k;
  if ((dA && ld_dA < n) || (dB && ld_dB < pp) || (Gk && ldg < pp) || (dT0 && ld_dT0 < pp))
    return fail(LINVIEW_ESHAPE, "bad leading dims");
  LV_TRY(check_dev_ptr(Gk, p->device, "Gk"));
  LV_TRY(check_dev_ptr(dA, p->device, "dA"));
  LV_TRY(check_dev_ptr(dB, p->device, "dB"));
  LV_TRY(check_dev_ptr(dT0, p->device, "dT0"));
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->Gpanel) {
    p->ldG = rup((int64_t)k * pp, 64);
    LV_TRY(dalloc(p, (size_t)n * p->ldG * p->elem, &p->Gpanel, s));
  }
  const int e = p->elem;
  char* G = static_cast<char*>(p->Gpanel);
  char* T = static_cast<char*>(p->Tpanel);
  int64_t ldT = p->ldT;
  View& a = p->views[0];
  // split operands of the tensor-core products (FP32): up to n rows each, inner
  // length up to max(n, k p)
  TcScratch sc;
  LV_TRY(tc_scratch(p, &sc, n, n, n > k * pp ? n : k * pp, s));
  // a few columns (FP32): the products with A and A^T are products passes over A
  const bool narrow = e == 4 && view_panel_fits<float>(p, a, (int)pp);
  if (iter_exp(p)) {
    // the exponential and skip models keep only some T_i: the reverse pass
    // needs T_0 .. T_k, recomputed here as T_i = A T_{i-1} + B (the same
    // function of (A, B, T_0), so the same gradient)
    if (!p->Tfull) {
      p->ldTf = rup((int64_t)(k + 1) * pp, 64);
      LV_TRY(dalloc(p, (size_t)n * p->ldTf * p->elem, &p->Tfull, s));
    }
    T = static_cast<char*>(p->Tfull);
    ldT = p->ldTf;
    const View& t0 = p->views[p->ie_NT + 2];
    LV_CUDA(cudaMemcpy2DAsync(T, ldT * e, t0.ptr, t0.ld * e, pp * e, n, cudaMemcpyDeviceToDevice,
                              s));
    for (int i = 1; i <= k; ++i) {
      char* tp = T + (size_t)(i - 1) * pp * e;
      char* ti = T + (size_t)i * pp * e;
      if (narrow)
        LV_TRY(view_panel_product<float>(p, a, false, reinterpret_cast<const float*>(tp), ldT,
                                         (int)pp, static_cast<const float*>(p->Bm), p->ldB,
                                         reinterpret_cast<float*>(ti), ldT, s));
      else
        LV_TRY(gemm_ab(p, n, pp, n, 1.0, rows_of(a.ptr, a.ld), cols_of(tp, ldT), 1.0, p->Bm,
                       p->ldB, ti, ldT, s, &sc, i > 1));
    }
  }
  // G_k = seed; G_i = A^T G_{i+1}
  void* gk = G + (size_t)(k - 1) * pp * e;
  const void* src = Gk ? Gk : T + (size_t)k * pp * e;
  const int64_t lds = Gk ? ldg : ldT;
  if (e == 4)
    LV_CUDA(launch_scale_copy<float>(static_cast<float*>(gk), p->ldG,
                                     static_cast<const float*>(src), lds, Gk ? 1.0f : 2.0f,
                                     (int)n, (int)pp, s));
  else
    LV_CUDA(launch_scale_copy<double>(static_cast<double*>(gk), p->ldG,
                                      static_cast<const double*>(src), lds, Gk ? 1.0 : 2.0,
                                      (int)n, (int)pp, s));
  p->all_launches++;
  // the rows of A^T are split once for all the products A^T G
  bool at_split = false;
  for (int i = k - 1; i >= 1; --i) {
    void* gi = G + (size_t)(i - 1) * pp * e;
    void* gn = G + (size_t)i * pp * e;
    if (narrow) {
      LV_TRY(view_panel_product<float>(p, a, true, static_cast<const float*>(gn), p->ldG, (int)pp,
                                       nullptr, 0, static_cast<float*>(gi), p->ldG, s));
    } else {
      LV_TRY(gemm_ab(p, n, pp, n, 1.0, cols_of(a.ptr, a.ld), cols_of(gn, p->ldG), 0.0, nullptr,
                     0, gi, p->ldG, s, &sc, at_split));
      at_split = true;
    }
  }
  if (dT0) {
    // dL/dT_0 = A^T G_1
    if (narrow)
      LV_TRY(view_panel_product<float>(p, a, true, static_cast<const float*>(static_cast<void*>(G)),
                                       p->ldG, (int)pp, nullptr, 0, static_cast<float*>(dT0),
                                       ld_dT0, s));
    else
      LV_TRY(gemm_ab(p, n, pp, n, 1.0, cols_of(a.ptr, a.ld), cols_of(G, p->ldG), 0.0, nullptr, 0,
                     dT0, ld_dT0, s, &sc, at_split));
  }
  if (dB) {
    LV_CUDA(cudaMemcpy2DAsync(dB, ld_dB * e, G, p->ldG * e, pp * e, n, cudaMemcpyDeviceToDevice, s));
    for (int i = 2; i <= k; ++i) {
      void* gi = G + (size_t)(i - 1) * pp * e;
      if (e == 4)
        LV_CUDA(launch_axpy_rows<float>(static_cast<float*>(dB), ld_dB, static_cast<float*>(gi),
                                        p->ldG, 1.0f, (int)n, (int)pp, s));
      else
        LV_CUDA(launch_axpy_rows<double>(static_cast<double*>(dB), ld_dB,
                                         static_cast<double*>(gi), p->ldG, 1.0, (int)n, (int)pp, s));
      p->all_launches++;
    }
  }
  if (dA) {
    // dA = [G_1 .. G_k] [T_0 .. T_{k-1}]^T, one product with inner dimension k p
    LV_TRY(gemm_ab(p, n, n, (int64_t)k * pp, 1.0, rows_of(G, p->ldG), rows_of(T, ldT), 0.0,
                   nullptr, 0, dA, ld_dA, s, &sc));
  }
  return LINVIEW_OK;
}

linview_status linview_adjoint_iteration(linview_program* p, void* dA, int64_t ld_dA, void* dB,
                                         int64_t ld_dB, void* stream) {
  return adjoint_iteration(p, nullptr, 0, dA, ld_dA, dB, ld_dB, nullptr, 0, stream);
}

linview_status linview_adjoint_iteration_seed(linview_program* p, const void* Gk, int64_t ldg,
                                              void* dA, int64_t ld_dA, void* dB, int64_t ld_dB,
                                              void* dT0, int64_t ld_dT0, void* stream) {
  if (!Gk) return fail(LINVIEW_EINVAL, "null seed");
  return adjoint_iteration(p, Gk, ldg, dA, ld_dA, dB, ld_dB, dT0, ld_dT0, stream);
}

linview_status linview_adjoint_power(linview_program* p, const void* G, int64_t ldg, void* dA,
                                     int64_t ld_dA, void* stream) {
  if (!p || !G || !dA) return fail(LINVIEW_EINVAL, "null argument");
  if (p->d.kind != LINVIEW_POWER && p->d.kind != LINVIEW_POWER_SUM)
    return fail(LINVIEW_EINVAL, "not a power program");
  LV_TRY(check_dev_ptr(G, p->device, "G"));
  LV_TRY(check_dev_ptr(dA, p->device, "dA"));
  if (p->d.model != LINVIEW_MODEL_EXP)
    return fail(LINVIEW_EUNSUPPORTED, "the power adjoint runs on the squaring chain (exponential model)");
  const int64_t n = p->d.n;
  if (ldg < n || ld_dA < n) return fail(LINVIEW_ESHAPE, "bad leading dims");
  LV_CUDA(cudaSetDevice(p->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int e = p->elem;
  const int64_t ldw = rup(n, 64);
  if (!p->Gw0) {
    LV_TRY(dalloc(p, (size_t)n * ldw * e, &p->Gw0, s));
    LV_TRY(dalloc(p, (size_t)n * ldw * e, &p->Gw1, s));
  }
  LV_CUDA(cudaMemcpy2DAsync(p->Gw0, ldw * e, G, ldg * e, n * e, n, cudaMemcpyDeviceToDevice, s));
  void* cur = p->Gw0;
  void* nxt = p->Gw1;
  TcScratch sc;
  LV_TRY(tc_scratch(p, &sc, n, n, n, s));
  // Gbar_h = Gbar_{2h} P_h^T + P_h^T Gbar_{2h}, h = k/2, ..., 1
  for (int l = p->L - 1; l >= 0; --l) {
    View& ph = pview(p, l);
    LV_TRY(gemm_ab(p, n, n, n, 1.0, rows_of(cur, ldw), rows_of(ph.ptr, ph.ld), 0.0, nullptr, 0,
                   nxt, ldw, s, &sc));
    LV_TRY(gemm_ab(p, n, n, n, 1.0, cols_of(ph.ptr, ph.ld), cols_of(cur, ldw), 1.0, nxt, ldw, nxt,
                   ldw, s, &sc));
    void* t = cur;
    cur = nxt;
    nxt = t;
  }
  LV_CUDA(cudaMemcpy2DAsync(dA, ld_dA * e, cur, ldw * e, n * e, n, cudaMemcpyDeviceToDevice, s));
  return LINVIEW_OK;
}

// ------------------------------------------------------ stand-alone product
linview_status linview_gemm(int precision, int ta, int tb, int64_t M, int64_t N, int64_t K,
                            double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                            double beta, void* C, int64_t ldc, void* stream) {
  if (precision != LINVIEW_F32 && precision != LINVIEW_F64)
    return fail(LINVIEW_EINVAL, "bad precision");
  if (M < 0 || N < 0 || K < 1 || M > (1 << 30) || N > (1 << 30) || K > (1 << 30))
    return fail(LINVIEW_EINVAL, "need M, N >= 0 and K >= 1");
  if (M == 0 || N == 0) return LINVIEW_OK;  // empty result: nothing to read or write
  if (!A || !B || !C) return fail(LINVIEW_EINVAL, "null argument");
  if (ldc < N || lda < (ta ? M : K) || ldb < (tb ? K : N))
    return fail(LINVIEW_ESHAPE, "leading dimension smaller than the row length");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  linview_program tmp;  // borrowed machinery, no views owned
  tmp.elem = precision == LINVIEW_F64 ? 8 : 4;
  cudaGetDevice(&tmp.device);
  LV_TRY(check_dev_ptr(A, tmp.device, "A"));
  LV_TRY(check_dev_ptr(B, tmp.device, "B"));
  LV_TRY(check_dev_ptr(C, tmp.device, "C"));
  cudaDeviceGetAttribute(&tmp.sms, cudaDevAttrMultiProcessorCount, tmp.device);
  void* work = nullptr;
  LV_TRY(talloc(&tmp, kGemmWorkBytes + 256, &work, s));
  tmp.status = static_cast<unsigned*>(work);
  tmp.gwork = static_cast<char*>(work) + 256;
  tmp.gwork_elems = (int64_t)kGemmWorkBytes / tmp.elem;
  cudaError_t ce = cudaMemsetAsync(work, 0, 256, s);
  linview_status st = ce == cudaSuccess ? LINVIEW_OK : fail(LINVIEW_EDEVICE, "memset failed");
  if (st == LINVIEW_OK) {
    TcScratch sc;
    st = tc_scratch(&tmp, &sc, M, N, K, s);
    // op(A) rows; op(B)^T rows (op(B) is K x N)
    const Opnd a = ta ? cols_of(A, lda) : rows_of(A, lda);
    const Opnd b = tb ? rows_of(B, ldb) : cols_of(B, ldb);
    if (st == LINVIEW_OK) st = gemm_ab(&tmp, M, N, K, alpha, a, b, beta, C, ldc, C, ldc, s, &sc);
  }
  unsigned hs = 0;
  cudaMemcpyAsync(&hs, tmp.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  tfree(&tmp, work, kGemmWorkBytes + 256, s);
  LV_CUDA(cudaStreamSynchronize(s));
  if (st == LINVIEW_OK && (hs & kStatusTimeout)) st = fail(LINVIEW_ETIMEOUT, "bounded wait expired");
  return st;
}

// ------------------------------------------------------ stand-alone level pass
linview_status linview_level_pass(int precision, int64_t n, void* P, int64_t ldp, const void* U,
                                  const void* V, int64_t ldf, int64_t r, void* X, void* Y,
                                  int do_update, void* stream) {
  if (precision != LINVIEW_F32 && precision != LINVIEW_F64)
    return fail(LINVIEW_EINVAL, "bad precision");
  if (!P || !U || !V) return fail(LINVIEW_EINVAL, "null argument");
  if (n < 1 || r < 1 || r > 64) return fail(LINVIEW_EINVAL, "need n >= 1 and 1 <= r <= 64");
  const int e = precision == LINVIEW_F64 ? 8 : 4;
  if (precision == LINVIEW_F64 && r > 32)
    return fail(LINVIEW_EUNSUPPORTED, "FP64 level pass takes r <= 32");
  if (ldp < n || ldf < n) return fail(LINVIEW_ESHAPE, "ldp/ldf < n");
  if ((ldp * e) % 16 != 0 || (reinterpret_cast<uintptr_t>(P) % 16) != 0)
    return fail(LINVIEW_ESHAPE, "P must be 16-byte aligned with ldp*elem a multiple of 16");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  linview_program tmp;  // borrowed machinery, no views owned
  tmp.elem = e;
  cudaGetDevice(&tmp.device);
  {
    const void* ptrs[5] = {P, U, V, X, Y};
    const char* names[5] = {"P", "U", "V", "X", "Y"};
    for (int i = 0; i < 5; ++i) LV_TRY(check_dev_ptr(ptrs[i], tmp.device, names[i]));
  }
  cudaDeviceGetAttribute(&tmp.sms, cudaDevAttrMultiProcessorCount, tmp.device);
  View v;
  v.ptr = P;
  v.rows = n;
  v.cols = n;
  v.ld = ldp;
  v.square = true;
  if (!make_tmap(&v.tmap, P, e, n, n, ldp)) return fail(LINVIEW_EDEVICE, "tensor map encode failed");
  v.tma_store = (n * e) % 16 == 0;
  const PassGeom g = fused_geom(e, (int)n, tmp.sms);
  tmp.fs = ldf;
  tmp.part_cs = rup(n, 64);
  tmp.xp_s = r * tmp.part_cs;
  tmp.yp_q = r * tmp.part_cs;
  const bool products = (X != nullptr) || (Y != nullptr);
  // FP32 blocks wider than 16 columns: the tensor-core products pass (its own
  // K parts, up to kTpMaxParts partial sets)
  const bool tp = e == 4 && products && r > kMaxProductR && ldf % 64 == 0;
  tmp.xslots = tp && g.gC < kTpMaxParts ? kTpMaxParts : g.gC;
  tmp.yslots = tp && g.gR < kTpMaxParts ? kTpMaxParts : g.gR;
  // the call's temporaries, returned in stream order on every exit path
  struct Temps {
    cudaStream_t s;
    std::vector<void*> ptrs;
    ~Temps() {
      for (void* q : ptrs) cudaFreeAsync(q, s);
    }
  } temps{s, {}};
  auto talloc_s = [&](void** out, size_t bytes) {
    const cudaError_t ce = cudaMallocAsync(out, bytes, s);
    if (ce == cudaSuccess) temps.ptrs.push_back(*out);
    return ce;
  };
  void* xp = nullptr;
  void* yp = nullptr;
  void* stw = nullptr;
  void* tpf = nullptr;
  if (products) {
    LV_CUDA(talloc_s(&xp, (size_t)tmp.xslots * tmp.xp_s * e));
    LV_CUDA(talloc_s(&yp, (size_t)tmp.yslots * tmp.yp_q * e));
  }
  if (tp) {
    LV_CUDA(talloc_s(&tpf, sizeof(float) * 128 * ldf));
    tmp.tpF = static_cast<float*>(tpf);
  }
  LV_CUDA(talloc_s(&stw, sizeof(unsigned) * 4));
  LV_CUDA(cudaMemsetAsync(stw, 0, sizeof(unsigned) * 4, s));
  tmp.status = static_cast<unsigned*>(stw);
  void* tcs = nullptr;  // split factors of the tensor-core update pass (FP32, r > 16)
  if (e == 4 && do_update && r > kMaxProductR) {
    LV_CUDA(talloc_s(&tcs, (size_t)tc_split_floats(n) * sizeof(float)));
    tmp.tcA = static_cast<float*>(tcs);
    tmp.tcB = tmp.tcA + tc_split_floats(n) / 2;
    if (!make_tmap_sw128(&tmp.tmA, tmp.tcA, 128, n, 128, 128) ||
        !make_tmap_sw128(&tmp.tmB, tmp.tcB, 128, n, 128, 32) ||
        !make_tmap_sw128(&v.tmap_tc, P, n, n, ldp, 128))
      return fail(LINVIEW_EDEVICE, "tensor map encode failed");
  }
  tmp.Xpart = xp;
  tmp.Ypart = yp;
  linview_status st = LINVIEW_OK;
  if (e == 4) {
    const float* u = static_cast<const float*>(U);
    const float* vv = static_cast<const float*>(V);
    if (products)
      st = run_products_update<float>(&tmp, v, (int)r, u, vv, do_update ? u : nullptr,
                                      do_update ? vv : nullptr, s, nullptr, /*allow_tc=*/tp);
    else if (do_update)
      st = run_update<float>(&tmp, v, u, vv, (int)r, s);
    if (st == LINVIEW_OK && X)
      st = launch_sum_partials<float>(static_cast<float*>(xp), tmp.pc_x, tmp.xp_s, tmp.part_cs,
                                      (int)n, (int)r, static_cast<float*>(X), ldf, s) == cudaSuccess
               ? LINVIEW_OK : fail(LINVIEW_EDEVICE, "sum_partials launch failed");
    if (st == LINVIEW_OK && Y)
      st = launch_sum_partials<float>(static_cast<float*>(yp), tmp.pc_y, tmp.yp_q, tmp.part_cs,
                                      (int)n, (int)r, static_cast<float*>(Y), ldf, s) == cudaSuccess
               ? LINVIEW_OK : fail(LINVIEW_EDEVICE, "sum_partials launch failed");
  } else {
    const double* u = static_cast<const double*>(U);
    const double* vv = static_cast<const double*>(V);
    if (products)
      st = run_products_update<double>(&tmp, v, (int)r, u, vv, do_update ? u : nullptr,
                                       do_update ? vv : nullptr, s);
    else if (do_update)
      st = run_update<double>(&tmp, v, u, vv, (int)r, s);
    if (st == LINVIEW_OK && X)
      st = launch_sum_partials<double>(static_cast<double*>(xp), g.gC, tmp.xp_s, tmp.part_cs,
                                       (int)n, (int)r, static_cast<double*>(X), ldf, s) == cudaSuccess
               ? LINVIEW_OK : fail(LINVIEW_EDEVICE, "sum_partials launch failed");
    if (st == LINVIEW_OK && Y)
      st = launch_sum_partials<double>(static_cast<double*>(yp), g.gR, tmp.yp_q, tmp.part_cs,
                                       (int)n, (int)r, static_cast<double*>(Y), ldf, s) == cudaSuccess
               ? LINVIEW_OK : fail(LINVIEW_EDEVICE, "sum_partials launch failed");
  }
  unsigned hs = 0;
  cudaMemcpyAsync(&hs, stw, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  LV_CUDA(cudaStreamSynchronize(s));
  if (st == LINVIEW_OK && (hs & kStatusTimeout)) st = fail(LINVIEW_ETIMEOUT, "bounded wait expired");
  return st;
}

// ------------------------------------------------------------- profiling
linview_status linview_set_profiling(linview_program* p, int enable) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  p->prof = enable != 0;
  return LINVIEW_OK;
}

linview_status linview_reset_stats(linview_program* p) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pool.clear();
  p->ev_recs.clear();
  for (auto& ge : p->graphs) ge.replayed = false;
  p->all_launches = 0;
  return LINVIEW_OK;
}

linview_status linview_pass_stats(linview_program* p, int kernel, int64_t* launches, double* ms,
                                  double* bytes, int64_t* all_launches) {
  if (!p) return fail(LINVIEW_EINVAL, "null program");
  if (kernel < 0 || kernel > 2) return fail(LINVIEW_EINVAL, "bad kernel selector %d", kernel);
  double tot = 0.0, by = 0.0;
  int64_t cnt = 0;
  auto add = [&](const std::vector<linview_program::Rec>& recs) -> linview_status {
    for (auto& rc : recs) {
      if (kernel != 0 && rc.kind != kernel) continue;
      float t = 0.f;
      LV_CUDA(cudaEventSynchronize(rc.e1));
      LV_CUDA(cudaEventElapsedTime(&t, rc.e0, rc.e1));
      tot += t;
      by += rc.bytes;
      ++cnt;
    }
    return LINVIEW_OK;
  };
  LV_TRY(add(p->ev_recs));
  // instrumented graph copies replayed since the reset: their last replay
  for (auto& ge : p->graphs)
    if (ge.instrumented && ge.replayed) LV_TRY(add(ge.recs));
  if (launches) *launches = cnt;
  if (ms) *ms = tot;
  if (bytes) *bytes = by;
  if (all_launches) *all_launches = p->all_launches;
  return LINVIEW_OK;
}

}  // extern "C"
