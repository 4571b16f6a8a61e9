// linview_level_pass_noalloc: the stand-alone level pass for callers that
// are not allowed to allocate device memory.
//
// Who needs it: code that runs where the device memory has already been
// handed out -- a serving process or an inference-engine plugin that reserves
// the whole GPU up front and forbids allocation on its enqueue path, or a
// latency-critical loop that cannot afford the implicit device-wide
// synchronisation a cudaMalloc/cudaFree may cause.  linview_level_pass gets
// its cross-block partial sums from the stream-ordered allocator; this
// variant takes them from one fixed array compiled into the library instead.
// It launches the CUDA-core products passes (FP32 in blocks of 16 columns,
// FP64 in blocks of 8) and partial-sum reductions of the allocating entry.
// One difference: FP32 blocks wider than 16 columns run on the CUDA-core
// passes here (products in blocks of 16, updates in blocks of 32), where the
// allocating entry splits the factors into scratch buffers for the
// tensor-core products and update passes; both are FP32-accurate, so those
// results agree within FP32 rounding, not bit for bit.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes
// (16 MiB).  Under CUDA's lazy module loading it is reserved on a device once
// the library's kernels are first used there, and stays reserved until the
// process exits.  Host code cannot use the variable's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it per device;
// make that first call before any stream capture begins.  All calls share
// the array and it keeps whatever the last call left in it, so two calls
// whose work overlaps on the GPU (e.g. on two streams) race on it: serialise
// them.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/linview.h"
#include "lv_device.cuh"
#include "lv_internal.h"

namespace lv {
// sets the thread-local message returned by linview_last_error (lv_capi.cu)
linview_status lv_set_error(linview_status st, const char* fmt, ...);
// EINVAL unless a non-null ``ptr`` is device or managed memory of ``device``
// (lv_capi.cu)
linview_status check_dev_ptr(const void* ptr, int device, const char* name);
}  // namespace lv

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr size_t kStatusBytes = 256;  // device status word, padded to the array's alignment
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device with that device current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int64_t rup64(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// The allocating entry point's launch sequence: one fused products + update
// pass up to kMaxFusedR columns, else products-only passes in blocks of
// kMaxProductR (FP32) or kMaxFusedR (FP64) columns and update-only passes of
// up to kMaxUpdateR columns, then the fixed-order sums of the partials into X
// and Y.
template <typename T>
cudaError_t run(lv::PassParams base, const CUtensorMap& tm, int n, int r, int sms, const T* U,
                const T* V, T* X, T* Y, bool do_update, cudaStream_t s) {
  using namespace lv;
  const bool products = (X != nullptr) || (Y != nullptr);
  const PassGeom g = fused_geom(sizeof(T), n, sms);
  cudaError_t e = cudaSuccess;
  if (products) {
    base.gC = g.gC;
    base.gR = g.gR;
    base.rows_per_cta = g.rows_per_cta;
    if (r <= kMaxFusedR) {
      PassParams pp = base;
      pp.Xf = U;
      pp.Yf = V;
      pp.Uu = do_update ? U : nullptr;
      pp.Wu = do_update ? V : nullptr;
      pp.r = r;
      e = launch_fused<T>(pp, tm, r, do_update ? kModeXYU : kModeXY, s);
      if (e != cudaSuccess) return e;
      do_update = false;
    } else {
      constexpr int MW = sizeof(T) == 4 ? kMaxProductR : kMaxFusedR;
      for (int c0 = 0; c0 < r; c0 += MW) {
        const int w = (r - c0 < MW) ? (r - c0) : MW;
        PassParams pp = base;
        pp.Xf = U + (int64_t)c0 * base.fs;
        pp.Yf = V + (int64_t)c0 * base.fs;
        pp.r = w;
        pp.Xpart = static_cast<T*>(base.Xpart) + (int64_t)c0 * base.part_cs;
        pp.Ypart = static_cast<T*>(base.Ypart) + (int64_t)c0 * base.part_cs;
        e = launch_fused<T>(pp, tm, w, kModeXY, s);
        if (e != cudaSuccess) return e;
      }
    }
  }
  if (do_update) {
    const int MU = kMaxUpdateR;
    for (int c0 = 0; c0 < r; c0 += MU) {
      const int w = (r - c0 < MU) ? (r - c0) : MU;
      const PassGeom gu = update_geom(sizeof(T), w, n, sms);
      PassParams pp = base;
      pp.Xf = nullptr;
      pp.Yf = nullptr;
      pp.Uu = U + (int64_t)c0 * base.fs;
      pp.Wu = V + (int64_t)c0 * base.fs;
      pp.r = w;
      pp.gC = gu.gC;
      pp.gR = gu.gR;
      pp.rows_per_cta = gu.rows_per_cta;
      // a block after the first follows a pass that wrote this view
      e = launch_update<T>(pp, tm, w, s, /*programmatic=*/c0 == 0);
      if (e != cudaSuccess) return e;
    }
  }
  if (X) {
    e = launch_sum_partials<T>(static_cast<const T*>(base.Xpart), g.gC, base.xp_s, base.part_cs,
                               n, r, X, base.fs, s);
    if (e != cudaSuccess) return e;
  }
  if (Y)
    e = launch_sum_partials<T>(static_cast<const T*>(base.Ypart), g.gR, base.yp_q, base.part_cs, n,
                               r, Y, base.fs, s);
  return e;
}

}  // namespace

extern "C" linview_status linview_level_pass_noalloc(int precision, int64_t n, void* P,
                                                     int64_t ldp, const void* U, const void* V,
                                                     int64_t ldf, int64_t r, void* X, void* Y,
                                                     int do_update, void* stream) {
  using namespace lv;
  if (precision != LINVIEW_F32 && precision != LINVIEW_F64)
    return lv_set_error(LINVIEW_EINVAL, "bad precision");
  if (!P || !U || !V) return lv_set_error(LINVIEW_EINVAL, "null argument");
  if (n < 1 || r < 1 || r > 64) return lv_set_error(LINVIEW_EINVAL, "need n >= 1 and 1 <= r <= 64");
  const int e = precision == LINVIEW_F64 ? 8 : 4;
  if (e == 8 && r > 32) return lv_set_error(LINVIEW_EUNSUPPORTED, "FP64 level pass takes r <= 32");
  if (ldp < n || ldf < n) return lv_set_error(LINVIEW_ESHAPE, "ldp/ldf < n");
  if ((ldp * e) % 16 != 0 || (reinterpret_cast<uintptr_t>(P) % 16) != 0)
    return lv_set_error(LINVIEW_ESHAPE, "P must be 16-byte aligned with ldp*elem a multiple of 16");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return lv_set_error(LINVIEW_EDEVICE, "no CUDA device");
  }
  {
    const void* ptrs[5] = {P, U, V, X, Y};
    const char* names[5] = {"P", "U", "V", "X", "Y"};
    for (int i = 0; i < 5; ++i) {
      const linview_status st = check_dev_ptr(ptrs[i], dev, names[i]);
      if (st != LINVIEW_OK) return st;
    }
  }
  // scratch layout: [status word | row-sum partials | column-sum partials]
  const PassGeom g = fused_geom(e, (int)n, sms);
  const int64_t part_cs = rup64(n, 64);
  const bool products = (X != nullptr) || (Y != nullptr);
  const size_t xbytes = products ? (size_t)g.gC * r * part_cs * e : 0;
  const size_t ybytes = products ? (size_t)g.gR * r * part_cs * e : 0;
  const size_t need = kStatusBytes + rup64((int64_t)xbytes, 256) + ybytes;
  if (need > kNoAllocScratchBytes)
    return lv_set_error(LINVIEW_ESHAPE,
                        "n=%lld, r=%lld needs %zu bytes of scratch; the built-in array holds %zu",
                        (long long)n, (long long)r, need, kNoAllocScratchBytes);
  void* scratch = nullptr;
  cudaError_t ce = scratch_address(&scratch);
  if (ce != cudaSuccess)
    return lv_set_error(LINVIEW_EDEVICE, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(ce));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* status = static_cast<unsigned*>(scratch);
  ce = cudaMemsetAsync(status, 0, sizeof(unsigned), s);  // the status word must start at zero
  if (ce != cudaSuccess)
    return lv_set_error(LINVIEW_EDEVICE, "cudaMemsetAsync failed: %s", cudaGetErrorString(ce));
  CUtensorMap tm;
  if (!make_tmap(&tm, P, e, n, n, ldp)) return lv_set_error(LINVIEW_EDEVICE, "tensor map encode failed");
  PassParams base{};
  base.P = P;
  base.ldp = ldp;
  base.n = (int)n;
  base.fs = ldf;
  base.part_cs = part_cs;
  base.xp_s = r * part_cs;
  base.yp_q = r * part_cs;
  base.Xpart = static_cast<char*>(scratch) + kStatusBytes;
  base.Ypart = static_cast<char*>(base.Xpart) + rup64((int64_t)xbytes, 256);
  base.status = status;
  base.tma_store = (n * e) % 16 == 0 ? 1 : 0;
  if (e == 4)
    ce = run<float>(base, tm, (int)n, (int)r, sms, static_cast<const float*>(U),
                    static_cast<const float*>(V), static_cast<float*>(X), static_cast<float*>(Y),
                    do_update != 0, s);
  else
    ce = run<double>(base, tm, (int)n, (int)r, sms, static_cast<const double*>(U),
                     static_cast<const double*>(V), static_cast<double*>(X),
                     static_cast<double*>(Y), do_update != 0, s);
  if (ce != cudaSuccess)
    return lv_set_error(LINVIEW_EDEVICE, "kernel launch failed: %s", cudaGetErrorString(ce));
  unsigned hs = 0;
  ce = cudaMemcpyAsync(&hs, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess)
    return lv_set_error(LINVIEW_EDEVICE, "status read failed: %s", cudaGetErrorString(ce));
  if (hs & kStatusTimeout) return lv_set_error(LINVIEW_ETIMEOUT, "bounded wait expired");
  return LINVIEW_OK;
}
