// Serving many maintained matrix-power programs under a stream of factored
// updates (the linview_server_* calls of linview.h).
//
// One scheduler thread per server issues all GPU work.  Each resident view
// has its own CUDA stream, a pinned staging buffer for its coalesced factors
// and a completion event.  A request that arrives for a view that is idle is
// issued at once if a slot (max_inflight) is free; requests that arrive while
// the view refreshes wait in its queue and leave together as one delta
// [U_1 .. U_m][V_1 .. V_m]^T (Section 3.2: deltas in factored form sum by
// concatenating their factors).  Each refresh is linview_apply_delta on the
// view's stream, i.e. the propagation of Appendix A through the squarings.
// A request of rank above the coalescing cap takes the re-evaluation strategy
// instead (Section 4.2.2: apply the delta, recompute): it and every request
// queued behind it are added to A by update-only level passes, and every view
// of the program is recomputed from the new A (linview_reeval).  A view's
// propagation graphs for ranks 1..r_cap are captured when it is admitted.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "linview.h"

namespace lv {
linview_status lv_set_error(linview_status st, const char* fmt, ...);
}

#define LV_TRY(expr)                 \
  do {                               \
    linview_status s_ = (expr);      \
    if (s_ != LINVIEW_OK) return s_; \
  } while (0)

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int32_t rank = 0;
  int64_t row = -1;          // >= 0: row update dA = e_row v^T (V = v, U unused)
  const float* U = nullptr;  // n x rank row-major, ld = rank
  const float* V = nullptr;
  std::vector<float> own;    // storage when the server copied the factors
  double arrival = 0.0;
};

enum ViewState : int32_t { kWaiting = 0, kResident = 1, kRemoved = 2 };

struct ServedView {
  int32_t id = 0;
  int64_t n = 0;
  int32_t k = 0;
  int32_t state = kWaiting;
  bool removing = false;
  int64_t bytes = 0;                // device bytes of the program
  linview_program* prog = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* pin = nullptr;             // pinned [U | V] staging, 2 x n x r_cap floats
  std::vector<float> A_host;        // the input while waiting for admission
  std::deque<Request> queue;
  // the refresh in flight
  bool busy = false;
  std::vector<Request> batch;
  std::vector<int64_t> batch_rows;  // distinct rows of the batch's row updates
  int32_t batch_rank = 0;
  bool batch_reeval = false;        // the batch is served by re-evaluation
  double start = 0.0;
};

}  // namespace

struct linview_server {
  int device = 0;
  int32_t max_inflight = 1;
  int32_t r_cap = 1;
  int64_t budget = 0;
  int64_t used = 0;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable work_cv;  // scheduler: new requests / views / removals
  std::condition_variable done_cv;  // drain: completions
  std::vector<std::unique_ptr<ServedView>> views;
  std::deque<linview_completion> completions;
  uint64_t next_ticket = 1;
  int32_t inflight = 0;
  linview_server_stats st{};
  std::atomic<bool> stop{false};
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(Clock::now() - t0).count();
  }
};

namespace {

linview_status set_err(linview_status s, const char* msg) { return lv::lv_set_error(s, "%s", msg); }

linview_program_desc power_desc(int64_t n, int32_t k, int32_t r_cap) {
  linview_program_desc d{};
  d.kind = LINVIEW_POWER;
  d.precision = LINVIEW_F32;
  d.n = n;
  d.k = k;
  d.r_max = r_cap;
  d.correction_period = 0;
  d.reeval_mode = LINVIEW_REEVAL_DEFAULT;
  return d;
}

// Free device memory that may still be promised to new views.
int64_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return (int64_t)fr;
}

constexpr int64_t kReserveBytes = int64_t(1) << 30;

// Create the program of view v from host or device input (on the calling
// thread); returns the status.  The view's stream and event exist already.
linview_status create_view_program(linview_server* s, ServedView* v, const void* A, int64_t lda,
                                   int on_device) {
  const linview_program_desc d = power_desc(v->n, v->k, s->r_cap);
  const void* inputs[1] = {A};
  const int64_t lds[1] = {lda};
  linview_program* prog = nullptr;
  linview_status st = linview_create_program(&d, inputs, lds, on_device, v->stream, &prog);
  if (st != LINVIEW_OK) return st;
  if (cudaStreamSynchronize(v->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    linview_destroy(prog);
    return set_err(LINVIEW_EDEVICE, "view creation failed on the device");
  }
  // every coalesced rank the view can see, captured now rather than by the
  // first request of each rank
  st = linview_prepare_updates(prog, s->r_cap, v->stream);
  if (st != LINVIEW_OK) {
    linview_destroy(prog);
    return st;
  }
  v->prog = prog;
  return LINVIEW_OK;
}

void complete_batch(linview_server* s, ServedView* v, int32_t status, double t) {
  for (Request& r : v->batch) {
    linview_completion c{};
    c.ticket = r.ticket;
    c.view = v->id;
    c.rank = r.rank;
    c.batch_rank = v->batch_rank;
    c.batch_size = (int32_t)v->batch.size();
    c.status = status;
    c.arrival_s = r.arrival;
    c.start_s = v->start;
    c.done_s = t;
    s->completions.push_back(c);
    s->st.completed++;
    if (status != LINVIEW_OK) s->st.failed++;
  }
  v->batch.clear();
  v->busy = false;
  s->inflight--;
}

void cancel_queue(linview_server* s, ServedView* v, double t) {
  for (Request& r : v->queue) {
    linview_completion c{};
    c.ticket = r.ticket;
    c.view = v->id;
    c.rank = r.rank;
    c.status = LINVIEW_EINVAL;
    c.arrival_s = r.arrival;
    c.start_s = t;
    c.done_s = t;
    s->completions.push_back(c);
    s->st.completed++;
    s->st.failed++;
  }
  v->queue.clear();
}

// Pack the batch's factors into the view's pinned buffer ([U | V], each
// n x R row-major) and issue the refresh; returns the status of the issue.
// The re-evaluation batch: A += sum_j U_j V_j^T by update-only level passes
// of at most 64 columns (the factors of all requests concatenated, column-major
// in a stream-ordered device buffer), then every view recomputed from A.
linview_status issue_reeval_batch(linview_server* s, ServedView* v) {
  const int64_t n = v->n;
  const int64_t ldf = (n + 63) / 64 * 64;
  int64_t R = 0;
  for (const Request& r : v->batch) R += r.rank;
  std::vector<float> host((size_t)2 * ldf * R, 0.f);  // U columns, then V columns
  float* hu = host.data();
  float* hv = host.data() + (size_t)ldf * R;
  int64_t c0 = 0;
  for (const Request& r : v->batch) {
    if (r.row >= 0) {
      hu[c0 * ldf + r.row] = 1.f;
      std::memcpy(hv + c0 * ldf, r.V, sizeof(float) * n);
    } else {
      for (int64_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < r.rank; ++c) {
          hu[(c0 + c) * ldf + i] = r.U[i * r.rank + c];
          hv[(c0 + c) * ldf + i] = r.V[i * r.rank + c];
        }
    }
    c0 += r.rank;
  }
  void* A = nullptr;
  int64_t lda = 0;
  LV_TRY(linview_view_device_ptr(v->prog, 0, &A, &lda));
  float* d = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), host.size() * sizeof(float), v->stream) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return set_err(LINVIEW_ENOMEM, "no device memory for the re-evaluation batch's factors");
  }
  linview_status st = LINVIEW_OK;
  if (cudaMemcpyAsync(d, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice,
                      v->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    st = set_err(LINVIEW_EDEVICE, "factor copy failed");
  }
  for (int64_t b = 0; b < R && st == LINVIEW_OK; b += 64) {
    const int64_t w = R - b < 64 ? R - b : 64;
    st = linview_level_pass(LINVIEW_F32, n, A, lda, d + b * ldf, d + (R + b) * ldf, ldf, w,
                            nullptr, nullptr, 1, v->stream);
  }
  // (a copy from pageable memory has been staged when cudaMemcpyAsync
  // returns, so ``host`` may go now)
  if (cudaFreeAsync(d, v->stream) != cudaSuccess) (void)cudaGetLastError();
  if (st != LINVIEW_OK) return st;
  LV_TRY(linview_reeval(v->prog, v->stream));
  if (cudaEventRecord(v->done, v->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return set_err(LINVIEW_EDEVICE, "cudaEventRecord failed");
  }
  return LINVIEW_OK;
}

linview_status issue_batch(linview_server* s, ServedView* v) {
  if (v->batch_reeval) return issue_reeval_batch(s, v);
  const int64_t n = v->n;
  const int R = v->batch_rank;
  float* U = v->pin;
  float* V = v->pin + (size_t)n * R;
  int c0 = 0;
  for (const Request& r : v->batch) {
    if (r.row >= 0) continue;
    const int rk = r.rank;
    for (int64_t i = 0; i < n; ++i) {
      std::memcpy(U + i * R + c0, r.U + i * rk, sizeof(float) * rk);
      std::memcpy(V + i * R + c0, r.V + i * rk, sizeof(float) * rk);
    }
    c0 += rk;
  }
  // one column per distinct row: U = e_row, V = the sum of its v's in arrival order
  for (const int64_t row : v->batch_rows) {
    for (int64_t i = 0; i < n; ++i) {
      U[i * R + c0] = 0.f;
      V[i * R + c0] = 0.f;
    }
    U[row * R + c0] = 1.f;
    for (const Request& r : v->batch) {
      if (r.row != row) continue;
      for (int64_t i = 0; i < n; ++i) V[i * R + c0] += r.V[i];
    }
    ++c0;
  }
  linview_status st = linview_apply_delta(v->prog, 0, R, U, R, V, R, 0, v->stream);
  if (st != LINVIEW_OK) return st;
  if (cudaEventRecord(v->done, v->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return set_err(LINVIEW_EDEVICE, "cudaEventRecord failed");
  }
  return LINVIEW_OK;
}

void release_view(ServedView* v) {
  if (v->prog) linview_destroy(v->prog);
  v->prog = nullptr;
  if (v->done) cudaEventDestroy(v->done);
  v->done = nullptr;
  if (v->stream) cudaStreamDestroy(v->stream);
  v->stream = nullptr;
  if (v->pin) cudaFreeHost(v->pin);
  v->pin = nullptr;
  v->A_host.clear();
  v->A_host.shrink_to_fit();
}

// The scheduler: completions, removals, admissions, then new refreshes in
// order of the oldest waiting request.
void scheduler(linview_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    const double t = s->now();
    // 1. refreshes that finished
    for (auto& vp : s->views) {
      ServedView* v = vp.get();
      if (!v->busy) continue;
      const cudaError_t e = cudaEventQuery(v->done);
      if (e == cudaErrorNotReady) continue;
      int32_t status = LINVIEW_OK;
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        status = LINVIEW_EDEVICE;
      }
      complete_batch(s, v, status, s->now());
      progressed = true;
    }
    if (progressed) s->done_cv.notify_all();
    if (s->stop.load() && s->inflight == 0) break;
    // 2. removals (program destroyed outside the lock).  Views are visited
    // by index: add_view may append while the lock is released.
    for (size_t iv = 0; iv < s->views.size(); ++iv) {
      ServedView* v = s->views[iv].get();
      if (!v->removing || v->busy || v->state == kRemoved) continue;
      cancel_queue(s, v, t);
      const bool was_resident = v->state == kResident;
      lk.unlock();
      release_view(v);
      lk.lock();
      if (was_resident) {
        s->used -= v->bytes;
        s->st.views_resident--;
      } else {
        s->st.views_waiting--;
      }
      v->state = kRemoved;
      progressed = true;
      s->done_cv.notify_all();
    }
    // 3. admissions of waiting views, in id order
    for (size_t iv = 0; iv < s->views.size(); ++iv) {
      ServedView* v = s->views[iv].get();
      if (v->state != kWaiting || v->removing || s->stop.load()) continue;
      if (s->used + v->bytes > s->budget || v->bytes + kReserveBytes > free_device_bytes()) break;
      s->used += v->bytes;
      lk.unlock();
      const linview_status st = create_view_program(s, v, v->A_host.data(), v->n, 0);
      lk.lock();
      if (st == LINVIEW_OK) {
        v->A_host.clear();
        v->A_host.shrink_to_fit();
        v->state = kResident;
        s->st.views_waiting--;
        s->st.views_resident++;
      } else {
        s->used -= v->bytes;  // keep waiting; retried when memory frees up again
        break;
      }
      progressed = true;
    }
    // 4. new refreshes: the idle resident view whose oldest request waited longest
    while (s->inflight < s->max_inflight && !s->stop.load()) {
      ServedView* pick = nullptr;
      for (auto& vp : s->views) {
        ServedView* v = vp.get();
        if (v->state != kResident || v->busy || v->removing || v->queue.empty()) continue;
        if (!pick || v->queue.front().arrival < pick->queue.front().arrival) pick = v;
      }
      if (!pick) break;
      // Take, in arrival order, every queued request that fits the rank cap
      // (the oldest always does).  Row updates to a row already in the batch
      // add no rank: their v's are summed into that row's column
      // (e_i v1^T + e_i v2^T = e_i (v1 + v2)^T).  Deltas add, so a request
      // may join a batch ahead of an older one that did not fit; that one
      // leads the next batch.
      int32_t R = 0;
      std::vector<int64_t>& rows = pick->batch_rows;
      rows.clear();
      std::deque<Request> rest;
      // a request past the rank cap: re-evaluation, which serves every
      // request queued for the view at once
      pick->batch_reeval = pick->queue.front().rank > s->r_cap;
      if (pick->batch_reeval) {
        for (Request& f : pick->queue) {
          R += f.rank;
          pick->batch.push_back(std::move(f));
        }
        pick->queue.clear();
      }
      while (!pick->queue.empty()) {
        Request f = std::move(pick->queue.front());
        pick->queue.pop_front();
        int32_t add = f.rank;
        if (f.row >= 0) add = std::find(rows.begin(), rows.end(), f.row) == rows.end() ? 1 : 0;
        if (R + add > s->r_cap) {
          rest.push_back(std::move(f));
          continue;
        }
        if (f.row >= 0 && add) rows.push_back(f.row);
        R += add;
        pick->batch.push_back(std::move(f));
      }
      pick->queue.swap(rest);
      pick->batch_rank = R;
      pick->busy = true;
      pick->start = s->now();
      s->inflight++;
      s->st.max_inflight_seen = std::max(s->st.max_inflight_seen, s->inflight);
      s->st.refreshes++;
      s->st.coalesced_rank_sum += R;
      if (pick->batch_reeval) s->st.reevals++;
      lk.unlock();
      const linview_status st = issue_batch(s, pick);
      lk.lock();
      if (st != LINVIEW_OK) {
        complete_batch(s, pick, st, s->now());
        s->done_cv.notify_all();
      }
      progressed = true;
    }
    if (progressed) continue;
    if (s->inflight > 0) {
      // poll the completion events closely: latency is measured here
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      if (s->stop.load()) break;
      s->work_cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

}  // namespace

extern "C" {

linview_status linview_server_create(int64_t hbm_budget_bytes, int32_t max_inflight, int32_t r_cap,
                                     linview_server** out) {
  if (!out) return set_err(LINVIEW_EINVAL, "null argument");
  *out = nullptr;
  if (max_inflight < 1) return set_err(LINVIEW_EINVAL, "max_inflight must be >= 1");
  if (r_cap < 1 || r_cap > 128) return set_err(LINVIEW_EINVAL, "r_cap must be in 1..128");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    (void)cudaGetLastError();
    return set_err(LINVIEW_EDEVICE, "no CUDA device");
  }
  auto* s = new linview_server();
  cudaGetDevice(&s->device);
  s->max_inflight = max_inflight;
  s->r_cap = r_cap;
  const int64_t fr = free_device_bytes();
  s->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : std::max<int64_t>(0, fr - kReserveBytes);
  s->st.bytes_budget = s->budget;
  s->t0 = Clock::now();
  s->worker = std::thread(scheduler, s);
  *out = s;
  return LINVIEW_OK;
}

double linview_server_clock(const linview_server* s) { return s ? s->now() : 0.0; }

linview_status linview_server_add_view(linview_server* s, int64_t n, int32_t k, const void* A,
                                       int64_t lda, int on_device, int32_t* view) {
  if (!s || !A || !view) return set_err(LINVIEW_EINVAL, "null argument");
  if (n < 1 || lda < n) return set_err(LINVIEW_ESHAPE, "bad n or lda");
  if (k < 2 || (k & (k - 1)) != 0) return set_err(LINVIEW_EINVAL, "k must be a power of two >= 2");
  if ((int64_t)s->r_cap * k > 128) return set_err(LINVIEW_EUNSUPPORTED, "r_cap * k exceeds 128");
  cudaSetDevice(s->device);
  auto v = std::make_unique<ServedView>();
  v->n = n;
  v->k = k;
  const linview_program_desc d = power_desc(n, k, s->r_cap);
  LV_TRY(linview_estimate_device_bytes(&d, &v->bytes));
  if (cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&v->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void**>(&v->pin), sizeof(float) * 2 * n * s->r_cap,
                    cudaHostAllocDefault) != cudaSuccess) {
    (void)cudaGetLastError();
    release_view(v.get());
    return set_err(LINVIEW_EDEVICE, "stream, event or pinned buffer allocation failed");
  }
  std::unique_lock<std::mutex> lk(s->mu);
  const bool fits = s->used + v->bytes <= s->budget &&
                    v->bytes + kReserveBytes <= free_device_bytes();
  bool waiting_before = false;  // earlier views waiting keep their turn
  for (auto& w : s->views)
    if (w->state == kWaiting && !w->removing) waiting_before = true;
  if (fits && !waiting_before) {
    s->used += v->bytes;
    lk.unlock();
    const linview_status st = create_view_program(s, v.get(), A, lda, on_device);
    lk.lock();
    if (st != LINVIEW_OK) {
      s->used -= v->bytes;
      lk.unlock();
      release_view(v.get());
      return st;
    }
    v->state = kResident;
    s->st.views_resident++;
  } else {
    v->A_host.resize((size_t)n * n);
    lk.unlock();
    const cudaError_t e = cudaMemcpy2D(v->A_host.data(), sizeof(float) * n, A, sizeof(float) * lda,
                                       sizeof(float) * n, n,
                                       on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    lk.lock();
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      lk.unlock();
      release_view(v.get());
      return set_err(LINVIEW_EDEVICE, "copy of the input failed");
    }
    v->state = kWaiting;
    s->st.views_waiting++;
  }
  v->id = (int32_t)s->views.size();
  *view = v->id;
  s->views.push_back(std::move(v));
  s->work_cv.notify_all();
  return LINVIEW_OK;
}

static linview_status enqueue(linview_server* s, int32_t view, Request&& r) {
  if (view < 0 || view >= (int32_t)s->views.size())
    return set_err(LINVIEW_EINVAL, "bad view id");
  ServedView* v = s->views[view].get();
  if (v->state == kRemoved || v->removing) return set_err(LINVIEW_EINVAL, "view was removed");
  r.ticket = s->next_ticket++;
  v->queue.push_back(std::move(r));
  s->st.submitted++;
  return LINVIEW_OK;
}

linview_status linview_server_submit(linview_server* s, int32_t view, int32_t rank, const void* U,
                                     int64_t ldu, const void* V, int64_t ldv, double arrival_s,
                                     uint64_t* ticket) {
  if (!s || !U || !V) return set_err(LINVIEW_EINVAL, "null argument");
  if (rank < 1) return set_err(LINVIEW_ERANK, "rank must be >= 1");
  if (ldu < rank || ldv < rank) return set_err(LINVIEW_ESHAPE, "ldu/ldv < rank");
  int64_t n = 0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (view < 0 || view >= (int32_t)s->views.size())
      return set_err(LINVIEW_EINVAL, "bad view id");
    n = s->views[view]->n;
  }
  if (rank > n) return set_err(LINVIEW_ERANK, "rank must be <= n");
  Request r;
  r.rank = rank;
  r.own.resize((size_t)2 * n * rank);
  const float* u = static_cast<const float*>(U);
  const float* v = static_cast<const float*>(V);
  for (int64_t i = 0; i < n; ++i) {
    std::memcpy(r.own.data() + i * rank, u + i * ldu, sizeof(float) * rank);
    std::memcpy(r.own.data() + (n + i) * rank, v + i * ldv, sizeof(float) * rank);
  }
  r.U = r.own.data();
  r.V = r.own.data() + (size_t)n * rank;
  std::lock_guard<std::mutex> g(s->mu);
  r.arrival = arrival_s >= 0 ? arrival_s : s->now();
  const uint64_t tk = s->next_ticket;
  LV_TRY(enqueue(s, view, std::move(r)));
  if (ticket) *ticket = tk;
  s->work_cv.notify_all();
  return LINVIEW_OK;
}

linview_status linview_server_submit_row(linview_server* s, int32_t view, int64_t row,
                                         const void* v, double arrival_s, uint64_t* ticket) {
  if (!s || !v) return set_err(LINVIEW_EINVAL, "null argument");
  int64_t n = 0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (view < 0 || view >= (int32_t)s->views.size())
      return set_err(LINVIEW_EINVAL, "bad view id");
    n = s->views[view]->n;
  }
  if (row < 0 || row >= n) return set_err(LINVIEW_EINVAL, "row out of range");
  Request r;
  r.rank = 1;
  r.row = row;
  r.own.assign(static_cast<const float*>(v), static_cast<const float*>(v) + n);
  r.V = r.own.data();
  std::lock_guard<std::mutex> g(s->mu);
  r.arrival = arrival_s >= 0 ? arrival_s : s->now();
  const uint64_t tk = s->next_ticket;
  LV_TRY(enqueue(s, view, std::move(r)));
  if (ticket) *ticket = tk;
  s->work_cv.notify_all();
  return LINVIEW_OK;
}

linview_status linview_server_replay(linview_server* s, int64_t count, const double* t_s,
                                     const int32_t* view, const int32_t* rank, const void* factors,
                                     const int64_t* offset, const int64_t* rows) {
  if (!s || (count > 0 && (!t_s || !view || !rank || !factors || !offset)))
    return set_err(LINVIEW_EINVAL, "null argument");
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (int64_t i = 0; i < count; ++i) {
      if (view[i] < 0 || view[i] >= (int32_t)s->views.size())
        return set_err(LINVIEW_EINVAL, "bad view id in the trace");
      if (rows && rows[i] >= s->views[view[i]]->n)
        return set_err(LINVIEW_EINVAL, "row out of range in the trace");
      if (!(rows && rows[i] >= 0) && (rank[i] < 1 || rank[i] > s->views[view[i]]->n))
        return set_err(LINVIEW_ERANK, "rank outside 1..n");
      if (i > 0 && t_s[i] < t_s[i - 1]) return set_err(LINVIEW_EINVAL, "t_s must be non-decreasing");
    }
  }
  const float* f = static_cast<const float*>(factors);
  const double t0 = s->now();
  for (int64_t i = 0; i < count; ++i) {
    const double due = t0 + t_s[i];
    for (;;) {  // sleep while far from the arrival, then spin
      const double wait = due - s->now();
      if (wait <= 0) break;
      if (wait > 2e-4)
        std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
      else
        std::this_thread::yield();
    }
    Request r;
    std::lock_guard<std::mutex> g(s->mu);
    const int64_t n = s->views[view[i]]->n;
    if (rows && rows[i] >= 0) {
      r.rank = 1;
      r.row = rows[i];
      r.V = f + offset[i];
    } else {
      r.rank = rank[i];
      r.U = f + offset[i];
      r.V = r.U + n * r.rank;
    }
    r.arrival = due;
    LV_TRY(enqueue(s, view[i], std::move(r)));
    s->work_cv.notify_all();
  }
  return LINVIEW_OK;
}

linview_status linview_server_poll(linview_server* s, linview_completion* out, int32_t max,
                                   int32_t* count) {
  if (!s || !count || (max > 0 && !out)) return set_err(LINVIEW_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  int32_t c = 0;
  while (c < max && !s->completions.empty()) {
    out[c++] = s->completions.front();
    s->completions.pop_front();
  }
  *count = c;
  return LINVIEW_OK;
}

linview_status linview_server_drain(linview_server* s, double timeout_s) {
  if (!s) return set_err(LINVIEW_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto all_done = [s] {
    if (s->st.completed < s->st.submitted) return false;
    for (auto& v : s->views)
      if (v->removing && v->state != kRemoved) return false;
    return true;
  };
  if (timeout_s <= 0) {
    s->done_cv.wait(lk, all_done);
    return LINVIEW_OK;
  }
  if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), all_done))
    return set_err(LINVIEW_ETIMEOUT, "requests still pending after the timeout");
  return LINVIEW_OK;
}

linview_status linview_server_view_state(linview_server* s, int32_t view, int32_t* state) {
  if (!s || !state) return set_err(LINVIEW_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  if (view < 0 || view >= (int32_t)s->views.size()) return set_err(LINVIEW_EINVAL, "bad view id");
  *state = s->views[view]->state;
  return LINVIEW_OK;
}

linview_status linview_server_view_program(linview_server* s, int32_t view,
                                           linview_program** prog) {
  if (!s || !prog) return set_err(LINVIEW_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  if (view < 0 || view >= (int32_t)s->views.size()) return set_err(LINVIEW_EINVAL, "bad view id");
  ServedView* v = s->views[view].get();
  if (v->state != kResident || v->removing) return set_err(LINVIEW_EINVAL, "view is not resident");
  *prog = v->prog;
  return LINVIEW_OK;
}

linview_status linview_server_remove_view(linview_server* s, int32_t view) {
  if (!s) return set_err(LINVIEW_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  if (view < 0 || view >= (int32_t)s->views.size()) return set_err(LINVIEW_EINVAL, "bad view id");
  ServedView* v = s->views[view].get();
  if (v->state == kRemoved || v->removing) return set_err(LINVIEW_EINVAL, "view already removed");
  v->removing = true;
  s->work_cv.notify_all();
  return LINVIEW_OK;
}

linview_status linview_server_stats_get(linview_server* s, linview_server_stats* out) {
  if (!s || !out) return set_err(LINVIEW_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  s->st.bytes_used = s->used;
  *out = s->st;
  return LINVIEW_OK;
}

void linview_server_destroy(linview_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop.store(true);
    s->work_cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& v : s->views) release_view(v.get());
  delete s;
}

}  // extern "C"
