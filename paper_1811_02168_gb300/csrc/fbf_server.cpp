// Serving loop: continuous batching of filter requests under an HBM budget.
//
// Requests (a host image, theta, sigma, K or eps) arrive at any time from any thread.  One
// worker thread per server runs the loop:
//   admission  in arrival order, while the request's device buffers (input and output,
//              8 B per pixel) fit the HBM budget and the next launch has room; buffers come
//              from the server's own stream-ordered memory pool and the image is copied in
//              at once on the upload stream;
//   launch     whenever fewer than max_inflight launches are in flight, everything admitted
//              so far goes into one batched launch (fbf_batch_submit / fbf_launch: one persistent
//              stream-K kernel per precision form and radius class) on the compute stream,
//              after the uploads it needs (events); requests that arrive meanwhile join the
//              next launch instead of waiting for a fixed batch;
//   results    the download stream waits for the launch, copies every result to its host
//              buffer and frees the device buffers (stream-ordered); an event per launch
//              marks completion, which the worker polls and turns into per-request status,
//              latency (submit -> result on the host) and released budget.
// Uploads and downloads run on separate streams, so admission never waits for a launch.
// Nothing here is in the paper (Section III filters one image at a time); the arithmetic
// per request is exactly fbf_filter's.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "fbf.h"
#include "fbf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Req {
  fbf_ticket_t id = 0;
  const float* host_in = nullptr;
  float* host_out = nullptr;
  int H = 0, W = 0;
  fbf_plan_t plan = nullptr;
  uint64_t bytes = 0;             // device bytes held while admitted
  double t_submit = 0, t_admit = 0, t_launch = 0;
  float* d_in = nullptr;
  float* d_out = nullptr;
  cudaEvent_t up = nullptr;       // upload complete
  int batch = 0;                  // requests in its launch
  bool deferred = false;          // counted once in waited_for_budget
  bool released = false;          // its device buffers' frees are enqueued
};

struct Launch {
  std::vector<Req*> reqs;
  cudaEvent_t done = nullptr;     // results on the host, device buffers released
};

using PlanKey = std::tuple<double, int, double, int, double>;   // sigma, R, theta, K, eps

// the slowest requests: mean of each latency part over the requests at or above q
struct Tail {
  double n = 0, queued = 0, wait = 0, l2r = 0, mpix = 0, batch = 0;
};

}  // namespace

struct fbf_server_s {
  int device = 0, precision = 0, max_batch = 1, max_inflight = 1;
  uint64_t budget = 0;
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  cudaMemPool_t pool = nullptr;
  fbf_batch_t batch = nullptr;

  std::mutex mu;                  // guards every member below
  std::condition_variable work;   // a submit or stop for the worker
  std::condition_variable idle;   // a completion for fbf_server_drain
  std::map<PlanKey, fbf_plan_t> plans;
  std::deque<Req*> waiting;       // submitted, not admitted
  std::unordered_map<fbf_ticket_t, int> status;
  fbf_ticket_t next_id = 1;
  uint64_t pending = 0;           // submitted and not finished
  bool stop = false;
  // worker state
  std::vector<Req*> admitted;
  std::deque<Launch> inflight;
  uint64_t used = 0;
  // statistics
  uint64_t requests = 0, pixels = 0, launches = 0, failed = 0, high_water = 0, waited = 0;
  uint32_t max_inflight_seen = 0;
  double t_first = -1, t_last = -1;
  std::vector<std::array<double, 6>> trace;   // latency, queued, wait, launch->result, px, batch
  std::thread worker;
  // test hook (fbf_debug_server_inject): uploads / launches still to fail on the host
  std::atomic<int> inject_upload{0}, inject_launch{0};
};

namespace {

// one injected failure of a stage, if any is left (test hook)
bool take_injected(std::atomic<int>& n) {
  int v = n.load();
  while (v > 0)
    if (n.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

// After a failed upload or launch: wait (best effort) for the copies and kernels that may
// still use a request's buffers, then give the buffers back to the pool (called without
// the lock).
void release_after_error(fbf_server_s* s, const std::vector<Req*>& reqs) {
  cudaStreamSynchronize(s->up);
  cudaStreamSynchronize(s->comp);
  cudaStreamSynchronize(s->down);
  for (Req* r : reqs) {
    if (r->released) continue;
    if (r->d_in) cudaFreeAsync(r->d_in, s->down);
    if (r->d_out) cudaFreeAsync(r->d_out, s->down);
    r->d_in = r->d_out = nullptr;
    r->released = true;
  }
  cudaStreamSynchronize(s->down);
}

// Device buffers and the upload of one admitted request (called without the lock).
int upload(fbf_server_s* s, Req* r) {
  const fbf::NvtxRange tr("fbf_server admit: upload");
  if (take_injected(s->inject_upload)) {
    const int rc = fbf::set_error(FBF_ECUDA, "fbf_server: upload: injected failure");
    release_after_error(s, {r});
    return rc;
  }
  const size_t n = (size_t)r->H * r->W * sizeof(float);
  void* a = nullptr;
  void* b = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&a, n, s->pool, s->up);
  if (e == cudaSuccess) r->d_in = static_cast<float*>(a);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&b, n, s->pool, s->up);
  if (e == cudaSuccess) r->d_out = static_cast<float*>(b);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_in, r->host_in, n, cudaMemcpyHostToDevice, s->up);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->up, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->up, s->up);
  if (e != cudaSuccess) {
    const int rc = fbf::set_error(FBF_ECUDA, std::string("fbf_server: upload: ") + cudaGetErrorString(e));
    release_after_error(s, {r});
    return rc;
  }
  return FBF_OK;
}

// One batched launch of the admitted requests, the downloads and the releases behind it
// (called without the lock).
int launch(fbf_server_s* s, Launch& L) {
  const fbf::NvtxRange tr("fbf_server launch");
  cudaError_t e = cudaSuccess;
  for (Req* r : L.reqs) {
    e = cudaStreamWaitEvent(s->comp, r->up, 0);
    if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_server: ") + cudaGetErrorString(e));
    const int rc = fbf_batch_submit(s->batch, r->plan, r->d_in, r->d_out, r->H, r->W, (size_t)r->W, nullptr);
    if (rc != FBF_OK) return rc;
  }
  // test hook: fail with the images queued in the batch, as a failing submit would leave them
  if (take_injected(s->inject_launch)) return fbf::set_error(FBF_ECUDA, "fbf_server: launch: injected failure");
  int rc = fbf_launch(s->batch, s->comp);
  if (rc != FBF_OK) return rc;
  cudaEvent_t kd = nullptr;
  e = cudaEventCreateWithFlags(&kd, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(kd, s->comp);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->down, kd, 0);
  if (kd) cudaEventDestroy(kd);
  for (Req* r : L.reqs) {
    if (e != cudaSuccess) break;
    const size_t n = (size_t)r->H * r->W * sizeof(float);
    e = cudaMemcpyAsync(r->host_out, r->d_out, n, cudaMemcpyDeviceToHost, s->down);
    if (e == cudaSuccess) e = cudaFreeAsync(r->d_in, s->down);
    if (e == cudaSuccess) r->d_in = nullptr;
    if (e == cudaSuccess) e = cudaFreeAsync(r->d_out, s->down);
    if (e == cudaSuccess) {
      r->d_out = nullptr;
      r->released = true;
    }
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, s->down);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_server: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

// Retire one request (lock held).
void retire(fbf_server_s* s, Req* r, int st, double t) {
  s->status[r->id] = st;
  s->used -= r->bytes;
  if (st == FBF_DONE) {
    ++s->requests;
    s->pixels += (uint64_t)r->H * r->W;
    s->trace.push_back({t - r->t_submit, r->t_admit - r->t_submit, r->t_launch - r->t_admit, t - r->t_launch,
                        (double)r->H * r->W, (double)r->batch});
  } else {
    ++s->failed;
  }
  s->t_last = t;
  if (r->up) cudaEventDestroy(r->up);
  delete r;
  --s->pending;
}

void worker_main(fbf_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool busy = false;
    // admission: arrival order, HBM budget, room in the next launch
    while (!s->waiting.empty() && (int)s->admitted.size() < s->max_batch) {
      Req* r = s->waiting.front();
      if (s->used + r->bytes > s->budget) {
        if (!r->deferred) { r->deferred = true; ++s->waited; }
        break;
      }
      s->waiting.pop_front();
      s->used += r->bytes;
      s->high_water = std::max(s->high_water, s->used);
      r->t_admit = now_s();
      lk.unlock();
      const int rc = upload(s, r);
      lk.lock();
      if (rc != FBF_OK) retire(s, r, rc, now_s());
      else s->admitted.push_back(r);
      busy = true;
    }
    // continuous batching: launch whatever is admitted whenever a launch slot is free
    if (!s->admitted.empty() && (int)s->inflight.size() < s->max_inflight) {
      Launch L;
      L.reqs.swap(s->admitted);
      const double t = now_s();
      for (Req* r : L.reqs) {
        r->t_launch = t;
        r->batch = (int)L.reqs.size();
      }
      lk.unlock();
      const int rc = launch(s, L);
      lk.lock();
      if (rc != FBF_OK) {
        // the stream state is unknown: wait for what was enqueued, free what was not freed.
        // fbf_launch empties the batch's queue on failure too; if an fbf_batch_submit failed
        // before it, images stay queued, and the batch (idle now) is made anew
        lk.unlock();
        release_after_error(s, L.reqs);
        int queued = 0;
        if (!s->batch || fbf_batch_pending(s->batch, &queued) != FBF_OK || queued > 0) {
          if (s->batch) fbf_batch_destroy(s->batch);
          s->batch = nullptr;
          fbf_batch_create(&s->batch, s->max_batch, 0);   // if this fails, launches fail
        }
        lk.lock();
        if (L.done) cudaEventDestroy(L.done);
        for (Req* r : L.reqs) retire(s, r, rc, now_s());
      } else {
        s->inflight.push_back(L);
        ++s->launches;
        s->max_inflight_seen = std::max(s->max_inflight_seen, (uint32_t)s->inflight.size());
      }
      busy = true;
    }
    // completions, in launch order
    while (!s->inflight.empty()) {
      Launch& L = s->inflight.front();
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaErrorNotReady) break;
      const fbf::NvtxRange tr("fbf_server complete");
      const double t = now_s();
      const int st = (q == cudaSuccess) ? FBF_DONE : FBF_ECUDA;
      if (st != FBF_DONE) fbf::set_error(FBF_ECUDA, std::string("fbf_server: ") + cudaGetErrorString(q));
      for (Req* r : L.reqs) retire(s, r, st, t);
      cudaEventDestroy(L.done);
      s->inflight.pop_front();
      busy = true;
    }
    if (busy) s->idle.notify_all();
    if (s->stop && s->waiting.empty() && s->admitted.empty() && s->inflight.empty()) break;
    if (!busy) {
      if (s->waiting.empty() && s->admitted.empty() && s->inflight.empty()) {
        s->work.wait(lk);                       // nothing on the GPU: sleep until a submit
      } else {
        lk.unlock();                            // GPU work in flight: poll its events
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
}

// The server's plan for (sigma, R, theta, K, eps), created on first use (lock not held).
int get_plan(fbf_server_s* s, double sigma, int R, double theta, int K, double eps, fbf_plan_t* out) {
  const PlanKey key{sigma, R, theta, K, eps};
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) { *out = it->second; return FBF_OK; }
  }
  fbf_plan_t p = nullptr;
  int rc = fbf_plan(&p, sigma, R, theta, K, eps, s->precision, 0);
  if (rc != FBF_OK) return rc;
  int r = 0;
  fbf_plan_radius(p, &r);
  const int rmax = (s->precision == FBF_FP32 || s->precision == FBF_FAST) ? FBF_MAX_RADIUS : FBF_MAX_RADIUS_TC;
  if (r > rmax) {
    fbf_plan_destroy(p);
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_server_submit: radius beyond the form's limit");
  }
  std::lock_guard<std::mutex> g(s->mu);
  auto ins = s->plans.emplace(key, p);
  if (!ins.second) fbf_plan_destroy(p);      // another thread made it first
  *out = ins.first->second;
  return FBF_OK;
}

void percentiles(std::vector<double> xs, double* p50, double* p99) {
  if (xs.empty()) { *p50 = *p99 = NAN; return; }
  std::sort(xs.begin(), xs.end());
  auto at = [&](double q) {
    size_t i = (size_t)std::ceil(q / 100.0 * xs.size());
    i = i == 0 ? 0 : i - 1;
    return xs[std::min(i, xs.size() - 1)];
  };
  *p50 = at(50);
  *p99 = at(99);
}

}  // namespace

extern "C" {

int fbf_server_create(fbf_server_t* out, int device, int precision, uint64_t hbm_budget_bytes,
                      int max_batch, int max_inflight) try {
  if (!out) return fbf::set_error(FBF_EINVAL, "fbf_server_create: out is NULL");
  *out = nullptr;
  if (precision != FBF_FP32 && precision != FBF_FP16_TC && precision != FBF_BF16_TC && precision != FBF_FAST)
    return fbf::set_error(FBF_EINVAL, "fbf_server_create: unknown precision form");
  if (max_batch < 1 || max_inflight < 1 || hbm_budget_bytes == 0)
    return fbf::set_error(FBF_EINVAL, "fbf_server_create: max_batch, max_inflight and the budget must be >= 1");
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_server_create: ") + cudaGetErrorString(e));
  fbf_server_s* s = new (std::nothrow) fbf_server_s();
  if (!s) return fbf::set_error(FBF_ENOMEM, "fbf_server_create: out of host memory");
  s->device = device;
  s->precision = precision;
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  s->max_inflight = max_inflight;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&s->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = hbm_budget_bytes;   // freed buffers stay in the pool up to the budget
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaSetDevice(cur);
  int rc = FBF_OK;
  if (e != cudaSuccess) rc = fbf::set_error(FBF_ECUDA, std::string("fbf_server_create: ") + cudaGetErrorString(e));
  if (rc == FBF_OK) rc = fbf_batch_create(&s->batch, max_batch, 0);
  if (rc != FBF_OK) {
    if (s->up) cudaStreamDestroy(s->up);
    if (s->comp) cudaStreamDestroy(s->comp);
    if (s->down) cudaStreamDestroy(s->down);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return rc;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_create")

int fbf_server_submit(fbf_server_t s, const float* host_in, float* host_out, int H, int W, double theta,
                      double sigma, int R, int K, double eps, fbf_ticket_t* ticket) try {
  if (!s || !host_in || !host_out) return fbf::set_error(FBF_EINVAL, "fbf_server_submit: NULL argument");
  if (H < 1 || W < 1) return fbf::set_error(FBF_EINVAL, "fbf_server_submit: H and W must be >= 1");
  const uint64_t bytes = 8ull * (uint64_t)H * (uint64_t)W;
  if (bytes > s->budget) return fbf::set_error(FBF_EINVAL, "fbf_server_submit: image larger than the HBM budget");
  fbf_plan_t plan = nullptr;
  int rc = get_plan(s, sigma, R, theta, K, eps, &plan);
  if (rc != FBF_OK) return rc;
  Req* r = new (std::nothrow) Req();
  if (!r) return fbf::set_error(FBF_ENOMEM, "fbf_server_submit: out of host memory");
  r->host_in = host_in;
  r->host_out = host_out;
  r->H = H;
  r->W = W;
  r->plan = plan;
  r->bytes = bytes;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) {
      delete r;
      return fbf::set_error(FBF_EINVAL, "fbf_server_submit: server is shutting down");
    }
    r->t_submit = now_s();
    if (s->t_first < 0) s->t_first = r->t_submit;
    r->id = s->next_id++;
    s->status[r->id] = FBF_PENDING;
    s->waiting.push_back(r);
    ++s->pending;
    if (ticket) *ticket = r->id;
  }
  s->work.notify_one();
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_submit")

int fbf_server_replay(fbf_server_t s, int n, const double* arrival_s, const float* const* host_in,
                      float* const* host_out, const int* H, const int* W, const double* theta,
                      const double* sigma, const int* R, const int* K, const double* eps,
                      fbf_ticket_t* tickets) try {
  if (!s || n < 0 || (n > 0 && (!arrival_s || !host_in || !host_out || !H || !W || !theta || !sigma || !R ||
                                !K || !eps)))
    return fbf::set_error(FBF_EINVAL, "fbf_server_replay: NULL argument");
  for (int i = 1; i < n; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return fbf::set_error(FBF_EINVAL, "fbf_server_replay: arrivals not sorted");
  // plans first, so that fitting does not delay the submissions
  for (int i = 0; i < n; ++i) {
    fbf_plan_t p = nullptr;
    const int rc = get_plan(s, sigma[i], R[i], theta[i], K[i], eps[i], &p);
    if (rc != FBF_OK) return rc;
  }
  const Clock::time_point t0 = Clock::now();
  for (int i = 0; i < n; ++i) {
    const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
    // sleep to within 100 us of the arrival, then poll the clock
    const Clock::time_point coarse = due - std::chrono::microseconds(100);
    if (Clock::now() < coarse) std::this_thread::sleep_until(coarse);
    while (Clock::now() < due) {
    }
    const int rc = fbf_server_submit(s, host_in[i], host_out[i], H[i], W[i], theta[i], sigma[i], R[i], K[i],
                                     eps[i], tickets ? tickets + i : nullptr);
    if (rc != FBF_OK) return rc;
  }
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_replay")

int fbf_server_poll(fbf_server_t s, fbf_ticket_t ticket, int* status) try {
  if (!s || !status) return fbf::set_error(FBF_EINVAL, "fbf_server_poll: NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->status.find(ticket);
  if (it == s->status.end()) return fbf::set_error(FBF_EINVAL, "fbf_server_poll: unknown ticket");
  *status = it->second;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_poll")

int fbf_server_drain(fbf_server_t s, double timeout_s) try {
  if (!s) return fbf::set_error(FBF_EINVAL, "fbf_server_drain: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->idle.wait_for(lk, std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s),
                                   [s] { return s->pending == 0; });
  if (!ok) return fbf::set_error(FBF_ETIMEDOUT, "fbf_server_drain: requests still pending");
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_drain")

int fbf_server_stats(fbf_server_t s, fbf_server_stats_t* out) try {
  if (!s || !out) return fbf::set_error(FBF_EINVAL, "fbf_server_stats: NULL argument");
  std::vector<std::array<double, 6>> tr;
  {
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->requests = s->requests;
    out->pixels = s->pixels;
    out->launches = s->launches;
    out->failed = s->failed;
    out->hbm_high_water = s->high_water;
    out->waited_for_budget = s->waited;
    out->max_inflight_seen = s->max_inflight_seen;
    out->wall_s = (s->t_first >= 0 && s->t_last >= s->t_first) ? s->t_last - s->t_first : 0.0;
    tr = s->trace;
  }
  std::vector<double> lat(tr.size());
  for (size_t i = 0; i < tr.size(); ++i) lat[i] = tr[i][0];
  double p50 = NAN, p99 = NAN;
  percentiles(lat, &p50, &p99);
  out->p50_ms = 1e3 * p50;
  out->p99_ms = 1e3 * p99;
  Tail t;
  for (const auto& x : tr) {
    if (!(x[0] >= p99)) continue;
    t.n += 1;
    t.queued += x[1];
    t.wait += x[2];
    t.l2r += x[3];
    t.mpix += x[4] / 1e6;
    t.batch += x[5];
  }
  out->tail_requests = t.n;
  if (t.n > 0) {
    out->tail_queued_ms = 1e3 * t.queued / t.n;
    out->tail_wait_for_launch_ms = 1e3 * t.wait / t.n;
    out->tail_launch_to_result_ms = 1e3 * t.l2r / t.n;
    out->tail_mpix = t.mpix / t.n;
    out->tail_batch = t.batch / t.n;
  }
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_stats")

int fbf_server_reset_stats(fbf_server_t s) try {
  if (!s) return fbf::set_error(FBF_EINVAL, "fbf_server_reset_stats: NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  if (s->pending != 0) return fbf::set_error(FBF_EBUSY, "fbf_server_reset_stats: requests pending");
  s->requests = s->pixels = s->launches = s->failed = s->waited = 0;
  s->high_water = s->used;
  s->max_inflight_seen = 0;
  s->t_first = s->t_last = -1;
  s->trace.clear();
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_reset_stats")

int fbf_server_destroy(fbf_server_t s) try {
  if (!s) return FBF_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  if (s->batch) fbf_batch_destroy(s->batch);
  for (auto& kv : s->plans) fbf_plan_destroy(kv.second);
  if (s->up) cudaStreamDestroy(s->up);
  if (s->comp) cudaStreamDestroy(s->comp);
  if (s->down) cudaStreamDestroy(s->down);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  cudaSetDevice(cur);
  delete s;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_server_destroy")

int fbf_debug_server_inject(fbf_server_t s, int stage, int count) try {
  if (!s || count < 0 || (stage != 1 && stage != 2))
    return fbf::set_error(FBF_EINVAL, "fbf_debug_server_inject: bad arguments");
  (stage == 1 ? s->inject_upload : s->inject_launch).store(count);
  return FBF_OK;
} FBF_ABI_CATCH("fbf_debug_server_inject")

}  // extern "C"
