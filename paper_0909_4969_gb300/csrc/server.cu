// Served decompositions of a tensor stream (the monitoring setting of
// Section 1 and Section 4: windows of hosts x measurement types x timeticks
// arriving over time).  Each request is one MACH-HOOI (Algorithm 2) of one
// window; windows of the same stream warm-start HOOI from the previous
// window's factors, kept resident on the device.
//
// Continuous batching: a fixed number of slots, each a host worker thread
// with its own CUDA stream.  A request is admitted as soon as a slot is
// free, its estimated device memory fits in what the HBM budget has left,
// and no earlier request of the same stream is pending or running (so warm
// starts follow window order).  Admitted requests run concurrently on their
// slots' streams; later arrivals are admitted as slots and memory free up.
// A request whose shape differs from its stream's resident state (a resized
// window) starts cold from the HOSVD and leaves the state untouched.
#include "mach_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace mach {
namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket = 0;
  int64_t stream_id = 0;
  const void* x = nullptr;
  mach_dtype dt = MACH_F32;
  int d = 0;
  int64_t dims[kMaxModes] = {0, 0, 0, 0};
  int ranks[kMaxModes] = {0, 0, 0, 0};
  double p = 1.0;
  uint64_t seed = 0;
  int sweeps = 0;
  mach_prec prec = MACH_PREC_FP32;
  size_t est = 0;
  int passed_over = 0;
  // results
  bool done = false;
  mach_status status = MACH_OK;
  std::string error;
  std::vector<double> core;
  std::vector<double> factors[kMaxModes];
  double err = 0.0;
  bool warm = false;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

// Resident per-stream state: the last window's factors (FP64 column-major).
struct StreamState {
  int d = 0;
  int64_t dims[kMaxModes] = {0, 0, 0, 0};
  int ranks[kMaxModes] = {0, 0, 0, 0};
  double* fac[kMaxModes] = {nullptr, nullptr, nullptr, nullptr};
  bool valid = false;
  bool busy = false;
};

bool same_shape(const StreamState& s, const Request& r) {
  if (!s.valid || s.d != r.d) return false;
  for (int k = 0; k < r.d; ++k)
    if (s.dims[k] != r.dims[k] || s.ranks[k] != r.ranks[k]) return false;
  return true;
}

// Device memory of one decomposition, from the sizes of everything
// mach_sample and mach_hooi allocate (kept set, per-mode orderings and
// fibre indices, sort and build scratch, workspace), with 3 sigma on K.
size_t estimate_bytes(const Request& r) {
  double N = 1.0;
  int64_t maxI = 1;
  for (int k = 0; k < r.d; ++k) {
    N *= (double)r.dims[k];
    maxI = std::max<int64_t>(maxI, r.dims[k]);
  }
  const double q = std::min(1.0, r.p);
  const double K = std::min(N, N * q + 3.0 * std::sqrt(N * q * (1.0 - q) + 1.0) + 4096.0);
  const double vs = r.dt == MACH_F32 ? 4.0 : 8.0;
  const double ts = r.prec == MACH_PREC_FP64 ? 8.0 : 4.0;
  double bytes = K * (8.0 + vs);                                  // kept set
  bytes += r.d * (K * (vs + 2.0 + 4.0 + 4.0) + 3.0 * 4.0 * maxI);  // orderings + fibres
  bytes += (double)sort_scratch_bytes((int64_t)K, maxI) + (double)csf_scratch_bytes((int64_t)K, maxI);
  double ws = 0.0;
  for (int n = 0; n < r.d; ++n) {
    double J = 1.0;
    for (int k = 0; k < r.d; ++k)
      if (k != n) J *= r.ranks[k];
    const double M = std::min((double)r.dims[n], J);
    ws = std::max(ws, (double)r.dims[n] * J * ts * 2.0 + std::max(M, (double)r.dims[n]) *
                                                                  std::max(M, (double)r.dims[n]) * ts);
  }
  bytes += ws + 64.0 * maxI * kMaxRank * 8.0 + (double)(32u << 20);
  double out = 0.0;
  for (int k = 0; k < r.d; ++k) out += (double)r.dims[k] * r.ranks[k] * 8.0;
  double core = 1.0;
  for (int k = 0; k < r.d; ++k) core *= r.ranks[k];
  bytes += out + core * 8.0;
  return (size_t)bytes;
}

}  // namespace

struct Server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::unordered_map<int64_t, Request*> tickets;
  std::unordered_map<int64_t, StreamState> streams;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> slot_streams;
  bool stop = false;
  size_t used = 0;
  int64_t next_ticket = 1;
  int active = 0;
  int max_active = 0;
  int64_t completed = 0;
  std::vector<double> latencies;

  // First admissible pending request (FIFO order), or null.  A request that
  // does not fit the remaining budget is passed over, but once it has been
  // passed over 2 * max_slots times nothing behind it is admitted until it
  // fits (no starvation of large windows).
  Request* pick() {
    std::unordered_map<int64_t, bool> seen;   // streams with an earlier pending request
    for (auto it = pending.begin(); it != pending.end(); ++it) {
      Request* r = *it;
      const bool stream_blocked = seen.count(r->stream_id) || streams[r->stream_id].busy;
      seen[r->stream_id] = true;
      if (stream_blocked) continue;
      if (used + r->est <= budget) {
        pending.erase(it);
        return r;
      }
      if (++r->passed_over > 2 * max_slots) return nullptr;
    }
    return nullptr;
  }

  void run(Request* r, cudaStream_t st);
  void worker(int slot);
};

void Server::run(Request* r, cudaStream_t st) {
  r->t_start = now_ms();
  mach_status s = MACH_OK;
  mach_sample_t smp = nullptr;
  double* fac[kMaxModes] = {nullptr, nullptr, nullptr, nullptr};
  double* core = nullptr;
  int64_t R = 1;
  for (int k = 0; k < r->d; ++k) R *= r->ranks[k];
  auto fail = [&](mach_status e) {
    s = e;
    r->error = mach_last_error();
  };
  // factors and core of this request (device, FP64)
  for (int k = 0; k < r->d && s == MACH_OK; ++k)
    if (cudaMallocAsync(&fac[k], (size_t)r->dims[k] * r->ranks[k] * sizeof(double), st) != cudaSuccess)
      fail(MACH_ENOMEM);
  if (s == MACH_OK && cudaMallocAsync(&core, (size_t)R * sizeof(double), st) != cudaSuccess) fail(MACH_ENOMEM);
  bool warm = false;
  if (s == MACH_OK) {
    std::unique_lock<std::mutex> lk(mu);
    StreamState& ss = streams[r->stream_id];
    if (same_shape(ss, *r)) {
      warm = true;
      for (int k = 0; k < r->d; ++k)
        cudaMemcpyAsync(fac[k], ss.fac[k], (size_t)r->dims[k] * r->ranks[k] * sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
    }
  }
  mach_status e;
  if (s == MACH_OK && (e = mach_sample(r->x, r->dt, r->d, r->dims, r->p, r->seed, st, &smp)) != MACH_OK) fail(e);
  if (s == MACH_OK &&
      (e = mach_hooi(smp, r->ranks, r->sweeps, r->prec, fac, core, warm ? 1 : 0, st)) != MACH_OK)
    fail(e);
  if (s == MACH_OK &&
      (e = mach_error(r->x, r->dt, r->d, r->dims, r->ranks, fac, core, &r->err, nullptr, st)) != MACH_OK)
    fail(e);
  if (s == MACH_OK) {
    r->core.resize((size_t)R);
    for (int k = 0; k < r->d; ++k) r->factors[k].resize((size_t)r->dims[k] * r->ranks[k]);
    bool ok = cudaMemcpyAsync(r->core.data(), core, (size_t)R * sizeof(double), cudaMemcpyDeviceToHost, st) ==
              cudaSuccess;
    for (int k = 0; k < r->d; ++k)
      ok = ok && cudaMemcpyAsync(r->factors[k].data(), fac[k], r->factors[k].size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (!ok || cudaStreamSynchronize(st) != cudaSuccess) fail(MACH_ECUDA);
  }
  if (smp) mach_sample_free(smp);
  {
    std::unique_lock<std::mutex> lk(mu);
    StreamState& ss = streams[r->stream_id];
    // the stream's resident factors: set by the first window, advanced by
    // every window of the same shape, untouched by resized windows
    if (s == MACH_OK && (!ss.valid || same_shape(ss, *r))) {
      for (int k = 0; k < kMaxModes; ++k) {
        if (ss.fac[k]) cudaFreeAsync(ss.fac[k], st);
        ss.fac[k] = nullptr;
      }
      ss.d = r->d;
      for (int k = 0; k < r->d; ++k) {
        ss.dims[k] = r->dims[k];
        ss.ranks[k] = r->ranks[k];
        ss.fac[k] = fac[k];
        fac[k] = nullptr;
      }
      ss.valid = true;
    }
  }
  for (int k = 0; k < r->d; ++k)
    if (fac[k]) cudaFreeAsync(fac[k], st);
  if (core) cudaFreeAsync(core, st);
  cudaStreamSynchronize(st);
  r->warm = warm;
  r->status = s;
  r->t_done = now_ms();
}

void Server::worker(int slot) {
  cudaSetDevice(device);
  cudaStream_t st = slot_streams[slot];
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || (r = pick()) != nullptr; });
      if (!r) return;   // stop
      used += r->est;
      streams[r->stream_id].busy = true;
      ++active;
      max_active = std::max(max_active, active);
    }
    run(r, st);
    {
      std::unique_lock<std::mutex> lk(mu);
      used -= r->est;
      streams[r->stream_id].busy = false;
      --active;
      ++completed;
      latencies.push_back(r->t_done - r->t_submit);
      r->done = true;
    }
    cv.notify_all();
  }
}

}  // namespace mach

using mach::Request;
using mach::Server;

extern "C" {

mach_status mach_server_create(size_t hbm_budget_bytes, int max_slots, void** srv) {
  if (!srv || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return MACH_EINVAL;
  Server* s = new Server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return MACH_ECUDA;
  }
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  for (int i = 0; i < max_slots; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t q : s->slot_streams) cudaStreamDestroy(q);
      delete s;
      return MACH_ECUDA;
    }
    s->slot_streams.push_back(st);
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(&Server::worker, s, i);
  *srv = s;
  return MACH_OK;
}

mach_status mach_submit(void* srv, int64_t stream_id, const void* x_dev, mach_dtype dtype, int d,
                        const int64_t* dims, const int* ranks, double p, uint64_t seed, int sweeps, mach_prec prec,
                        int64_t* ticket) {
  Server* s = static_cast<Server*>(srv);
  if (!s || !x_dev || !dims || !ranks || !ticket) return MACH_EINVAL;
  if (d < 2 || d > mach::kMaxModes || !(p > 0.0 && p <= 1.0) || sweeps < 0) return MACH_EINVAL;
  if (dtype != MACH_F32 && dtype != MACH_F64) return MACH_EINVAL;
  if (prec != MACH_PREC_FP64 && prec != MACH_PREC_FP32 && prec != MACH_PREC_BF16_REFINE) return MACH_EINVAL;
  Request* r = new Request();
  r->stream_id = stream_id;
  r->x = x_dev;
  r->dt = dtype;
  r->d = d;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > mach::kMaxDim || ranks[k] < 1 || ranks[k] > mach::kMaxRank ||
        ranks[k] > dims[k]) {
      delete r;
      return MACH_EINVAL;
    }
    r->dims[k] = dims[k];
    r->ranks[k] = ranks[k];
  }
  r->p = p;
  r->seed = seed;
  r->sweeps = sweeps;
  r->prec = prec;
  r->est = mach::estimate_bytes(*r);
  if (r->est > s->budget) {
    delete r;
    return MACH_ENOMEM_BUDGET;
  }
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return MACH_EBUSY;
    }
    if (s->pending.size() >= 65536) {
      delete r;
      return MACH_EAGAIN;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = mach::now_ms();
    s->tickets[r->ticket] = r;
    s->pending.push_back(r);
  }
  s->cv.notify_all();
  *ticket = r->ticket;
  return MACH_OK;
}

mach_status mach_poll(void* srv, int64_t ticket, int* done, double* core_host, double* const* factors_host,
                      double* err_out) {
  Server* s = static_cast<Server*>(srv);
  if (!s || !done) return MACH_EINVAL;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return MACH_EINVAL;
    r = it->second;
    if (!r->done) {
      *done = 0;
      return MACH_EAGAIN;
    }
    s->tickets.erase(it);
  }
  *done = 1;
  const mach_status st = r->status;
  if (st == MACH_OK) {
    if (core_host) std::memcpy(core_host, r->core.data(), r->core.size() * sizeof(double));
    if (factors_host)
      for (int k = 0; k < r->d; ++k)
        if (factors_host[k]) std::memcpy(factors_host[k], r->factors[k].data(), r->factors[k].size() * sizeof(double));
    if (err_out) *err_out = r->err;
  }
  delete r;
  return st;
}

mach_status mach_server_stats(void* srv, int64_t* completed, double* p50_ms, double* p99_ms, int* max_in_flight,
                              size_t* budget_in_use) {
  Server* s = static_cast<Server*>(srv);
  if (!s) return MACH_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<double> v = s->latencies;
  std::sort(v.begin(), v.end());
  auto q = [&](double f) -> double {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::ceil(f * (double)v.size());
    i = i == 0 ? 0 : i - 1;
    return v[std::min(i, v.size() - 1)];
  };
  if (completed) *completed = s->completed;
  if (p50_ms) *p50_ms = q(0.50);
  if (p99_ms) *p99_ms = q(0.99);
  if (max_in_flight) *max_in_flight = s->max_active;
  if (budget_in_use) *budget_in_use = s->used;
  return MACH_OK;
}

mach_status mach_request_bytes(mach_dtype dtype, int d, const int64_t* dims, const int* ranks, double p,
                               mach_prec prec, size_t* bytes) {
  if (!dims || !ranks || !bytes || d < 2 || d > mach::kMaxModes || !(p > 0.0 && p <= 1.0)) return MACH_EINVAL;
  Request r;
  r.dt = dtype;
  r.d = d;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || ranks[k] < 1) return MACH_EINVAL;
    r.dims[k] = dims[k];
    r.ranks[k] = ranks[k];
  }
  r.p = p;
  r.prec = prec;
  *bytes = mach::estimate_bytes(r);
  return MACH_OK;
}

mach_status mach_server_destroy(void* srv) {
  Server* s = static_cast<Server*>(srv);
  if (!s) return MACH_EINVAL;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stop = true;
    // requests not yet admitted are dropped
    for (Request* r : s->pending) {
      s->tickets.erase(r->ticket);
      delete r;
    }
    s->pending.clear();
  }
  s->cv.notify_all();
  for (std::thread& t : s->workers) t.join();
  for (auto& kv : s->tickets) delete kv.second;
  cudaSetDevice(s->device);
  for (auto& kv : s->streams)
    for (int k = 0; k < mach::kMaxModes; ++k)
      if (kv.second.fac[k]) cudaFree(kv.second.fac[k]);
  for (cudaStream_t q : s->slot_streams) {
    cudaStreamSynchronize(q);
    cudaStreamDestroy(q);
  }
  delete s;
  return MACH_OK;
}

}  // extern "C"
