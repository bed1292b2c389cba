// C ABI of libmach (declared in include/mach.h): argument checking, device
// memory ownership and the orchestration of the kernels of Algorithm 2.
#include "mach_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <type_traits>
#include <vector>

namespace mach {

// ---- error state -------------------------------------------------------------
static thread_local char g_last_error[512] = "";

void set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

mach_status dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s) {
  b.bytes = bytes;
  b.ptr = nullptr;
  if (bytes == 0) return MACH_OK;
  // 256 bytes of slack past the end: 16-byte-granular bulk copies may round a
  // range end up by up to 15 bytes (never used, never written).
  const size_t padded = ((bytes + 255) & ~(size_t)255) + 256;
  cudaError_t e = cudaMallocAsync(&b.ptr, padded, s);
  if (e != cudaSuccess) {
    set_last_error("cudaMallocAsync(%zu) -> %s", padded, cudaGetErrorString(e));
    b.ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? MACH_ENOMEM : MACH_ECUDA;
  }
  return MACH_OK;
}

void dev_free(DevBuf& b, cudaStream_t s) {
  if (b.ptr) cudaFreeAsync(b.ptr, s);
  b.ptr = nullptr;
  b.bytes = 0;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- profiling -----------------------------------------------------------------
struct ProfRec {
  cudaEvent_t a, b;
  int kind;
  double bytes;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;
static cudaEvent_t g_open[PROF_NKINDS];

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// While a stream is being captured, the record must become an event-record
// node of the graph (re-armed with fresh events for every replay).
static void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

void prof_begin(int kind, cudaStream_t s) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on) return;
  g_open[kind] = prof_event();
  prof_record(g_open[kind], s);
}

void prof_end(int kind, cudaStream_t s, double bytes) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on || !g_open[kind]) return;
  cudaEvent_t e = prof_event();
  prof_record(e, s);
  g_prof.push_back(ProfRec{g_open[kind], e, kind, bytes});
  g_open[kind] = nullptr;
}

// Helpers for replayed CUDA graphs: the records made while a sweep was
// captured are taken out (that sweep never ran) and every replay pushes its
// own records with fresh events.
static size_t prof_mark() {
  std::lock_guard<std::mutex> g(g_prof_mu);
  return g_prof.size();
}

static std::vector<ProfRec> prof_take_since(size_t i) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  std::vector<ProfRec> out;
  if (i < g_prof.size()) {
    out.assign(g_prof.begin() + (std::ptrdiff_t)i, g_prof.end());
    g_prof.resize(i);
  }
  return out;
}

static bool prof_replay_push(cudaEvent_t* a, cudaEvent_t* b, int kind, double bytes) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on) return false;
  *a = prof_event();
  *b = prof_event();
  g_prof.push_back(ProfRec{*a, *b, kind, bytes});
  return true;
}

static void prof_release(cudaEvent_t e) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_pool.push_back(e);
}

static void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_patch_last_bytes(int kind, double bytes) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto it = g_prof.rbegin(); it != g_prof.rend(); ++it)
    if (it->kind == kind) {
      it->bytes = bytes;
      return;
    }
}

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached = n > 0 ? n : 1;
  }
  return cached;
}

}  // namespace mach

using namespace mach;

// Device scalars of a sample object.
struct SampleScalars {
  int64_t count;
  unsigned err;
  uint32_t nfib[kMaxModes];
  uint32_t ntask[kMaxModes];
  unsigned long long eig_stats[3];   // eigensolver calls, iterations, unconverged
  unsigned long long eig_ctl[8];     // split-path iteration control
  unsigned counter;
  double acc[2];
};

struct ModeCsf {
  DevBuf idx;        // mode-ordered l (only while building; mode 0 keeps it)
  DevBuf val;        // mode-ordered values
  DevBuf val16;      // BF16 copy of val (made by the first BF16_REFINE sweep)
  DevBuf leaf;       // uint16
  DevBuf fib_start;  // uint32 K + 1
  DevBuf fib_mid;    // uint32 K
  DevBuf row_fib;    // uint32 I + 1
  DevBuf row_task;   // uint32 I + 1
  DevBuf tasks;      // int4
  int64_t ntask_cap = 0;
  uint32_t emax = 0;
};

// HOOI workspace, one per precision.
struct Workspace {
  bool ready = false;
  int ranks[kMaxModes] = {0, 0, 0, 0};
  DevBuf fac[kMaxModes];  // T row-major I_k x r_k
  DevBuf Y, partial, C, gram_part, V, W, U, Vout, theta, A64, gram64, rinv;
  DevBuf eig_part;           // split-path partial Grams
  DevBuf ytpart;             // partials of the warm-start product Y^T A
  DevBuf basis[kMaxModes];   // per mode: last Ritz block (M x b, T)
  int basis_M[kMaxModes] = {0, 0, 0, 0};   // its M and b (0 = none)
  int basis_b[kMaxModes] = {0, 0, 0, 0};
  int64_t partial_cap_elems = 0;
  int64_t gram_part_cap = 0;
};

struct mach_sample_s {
  int d = 0;
  int64_t dims[kMaxModes] = {1, 1, 1, 1};
  mach_dtype dt = MACH_F32;
  double p = 1.0;
  uint64_t seed = 0;
  uint64_t T = 0;
  int64_t N = 0;
  int64_t K = 0;
  cudaStream_t stream = nullptr;
  DevBuf idx, val;  // sampler output, increasing l (mode 0 order)
  ModeCsf mode[kMaxModes];
  DevBuf scal;      // SampleScalars
  int64_t nfib[kMaxModes] = {0, 0, 0, 0};   // host copies after the build
  int64_t ntask[kMaxModes] = {0, 0, 0, 0};
  Workspace ws[2];  // [0] FP32, [1] FP64
  SampleScalars* dscal() { return static_cast<SampleScalars*>(scal.ptr); }
};

namespace {

size_t dtype_size(mach_dtype dt) { return dt == MACH_F32 ? 4 : 8; }

void free_mode(ModeCsf& m, cudaStream_t s, bool keep_idx) {
  if (!keep_idx) dev_free(m.idx, s);
  dev_free(m.val, s);
  dev_free(m.val16, s);
  dev_free(m.leaf, s);
  dev_free(m.fib_start, s);
  dev_free(m.fib_mid, s);
  dev_free(m.row_fib, s);
  dev_free(m.row_task, s);
  dev_free(m.tasks, s);
}

void free_ws(Workspace& w, cudaStream_t s) {
  for (auto& f : w.fac) dev_free(f, s);
  for (int k = 0; k < kMaxModes; ++k) {
    dev_free(w.basis[k], s);
    w.basis_M[k] = w.basis_b[k] = 0;
  }
  dev_free(w.Y, s);
  dev_free(w.partial, s);
  dev_free(w.C, s);
  dev_free(w.gram_part, s);
  dev_free(w.V, s);
  dev_free(w.W, s);
  dev_free(w.U, s);
  dev_free(w.Vout, s);
  dev_free(w.theta, s);
  dev_free(w.A64, s);
  dev_free(w.gram64, s);
  dev_free(w.rinv, s);
  dev_free(w.eig_part, s);
  dev_free(w.ytpart, s);
  w.ready = false;
}

void free_sample(mach_sample_s* h) {
  cudaStream_t s = h->stream;
  for (int k = 0; k < kMaxModes; ++k) {
    if (k == 0) {
      // mode 0 aliases idx/val of the sampler output
      h->mode[0].idx.ptr = nullptr;
      h->mode[0].val.ptr = nullptr;
    }
    free_mode(h->mode[k], s, false);
  }
  dev_free(h->idx, s);
  dev_free(h->val, s);
  free_ws(h->ws[0], s);
  free_ws(h->ws[1], s);
  dev_free(h->scal, s);
}

// Modes of the cyclic ordering of mode n.
struct Cyc {
  int row, leaf, nmid, mid[2];
};
Cyc cyc(int d, int n) {
  Cyc c;
  c.row = n;
  c.leaf = (n + d - 1) % d;
  c.nmid = d - 2;
  c.mid[0] = (n + 1) % d;
  c.mid[1] = (n + 2) % d;
  return c;
}

// Block width of the subspace iteration: the leading r eigenvectors converge
// like (lambda_{b+1} / lambda_r)^k, so a wider block pays off when the
// spectrum is crowded near r.  Warm-started HOOI updates use at least 16
// columns; the cold HOSVD start always uses the full 32.
int block_size_for(int M, int r, bool cold, bool fp64) {
  // warm starts (previous factor + previous Ritz directions) need few
  // iterations, so the block carries only a few guard directions past r;
  // FP64 cold starts carry the widest block (their results are compared at
  // 1e-10); FP32 cold starts the warm width: the b-space step, whose Jacobi
  // costs ~b^3 per sweep on one warp, bounds the multi-CTA route, and the
  // HOOI sweeps refine the start
  int b = cold && fp64 ? 32 : std::max(r + 6, 16);
  b = std::min(b, 32);
  return std::min(b, M);
}

}  // namespace

// ---------------------------------------------------------------------------
// Public entry points
// ---------------------------------------------------------------------------
extern "C" {

const char* mach_strerror(mach_status s) {
  switch (s) {
    case MACH_OK: return "ok";
    case MACH_EINVAL: return "invalid argument";
    case MACH_ENOMEM: return "out of device memory";
    case MACH_ENOMEM_BUDGET: return "request exceeds the HBM budget";
    case MACH_ECUDA: return "CUDA error";
    case MACH_ETIMEOUT: return "device-side wait timed out";
    case MACH_EBUSY: return "busy";
    case MACH_EAGAIN: return "not ready, retry";
    case MACH_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* mach_last_error(void) { return g_last_error; }

const char* mach_version(void) { return "libmach 0.1 (sm_103a)"; }

mach_status mach_profile_enable(int enable) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto& r : g_prof) {
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof.clear();
  for (auto& e : g_open) e = nullptr;
  g_prof_on = enable != 0;
  return MACH_OK;
}

mach_status mach_profile_query(int kind, double* total_ms, int64_t* launches, double* bytes) {
  if (kind < 0 || kind >= PROF_NKINDS || !total_ms || !launches || !bytes) return MACH_EINVAL;
  std::lock_guard<std::mutex> g(g_prof_mu);
  double t = 0.0, by = 0.0;
  int64_t n = 0;
  for (auto& r : g_prof) {
    if (r.kind != kind) continue;
    MACH_CUDA_TRY(cudaEventSynchronize(r.b));
    float ms = 0.f;
    MACH_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    by += r.bytes;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  *bytes = by;
  return MACH_OK;
}

int64_t mach_launch_count(void) { return (int64_t)g_launches.load(); }

mach_status mach_check_bounded_wait(long long limit, int arrive, void* stream) {
  if (limit < 1 || limit > kSpinLimit) return MACH_EINVAL;
  return run_bounded_wait_check(limit, arrive, static_cast<cudaStream_t>(stream));
}

// The input streamed from host memory: chunk_entries > 0 entries of x_host
// at a time, copied into a ring of two device buffers on a copy stream while
// the sampler runs on the previous chunk.
struct HostStream {
  int64_t chunk_entries = 0;   // 0: x is a device pointer
};

static mach_status sample_impl(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims, double p, uint64_t seed,
                               void* stream, mach_sample_t* out, bool skip, HostStream hst = HostStream()) {
  if (!x_dev || !dims || !out) return MACH_EINVAL;
  if (d < 2 || d > kMaxModes) return MACH_EINVAL;
  if (dtype != MACH_F32 && dtype != MACH_F64) return MACH_EINVAL;
  if (!(p > 0.0 && p <= 1.0)) return MACH_EINVAL;
  if (((uintptr_t)x_dev & 15u) != 0) {
    set_last_error("input tensor must be 16-byte aligned");
    return MACH_EINVAL;
  }
  int64_t N = 1;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > kMaxDim) {
      set_last_error("dims[%d] = %lld outside [1, %d]", k, (long long)dims[k], kMaxDim);
      return MACH_EINVAL;
    }
    N *= dims[k];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mach_sample_s* h = new mach_sample_s();
  h->d = d;
  for (int k = 0; k < d; ++k) h->dims[k] = dims[k];
  h->dt = dtype;
  h->p = p;
  h->seed = seed;
  h->T = (uint64_t)std::floor(p * 4294967296.0);
  h->N = N;
  h->stream = st;
  auto fail = [&](mach_status s) {
    cudaStreamSynchronize(st);
    free_sample(h);
    delete h;
    return s;
  };
  mach_status s;
  if ((s = dev_alloc(h->scal, sizeof(SampleScalars), st)) != MACH_OK) return fail(s);
  SampleScalars* ds = h->dscal();
  if (cudaMemsetAsync(ds, 0, sizeof(SampleScalars), st) != cudaSuccess) return fail(MACH_ECUDA);
  // coin + compaction: per-warp segments, then an ordered gather into idx / val
  // (sized for the segments' capacity, so no host round trip in between)
  const double q = h->T >= (1ull << 32) ? 1.0 : (double)h->T / 4294967296.0;
  const bool from_host = hst.chunk_entries > 0;
  const int64_t CE = from_host ? std::min<int64_t>(hst.chunk_entries, N) : N;   // entries per input chunk
  const int64_t nchunks = from_host ? ceil_div(N, CE) : 1;
  SegPlan pl = plan_segments(CE, dtype, q);
  const size_t vs = dtype_size(dtype);
  ScopedDevBuf ring[2] = {ScopedDevBuf(st), ScopedDevBuf(st)};
  cudaStream_t cst = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  auto release_stream = [&]() {
    for (int b = 0; b < 2; ++b) {
      if (copied[b]) cudaEventDestroy(copied[b]);
      if (consumed[b]) cudaEventDestroy(consumed[b]);
      copied[b] = consumed[b] = nullptr;
    }
    if (cst) {
      cudaStreamSynchronize(cst);   // no copy into the ring is left in flight
      cudaStreamDestroy(cst);
    }
    cst = nullptr;
  };
  if (from_host) {
    for (int b = 0; b < 2 && b < nchunks; ++b)
      if ((s = dev_alloc(ring[b], (size_t)CE * vs, st)) != MACH_OK) return fail(s);
    if (cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&consumed[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&consumed[1], cudaEventDisableTiming) != cudaSuccess) {
      release_stream();
      set_last_error("host-streamed sampler: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(MACH_ECUDA);
    }
    // the ring buffers come from stream-ordered allocations on st
    if (cudaEventRecord(consumed[0], st) != cudaSuccess || cudaEventRecord(consumed[1], st) != cudaSuccess) {
      release_stream();
      return fail(MACH_ECUDA);
    }
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    ScopedDevBuf seg_off(st), seg_val(st), seg_cnt(st);
    const int64_t nseg_all = pl.nseg * nchunks;
    const int64_t cap_all = nseg_all * pl.seg_cap;
    if ((s = dev_alloc(h->idx, (size_t)cap_all * 8, st)) != MACH_OK) return release_stream(), fail(s);
    if ((s = dev_alloc(h->val, (size_t)cap_all * vs, st)) != MACH_OK) return release_stream(), fail(s);
    if ((s = dev_alloc(seg_off, (size_t)cap_all * 4, st)) != MACH_OK) return release_stream(), fail(s);
    if ((s = dev_alloc(seg_val, (size_t)cap_all * vs, st)) != MACH_OK) return release_stream(), fail(s);
    if ((s = dev_alloc(seg_cnt, (size_t)nseg_all * 8, st)) != MACH_OK) return release_stream(), fail(s);
    prof_begin(PROF_SAMPLER, st);
    for (int64_t c = 0; c < nchunks; ++c) {
      const int64_t l0 = c * CE, n = std::min<int64_t>(CE, N - l0);
      const void* xc = x_dev;
      if (from_host) {
        const int b = (int)(c & 1);
        // copy chunk c once the sampler has finished with the chunk two back
        if (cudaStreamWaitEvent(cst, consumed[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(ring[b].ptr, static_cast<const char*>(x_dev) + (size_t)l0 * vs, (size_t)n * vs,
                            cudaMemcpyHostToDevice, cst) != cudaSuccess ||
            cudaEventRecord(copied[b], cst) != cudaSuccess || cudaStreamWaitEvent(st, copied[b], 0) != cudaSuccess) {
          set_last_error("host-streamed sampler: %s", cudaGetErrorString(cudaGetLastError()));
          release_stream();
          return fail(MACH_ECUDA);
        }
        xc = ring[b].ptr;
      }
      const size_t so = (size_t)c * pl.nseg * pl.seg_cap;
      if ((s = launch_sampler_seg(xc, dtype, n, l0, seed, h->T, pl, static_cast<uint32_t*>(seg_off.ptr) + so,
                                  static_cast<char*>(seg_val.ptr) + so * vs,
                                  static_cast<int64_t*>(seg_cnt.ptr) + c * pl.nseg, st, skip)) != MACH_OK)
        return release_stream(), fail(s);
      if (from_host && cudaEventRecord(consumed[c & 1], st) != cudaSuccess) return release_stream(), fail(MACH_ECUDA);
    }
    // output position of every segment: one exclusive scan of the counts
    ScopedDevBuf seg_scan(st);
    if ((s = dev_alloc(seg_scan, (size_t)(nseg_all + scan_tmp_elems_total(nseg_all)) * 8, st)) != MACH_OK)
      return release_stream(), fail(s);
    long long* cnt_ll = static_cast<long long*>(seg_cnt.ptr);
    long long* scan_ll = static_cast<long long*>(seg_scan.ptr);
    if ((s = scan_exclusive<long long>(cnt_ll, scan_ll, nseg_all, nullptr, scan_ll + nseg_all, st)) != MACH_OK)
      return release_stream(), fail(s);
    if ((s = launch_seg_gather(dtype, pl, nseg_all, CE, static_cast<const int64_t*>(seg_cnt.ptr),
                               static_cast<const int64_t*>(seg_scan.ptr), static_cast<const uint32_t*>(seg_off.ptr),
                               seg_val.ptr, static_cast<int64_t*>(h->idx.ptr), h->val.ptr, cap_all, &ds->err,
                               st)) != MACH_OK)
      return release_stream(), fail(s);
    dev_free(seg_scan, st);
    prof_end(PROF_SAMPLER, st, 0.0);
    std::vector<int64_t> cnt((size_t)nseg_all);
    SampleScalars hs;
    if (cudaMemcpyAsync(cnt.data(), seg_cnt.ptr, cnt.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&hs, ds, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_last_error("sampler: %s", cudaGetErrorString(cudaGetLastError()));
      return release_stream(), fail(MACH_ECUDA);
    }
    dev_free(seg_off, st);
    dev_free(seg_val, st);
    dev_free(seg_cnt, st);
    if (hs.err & DEV_TIMEOUT) return release_stream(), fail(MACH_ETIMEOUT);
    int64_t K = 0, mx = 0;
    for (int64_t c : cnt) {
      K += c;
      mx = std::max(mx, c);
    }
    h->K = K;
    prof_patch_last_bytes(PROF_SAMPLER, (double)N * vs + (double)K * (vs + 8));
    if (!(hs.err & DEV_OVERFLOW) && mx <= pl.seg_cap) break;
    // a segment exceeded its capacity (an 8-sigma event): rerun with the exact one
    dev_free(h->idx, st);
    dev_free(h->val, st);
    cudaMemsetAsync(&ds->err, 0, sizeof(unsigned), st);
    pl.seg_cap = std::max<int64_t>(mx, 1);
  }
  // the ring is idle once the stream has synchronised above
  release_stream();
  for (int b = 0; b < 2; ++b) dev_free(ring[b], st);
  if (cudaMemcpyAsync(&ds->count, &h->K, sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(MACH_ECUDA);
  const int64_t K = h->K;
  if (K >= (1ll << 31)) {
    set_last_error("too many kept entries (%lld) for 32-bit fibre indices", (long long)K);
    return fail(MACH_EINVAL);
  }
  // ---- per-mode orderings and CSF --------------------------------------------
  const Decoder dec = make_decoder(d, h->dims);
  prof_begin(PROF_CSF, st);
  h->mode[0].idx = h->idx;
  h->mode[0].val = h->val;
  int64_t maxdim = 1;
  for (int k = 0; k < d; ++k) maxdim = std::max(maxdim, h->dims[k]);
  ScopedDevBuf sort_scr(st), csf_scr(st);
  if ((s = dev_alloc(sort_scr, sort_scratch_bytes(K, maxdim), st)) != MACH_OK) return fail(s);
  if ((s = dev_alloc(csf_scr, csf_scratch_bytes(K, maxdim), st)) != MACH_OK) return fail(s);
  const int64_t Kc = std::max<int64_t>(K, 1);
  for (int m = d - 1; m >= 1; --m) {
    ModeCsf& dst = h->mode[m];
    const ModeCsf& srcm = h->mode[(m + 1) % d];
    if ((s = dev_alloc(dst.idx, (size_t)Kc * 8, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(dst.val, (size_t)Kc * vs, st)) != MACH_OK) return fail(s);
    if (dtype == MACH_F32)
      s = counting_sort<float>(static_cast<const int64_t*>(srcm.idx.ptr), static_cast<const float*>(srcm.val.ptr), K,
                               &ds->count, dec, m, static_cast<int64_t*>(dst.idx.ptr),
                               static_cast<float*>(dst.val.ptr), sort_scr.ptr, st);
    else
      s = counting_sort<double>(static_cast<const int64_t*>(srcm.idx.ptr), static_cast<const double*>(srcm.val.ptr),
                                K, &ds->count, dec, m, static_cast<int64_t*>(dst.idx.ptr),
                                static_cast<double*>(dst.val.ptr), sort_scr.ptr, st);
    if (s != MACH_OK) return fail(s);
  }
  const int64_t target_tasks = (int64_t)num_sms() * 64;
  for (int m = 0; m < d; ++m) {
    ModeCsf& M = h->mode[m];
    const int64_t In = h->dims[m];
    int64_t emax = K / std::max<int64_t>(1, target_tasks);
    emax = std::max<int64_t>(256, std::min<int64_t>(emax, (int64_t)ttmc_task_max()));
    M.emax = (uint32_t)emax;
    M.ntask_cap = K / emax + In + 1;
    if ((s = dev_alloc(M.leaf, (size_t)Kc * 2, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(M.fib_start, (size_t)(Kc + 1) * 4, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(M.fib_mid, (size_t)Kc * 4, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(M.row_fib, (size_t)(In + 1) * 4, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(M.row_task, (size_t)(In + 1) * 4, st)) != MACH_OK) return fail(s);
    if ((s = dev_alloc(M.tasks, (size_t)M.ntask_cap * 16, st)) != MACH_OK) return fail(s);
    CsfBuildArgs a;
    a.idx = static_cast<const int64_t*>(M.idx.ptr);
    a.d_count = &ds->count;
    a.K = K;
    a.dec = dec;
    a.mode = m;
    a.emax = M.emax;
    a.leaf = static_cast<uint16_t*>(M.leaf.ptr);
    a.fib_start = static_cast<uint32_t*>(M.fib_start.ptr);
    a.fib_mid = static_cast<uint32_t*>(M.fib_mid.ptr);
    a.row_fib = static_cast<uint32_t*>(M.row_fib.ptr);
    a.row_task = static_cast<uint32_t*>(M.row_task.ptr);
    a.tasks = static_cast<int4*>(M.tasks.ptr);
    a.d_nfib = &ds->nfib[m];
    a.d_ntask = &ds->ntask[m];
    a.d_err = &ds->err;
    a.scratch = csf_scr.ptr;
    if ((s = build_csf(a, st)) != MACH_OK) return fail(s);
  }
  prof_end(PROF_CSF, st, 0.0);
  for (int m = 1; m < d; ++m) dev_free(h->mode[m].idx, st);
  dev_free(sort_scr, st);
  dev_free(csf_scr, st);
  {
    SampleScalars hs;
    if (cudaMemcpyAsync(&hs, ds, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_last_error("csf build: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(MACH_ECUDA);
    }
    if (hs.err & (DEV_BADINDEX | DEV_TIMEOUT)) {
      set_last_error("csf build consistency check failed (0x%x)", hs.err);
      return fail(MACH_EINTERNAL);
    }
    for (int m = 0; m < d; ++m) {
      h->nfib[m] = hs.nfib[m];
      h->ntask[m] = hs.ntask[m];
    }
  }
  *out = h;
  return MACH_OK;
}

mach_status mach_sample(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims, double p, uint64_t seed,
                        void* stream, mach_sample_t* out) {
  return sample_impl(x_dev, dtype, d, dims, p, seed, stream, out, false);
}

mach_status mach_sample_host(const void* x_host, mach_dtype dtype, int d, const int64_t* dims, double p,
                             uint64_t seed, int64_t chunk_entries, void* stream, mach_sample_t* out) {
  const int64_t align = sampler_chunk_align();
  if (chunk_entries == 0) chunk_entries = (int64_t)1 << 28;
  if (chunk_entries < 0 || chunk_entries % align != 0) {
    set_last_error("chunk_entries must be a positive multiple of %lld", (long long)align);
    return MACH_EINVAL;
  }
  HostStream hst;
  hst.chunk_entries = chunk_entries;
  return sample_impl(x_host, dtype, d, dims, p, seed, stream, out, false, hst);
}

mach_status mach_sample_skip(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims, double p,
                             uint64_t seed, void* stream, mach_sample_t* out) {
  return sample_impl(x_dev, dtype, d, dims, p, seed, stream, out, true);
}

mach_status mach_sample_count(mach_sample_t s, int64_t* n_kept) {
  if (!s || !n_kept) return MACH_EINVAL;
  *n_kept = s->K;
  return MACH_OK;
}

mach_status mach_sample_indices(mach_sample_t s, int64_t* idx_dev, int64_t cap, void* stream) {
  if (!s || (!idx_dev && s->K > 0)) return MACH_EINVAL;
  if (cap < s->K) return MACH_EINVAL;
  if (s->K == 0) return MACH_OK;
  MACH_CUDA_TRY(cudaMemcpyAsync(idx_dev, s->idx.ptr, (size_t)s->K * 8, cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
  return MACH_OK;
}

mach_status mach_sample_values(mach_sample_t s, void* val_dev, int64_t cap, void* stream) {
  if (!s || (!val_dev && s->K > 0)) return MACH_EINVAL;
  if (cap < s->K) return MACH_EINVAL;
  if (s->K == 0) return MACH_OK;
  MACH_CUDA_TRY(cudaMemcpyAsync(val_dev, s->val.ptr, (size_t)s->K * dtype_size(s->dt), cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
  return MACH_OK;
}

mach_status mach_sample_fibers(mach_sample_t s, int mode, int64_t* n_fibers) {
  if (!s || !n_fibers || mode < 0 || mode >= s->d) return MACH_EINVAL;
  uint32_t v = 0;
  MACH_CUDA_TRY(cudaMemcpyAsync(&v, &s->dscal()->nfib[mode], 4, cudaMemcpyDeviceToHost, s->stream));
  MACH_CUDA_TRY(cudaStreamSynchronize(s->stream));
  *n_fibers = v;
  return MACH_OK;
}

mach_status mach_sample_stats(mach_sample_t s, int64_t* eig_calls, int64_t* eig_iters, int64_t* eig_unconverged,
                              unsigned* device_flags) {
  if (!s) return MACH_EINVAL;
  SampleScalars hs;
  MACH_CUDA_TRY(cudaMemcpyAsync(&hs, s->dscal(), sizeof(hs), cudaMemcpyDeviceToHost, s->stream));
  MACH_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (eig_calls) *eig_calls = (int64_t)hs.eig_stats[0];
  if (eig_iters) *eig_iters = (int64_t)hs.eig_stats[1];
  if (eig_unconverged) *eig_unconverged = (int64_t)hs.eig_stats[2];
  if (device_flags) *device_flags = hs.err;
  return MACH_OK;
}

mach_status mach_sample_free(mach_sample_t s) {
  if (!s) return MACH_EINVAL;
  cudaStreamSynchronize(s->stream);
  free_sample(s);
  cudaStreamSynchronize(s->stream);
  delete s;
  return MACH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// HOOI driver
// ---------------------------------------------------------------------------
namespace {

mach_status check_ranks(const mach_sample_s* h, const int* ranks) {
  const int d = h->d;
  for (int k = 0; k < d; ++k) {
    if (ranks[k] < 1 || ranks[k] > kMaxRank || ranks[k] > h->dims[k]) {
      set_last_error("rank %d of mode %d outside [1, min(I_k, %d)]", ranks[k], k, kMaxRank);
      return MACH_EINVAL;
    }
  }
  for (int n = 0; n < d; ++n) {
    int64_t J = 1;
    for (int k = 0; k < d; ++k)
      if (k != n) J *= ranks[k];
    if (J > kMaxJ || ranks[n] > J) {
      set_last_error("mode %d: prod of other ranks %lld must be in [r_n, %d]", n, (long long)J, kMaxJ);
      return MACH_EINVAL;
    }
    if (d == 4) {
      const Cyc c = cyc(d, n);
      const int Q = ranks[c.mid[1]] * ranks[c.leaf];
      const int SQ = (Q + 31) / 32;
      if (SQ > 8 || ranks[c.mid[0]] * SQ > kMaxJ / 32) {
        set_last_error("mode %d: rank combination not supported by the 4-way chain kernel", n);
        return MACH_EINVAL;
      }
    }
  }
  return MACH_OK;
}

template <typename T>
mach_status ensure_ws(mach_sample_s* h, const int* ranks, Workspace& w) {
  const int d = h->d;
  bool same = w.ready;
  for (int k = 0; k < d && same; ++k) same = (w.ranks[k] == ranks[k]);
  if (same) return MACH_OK;
  cudaStream_t st = h->stream;
  free_ws(w, st);
  int64_t maxY = 1, maxP = 1, maxM = 1, maxIr = 1, maxI = 1;
  int maxr = 1;
  for (int n = 0; n < d; ++n) {
    int64_t J = 1;
    for (int k = 0; k < d; ++k)
      if (k != n) J *= ranks[k];
    maxY = std::max(maxY, h->dims[n] * J);
    maxP = std::max(maxP, h->mode[n].ntask_cap * J);
    maxM = std::max(maxM, std::min<int64_t>(h->dims[n], J));
    maxM = std::max(maxM, h->dims[n]);  // HOSVD Gram is I_n x I_n
    maxIr = std::max(maxIr, h->dims[n] * ranks[n]);
    maxI = std::max(maxI, h->dims[n]);
    maxr = std::max(maxr, ranks[n]);
  }
  MACH_TRY(dev_alloc(w.Y, (size_t)maxY * sizeof(T), st));
  MACH_TRY(dev_alloc(w.partial, (size_t)maxP * sizeof(T), st));
  w.partial_cap_elems = maxP;
  MACH_TRY(dev_alloc(w.C, (size_t)maxM * maxM * sizeof(T), st));
  w.gram_part_cap = std::min<int64_t>((int64_t)64 * kMaxJ * kMaxJ, 16 * maxM * maxM);
  MACH_TRY(dev_alloc(w.gram_part, (size_t)w.gram_part_cap * sizeof(T), st));
  MACH_TRY(dev_alloc(w.V, (size_t)maxM * 32 * sizeof(T), st));
  MACH_TRY(dev_alloc(w.W, (size_t)maxM * 32 * sizeof(T), st));
  MACH_TRY(dev_alloc(w.U, (size_t)maxM * 32 * sizeof(T), st));
  MACH_TRY(dev_alloc(w.Vout, eig_out_bytes((int)maxM), st));
  MACH_TRY(dev_alloc(w.theta, (size_t)32 * sizeof(double), st));
  MACH_TRY(dev_alloc(w.A64, (size_t)maxIr * sizeof(double), st));
  // per-CTA partial Grams of the FP64 Cholesky QR (lsv_finish grid <= 2 SMs worth)
  MACH_TRY(dev_alloc(w.gram64, (size_t)(2 * num_sms() + 2) * kMaxRank * kMaxRank * sizeof(double), st));
  MACH_TRY(dev_alloc(w.ytpart, (size_t)64 * std::max<int64_t>(maxM, 1) * kMaxRank * sizeof(T), st));
  MACH_TRY(dev_alloc(w.rinv, (size_t)kMaxRank * kMaxRank * sizeof(double), st));
  for (int k = 0; k < d; ++k) MACH_TRY(dev_alloc(w.fac[k], (size_t)h->dims[k] * ranks[k] * sizeof(T) + 64, st));
  for (int k = 0; k < d; ++k) MACH_TRY(dev_alloc(w.basis[k], (size_t)maxM * 32 * sizeof(T), st));
  MACH_TRY(dev_alloc(w.eig_part, eig_part_elems((int)maxM) * sizeof(T), st));
#ifdef MACH_POISON_WS
  // debugging aid: every workspace word starts as a NaN, so that a read of a
  // word no kernel has written shows in the results
  {
    DevBuf* bufs[] = {&w.Y, &w.partial, &w.C, &w.gram_part, &w.V, &w.W, &w.U, &w.Vout, &w.theta, &w.A64,
                      &w.gram64, &w.ytpart, &w.rinv, &w.eig_part, &w.fac[0], &w.fac[1], &w.fac[2], &w.fac[3],
                      &w.basis[0], &w.basis[1], &w.basis[2], &w.basis[3]};
    for (DevBuf* b : bufs)
      if (b->ptr) MACH_CUDA_TRY(cudaMemsetAsync(b->ptr, 0xFF, b->bytes, st));
  }
#endif
  for (int k = 0; k < d; ++k) w.ranks[k] = ranks[k];
  w.ready = true;
  (void)maxI;
  (void)maxr;
  return MACH_OK;
}

template <typename T>
mach_status run_ttmc(mach_sample_s* h, Workspace& w, const int* ranks, int n, cudaStream_t st, bool bf16 = false) {
  const int d = h->d;
  const Cyc c = cyc(d, n);
  const ModeCsf& M = h->mode[n];
  TtmcLaunch L;
  L.d = d;
  L.val = bf16 ? M.val16.ptr : M.val.ptr;
  L.vdt = h->dt;
  L.bf16 = bf16;
  L.leaf = static_cast<const uint16_t*>(M.leaf.ptr);
  L.fib_start = static_cast<const uint32_t*>(M.fib_start.ptr);
  L.fib_mid = static_cast<const uint32_t*>(M.fib_mid.ptr);
  L.tasks = static_cast<const int4*>(M.tasks.ptr);
  L.d_ntask = &h->dscal()->ntask[n];
  L.d_nfib = &h->dscal()->nfib[n];
  L.row_task = static_cast<const uint32_t*>(M.row_task.ptr);
  L.ntask_cap = M.ntask_cap;
  L.nrows = (int)h->dims[n];
  L.A_leaf = w.fac[c.leaf].ptr;
  L.A_mid0 = d >= 3 ? w.fac[c.mid[0]].ptr : nullptr;
  L.A_mid1 = d >= 4 ? w.fac[c.mid[1]].ptr : nullptr;
  L.I_leaf = (int)h->dims[c.leaf];
  L.I_mid0 = d >= 3 ? (int)h->dims[c.mid[0]] : 0;
  L.I_mid1 = d >= 4 ? (int)h->dims[c.mid[1]] : 0;
  L.r_leaf = ranks[c.leaf];
  L.r_mid0 = d >= 3 ? ranks[c.mid[0]] : 1;
  L.r_mid1 = d >= 4 ? ranks[c.mid[1]] : 1;
  int J = 1;
  for (int k = 0; k < d; ++k)
    if (k != n) J *= ranks[k];
  L.J = J;
  L.Y = w.Y.ptr;
  L.partial = w.partial.ptr;
  L.err = &h->dscal()->err;
  prof_begin(PROF_TTMC, st);
  MACH_TRY(launch_ttmc(L, sizeof(T) == 8, st));
  prof_end(PROF_TTMC, st,
           (double)h->K * ((bf16 ? 2 : dtype_size(h->dt)) + 2) + (double)h->nfib[n] * 8 +
               (double)h->dims[n] * J * sizeof(T));
  return MACH_OK;
}

// Leading r eigenvectors of the M x M Gram in w.C -> factor n (FP64 out + T copy).
template <typename T>
mach_status solve_factor(mach_sample_s* h, Workspace& w, int n, int r, int I, int J, bool jroute, bool warm,
                         int maxit, double* fac_out, cudaStream_t st, const T* Y = nullptr) {
  const int M = jroute ? J : I;
  const int b = block_size_for(M, r, !warm, sizeof(T) == 8);
  if (!Y) Y = static_cast<const T*>(w.Y.ptr);
  // Start block [Y^T A_prev, previous Ritz vectors r..b] for a warm solve
  // whose previous solve (the same mode in the previous sweep) had the same
  // Gram shape: Y^T A_prev carries one power step on the new data, the
  // previous Ritz vectors the next directions.  Otherwise [Y^T A_prev,
  // random] (warm) or random (cold).
  const bool have_prev = warm && w.basis_M[n] == M && w.basis_b[n] == b && b > r;
  MACH_TRY(launch_start_block<T>(Y, static_cast<const T*>(w.fac[n].ptr), I, J, r, b, jroute, warm,
                                 static_cast<T*>(w.V.ptr), static_cast<T*>(w.ytpart.ptr), 0x1000u + (uint32_t)n,
                                 have_prev ? static_cast<const T*>(w.basis[n].ptr) : nullptr, st));
  w.basis_M[n] = M;
  w.basis_b[n] = b;
  EigLaunch e;
  e.M = M;
  e.r = r;
  e.b = b;
  e.maxit = maxit;
  e.tol = sizeof(T) == 8 ? 1e-14 : 2e-6;
  e.V = w.V.ptr;
  e.W = w.W.ptr;
  e.U = w.U.ptr;
  e.Vout = static_cast<double*>(w.Vout.ptr);
  e.theta = static_cast<double*>(w.theta.ptr);
  e.part = w.eig_part.ptr;
  e.stats = h->dscal()->eig_stats;
  e.basis_out = w.basis[n].ptr;
  e.rr = static_cast<double*>(w.Vout.ptr);   // the split path's rotation (the factor kernel reads it)
  e.ctl = h->dscal()->eig_ctl;
  MACH_TRY(launch_eig<T>(static_cast<const T*>(w.C.ptr), e, st));
  return launch_lsv_finish<T>(Y, eig_result<T>(e), I, J, r, jroute,
                              static_cast<double*>(w.A64.ptr), static_cast<double*>(w.gram64.ptr),
                              &h->dscal()->counter, static_cast<double*>(w.rinv.ptr), &h->dscal()->err, fac_out,
                              static_cast<T*>(w.fac[n].ptr), st);
}

// The HOSVD Gram of mode n, X^_(n) X^_(n)^T (raw values), from the fibres
// along mode n (the CSF whose leaf is n: mode (n + 1) mod d), into C (I_n x
// I_n row-major).  method 0: exact, every pair of kept entries of a fibre
// accumulated in T; 1 / 2: on the tensor cores with 1 / 2 BF16 terms
// (T = float only).
template <typename T>
mach_status hosvd_gram(mach_sample_s* h, int n, int method, T* C, cudaStream_t st) {
  const int d = h->d;
  const int src = (n + 1) % d;
  const ModeCsf& M = h->mode[src];
  const int In = (int)h->dims[n];
  if (method > 0) {
    ScopedDevBuf scr(st);
    MACH_TRY(dev_alloc(scr, tc_gram_scratch_bytes(In), st));
    return launch_tc_gram<T>(M.val.ptr, h->dt, static_cast<const uint16_t*>(M.leaf.ptr),
                             static_cast<const uint32_t*>(M.fib_start.ptr), h->nfib[src], In, method,
                             static_cast<float*>(scr.ptr), C, &h->dscal()->err, st);
  }
  if (h->dt == MACH_F32)
    return launch_init_gram<float, T>(M.val.ptr, static_cast<const uint16_t*>(M.leaf.ptr),
                                      static_cast<const uint32_t*>(M.fib_start.ptr), &h->dscal()->nfib[src], h->K, In,
                                      C, st);
  return launch_init_gram<double, T>(M.val.ptr, static_cast<const uint16_t*>(M.leaf.ptr),
                                     static_cast<const uint32_t*>(M.fib_start.ptr), &h->dscal()->nfib[src], h->K, In,
                                     C, st);
}

// Keep probability from which the HOSVD Gram of the FP32 sweeps runs on the
// tensor cores: the dense tile work grows like I N and the pairwise
// products like p^2 I N, so the tiles win once a few percent are kept.
constexpr double kTcGramMinP = 0.02;

// Method of the HOSVD Gram that starts HOOI: the tensor cores for FP32 sweeps
// (2 BF16 terms; 1 for BF16_REFINE) when sweeps follow to refine the start
// and the sample is dense enough; else the exact pairwise sums.
template <typename T>
int hosvd_gram_method(const mach_sample_s* h, int n, int sweeps, bool bf16) {
  if (!std::is_same<T, float>::value || sweeps <= 0 || h->p < kTcGramMinP) return 0;
  if (h->dims[n] > tc_gram_max_order()) return 0;
  return bf16 ? 1 : 2;
}

// Iteration cap of the HOSVD eigensolve (it stops earlier once the Ritz
// residuals meet the path's tolerance; FP64 on long modes runs the cap).
// HOOI stopped after a fixed number of sweeps depends on its start, so with
// few sweeps to follow the start must be the HOSVD itself (up to 40
// iterations; 400 for MACH-HOSVD alone).  With 15 or more sweeps HOOI's own
// contraction removes the start's error (at 1000^3 with 20 sweeps, starts
// 8 and 40 iterations in give the same result to rounding), so 8 suffice.
inline int hosvd_iterations(int sweeps) { return sweeps <= 0 ? 400 : sweeps >= 15 ? 8 : 40; }

// HOSVD of X^: A_n = leading eigenvectors of X^_(n) X^_(n)^T.
template <typename T>
mach_status hosvd_start(mach_sample_s* h, Workspace& w, const int* ranks, int sweeps, double* const* factors,
                        cudaStream_t st, bool bf16 = false) {
  const int d = h->d;
  for (int n = 0; n < d; ++n) {
    const int In = (int)h->dims[n];
    prof_begin(PROF_INITGRAM, st);
    MACH_TRY(hosvd_gram<T>(h, n, hosvd_gram_method<T>(h, n, sweeps, bf16), static_cast<T*>(w.C.ptr), st));
    const int init_it = hosvd_iterations(sweeps);
    MACH_TRY(solve_factor<T>(h, w, n, ranks[n], In, In, false, false, init_it, factors[n], st));
    prof_end(PROF_INITGRAM, st, 0.0);
  }
  return MACH_OK;
}

// Runs `count` more sweeps by capturing one (`body`) into a CUDA graph and
// replaying it: sweeps after the first issue the same launches with the same
// arguments, so the replays remove the launch gaps between the ~10 stream
// operations of every mode update.  *done counts the sweeps run.  When the
// capture or instantiation fails nothing has run, and the caller runs the
// remaining sweeps directly.
template <typename F>
mach_status replay_sweeps(cudaStream_t st, int count, F body, int* done) {
  if (count < 4) return MACH_OK;   // too few replays to repay the capture
  const size_t mark = prof_mark();
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return MACH_OK;
  }
  const long long l0 = (long long)mach_launch_count();
  const mach_status sb = body();
  const long long nlaunch = (long long)mach_launch_count() - l0;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  add_launches(-nlaunch);   // counted while capturing; they run in the replays
  std::vector<ProfRec> recs = prof_take_since(mark);
  cudaGraphExec_t ge = nullptr;
  const bool ok = sb == MACH_OK && ec == cudaSuccess && g != nullptr &&
                  cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  // event-record nodes of the profiling scopes, matched to their records
  std::vector<std::pair<cudaGraphNode_t, cudaGraphNode_t>> pnodes;
  bool profile_ok = ok;
  if (ok && !recs.empty()) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    std::map<cudaEvent_t, cudaGraphNode_t> ev2node;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      cudaEvent_t e = nullptr;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeEventRecord &&
          cudaGraphEventRecordNodeGetEvent(nd, &e) == cudaSuccess)
        ev2node[e] = nd;
    }
    for (const ProfRec& r : recs) {
      auto ia = ev2node.find(r.a), ib = ev2node.find(r.b);
      if (ia == ev2node.end() || ib == ev2node.end()) {
        profile_ok = false;
        break;
      }
      pnodes.emplace_back(ia->second, ib->second);
    }
  }
  for (const ProfRec& r : recs) {
    prof_release(r.a);
    prof_release(r.b);
  }
  if (!ok) {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return MACH_OK;
  }
  mach_status s = MACH_OK;
  for (int k = 0; k < count; ++k) {
    if (profile_ok)
      for (size_t i = 0; i < pnodes.size(); ++i) {
        cudaEvent_t a, b;
        if (!prof_replay_push(&a, &b, recs[i].kind, recs[i].bytes)) break;
        cudaGraphExecEventRecordNodeSetEvent(ge, pnodes[i].first, a);
        cudaGraphExecEventRecordNodeSetEvent(ge, pnodes[i].second, b);
      }
    if (cudaGraphLaunch(ge, st) != cudaSuccess) {
      set_last_error("sweep graph launch: %s", cudaGetErrorString(cudaGetLastError()));
      s = MACH_ECUDA;
      break;
    }
    add_launches(nlaunch);
    ++*done;
  }
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  return s;
}

constexpr int kBf16Refine = 3;   // FP32 refinement sweeps after the BF16 sweeps

template <typename T>
mach_status hooi_impl(mach_sample_s* h, const int* ranks, int sweeps, double* const* factors, double* core,
                      bool warm, cudaStream_t st, bool bf16 = false) {
  const int d = h->d;
  Workspace& w = h->ws[sizeof(T) == 8 ? 1 : 0];
  MACH_TRY(ensure_ws<T>(h, ranks, w));
  if (warm) {
    for (int k = 0; k < d; ++k)
      MACH_TRY(launch_factor_to_rowmajor<T>(factors[k], (int)h->dims[k], ranks[k], static_cast<T*>(w.fac[k].ptr),
                                            st));
  } else {
    MACH_TRY(hosvd_start<T>(h, w, ranks, sweeps, factors, st, bf16));
  }
  if (bf16 && sweeps > 0) {
    for (int n = 0; n < d; ++n) {
      ModeCsf& M = h->mode[n];
      if (!M.val16.ptr) {
        MACH_TRY(dev_alloc(M.val16, (size_t)std::max<int64_t>(h->K, 1) * 2, st));
        MACH_TRY(launch_to_bf16(M.val.ptr, h->dt, h->K, M.val16.ptr, st));
      }
    }
  }
  // BF16_REFINE: the requested sweeps read BF16 values, then kBf16Refine
  // more sweeps with the input values refine every factor (subspace
  // iteration from the BF16 solution; each sweep contracts the BF16 error
  // by the HOOI convergence factor)
  const int total = bf16 && sweeps > 0 ? sweeps + kBf16Refine : sweeps;
  auto one_sweep = [&](bool low) -> mach_status {
    for (int n = 0; n < d; ++n) {
      int J = 1;
      for (int k = 0; k < d; ++k)
        if (k != n) J *= ranks[k];
      const int In = (int)h->dims[n];
      MACH_TRY(run_ttmc<T>(h, w, ranks, n, st, low));
      prof_begin(PROF_LSV, st);
      const bool jroute = J < In;
      const int M = jroute ? J : In;
      const T* Y = static_cast<const T*>(w.Y.ptr);
      if (jroute)
        MACH_TRY(launch_gram<T>(Y, In, M, J, 1, static_cast<T*>(w.C.ptr), static_cast<T*>(w.gram_part.ptr),
                                w.gram_part_cap, st));
      else
        MACH_TRY(launch_gram<T>(Y, J, M, 1, J, static_cast<T*>(w.C.ptr), static_cast<T*>(w.gram_part.ptr),
                                w.gram_part_cap, st));
      MACH_TRY(solve_factor<T>(h, w, n, ranks[n], In, J, jroute, true, 100, factors[n], st));
      prof_end(PROF_LSV, st, 0.0);
    }
    return MACH_OK;
  };
  int sweep = 0;
  if (!bf16 && total >= 5) {
    // the first sweep settles the warm-start state of every mode; the rest
    // repeat its launches exactly and run as replays of one captured sweep
    MACH_TRY(one_sweep(false));
    sweep = 1;
    MACH_TRY(replay_sweeps(st, total - 1, [&]() { return one_sweep(false); }, &sweep));
  }
  for (; sweep < total; ++sweep) MACH_TRY(one_sweep(bf16 && sweep < sweeps));
  if (core) {
    const int n = d - 1;
    int J = 1;
    for (int k = 0; k < d; ++k)
      if (k != n) J *= ranks[k];
    if (sweeps == 0) MACH_TRY(run_ttmc<T>(h, w, ranks, n, st));
    MACH_TRY(launch_core<T>(static_cast<const T*>(w.Y.ptr), factors[n], (int)h->dims[n], J, ranks[n], 1.0 / h->p,
                            core, st));
  }
  return MACH_OK;
}

// Tucker2 (mode c kept whole, the other two compressed), Algorithm 2 with
// the n-mode products of the kept mode left out: HOSVD starts for the
// compressed modes, then sweeps over them (Gauss-Seidel), then the core.
template <typename T>
mach_status tucker2_impl(mach_sample_s* h, const int* ranks, int c, int sweeps, double* const* factors, double* core,
                         bool warm, cudaStream_t st) {
  const int cm[2] = {c == 0 ? 1 : 0, c == 2 ? 1 : 2};   // the compressed modes, increasing
  int wranks[3];
  for (int k = 0; k < 3; ++k) wranks[k] = k == c ? 1 : ranks[k];
  Workspace& w = h->ws[sizeof(T) == 8 ? 1 : 0];
  MACH_TRY(ensure_ws<T>(h, wranks, w));
  const int I_c = (int)h->dims[c];
  int64_t ymax = 1;
  for (int q = 0; q < 2; ++q) ymax = std::max<int64_t>(ymax, h->dims[cm[q]] * ranks[cm[1 - q]] * (int64_t)I_c);
  DevBuf Y2;
  MACH_TRY(dev_alloc(Y2, (size_t)ymax * sizeof(T), st));
  T* Y = static_cast<T*>(Y2.ptr);
  auto done = [&](mach_status s) {
    dev_free(Y2, st);
    return s;
  };
  mach_status s = MACH_OK;
  if (factors[c] && (s = launch_identity_colmajor(factors[c], I_c, st)) != MACH_OK) return done(s);
  if (warm) {
    for (int q = 0; q < 2; ++q)
      if ((s = launch_factor_to_rowmajor<T>(factors[cm[q]], (int)h->dims[cm[q]], ranks[cm[q]],
                                            static_cast<T*>(w.fac[cm[q]].ptr), st)) != MACH_OK)
        return done(s);
  } else {
    for (int q = 0; q < 2; ++q) {
      const int n = cm[q], In = (int)h->dims[n];
      s = hosvd_gram<T>(h, n, hosvd_gram_method<T>(h, n, sweeps, false), static_cast<T*>(w.C.ptr), st);
      if (s != MACH_OK) return done(s);
      const int init_it = hosvd_iterations(sweeps);
      if ((s = solve_factor<T>(h, w, n, ranks[n], In, In, false, false, init_it, factors[n], st)) != MACH_OK)
        return done(s);
    }
  }
  // Y_(n) for compressed mode n: the leaf level of the CSF whose leaf is the
  // other compressed mode m
  auto mode_y = [&](int q) -> mach_status {
    const int n = cm[q], m = cm[1 - q], src = (m + 1) % 3;
    const ModeCsf& M = h->mode[src];
    Tucker2Leaf a;
    a.val = M.val.ptr;
    a.leaf = static_cast<const uint16_t*>(M.leaf.ptr);
    a.fib_start = static_cast<const uint32_t*>(M.fib_start.ptr);
    a.fib_mid = static_cast<const uint32_t*>(M.fib_mid.ptr);
    a.row_fib = static_cast<const uint32_t*>(M.row_fib.ptr);
    a.rows = (int)h->dims[src];
    a.Am = w.fac[m].ptr;
    a.rm = ranks[m];
    a.row_is_n = src == n ? 1 : 0;
    a.I_n = (int)h->dims[n];
    a.I_c = I_c;
    a.Y = Y;
    return launch_tucker2_leaf<T>(a, h->dt, st);
  };
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int q = 0; q < 2; ++q) {
      const int n = cm[q], m = cm[1 - q], In = (int)h->dims[n];
      const int J = ranks[m] * I_c;
      if ((s = mode_y(q)) != MACH_OK) return done(s);
      const bool jroute = J < In;
      const int Mg = jroute ? J : In;
      prof_begin(PROF_LSV, st);
      if (jroute)
        s = launch_gram<T>(Y, In, Mg, J, 1, static_cast<T*>(w.C.ptr), static_cast<T*>(w.gram_part.ptr),
                           w.gram_part_cap, st);
      else
        s = launch_gram<T>(Y, J, Mg, 1, J, static_cast<T*>(w.C.ptr), static_cast<T*>(w.gram_part.ptr),
                           w.gram_part_cap, st);
      if (s != MACH_OK) return done(s);
      if ((s = solve_factor<T>(h, w, n, ranks[n], In, J, jroute, true, 100, factors[n], st, Y)) != MACH_OK)
        return done(s);
      prof_end(PROF_LSV, st, 0.0);
    }
  }
  if (core) {
    const int L = cm[1], O = cm[0];
    if (sweeps == 0 && (s = mode_y(1)) != MACH_OK) return done(s);
    if ((s = launch_tucker2_core<T>(Y, factors[L], (int)h->dims[L], ranks[L], ranks[O], I_c, L, O, c, 1.0 / h->p,
                                    core, st)) != MACH_OK)
      return done(s);
  }
  return done(MACH_OK);
}

}  // namespace

extern "C" {

mach_status mach_hooi(mach_sample_t s, const int* ranks, int sweeps, mach_prec prec, double* const* factors_dev,
                      double* core_dev, int warm_start, void* stream) {
  if (!s || !ranks || !factors_dev || sweeps < 0) return MACH_EINVAL;
  for (int k = 0; k < s->d; ++k)
    if (!factors_dev[k]) return MACH_EINVAL;
  MACH_TRY(check_ranks(s, ranks));
  if (s->K == 0) {
    set_last_error("the sample kept no entries: nothing to decompose");
    return MACH_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->stream = st;
  switch (prec) {
    case MACH_PREC_FP64: return hooi_impl<double>(s, ranks, sweeps, factors_dev, core_dev, warm_start != 0, st);
    case MACH_PREC_FP32: return hooi_impl<float>(s, ranks, sweeps, factors_dev, core_dev, warm_start != 0, st);
    case MACH_PREC_BF16_REFINE:
      return hooi_impl<float>(s, ranks, sweeps, factors_dev, core_dev, warm_start != 0, st, true);
  }
  return MACH_EINVAL;
}

mach_status mach_hooi_tucker2(mach_sample_t s, const int* ranks, int keep_mode, int sweeps, mach_prec prec,
                              double* const* factors_dev, double* core_dev, int warm_start, void* stream) {
  if (!s || !ranks || !factors_dev || sweeps < 0) return MACH_EINVAL;
  if (s->d != 3) {
    set_last_error("Tucker2 takes a 3-way sample");
    return MACH_EINVAL;
  }
  if (keep_mode < 0 || keep_mode > 2) return MACH_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (!factors_dev[k] && k != keep_mode) return MACH_EINVAL;
  const int c = keep_mode;
  for (int k = 0; k < 3; ++k) {
    if (k == c) continue;
    const int other = 3 - c - k;
    const int64_t J = (int64_t)ranks[other] * s->dims[c];
    if (ranks[k] < 1 || ranks[k] > kMaxRank || ranks[k] > s->dims[k] || ranks[k] > J) {
      set_last_error("rank %d of mode %d outside [1, min(I_k, %d, r_other * I_keep)]", ranks[k], k, kMaxRank);
      return MACH_EINVAL;
    }
  }
  if (s->K == 0) {
    set_last_error("the sample kept no entries: nothing to decompose");
    return MACH_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->stream = st;
  switch (prec) {
    case MACH_PREC_FP64: return tucker2_impl<double>(s, ranks, c, sweeps, factors_dev, core_dev, warm_start != 0, st);
    case MACH_PREC_FP32: return tucker2_impl<float>(s, ranks, c, sweeps, factors_dev, core_dev, warm_start != 0, st);
    default: break;
  }
  set_last_error("Tucker2 runs FP64 or FP32 sweeps");
  return MACH_EINVAL;
}

mach_status mach_hooi_batched(const mach_sample_t* samples, int B, const int* ranks, int sweeps, mach_prec prec,
                              double* const* factors_io_dev, double* const* cores_dev, int warm_start, void* stream) {
  if (B < 0 || sweeps < 0 || (B > 0 && (!samples || !ranks || !factors_io_dev))) return MACH_EINVAL;
  if (B == 0) return MACH_OK;
  if (prec != MACH_PREC_FP32) {
    set_last_error("batched HOOI runs FP32 sweeps (prec must be MACH_PREC_FP32)");
    return MACH_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mach_dtype dt = samples[0] ? samples[0]->dt : MACH_F32;
  int64_t ws_per = 0;
  for (int b = 0; b < B; ++b) {
    mach_sample_s* h = samples[b];
    if (!h) return MACH_EINVAL;
    if (h->d != 3) {
      set_last_error("batched HOOI takes 3-way samples (sample %d has %d modes)", b, h->d);
      return MACH_EINVAL;
    }
    if (h->dt != dt) {
      set_last_error("batched HOOI: every sample must hold the same value type");
      return MACH_EINVAL;
    }
    if (h->K == 0) {
      set_last_error("sample %d kept no entries: nothing to decompose", b);
      return MACH_EINVAL;
    }
    MACH_TRY(check_ranks(h, ranks));
    int64_t need = 0, ymax = 0, imax = 0;
    for (int n = 0; n < 3; ++n) {
      imax = std::max<int64_t>(imax, h->dims[n]);
      const int J = ranks[(n + 1) % 3] * ranks[(n + 2) % 3];
      if (J > batched_max_j()) {
        set_last_error("batched HOOI: mode %d has J = %d > %d (use mach_hooi)", n, J, batched_max_j());
        return MACH_EINVAL;
      }
      if (!factors_io_dev[(size_t)b * 3 + n]) return MACH_EINVAL;
      need += (h->dims[n] * ranks[n] + 31) & ~(int64_t)31;
      ymax = std::max<int64_t>(ymax, h->dims[n] * J);
    }
    if (!warm_start) ymax = std::max<int64_t>(ymax, batched_hosvd_scratch(imax));
    ws_per = std::max<int64_t>(ws_per, need + ymax);
  }
  // CTAs claim items in this order: largest first, so the long
  // decompositions start at once and the short ones fill in behind them
  std::vector<int> order((size_t)B);
  for (int b = 0; b < B; ++b) order[(size_t)b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return samples[x]->K > samples[y]->K; });
  std::vector<BatItem> items((size_t)B);
  for (int o = 0; o < B; ++o) {
    const int b = order[(size_t)o];
    mach_sample_s* h = samples[b];
    BatItem& it = items[(size_t)o];
    for (int n = 0; n < 3; ++n) {
      const ModeCsf& M = h->mode[n];
      it.mode[n].val = M.val.ptr;
      it.mode[n].leaf = static_cast<const uint16_t*>(M.leaf.ptr);
      it.mode[n].fib_start = static_cast<const uint32_t*>(M.fib_start.ptr);
      it.mode[n].fib_mid = static_cast<const uint32_t*>(M.fib_mid.ptr);
      it.mode[n].row_fib = static_cast<const uint32_t*>(M.row_fib.ptr);
      it.dims[n] = (int)h->dims[n];
      it.fac[n] = factors_io_dev[(size_t)b * 3 + n];
    }
    it.inv_p = 1.0 / h->p;
    it.core = cores_dev ? cores_dev[b] : nullptr;
    it.err = &h->dscal()->err;
    it.seed = h->seed;
  }
  const int grid = batched_grid(B);
  DevBuf items_dev, ws;
  MACH_TRY(dev_alloc(items_dev, items.size() * sizeof(BatItem) + 64, st));
  mach_status s = dev_alloc(ws, (size_t)grid * (size_t)ws_per * sizeof(float), st);
  if (s != MACH_OK) {
    dev_free(items_dev, st);
    return s;
  }
  BatArgs a;
  a.items = static_cast<const BatItem*>(items_dev.ptr);
  a.B = B;
  for (int n = 0; n < 3; ++n) a.r[n] = ranks[n];
  a.sweeps = sweeps;
  a.warm = warm_start ? 1 : 0;
  a.next = reinterpret_cast<unsigned*>(static_cast<char*>(items_dev.ptr) + items.size() * sizeof(BatItem));
  a.ws = static_cast<float*>(ws.ptr);
  a.ws_stride = ws_per;
  if (cudaMemcpyAsync(items_dev.ptr, items.data(), items.size() * sizeof(BatItem), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(a.next, 0, sizeof(unsigned), st) != cudaSuccess) {
    set_last_error("batched HOOI: %s", cudaGetErrorString(cudaGetLastError()));
    s = MACH_ECUDA;
  } else {
    s = launch_batched_hooi(a, dt, grid, st);
  }
  dev_free(items_dev, st);
  dev_free(ws, st);
  return s;
}

mach_status mach_sample_gram(mach_sample_t s, int mode, int method, double* gram_dev, void* stream) {
  if (!s || !gram_dev || mode < 0 || mode >= s->d || method < 0 || method > 2) return MACH_EINVAL;
  if (method > 0 && s->dims[mode] > tc_gram_max_order()) {
    set_last_error("tensor-core Gram: I_n = %lld above %d", (long long)s->dims[mode], tc_gram_max_order());
    return MACH_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->stream = st;
  if (s->K == 0)
    return cudaMemsetAsync(gram_dev, 0, sizeof(double) * (size_t)(s->dims[mode] * s->dims[mode]), st) == cudaSuccess
               ? MACH_OK
               : MACH_ECUDA;
  return hosvd_gram<double>(s, mode, method, gram_dev, st);
}

mach_status mach_core(mach_sample_t s, const int* ranks, double* const* factors_dev, double* core_dev,
                      void* stream) {
  if (!s || !ranks || !factors_dev || !core_dev) return MACH_EINVAL;
  MACH_TRY(check_ranks(s, ranks));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s->stream = st;
  Workspace& w = s->ws[1];
  MACH_TRY(ensure_ws<double>(s, ranks, w));
  const int d = s->d;
  for (int k = 0; k < d; ++k)
    MACH_TRY(launch_factor_to_rowmajor<double>(factors_dev[k], (int)s->dims[k], ranks[k],
                                               static_cast<double*>(w.fac[k].ptr), st));
  const int n = d - 1;
  int J = 1;
  for (int k = 0; k < d; ++k)
    if (k != n) J *= ranks[k];
  MACH_TRY(run_ttmc<double>(s, w, ranks, n, st));
  return launch_core<double>(static_cast<const double*>(w.Y.ptr), factors_dev[n], (int)s->dims[n], J, ranks[n],
                             1.0 / s->p, core_dev, st);
}

mach_status mach_sample_noalloc(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims, double p,
                                uint64_t seed, int64_t* idx_dev, void* val_dev, int64_t cap, int64_t* n_kept,
                                void* stream) {
  if (!x_dev || !dims || !n_kept || cap < 0) return MACH_EINVAL;
  if (cap > 0 && (!idx_dev || !val_dev)) return MACH_EINVAL;
  if (d < 2 || d > kMaxModes) return MACH_EINVAL;
  if (dtype != MACH_F32 && dtype != MACH_F64) return MACH_EINVAL;
  if (!(p > 0.0 && p <= 1.0)) return MACH_EINVAL;
  const size_t vs = dtype_size(dtype);
  if (((uintptr_t)x_dev & 15u) != 0 || ((uintptr_t)idx_dev & 7u) != 0 || ((uintptr_t)val_dev & (vs - 1)) != 0) {
    set_last_error("x_dev must be 16-byte aligned, idx_dev and val_dev aligned to their element size");
    return MACH_EINVAL;
  }
  int64_t N = 1;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || dims[k] > kMaxDim) {
      set_last_error("dims[%d] = %lld outside [1, %d]", k, (long long)dims[k], kMaxDim);
      return MACH_EINVAL;
    }
    N *= dims[k];
  }
  const int64_t max_n = sampler_fixed_max_entries(dtype);
  if (N > max_n) {
    set_last_error("mach_sample_noalloc: %lld entries exceed the fixed scratch limit of %lld entries for this dtype",
                   (long long)N, (long long)max_n);
    return MACH_EINVAL;
  }
  unsigned long long* fixed = nullptr;
  MACH_TRY(sampler_fixed_scratch(&fixed));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t T = (uint64_t)std::floor(p * 4294967296.0);
  int64_t* d_count = reinterpret_cast<int64_t*>(fixed);
  unsigned* d_err = reinterpret_cast<unsigned*>(fixed + 1);
  // the status word starts at zero; the count and the look-back words are
  // cleared by the launcher
  MACH_CUDA_TRY(cudaMemsetAsync(fixed + 1, 0, sizeof(unsigned long long), st));
  MACH_TRY(launch_sampler(x_dev, dtype, N, seed, T, cap, idx_dev, val_dev, d_count, d_err, fixed + 2, st));
  unsigned long long h[2] = {0, 0};
  MACH_CUDA_TRY(cudaMemcpyAsync(h, fixed, sizeof(h), cudaMemcpyDeviceToHost, st));
  MACH_CUDA_TRY(cudaStreamSynchronize(st));
  if (h[1] & DEV_TIMEOUT) return MACH_ETIMEOUT;
  *n_kept = (int64_t)h[0];
  if ((int64_t)h[0] > cap) {
    set_last_error("mach_sample_noalloc: %lld entries kept, capacity %lld", (long long)h[0], (long long)cap);
    return MACH_EINVAL;
  }
  return MACH_OK;
}

mach_status mach_error(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims, const int* ranks,
                       double* const* factors_dev, const double* core_dev, double* rel_err, double* x_norm,
                       void* stream) {
  if (!x_dev || !dims || !ranks || !factors_dev || !core_dev || !rel_err) return MACH_EINVAL;
  if (d < 2 || d > kMaxModes) return MACH_EINVAL;
  int64_t R = 1;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || ranks[k] < 1 || ranks[k] > kMaxRank || !factors_dev[k]) return MACH_EINVAL;
    R *= ranks[k];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf acc;
  MACH_TRY(dev_alloc(acc, 2 * sizeof(double), st));
  mach_status s = launch_error(x_dev, dtype, d, dims, ranks, factors_dev, core_dev, static_cast<double*>(acc.ptr), st);
  double h[2] = {0, 0};
  std::vector<double> g((size_t)R);
  if (s == MACH_OK) {
    if (cudaMemcpyAsync(h, acc.ptr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(g.data(), core_dev, sizeof(double) * R, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = MACH_ECUDA;
  }
  dev_free(acc, st);
  if (s != MACH_OK) return s;
  double g2 = 0.0;
  for (double v : g) g2 += v * v;
  const double e2 = h[0] - 2.0 * h[1] + g2;
  *rel_err = h[0] > 0 ? std::sqrt(std::max(e2, 0.0) / h[0]) : 0.0;
  if (x_norm) *x_norm = std::sqrt(h[0]);
  return MACH_OK;
}

}  // extern "C"
