// The MACH coin (Section 3 Remark 1; Algorithm 1 and Algorithm 2, first block;
// Theorem 1's sampling law): one Philox4x32-10 word per linear index decides
// whether the entry is kept; kept (l, value) pairs are compacted in increasing
// l.  The coin is value-independent, so the dense input is streamed once.
//
// GB300 design: persistent CTAs (4 per SM) claim 16 KiB tiles of X through
// one atomic counter and stream them into a 3-stage shared-memory ring with
// 1-D TMA bulk copies completed on mbarriers.  Because the coin does not
// depend on the data, a CTA settles a tile's place in the output as soon as
// it claims it, while the tile's bytes are still in flight: each thread
// evaluates Philox for 4 (FP32) or 2 (FP64) consecutive counters, i.e. 16 / 8
// consecutive entries; the keep masks and per-thread prefixes are cached in
// shared memory; the tile's aggregate is published and its exclusive prefix
// is found by a decoupled look-back over the per-tile status words (bounded
// spin-waits), which only walks over tiles claimed just before.  When the
// data has landed, the kept (l, value) pairs are written in order.  Philox is
// evaluated exactly once per counter.
#include "mach_internal.cuh"

namespace mach {

namespace {

constexpr int kSampThreads = 256;
constexpr int kSampWarps = kSampThreads / 32;
constexpr int kSampStages = 3;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

template <typename V>
struct SampCfg {
  static constexpr int kCPT = sizeof(V) == 4 ? 4 : 2;     // Philox counters per thread
  static constexpr int kEPT = 4 * kCPT;                      // entries per thread
  static constexpr int kTile = kSampThreads * kEPT;          // entries per tile
  static constexpr size_t kStageBytes = (size_t)kTile * sizeof(V);
};

struct SampleArgs {
  const void* x;
  int64_t n;
  uint32_t key0, key1;
  uint32_t t32;        // threshold when not keeping everything
  int keep_all;        // p == 1
  int64_t num_tiles;
  unsigned long long* tile_counter;
  unsigned long long* tile_status;
  int64_t cap;
  int64_t* out_idx;
  void* out_val;
  int64_t* out_count;
  unsigned* err;
};

// Exclusive prefix of tile t (warp 0): walk predecessors 32 at a time until
// an inclusive prefix is met; every wait is bounded.
__device__ long long lookback(const SampleArgs& a, long long t, int lane) {
  unsigned long long* st = a.tile_status;
  long long excl = 0;
  long long base = t - 1;
  long long spins = 0;
  for (;;) {
    const long long j = base - lane;
    unsigned long long v = j >= 0 ? ld_acquire_u64(&st[j]) : kFlagPre;
    while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicOr(a.err, DEV_TIMEOUT);
        return excl;
      }
      __nanosleep(32);
      if ((v >> 62) == 0) v = ld_acquire_u64(&st[j]);
    }
    const unsigned pre = __ballot_sync(0xffffffffu, (v >> 62) == 2);
    const long long val = (long long)(v & kValMask);
    if (pre) {
      const int first = __ffs(pre) - 1;
      excl += warp_sum(lane <= first ? val : 0LL);
      break;
    }
    excl += warp_sum(val);
    base -= 32;
  }
  return excl;
}

template <typename V>
__global__ void __launch_bounds__(kSampThreads) sample_kernel(SampleArgs a) {
  using C = SampCfg<V>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  V* stage_buf = reinterpret_cast<V*>(smem_raw);
  __shared__ uint64_t bars[kSampStages];
  __shared__ long long stage_tile[kSampStages];
  __shared__ uint32_t s_mask[kSampStages][kSampThreads];
  __shared__ int s_pre[kSampStages][kSampThreads];   // per-thread exclusive prefix in the tile
  __shared__ long long s_excl[kSampStages];
  __shared__ int warp_tot[kSampWarps];

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const V* x = static_cast<const V*>(a.x);
  V* out_val = static_cast<V*>(a.out_val);

  if (tid == 0) {
    for (int s = 0; s < kSampStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Thread 0: claim the next tile for stage s and start its copy.
  auto issue = [&](int s) {
    const long long t = (long long)atomicAdd(a.tile_counter, 1ull);
    stage_tile[s] = t;
    uint32_t bytes = 0;
    if (t < a.num_tiles) {
      const int64_t e0 = (int64_t)t * C::kTile;
      const int64_t ne = min((int64_t)C::kTile, a.n - e0);
      bytes = (uint32_t)(((uint64_t)ne * sizeof(V)) & ~(uint64_t)15);
    }
    if (bytes) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[s], bytes);
      bulk_g2s(stage_buf + (size_t)s * C::kTile, x + (int64_t)t * C::kTile, bytes, &bars[s]);
    } else {
      mbar_arrive(&bars[s]);
    }
  };

  // All threads: evaluate the coin for the tile claimed into stage s, cache
  // masks and prefixes, publish the aggregate, look back for the exclusive
  // prefix and publish the inclusive one.  Must be called after a
  // __syncthreads that made stage_tile[s] visible.
  auto count_ahead = [&](int s) {
    const long long t = stage_tile[s];
    if (t >= a.num_tiles) return;  // uniform
    const int64_t e_thr = (int64_t)t * C::kTile + (int64_t)tid * C::kEPT;
    const uint64_t q0 = (uint64_t)e_thr >> 2;
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < C::kCPT; ++j) {
      const uint64_t q = q0 + j;
      const uint4 w = philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), a.key0, a.key1);
      uint32_t b;
      if (a.keep_all) {
        b = 0xFu;
      } else {
        b = (uint32_t)(w.x < a.t32) | ((uint32_t)(w.y < a.t32) << 1) | ((uint32_t)(w.z < a.t32) << 2) |
            ((uint32_t)(w.w < a.t32) << 3);
      }
      mask |= b << (4 * j);
    }
    const int64_t valid = a.n - e_thr;
    if (valid < C::kEPT) mask &= valid <= 0 ? 0u : ((1u << valid) - 1u);
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int warp_off = 0, blk = 0;
#pragma unroll
    for (int w = 0; w < kSampWarps; ++w) {
      const int v = warp_tot[w];
      warp_off += (w < warp) ? v : 0;
      blk += v;
    }
    s_mask[s][tid] = mask;
    s_pre[s][tid] = warp_off + incl - cnt;
    if (warp == 0) {
      long long e = 0;
      if (t == 0) {
        if (lane == 0) st_release_u64(&a.tile_status[0], kFlagPre | (unsigned long long)blk);
      } else {
        if (lane == 0) st_release_u64(&a.tile_status[t], kFlagAgg | (unsigned long long)blk);
        e = lookback(a, t, lane);
        if (lane == 0) st_release_u64(&a.tile_status[t], kFlagPre | (unsigned long long)(e + blk));
      }
      if (lane == 0) {
        s_excl[s] = e;
        if (t == a.num_tiles - 1) *a.out_count = e + blk;
      }
    }
    __syncthreads();  // warp_tot reuse, s_excl visible
  };

  for (int s = 0; s < kSampStages; ++s) {
    if (tid == 0) issue(s);
    __syncthreads();
    count_ahead(s);
  }

  uint32_t parity = 0;
  int s = 0;
  for (;;) {
    const bool ok = mbar_wait_bounded(&bars[s], (parity >> s) & 1u);
    parity ^= 1u << s;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.err, DEV_TIMEOUT);
      for (int k = 1; k < kSampStages; ++k) {
        const int s2 = (s + k) % kSampStages;
        (void)mbar_wait_bounded(&bars[s2], (parity >> s2) & 1u);
      }
      break;
    }
    const long long t = stage_tile[s];
    if (t >= a.num_tiles) break;

    const V* buf = stage_buf + (size_t)s * C::kTile;
    const int64_t e_tile = (int64_t)t * C::kTile;
    const int64_t tile_n = min((int64_t)C::kTile, a.n - e_tile);
    const int64_t n_staged = (int64_t)((((uint64_t)tile_n * sizeof(V)) & ~(uint64_t)15) / sizeof(V));
    const int64_t e_thr = e_tile + (int64_t)tid * C::kEPT;
    uint32_t mask = s_mask[s][tid];
    long long pos = s_excl[s] + s_pre[s][tid];
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const int64_t l = e_thr + b;
      const int64_t in_tile = l - e_tile;
      const V v = in_tile < n_staged ? buf[in_tile] : x[l];
      if (pos < a.cap) {
        a.out_idx[pos] = l;
        out_val[pos] = v;
      } else {
        atomicOr(a.err, DEV_OVERFLOW);
      }
      ++pos;
    }
    __syncthreads();
    if (tid == 0) issue(s);
    __syncthreads();
    count_ahead(s);
    s = (s + 1 == kSampStages) ? 0 : s + 1;
  }
}

template <typename V>
mach_status launch_sampler_t(const void* x, int64_t n, uint64_t seed, uint64_t T, int64_t cap, int64_t* idx,
                             void* val, int64_t* d_count, unsigned* d_err, unsigned long long* scratch,
                             cudaStream_t st) {
  using C = SampCfg<V>;
  const int64_t num_tiles = ceil_div(n, C::kTile);
  // scratch: [0] tile counter, [1..num_tiles] tile status
  MACH_CUDA_TRY(cudaMemsetAsync(scratch, 0, (size_t)(num_tiles + 1) * sizeof(unsigned long long), st));
  MACH_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
  const size_t smem = kSampStages * C::kStageBytes;
  MACH_CUDA_TRY(cudaFuncSetAttribute(sample_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MACH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_kernel<V>, kSampThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > num_tiles) grid = num_tiles;
  if (grid < 1) grid = 1;
  SampleArgs a;
  a.x = x;
  a.n = n;
  a.key0 = (uint32_t)(seed & 0xffffffffu);
  a.key1 = (uint32_t)(seed >> 32);
  a.keep_all = T >= (1ull << 32) ? 1 : 0;
  a.t32 = a.keep_all ? 0xffffffffu : (uint32_t)T;
  a.num_tiles = num_tiles;
  a.tile_counter = scratch;
  a.tile_status = scratch + 1;
  a.cap = cap;
  a.out_idx = idx;
  a.out_val = val;
  a.out_count = d_count;
  a.err = d_err;
  sample_kernel<V><<<(unsigned)grid, kSampThreads, smem, st>>>(a);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

}  // namespace

int64_t sampler_scratch_words(int64_t n, mach_dtype dt) {
  const int64_t tile = dt == MACH_F32 ? SampCfg<float>::kTile : SampCfg<double>::kTile;
  return ceil_div(n, tile) + 1;
}

mach_status launch_sampler(const void* x, mach_dtype dt, int64_t n, uint64_t seed, uint64_t T, int64_t cap,
                           int64_t* idx, void* val, int64_t* d_count, unsigned* d_err,
                           unsigned long long* scratch, cudaStream_t st) {
  if (dt == MACH_F32)
    return launch_sampler_t<float>(x, n, seed, T, cap, idx, val, d_count, d_err, scratch, st);
  return launch_sampler_t<double>(x, n, seed, T, cap, idx, val, d_count, d_err, scratch, st);
}

}  // namespace mach
