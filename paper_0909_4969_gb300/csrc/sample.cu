// The MACH coin (Section 3 Remark 1; Algorithm 1 and Algorithm 2, first block;
// Theorem 1's sampling law): one Philox4x32-10 word per linear index decides
// whether the entry is kept; kept (l, value) pairs are compacted in increasing
// l.  The coin is value-independent, so the dense input is streamed once.
//
// Two kernels.  The product path of mach_sample (sample_seg_kernel, below)
// gives every warp its own contiguous segment of X and concatenates the
// segments afterwards, so no warp ever waits for another.  The decoupled
// look-back kernel (sample_kernel, first) writes final positions directly
// and needs only a small fixed scratch, which suits the allocation-free
// entry point: per CTA one control warp claims 16 KiB tiles of X (one
// atomic counter, so claim order is tile order), starts their 1-D TMA bulk
// copies into a 4-stage shared-memory ring and runs the look-back; eight
// compute warps evaluate Philox for each claimed tile, scan the keep counts
// inside the tile, and, once the tile's global offset is known and its
// bytes have landed, write the kept (l, value) pairs in order.  Every wait
// is bounded.
#include "mach_internal.cuh"

#include <cmath>
#include <mutex>

namespace mach {

namespace {

constexpr int kCompWarps = 8;
constexpr int kCompThreads = 32 * kCompWarps;
constexpr int kSampThreads = kCompThreads + 32;   // + control warp
constexpr int kSampStages = 4;
constexpr int kLag = 2;                           // compute writes tile j - kLag after counting tile j
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

template <typename V>
struct SampCfg {
  static constexpr int kCPT = sizeof(V) == 4 ? 4 : 2;     // Philox counters per thread
  static constexpr int kEPT = 4 * kCPT;                      // entries per thread
  static constexpr int kTile = kCompThreads * kEPT;          // entries per tile
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

// Exclusive prefix of tile t (one warp): walk predecessors 32 at a time until
// an inclusive prefix is met; every wait is bounded.  Returns false on timeout.
__device__ bool lookback(const SampleArgs& a, long long t, int lane, long long* out) {
  unsigned long long* st = a.tile_status;
  long long excl = 0;
  long long base = t - 1;
  long long spins = 0;
  for (;;) {
    const long long j = base - lane;
    unsigned long long v = j >= 0 ? ld_acquire_u64(&st[j]) : kFlagPre;
    while (__any_sync(0xffffffffu, (v >> 62) == 0)) {
      if (++spins > kSpinLimit) return false;
      if (spins > 16) __nanosleep(32);
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
  *out = excl;
  return true;
}

__device__ __forceinline__ void compute_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(kCompThreads) : "memory");
}

template <typename V>
__global__ void __launch_bounds__(kSampThreads) sample_kernel(SampleArgs a) {
  using C = SampCfg<V>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  V* stage_buf = reinterpret_cast<V*>(smem_raw);
  __shared__ uint64_t bar_claimed[kSampStages], bar_full[kSampStages], bar_counted[kSampStages],
      bar_prefixed[kSampStages], bar_empty[kSampStages];
  __shared__ long long stage_tile[kSampStages];
  __shared__ long long s_excl[kSampStages];
  __shared__ int s_agg[kSampStages];
  __shared__ uint32_t s_mask[kSampStages][kCompThreads];
  __shared__ int s_pre[kSampStages][kCompThreads];
  __shared__ int warp_tot[kSampStages][kCompWarps];
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const V* x = static_cast<const V*>(a.x);
  V* out_val = static_cast<V*>(a.out_val);

  if (tid == 0) {
    for (int s = 0; s < kSampStages; ++s) {
      mbar_init(&bar_claimed[s], 1);
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_counted[s], kCompWarps);
      mbar_init(&bar_prefixed[s], 1);
      mbar_init(&bar_empty[s], kCompWarps);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kCompWarps) {
    // ------------------------------- control warp -------------------------------
    auto claim = [&](int s) {  // lane 0
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
        mbar_arrive_expect_tx(&bar_full[s], bytes);
        bulk_g2s(stage_buf + (size_t)s * C::kTile, x + (int64_t)t * C::kTile, bytes, &bar_full[s]);
      } else {
        mbar_arrive(&bar_full[s]);
      }
      mbar_arrive(&bar_claimed[s]);
      return t;
    };
    bool fail = false;
    if (lane == 0)
      for (int s = 0; s < kSampStages; ++s) claim(s);
    __syncwarp();
    for (long long i = 0;; ++i) {
      const int s = (int)(i % kSampStages);
      const uint32_t ph = (uint32_t)((i / kSampStages) & 1);
      if (!mbar_wait_bounded(&bar_counted[s], ph)) {
        fail = true;
        break;
      }
      const long long t = stage_tile[s];
      if (t >= a.num_tiles) break;
      const int agg = s_agg[s];
      long long e = 0;
      if (t == 0) {
        if (lane == 0) st_release_u64(&a.tile_status[0], kFlagPre | (unsigned long long)agg);
      } else {
        if (!lookback(a, t, lane, &e)) {
          fail = true;
          break;
        }
        if (lane == 0) st_release_u64(&a.tile_status[t], kFlagPre | (unsigned long long)(e + agg));
      }
      if (lane == 0) {
        s_excl[s] = e;
        if (t == a.num_tiles - 1) *a.out_count = e + agg;
        mbar_arrive(&bar_prefixed[s]);
      }
      __syncwarp();
      // refill the previous tile's stage with tile (i - 1) + stages once
      // compute has written tile i - 1 (after this look-back, so the next
      // look-back never waits behind a write)
      if (i >= 1 && lane == 0) {
        const int sp = (int)((i - 1) % kSampStages);
        const uint32_t php = (uint32_t)(((i - 1) / kSampStages) & 1);
        if (!mbar_wait_bounded(&bar_empty[sp], php)) fail = true;
        else claim(sp);
      }
      if (__any_sync(0xffffffffu, fail)) {
        fail = true;
        break;
      }
    }
    if (fail && lane == 0) {
      atomicOr(a.err, DEV_TIMEOUT);
      atomicExch(&s_abort, 1);
      // leave no bulk copy in flight: bounded wait on every stage's current phase
      for (int s = 0; s < kSampStages; ++s) {
        (void)mbar_wait_bounded(&bar_full[s], 0);
        (void)mbar_wait_bounded(&bar_full[s], 1);
      }
    }
    return;
  }

  // ------------------------------- compute warps -------------------------------
  auto count = [&](int s, long long t) {
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
    if (lane == 31) warp_tot[s][warp] = incl;
    compute_bar();
    int warp_off = 0, blk = 0;
#pragma unroll
    for (int w = 0; w < kCompWarps; ++w) {
      const int v = warp_tot[s][w];
      warp_off += (w < warp) ? v : 0;
      blk += v;
    }
    s_mask[s][tid] = mask;
    s_pre[s][tid] = warp_off + incl - cnt;
    if (tid == 0) {
      s_agg[s] = blk;
      // publish the aggregate at once (decoupled from this CTA's look-backs)
      if (t > 0) st_release_u64(&a.tile_status[t], kFlagAgg | (unsigned long long)blk);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&bar_counted[s]);
  };

  auto write = [&](long long j) -> bool {
    const int s = (int)(j % kSampStages);
    const uint32_t ph = (uint32_t)((j / kSampStages) & 1);
    if (!mbar_wait_bounded(&bar_prefixed[s], ph) || !mbar_wait_bounded(&bar_full[s], ph)) return false;
    const long long t = stage_tile[s];
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
    __syncwarp();
    if (lane == 0) mbar_arrive(&bar_empty[s]);
    return true;
  };

  long long i = 0;
  bool ok = true;
  for (;; ++i) {
    const int s = (int)(i % kSampStages);
    const uint32_t ph = (uint32_t)((i / kSampStages) & 1);
    if (!mbar_wait_bounded(&bar_claimed[s], ph)) {
      ok = false;
      break;
    }
    const long long t = stage_tile[s];
    if (t >= a.num_tiles) {
      // end marker: let the control warp see it, then drain the last writes
      if (lane == 0) mbar_arrive(&bar_counted[s]);
      break;
    }
    count(s, t);
    if (i >= kLag && !write(i - kLag)) {
      ok = false;
      break;
    }
    if (s_abort) break;
  }
  if (ok) {
    for (long long j = (i >= kLag ? i - kLag : 0); j < i; ++j)
      if (!write(j)) break;
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
  MACH_TRY(allow_max_dyn_smem(sample_kernel<V>));
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

// ----------------------------------------------------------------------------
// Segmented sampler (the product path of mach_sample).  Every warp owns a
// contiguous range of 2048-entry chunks of X and works alone.  Lane 0 keeps
// the chunk D ahead in flight from HBM into L2 with one bulk prefetch
// (cp.async.bulk.prefetch.L2), so X crosses HBM exactly once; the lanes
// evaluate the coin of their 64 consecutive entries (16 Philox calls, the
// key schedule comes with the launch), scan the keep counts with warp
// shuffles, and read only the kept values (from L2) while writing the kept
// (offset in the segment, value) pairs, in increasing l, into the warp's own
// segment of a staging buffer; seg_gather_kernel then concatenates the
// segments in warp order and restores l.  No shared memory, no block barrier and no wait on another warp:
// occupancy is set by registers alone, which keeps the integer pipes that
// carry Philox busy.
// ----------------------------------------------------------------------------
constexpr int kSegWarps = 8;
constexpr int kSegThreads = 32 * kSegWarps;
constexpr int kSegCtasPerSm = 4;
constexpr int kCallsPerLane = 16;
constexpr int kEntriesPerLane = 4 * kCallsPerLane;       // 64
constexpr int kChunk = 32 * kEntriesPerLane;             // 2048 entries per chunk
constexpr int kPrefetchAhead = 1;                        // chunks in flight per warp (more thrashes L2 at large p)

struct SegArgs {
  const void* x;
  int64_t n;
  int64_t l0;           // linear index of x[0] (a multiple of kChunk): the coin is keyed on l0 + e
  PhiloxSched ks;
  uint32_t t32;
  int keep_all;
  int64_t num_chunks;
  int64_t chunks_per_seg;
  int64_t nseg;
  int64_t seg_cap;
  uint32_t* seg_off;    // l - (first entry of the segment); a segment spans < 2^32 entries
  void* seg_val;
  int64_t* seg_count;
};

__device__ __forceinline__ void prefetch_l2_bulk(const void* g, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(bytes) : "memory");
}

// Keep bits of 8 Philox calls (32 consecutive entries from counter q_lo | k0).
__device__ __forceinline__ uint32_t coin_bits8(uint32_t q_lo, uint32_t q_hi, int k0, const SegArgs& a) {
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint4 w = philox4x32_10_sched(q_lo | (uint32_t)(k0 + k), q_hi, a.ks);
    const uint32_t b = (uint32_t)(w.x < a.t32) | ((uint32_t)(w.y < a.t32) << 1) |
                       ((uint32_t)(w.z < a.t32) << 2) | ((uint32_t)(w.w < a.t32) << 3);
    m |= b << (4 * k);
  }
  return m;
}

// STREAM: prefetch every chunk into L2 (the one-pass form, X crosses HBM
// once).  Without it (the sector-skipping form, for HBM-resident inputs)
// only the 32-byte sectors that hold kept entries leave HBM
// (1 - (1 - p)^(32 / s_in) of X); the kept set is the same.
template <typename V, bool STREAM>
__global__ void __launch_bounds__(kSegThreads, kSegCtasPerSm) sample_seg_kernel(SegArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (int64_t)blockIdx.x * kSegWarps + warp;
  if (seg >= a.nseg) return;
  const V* x = static_cast<const V*>(a.x);
  const int64_t c0 = seg * a.chunks_per_seg;
  const int64_t c1 = min(a.num_chunks, c0 + a.chunks_per_seg);
  auto prefetch = [&](int64_t c) {
    const int64_t e0 = c * kChunk;
    const int64_t ne = min((int64_t)kChunk, a.n - e0);
    const uint32_t bytes = (uint32_t)(((uint64_t)ne * sizeof(V)) & ~(uint64_t)15);
    if (bytes) prefetch_l2_bulk(x + e0, bytes);
  };
  if (STREAM && lane == 0)
    for (int d = 0; d < kPrefetchAhead && c0 + d < c1; ++d) prefetch(c0 + d);
  uint32_t* out_off = a.seg_off + (size_t)seg * a.seg_cap;
  V* out_val = static_cast<V*>(a.seg_val) + (size_t)seg * a.seg_cap;
  const V* x_seg = x + c0 * kChunk;
  const uint32_t cap = (uint32_t)a.seg_cap;
  uint32_t base = 0;
  for (int64_t c = c0; c < c1; ++c) {
    if (STREAM && lane == 0 && c + kPrefetchAhead < c1) prefetch(c + kPrefetchAhead);
    const int64_t e_lane = c * kChunk + (int64_t)lane * kEntriesPerLane;
    // q0 = (l0 + e_lane) / 4 is a multiple of 16, so the lane's 16 counters
    // differ in the low word only
    const uint64_t q0 = (uint64_t)(a.l0 + e_lane) >> 2;
    const uint32_t q_lo = (uint32_t)q0, q_hi = (uint32_t)(q0 >> 32);
    uint64_t mask;
    if (a.keep_all) {
      mask = ~0ull;
    } else {
      const uint32_t lo = coin_bits8(q_lo, q_hi, 0, a);
      const uint32_t hi = coin_bits8(q_lo, q_hi, 8, a);
      mask = ((uint64_t)hi << 32) | lo;
    }
    if (c == a.num_chunks - 1) {
      const int64_t valid = a.n - e_lane;
      if (valid < kEntriesPerLane) mask &= valid <= 0 ? 0ull : ((1ull << valid) - 1ull);
    }
    const int cnt = __popcll(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t pos = base + (uint32_t)(incl - cnt);
    const uint32_t off_lane = (uint32_t)((c - c0) * kChunk) + (uint32_t)(lane * kEntriesPerLane);
    while (mask) {
      const uint32_t off = off_lane + (uint32_t)(__ffsll((long long)mask) - 1);
      mask &= mask - 1;
      if (pos < cap) {
        out_off[pos] = off;
        out_val[pos] = __ldg(x_seg + off);
      }
      ++pos;
    }
    base += (uint32_t)tot;
  }
  if (lane == 0) a.seg_count[seg] = base;
}

// Concatenate the segments in warp order into idx / val[0, K); block c
// copies segment c.  Segments that overflowed their capacity are flagged
// (the host then reruns with the exact capacity).
template <typename V>
__global__ void __launch_bounds__(256) seg_gather_kernel(const int64_t* __restrict__ seg_count,
                                                         const int64_t* __restrict__ seg_start, int64_t seg_cap,
                                                         int64_t seg_span, int64_t nseg_chunk, int64_t chunk_entries,
                                                         const uint32_t* __restrict__ seg_off,
                                                         const V* __restrict__ seg_val, int64_t* __restrict__ idx,
                                                         V* __restrict__ val, int64_t out_cap, unsigned* err) {
  const int64_t c = blockIdx.x;
  const int64_t off = seg_start[c];   // exclusive scan of the segment counts
  const int64_t cnt = seg_count[c];
  if (cnt > seg_cap) {
    if (threadIdx.x == 0) atomicOr(err, DEV_OVERFLOW);
    return;
  }
  if (off + cnt > out_cap) {
    if (threadIdx.x == 0) atomicOr(err, DEV_OVERFLOW);
    return;
  }
  // segment c is segment c % nseg_chunk of input chunk c / nseg_chunk
  const int64_t l0 = (int64_t)(c / nseg_chunk) * chunk_entries + (int64_t)(c % nseg_chunk) * seg_span;
  const uint32_t* so = seg_off + (size_t)c * seg_cap;
  const V* sv = seg_val + (size_t)c * seg_cap;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    idx[off + i] = l0 + so[i];
    val[off + i] = sv[i];
  }
}

template <typename V, bool STREAM>
mach_status launch_seg_t(const void* x, int64_t n, int64_t l0, uint64_t seed, uint64_t T, const SegPlan& pl,
                         uint32_t* seg_off, void* seg_val, int64_t* seg_count, cudaStream_t st) {
  SegArgs a;
  a.x = x;
  a.n = n;
  a.l0 = l0;
  a.ks = make_philox_sched(seed);
  a.keep_all = T >= (1ull << 32) ? 1 : 0;
  a.t32 = a.keep_all ? 0xffffffffu : (uint32_t)T;
  a.num_chunks = ceil_div(n, kChunk);
  a.chunks_per_seg = pl.chunks_per_seg;
  a.nseg = pl.nseg;
  a.seg_cap = pl.seg_cap;
  a.seg_off = seg_off;
  a.seg_val = seg_val;
  a.seg_count = seg_count;
  const int64_t grid = ceil_div(pl.nseg, kSegWarps);
  sample_seg_kernel<V, STREAM><<<(unsigned)grid, kSegThreads, 0, st>>>(a);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

}  // namespace

SegPlan plan_segments(int64_t n, mach_dtype dt, double q) {
  (void)dt;
  // one segment per resident warp
  const int64_t num_chunks = std::max<int64_t>(1, ceil_div(n, kChunk));
  int64_t nseg = std::min<int64_t>(num_chunks, (int64_t)num_sms() * kSegCtasPerSm * kSegWarps);
  SegPlan pl;
  pl.chunks_per_seg = ceil_div(num_chunks, nseg);
  pl.nseg = ceil_div(num_chunks, pl.chunks_per_seg);
  const double per = (double)pl.chunks_per_seg * (double)kChunk;
  const double mean = per * q;
  int64_t cap = (int64_t)(mean + 8.0 * std::sqrt(mean * (1.0 - q) + 1.0) + 64.0);
  if (cap > (int64_t)per || q >= 1.0) cap = (int64_t)per;
  pl.seg_cap = std::max<int64_t>(cap, 1);
  return pl;
}

mach_status launch_sampler_seg(const void* x, mach_dtype dt, int64_t n, int64_t l0, uint64_t seed, uint64_t T,
                               const SegPlan& pl, uint32_t* seg_off, void* seg_val, int64_t* seg_count,
                               cudaStream_t st, bool skip) {
  if (l0 % kChunk != 0) return MACH_EINVAL;
  if (dt == MACH_F32)
    return skip ? launch_seg_t<float, false>(x, n, l0, seed, T, pl, seg_off, seg_val, seg_count, st)
                : launch_seg_t<float, true>(x, n, l0, seed, T, pl, seg_off, seg_val, seg_count, st);
  return skip ? launch_seg_t<double, false>(x, n, l0, seed, T, pl, seg_off, seg_val, seg_count, st)
              : launch_seg_t<double, true>(x, n, l0, seed, T, pl, seg_off, seg_val, seg_count, st);
}

mach_status launch_seg_gather(mach_dtype dt, const SegPlan& pl, int64_t nseg_total, int64_t chunk_entries,
                              const int64_t* seg_count, const int64_t* seg_start, const uint32_t* seg_off,
                              const void* seg_val, int64_t* idx, void* val, int64_t out_cap, unsigned* d_err,
                              cudaStream_t st) {
  const int64_t span = pl.chunks_per_seg * kChunk;
  if (dt == MACH_F32)
    seg_gather_kernel<float><<<(unsigned)nseg_total, 256, 0, st>>>(
        seg_count, seg_start, pl.seg_cap, span, pl.nseg, chunk_entries, seg_off, static_cast<const float*>(seg_val),
        idx, static_cast<float*>(val), out_cap, d_err);
  else
    seg_gather_kernel<double><<<(unsigned)nseg_total, 256, 0, st>>>(
        seg_count, seg_start, pl.seg_cap, span, pl.nseg, chunk_entries, seg_off,
        static_cast<const double*>(seg_val), idx, static_cast<double*>(val), out_cap, d_err);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

int64_t sampler_chunk_align() { return kChunk; }

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

// ----------------------------------------------------------------------------
// Fixed device scratch of the allocation-free sampling entry point: word 0
// the kept count, word 1 the status bits, word 2 the tile counter, words
// 3.. the look-back status of each tile.  4 MiB: 524285 tiles, i.e. up to
// 2,147,471,360 FP32 or 1,073,735,680 FP64 entries per call.  One copy per
// device, so calls that overlap on one device race on it.
// ----------------------------------------------------------------------------
static __device__ __align__(256) unsigned long long g_sampler_fixed_scratch[mach::kFixedScratchWords];

namespace mach {

int64_t sampler_fixed_max_entries(mach_dtype dt) {
  const int64_t tile = dt == MACH_F32 ? SampCfg<float>::kTile : SampCfg<double>::kTile;
  return (kFixedScratchWords - 3) * tile;
}

mach_status sampler_fixed_scratch(unsigned long long** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static unsigned long long* addr[kMaxDevices] = {};
  int dev = 0;
  MACH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MACH_EINVAL;
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    MACH_CUDA_TRY(cudaGetSymbolAddress(&p, g_sampler_fixed_scratch));
    addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = addr[dev];
  return MACH_OK;
}

}  // namespace mach
