// Per-mode orderings of the kept entries (needed by the mode-n TTM chain of
// Algorithm 2) and their compressed-fibre (CSF) index.
//
// Mode n uses the cyclic order (i_n, i_{n+1}, .., i_d, i_1, .., i_{n-1}); its
// fibres are the runs of entries that agree on every index but the leaf
// i_{n-1}.  Mode 1's order is the sampler's increasing-l order.  Mode n's order
// is a STABLE counting sort of mode (n+1)'s order by i_n (mode d+1 = mode 1),
// so d-1 single-key sorts produce every ordering.  A stable counting sort of
// small keys is the GPU-natural choice: per-warp-tile histograms, one device
// scan over (bin, tile), then a scatter in which each warp ranks equal keys
// of a 32-entry chunk with __match_any_sync and keeps per-bin running counts
// in shared memory.
#include "mach_internal.cuh"

#include <vector>

namespace mach {

// ----------------------------------------------------------------------------
// Generic exclusive scan (three-phase: tile sums, scan of sums, tile scan).
// ----------------------------------------------------------------------------
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_excl_scan(T v, T* total, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < (int)(blockDim.x >> 5)) sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const T r = sh[warp] + incl - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const T* in, int64_t n, T* sums) {
  __shared__ T sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  T tot;
  block_excl_scan<T>(s, &tot, sh);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
    scan_tiles(const T* in, int64_t n, T* out, const T* offsets, T* total_out) {
  __shared__ T sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = base + i < n ? in[base + i] : T(0);
    s += loc[i];
  }
  T tot;
  T run = block_excl_scan<T>(s, &tot, sh) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += loc[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *total_out = run;
}

}  // namespace

// Exclusive scan of n elements; *total_dev (if non-null) receives the sum.
// `tmp` must hold scan_tmp_elems(n) elements.
int64_t scan_tmp_elems(int64_t n) {
  int64_t tot = 0;
  while (n > kScanTile) {
    n = ceil_div(n, kScanTile);
    tot += n + 1;
  }
  return tot + 2;
}

template <typename T>
mach_status scan_exclusive(const T* in, T* out, int64_t n, T* total_dev, T* tmp, cudaStream_t st) {
  if (n <= 0) {
    if (total_dev) MACH_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(T), st));
    return MACH_OK;
  }
  const int64_t nb = ceil_div(n, kScanTile);
  if (nb == 1) {
    scan_tiles<T><<<1, kScanThreads, 0, st>>>(in, n, out, nullptr, total_dev);
    MACH_LAUNCH_CHECK();
    return MACH_OK;
  }
  T* sums = tmp;
  T* sums_scanned = tmp + nb;
  scan_tile_sums<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
  MACH_LAUNCH_CHECK();
  MACH_TRY(scan_exclusive<T>(sums, sums_scanned, nb, nullptr, tmp + 2 * nb, st));
  scan_tiles<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, sums_scanned, total_dev);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

int64_t scan_tmp_elems_total(int64_t n) {
  // generous bound for the recursive layout used above (2 nb per level)
  int64_t tot = 0;
  while (n > kScanTile) {
    n = ceil_div(n, kScanTile);
    tot += 2 * n;
  }
  return tot + 4;
}

template mach_status scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, uint32_t*,
                                              cudaStream_t);
template mach_status scan_exclusive<long long>(const long long*, long long*, int64_t, long long*, long long*,
                                               cudaStream_t);

// ----------------------------------------------------------------------------
// Stable counting sort of (l, value) by one coordinate.
// ----------------------------------------------------------------------------
namespace {

constexpr int kWT = 4096;          // entries per warp tile (128 chunks of 32)
constexpr int kWTChunks = kWT / 32;

__device__ __forceinline__ uint32_t coord_of(const Decoder& dec, uint64_t l, int mode) {
  uint32_t c[kMaxModes];
  decode(dec, l, c);
  return c[mode];
}

__global__ void cs_hist_kernel(const int64_t* __restrict__ idx, const int64_t* d_count, Decoder dec, int mode,
                               uint32_t nbins, int64_t nwt, uint32_t* __restrict__ counts) {
  extern __shared__ uint32_t hist[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* h = hist + (size_t)wib * nbins;
  for (uint32_t b = lane; b < nbins; b += 32) h[b] = 0;
  __syncwarp();
  if (wt >= nwt) return;
  const int64_t K = *d_count;
  const int64_t e0 = wt * kWT;
  for (int c = 0; c < kWTChunks; ++c) {
    const int64_t e = e0 + (int64_t)c * 32 + lane;
    if (e < K) atomicAdd(&h[coord_of(dec, (uint64_t)idx[e], mode)], 1u);
  }
  __syncwarp();
  for (uint32_t b = lane; b < nbins; b += 32) counts[(int64_t)b * nwt + wt] = h[b];
}

template <typename V>
__global__ void cs_scatter_kernel(const int64_t* __restrict__ idx, const V* __restrict__ val,
                                  const int64_t* d_count, Decoder dec, int mode, uint32_t nbins, int64_t nwt,
                                  const uint32_t* __restrict__ base, int64_t* __restrict__ idx_out,
                                  V* __restrict__ val_out) {
  extern __shared__ uint32_t run_all[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* run = run_all + (size_t)wib * nbins;
  for (uint32_t b = lane; b < nbins; b += 32) run[b] = 0;
  __syncwarp();
  if (wt >= nwt) return;
  const int64_t K = *d_count;
  const int64_t e0 = wt * kWT;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kWTChunks; ++c) {
    const int64_t e = e0 + (int64_t)c * 32 + lane;
    const bool valid = e < K;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!act) break;
    int64_t l = 0;
    V v = V(0);
    uint32_t key = 0xffffffffu;
    if (valid) {
      l = idx[e];
      v = val[e];
      key = coord_of(dec, (uint64_t)l, mode);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (valid) {
      const uint32_t rank = __popc(peers & lt);
      const uint32_t pos = base[(int64_t)key * nwt + wt] + run[key] + rank;
      idx_out[pos] = l;
      val_out[pos] = v;
    }
    __syncwarp();
    if (valid && (peers & lt) == 0) run[key] += __popc(peers);
    __syncwarp();
  }
}

}  // namespace

int64_t sort_num_wt(int64_t K) { return ceil_div(K > 0 ? K : 1, kWT); }

// Bytes of scratch for one counting sort (counts + scanned + scan tmp).
size_t sort_scratch_bytes(int64_t K, int64_t nbins) {
  const int64_t nwt = sort_num_wt(K);
  const int64_t cells = nwt * nbins;
  return (size_t)(2 * cells + scan_tmp_elems_total(cells) + 8) * sizeof(uint32_t);
}

template <typename V>
mach_status counting_sort(const int64_t* idx, const V* val, int64_t K, const int64_t* d_count, const Decoder& dec,
                          int mode, int64_t* idx_out, V* val_out, void* scratch, cudaStream_t st) {
  const uint32_t nbins = (uint32_t)dec.dims[mode];
  const int64_t nwt = sort_num_wt(K);
  const int64_t cells = nwt * nbins;
  uint32_t* counts = static_cast<uint32_t*>(scratch);
  uint32_t* scanned = counts + cells;
  uint32_t* tmp = scanned + cells;
  int wpb = (int)((96 * 1024) / ((size_t)nbins * 4));
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  const size_t smem = (size_t)wpb * nbins * 4;
  MACH_TRY(allow_max_dyn_smem(cs_hist_kernel));
  MACH_TRY(allow_max_dyn_smem(cs_scatter_kernel<V>));
  const unsigned grid = (unsigned)ceil_div(nwt, wpb);
  cs_hist_kernel<<<grid, 32 * wpb, smem, st>>>(idx, d_count, dec, mode, nbins, nwt, counts);
  MACH_LAUNCH_CHECK();
  MACH_TRY(scan_exclusive<uint32_t>(counts, scanned, cells, nullptr, tmp, st));
  cs_scatter_kernel<V><<<grid, 32 * wpb, smem, st>>>(idx, val, d_count, dec, mode, nbins, nwt, scanned, idx_out,
                                                     val_out);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template mach_status counting_sort<float>(const int64_t*, const float*, int64_t, const int64_t*, const Decoder&,
                                          int, int64_t*, float*, void*, cudaStream_t);
template mach_status counting_sort<double>(const int64_t*, const double*, int64_t, const int64_t*,
                                           const Decoder&, int, int64_t*, double*, void*, cudaStream_t);

// ----------------------------------------------------------------------------
// CSF of one mode ordering.
// ----------------------------------------------------------------------------
namespace {

// Cyclic mode layout of mode n: position 0 = n (row), positions 1..d-2 = mids,
// position d-1 = leaf = (n - 1) mod d.
struct ModeLayout {
  int d;
  int row;
  int mids[2];
  int nmid;
  int leaf;
};

__device__ __forceinline__ uint32_t pack_mid(const ModeLayout& L, const uint32_t* c) {
  if (L.nmid == 0) return 0u;
  if (L.nmid == 1) return c[L.mids[0]];
  return (c[L.mids[0]] << 16) | c[L.mids[1]];
}

__global__ void csf_flags_kernel(const int64_t* __restrict__ idx, const int64_t* d_count, Decoder dec,
                                 ModeLayout L, uint32_t* __restrict__ flags, uint16_t* __restrict__ leaf,
                                 unsigned* err) {
  const int64_t K = *d_count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[kMaxModes], p[kMaxModes];
    decode(dec, (uint64_t)idx[e], c);
    leaf[e] = (uint16_t)c[L.leaf];
    uint32_t f = 1u;
    if (e > 0) {
      decode(dec, (uint64_t)idx[e - 1], p);
      f = 0u;
      for (int k = 0; k < L.d; ++k)
        if (k != L.leaf && c[k] != p[k]) f = 1u;
      // ordering check: rows must be non-decreasing
      if (c[L.row] < p[L.row]) atomicOr(err, DEV_BADINDEX);
    }
    flags[e] = f;
  }
}

__global__ void csf_fill_kernel(const int64_t* __restrict__ idx, const int64_t* d_count, Decoder dec,
                                ModeLayout L, const uint32_t* __restrict__ flags,
                                const uint32_t* __restrict__ fid, uint32_t* __restrict__ fib_start,
                                uint32_t* __restrict__ fib_mid, uint32_t* __restrict__ row_fib,
                                const uint32_t* d_nfib) {
  const int64_t K = *d_count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K; e += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[e]) continue;
    uint32_t c[kMaxModes];
    decode(dec, (uint64_t)idx[e], c);
    const uint32_t f = fid[e];
    fib_start[f] = (uint32_t)e;
    fib_mid[f] = pack_mid(L, c);
    bool new_row = (e == 0);
    if (!new_row) {
      uint32_t p[kMaxModes];
      decode(dec, (uint64_t)idx[e - 1], p);
      new_row = p[L.row] != c[L.row];
    }
    if (new_row) row_fib[c[L.row]] = f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) fib_start[*d_nfib] = (uint32_t)K;
}

__global__ void fill_u32(uint32_t* p, int64_t n, uint32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void fill_u32_dev(uint32_t* p, int64_t n, const uint32_t* v) {
  const uint32_t x = *v;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = x;
}

// row_fib[r] = min(row_fib[r], row_fib[r+1]) from the end (empty rows point at
// the next non-empty row's first fibre).  One block; rows <= kMaxDim + 1.
__global__ void suffix_min_kernel(uint32_t* row_fib, int nrows1) {
  __shared__ uint32_t sh[1024];
  const int per = (nrows1 + 1023) / 1024;
  const int b0 = nrows1 - (threadIdx.x + 1) * per;   // thread 0 takes the LAST chunk
  uint32_t m = 0xffffffffu;
  for (int i = per - 1; i >= 0; --i) {
    const int r = b0 + i;
    if (r >= 0 && r < nrows1) {
      m = min(m, row_fib[r]);
      row_fib[r] = m;
    }
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  // exclusive suffix-min carry from chunks nearer the end (lower thread ids)
  uint32_t carry = 0xffffffffu;
  for (int t = 0; t < (int)threadIdx.x; ++t) carry = min(carry, sh[t]);
  for (int i = per - 1; i >= 0; --i) {
    const int r = b0 + i;
    if (r >= 0 && r < nrows1) row_fib[r] = min(row_fib[r], carry);
  }
}

__global__ void task_count_kernel(const uint32_t* __restrict__ row_fib, const uint32_t* __restrict__ fib_start,
                                  int nrows, uint32_t emax, uint32_t* __restrict__ ntask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const uint32_t e0 = fib_start[row_fib[r]];
  const uint32_t e1 = fib_start[row_fib[r + 1]];
  ntask[r] = (e1 - e0 + emax - 1) / emax;
}

__global__ void task_fill_kernel(const uint32_t* __restrict__ row_fib, const uint32_t* __restrict__ fib_start,
                                 int nrows, uint32_t emax, const uint32_t* __restrict__ row_task,
                                 int4* __restrict__ tasks) {
  const int r = blockIdx.x;
  const uint32_t f_lo = row_fib[r], f_hi = row_fib[r + 1];
  const uint32_t e_lo = fib_start[f_lo], e_hi = fib_start[f_hi];
  const uint32_t t0 = row_task[r];
  const uint32_t nt = row_task[r + 1] - t0;
  for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
    const uint32_t e0 = e_lo + k * emax;
    const uint32_t e1 = min(e0 + emax, e_hi);
    // fibre containing e0: last f in [f_lo, f_hi) with fib_start[f] <= e0
    uint32_t lo = f_lo, hi = f_hi;   // invariant: fib_start[lo] <= e0 < fib_start[hi]
    while (hi - lo > 1) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (fib_start[mid] <= e0) lo = mid; else hi = mid;
    }
    tasks[t0 + k] = make_int4(r, (int)e0, (int)e1, (int)lo);
  }
}

}  // namespace



size_t csf_scratch_bytes(int64_t K, int64_t nrows) {
  const int64_t n = K > nrows + 1 ? K : nrows + 1;
  return (size_t)(2 * n + scan_tmp_elems_total(n) + 16) * sizeof(uint32_t);
}

mach_status build_csf(const CsfBuildArgs& a, cudaStream_t st) {
  const int d = a.dec.d;
  ModeLayout L;
  L.d = d;
  L.row = a.mode;
  L.leaf = (a.mode + d - 1) % d;
  L.nmid = d - 2;
  for (int j = 0; j < 2; ++j) L.mids[j] = (a.mode + 1 + j) % d;
  const int nrows = (int)a.dec.dims[a.mode];
  uint32_t* flags = static_cast<uint32_t*>(a.scratch);
  const int64_t n = a.K > nrows + 1 ? a.K : nrows + 1;
  uint32_t* fid = flags + n;
  uint32_t* tmp = fid + n;
  const int threads = 256;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a.K, threads), 152 * 16));
  csf_flags_kernel<<<grid, threads, 0, st>>>(a.idx, a.d_count, a.dec, L, flags, a.leaf, a.d_err);
  MACH_LAUNCH_CHECK();
  MACH_TRY(scan_exclusive<uint32_t>(flags, fid, a.K, a.d_nfib, tmp, st));
  fill_u32_dev<<<(unsigned)ceil_div(nrows + 1, 256), 256, 0, st>>>(a.row_fib, nrows + 1, a.d_nfib);
  MACH_LAUNCH_CHECK();
  csf_fill_kernel<<<grid, threads, 0, st>>>(a.idx, a.d_count, a.dec, L, flags, fid, a.fib_start, a.fib_mid,
                                            a.row_fib, a.d_nfib);
  MACH_LAUNCH_CHECK();
  if (a.K == 0) {
    MACH_CUDA_TRY(cudaMemsetAsync(a.fib_start, 0, sizeof(uint32_t), st));
  }
  suffix_min_kernel<<<1, 1024, 0, st>>>(a.row_fib, nrows + 1);
  MACH_LAUNCH_CHECK();
  // tasks: per-row counts -> scan -> fill
  uint32_t* ntask = flags;  // reuse (nrows + 1 <= n)
  MACH_CUDA_TRY(cudaMemsetAsync(ntask, 0, sizeof(uint32_t) * (nrows + 1), st));
  task_count_kernel<<<(unsigned)ceil_div(nrows, 256), 256, 0, st>>>(a.row_fib, a.fib_start, nrows, a.emax, ntask);
  MACH_LAUNCH_CHECK();
  MACH_TRY(scan_exclusive<uint32_t>(ntask, a.row_task, nrows + 1, a.d_ntask, tmp, st));
  task_fill_kernel<<<nrows, 128, 0, st>>>(a.row_fib, a.fib_start, nrows, a.emax, a.row_task, a.tasks);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

}  // namespace mach
