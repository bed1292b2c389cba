// Sparse tensor-times-matrix chain of Algorithm 2:
//   Y = X^ x_1 A_1^T ... x_{n-1} A_{n-1}^T x_{n+1} A_{n+1}^T ... x_d A_d^T,
// produced directly as the mode-n matricization Y_(n) (I_n x J_n, row-major).
// The n-mode products commute (Section 2.1, products along different modes),
// so the chain is evaluated fibre by fibre over the mode-n CSF:
//   z_f   = sum_{e in fibre f} x_e A_leaf[i_leaf(e), :]           (leaf level)
//   Y[i_n, (a, b)] += A_mid[i_mid(f), a] z_f[b]                     (d = 3)
//   w[(a2, b)] += A_mid2[i_mid2(f), a2] z_f[b];  on a change of i_mid1:
//   Y[i_n, (a1, a2, b)] += A_mid1[i_mid1, a1] w[(a2, b)]             (d = 4)
// Column order of Y_(n) is C-order over (r_mid1, r_mid2, r_leaf), i.e. over
// the cyclic mode order n+1, .., n-1.  Column order does not change the left
// singular vectors; for mode d it is the natural order (r_1 .. r_{d-1}).
//
// GB300 mapping: one warp per task (a segment of <= E entries of one row);
// lanes own fibres for the leaf level (factor rows of the leaf mode staged in
// shared memory with one TMA bulk copy per CTA), the warp then owns the row's
// J_n accumulators (lane j holds columns j, j+32, ..) and folds the 32 fibre
// vectors in from shared memory.  A row split over several tasks is reduced in
// task order by a fix-up kernel, so results are deterministic.
#include "mach_internal.cuh"

namespace mach {

namespace {

constexpr int kTtmcWarps = 8;
constexpr int kTtmcThreads = 32 * kTtmcWarps;
constexpr int kAcc = kMaxJ / 32;   // 32 row accumulators per lane
constexpr int kSQ = 8;             // level-2 accumulators per lane (d = 4)

template <typename T>
struct TtmcArgs {
  const void* val;            // mode-ordered values (V)
  const uint16_t* leaf;       // leaf index per entry
  const uint32_t* fib_start;  // F + 1
  const uint32_t* fib_mid;    // packed mid indices per fibre
  const int4* tasks;          // (row, e0, e1, f0)
  const uint32_t* d_ntask;
  const uint32_t* d_nfib;
  const uint32_t* row_task;   // I_n + 1
  const T* A_leaf;            // I_leaf x r_leaf row-major
  const T* A_mid0;            // I_mid0 x r_mid0 row-major (d >= 3)
  const T* A_mid1;            // I_mid1 x r_mid1 row-major (d == 4)
  int r_leaf, r_mid0, r_mid1;
  int J;                      // row length of Y
  int Q;                      // level-2 width: d == 4: r_mid1 * r_leaf, else J
  uint32_t leaf_bytes_staged; // 0 = read A_leaf from global
  T* Y;                       // I_n x J
  T* partial;                 // ntask x J
};

template <typename V, typename T, int D>
__global__ void __launch_bounds__(kTtmcThreads) ttmc_kernel(TtmcArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  __shared__ T sz[kTtmcWarps][32][kMaxRank + 1];
  __shared__ uint32_t smid[kTtmcWarps][32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const V* val = static_cast<const V*>(a.val);

  // Stage the leaf factor (the hottest gather) in shared memory.
  const T* Aleaf = a.A_leaf;
  if (a.leaf_bytes_staged) {
    T* sA = reinterpret_cast<T*>(smem_raw);
    if (tid == 0) {
      mbar_init(&bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar, a.leaf_bytes_staged);
      bulk_g2s(sA, a.A_leaf, a.leaf_bytes_staged, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0)) {
      return;  // the copy never landed; Y is left unwritten (host sees garbage, never a hang)
    }
    Aleaf = sA;
  }

  const int rl = a.r_leaf;
  const int Q = a.Q;
  const int SQ = (Q + 31) >> 5;
  int qa[kSQ > kAcc ? kSQ : kAcc], qb[kSQ > kAcc ? kSQ : kAcc];
#pragma unroll
  for (int s = 0; s < (D == 4 ? kSQ : kAcc); ++s) {
    const int q = lane + 32 * s;
    qa[s] = q / rl;
    qb[s] = q - qa[s] * rl;
  }

  const uint32_t ntask = *a.d_ntask;
  const uint32_t nfib = *a.d_nfib;
  const int gwarp = blockIdx.x * kTtmcWarps + warp;
  const int nwarps = gridDim.x * kTtmcWarps;

  for (uint32_t t = gwarp; t < ntask; t += nwarps) {
    const int4 tk = a.tasks[t];
    const int row = tk.x;
    const uint32_t e0 = (uint32_t)tk.y, e1 = (uint32_t)tk.z;
    T acc[kAcc];
#pragma unroll
    for (int s = 0; s < kAcc; ++s) acc[s] = T(0);
    T w[kSQ];
#pragma unroll
    for (int s = 0; s < kSQ; ++s) w[s] = T(0);
    uint32_t cur_a1 = 0xffffffffu;

    auto flush_w = [&]() {
      if (D == 4 && cur_a1 != 0xffffffffu) {
        const T* arow = a.A_mid0 + (size_t)cur_a1 * a.r_mid0;
#pragma unroll
        for (int r1 = 0; r1 < kMaxRank; ++r1) {
          if (r1 < a.r_mid0) {
            const T m = arow[r1];
#pragma unroll
            for (int s = 0; s < kSQ; ++s)
              if (s < SQ && r1 * SQ + s < kAcc) acc[r1 * SQ + s] += m * w[s];
          }
        }
#pragma unroll
        for (int s = 0; s < kSQ; ++s) w[s] = T(0);
      }
    };

    for (uint32_t fb = (uint32_t)tk.w;; fb += 32) {
      const uint32_t f = fb + lane;
      uint32_t fs = 0xffffffffu, fe = 0;
      if (f < nfib) {
        fs = a.fib_start[f];
        fe = a.fib_start[f + 1];
      }
      const bool valid = f < nfib && fs < e1;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      if (!vm) break;
      T z[kMaxRank];
#pragma unroll
      for (int b = 0; b < kMaxRank; ++b) z[b] = T(0);
      uint32_t mid = 0;
      if (valid) {
        const uint32_t s0 = fs > e0 ? fs : e0;
        const uint32_t s1 = fe < e1 ? fe : e1;
        for (uint32_t e = s0; e < s1; ++e) {
          const T v = (T)val[e];
          const T* ar = Aleaf + (size_t)a.leaf[e] * rl;
#pragma unroll
          for (int b = 0; b < kMaxRank; ++b)
            if (b < rl) z[b] += v * ar[b];
        }
        mid = a.fib_mid[f];
      }
#pragma unroll
      for (int b = 0; b < kMaxRank; ++b)
        if (b < rl) sz[warp][lane][b] = z[b];
      smid[warp][lane] = mid;
      __syncwarp();
      const int nv = __popc(vm);
      for (int j = 0; j < nv; ++j) {
        const T* zj = sz[warp][j];
        if (D == 2) {
#pragma unroll
          for (int s = 0; s < kAcc; ++s) {
            const int q = lane + 32 * s;
            if (q < rl) acc[s] += zj[q];
          }
        } else if (D == 3) {
          const T* arow = a.A_mid0 + (size_t)smid[warp][j] * a.r_mid0;
#pragma unroll
          for (int s = 0; s < kAcc; ++s)
            if (lane + 32 * s < Q) acc[s] += arow[qa[s]] * zj[qb[s]];
        } else {
          const uint32_t m = smid[warp][j];
          const uint32_t a1 = m >> 16, a2 = m & 0xffffu;
          if (a1 != cur_a1) {
            flush_w();
            cur_a1 = a1;
          }
          const T* arow = a.A_mid1 + (size_t)a2 * a.r_mid1;
#pragma unroll
          for (int s = 0; s < kSQ; ++s)
            if (lane + 32 * s < Q) w[s] += arow[qa[s]] * zj[qb[s]];
        }
      }
      __syncwarp();
    }
    flush_w();

    const bool single = (a.row_task[row + 1] - a.row_task[row]) == 1;
    T* dst = single ? a.Y + (size_t)row * a.J : a.partial + (size_t)t * a.J;
    if (D == 4) {
#pragma unroll
      for (int r1 = 0; r1 < kMaxRank; ++r1) {
        if (r1 < a.r_mid0) {
#pragma unroll
          for (int s = 0; s < kSQ; ++s) {
            const int q = lane + 32 * s;
            if (s < SQ && q < Q && r1 * SQ + s < kAcc) dst[r1 * Q + q] = acc[r1 * SQ + s];
          }
        }
      }
    } else {
#pragma unroll
      for (int s = 0; s < kAcc; ++s) {
        const int q = lane + 32 * s;
        if (q < a.J) dst[q] = acc[s];
      }
    }
  }
}

template <typename T>
__global__ void ttmc_fixup_kernel(const uint32_t* __restrict__ row_task, int J, const T* __restrict__ partial,
                                  T* __restrict__ Y) {
  const int row = blockIdx.x;
  const uint32_t t0 = row_task[row], t1 = row_task[row + 1];
  if (t1 - t0 == 1) return;
  for (int c = threadIdx.x; c < J; c += blockDim.x) {
    T s = T(0);
    for (uint32_t t = t0; t < t1; ++t) s += partial[(size_t)t * J + c];
    Y[(size_t)row * J + c] = s;
  }
}

}  // namespace



template <typename V, typename T, int D>
static mach_status launch_ttmc_t(const TtmcLaunch& L, cudaStream_t st) {
  TtmcArgs<T> a;
  a.val = L.val;
  a.leaf = L.leaf;
  a.fib_start = L.fib_start;
  a.fib_mid = L.fib_mid;
  a.tasks = L.tasks;
  a.d_ntask = L.d_ntask;
  a.d_nfib = L.d_nfib;
  a.row_task = L.row_task;
  a.A_leaf = static_cast<const T*>(L.A_leaf);
  a.A_mid0 = static_cast<const T*>(L.A_mid0);
  a.A_mid1 = static_cast<const T*>(L.A_mid1);
  a.r_leaf = L.r_leaf;
  a.r_mid0 = L.r_mid0;
  a.r_mid1 = L.r_mid1;
  a.J = L.J;
  a.Q = D == 4 ? L.r_mid1 * L.r_leaf : L.J;
  a.Y = static_cast<T*>(L.Y);
  a.partial = static_cast<T*>(L.partial);
  const size_t leaf_bytes = (size_t)L.I_leaf * L.r_leaf * sizeof(T);
  const size_t staged = (leaf_bytes + 15) & ~(size_t)15;
  a.leaf_bytes_staged = staged <= 96 * 1024 ? (uint32_t)staged : 0u;
  const size_t smem = a.leaf_bytes_staged;
  MACH_CUDA_TRY(cudaFuncSetAttribute(ttmc_kernel<V, T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(smem > 0 ? smem : 1)));
  int per_sm = 0;
  MACH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ttmc_kernel<V, T, D>, kTtmcThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  const int64_t need = ceil_div(L.ntask_cap, kTtmcWarps);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  ttmc_kernel<V, T, D><<<(unsigned)grid, kTtmcThreads, smem, st>>>(a);
  MACH_LAUNCH_CHECK();
  ttmc_fixup_kernel<T><<<L.nrows, 128, 0, st>>>(L.row_task, L.J, static_cast<const T*>(L.partial),
                                                 static_cast<T*>(L.Y));
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename V, typename T>
static mach_status launch_ttmc_vt(const TtmcLaunch& L, cudaStream_t st) {
  switch (L.d) {
    case 2: return launch_ttmc_t<V, T, 2>(L, st);
    case 3: return launch_ttmc_t<V, T, 3>(L, st);
    case 4: return launch_ttmc_t<V, T, 4>(L, st);
    default: return MACH_EINVAL;
  }
}

mach_status launch_ttmc(const TtmcLaunch& L, bool compute_fp64, cudaStream_t st) {
  if (L.vdt == MACH_F32) {
    return compute_fp64 ? launch_ttmc_vt<float, double>(L, st) : launch_ttmc_vt<float, float>(L, st);
  }
  return compute_fp64 ? launch_ttmc_vt<double, double>(L, st) : launch_ttmc_vt<double, float>(L, st);
}

}  // namespace mach
