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
// GB300 mapping: one warp per task (a segment of <= E entries of one row).
// The task's values and leaf indices are staged into the warp's shared-memory
// buffer with two 1-D TMA bulk copies completed on a per-warp mbarrier (one
// elected lane issues them; the warp waits on the phase).  Lanes then own
// fibres for the leaf level, reading entries from shared memory and factor
// rows of the leaf mode from shared memory (small factors, staged once per
// CTA) or through L1.  The warp owns the row's J_n accumulators (lane j holds
// columns j, j+32, ..) and folds the 32 fibre vectors in from shared memory.
// A row split over several tasks is reduced in task order by a fix-up kernel,
// so results are deterministic.
#include "mach_internal.cuh"

#include <cuda_bf16.h>

namespace mach {

namespace {

// warps per CTA: 16 for FP32 arithmetic, 8 for FP64 (register budget)
template <typename T>
struct TtmcWarps {
  static constexpr int value = sizeof(T) == 4 ? 16 : 8;
};
constexpr int kSQ = 8;                 // level-2 accumulators per lane (d = 4)
constexpr uint32_t kTaskMax = 512;     // entries per task (shared-memory staging, double-buffered)

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
  uint32_t leaf_bytes_staged; // bytes of each factor copied to shared memory
  uint32_t mid0_bytes_staged; // (0 = read it through L1)
  uint32_t mid1_bytes_staged;
  T* Y;                       // I_n x J
  T* partial;                 // ntask x J
  unsigned* err;
};

// Per-warp staging buffer: values (padded) then leaf indices (padded).
template <typename V>
struct WarpStage {
  static constexpr uint32_t kValBytes = (kTaskMax + 16) * sizeof(V);
  static constexpr uint32_t kLeafBytes = (kTaskMax + 16) * 2;
  static constexpr uint32_t kBytes = kValBytes + kLeafBytes;
};

template <typename V, typename T, int D, int ACC, int RLM>
__global__ void __launch_bounds__(32 * TtmcWarps<T>::value) ttmc_kernel(TtmcArgs<T> a) {
  constexpr int kW = TtmcWarps<T>::value;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar_fac;
  __shared__ uint64_t bar_warp[kW][2];
  __shared__ T sz[kW][32][RLM + 1];
  __shared__ uint32_t smid[kW][32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const V* val = static_cast<const V*>(a.val);
  const uint32_t fac_bytes = a.leaf_bytes_staged + a.mid0_bytes_staged + a.mid1_bytes_staged;
  unsigned char* wbuf0 = smem_raw + fac_bytes + (size_t)warp * 2 * WarpStage<V>::kBytes;

  if (tid == 0) {
    mbar_init(&bar_fac, 1);
    for (int w = 0; w < kW; ++w) {
      mbar_init(&bar_warp[w][0], 1);
      mbar_init(&bar_warp[w][1], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  // Stage the factor matrices (gathered per entry and per fibre) in shared
  // memory with TMA bulk copies, as far as they fit.
  const T* Aleaf = a.A_leaf;
  const T* Amid0 = a.A_mid0;
  const T* Amid1 = a.A_mid1;
  if (fac_bytes) {
    T* sLeaf = reinterpret_cast<T*>(smem_raw);
    T* sMid0 = reinterpret_cast<T*>(smem_raw + a.leaf_bytes_staged);
    T* sMid1 = reinterpret_cast<T*>(smem_raw + a.leaf_bytes_staged + a.mid0_bytes_staged);
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar_fac, fac_bytes);
      if (a.leaf_bytes_staged) bulk_g2s(sLeaf, a.A_leaf, a.leaf_bytes_staged, &bar_fac);
      if (a.mid0_bytes_staged) bulk_g2s(sMid0, a.A_mid0, a.mid0_bytes_staged, &bar_fac);
      if (a.mid1_bytes_staged) bulk_g2s(sMid1, a.A_mid1, a.mid1_bytes_staged, &bar_fac);
    }
    if (!mbar_wait_bounded(&bar_fac, 0)) {
      if (tid == 0) atomicOr(a.err, DEV_TIMEOUT);
      return;
    }
    if (a.leaf_bytes_staged) Aleaf = sLeaf;
    if (a.mid0_bytes_staged) Amid0 = sMid0;
    if (a.mid1_bytes_staged) Amid1 = sMid1;
  }

  const int rl = a.r_leaf;
  const int Q = a.Q;
  const int SQ = (Q + 31) >> 5;
  constexpr int NQ = D == 4 ? kSQ : ACC;
  int qa[NQ], qb[NQ];
#pragma unroll
  for (int s = 0; s < NQ; ++s) {
    const int q = lane + 32 * s;
    qa[s] = q / rl;
    qb[s] = q - qa[s] * rl;
  }

  const uint32_t ntask = *a.d_ntask;
  const uint32_t nfib = *a.d_nfib;
  const int gwarp = blockIdx.x * kW + warp;
  const int nwarps = gridDim.x * kW;
  uint32_t phase_bits = 0;
  // entries [e0, e1) of a task are staged from the 16-byte boundary below e0
  constexpr uint32_t kAlign = 16 / sizeof(uint16_t);   // 8 entries (also a multiple of 16 B of V)
  // lane 0: start the bulk copies of task tt into staging buffer `buf`
  auto stage_task = [&](uint32_t tt, int buf) {
    if (lane == 0) {
      const int4 tk = a.tasks[tt];
      const uint32_t b0 = (uint32_t)tk.y & ~(kAlign - 1);
      const uint32_t ns = (((uint32_t)tk.z - b0) + kAlign - 1) & ~(kAlign - 1);
      const uint32_t vb = ns * (uint32_t)sizeof(V), lb = ns * 2u;
      unsigned char* wb = wbuf0 + (size_t)buf * WarpStage<V>::kBytes;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar_warp[warp][buf], vb + lb);
      bulk_g2s(wb, val + b0, vb, &bar_warp[warp][buf]);
      bulk_g2s(wb + WarpStage<V>::kValBytes, a.leaf + b0, lb, &bar_warp[warp][buf]);
    }
  };
  // each warp takes a contiguous block of tasks [tb, te) and keeps its
  // accumulators across consecutive tasks of one row: one output per (warp,
  // row) run, written straight to Y when the row lies inside the block, else
  // to the partial slot of the run's first task (summed by the fix-up)
  const uint32_t per = (ntask + (uint32_t)nwarps - 1u) / (uint32_t)nwarps;
  const uint32_t tb = min(ntask, (uint32_t)gwarp * per), te = min(ntask, tb + per);
  if (tb < te) stage_task(tb, 0);
  int cur = 0;
  T acc[ACC];
#pragma unroll
  for (int s = 0; s < ACC; ++s) acc[s] = T(0);
  // d = 3: lane (h, am) = (lane >> 4, lane & 15) folds the fibres j = h,
  // h + 2, .. into row am of the (r_mid x r_leaf) block: acc3[b] +=
  // A_mid[i_mid(f_j), am] z_j[b]  (z_j read as a broadcast)
  T acc3[D == 3 ? RLM : 1];
#pragma unroll
  for (int b = 0; b < (D == 3 ? RLM : 1); ++b) acc3[b] = T(0);
  const int half = lane >> 4, am = lane & 15;
  T w[D == 4 ? kSQ : 1];
#pragma unroll
  for (int s = 0; s < (D == 4 ? kSQ : 1); ++s) w[s] = T(0);
  uint32_t cur_a1 = 0xffffffffu;
  int cur_row = -1;
  uint32_t head = 0;

  auto flush_w = [&]() {
      if (D == 4 && cur_a1 != 0xffffffffu) {
        const T* arow = Amid0 + (size_t)cur_a1 * a.r_mid0;
#pragma unroll
        for (int r1 = 0; r1 < kMaxRank; ++r1) {
          if (r1 < a.r_mid0) {
            const T m = arow[r1];
#pragma unroll
            for (int s = 0; s < kSQ; ++s)
              if (s < SQ && r1 * SQ + s < ACC) acc[r1 * SQ + s] += m * w[s];
          }
        }
#pragma unroll
        for (int s = 0; s < (D == 4 ? kSQ : 1); ++s) w[s] = T(0);
      }
    };

  auto flush_row = [&]() {
    flush_w();
    cur_a1 = 0xffffffffu;
    const uint32_t rt0 = a.row_task[cur_row], rt1 = a.row_task[cur_row + 1];
    const bool whole = rt0 >= tb && rt1 <= te;
    T* dst = whole ? a.Y + (size_t)cur_row * a.J : a.partial + (size_t)head * a.J;
    if (D == 4) {
#pragma unroll
      for (int r1 = 0; r1 < kMaxRank; ++r1) {
        if (r1 < a.r_mid0) {
#pragma unroll
          for (int s = 0; s < kSQ; ++s) {
            const int q = lane + 32 * s;
            if (s < SQ && q < Q && r1 * SQ + s < ACC) dst[r1 * Q + q] = acc[r1 * SQ + s];
          }
        }
      }
    } else if (D == 3) {
#pragma unroll
      for (int b = 0; b < (D == 3 ? RLM : 1); ++b) acc3[b] += __shfl_xor_sync(0xffffffffu, acc3[b], 16);
      if (half == 0 && am < a.r_mid0) {
#pragma unroll
        for (int b = 0; b < (D == 3 ? RLM : 1); ++b)
          if (b < rl) dst[am * rl + b] = acc3[b];
      }
    } else {
#pragma unroll
      for (int s = 0; s < ACC; ++s) {
        const int q = lane + 32 * s;
        if (q < a.J) dst[q] = acc[s];
      }
    }
#pragma unroll
    for (int s = 0; s < ACC; ++s) acc[s] = T(0);
#pragma unroll
    for (int b = 0; b < (D == 3 ? RLM : 1); ++b) acc3[b] = T(0);
  };

  for (uint32_t t = tb; t < te; ++t, cur ^= 1) {
    // prefetch the next task into the other buffer (freed at the end of the
    // previous iteration) while this one is processed
    if (t + 1 < te) stage_task(t + 1, cur ^ 1);
    const int4 tk = a.tasks[t];
    const int row = tk.x;
    const uint32_t e0 = (uint32_t)tk.y, e1 = (uint32_t)tk.z;
    const uint32_t base = e0 & ~(kAlign - 1);
    unsigned char* wbuf = wbuf0 + (size_t)cur * WarpStage<V>::kBytes;
    const V* sval = reinterpret_cast<const V*>(wbuf);
    const uint16_t* sleaf = reinterpret_cast<const uint16_t*>(wbuf + WarpStage<V>::kValBytes);
    if (row != cur_row) {
      if (cur_row >= 0) flush_row();
      cur_row = row;
      head = t;
    }
    if (!mbar_wait_bounded(&bar_warp[warp][cur], (phase_bits >> cur) & 1u)) {
      if (lane == 0) atomicOr(a.err, DEV_TIMEOUT);
      // drain the prefetch of the other buffer (bounded) before leaving
      if (t + 1 < te) (void)mbar_wait_bounded(&bar_warp[warp][cur ^ 1], (phase_bits >> (cur ^ 1)) & 1u);
      return;
    }
    phase_bits ^= 1u << cur;

    // fibre metadata of batch k + 1 is loaded while batch k is processed:
    // lane l holds fib_start / fib_mid of fibre fb + l, lane 31 also the
    // start of the fibre after the batch (the end of its own fibre)
    uint32_t fs_n, mid_n, fl_n = 0;
    {
      const uint32_t f = (uint32_t)tk.w + lane;
      fs_n = f < nfib ? a.fib_start[f] : 0xffffffffu;
      mid_n = f < nfib ? a.fib_mid[f] : 0u;
      if (lane == 31 && f + 1 <= nfib) fl_n = a.fib_start[f + 1];
    }
    for (uint32_t fb = (uint32_t)tk.w;; fb += 32) {
      const uint32_t f = fb + lane;
      const uint32_t fs = fs_n, mid_f = mid_n;
      uint32_t fe = __shfl_down_sync(0xffffffffu, fs, 1);
      if (lane == 31) fe = fl_n;
      const bool valid = f < nfib && fs < e1;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      if (!vm) break;
      {
        const uint32_t fn = f + 32;
        fs_n = fn < nfib ? a.fib_start[fn] : 0xffffffffu;
        mid_n = fn < nfib ? a.fib_mid[fn] : 0u;
        if (lane == 31 && fn + 1 <= nfib) fl_n = a.fib_start[fn + 1];
      }
      T z[RLM];
#pragma unroll
      for (int b = 0; b < RLM; ++b) z[b] = T(0);
      uint32_t mid = 0;
      if (valid) {
        const uint32_t s0 = (fs > e0 ? fs : e0) - base;
        const uint32_t s1 = (fe < e1 ? fe : e1) - base;
        if (rl == RLM && (RLM % 2) == 0 && sizeof(T) == 4) {
          // exact even rank: 8-byte loads of the factor row
          for (uint32_t e = s0; e < s1; ++e) {
            const T v = (T)sval[e];
            const float2* ar = reinterpret_cast<const float2*>(Aleaf + (size_t)sleaf[e] * RLM);
#pragma unroll
            for (int b = 0; b < RLM / 2; ++b) {
              const float2 w2 = ar[b];
              z[2 * b] += v * (T)w2.x;
              z[2 * b + 1] += v * (T)w2.y;
            }
          }
        } else {
          for (uint32_t e = s0; e < s1; ++e) {
            const T v = (T)sval[e];
            const T* ar = Aleaf + (size_t)sleaf[e] * rl;
#pragma unroll
            for (int b = 0; b < RLM; ++b)
              if (b < rl) z[b] += v * ar[b];
          }
        }
        mid = mid_f;
      }
#pragma unroll
      for (int b = 0; b < RLM; ++b)
        if (b < rl) sz[warp][lane][b] = z[b];
      smid[warp][lane] = mid;
      __syncwarp();
      const int nv = __popc(vm);
      if (D == 3) {
        if (am < a.r_mid0) {
          for (int j = half; j < nv; j += 2) {
            const T m = Amid0[(size_t)smid[warp][j] * a.r_mid0 + am];
            const T* zj = sz[warp][j];
#pragma unroll
            for (int b = 0; b < RLM; ++b) acc3[b] += m * zj[b];
          }
        }
        __syncwarp();
        continue;
      }
      for (int j = 0; j < nv; ++j) {
        const T* zj = sz[warp][j];
        if (D == 2) {
          if (lane < rl) acc[0] += zj[lane];
        } else if (D == 3) {
          const T* arow = Amid0 + (size_t)smid[warp][j] * a.r_mid0;
#pragma unroll
          for (int s = 0; s < ACC; ++s)
            if (lane + 32 * s < Q) acc[s] += arow[qa[s]] * zj[qb[s]];
        } else {
          const uint32_t m = smid[warp][j];
          const uint32_t a1 = m >> 16, a2 = m & 0xffffu;
          if (a1 != cur_a1) {
            flush_w();
            cur_a1 = a1;
          }
          const T* arow = Amid1 + (size_t)a2 * a.r_mid1;
#pragma unroll
          for (int s = 0; s < kSQ; ++s)
            if (s < SQ && lane + 32 * s < Q) w[s] += arow[qa[s]] * zj[qb[s]];
        }
      }
      __syncwarp();
    }
    __syncwarp();   // the staging buffer is reused by the next task
  }
  if (cur_row >= 0) flush_row();
}

// The 3-way chain with the fold kept in registers: lane j owns fibre j of a
// batch of 32, forms z_f (leaf level, as above), reads the mid factor row
// of the fibre and adds the outer product A_mid[i_mid(f), :] (x) z_f to its
// own copy of the row's RM x RL accumulators.  The 32 copies are summed once
// per (warp, row) run, in lane order, through a shared-memory transpose.
// Compared with the shared-memory fold above this reads no z vectors back
// from shared memory (about a third of the shared-memory loads per fibre);
// it holds RM * RL accumulators per lane, so it serves FP32 arithmetic and
// RM * RL <= 100.
template <typename V, int RM, int RL, int KW>
__global__ void __launch_bounds__(32 * KW, 1) ttmc3_kernel(TtmcArgs<float> a) {
  using T = float;
  constexpr int J = RM * RL;
  constexpr int NC = (J + 31) / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar_fac;
  __shared__ uint64_t bar_warp[KW][2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const V* val = static_cast<const V*>(a.val);
  const uint32_t fac_bytes = a.leaf_bytes_staged + a.mid0_bytes_staged;
  unsigned char* wbuf0 = smem_raw + fac_bytes + (size_t)warp * 2 * WarpStage<V>::kBytes;
  float* red = reinterpret_cast<float*>(smem_raw + fac_bytes + (size_t)KW * 2 * WarpStage<V>::kBytes) +
               (size_t)warp * 32 * 33;

  if (tid == 0) {
    mbar_init(&bar_fac, 1);
    for (int w = 0; w < KW; ++w) {
      mbar_init(&bar_warp[w][0], 1);
      mbar_init(&bar_warp[w][1], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const T* Aleaf = a.A_leaf;
  const T* Amid = a.A_mid0;
  if (fac_bytes) {
    T* sLeaf = reinterpret_cast<T*>(smem_raw);
    T* sMid = reinterpret_cast<T*>(smem_raw + a.leaf_bytes_staged);
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar_fac, fac_bytes);
      if (a.leaf_bytes_staged) bulk_g2s(sLeaf, a.A_leaf, a.leaf_bytes_staged, &bar_fac);
      if (a.mid0_bytes_staged) bulk_g2s(sMid, a.A_mid0, a.mid0_bytes_staged, &bar_fac);
    }
    if (!mbar_wait_bounded(&bar_fac, 0)) {
      if (tid == 0) atomicOr(a.err, DEV_TIMEOUT);
      return;
    }
    if (a.leaf_bytes_staged) Aleaf = sLeaf;
    if (a.mid0_bytes_staged) Amid = sMid;
  }

  const uint32_t ntask = *a.d_ntask;
  const uint32_t nfib = *a.d_nfib;
  const int gwarp = blockIdx.x * KW + warp;
  const int nwarps = gridDim.x * KW;
  uint32_t phase_bits = 0;
  constexpr uint32_t kAlign = 16 / sizeof(uint16_t);
  auto stage_task = [&](uint32_t tt, int buf) {
    if (lane == 0) {
      const int4 tk = a.tasks[tt];
      const uint32_t b0 = (uint32_t)tk.y & ~(kAlign - 1);
      const uint32_t ns = (((uint32_t)tk.z - b0) + kAlign - 1) & ~(kAlign - 1);
      const uint32_t vb = ns * (uint32_t)sizeof(V), lb = ns * 2u;
      unsigned char* wb = wbuf0 + (size_t)buf * WarpStage<V>::kBytes;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar_warp[warp][buf], vb + lb);
      bulk_g2s(wb, val + b0, vb, &bar_warp[warp][buf]);
      bulk_g2s(wb + WarpStage<V>::kValBytes, a.leaf + b0, lb, &bar_warp[warp][buf]);
    }
  };
  const uint32_t per = (ntask + (uint32_t)nwarps - 1u) / (uint32_t)nwarps;
  const uint32_t tb = min(ntask, (uint32_t)gwarp * per), te = min(ntask, tb + per);
  if (tb < te) stage_task(tb, 0);
  int cur = 0;
  T acc[J];
#pragma unroll
  for (int q = 0; q < J; ++q) acc[q] = T(0);
  int cur_row = -1;
  uint32_t head = 0;

  auto flush_row = [&]() {
    const uint32_t rt0 = a.row_task[cur_row], rt1 = a.row_task[cur_row + 1];
    const bool whole = rt0 >= tb && rt1 <= te;
    T* dst = whole ? a.Y + (size_t)cur_row * a.J : a.partial + (size_t)head * a.J;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (32 * c + j < J) red[lane * 33 + j] = acc[32 * c + j];
      __syncwarp();
      if (32 * c + lane < J) {
        T sum = T(0);
#pragma unroll 8
        for (int l = 0; l < 32; ++l) sum += red[l * 33 + lane];
        dst[32 * c + lane] = sum;
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < J; ++q) acc[q] = T(0);
  };

  for (uint32_t t = tb; t < te; ++t, cur ^= 1) {
    if (t + 1 < te) stage_task(t + 1, cur ^ 1);
    const int4 tk = a.tasks[t];
    const int row = tk.x;
    const uint32_t e0 = (uint32_t)tk.y, e1 = (uint32_t)tk.z;
    const uint32_t base = e0 & ~(kAlign - 1);
    unsigned char* wbuf = wbuf0 + (size_t)cur * WarpStage<V>::kBytes;
    const V* sval = reinterpret_cast<const V*>(wbuf);
    const uint16_t* sleaf = reinterpret_cast<const uint16_t*>(wbuf + WarpStage<V>::kValBytes);
    if (row != cur_row) {
      if (cur_row >= 0) flush_row();
      cur_row = row;
      head = t;
    }
    if (!mbar_wait_bounded(&bar_warp[warp][cur], (phase_bits >> cur) & 1u)) {
      if (lane == 0) atomicOr(a.err, DEV_TIMEOUT);
      if (t + 1 < te) (void)mbar_wait_bounded(&bar_warp[warp][cur ^ 1], (phase_bits >> (cur ^ 1)) & 1u);
      return;
    }
    phase_bits ^= 1u << cur;
    uint32_t fs_n, mid_n, fl_n = 0;
    {
      const uint32_t f = (uint32_t)tk.w + lane;
      fs_n = f < nfib ? a.fib_start[f] : 0xffffffffu;
      mid_n = f < nfib ? a.fib_mid[f] : 0u;
      if (lane == 31 && f + 1 <= nfib) fl_n = a.fib_start[f + 1];
    }
    for (uint32_t fb = (uint32_t)tk.w;; fb += 32) {
      const uint32_t f = fb + lane;
      const uint32_t fs = fs_n, mid_f = mid_n;
      uint32_t fe = __shfl_down_sync(0xffffffffu, fs, 1);
      if (lane == 31) fe = fl_n;
      const bool valid = f < nfib && fs < e1;
      if (!__ballot_sync(0xffffffffu, valid)) break;
      {
        const uint32_t fn = f + 32;
        fs_n = fn < nfib ? a.fib_start[fn] : 0xffffffffu;
        mid_n = fn < nfib ? a.fib_mid[fn] : 0u;
        if (lane == 31 && fn + 1 <= nfib) fl_n = a.fib_start[fn + 1];
      }
      if (valid) {
        T z[RL];
#pragma unroll
        for (int b = 0; b < RL; ++b) z[b] = T(0);
        const uint32_t s0 = (fs > e0 ? fs : e0) - base;
        const uint32_t s1 = (fe < e1 ? fe : e1) - base;
        for (uint32_t e = s0; e < s1; ++e) {
          const T v = (T)sval[e];
          const T* ar = Aleaf + (size_t)sleaf[e] * RL;
          if ((RL % 2) == 0) {
#pragma unroll
            for (int b = 0; b < RL / 2; ++b) {
              const float2 w2 = reinterpret_cast<const float2*>(ar)[b];
              z[2 * b] += v * w2.x;
              z[2 * b + 1] += v * w2.y;
            }
          } else {
#pragma unroll
            for (int b = 0; b < RL; ++b) z[b] += v * ar[b];
          }
        }
        T m[RM];
        const T* mr = Amid + (size_t)mid_f * RM;
        if ((RM % 2) == 0) {
#pragma unroll
          for (int i = 0; i < RM / 2; ++i) {
            const float2 w2 = reinterpret_cast<const float2*>(mr)[i];
            m[2 * i] = w2.x;
            m[2 * i + 1] = w2.y;
          }
        } else {
#pragma unroll
          for (int i = 0; i < RM; ++i) m[i] = mr[i];
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int b = 0; b < RL; ++b) acc[i * RL + b] += m[i] * z[b];
      }
    }
    __syncwarp();   // the staging buffer is reused by the next task
  }
  if (cur_row >= 0) flush_row();
}

// Rows split over several warps' task blocks: Y_row = sum of the partials of
// the runs, i.e. of the row's first task and of every later task that starts
// a warp block (t a multiple of `per`), in increasing task order.  Rows that
// lie in one block were written directly; rows without tasks are zero.
template <typename T>
__global__ void ttmc_fixup_kernel(const uint32_t* __restrict__ row_task, const uint32_t* __restrict__ d_ntask,
                                  uint32_t nwarps, int J, const T* __restrict__ partial, T* __restrict__ Y) {
  const uint32_t per = (*d_ntask + nwarps - 1u) / nwarps;   // the task kernel's block size
  const int row = blockIdx.x;
  const uint32_t t0 = row_task[row], t1 = row_task[row + 1];
  if (t1 > t0 && t0 / per == (t1 - 1) / per) return;
  for (int c = threadIdx.x; c < J; c += blockDim.x) {
    T s = T(0);
    if (t1 > t0) {
      s = partial[(size_t)t0 * J + c];
      for (uint32_t h = (t0 / per + 1) * per; h < t1; h += per) s += partial[(size_t)h * J + c];
    }
    Y[(size_t)row * J + c] = s;
  }
}

}  // namespace

uint32_t ttmc_task_max() { return kTaskMax; }

template <typename V, typename T, int D, int ACC, int RLM>
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
  a.err = L.err;
  constexpr int kW = TtmcWarps<T>::value;
  auto kern = ttmc_kernel<V, T, D, ACC, RLM>;
  cudaFuncAttributes fa;
  MACH_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0;
  MACH_CUDA_TRY(cudaGetDevice(&dev));
  MACH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t warp_bytes = (size_t)kW * 2 * WarpStage<V>::kBytes;
  size_t budget = (size_t)optin > fa.sharedSizeBytes + warp_bytes + 1024
                      ? (size_t)optin - fa.sharedSizeBytes - warp_bytes - 1024 : 0;
  // greedy: leaf factor (gathered per entry) first, then the mid factors
  auto take = [&](size_t elems) -> uint32_t {
    const size_t by = (elems * sizeof(T) + 15) & ~(size_t)15;
    if (elems == 0 || by > budget) return 0u;
    budget -= by;
    return (uint32_t)by;
  };
  a.leaf_bytes_staged = take((size_t)L.I_leaf * L.r_leaf);
  a.mid0_bytes_staged = D >= 3 ? take((size_t)L.I_mid0 * L.r_mid0) : 0u;
  a.mid1_bytes_staged = D >= 4 ? take((size_t)L.I_mid1 * L.r_mid1) : 0u;
  const size_t smem = (size_t)a.leaf_bytes_staged + a.mid0_bytes_staged + a.mid1_bytes_staged + warp_bytes;
  MACH_TRY(allow_max_dyn_smem(kern));
  int per_sm = 0;
  MACH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kW, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  const int64_t need = ceil_div(L.ntask_cap, kW);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 32 * kW, smem, st>>>(a);
  MACH_LAUNCH_CHECK();
  ttmc_fixup_kernel<T><<<L.nrows, 128, 0, st>>>(L.row_task, L.d_ntask, (uint32_t)(grid * kW), L.J,
                                                 static_cast<const T*>(L.partial), static_cast<T*>(L.Y));
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

// The register-fold 3-way chain (ttmc3_kernel) for FP32 arithmetic and the
// (r_mid, r_leaf) pairs instantiated here; false when it does not apply.
template <typename V, int RM, int RL>
static mach_status launch_ttmc3_t(const TtmcLaunch& L, cudaStream_t st) {
  constexpr int KW = RM * RL > 64 ? 12 : 16;
  TtmcArgs<float> a;
  a.val = L.val;
  a.leaf = L.leaf;
  a.fib_start = L.fib_start;
  a.fib_mid = L.fib_mid;
  a.tasks = L.tasks;
  a.d_ntask = L.d_ntask;
  a.d_nfib = L.d_nfib;
  a.row_task = L.row_task;
  a.A_leaf = static_cast<const float*>(L.A_leaf);
  a.A_mid0 = static_cast<const float*>(L.A_mid0);
  a.A_mid1 = nullptr;
  a.r_leaf = L.r_leaf;
  a.r_mid0 = L.r_mid0;
  a.r_mid1 = 1;
  a.J = L.J;
  a.Q = L.J;
  a.Y = static_cast<float*>(L.Y);
  a.partial = static_cast<float*>(L.partial);
  a.err = L.err;
  auto kern = ttmc3_kernel<V, RM, RL, KW>;
  cudaFuncAttributes fa;
  MACH_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0;
  MACH_CUDA_TRY(cudaGetDevice(&dev));
  MACH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t fixed = (size_t)KW * 2 * WarpStage<V>::kBytes + (size_t)KW * 32 * 33 * sizeof(float);
  size_t budget = (size_t)optin > fa.sharedSizeBytes + fixed + 1024 ? (size_t)optin - fa.sharedSizeBytes - fixed - 1024
                                                                    : 0;
  auto take = [&](size_t elems) -> uint32_t {
    const size_t by = (elems * sizeof(float) + 15) & ~(size_t)15;
    if (elems == 0 || by > budget) return 0u;
    budget -= by;
    return (uint32_t)by;
  };
  a.leaf_bytes_staged = take((size_t)L.I_leaf * L.r_leaf);
  a.mid0_bytes_staged = take((size_t)L.I_mid0 * L.r_mid0);
  a.mid1_bytes_staged = 0;
  const size_t smem = (size_t)a.leaf_bytes_staged + a.mid0_bytes_staged + fixed;
  MACH_TRY(allow_max_dyn_smem(kern));
  int per_sm = 0;
  MACH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * KW, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  const int64_t need = ceil_div(L.ntask_cap, KW);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 32 * KW, smem, st>>>(a);
  MACH_LAUNCH_CHECK();
  ttmc_fixup_kernel<float><<<L.nrows, 128, 0, st>>>(L.row_task, L.d_ntask, (uint32_t)(grid * KW), L.J,
                                                     static_cast<const float*>(L.partial), static_cast<float*>(L.Y));
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename V>
static bool launch_ttmc3(const TtmcLaunch& L, cudaStream_t st, mach_status* s) {
  const int rm = L.r_mid0, rl = L.r_leaf;
#define MACH_TTMC3(RM_, RL_)                          \
  if (rm == RM_ && rl == RL_) {                       \
    *s = launch_ttmc3_t<V, RM_, RL_>(L, st);          \
    return true;                                      \
  }
  MACH_TTMC3(10, 10)
  MACH_TTMC3(4, 8)
  MACH_TTMC3(8, 4)
  MACH_TTMC3(4, 4)
  MACH_TTMC3(8, 8)
  MACH_TTMC3(5, 5)
#undef MACH_TTMC3
  return false;
}

template <typename V, typename T, int D, int ACC>
static mach_status launch_ttmc_rl(const TtmcLaunch& L, cudaStream_t st) {
  // leaf-rank widths: exact for the common ranks 4, 5, 8, 10, padded otherwise
  if (L.r_leaf <= 4) return launch_ttmc_t<V, T, D, ACC, 4>(L, st);
  if (L.r_leaf == 5) return launch_ttmc_t<V, T, D, ACC, 5>(L, st);
  if (L.r_leaf <= 8) return launch_ttmc_t<V, T, D, ACC, 8>(L, st);
  if (L.r_leaf <= 10) return launch_ttmc_t<V, T, D, ACC, 10>(L, st);
  return launch_ttmc_t<V, T, D, ACC, 16>(L, st);
}

template <typename V, typename T>
static mach_status launch_ttmc_vt(const TtmcLaunch& L, cudaStream_t st) {
  if (L.d == 2) return launch_ttmc_rl<V, T, 2, 1>(L, st);
  if (L.d == 3) return launch_ttmc_rl<V, T, 3, 1>(L, st);   // half-warp fold: no ACC slots
  if (L.d == 4) {
    const int Q = L.r_mid1 * L.r_leaf;
    const int need = L.r_mid0 * ((Q + 31) / 32);
    if (need <= 4) return launch_ttmc_rl<V, T, 4, 4>(L, st);
    if (need <= 8) return launch_ttmc_rl<V, T, 4, 8>(L, st);
    if (need <= 16) return launch_ttmc_rl<V, T, 4, 16>(L, st);
    return launch_ttmc_rl<V, T, 4, 32>(L, st);
  }
  return MACH_EINVAL;
}

namespace {
template <typename V>
__global__ void to_bf16_kernel(const V* __restrict__ in, int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn((float)in[i]);
}
}  // namespace

mach_status launch_to_bf16(const void* val, mach_dtype dt, int64_t K, void* out, cudaStream_t st) {
  if (K <= 0) return MACH_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(K, 256), (int64_t)num_sms() * 16);
  if (dt == MACH_F32)
    to_bf16_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(val), K, static_cast<__nv_bfloat16*>(out));
  else
    to_bf16_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(val), K,
                                                 static_cast<__nv_bfloat16*>(out));
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

mach_status launch_ttmc(const TtmcLaunch& L, bool compute_fp64, cudaStream_t st) {
  mach_status s = MACH_OK;
  if (L.bf16) {
    if (compute_fp64) return MACH_EINVAL;
    if (L.d == 3 && launch_ttmc3<__nv_bfloat16>(L, st, &s)) return s;
    return launch_ttmc_vt<__nv_bfloat16, float>(L, st);
  }
  if (L.vdt == MACH_F32) {
    if (!compute_fp64 && L.d == 3 && launch_ttmc3<float>(L, st, &s)) return s;
    return compute_fp64 ? launch_ttmc_vt<float, double>(L, st) : launch_ttmc_vt<float, float>(L, st);
  }
  return compute_fp64 ? launch_ttmc_vt<double, double>(L, st) : launch_ttmc_vt<double, float>(L, st);
}

}  // namespace mach
