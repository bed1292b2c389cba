// HOSVD Gram on the tensor cores: C = X^_(n) X^_(n)^T (Algorithm 2's HOSVD
// initialisation; Section 2.1 HOSVD: the leading left singular vectors of
// the mode-n matricization are the leading eigenvectors of this Gram).
//
// Every fibre along mode n is one column of X^_(n).  The fibres are taken
// 64 at a time; a chunk of 64 fibres is written densely (zeros where the
// coin dropped the entry) into shared memory as BF16 operand tiles, and the
// tile's outer product is accumulated by tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulators in tensor memory).  Where the sampled
// matricization is dense enough (a few percent of entries kept) this is far
// cheaper than accumulating the products of every pair of kept entries of a
// fibre one by one.
//
// Precision: each value x is split as x = h + l with h = bf16(x) and
// l = bf16(x - h) (about 16 significant bits together).  With terms = 2 the
// accumulator receives H H^T + H (2L)^T, whose symmetric part
// H H^T + H L^T + L H^T is the Gram of H + L up to the L L^T term; with
// terms = 1 it receives H H^T.  HOOI's sweeps refine the start this Gram
// gives; the exact FP32 / FP64 routes are kept for MACH-HOSVD alone.
//
// Work split: the I x I Gram is cut into 256 x 256 blocks (a, b); a CTA
// owns one block and a contiguous range of fibre chunks, and accumulates the
// block as two M = 128 tiles (TMEM columns 0..255 and 256..511).  Partial
// blocks go to global memory and a second kernel sums them over the chunk
// ranges in a fixed order (deterministic) and symmetrises.
//
// Shared-memory operand layout (K-major, no swizzle): core matrices of
// 8 rows x 16 bytes (8 BF16 along K) stored contiguously; core matrices
// adjacent along K are 128 bytes apart (the descriptor's leading byte
// offset), adjacent along the rows (kTcK / 8) * 128 bytes apart (its stride
// byte offset).
#include "mach_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace mach {

namespace {

constexpr int kTcK = 64;                         // fibres per chunk (MMA K per chunk)
constexpr int kTcRows = 256;                     // operand tile rows (two M = 128 MMAs)
constexpr int kTcThreads = 256;
constexpr uint32_t kTileBytes = kTcRows * kTcK * 2;   // 32 KB per BF16 tile
constexpr uint32_t kLbo = 128;                   // K-adjacent core matrices
constexpr uint32_t kSbo = (kTcK / 8) * 128;      // row-adjacent core matrices
constexpr int kTcStages = 2;
constexpr uint32_t kTmemCols = 512;
constexpr size_t kTcSmem = 2 * 3 * kTileBytes;   // two stages of three tiles (192 KB): one CTA per SM, which owns
                                                 // all 512 TMEM columns

__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(((row >> 3) * (kTcK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride
// byte offsets (all >> 4), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((kLbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((kSbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcGramArgs {
  const void* val;
  int vdt;                    // 0: float values, 1: double
  const uint16_t* leaf;
  const uint32_t* fib_start;
  int64_t nfib;
  int I;                      // order of the Gram
  int nrb;                    // 256-row blocks per side
  int splits;                 // fibre-chunk ranges per block
  int terms;                  // 1: H H^T; 2: H H^T + H (2L)^T
  float* part;                // [splits][nrb * nrb][256][256]
  unsigned* err;
};

__device__ __forceinline__ float load_val(const void* v, int vdt, uint32_t i) {
  return vdt ? (float)static_cast<const double*>(v)[i] : static_cast<const float*>(v)[i];
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_gram_kernel(TcGramArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t bar_mma[kTcStages];
  __shared__ uint32_t tmem_base_sh;
  __shared__ uint32_t fst[kTcK + 1];   // entry offsets of the chunk's fibres (and the end)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nblk = a.nrb * a.nrb;
  const int blk = (int)(blockIdx.x % (unsigned)nblk), sp = (int)(blockIdx.x / (unsigned)nblk);
  const int r0 = (blk / a.nrb) * kTcRows, c0 = (blk % a.nrb) * kTcRows;
  const int ra = min(kTcRows, a.I - r0), rb = min(kTcRows, a.I - c0);
  const int mtiles = (ra + 127) >> 7;
  const int N = (rb + 15) & ~15;
  const bool shared_tile = r0 == c0;
  const int64_t nchunk = (a.nfib + kTcK - 1) / kTcK;
  const int64_t ch0 = nchunk * sp / a.splits, ch1 = nchunk * (sp + 1) / a.splits;
  // stage s: tile A (H rows r0..), tile B (H rows c0.., absent when shared),
  // tile L (2L rows c0.., terms == 2)
  const uint32_t sbase = smem_addr(tc_smem);
  const uint32_t stage_bytes = 3 * kTileBytes;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) mbar_init(&bar_mma[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t idesc = idesc_bf16_f32(128, N);
  bool timed_out = false;
  int uses[kTcStages] = {0, 0};
  for (int64_t ch = ch0; ch < ch1 && !timed_out; ++ch) {
    const int s = (int)((ch - ch0) & 1);
    unsigned char* st = tc_smem + (size_t)s * stage_bytes;
    if (uses[s] > 0) {
      // the MMAs that read this stage two chunks ago have completed
      if (!mbar_wait_bounded(&bar_mma[s], (uint32_t)((uses[s] - 1) & 1))) {
        timed_out = true;
        break;
      }
    }
    // the chunk's fibre starts (one coalesced load, clamped past the last
    // fibre), then zero the stage's tiles while they arrive
    if (tid <= kTcK) {
      const int64_t f = ch * kTcK + tid;
      fst[tid] = a.fib_start[f < a.nfib ? f : a.nfib];
    }
    {
      const int ntile = 1 + (shared_tile ? 0 : 1) + (a.terms == 2 ? 1 : 0);
      uint4* z = reinterpret_cast<uint4*>(st);
      const int n16 = ntile * (int)(kTileBytes / 16);
      for (int i = tid; i < n16; i += kTcThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    unsigned char* tA = st;
    unsigned char* tB = shared_tile ? st : st + kTileBytes;
    unsigned char* tL = st + (shared_tile ? 1 : 2) * kTileBytes;
    // scatter: the chunk's entries are contiguous; thread t takes entries
    // t, t + 256, .. and finds its fibre (column k) by binary search in fst
    {
      const uint32_t s0 = fst[0], s1 = fst[kTcK];
      for (uint32_t e = s0 + (uint32_t)tid; e < s1; e += kTcThreads) {
        int lo = 0, hi = kTcK;   // fst[lo] <= e < fst[hi]
#pragma unroll
        for (int step = 0; step < 6; ++step) {
          const int mid = (lo + hi) >> 1;
          if (fst[mid] <= e) lo = mid;
          else hi = mid;
        }
        const int k = lo;
        const int li = (int)a.leaf[e];
        const float x = load_val(a.val, a.vdt, e);
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float lo_part = x - __bfloat162float(h);
        const unsigned ia = (unsigned)(li - r0), ib = (unsigned)(li - c0);
        if (ia < (unsigned)kTcRows) *reinterpret_cast<__nv_bfloat16*>(tA + tile_off((int)ia, k)) = h;
        if (ib < (unsigned)kTcRows) {
          if (!shared_tile) *reinterpret_cast<__nv_bfloat16*>(tB + tile_off((int)ib, k)) = h;
          if (a.terms == 2)
            *reinterpret_cast<__nv_bfloat16*>(tL + tile_off((int)ib, k)) = __float2bfloat16_rn(2.0f * lo_part);
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t aA = sbase + (uint32_t)s * stage_bytes;
      const uint32_t aB = shared_tile ? aA : aA + kTileBytes;
      const uint32_t aL = aA + (shared_tile ? 1u : 2u) * kTileBytes;
      for (int mt = 0; mt < mtiles; ++mt) {
        const uint32_t d = tmem + (uint32_t)(mt * 256);
        for (int t = 0; t < a.terms; ++t) {
#pragma unroll
          for (int ks = 0; ks < kTcK / 16; ++ks) {
            const uint64_t da = smem_desc(aA + (uint32_t)mt * 16u * kSbo + (uint32_t)ks * 2u * kLbo);
            const uint64_t db = smem_desc((t == 0 ? aB : aL) + (uint32_t)ks * 2u * kLbo);
            const uint32_t acc = (ch > ch0 || t > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(d, da, db, idesc, acc);
          }
        }
      }
      mma_commit(&bar_mma[s]);
    }
    ++uses[s];
  }
  // wait for the last MMAs (the latest commit covers every earlier one)
  const int64_t done = min(ch1, ch0 + (int64_t)(uses[0] + uses[1])) - ch0;
  bool have = done > 0;
  if (have) {
    const int s_last = (int)((done - 1) & 1);
    if (!mbar_wait_bounded(&bar_mma[s_last], (uint32_t)((uses[s_last] - 1) & 1))) {
      timed_out = true;
      // wait (bounded) once more for the MMAs still in flight before TMEM is freed
      (void)mbar_wait_bounded(&bar_mma[s_last], (uint32_t)((uses[s_last] - 1) & 1));
    }
  }
  if (timed_out && tid == 0) atomicOr(a.err, DEV_TIMEOUT);
  tc_fence_after();
  // accumulators -> partial block (rows of M tile w / 4, lanes 32 (w % 4) ..)
  float* out = a.part + ((size_t)sp * nblk + blk) * (size_t)kTcRows * kTcRows;
  const int mt = warp >> 2;
  const int row = mt * 128 + (warp & 3) * 32 + lane;
  if (mt < mtiles) {
    for (int g = 0; g < N / 16; ++g) {
      float v[16];
      if (have && !timed_out) {
        tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(mt * 256 + g * 16), v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      float4* o = reinterpret_cast<float4*>(out + (size_t)row * kTcRows + g * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// C[i][j] = (D(i, j) + D(j, i)) / 2 with D = the partial blocks summed over
// the chunk ranges in range order.
template <typename T>
__global__ void tc_gram_reduce(const float* __restrict__ part, int I, int nrb, int splits, T* __restrict__ C) {
  const int64_t n = (int64_t)I * I;
  const int nblk = nrb * nrb;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(o / I), j = (int)(o - (o / I) * I);
    const size_t bij = (size_t)((i >> 8) * nrb + (j >> 8)) * kTcRows * kTcRows + (size_t)(i & 255) * kTcRows + (j & 255);
    const size_t bji = (size_t)((j >> 8) * nrb + (i >> 8)) * kTcRows * kTcRows + (size_t)(j & 255) * kTcRows + (i & 255);
    float dij = 0.f, dji = 0.f;
    for (int s = 0; s < splits; ++s) {
      const size_t base = (size_t)s * nblk * kTcRows * kTcRows;
      dij += part[base + bij];
      dji += part[base + bji];
    }
    C[o] = (T)(0.5f * (dij + dji));
  }
}

}  // namespace

int tc_gram_max_order() { return 4096; }

size_t tc_gram_scratch_bytes(int I) {
  const int nrb = (I + kTcRows - 1) / kTcRows;
  const int nblk = nrb * nrb;
  const int splits = std::max(1, num_sms() / nblk);
  return (size_t)splits * nblk * kTcRows * kTcRows * sizeof(float);
}

template <typename T>
mach_status launch_tc_gram(const void* val, mach_dtype vdt, const uint16_t* leaf, const uint32_t* fib_start,
                           int64_t nfib, int I, int terms, float* scratch, T* C, unsigned* err, cudaStream_t st) {
  if (I < 1 || I > tc_gram_max_order() || (terms != 1 && terms != 2)) return MACH_EINVAL;
  TcGramArgs a;
  a.val = val;
  a.vdt = vdt == MACH_F64 ? 1 : 0;
  a.leaf = leaf;
  a.fib_start = fib_start;
  a.nfib = nfib;
  a.I = I;
  a.nrb = (I + kTcRows - 1) / kTcRows;
  const int nblk = a.nrb * a.nrb;
  a.splits = std::max(1, num_sms() / nblk);
  a.terms = terms;
  a.part = scratch;
  a.err = err;
  MACH_CUDA_TRY(cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  tc_gram_kernel<<<(unsigned)(nblk * a.splits), kTcThreads, kTcSmem, st>>>(a);
  MACH_LAUNCH_CHECK();
  const int64_t n = (int64_t)I * I;
  tc_gram_reduce<T><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, st>>>(scratch, I, a.nrb, a.splits,
                                                                                          C);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template mach_status launch_tc_gram<float>(const void*, mach_dtype, const uint16_t*, const uint32_t*, int64_t, int,
                                           int, float*, float*, unsigned*, cudaStream_t);
template mach_status launch_tc_gram<double>(const void*, mach_dtype, const uint16_t*, const uint32_t*, int64_t, int,
                                            int, float*, double*, unsigned*, cudaStream_t);

}  // namespace mach
