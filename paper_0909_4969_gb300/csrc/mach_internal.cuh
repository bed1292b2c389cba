// Internal helpers shared by the libmach translation units (device + host).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "mach.h"

namespace mach {

// ----------------------------------------------------------------------------
// Error reporting
// ----------------------------------------------------------------------------
void set_last_error(const char* fmt, ...);

#define MACH_CUDA_TRY(expr)                                                            \
  do {                                                                                 \
    cudaError_t mach_e_ = (expr);                                                      \
    if (mach_e_ != cudaSuccess) {                                                      \
      ::mach::set_last_error("%s:%d %s -> %s", __FILE__, __LINE__, #expr,              \
                             cudaGetErrorString(mach_e_));                             \
      return mach_e_ == cudaErrorMemoryAllocation ? MACH_ENOMEM : MACH_ECUDA;          \
    }                                                                                  \
  } while (0)

#define MACH_TRY(expr)                          \
  do {                                          \
    mach_status mach_s_ = (expr);               \
    if (mach_s_ != MACH_OK) return mach_s_;     \
  } while (0)

// Every kernel launch in libmach is followed by MACH_LAUNCH_CHECK(), which
// also counts it (mach_launch_count).
void count_launch();
#define MACH_LAUNCH_CHECK()          \
  do {                               \
    ::mach::count_launch();          \
    MACH_CUDA_TRY(cudaGetLastError()); \
  } while (0)

// Profiling scopes (event pairs on the launching stream), see mach.h.
enum ProfKind { PROF_SAMPLER = 0, PROF_TTMC = 1, PROF_LSV = 2, PROF_CSF = 3, PROF_INITGRAM = 4, PROF_NKINDS = 5 };
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s, double bytes);

// Device-side status word bits (a kernel never traps: it records and returns).
enum : unsigned {
  DEV_TIMEOUT = 1u,    // a bounded spin-wait gave up
  DEV_OVERFLOW = 2u,   // output capacity exceeded (sizes are recomputed by the host)
  DEV_BADINDEX = 4u,   // an index fell outside its declared range (skipped)
  DEV_NOTPD = 8u       // a Gram matrix that must be positive definite was not
};

// Upper bound of every device spin-wait, in polling iterations (each iteration
// sleeps ~64-256 ns): about one second, after which the kernel flags
// DEV_TIMEOUT and returns.
constexpr long long kSpinLimit = 1LL << 23;

constexpr int kMaxModes = 4;
constexpr int kMaxRank = 16;
constexpr int kMaxJ = 1024;
constexpr int kMaxDim = 16384;

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Round: multiply words 0 and 2 by the
// round multipliers (full 64-bit products), new state
// (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)); the key is
// bumped by the Weyl constants (fractional parts of the golden ratio and of
// sqrt 3) before every round but the first.  The product is formed as
// __umulhi + 32-bit multiply, the faster pair on sm_103a.
// ----------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1) {
  uint32_t x0 = c0, x1 = c1, x2 = 0u, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, x0);
    const uint32_t lo0 = kPhiloxM0 * x0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, x2);
    const uint32_t lo1 = kPhiloxM1 * x2;
    const uint32_t n0 = hi1 ^ x1 ^ k0;
    const uint32_t n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
  }
  return make_uint4(x0, x1, x2, x3);
}

// The same generator with the key schedule supplied by the launch
// (k0[r] = key0 + r W0, k1[r] = key1 + r W1, mod 2^32), so the per-round key
// bumps leave the integer pipe; counter words 2 and 3 are zero, so round 0
// has one product.  Returns the same words as philox4x32_10.
struct PhiloxSched {
  uint32_t k0[10];
  uint32_t k1[10];
};

inline PhiloxSched make_philox_sched(uint64_t seed) {
  PhiloxSched ks;
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = k0;
    ks.k1[r] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return ks;
}

// Both halves of the 32 x 32 -> 64-bit product, written as separate
// mul.hi / mul.lo (measured on sm_103a: the form that leaves the integer
// multiply pipe with the product work only).
__device__ __forceinline__ void mul_hilo(uint32_t m, uint32_t x, uint32_t& hi, uint32_t& lo) {
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(hi) : "r"(x), "r"(m));
  asm("mul.lo.u32 %0, %1, %2;" : "=r"(lo) : "r"(x), "r"(m));
}

__device__ __forceinline__ uint4 philox4x32_10_sched(uint32_t c0, uint32_t c1, const PhiloxSched& ks) {
  uint32_t h, l;
  mul_hilo(kPhiloxM0, c0, h, l);
  uint32_t x0 = c1 ^ ks.k0[0];
  uint32_t x1 = 0u;
  uint32_t x2 = h ^ ks.k1[0];
  uint32_t x3 = l;
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_hilo(kPhiloxM0, x0, hi0, lo0);
    mul_hilo(kPhiloxM1, x2, hi1, lo1);
    x0 = hi1 ^ x1 ^ ks.k0[r];
    x1 = lo1;
    x2 = hi0 ^ x3 ^ ks.k1[r];
    x3 = lo0;
  }
  return make_uint4(x0, x1, x2, x3);
}

// ----------------------------------------------------------------------------
// Division of 64-bit unsigned integers by a run-time invariant divisor using
// one multiply-high, after Granlund & Montgomery, "Division by invariant
// integers using multiplication" (PLDI 1994), unsigned case: with
// l = ceil(log2 d) and m = floor(2^64 (2^l - d) / d) + 1,
// q = (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = mulhi(m, n).
// ----------------------------------------------------------------------------
struct FastDiv {
  uint64_t d;
  uint64_t m;
  uint32_t s1;
  uint32_t s2;
};

inline FastDiv make_fastdiv(uint64_t d) {
  // d in [1, 2^63]
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while (((uint64_t)1 << l) < d) ++l;
  const unsigned __int128 num = ((unsigned __int128)(((uint64_t)1 << l) - d)) << 64;
  f.m = (uint64_t)(num / d) + 1;
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 0 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint64_t fdiv(const FastDiv& f, uint64_t n) {
  const uint64_t t = __umul64hi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Mixed-radix decoder: C-order linear index -> coordinates.
struct Decoder {
  int d;
  FastDiv div[kMaxModes];   // divisor = dims[k]
  int64_t dims[kMaxModes];
};

inline Decoder make_decoder(int d, const int64_t* dims) {
  Decoder dec;
  dec.d = d;
  for (int k = 0; k < kMaxModes; ++k) {
    dec.dims[k] = k < d ? dims[k] : 1;
    dec.div[k] = make_fastdiv(k < d ? (uint64_t)dims[k] : 1u);
  }
  return dec;
}

__device__ __forceinline__ void decode(const Decoder& dec, uint64_t l, uint32_t* coord) {
#pragma unroll
  for (int k = kMaxModes - 1; k >= 0; --k) {
    if (k < dec.d) {
      const uint64_t q = fdiv(dec.div[k], l);
      coord[k] = (uint32_t)(l - q * dec.div[k].d);
      l = q;
    }
  }
}

// ----------------------------------------------------------------------------
// mbarrier and bulk (TMA) copies, global -> shared, 1-D (no tensor map).
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; returns false (and the caller flags
// DEV_TIMEOUT) when the limit is reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kSpinLimit) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// One bulk copy of `bytes` (multiple of 16, both addresses 16-B aligned) that
// completes `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Release / acquire accesses to 64-bit flags in global memory.
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Raise a kernel's dynamic shared-memory limit to the most it may use on
// this device.  The value is the same on every call, so launches from
// several host threads never lower the limit under one another.
template <typename F>
inline mach_status allow_max_dyn_smem(F kern) {
  cudaFuncAttributes fa;
  MACH_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0;
  MACH_CUDA_TRY(cudaGetDevice(&dev));
  MACH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  MACH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes));
  return MACH_OK;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device memory owned by the library, allocated stream-ordered.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

mach_status dev_alloc(DevBuf& b, size_t bytes, cudaStream_t s);
void dev_free(DevBuf& b, cudaStream_t s);

// A DevBuf released (stream-ordered) when it goes out of scope, so that
// every early return of a host routine frees its temporaries.
struct ScopedDevBuf : DevBuf {
  cudaStream_t st;
  explicit ScopedDevBuf(cudaStream_t s) : st(s) {}
  ~ScopedDevBuf() { dev_free(*this, st); }
  ScopedDevBuf(const ScopedDevBuf&) = delete;
  ScopedDevBuf& operator=(const ScopedDevBuf&) = delete;
};

int num_sms();

// HOSVD Gram X^_(n) X^_(n)^T on the tensor cores (tcgram.cu), from the
// fibres along mode n; terms = 1 (BF16 values) or 2 (BF16 pair, about 16
// significant bits).  scratch: tc_gram_scratch_bytes(I) bytes.
int tc_gram_max_order();
size_t tc_gram_scratch_bytes(int I);
template <typename T>
mach_status launch_tc_gram(const void* val, mach_dtype vdt, const uint16_t* leaf, const uint32_t* fib_start,
                           int64_t nfib, int I, int terms, float* scratch, T* C, unsigned* err, cudaStream_t st);

// Self-check of the bounded mbarrier wait (selfcheck.cu).
mach_status run_bounded_wait_check(long long limit, int arrive, cudaStream_t st);

// ----------------------------------------------------------------------------
// Kernel launchers (one definition each, in sample.cu / sort.cu / ttmc.cu /
// linalg.cu / error.cu) and their argument blocks.
// ----------------------------------------------------------------------------
int64_t sampler_scratch_words(int64_t n, mach_dtype dt);
// Segmented sampler (sample.cu): nseg CTAs, each writing up to seg_cap kept
// pairs of its contiguous tiles into its own segment; then an ordered gather.
struct SegPlan {
  int64_t nseg = 0;
  int64_t chunks_per_seg = 0;
  int64_t seg_cap = 0;
};
SegPlan plan_segments(int64_t n, mach_dtype dt, double q);
// l0: linear index of x[0] (a multiple of sampler_chunk_align()), for a
// tensor sampled chunk by chunk.
mach_status launch_sampler_seg(const void* x, mach_dtype dt, int64_t n, int64_t l0, uint64_t seed, uint64_t T,
                               const SegPlan& pl, uint32_t* seg_off, void* seg_val, int64_t* seg_count,
                               cudaStream_t st, bool skip);
// Gathers nseg_total segments: segment c belongs to input chunk c / pl.nseg,
// whose first linear index is (c / pl.nseg) * chunk_entries, and starts at
// output position seg_start[c] (the exclusive scan of seg_count).
mach_status launch_seg_gather(mach_dtype dt, const SegPlan& pl, int64_t nseg_total, int64_t chunk_entries,
                              const int64_t* seg_count, const int64_t* seg_start, const uint32_t* seg_off,
                              const void* seg_val, int64_t* idx, void* val, int64_t out_cap, unsigned* d_err,
                              cudaStream_t st);
// Exclusive scan (sort.cu; instantiated for uint32_t and long long); `tmp`
// holds scan_tmp_elems_total(n) elements.
template <typename T>
mach_status scan_exclusive(const T* in, T* out, int64_t n, T* total_dev, T* tmp, cudaStream_t st);
int64_t scan_tmp_elems_total(int64_t n);
int64_t sampler_chunk_align();
// Tucker2 of a 3-way sample (tucker2.cu).
struct Tucker2Leaf {
  const void* val;             // the source CSF (leaf index = the contracted mode m)
  const uint16_t* leaf;
  const uint32_t* fib_start;
  const uint32_t* fib_mid;
  const uint32_t* row_fib;
  int rows;                    // rows of the source CSF
  const void* Am;              // A_m, I_m x r_m row-major (T)
  int rm;
  int row_is_n;                // the source CSF's row index is i_n (else it is i_c)
  int I_n, I_c;
  void* Y;                     // I_n x (r_m * I_c), row-major (T)
};
template <typename T>
mach_status launch_tucker2_leaf(const Tucker2Leaf& a, mach_dtype vdt, cudaStream_t st);
template <typename T>
mach_status launch_tucker2_core(const T* Y, const double* A_L, int I_L, int r_L, int r_O, int I_c, int L, int O,
                                int c, double scale, double* G, cudaStream_t st);
mach_status launch_identity_colmajor(double* A, int n, cudaStream_t st);

// Batched HOOI (batched.cu): one persistent launch over many 3-way samples.
struct BatMode {             // the mode-n CSF of one sample
  const void* val;           // mode-ordered values (the sample's dtype)
  const uint16_t* leaf;      // leaf index per entry
  const uint32_t* fib_start; // nfib + 1
  const uint32_t* fib_mid;   // mid index per fibre
  const uint32_t* row_fib;   // I_n + 1
};
struct BatItem {
  BatMode mode[3];
  int dims[3];
  double inv_p;
  double* fac[3];            // FP64 column-major I_k x r_k: start factors in, results out
  double* core;              // r_1 r_2 r_3 FP64 (C order), or null
  unsigned* err;             // the sample's status word
  uint64_t seed;             // seeds the HOSVD start block
};
struct BatArgs {
  const BatItem* items;
  int B;
  int r[3];
  int sweeps;
  int warm;                  // 0: HOSVD start inside the launch
  unsigned* next;            // item counter (zero at launch)
  float* ws;                 // grid x ws_stride floats
  int64_t ws_stride;
};
int batched_max_j();
int64_t batched_hosvd_scratch(int64_t max_dim);
int batched_grid(int B);
mach_status launch_batched_hooi(const BatArgs& a, mach_dtype dt, int grid, cudaStream_t st);

// Fixed scratch of the allocation-free sampler (sample.cu): its size in
// 8-byte words, the largest tensor it serves, and this device's address of it.
constexpr int64_t kFixedScratchWords = 524288;
int64_t sampler_fixed_max_entries(mach_dtype dt);
mach_status sampler_fixed_scratch(unsigned long long** out);
mach_status launch_sampler(const void* x, mach_dtype dt, int64_t n, uint64_t seed, uint64_t T, int64_t cap,
                           int64_t* idx, void* val, int64_t* d_count, unsigned* d_err,
                           unsigned long long* scratch, cudaStream_t st);
size_t sort_scratch_bytes(int64_t K, int64_t nbins);
template <typename V>
mach_status counting_sort(const int64_t* idx, const V* val, int64_t K, const int64_t* d_count, const Decoder& dec,
                          int mode, int64_t* idx_out, V* val_out, void* scratch, cudaStream_t st);
struct CsfBuildArgs {
  const int64_t* idx;
  const int64_t* d_count;
  int64_t K;
  Decoder dec;
  int mode;
  uint32_t emax;
  uint16_t* leaf;
  uint32_t* fib_start;
  uint32_t* fib_mid;
  uint32_t* row_fib;
  uint32_t* row_task;
  int4* tasks;
  uint32_t* d_nfib;
  uint32_t* d_ntask;
  unsigned* d_err;
  void* scratch;
};
size_t csf_scratch_bytes(int64_t K, int64_t nrows);
mach_status build_csf(const CsfBuildArgs& a, cudaStream_t st);
struct TtmcLaunch {
  int d;
  const void* val;
  mach_dtype vdt;
  bool bf16 = false;          // val holds BF16 copies of the values
  const uint16_t* leaf;
  const uint32_t* fib_start;
  const uint32_t* fib_mid;
  const int4* tasks;
  const uint32_t* d_ntask;
  const uint32_t* d_nfib;
  const uint32_t* row_task;
  int64_t ntask_cap;
  int nrows;
  const void* A_leaf;
  const void* A_mid0;
  const void* A_mid1;
  int I_leaf, I_mid0, I_mid1;
  int r_leaf, r_mid0, r_mid1;
  int J;
  void* Y;
  void* partial;
  unsigned* err;
};
uint32_t ttmc_task_max();
// BF16 copy (round to nearest even) of K values of dtype dt.
mach_status launch_to_bf16(const void* val, mach_dtype dt, int64_t K, void* out, cudaStream_t st);
mach_status launch_ttmc(const TtmcLaunch& L, bool compute_fp64, cudaStream_t st);
template <typename T>
mach_status launch_gram(const T* Z, int64_t L, int M, int64_t sl, int64_t sm, T* C, T* partial_scratch,
                        int64_t partial_cap, cudaStream_t st);
template <typename V, typename T>
mach_status launch_init_gram(const void* val, const uint16_t* leaf, const uint32_t* fib_start,
                             const uint32_t* d_nfib, int64_t nfib_cap, int M, T* C, cudaStream_t st);
struct EigLaunch {
  int M, r, b;
  int maxit;
  double tol;
  void* V;
  void* W;
  void* U;
  double* Vout;
  double* theta;
  void* part;                  // >= eig_part_elems(M) elements of T (split path)
  unsigned long long* stats;   // device counters: calls, iterations, unconverged
  void* basis_out;             // M x b T: final Ritz block, or null
  double* rr;                  // >= kMaxRank * (kMaxRank + 1) doubles (split path); may alias Vout
  unsigned long long* ctl = nullptr;   // 3 device words: the FP32 split path's convergence test and early exit
};
int eig_split_threshold();
size_t eig_part_elems(int M);
template <typename T>
mach_status launch_eig(const T* C, const EigLaunch& e, cudaStream_t st);
// Where a finished launch_eig left its result: the leading Ritz basis U_r
// (M x r, T, leading dimension ldu), the FP64 rotation X (r x r row-major)
// with U_r X = the eigenvectors, and theta (r eigenvalues, descending).
template <typename T>
struct EigResult {
  const T* U;
  int ldu;
  const double* X;
  const double* theta;
};
template <typename T>
EigResult<T> eig_result(const EigLaunch& e);
// Bytes of the output area e.Vout for orders up to M.
size_t eig_out_bytes(int M);
template <typename T>
mach_status launch_start_block(const T* Y, const T* Aprev, int I, int J, int r, int b, bool jroute, bool warm,
                               T* V, T* scratch, uint32_t salt, const T* prev_ritz, cudaStream_t st);
template <typename T>
mach_status launch_lsv_finish(const T* Y, const EigResult<T>& ev, int I, int J, int r, bool jroute,
                              double* A64, double* gram64, unsigned* counter, double* rinv, unsigned* err,
                              double* out_colmajor, T* out_rowmajor, cudaStream_t st);
template <typename T>
mach_status launch_factor_to_rowmajor(const double* A, int I, int r, T* out, cudaStream_t st);
template <typename T>
mach_status launch_core(const T* Y, const double* A, int I, int J, int r, double scale, double* G,
                        cudaStream_t st);
mach_status launch_error(const void* x, mach_dtype dt, int d, const int64_t* dims, const int* ranks,
                         double* const* factors, const double* core, double* acc, cudaStream_t st);

}  // namespace mach
