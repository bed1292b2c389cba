/*
 * mach.h — C ABI of libmach: MACH (Tsourakakis, "MACH: Fast Randomized Tensor
 * Decompositions", arXiv 0909.4969) on one NVIDIA GB300 (sm_103a).
 *
 * MACH keeps every entry of a dense d-way tensor X independently with
 * probability p and reweighs kept entries by 1/p (Section 3, Remark 1;
 * Algorithm 1 and Algorithm 2, first block; Theorem 1's sampling law), then
 * computes the Tucker decomposition of the sampled tensor X^ by HOOI
 * (Algorithm 2): HOSVD initialisation, sweeps that update every factor from
 * the tensor-times-matrix chain Y = X^ x_{k != i} A_k^T, and the core
 * G = X^ x_1 A_1^T ... x_d A_d^T.
 *
 * Conventions shared by every entry point:
 *  - Tensors are dense, C-order (last index fastest).  The linear index of
 *    entry (i_1..i_d) (zero-based) is l = (..(i_1 I_2 + i_2) I_3 + ..) I_d + i_d.
 *  - Device pointers come from cudaMalloc (or a caching allocator over it) on
 *    the current device; every input tensor must be 16-byte aligned.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Factors cross the boundary as FP64, column-major I_k x r_k (entry (i, j)
 *    at i + j*I_k), one device pointer per mode.  The core crosses as FP64,
 *    C-order r_1 x ... x r_d.
 *  - Supported orders d in {2, 3, 4}; dims 1 <= I_k <= 16384; ranks
 *    1 <= r_k <= min(I_k, 16, prod_{j != k} r_j); prod_{j != k} r_j <= 1024;
 *    fewer than 2^31 kept entries.
 *  - No exception crosses the ABI; every call returns a mach_status.  On
 *    error nothing the caller owns has been freed; outputs are unspecified.
 *  - The library allocates its own scratch with cudaMallocAsync (stream
 *    ordered) and frees it when the owning object is freed.
 */
#ifndef MACH_H
#define MACH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mach_status {
  MACH_OK = 0,
  MACH_EINVAL = 1,         /* invalid argument (shape, rank, p, alignment, null) */
  MACH_ENOMEM = 2,         /* device allocation failed */
  MACH_ENOMEM_BUDGET = 3,  /* a request exceeds the server's HBM budget */
  MACH_ECUDA = 4,          /* a CUDA runtime call failed; see mach_last_error() */
  MACH_ETIMEOUT = 5,       /* a bounded device-side wait gave up */
  MACH_EBUSY = 6,          /* object in use by in-flight work */
  MACH_EAGAIN = 7,         /* not ready yet / no free slot: retry later */
  MACH_EINTERNAL = 8       /* internal consistency check failed */
} mach_status;

typedef enum mach_dtype { MACH_F32 = 0, MACH_F64 = 1 } mach_dtype;

/* Arithmetic of the HOOI sweep.  FP64: every contraction, Gram, eigensolve
 * and re-orthonormalisation in FP64 (the small b x b rotations of the
 * intermediate subspace iterations are found in FP32, as they only orient
 * the next basis; the rotation that is kept is computed in FP64).  FP32:
 * tensor-times-matrix chain and Gram in FP32 with FP32 accumulation; the
 * R x R eigensolve and the re-orthonormalisation of the factors in FP64.
 * BF16_REFINE: the requested sweeps read BF16 copies of the sampled values
 * (chain in FP32 accumulation), then three more sweeps with the input values
 * refine the factors (subspace iteration from the BF16 solution; the core is
 * formed from the input values); the small eigensolve and the
 * re-orthonormalisation in FP64. */
typedef enum mach_prec {
  MACH_PREC_FP64 = 0,
  MACH_PREC_FP32 = 1,
  MACH_PREC_BF16_REFINE = 2
} mach_prec;

typedef struct mach_sample_s* mach_sample_t;

/* Human-readable name of a status code (static storage). */
const char* mach_strerror(mach_status status);

/* Last CUDA/internal error message seen by this thread (static per thread). */
const char* mach_last_error(void);

/* Library version string (static storage). */
const char* mach_version(void);

/* ---------------------------------------------------------------------------
 * mach_sample — the coin of Algorithm 1/2 (Section 3 Remark 1; Theorem 1).
 *
 * Every linear index l of the dense tensor x_dev (dtype, d modes, dims[0..d-1])
 * is kept iff Philox4x32-10(key = (seed mod 2^32, seed div 2^32),
 * counter = (q mod 2^32, q div 2^32, 0, 0), q = l div 4)[l mod 4] < T with
 * T = floor(p * 2^32) (T = 2^32 when p = 1).  The kept (value, l) pairs are
 * compacted in increasing l; the values are stored unscaled (the 1/p
 * reweighing is applied once, in the core and the norms).  The call then
 * builds, for every mode n, the entries re-ordered by (i_n, i_{n+1}, ..,
 * i_d, i_1, .., i_{n-1}) with fibre and row pointers, which the HOOI sweep
 * streams.
 *
 *   x_dev   device pointer, N = prod(dims) elements of `dtype`, 16-B aligned;
 *           read only; the caller keeps ownership and may free it once this
 *           call returns (the kept values are copied).
 *   p       keep probability, 0 < p <= 1.
 *   seed    64-bit Philox key.
 *   stream  work is ordered on it.  The call synchronises `stream` twice:
 *           after compaction (to size its buffers) and at the end (fibre
 *           counts and consistency checks).
 *   out     receives the new sample object; free it with mach_sample_free.
 * Errors: MACH_EINVAL (null pointers, d not in {2,3,4}, dims outside
 * [1, 16384], p outside (0,1], misaligned x_dev, 2^31 or more kept entries),
 * MACH_ENOMEM, MACH_ECUDA, MACH_ETIMEOUT, MACH_EINTERNAL (ordering check).
 */
mach_status mach_sample(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims,
                        double p, uint64_t seed, void* stream, mach_sample_t* out);

/* ---------------------------------------------------------------------------
 * mach_sample_host — mach_sample for an input that stays in HOST memory, the
 * setting the paper motivates MACH with (a tensor too large to hold in
 * memory, Section 1; the exact decomposition running out of memory in
 * Section 4): X is streamed chunk by chunk into a ring of two device
 * buffers of chunk_entries entries, each copy (on a stream of the library's
 * own) overlapping the coin of the previous chunk; only the kept entries
 * and their orderings stay on the device.  The coin of entry l is the same
 * as mach_sample's (keyed on the global l), so the kept set, values,
 * orderings and every later result are identical to mach_sample on the same
 * data.
 *
 *   x_host         host pointer to the dense C-order tensor (16-byte
 *                  aligned; page-locked memory lets the copies overlap the
 *                  sampler, pageable memory works but serialises them).
 *   chunk_entries  entries per streamed chunk: 0 = 2^28, else a positive
 *                  multiple of 2048.  The ring holds 2 chunks of device
 *                  memory.
 *   other arguments and errors as mach_sample (MACH_EINVAL also for a bad
 *   chunk_entries).  Synchronises `stream`.
 */
mach_status mach_sample_host(const void* x_host, mach_dtype dtype, int d, const int64_t* dims,
                             double p, uint64_t seed, int64_t chunk_entries, void* stream,
                             mach_sample_t* out);

/* ---------------------------------------------------------------------------
 * mach_sample_skip — mach_sample for an input resident in device memory,
 * reading only what the coin keeps.  The coin depends on the index alone
 * (Section 3 Remark 1), so the kept entries are known before X is read:
 * only the 32-byte sectors that hold kept entries are fetched, i.e.
 * 1 - (1 - p)^(32 / s_in) of X (7.7 % of an FP32 tensor at p = 0.01) instead
 * of all of it.  Same arguments, same kept set and orderings, same errors
 * as mach_sample.  The paper samples a stream it reads once in full; this
 * form is for data already in HBM.
 */
mach_status mach_sample_skip(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims,
                             double p, uint64_t seed, void* stream, mach_sample_t* out);

/* ---------------------------------------------------------------------------
 * mach_sample_noalloc — the same coin and compaction as mach_sample, written
 * straight into caller-owned buffers, with NO allocation of any kind: no
 * device or host heap memory, no memory pool, no library routine that
 * allocates.  The paper
 * has no counterpart; it exists for callers that must not allocate while
 * they sample: a process whose device memory is entirely committed to
 * resident tensors and preallocated output slabs (an allocation would fail
 * or evict), and a caller on a latency-critical path where an allocator
 * call could synchronise the device or stall behind other users of the
 * pool.  The look-back scratch lives in a fixed 4 MiB device array inside
 * libmach (one copy per device), which limits one call to
 * 2,147,471,360 FP32 or 1,073,735,680 FP64 entries.
 *
 *   x_dev, dtype, d, dims, p, seed  as for mach_sample.
 *   idx_dev  device int64[cap]: receives the kept linear indices, increasing.
 *   val_dev  device buffer of cap elements of `dtype`: the kept values,
 *            unscaled, in the same order.  Both caller-owned, written only
 *            in [0, min(cap, n_kept)).
 *   cap      capacity of idx_dev / val_dev in entries (may be 0).
 *   n_kept   host pointer receiving the number of kept entries, also when
 *            it exceeds cap.
 *   stream   work is ordered on it; the call synchronises it once, at the
 *            end, to read the count.
 * The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress), which may load the library's device code; make it
 * once on every device before any stream capture or other context in which
 * that lookup is not allowed.  Calls that overlap in time on one device
 * (several host threads or streams) race on the single scratch array and
 * give wrong results: serialise them.
 * Errors: MACH_EINVAL (as for mach_sample; misaligned idx_dev / val_dev;
 * N above the fixed-scratch limit, checked before any device work; cap <
 * n_kept, after the work, with n_kept set and the first cap entries
 * written), MACH_ECUDA, MACH_ETIMEOUT.
 */
mach_status mach_sample_noalloc(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims,
                                double p, uint64_t seed, int64_t* idx_dev, void* val_dev,
                                int64_t cap, int64_t* n_kept, void* stream);

/* Number of kept entries (host value; no device work). */
mach_status mach_sample_count(mach_sample_t s, int64_t* n_kept);

/* Copy the kept linear indices (increasing, int64) into idx_dev[0..cap). Fails
 * with MACH_EINVAL if cap < n_kept.  Asynchronous on `stream`. */
mach_status mach_sample_indices(mach_sample_t s, int64_t* idx_dev, int64_t cap, void* stream);

/* Copy the kept values (unscaled, in the sample's dtype, in increasing l) into
 * val_dev[0..cap).  Asynchronous on `stream`. */
mach_status mach_sample_values(mach_sample_t s, void* val_dev, int64_t cap, void* stream);

/* Number of non-empty fibres of the mode-n ordering (entries sharing every
 * index but the leaf index i_{n-1}); host value.  Diagnostic. */
mach_status mach_sample_fibers(mach_sample_t s, int mode, int64_t* n_fibers);

/* Diagnostics accumulated over every mach_hooi / mach_core call on this
 * sample (synchronises its stream): number of leading-singular-vector solves,
 * their total subspace iterations, how many stopped at the iteration cap
 * before reaching the tolerance, and the device status bits (timeouts,
 * overflow, index and positive-definiteness checks; 0 = clean).  Any pointer
 * may be NULL. */
mach_status mach_sample_stats(mach_sample_t s, int64_t* eig_calls, int64_t* eig_iters,
                              int64_t* eig_unconverged, unsigned* device_flags);

/* ---------------------------------------------------------------------------
 * mach_sample_gram — the Gram X^_(n) X^_(n)^T of the sampled tensor's mode-n
 * matricization (raw kept values, no 1/p), whose leading eigenvectors are
 * the HOSVD factor A_n (Section 2.1 HOSVD; Algorithm 1, and Algorithm 2's
 * initialisation).  mach_hooi computes it to start HOOI; this call exposes
 * it.
 *   mode      0 .. d-1.
 *   method    0: exact, every pair of kept entries of each fibre along mode
 *             n multiplied and summed in FP64;
 *             1: tensor cores, BF16 values, FP32 accumulation (relative
 *             error of a few 2^-9);
 *             2: tensor cores, each value as a pair of BF16 numbers (about
 *             16 significant bits), FP32 accumulation.
 *             Methods 1 and 2 need I_n <= 4096.
 *   gram_dev  device FP64 buffer of I_n x I_n entries, row-major (written).
 * Asynchronous on `stream`.  Errors: MACH_EINVAL (arguments), MACH_ENOMEM,
 * MACH_ECUDA.  A device-side timeout sets the status bits of
 * mach_sample_stats.
 */
mach_status mach_sample_gram(mach_sample_t s, int mode, int method, double* gram_dev, void* stream);

/* Release a sample object and its device memory (synchronises its stream). */
mach_status mach_sample_free(mach_sample_t s);

/* ---------------------------------------------------------------------------
 * mach_hooi — HOOI on the sampled tensor (Algorithm 2, second block;
 * Section 2.1 "Tucker3 Algorithms").
 *
 * Unless warm_start != 0, every A_k is first initialised by HOSVD of X^
 * (the r_k leading left singular vectors of the mode-k matricization).  Then
 * `sweeps` Gauss-Seidel sweeps: for i = 1..d, Y = X^ x_{k != i} A_k^T with the
 * latest factors and A_i <- the r_i leading left singular vectors of Y_(i).
 * The singular vectors are computed to convergence by block subspace
 * iteration with Rayleigh-Ritz on the small Gram matrix of Y_(i) (the
 * "under-the-hood" solver of Section 3 Remark 4).
 *
 *   ranks        host array of d ranks.
 *   sweeps       >= 0 (0 = MACH-HOSVD, Algorithm 1, when warm_start == 0).
 *   prec         arithmetic of the sweep (see mach_prec).
 *   factors_dev  host array of d device pointers, each FP64 column-major
 *                I_k x r_k; read as the starting point when warm_start != 0,
 *                always overwritten with the result.  Caller-owned.
 *   core_dev     NULL, or device FP64 buffer of prod(r_k) entries receiving
 *                G = X^ x_1 A_1^T ... x_d A_d^T (X^ includes 1/p), C-order.
 * Errors: MACH_EINVAL (bad ranks or pointers), MACH_ENOMEM, MACH_ECUDA.
 */
mach_status mach_hooi(mach_sample_t s, const int* ranks, int sweeps, mach_prec prec,
                      double* const* factors_dev, double* core_dev, int warm_start,
                      void* stream);

/* ---------------------------------------------------------------------------
 * mach_hooi_tucker2 — Tucker2 of a 3-way sample: mode keep_mode stays whole,
 * the other two are compressed (Section 2.1: compressing n of the d modes
 * gives a Tucker-n decomposition; Section 4 applies a Tucker2 to the sensor
 * tensor).  Algorithm 2 with the kept mode's products left out: HOSVD starts
 * for the compressed modes (unless warm_start != 0), `sweeps` Gauss-Seidel
 * sweeps in which A_n (n compressed) is the r_n leading left singular vectors
 * of Y_(n), Y = X^ x_m A_m^T (m the other compressed mode, the kept mode not
 * multiplied), then the core.
 *
 *   ranks        host array of 3; entries of the compressed modes in
 *                [1, min(I_k, 16, r_other * I_keep)]; the kept mode's entry is
 *                ignored (its rank is I_keep).
 *   keep_mode    0, 1 or 2.
 *   prec         MACH_PREC_FP64 or MACH_PREC_FP32.
 *   factors_dev  3 device pointers, FP64 column-major: I_k x r_k for the
 *                compressed modes (read when warm_start != 0, overwritten);
 *                for the kept mode NULL (nothing written) or I_keep x I_keep
 *                (set to the identity).
 *   core_dev     NULL, or r'_1 r'_2 r'_3 FP64 entries (r'_keep = I_keep),
 *                C order, 1/p included.
 * Errors: MACH_EINVAL (not 3-way, bad ranks or mode, empty sample),
 * MACH_ENOMEM, MACH_ECUDA.
 */
mach_status mach_hooi_tucker2(mach_sample_t s, const int* ranks, int keep_mode, int sweeps,
                              mach_prec prec, double* const* factors_dev, double* core_dev,
                              int warm_start, void* stream);

/* ---------------------------------------------------------------------------
 * mach_hooi_batched — Algorithm 2 for B independent 3-way samples in ONE
 * persistent kernel launch (the loop and the core of Algorithm 2 for every
 * sample; Section 2.1 n-mode products and "Tucker3 Algorithms").  Each CTA
 * of the launch owns one decomposition at a time and runs all of its sweeps
 * without returning to the host, which removes the per-mode launches that
 * bound many small decompositions.  Unless warm_start != 0, every factor is
 * first initialised inside the same launch by HOSVD: the r_n leading
 * eigenvectors of X^_(n) X^_(n)^T from 40 block subspace iterations (width
 * 16, seeded by the sample's seed) applied through the fibres along mode n,
 * and a Rayleigh-Ritz step (the atomically accumulated products make this
 * start reproducible to rounding only).  The sweeps are
 * FP32: the TTM chain over the mode-n CSF, the
 * Gram of the smaller side of Y_(n) (M = min(I_n, J_n) <= 32), its full
 * eigendecomposition by cyclic Jacobi, A_n = Y V Lambda^-1/2 (or V), then a
 * Cholesky re-orthonormalisation with FP64 r x r Gram, factor and inverse.
 *
 *   samples        host array of B sample handles, all 3-way, all with the
 *                  same value type (MACH_F32 or MACH_F64), none empty.
 *   ranks          host array of 3 ranks shared by every sample; every
 *                  J_n = prod_{k != n} r_k must be <= 32.
 *   sweeps         >= 0 (0 with warm_start == 0: the HOSVD factors).
 *   prec           MACH_PREC_FP32 (others: MACH_EINVAL).
 *   factors_io_dev host array of 3B device pointers, entry 3b + k = factor k
 *                  of sample b, FP64 column-major I_k x r_k: read when
 *                  warm_start != 0, always overwritten.  Caller-owned.
 *   cores_dev      NULL, or host array of B device pointers (entries may be
 *                  NULL) receiving G of sample b, r_1 r_2 r_3 FP64, C-order,
 *                  1/p included.
 * Asynchronous on `stream` (its staging buffers are freed stream-ordered).  Errors: MACH_EINVAL (bad
 * handles, shapes outside the limits above, mixed value types), MACH_ENOMEM,
 * MACH_ECUDA.  Device checks (a Gram that is not positive definite) set the
 * status bits read by mach_sample_stats.
 */
mach_status mach_hooi_batched(const mach_sample_t* samples, int B, const int* ranks, int sweeps,
                              mach_prec prec, double* const* factors_io_dev,
                              double* const* cores_dev, int warm_start, void* stream);

/* ---------------------------------------------------------------------------
 * mach_core — G = X^ x_1 A_1^T ... x_d A_d^T for given factors (Algorithm 2
 * last step, Eq. eqcore), with X^ = kept values / p.  FP64 throughout.
 *   factors_dev  d device pointers, FP64 column-major I_k x r_k (read only).
 *   core_dev     device FP64 buffer, prod(r_k) entries, C-order (written).
 */
mach_status mach_core(mach_sample_t s, const int* ranks, double* const* factors_dev,
                      double* core_dev, void* stream);

/* ---------------------------------------------------------------------------
 * mach_error — the accuracy measure of Section 4 ("Speedups & Synthetic
 * Experiment"): ||X - G x_1 A_1 ... x_d A_d|| / ||X|| against the ORIGINAL
 * dense X, in one streaming pass over X (orthonormal factors assumed, so
 * ||G x A|| = ||G||).  Synchronises `stream`; the result is a host value.
 *   x_dev, dtype, d, dims  the original tensor (as for mach_sample).
 *   factors_dev, core_dev  as produced by mach_hooi / mach_core.
 *   rel_err      host pointer receiving the relative error.
 *   x_norm       host pointer (may be NULL) receiving ||X||.
 */
mach_status mach_error(const void* x_dev, mach_dtype dtype, int d, const int64_t* dims,
                       const int* ranks, double* const* factors_dev, const double* core_dev,
                       double* rel_err, double* x_norm, void* stream);

/* ---------------------------------------------------------------------------
 * Served decompositions of tensor streams (the monitoring setting of
 * Section 1 and Section 4: windows of a stream arrive over time).  Each
 * request is one mach_sample + mach_hooi (Algorithm 2) + mach_error of one
 * window.  Windows of one stream warm-start HOOI from the previous window's
 * factors, which the server keeps on the device; a window whose shape or
 * ranks differ from its stream's state (a resized window) starts cold from
 * the HOSVD and leaves that state as it was.
 *
 * Continuous batching: `max_slots` worker slots, each with its own CUDA
 * stream.  A request is admitted as soon as a slot is free, its estimated
 * device memory fits in what remains of `hbm_budget_bytes`, and no earlier
 * request of the same stream is pending or running; admitted requests run
 * concurrently, later ones are admitted as slots and memory free up.
 *
 * mach_server_create  budget in bytes (> 0), 1 <= max_slots <= 64, on the
 *                     current device.  *srv receives the server handle.
 * mach_submit         queues one window.  x_dev (device, C order, 16-B
 *                     aligned) stays owned by the caller; it must be fully
 *                     written when mach_submit is called (the server's
 *                     streams are not ordered after the caller's) and stay
 *                     valid and unchanged until mach_poll reports it done.  Ranks
 *                     1 <= r_k <= min(I_k, 16).  *ticket identifies the
 *                     request.  Errors: MACH_EINVAL (arguments),
 *                     MACH_ENOMEM_BUDGET (the window can never fit the
 *                     budget), MACH_EAGAIN (queue full: retry), MACH_EBUSY
 *                     (server shutting down).
 * mach_poll           non-blocking.  Not finished: *done = 0, MACH_EAGAIN.
 *                     Finished: *done = 1, the request's status is
 *                     returned and, on MACH_OK, the core (prod(r_k) FP64, C
 *                     order), the factors (FP64 column-major I_k x r_k, one
 *                     host pointer per mode) and the relative error of
 *                     Section 4 against the window are copied into the
 *                     caller's host buffers (any may be NULL).  The ticket
 *                     is released by that call.
 * mach_server_stats   completed requests, p50 / p99 of submit-to-done
 *                     latency (ms, host clock), the most requests ever in
 *                     flight at once, and the budget in use.  NULL outputs
 *                     are skipped.
 * mach_server_destroy drops requests not yet admitted, waits for the ones
 *                     running, and frees the server and the streams' state.
 * mach_request_bytes  the device memory the server reserves for one such
 *                     request (what admission compares with the budget).
 * Calls on one server may come from any host thread.
 */
mach_status mach_server_create(size_t hbm_budget_bytes, int max_slots, void** srv);
mach_status mach_submit(void* srv, int64_t stream_id, const void* x_dev, mach_dtype dtype, int d,
                        const int64_t* dims, const int* ranks, double p, uint64_t seed, int sweeps,
                        mach_prec prec, int64_t* ticket);
mach_status mach_poll(void* srv, int64_t ticket, int* done, double* core_host,
                      double* const* factors_host, double* err_out);
mach_status mach_server_stats(void* srv, int64_t* completed, double* p50_ms, double* p99_ms,
                              int* max_in_flight, size_t* budget_in_use);
mach_status mach_server_destroy(void* srv);
mach_status mach_request_bytes(mach_dtype dtype, int d, const int64_t* dims, const int* ranks, double p,
                               mach_prec prec, size_t* bytes);

/* ---------------------------------------------------------------------------
 * Profiling (for measurement harnesses).  While enabled, libmach records a
 * CUDA event pair on the launching stream around every launch of the kernel
 * classes below, together with that launch's algorithmic byte count.
 *   kind 0: sampler (coin + compaction), bytes = N s_in + K (s_in + 8)
 *   kind 1: TTM chain of one mode,  bytes = K (s_val + 2) + F 8 + I_n J_n s_T
 *   kind 2: leading singular vectors of one mode (Gram, eigensolver, QR)
 *   kind 3: mode orderings and CSF build of one sample
 *   kind 4: HOSVD Gram of one mode
 * mach_profile_enable(1) clears previous records.  mach_profile_query
 * synchronises the recorded events and returns, for one kind, the summed
 * event time in milliseconds, the number of launches and the summed bytes.
 * mach_launch_count returns the number of CUDA kernels libmach has launched
 * since it was loaded (all kinds, whether profiling is on or not).
 */
/* ---------------------------------------------------------------------------
 * mach_check_bounded_wait — self-check of the bounded device-side wait that
 * every libmach kernel uses on its barriers (a wait that gives up after a
 * fixed number of polls, flags a status bit and returns, so that a barrier
 * that never completes costs an error code rather than a hung GPU).  One
 * thread block waits on a barrier phase for at most `limit` polls (1 <=
 * limit <= 2^23; each poll sleeps ~64 ns or more).  arrive != 0: the block
 * completes the phase itself first and the call returns MACH_OK.  arrive ==
 * 0: nothing completes it, the wait runs out and the call returns
 * MACH_ETIMEOUT, with the device context still usable.  Synchronises
 * `stream`.  Diagnostic; not part of the method.
 * Errors: MACH_EINVAL (limit outside the range), MACH_ENOMEM, MACH_ECUDA.
 */
mach_status mach_check_bounded_wait(long long limit, int arrive, void* stream);

mach_status mach_profile_enable(int enable);
mach_status mach_profile_query(int kind, double* total_ms, int64_t* launches, double* bytes);
int64_t mach_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MACH_H */
