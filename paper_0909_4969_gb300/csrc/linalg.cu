// Leading left singular vectors ("the r_i leading left singular vectors of
// Y_(i)", Algorithm 2; HOSVD, Section 2.1) and the core (Eq. eqcore /
// Algorithm 2 last step), as small dense kernels.
//
// For Y_(i) of size I x J the leading left singular vectors are the leading
// eigenvectors of Y Y^T; when J < I they are Y V Sigma^-1 with V the leading
// eigenvectors of Y^T Y.  The eigenvectors of the M x M Gram (M = min(I, J))
// come from block subspace iteration with a Rayleigh-Ritz step every
// iteration (the Lanczos-class "under-the-hood" solver of Section 3 Remark 4),
// warm-started from the previous factor and run until the Ritz residuals fall
// below a tolerance.  The b x b Rayleigh-Ritz eigenproblems use cyclic Jacobi
// (round-robin ordering, one warp); the final r x r Rayleigh-Ritz problem and
// the re-orthonormalisation (Cholesky QR) of the I x r factor are FP64.
//
// GB300 FP64 throughput is 1/64 of FP32, so FP64 is confined to O(M r^2)
// and O(r^3) work; the O(M^2 b) products run in the path's precision T.
#include "mach_internal.cuh"

#include <cmath>

namespace mach {

namespace {

// ----------------------------------------------------------------------------
// Gram C = Z^T Z, Z: L x M, element (l, m) at Z[l * sl + m * sm].
// 32x32 output tiles (upper triangle), split over L into `nsplit` partials.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const T* __restrict__ Z, int64_t L, int M, int64_t sl,
                                                   int64_t sm, int nsplit, T* __restrict__ out) {
  const int bx = blockIdx.x, by = blockIdx.y;
  if (by > bx) return;
  __shared__ T sa[32][33];
  __shared__ T sb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t chunk = ceil_div(L, nsplit);
  const int64_t l_lo = (int64_t)blockIdx.z * chunk;
  const int64_t l_hi = min(L, l_lo + chunk);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t l0 = l_lo; l0 < l_hi; l0 += 32) {
    for (int k = ty; k < 32; k += 8) {
      const int64_t l = l0 + k;
      const int ma = by * 32 + tx, mb = bx * 32 + tx;
      sa[k][tx] = (l < l_hi && ma < M) ? Z[l * sl + ma * sm] : T(0);
      sb[k][tx] = (l < l_hi && mb < M) ? Z[l * sl + mb * sm] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const T b = sb[k][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] += sa[k][ty + 8 * i] * b;
    }
    __syncthreads();
  }
  T* o = out + (size_t)blockIdx.z * M * M;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = by * 32 + ty + 8 * i, c = bx * 32 + tx;
    if (r < M && c < M) {
      o[(size_t)r * M + c] = acc[i];
      o[(size_t)c * M + r] = acc[i];
    }
  }
}

template <typename T>
__global__ void sum_partials_kernel(const T* __restrict__ part, int nsplit, int64_t n, T* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * n + i];
    out[i] = s;
  }
}

// ----------------------------------------------------------------------------
// HOSVD Gram C = X^_(n) X^_(n)^T (raw values) from the fibres along mode n
// (every fibre is one column of the mode-n matricization): C[a][b] +=
// x_a x_b for every pair of entries of a fibre.  One warp per fibre, the
// lanes over its unordered pairs (one FP atomic each, into the upper
// triangle: half the atomics of adding both C[a][b] and C[b][a]), then one
// pass mirrors the upper triangle.
// ----------------------------------------------------------------------------
template <typename V, typename T>
__global__ void init_gram_kernel(const V* __restrict__ val, const uint16_t* __restrict__ leaf,
                                 const uint32_t* __restrict__ fib_start, const uint32_t* d_nfib, int M,
                                 T* __restrict__ C) {
  const uint32_t nfib = *d_nfib;
  const int lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t f = gw; f < nfib; f += nw) {
    const uint32_t s0 = fib_start[f], s1 = fib_start[f + 1];
    const uint32_t n = s1 - s0, npair = n * (n + 1) / 2;
    // the fibre's unordered pairs (i <= j) spread over the lanes; one atomic
    // per pair into the upper triangle (gram_symmetrize_kernel mirrors it)
    for (uint32_t k0 = lane; k0 < npair; k0 += 32) {
      uint32_t i = 0, k = k0;
      while (k >= n - i) {
        k -= n - i;
        ++i;
      }
      const uint32_t j = i + k;
      const uint32_t a = leaf[s0 + i], b2 = leaf[s0 + j];
      const T v = (T)val[s0 + i] * (T)val[s0 + j];
      const uint32_t lo = a < b2 ? a : b2, hi = a < b2 ? b2 : a;
      atomicAdd(&C[(size_t)lo * M + hi], v);
    }
  }
}

// C[hi][lo] = C[lo][hi] for lo < hi.
template <typename T>
__global__ void gram_symmetrize_kernel(T* __restrict__ C, int M) {
  const int64_t n = (int64_t)M * M;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(o / M), c = (int)(o - (o / M) * M);
    if (r > c) C[o] = C[(size_t)c * M + r];
  }
}

// ----------------------------------------------------------------------------
// Starting blocks.  Deterministic pseudo-random fill (Philox of (i, j)) for
// the columns not given by a warm start.
// ----------------------------------------------------------------------------
// Columns col0..b of the start block: the previous solve's Ritz vectors
// (same M x b shape) when `prev` is given, else the pseudo-random fill.
template <typename T>
__global__ void fill_random_block(T* V, int M, int b, int col0, uint32_t salt, const T* __restrict__ prev) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < M * b; o += gridDim.x * blockDim.x) {
    const int i = o / b, j = o - (o / b) * b;
    if (j < col0) continue;
    if (prev) {
      V[o] = prev[o];
      continue;
    }
    const uint4 w = philox4x32_10((uint32_t)i, (uint32_t)j, 0x4d414348u, salt);
    V[o] = (T)((double)w.x * (1.0 / 4294967296.0) - 0.5);
  }
}

// Partial products for V[:, :r] = Y^T A (Y: I x J row-major, A: I x r
// row-major T): CTA (jb, sp) handles columns [32 jb, 32 jb + 32) of Y over the
// rows i = sp, sp + nsplit, ..; threads (tx, ty): tx = column, ty = row
// phase; coalesced reads of Y rows, A rows broadcast.  Partials land in
// part[sp][j][k] and are summed in split order by yt_reduce_fill (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) yt_times_a_part(const T* __restrict__ Y, const T* __restrict__ A, int I,
                                                       int J, int r, int nsplit, T* __restrict__ part) {
  __shared__ T red[8][32][kMaxRank + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  const int sp = blockIdx.y;
  T acc[kMaxRank];
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) acc[k] = T(0);
  if (j < J) {
    for (int i = sp + ty * nsplit; i < I; i += 8 * nsplit) {
      const T y = Y[(size_t)i * J + j];
      const T* ar = A + (size_t)i * r;
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k)
        if (k < r) acc[k] += y * ar[k];
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) red[ty][tx][k] = acc[k];
  __syncthreads();
  if (ty == 0 && j < J) {
    for (int k = 0; k < r; ++k) {
      T s = T(0);
      for (int g = 0; g < 8; ++g) s += red[g][tx][k];
      part[((size_t)sp * J + j) * r + k] = s;
    }
  }
}

// The whole warm J-route start block in one pass: columns 0..r the sum of
// the Y^T A partials in split order, columns r..b the previous Ritz vectors
// (or the pseudo-random fill).
template <typename T>
__global__ void yt_reduce_fill(const T* __restrict__ part, int nsplit, int J, int r, T* __restrict__ V, int b,
                               uint32_t salt, const T* __restrict__ prev) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < J * b; o += gridDim.x * blockDim.x) {
    const int j = o / b, k = o - (o / b) * b;
    if (k < r) {
      T s = T(0);
      for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * J + j) * r + k];
      V[o] = s;
    } else if (prev) {
      V[o] = prev[o];
    } else {
      const uint4 w = philox4x32_10((uint32_t)j, (uint32_t)k, 0x4d414348u, salt);
      V[o] = (T)((double)w.x * (1.0 / 4294967296.0) - 0.5);
    }
  }
}

template <typename T>
__global__ void copy_cols(const T* __restrict__ A, int M, int r, T* V, int b) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= M * r) return;
  const int i = o / r, k = o - (o / r) * r;
  V[(size_t)i * b + k] = A[o];
}

// ----------------------------------------------------------------------------
// Factor from eigenvectors.  The eigensolver returns its leading Ritz basis
// U_r (M x r, T, leading dimension ldu) and the FP64 rotation X (r x r) that
// the final Rayleigh-Ritz refinement applied to it; the eigenvectors are
// U_r X, formed here (FP64 work spread over the CTAs):
//  J-route: A64[i][k] = sum_m (sum_j Y[i][j] U_r[j][m]) X[m][k] / sqrt(theta_k)
//  I-route: A64[i][k] = sum_m U_r[i][m] X[m][k].
// Then the FP64 re-orthonormalisation A <- A Z: every CTA writes its
// partial Gram A_blk^T A_blk to part[blockIdx] (register accumulation per
// lane, warp partials reduced in shared memory); the last CTA to finish sums
// the partials in block order (deterministic) and stores Z in rinv: the
// series G^-1/2 when G is within 1e-4 of the identity (always, for
// converged eigenvectors), else R^-1 of the Cholesky factor G = R^T R.
// ----------------------------------------------------------------------------
constexpr int kPairsPerLane = (kMaxRank * kMaxRank + 31) / 32;
constexpr size_t kLsvStageBytes = 48 * 1024;

template <typename T>
__global__ void __launch_bounds__(256) lsv_apply_kernel(const T* __restrict__ Y, const T* __restrict__ U, int ldu,
                                                        const double* __restrict__ X,
                                                        const double* __restrict__ theta, int I, int J, int r,
                                                        int jroute, double* __restrict__ A64, double* part,
                                                        unsigned* counter, double* rinv, unsigned* err) {
  __shared__ double wsum[8][kMaxRank * kMaxRank];
  __shared__ double sinv[kMaxRank];
  __shared__ double Xs[kMaxRank * kMaxRank];
  __shared__ bool last;
  // the row products Y U_r run in the arithmetic of Y (T); U_r is staged in
  // shared memory when it fits
  extern __shared__ __align__(16) unsigned char lsv_smem[];
  T* Us = reinterpret_cast<T*>(lsv_smem);
  const bool staged = jroute && (size_t)J * r * sizeof(T) <= kLsvStageBytes;
  if (staged)
    for (int e = threadIdx.x; e < J * r; e += blockDim.x) {
      const int j = e / r, m = e - (e / r) * r;
      Us[e] = U[(size_t)j * ldu + m];
    }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Xs[e] = X[e];
  if (threadIdx.x < r) sinv[threadIdx.x] = theta[threadIdx.x] > 0.0 ? 1.0 / sqrt(theta[threadIdx.x]) : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rr = r * r;
  double gacc[kPairsPerLane];
#pragma unroll
  for (int k = 0; k < kPairsPerLane; ++k) gacc[k] = 0.0;
  for (int i = blockIdx.x * nw + warp; i < I; i += gridDim.x * nw) {
    double u[kMaxRank];
    if (jroute) {
      T sacc[kMaxRank];
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k) sacc[k] = T(0);
      for (int j = lane; j < J; j += 32) {
        const T y = Y[(size_t)i * J + j];
        if (staged) {
#pragma unroll
          for (int k = 0; k < kMaxRank; ++k)
            if (k < r) sacc[k] += y * Us[j * r + k];
        } else {
#pragma unroll
          for (int k = 0; k < kMaxRank; ++k)
            if (k < r) sacc[k] += y * U[(size_t)j * ldu + k];
        }
      }
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k) u[k] = k < r ? (double)warp_sum(sacc[k]) : 0.0;
    } else {
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k) u[k] = k < r ? (double)U[(size_t)i * ldu + k] : 0.0;
    }
    // lane k forms entry k of the row (r FP64 products), then every lane
    // takes the whole row by shuffles for the Gram pairs
    double mine = 0.0;
    if (lane < r) {
#pragma unroll
      for (int m = 0; m < kMaxRank; ++m)
        if (m < r) mine += u[m] * Xs[m * r + lane];
      if (jroute) mine *= sinv[lane];
    }
    double arow[kMaxRank];
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) arow[k] = k < r ? __shfl_sync(0xffffffffu, mine, k) : 0.0;
    if (lane < r) A64[(size_t)i * r + lane] = arow[lane < kMaxRank ? lane : 0];
#pragma unroll
    for (int k = 0; k < kPairsPerLane; ++k) {
      const int pidx = lane + 32 * k;
      if (pidx < rr) {
        const int p = pidx / r, q = pidx - (pidx / r) * r;
        gacc[k] += arow[p] * arow[q];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kPairsPerLane; ++k) {
    const int pidx = lane + 32 * k;
    if (pidx < rr) wsum[warp][pidx] = gacc[k];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rr; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += wsum[w][e];
    part[(size_t)blockIdx.x * rr + e] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // deterministic sum of the partials in block order, one thread per entry
  // (the loads are independent, so they are all in flight at once)
  double* G = &wsum[0][0];
  for (int e = threadIdx.x; e < rr; e += blockDim.x) {
    double t = 0.0;
#pragma unroll 8
    for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(part + (size_t)k * rr + e);
    G[e] = t;
  }
  __syncthreads();
  // The rows are orthonormal up to the eigenvectors' accuracy and rounding,
  // so E = G - I is small: then the symmetric orthonormalisation
  // G^-1/2 = I - E/2 + 3/8 E^2 (the binomial series; the first omitted term,
  // 5/16 E^3, is below 4e-13 for max |E_ij| <= 1e-4) takes three parallel
  // steps instead of the serial FP64 Cholesky.
  __shared__ double emax_w[8];
  {
    double em = 0.0;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
      const int p = e / r, q = e - (e / r) * r;
      em = fmax(em, fabs(G[e] - (p == q ? 1.0 : 0.0)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    if (lane == 0) emax_w[warp] = em;
  }
  __syncthreads();
  double emax = 0.0;
  for (int w = 0; w < nw; ++w) emax = fmax(emax, emax_w[w]);
  if (emax <= 1e-4) {
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
      const int p = e / r, q = e - (e / r) * r;
      double e2 = 0.0;
      for (int k = 0; k < r; ++k)
        e2 += (G[p * r + k] - (p == k ? 1.0 : 0.0)) * (G[k * r + q] - (k == q ? 1.0 : 0.0));
      const double epq = G[e] - (p == q ? 1.0 : 0.0);
      rinv[e] = (p == q ? 1.0 : 0.0) - 0.5 * epq + 0.375 * e2;
    }
    if (threadIdx.x == 0) *counter = 0u;   // ready for the next launch
    return;
  }
  if (warp != 0) return;
  // otherwise: upper Cholesky G = R^T R in place (one warp, lane c owns
  // column c) and A R^-1
  for (int j = 0; j < r; ++j) {
    double djj = G[j * r + j];
    if (!(djj > 0.0)) {
      if (lane == 0) atomicOr(err, DEV_NOTPD);
      djj = 1e-300;
    }
    djj = sqrt(djj);
    __syncwarp();
    if (lane == j) G[j * r + j] = djj;
    if (lane > j && lane < r) G[j * r + lane] /= djj;
    __syncwarp();
    if (lane > j && lane < r)
      for (int c = lane; c < r; ++c) G[lane * r + c] -= G[j * r + lane] * G[j * r + c];
    __syncwarp();
  }
  // R^-1 (upper): lane j back-substitutes column j
  double* Ri = &wsum[1][0];
  if (lane < r) {
    const int j = lane;
    for (int i = r - 1; i >= 0; --i) {
      double v = i == j ? 1.0 : 0.0;
      for (int k = i + 1; k <= j; ++k) v -= G[i * r + k] * Ri[k * r + j];
      Ri[i * r + j] = i > j ? 0.0 : v / G[i * r + i];
    }
  }
  __syncwarp();
  for (int k = lane; k < rr; k += 32) rinv[k] = Ri[k];
  if (lane == 0) *counter = 0u;   // ready for the next launch (it starts at zero with the sample)
}

// A = A64 R^-1: FP64 column-major output (I x r) and the row-major copy in T.
template <typename T>
__global__ void lsv_finish_kernel(const double* __restrict__ A64, const double* __restrict__ rinv, int I, int r,
                                  double* __restrict__ out_colmajor, T* __restrict__ out_rowmajor) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= I * r) return;
  const int i = o / r, k = o - (o / r) * r;
  double s = 0.0;
  for (int j = 0; j < r; ++j) s += A64[(size_t)i * r + j] * rinv[j * r + k];
  out_colmajor[(size_t)k * I + i] = s;
  out_rowmajor[(size_t)i * r + k] = (T)s;
}

// FP64 column-major I x r  ->  row-major T.
template <typename T>
__global__ void factor_to_rowmajor(const double* __restrict__ A, int I, int r, T* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= I * r) return;
  const int i = o / r, k = o - (o / r) * r;
  out[o] = (T)A[(size_t)k * I + i];
}

// Core of the last mode: G[c * r + k] = scale * sum_i A[i][k] Y[i][c], with A
// FP64 column-major (I x r) and Y row-major I x J.  One warp per output.
template <typename T>
__global__ void core_kernel(const T* __restrict__ Y, const double* __restrict__ A, int I, int J, int r,
                            double scale, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= J * r) return;
  const int c = gw / r, k = gw - (gw / r) * r;
  double s = 0.0;
  for (int i = lane; i < I; i += 32) s += A[(size_t)k * I + i] * (double)Y[(size_t)i * J + c];
  s = warp_sum(s);
  if (lane == 0) G[(size_t)c * r + k] = s * scale;
}

}  // namespace

// ----------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------
template <typename T>
mach_status launch_gram(const T* Z, int64_t L, int M, int64_t sl, int64_t sm, T* C, T* partial_scratch,
                        int64_t partial_cap, cudaStream_t st) {
  const int tiles = (M + 31) / 32;
  const int ntiles = tiles * (tiles + 1) / 2;
  int nsplit = (int)std::min<int64_t>(std::max<int64_t>(1, L / 32), std::max(1, num_sms() / ntiles));
  nsplit = std::min(nsplit, 64);
  if ((int64_t)nsplit * M * M > partial_cap) nsplit = 1;
  dim3 grid(tiles, tiles, nsplit);
  if (nsplit == 1) {
    gram_kernel<T><<<grid, 256, 0, st>>>(Z, L, M, sl, sm, 1, C);
    MACH_LAUNCH_CHECK();
    return MACH_OK;
  }
  gram_kernel<T><<<grid, 256, 0, st>>>(Z, L, M, sl, sm, nsplit, partial_scratch);
  MACH_LAUNCH_CHECK();
  const int64_t n = (int64_t)M * M;
  sum_partials_kernel<T><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(partial_scratch,
                                                                                               nsplit, n, C);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename V, typename T>
mach_status launch_init_gram(const void* val, const uint16_t* leaf, const uint32_t* fib_start,
                             const uint32_t* d_nfib, int64_t nfib_cap, int M, T* C, cudaStream_t st) {
  MACH_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(T) * (size_t)M * M, st));
  const int threads = 256;
  const int64_t warps = std::max<int64_t>(1, std::min<int64_t>(nfib_cap, (int64_t)num_sms() * 64));
  init_gram_kernel<V, T><<<(unsigned)ceil_div(warps * 32, threads), threads, 0, st>>>(
      static_cast<const V*>(val), leaf, fib_start, d_nfib, M, C);
  MACH_LAUNCH_CHECK();
  gram_symmetrize_kernel<T><<<(unsigned)std::min<int64_t>(ceil_div((int64_t)M * M, 256), 4096), 256, 0, st>>>(C, M);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}



template <typename T>
mach_status launch_start_block(const T* Y, const T* Aprev, int I, int J, int r, int b, bool jroute, bool warm,
                               T* V, T* scratch, uint32_t salt, const T* prev_ritz, cudaStream_t st) {
  const int M = jroute ? J : I;
  const unsigned fill_grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)M * b, 256), 1024));
  if (!(warm && jroute)) {
    fill_random_block<T><<<fill_grid, 256, 0, st>>>(V, M, b, warm ? r : 0, salt, warm ? prev_ritz : nullptr);
    MACH_LAUNCH_CHECK();
  }
  if (warm) {
    if (jroute) {
      // partials (nsplit x J x r) live in `scratch` (>= 64 J kMaxRank elements)
      const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(
          std::min<int64_t>(64, std::max<int64_t>(1, I / 16)), num_sms() / std::max<int64_t>(1, ceil_div(J, 32))));
      T* part = scratch;
      yt_times_a_part<T><<<dim3((unsigned)ceil_div(J, 32), (unsigned)nsplit), 256, 0, st>>>(Y, Aprev, I, J, r, nsplit,
                                                                                           part);
      MACH_LAUNCH_CHECK();
      yt_reduce_fill<T><<<fill_grid, 256, 0, st>>>(part, nsplit, J, r, V, b, salt, prev_ritz);
    } else {
      copy_cols<T><<<(unsigned)ceil_div((int64_t)I * r, 128), 128, 0, st>>>(Aprev, I, r, V, b);
    }
    MACH_LAUNCH_CHECK();
  }
  return MACH_OK;
}

template <typename T>
mach_status launch_lsv_finish(const T* Y, const EigResult<T>& ev, int I, int J, int r, bool jroute, double* A64,
                              double* gram64, unsigned* counter, double* rinv, unsigned* err, double* out_colmajor,
                              T* out_rowmajor, cudaStream_t st) {
  // the completion counter is zero here: the sample's scalars start zeroed
  // and the last CTA of every launch resets it
  // few partial Grams for the last CTA to sum: at most 64 CTAs, several rows per warp
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 32), 64));
  const size_t vbytes = (size_t)J * r * sizeof(T);
  const size_t smem = jroute && vbytes <= kLsvStageBytes ? vbytes : 0;
  lsv_apply_kernel<T><<<blocks, 256, smem, st>>>(Y, ev.U, ev.ldu, ev.X, ev.theta, I, J, r, jroute ? 1 : 0, A64,
                                                  gram64, counter, rinv, err);
  MACH_LAUNCH_CHECK();
  lsv_finish_kernel<T><<<(unsigned)ceil_div((int64_t)I * r, 256), 256, 0, st>>>(A64, rinv, I, r, out_colmajor,
                                                                                 out_rowmajor);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename T>
mach_status launch_factor_to_rowmajor(const double* A, int I, int r, T* out, cudaStream_t st) {
  factor_to_rowmajor<T><<<(unsigned)ceil_div((int64_t)I * r, 256), 256, 0, st>>>(A, I, r, out);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename T>
mach_status launch_core(const T* Y, const double* A, int I, int J, int r, double scale, double* G,
                        cudaStream_t st) {
  const int64_t warps = (int64_t)J * r;
  core_kernel<T><<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(Y, A, I, J, r, scale, G);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

#define MACH_INST(T)                                                                                             \
  template mach_status launch_gram<T>(const T*, int64_t, int, int64_t, int64_t, T*, T*, int64_t, cudaStream_t);  \
  template mach_status launch_start_block<T>(const T*, const T*, int, int, int, int, bool, bool, T*, T*,       \
                                             uint32_t, const T*, cudaStream_t);                                  \
  template mach_status launch_lsv_finish<T>(const T*, const EigResult<T>&, int, int, int, bool, double*,        \
                                            double*, unsigned*, double*, unsigned*, double*, T*, cudaStream_t);  \
  template mach_status launch_factor_to_rowmajor<T>(const double*, int, int, T*, cudaStream_t);                  \
  template mach_status launch_core<T>(const T*, const double*, int, int, int, double, double*, cudaStream_t);
MACH_INST(float)
MACH_INST(double)
#undef MACH_INST

template mach_status launch_init_gram<float, float>(const void*, const uint16_t*, const uint32_t*,
                                                    const uint32_t*, int64_t, int, float*, cudaStream_t);
template mach_status launch_init_gram<float, double>(const void*, const uint16_t*, const uint32_t*,
                                                     const uint32_t*, int64_t, int, double*, cudaStream_t);
template mach_status launch_init_gram<double, float>(const void*, const uint16_t*, const uint32_t*,
                                                     const uint32_t*, int64_t, int, float*, cudaStream_t);
template mach_status launch_init_gram<double, double>(const void*, const uint16_t*, const uint32_t*,
                                                      const uint32_t*, int64_t, int, double*, cudaStream_t);

}  // namespace mach
