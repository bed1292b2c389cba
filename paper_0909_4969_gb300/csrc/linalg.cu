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
// x_a x_b for every pair of entries of a fibre.  One warp per fibre.
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
    for (uint32_t i = s0 + lane; i < s1; i += 32) {
      const uint32_t a = leaf[i];
      const T vi = (T)val[i];
      for (uint32_t j = i; j < s1; ++j) {
        const uint32_t b = leaf[j];
        const T v = vi * (T)val[j];
        atomicAdd(&C[(size_t)a * M + b], v);
        if (a != b) atomicAdd(&C[(size_t)b * M + a], v);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Cyclic Jacobi for a small symmetric matrix (n <= 32) held in shared memory
// (row-major, leading dimension ld), all threads of the CTA.  On return H is
// (nearly) diagonal and Qm holds the eigenvectors in its columns.
// Rotation (Golub & Van Loan, sym.schur2): tau = (h_qq - h_pp) / (2 h_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c;
// H <- J^T H J with J_pp = J_qq = c, J_pq = s, J_qp = -s.  Each round applies
// n/2 disjoint rotations (round-robin ordering); every element of the column
// and row updates belongs to exactly one thread.  Sweeps stop at the relative
// off-diagonal tolerance, or at the rounding floor (quadratic convergence: a
// sweep that no longer cuts the off-diagonal mass 4x near the floor).
template <typename T>
__device__ void jacobi_block(T* H, T* Qm, int n, int ld, int max_sweeps, T rel_tol, T* cs, int* pq, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    Qm[i * ld + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  if (n <= 1) return;
  const int np = (n + 1) & ~1;  // even number of players (a dummy when n is odd)
  const int npairs = np / 2;
  double prev_off = -1.0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e - (e / n) * n;
      const double h = (double)H[i * ld + j];
      if (i == j) dia += h * h; else off += h * h;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (lane == 0) {
      red[2 * warp] = off;
      red[2 * warp + 1] = dia;
    }
    __syncthreads();
    off = 0.0;
    dia = 0.0;
    for (int w = 0; w < nw; ++w) {
      off += red[2 * w];
      dia += red[2 * w + 1];
    }
    __syncthreads();
    if (off <= (double)rel_tol * (double)rel_tol * dia) break;
    const double floor_rel = sizeof(T) == 8 ? 1e-12 : 1e-4;
    if (prev_off >= 0.0 && off > 0.25 * prev_off && off <= floor_rel * floor_rel * dia) break;
    prev_off = off;
    for (int round = 0; round < np - 1; ++round) {
      if (tid < npairs) {
        const int pa = tid, pb = np - 1 - tid;
        int p = pa == 0 ? 0 : ((pa - 1 + round) % (np - 1)) + 1;
        int q = pb == 0 ? 0 : ((pb - 1 + round) % (np - 1)) + 1;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        T c = T(1), s = T(0);
        if (q < n) {
          const T hpq = H[p * ld + q];
          const T hpp = H[p * ld + p], hqq = H[q * ld + q];
          if (hpq != T(0)) {
            const T tau = (hqq - hpp) / (T(2) * hpq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            s = t * c;
          }
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        pq[2 * tid] = p;
        pq[2 * tid + 1] = q < n ? q : -1;
      }
      __syncthreads();
      // H <- H J and Qm <- Qm J (column rotations): element (i, pair k)
      for (int e = tid; e < npairs * n; e += nt) {
        const int k = e / n, i = e - (e / n) * n;
        const int q = pq[2 * k + 1];
        if (q < 0) continue;
        const int p = pq[2 * k];
        const T c = cs[2 * k], s = cs[2 * k + 1];
        const T hp = H[i * ld + p], hq = H[i * ld + q];
        H[i * ld + p] = c * hp - s * hq;
        H[i * ld + q] = s * hp + c * hq;
        const T qp = Qm[i * ld + p], qq = Qm[i * ld + q];
        Qm[i * ld + p] = c * qp - s * qq;
        Qm[i * ld + q] = s * qp + c * qq;
      }
      __syncthreads();
      // H <- J^T H (row rotations): element (pair k, j)
      for (int e = tid; e < npairs * n; e += nt) {
        const int k = e / n, j = e - (e / n) * n;
        const int q = pq[2 * k + 1];
        if (q < 0) continue;
        const int p = pq[2 * k];
        const T c = cs[2 * k], s = cs[2 * k + 1];
        const T hp = H[p * ld + j], hq = H[q * ld + j];
        H[p * ld + j] = c * hp - s * hq;
        H[q * ld + j] = s * hp + c * hq;
      }
      __syncthreads();
    }
  }
}

// Order of eigenvalues (diagonal of H) descending -> perm[0..n)
template <typename T>
__device__ void sort_desc_warp(const T* H, int n, int ld, int* perm) {
  const int lane = threadIdx.x & 31;
  if (lane < n) {
    const T v = H[lane * ld + lane];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T u = H[j * ld + j];
      rank += (u > v) || (u == v && j < lane);
    }
    perm[rank] = lane;
  }
  __syncwarp();
}

// Block-wide reduction of NV values per thread into out[0..NV) (smem result).
template <typename T, int NV>
__device__ void block_reduce_vec(T (&v)[NV], T* red /* [warps][NV] */, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * NV + k] = v[k];
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    T s = T(0);
    for (int w = 0; w < nw; ++w) s += red[w * NV + k];
    out[k] = s;
  }
  __syncthreads();
}

constexpr int kEigThreads = 256;
constexpr int kEigWarps = kEigThreads / 32;
constexpr int kBMax = 32;
constexpr int kEigSmallMax = 256;   // larger Grams take the split (multi-CTA) path
constexpr int kChunk = 32;          // rows per shared-memory chunk in streamed reductions

// Shared-memory state of one Rayleigh-Ritz step.
template <typename T>
struct RRShared {
  T H[kBMax * kBMax];
  T Qm[kBMax * kBMax];
  T G[kBMax * kBMax];
  T cs[kBMax * 2];
  T xa[kChunk * kBMax];   // row chunk of the left operand
  T xb[kChunk * kBMax];   // row chunk of the right operand
  int pq[kBMax * 2];
  int perm[kBMax];
  double red[kEigWarps * kBMax];
  double res[kBMax];
  int conv;
};

// Iteration control kept in global memory between split-path launches.
struct EigCtl {
  int done;
  int it;
  double prev_worst;
};

template <typename T>
struct EigArgs {
  const T* C;          // M x M symmetric (row-major), global
  int M, r, b;
  T* V;                // M x b, holds V0 on entry (global)
  T* W;                // M x b (global scratch)
  T* U;                // M x b (global scratch)
  double* Vout;        // M x r, FP64 leading eigenvectors (row-major)
  double* theta;       // r eigenvalues, FP64, descending
  int maxit;
  double tol;          // relative residual tolerance
  EigCtl* ctl;         // split path only
  unsigned long long* stats;  // [0] calls, [1] iterations, [2] unconverged
  T* basis_out;        // M x b: the final Ritz block (warm start of the next solve), or null
};

// W[:, :ncols] = C V[:, :ncols] (row stride b for V and W).  A warp owns RPW
// rows of C at a time, lane j owns column j of V: each step reads one
// coalesced row of V (shared by the RPW rows) and RPW broadcast entries of C.
// Rows [row0, row1) are shared among `nwarps` warps.
template <typename T, int RPW = 4>
__device__ void cv_rows(const T* C, int ldc, const T* V, T* W, int M, int b, int ncols, int row0, int row1,
                        int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  for (int i0 = row0 + RPW * warp; i0 < row1; i0 += RPW * nwarps) {
    const int nr = min(RPW, row1 - i0);
    const T* crow[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) crow[q] = C + (size_t)(i0 + (q < nr ? q : 0)) * ldc;
    T acc[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) acc[q] = T(0);
    if (lane < ncols) {
      const T* vc = V + lane;
#pragma unroll 4
      for (int k = 0; k < M; ++k) {
        const T v = vc[(size_t)k * b];
#pragma unroll
        for (int q = 0; q < RPW; ++q) acc[q] += crow[q][k] * v;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q)
        if (q < nr) W[(size_t)(i0 + q) * b + lane] = acc[q];
    }
  }
}

// H = X^T Y (b x b, row-major ld kBMax) for M x b row-major X, Y; rows are
// streamed through shared memory in chunks (works for global or shared
// sources).  Thread t owns the entries t, t + 256, .. of H.
template <typename T>
__device__ void gram_xty(const T* X, const T* Y, int M, int b, T* H, RRShared<T>& sh) {
  T acc[(kBMax * kBMax) / kEigThreads];
#pragma unroll
  for (int k = 0; k < (kBMax * kBMax) / kEigThreads; ++k) acc[k] = T(0);
  for (int c0 = 0; c0 < M; c0 += kChunk) {
    const int nr = min(kChunk, M - c0);
    for (int o = threadIdx.x; o < nr * b; o += blockDim.x) {
      sh.xa[o] = X[(size_t)c0 * b + o];
      sh.xb[o] = Y[(size_t)c0 * b + o];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (kBMax * kBMax) / kEigThreads; ++k) {
      const int e = threadIdx.x + k * kEigThreads;
      if (e < b * b) {
        const int p = e / b, q = e - (e / b) * b;
        T s = acc[k];
        for (int i = 0; i < nr; ++i) s += sh.xa[i * b + p] * sh.xb[i * b + q];
        acc[k] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < (kBMax * kBMax) / kEigThreads; ++k) {
    const int e = threadIdx.x + k * kEigThreads;
    if (e < b * b) H[(e / b) * kBMax + (e - (e / b) * b)] = acc[k];
  }
  __syncthreads();
}

// Orthonormalise the columns of X (M x b) in place in precision T: column
// scaling, then Cholesky QR twice (X <- X R^-1).  Used on blocks whose
// columns are already nearly orthogonal (C times Ritz vectors), so the Gram
// is well conditioned after scaling.
template <typename T>
__device__ void orth_block(T* X, int M, int b, RRShared<T>& sh) {
  for (int pass = 0; pass < 3; ++pass) {
    gram_xty<T>(X, X, M, b, sh.G, sh);
    if (pass == 0) {
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        T* xr = X + (size_t)i * b;
        for (int j = 0; j < b; ++j) {
          const T nrm = sqrt(sh.G[j * kBMax + j]);
          xr[j] = nrm > T(0) ? xr[j] / nrm : T(0);
        }
      }
      __syncthreads();
      continue;
    }
    // right-looking Cholesky G = R^T R (R upper, in place), warp 0
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int j = 0; j < b; ++j) {
        T djj = sh.G[j * kBMax + j];
        djj = djj > T(0) ? sqrt(djj) : T(1e-30);
        __syncwarp();
        if (lane == 0) sh.G[j * kBMax + j] = djj;
        for (int c = j + 1 + lane; c < b; c += 32) sh.G[j * kBMax + c] /= djj;
        __syncwarp();
        for (int c = j + 1 + lane; c < b; c += 32)
          for (int c2 = c; c2 < b; ++c2) sh.G[c * kBMax + c2] -= sh.G[j * kBMax + c] * sh.G[j * kBMax + c2];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      T xr[kBMax];
      for (int j = 0; j < b; ++j) xr[j] = X[(size_t)i * b + j];
      for (int j = 0; j < b; ++j) {
        T v = xr[j];
        for (int k = 0; k < j; ++k) v -= xr[k] * sh.G[k * kBMax + j];
        xr[j] = v / sh.G[j * kBMax + j];
      }
      for (int j = 0; j < b; ++j) X[(size_t)i * b + j] = xr[j];
    }
    __syncthreads();
  }
}

// One Rayleigh-Ritz step given V (orthonormal, M x b) and W = C V:
// H = V^T W, H = Q Theta Q^T (Jacobi), U = V Q (Ritz vectors), W <- W Q,
// residuals ||W_j - theta_j U_j|| of the leading r.  Converged when every
// residual is below tol * theta_1, or when the residual has reached the
// arithmetic's floor (below 10 tol and no longer halving).  If not
// converged, V <- orth(W) for the next power step.  Returns converged.
template <typename T>
__device__ bool rr_step(T* V, T* W, T* U, int M, int b, int r, double tol, double* prev_worst, RRShared<T>& sh) {
  gram_xty<T>(V, W, M, b, sh.H, sh);
  // symmetrise (rounding) before Jacobi
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e - (e / b) * b;
    if (p < q) {
      const T avg = (sh.H[p * kBMax + q] + sh.H[q * kBMax + p]) * T(0.5);
      sh.H[p * kBMax + q] = avg;
      sh.H[q * kBMax + p] = avg;
    }
  }
  __syncthreads();
  jacobi_block<T>(sh.H, sh.Qm, b, kBMax, 20, sizeof(T) == 8 ? T(1e-15) : T(1e-7), sh.cs, sh.pq, sh.red);
  if (threadIdx.x < 32) sort_desc_warp<T>(sh.H, b, kBMax, sh.perm);
  __syncthreads();
  double loc[kBMax];
  for (int j = 0; j < kBMax; ++j) loc[j] = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    T vr[kBMax], wr[kBMax];
    for (int k = 0; k < b; ++k) {
      vr[k] = V[(size_t)i * b + k];
      wr[k] = W[(size_t)i * b + k];
    }
    for (int j = 0; j < b; ++j) {
      const int pj = sh.perm[j];
      T su = T(0), sw = T(0);
      for (int k = 0; k < b; ++k) {
        const T q = sh.Qm[k * kBMax + pj];
        su += vr[k] * q;
        sw += wr[k] * q;
      }
      U[(size_t)i * b + j] = su;
      W[(size_t)i * b + j] = sw;
      if (j < r) {
        const double d = (double)sw - (double)sh.H[pj * kBMax + pj] * (double)su;
        loc[j] += d * d;
      }
    }
  }
  block_reduce_vec<double, kBMax>(loc, sh.red, sh.res);
  if (threadIdx.x == 0) {
    const double th0 = fabs((double)sh.H[sh.perm[0] * kBMax + sh.perm[0]]);
    double worst = 0.0;
    for (int j = 0; j < r; ++j) worst = fmax(worst, sqrt(sh.res[j]));
    const double rel = th0 > 0.0 ? worst / th0 : 0.0;
    const bool floor_hit = rel < 10.0 * tol && rel > 0.5 * (*prev_worst);
    sh.conv = (th0 == 0.0) || (rel <= tol) || floor_hit;
    *prev_worst = rel;
  }
  __syncthreads();
  if (sh.conv) return true;
  for (int o = threadIdx.x; o < M * b; o += blockDim.x) V[o] = W[o];
  __syncthreads();
  orth_block<T>(V, M, b, sh);
  return false;
}

// Final Rayleigh-Ritz of the leading r Ritz vectors in FP64: with
// W[:, :r] = C U[:, :r], H64 = U_r^T W_r (FP64 accumulation), FP64 Jacobi,
// Vout = U_r Q64 (FP64).
template <typename T>
__device__ void final_rr(const T* U, const T* W, int M, int b, int r, double* Vout, double* theta,
                         RRShared<T>& sh, double* H64, double* Q64, double* cs64) {
  for (int pidx = threadIdx.x; pidx < r * r; pidx += blockDim.x) {
    const int p = pidx / r, q = pidx - (pidx / r) * r;
    if (q < p) continue;
    double s = 0.0;
    for (int i = 0; i < M; ++i) s += (double)U[(size_t)i * b + p] * (double)W[(size_t)i * b + q];
    H64[p * kBMax + q] = s;
    H64[q * kBMax + p] = s;
  }
  __syncthreads();
  jacobi_block<double>(H64, Q64, r, kBMax, 30, 1e-15, cs64, sh.pq, sh.red);
  if (threadIdx.x < 32) sort_desc_warp<double>(H64, r, kBMax, sh.perm);
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double ur[kMaxRank];
    for (int k = 0; k < r; ++k) ur[k] = (double)U[(size_t)i * b + k];
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int k = 0; k < r; ++k) s += ur[k] * Q64[k * kBMax + sh.perm[j]];
      Vout[(size_t)i * r + j] = s;
    }
  }
  if (threadIdx.x < r) theta[threadIdx.x] = H64[sh.perm[threadIdx.x] * kBMax + sh.perm[threadIdx.x]];
  __syncthreads();
}

// Shared-memory plan of the fused kernel: V, W, U and then C when they fit
// in `budget` bytes of dynamic shared memory (mode 2: all in smem, 1: V/W/U
// only, 0: everything stays in global memory).
struct EigSmemPlan {
  int mode;
  size_t bytes;
};

inline EigSmemPlan eig_smem_plan(int M, int b, size_t elem, size_t budget) {
  EigSmemPlan p;
  const size_t vwu = (size_t)3 * M * b * elem;
  const size_t c = (size_t)M * M * elem;
  if (vwu + c <= budget) {
    p.mode = 2;
    p.bytes = vwu + c;
  } else if (vwu <= budget) {
    p.mode = 1;
    p.bytes = vwu;
  } else {
    p.mode = 0;
    p.bytes = 0;
  }
  return p;
}

// Fused path (one CTA, M <= kEigSmallMax): operands in shared memory, power
// step + Rayleigh-Ritz until converged, final FP64 Rayleigh-Ritz.
template <typename T>
__global__ void __launch_bounds__(kEigThreads) eig_kernel(EigArgs<T> a, int smem_mode) {
  extern __shared__ __align__(16) unsigned char eig_smem[];
  __shared__ RRShared<T> sh;
  __shared__ double H64[kBMax * kBMax];
  __shared__ double Q64[kBMax * kBMax];
  __shared__ double cs64[kBMax * 2];
  __shared__ double prev;
  const int M = a.M, b = a.b, r = a.r;
  T* V = a.V;
  T* W = a.W;
  T* U = a.U;
  const T* C = a.C;
  if (smem_mode >= 1) {
    V = reinterpret_cast<T*>(eig_smem);
    W = V + (size_t)M * b;
    U = W + (size_t)M * b;
    for (int o = threadIdx.x; o < M * b; o += blockDim.x) V[o] = a.V[o];
  }
  if (smem_mode == 2) {
    T* Cs = U + (size_t)M * b;
    for (int o = threadIdx.x; o < M * M; o += blockDim.x) Cs[o] = a.C[o];
    C = Cs;
  }
  if (threadIdx.x == 0) prev = 1e300;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  orth_block<T>(V, M, b, sh);
  int it = 0;
  bool conv = false;
  for (; it < a.maxit; ++it) {
    cv_rows<T>(C, M, V, W, M, b, b, 0, M, warp, kEigWarps);
    __syncthreads();
    if (rr_step<T>(V, W, U, M, b, r, a.tol, &prev, sh)) {
      conv = true;
      break;
    }
  }
  if (a.basis_out)
    for (int o = threadIdx.x; o < M * b; o += blockDim.x) a.basis_out[o] = U[o];
  cv_rows<T>(C, M, U, W, M, b, r, 0, M, warp, kEigWarps);
  __syncthreads();
  final_rr<T>(U, W, M, b, r, a.Vout, a.theta, sh, H64, Q64, cs64);
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[0], 1ull);
    atomicAdd(&a.stats[1], (unsigned long long)(it + (conv ? 1 : 0)));
    if (!conv) atomicAdd(&a.stats[2], 1ull);
  }
}

// Split path (large M): eig_begin (orth), then per iteration the multi-CTA
// product and the single-CTA Rayleigh-Ritz step, then the product with the
// leading Ritz vectors and eig_end (FP64 Rayleigh-Ritz).  Iterations after
// convergence return at once (device flag).
template <typename T>
__global__ void __launch_bounds__(kEigThreads) eig_begin_kernel(EigArgs<T> a) {
  __shared__ RRShared<T> sh;
  if (threadIdx.x == 0) {
    a.ctl->done = 0;
    a.ctl->it = 0;
    a.ctl->prev_worst = 1e300;
  }
  orth_block<T>(a.V, a.M, a.b, sh);
}

template <typename T>
__global__ void __launch_bounds__(256) symm_mul_kernel(EigArgs<T> a, const T* V, T* W, int ncols, int respect_done) {
  if (respect_done && a.ctl->done) return;
  const int row0 = blockIdx.x * 8;
  cv_rows<T, 1>(a.C, a.M, V, W, a.M, a.b, ncols, row0, min(a.M, row0 + 8), threadIdx.x >> 5, 8);
}

template <typename T>
__global__ void __launch_bounds__(kEigThreads) eig_step_kernel(EigArgs<T> a) {
  __shared__ RRShared<T> sh;
  __shared__ double prev;
  if (a.ctl->done) return;
  if (threadIdx.x == 0) prev = a.ctl->prev_worst;
  __syncthreads();
  const bool conv = rr_step<T>(a.V, a.W, a.U, a.M, a.b, a.r, a.tol, &prev, sh);
  if (threadIdx.x == 0) {
    a.ctl->it += 1;
    a.ctl->prev_worst = prev;
    if (conv || a.ctl->it >= a.maxit) a.ctl->done = conv ? 1 : 2;
  }
}

template <typename T>
__global__ void __launch_bounds__(kEigThreads) eig_end_kernel(EigArgs<T> a) {
  __shared__ RRShared<T> sh;
  __shared__ double H64[kBMax * kBMax];
  __shared__ double Q64[kBMax * kBMax];
  __shared__ double cs64[kBMax * 2];
  if (a.basis_out)
    for (int o = threadIdx.x; o < a.M * a.b; o += blockDim.x) a.basis_out[o] = a.U[o];
  final_rr<T>(a.U, a.W, a.M, a.b, a.r, a.Vout, a.theta, sh, H64, Q64, cs64);
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[0], 1ull);
    atomicAdd(&a.stats[1], (unsigned long long)a.ctl->it);
    if (a.ctl->done != 1) atomicAdd(&a.stats[2], 1ull);
  }
}

// ----------------------------------------------------------------------------
// Starting blocks.  Deterministic pseudo-random fill (Philox of (i, j)) for
// the columns not given by a warm start.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void fill_random_block(T* V, int M, int b, int col0, uint32_t salt) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < M * b; o += gridDim.x * blockDim.x) {
    const int i = o / b, j = o - (o / b) * b;
    if (j < col0) continue;
    const uint4 w = philox4x32_10((uint32_t)i, (uint32_t)j, 0x4d414348u, salt);
    V[o] = (T)((double)w.x * (1.0 / 4294967296.0) - 0.5);
  }
}

// Partial products for V[:, :r] = Y^T A (Y: I x J row-major, A: I x r
// row-major T): CTA (jb, sp) handles columns [32 jb, 32 jb + 32) of Y over the
// rows i = sp, sp + nsplit, ..; threads (tx, ty): tx = column, ty = row
// phase; coalesced reads of Y rows, A rows broadcast.  Partials land in
// part[sp][j][k] and are summed in split order by yt_reduce (deterministic).
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

template <typename T>
__global__ void yt_reduce(const T* __restrict__ part, int nsplit, int J, int r, T* __restrict__ V, int b) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= J * r) return;
  const int j = o / r, k = o - (o / r) * r;
  T s = T(0);
  for (int sp = 0; sp < nsplit; ++sp) s += part[(size_t)sp * J * r + o];
  V[(size_t)j * b + k] = s;
}

template <typename T>
__global__ void copy_cols(const T* __restrict__ A, int M, int r, T* V, int b) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= M * r) return;
  const int i = o / r, k = o - (o / r) * r;
  V[(size_t)i * b + k] = A[o];
}

// ----------------------------------------------------------------------------
// Factor from eigenvectors:
//  J-route: A64[i][k] = sum_j Y[i][j] Vout[j][k] / sqrt(theta_k)   (FP64)
//  I-route: A64 = Vout.
// Then FP64 Cholesky QR: G = A^T A (atomics into gram64), last block
// factors G = R^T R and stores R^-1 (upper) in rinv.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void lsv_apply_kernel(const T* __restrict__ Y, const double* __restrict__ Vout,
                                 const double* __restrict__ theta, int I, int J, int r, int jroute,
                                 double* __restrict__ A64, double* gram64, unsigned* counter, double* rinv,
                                 unsigned* err) {
  __shared__ double sG[kMaxRank * kMaxRank];
  __shared__ double sinv[kMaxRank];
  __shared__ bool last;
  for (int k = threadIdx.x; k < r * r; k += blockDim.x) sG[k] = 0.0;
  if (threadIdx.x < r) sinv[threadIdx.x] = theta[threadIdx.x] > 0.0 ? 1.0 / sqrt(theta[threadIdx.x]) : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = blockIdx.x * nw + warp; i < I; i += gridDim.x * nw) {
    double arow[kMaxRank];
    if (jroute) {
      double s[kMaxRank];
      for (int k = 0; k < kMaxRank; ++k) s[k] = 0.0;
      for (int j = lane; j < J; j += 32) {
        const double y = (double)Y[(size_t)i * J + j];
        for (int k = 0; k < r; ++k) s[k] += y * Vout[(size_t)j * r + k];
      }
      for (int k = 0; k < r; ++k) arow[k] = warp_sum(s[k]) * sinv[k];
    } else {
      for (int k = 0; k < r; ++k) arow[k] = Vout[(size_t)i * r + k];
    }
    if (lane < r) A64[(size_t)i * r + lane] = arow[lane];
    // partial Gram
    for (int pidx = lane; pidx < r * r; pidx += 32) {
      const int p = pidx / r, q = pidx - (pidx / r) * r;
      atomicAdd(&sG[pidx], arow[p] * arow[q]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r * r; k += blockDim.x) atomicAdd(&gram64[k], sG[k]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  // Cholesky of gram64 (volatile reads of the accumulated values)
  double R[kMaxRank * kMaxRank];
  for (int k = 0; k < r * r; ++k) R[k] = ((volatile double*)gram64)[k];
  for (int j = 0; j < r; ++j) {
    double djj = R[j * r + j];
    for (int k = 0; k < j; ++k) djj -= R[k * r + j] * R[k * r + j];
    if (!(djj > 0.0)) {
      atomicOr(err, DEV_NOTPD);
      djj = 1e-300;
    }
    djj = sqrt(djj);
    R[j * r + j] = djj;
    for (int c = j + 1; c < r; ++c) {
      double v = R[j * r + c];
      for (int k = 0; k < j; ++k) v -= R[k * r + j] * R[k * r + c];
      R[j * r + c] = v / djj;
    }
    for (int c = 0; c < j; ++c) R[j * r + c] = 0.0;
  }
  // inverse of upper-triangular R
  double Ri[kMaxRank * kMaxRank];
  for (int k = 0; k < r * r; ++k) Ri[k] = 0.0;
  for (int j = 0; j < r; ++j) {
    Ri[j * r + j] = 1.0 / R[j * r + j];
    for (int i = j - 1; i >= 0; --i) {
      double v = 0.0;
      for (int k = i + 1; k <= j; ++k) v += R[i * r + k] * Ri[k * r + j];
      Ri[i * r + j] = -v / R[i * r + i];
    }
  }
  for (int k = 0; k < r * r; ++k) rinv[k] = Ri[k];
}

// A = A64 R^-1: FP64 column-major output (I x r) and the row-major copy in T.
template <typename T>
__global__ void lsv_finish_kernel(const double* __restrict__ A64, const double* __restrict__ rinv, int I, int r,
                                  double* __restrict__ out_colmajor, T* __restrict__ out_rowmajor) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= I * r) return;
  const int i = o / r, k = o - (o / r) * r;
  double s = 0.0;
  for (int j = 0; j <= k; ++j) s += A64[(size_t)i * r + j] * rinv[j * r + k];
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
  int nsplit = (int)std::min<int64_t>(std::max<int64_t>(1, L / 256), 64);
  const int ntiles = tiles * (tiles + 1) / 2;
  while (nsplit > 1 && (int64_t)ntiles * nsplit > 4 * num_sms()) nsplit /= 2;
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
  return MACH_OK;
}



template <typename T>
mach_status launch_eig(const T* C, const EigLaunch& e, cudaStream_t st) {
  EigArgs<T> a;
  a.C = C;
  a.M = e.M;
  a.r = e.r;
  a.b = e.b;
  a.V = static_cast<T*>(e.V);
  a.W = static_cast<T*>(e.W);
  a.U = static_cast<T*>(e.U);
  a.Vout = e.Vout;
  a.theta = e.theta;
  a.maxit = e.maxit;
  a.tol = e.tol;
  a.ctl = static_cast<EigCtl*>(e.ctl);
  a.stats = e.stats;
  a.basis_out = static_cast<T*>(e.basis_out);
  if (e.M <= kEigSmallMax) {
    cudaFuncAttributes fa;
    MACH_CUDA_TRY(cudaFuncGetAttributes(&fa, eig_kernel<T>));
    int dev = 0, optin = 0;
    MACH_CUDA_TRY(cudaGetDevice(&dev));
    MACH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t budget = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
    const EigSmemPlan plan = eig_smem_plan(e.M, e.b, sizeof(T), budget);
    MACH_CUDA_TRY(cudaFuncSetAttribute(eig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.bytes));
    eig_kernel<T><<<1, kEigThreads, plan.bytes, st>>>(a, plan.mode);
    MACH_LAUNCH_CHECK();
    return MACH_OK;
  }
  const unsigned rows = (unsigned)ceil_div(e.M, 8);
  eig_begin_kernel<T><<<1, kEigThreads, 0, st>>>(a);
  MACH_LAUNCH_CHECK();
  for (int it = 0; it < e.maxit; ++it) {
    symm_mul_kernel<T><<<rows, 256, 0, st>>>(a, a.V, a.W, e.b, 1);
    MACH_LAUNCH_CHECK();
    eig_step_kernel<T><<<1, kEigThreads, 0, st>>>(a);
    MACH_LAUNCH_CHECK();
  }
  symm_mul_kernel<T><<<rows, 256, 0, st>>>(a, a.U, a.W, e.r, 0);
  MACH_LAUNCH_CHECK();
  eig_end_kernel<T><<<1, kEigThreads, 0, st>>>(a);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename T>
mach_status launch_start_block(const T* Y, const T* Aprev, int I, int J, int r, int b, bool jroute, bool warm,
                               T* V, T* scratch, uint32_t salt, cudaStream_t st) {
  const int M = jroute ? J : I;
  fill_random_block<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)M * b, 256), 1024)),
                         256, 0, st>>>(V, M, b, warm ? r : 0, salt);
  MACH_LAUNCH_CHECK();
  if (warm) {
    if (jroute) {
      // partials (nsplit x J x r) live in `scratch`, which holds J x 32
      // elements, so nsplit <= 32 / r
      const int nsplit = std::max(1, std::min(32 / std::max(r, 1), std::max(1, I / 64)));
      T* part = scratch;
      yt_times_a_part<T><<<dim3((unsigned)ceil_div(J, 32), (unsigned)nsplit), 256, 0, st>>>(Y, Aprev, I, J, r, nsplit,
                                                                                           part);
      MACH_LAUNCH_CHECK();
      yt_reduce<T><<<(unsigned)ceil_div((int64_t)J * r, 128), 128, 0, st>>>(part, nsplit, J, r, V, b);
    } else {
      copy_cols<T><<<(unsigned)ceil_div((int64_t)I * r, 128), 128, 0, st>>>(Aprev, I, r, V, b);
    }
    MACH_LAUNCH_CHECK();
  }
  return MACH_OK;
}

template <typename T>
mach_status launch_lsv_finish(const T* Y, const double* Vout, const double* theta, int I, int J, int r, bool jroute,
                              double* A64, double* gram64, unsigned* counter, double* rinv, unsigned* err,
                              double* out_colmajor, T* out_rowmajor, cudaStream_t st) {
  MACH_CUDA_TRY(cudaMemsetAsync(gram64, 0, sizeof(double) * r * r, st));
  MACH_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(I, 8), 2 * num_sms()));
  lsv_apply_kernel<T><<<blocks, 256, 0, st>>>(Y, Vout, theta, I, J, r, jroute ? 1 : 0, A64, gram64, counter, rinv,
                                               err);
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
  template mach_status launch_eig<T>(const T*, const EigLaunch&, cudaStream_t);                                  \
  template mach_status launch_start_block<T>(const T*, const T*, int, int, int, int, bool, bool, T*, T*,       \
                                             uint32_t, cudaStream_t);                                            \
  template mach_status launch_lsv_finish<T>(const T*, const double*, const double*, int, int, int, bool,         \
                                            double*, double*, unsigned*, double*, unsigned*, double*, T*,        \
                                            cudaStream_t);                                                       \
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
