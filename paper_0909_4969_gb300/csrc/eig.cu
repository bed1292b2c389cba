// Leading eigenvectors of a small symmetric positive semi-definite Gram matrix
// C (M x M): the "r_i leading left singular vectors" step of Algorithm 2 and
// of HOSVD (Section 2.1), computed by block subspace iteration with a
// Rayleigh-Ritz step in every iteration (the Lanczos-class "under-the-hood"
// solver of Section 3 Remark 4).
//
// One iteration, with V (M x b) orthonormal:
//   W = C V;  H = V^T W;  P = W^T W                       (M-length passes)
//   H = Q Theta Q^T (cyclic Jacobi, one warp)             (b-space)
//   E = W - V H,  F = E^T E;  residual of Ritz pair j:
//       ||C u_j - theta_j u_j|| = sqrt(q_j^T F q_j)       (no cancellation)
//   next basis V <- W Q D R^-1, R = chol(D Q^T P Q D), D = column scaling
// All b x b work (Jacobi, Cholesky, the small products) runs on one warp in
// shared memory; every M-length pass is a single sweep over rows.  Small
// Grams (M <= 256) run in one CTA with operands in shared memory; larger
// ones (HOSVD of long modes) run the same steps as multi-CTA launches with a
// fixed iteration count.  A final Rayleigh-Ritz of the leading r Ritz vectors
// is done in FP64.
#include "mach_internal.cuh"
#include "jacobi.cuh"

namespace mach {

namespace {

#ifdef MACH_EIG_PHASES
// debugging aid: clock cycles of the fused eigensolver's phases, summed
// over its launches (read with mach_debug_eig_phases in such a build)
__device__ unsigned long long g_eig_phase[16];
#define EIG_MARK(k)                                                              \
  do {                                                                           \
    __syncthreads();                                                             \
    const long long t_ = clock64();                                              \
    if (threadIdx.x == 0) atomicAdd(&g_eig_phase[k], (unsigned long long)(t_ - t_mark)); \
    t_mark = t_;                                                                 \
  } while (0)
#else
#define EIG_MARK(k) \
  do {            \
  } while (0)
#endif

constexpr int kEigThreads = 256;
constexpr int kB = 32;        // maximum block width
constexpr int kLd = kB + 1;   // padded leading dimension of b x b matrices
constexpr int kEigSmallMax = 256;

// ----------------------------------------------------------------------------
// b-space helpers: one warp, matrices in shared memory with leading dim kLd.
// ----------------------------------------------------------------------------

// Cyclic Jacobi on one warp: jacobi_reg in jacobi.cuh.
template <typename T>
__device__ void jacobi_warp(T* H, T* Qm, int n, T rel_tol, int max_sweeps) {
  if (n <= 8) jacobi_reg<T, 8>(H, Qm, kLd, n, rel_tol, max_sweeps);
  else if (n <= 12) jacobi_reg<T, 12>(H, Qm, kLd, n, rel_tol, max_sweeps);
  else if (n <= 16) jacobi_reg<T, 16>(H, Qm, kLd, n, rel_tol, max_sweeps);
  else if (n <= 20) jacobi_reg<T, 20>(H, Qm, kLd, n, rel_tol, max_sweeps);
  else if (n <= 24) jacobi_reg<T, 24>(H, Qm, kLd, n, rel_tol, max_sweeps);
  else jacobi_reg<T, 32>(H, Qm, kLd, n, rel_tol, max_sweeps);
}

// perm[0..n): indices of the diagonal of H in descending order (ties: lower index first).
template <typename T>
__device__ void sort_desc_warp(const T* H, int n, int* perm) {
  const int lane = threadIdx.x & 31;
  if (lane < n) {
    const T v = H[lane * kLd + lane];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T u = H[j * kLd + j];
      rank += (u > v) || (u == v && j < lane);
    }
    perm[rank] = lane;
  }
  __syncwarp();
}

// In place upper Cholesky G = R^T R of a Gram with unit (or zero) diagonal,
// rank-revealing: a column whose pivot falls below the arithmetic's floor
// depends numerically on the earlier ones; it is marked dead (dead[j] = 1,
// R row j = e_j^T) and its entries of the transform are zeroed.  All
// threads of the CTA, one entry each per step.  For the start blocks, which
// factor once per launch, these parallel steps measured 2.3x faster than the
// one-warp register form below (whose long unrolled code is fetched cold
// on its first use in a launch) and than one-warp loops over shared memory;
// the b-space step, which factors every iteration, keeps the register form.
// The lower triangle is left as it was.
template <typename T>
__device__ void chol_cta(T* G, int n, int* dead) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const T floor_piv = sizeof(T) == 8 ? T(1e-24) : T(1e-10);
#pragma unroll 1
  for (int j = 0; j < n; ++j) {
    const T piv = G[j * kLd + j];
    const bool ok = piv > floor_piv;
    const T djj = ok ? sqrt(piv) : T(1);
    const T inv = T(1) / djj;
    __syncthreads();
    if (tid < n && tid >= j) G[j * kLd + tid] = tid == j ? djj : (ok ? G[j * kLd + tid] * inv : T(0));
    if (tid == 0) dead[j] = ok ? 0 : 1;
    __syncthreads();
    const int m = n - 1 - j;   // trailing block rows/columns j+1..n-1
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e / m, c = j + 1 + (e - (e / m) * m);
      if (c >= i) G[i * kLd + c] -= G[j * kLd + i] * G[j * kLd + c];
    }
    __syncthreads();
  }
}

// Out = X D R^-1 with the columns of dead directions zeroed (X = I when
// null), R the upper factor of chol_cta; Ri (b x b, ld kLd) is scratch for
// R^-1, computed by rows from the bottom (one column per thread per step).
// Out must not alias X.  All threads of the CTA.
template <typename T>
__device__ void apply_rinv_cta(const T* X, const T* d, const T* R, const int* dead, int b, T* Ri, T* Out) {
  const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll 1
  for (int i = b - 1; i >= 0; --i) {
    if (tid < b && tid >= i) {
      T v = tid == i ? T(1) : T(0);
      for (int k = i + 1; k <= tid; ++k) v -= R[i * kLd + k] * Ri[k * kLd + tid];
      Ri[i * kLd + tid] = v / R[i * kLd + i];
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += nt) {
    const int a = e / b, c = e - (e / b) * b;
    T acc = T(0);
    if (!dead[c]) {
      if (X) {
        for (int k = 0; k <= c; ++k) acc += X[a * kLd + k] * d[k] * Ri[k * kLd + c];
      } else if (a <= c) {
        acc = d[a] * Ri[a * kLd + c];
      }
    }
    Out[a * kLd + c] = acc;
  }
}

// The same factorisation register resident (one warp), for the b-space step
// (called every iteration, so its unrolled code stays in the instruction
// cache after the first): lane i holds row i
// of the Gram in NB registers; column j takes the pivot from lane j by a
// shuffle, lane j scales its row into row j of R, and every later row i
// subtracts R[j][i] R[j][:] (R[j][i] is lane i's own entry of the
// symmetric Gram over the pivot).  Full rows are updated, so the Gram stays
// symmetric.  R (upper) is written back to G.
template <typename T, int NB>
__device__ __noinline__ void chol_reg(T* G, int n, int* dead) {
  const int lane = threadIdx.x & 31;
  const T floor_piv = sizeof(T) == 8 ? T(1e-24) : T(1e-10);
  T g[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) g[c] = (lane < n && c < n) ? G[lane * kLd + c] : T(0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < n) {
      const T piv = __shfl_sync(0xffffffffu, g[j], j);
      if (!(piv > floor_piv)) {
        // a numerically dependent column: row j of R is e_j^T
        if (lane == j) {
#pragma unroll
          for (int c = 0; c < NB; ++c) g[c] = c == j ? T(1) : T(0);
        }
        if (lane == 0) dead[j] = 1;
      } else {
        const T djj = sqrt(piv);
        const T inv = T(1) / djj;
        if (lane == j) {
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c > j) g[c] *= inv;
          g[j] = djj;
        }
        if (lane == 0) dead[j] = 0;
        const T rji = g[j] * inv;   // lane i > j: R[j][i]
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c > j) {
            const T rjc = __shfl_sync(0xffffffffu, g[c], j);
            if (lane > j) g[c] -= rji * rjc;
          }
        }
      }
    }
  }
  if (lane < n) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c < n) G[lane * kLd + c] = c >= lane ? g[c] : T(0);
  }
  __syncwarp();
}

template <typename T>
__device__ void chol_fast(T* G, int n, int* dead) {
  if (n <= 16) chol_reg<T, 16>(G, n, dead);
  else if (n <= 24) chol_reg<T, 24>(G, n, dead);
  else chol_reg<T, 32>(G, n, dead);
}

// Column scaling of a Gram: d_j = 1/sqrt(G_jj), or 0 for columns whose norm
// is negligible against the largest one.
template <typename T>
__device__ void col_scale_warp(const T* G, int n, T* d) {
  const int lane = threadIdx.x & 31;
  T g = lane < n ? G[lane * kLd + lane] : T(0);
  T gmax = g;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  const T rel = sizeof(T) == 8 ? T(1e-28) : T(1e-12);
  if (lane < n) d[lane] = (g > rel * gmax && g > T(0)) ? T(1) / sqrt(g) : T(0);
  __syncwarp();
}

// row[0..b) <- row D R^-1 for the upper factor R (shared memory, ld kLd)
// of a rank-revealing Cholesky (dead columns zeroed).  Unrolled over NB >= b
// columns so that the row stays in registers; solve_row picks NB.
template <typename T, int NB>
__device__ __forceinline__ void solve_row_nb(T (&row)[kB], const T* d, const T* R, const int* dead, int b) {
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < b) row[j] *= d[j];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < b) {
      T v = row[j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= row[k] * R[k * kLd + j];
      row[j] = dead[j] ? T(0) : v / R[j * kLd + j];
    }
  }
}

template <typename T>
__device__ __forceinline__ void solve_row(T (&row)[kB], const T* d, const T* R, const int* dead, int b) {
  if (b <= 16) solve_row_nb<T, 16>(row, d, R, dead, b);
  else if (b <= 24) solve_row_nb<T, 24>(row, d, R, dead, b);
  else solve_row_nb<T, 32>(row, d, R, dead, b);
}

// dst[i * ldd + j] = src[i * lds + j] for i < rows, j < cols: a CTA-wide
// copy with 8 independent loads in flight per thread
template <typename T>
__device__ void stage_rows(T* dst, int ldd, const T* __restrict__ src, int lds, int rows, int cols) {
  // warps take 4 rows at a time, lanes the columns: coalesced row segments,
  // 8 independent loads per lane in flight, no index division
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 4 * warp; i0 < rows; i0 += 4 * nw) {
    for (int j0 = 0; j0 < cols; j0 += 64) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + (u & 3), j = j0 + 32 * (u >> 2) + lane;
        v[u] = (i < rows && j < cols) ? src[(size_t)i * lds + j] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + (u & 3), j = j0 + 32 * (u >> 2) + lane;
        if (i < rows && j < cols) dst[i * ldd + j] = v[u];
      }
    }
  }
}

// Shared state of one b-space step.
template <typename T>
struct BSpace {
  T H[kB * kLd];    // V^T W, then diagonalised
  T P[kB * kLd];    // W^T W
  T F[kB * kLd];    // E^T E
  T Q[kB * kLd];    // eigenvectors of H (unsorted columns)
  T S[kB * kLd];    // next-basis transform (or sorted Q)
  T G[kB * kLd];    // scratch
  int perm[kB];
  T theta[kB];
  T d[kB];          // column scaling
  int dead[kB];     // columns dropped by the rank-revealing Cholesky
  int conv;
};

// All threads of the CTA (blockDim.x threads, b-space matrices in shared
// memory): warp 0 runs Jacobi on H and sorts; the residual test (needs F
// unless `check` is false) and, when not converged, S = Q_sorted D R^-1
// with R = chol(D Q^T P Q D).  The b x b products are spread over the CTA.
// When converged (or `final_rotation`), S = Q_sorted (Ritz vectors U = V S).
// *prev (shared) carries the previous residual between iterations.
template <typename T>
__device__ void bspace_step(BSpace<T>& s, int b, int r, double tol, double* prev, bool check, bool final_rotation) {
  const int tid = threadIdx.x, lane = tid & 31;
  // The Ritz rotation of an FP32 iteration that neither tests convergence
  // nor ends the solve only orients the next basis (span(C V) does not
  // depend on it, and the scaled Cholesky QR needs W S only roughly
  // orthogonal): three Jacobi sweeps there, full accuracy on testing and
  // final iterations.
  //
  // FP64: FP64 runs at 1/64 of FP32 on this part and a Jacobi sweep of the
  // b x b problem is ~6 b^3 dependent-round FP64 operations on one warp, so
  // every iteration rotates by an FP32 Jacobi of a scaled, rounded copy of H
  // (the rotation is exact in FP64 as a matrix; the next basis is
  // re-orthonormalised in FP64 and its span does not depend on the
  // rotation), and only the rotation that is kept (converged or last
  // iteration) is recomputed by the FP64 Jacobi below.
  if (sizeof(T) == 8) {
    float* Hf = reinterpret_cast<float*>(s.G);   // G is scratch until the residual test
    float* Qf = Hf + kB * kLd;
    if (tid < 32) {
      T hm = lane < b ? fabs(s.H[lane * kLd + lane]) : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hm = fmax(hm, __shfl_xor_sync(0xffffffffu, hm, o));
      if (lane == 0) s.d[0] = hm > T(0) ? T(1) / hm : T(1);   // d is free until the next basis
    }
    __syncthreads();
    const T sc = s.d[0];
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int a = e / b, j = e - a * b;
      Hf[a * kLd + j] = (float)(s.H[a * kLd + j] * sc);
    }
    __syncthreads();
    if (tid < 32) {
      jacobi_warp<float>(Hf, Qf, b, 1e-6f, 8);
      sort_desc_warp<float>(Hf, b, s.perm);
      if (lane < b) s.theta[lane] = (T)Hf[s.perm[lane] * kLd + s.perm[lane]] / sc;
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int a = e / b, j = e - a * b;
      s.S[a * kLd + j] = (T)Qf[a * kLd + s.perm[j]];
    }
    __syncthreads();
  } else {
    const int sweeps = check || final_rotation ? 8 : 3;
    if (tid < 32) {
      jacobi_warp<T>(s.H, s.Q, b, T(1e-6), sweeps);
      sort_desc_warp<T>(s.H, b, s.perm);
      if (lane < b) s.theta[lane] = s.H[s.perm[lane] * kLd + s.perm[lane]];
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int a = e / b, j = e - a * b;
      s.S[a * kLd + j] = s.Q[a * kLd + s.perm[j]];
    }
    __syncthreads();
  }
  if (check) {
    // res_j^2 = q_j^T F q_j for the leading r Ritz pairs
    for (int e = tid; e < b * r; e += blockDim.x) {
      const int a = e / r, j = e - a * r;
      T fq = T(0);
      for (int c = 0; c < b; ++c) fq += s.F[a * kLd + c] * s.S[c * kLd + j];
      s.G[a * kLd + j] = fq;
    }
    __syncthreads();
    if (tid < 32) {
      double res = 0.0;
      if (lane < r)
        for (int a = 0; a < b; ++a) res += (double)s.S[a * kLd + lane] * (double)s.G[a * kLd + lane];
      res = res > 0.0 ? sqrt(res) : 0.0;
      double worst = res;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
      const double th0 = fabs((double)s.theta[0]);
      const double rel = th0 > 0.0 ? worst / th0 : 0.0;
      const bool floor_hit = rel < 10.0 * tol && rel > 0.5 * (*prev);
      const bool conv = (th0 == 0.0) || rel <= tol || floor_hit;
      __syncwarp();
      if (lane == 0) {
        s.conv = conv ? 1 : 0;
        *prev = rel;
      }
    }
  } else if (tid == 0) {
    s.conv = 0;
  }
  __syncthreads();
  if (sizeof(T) == 8 && (s.conv || final_rotation)) {
    // the kept rotation in full FP64 precision (H is still unrotated)
    if (tid < 32) {
      jacobi_warp<T>(s.H, s.Q, b, T(1e-14), 12);
      sort_desc_warp<T>(s.H, b, s.perm);
      if (lane < b) s.theta[lane] = s.H[s.perm[lane] * kLd + s.perm[lane]];
    }
    __syncthreads();
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int a = e / b, j = e - a * b;
      s.S[a * kLd + j] = s.Q[a * kLd + s.perm[j]];
    }
    __syncthreads();
  }
  if (s.conv || final_rotation) return;
  // G = P S, then F = S^T G (F is free once the residual is taken)
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int a = e / b, j = e - a * b;
    T acc = T(0);
    for (int c = 0; c < b; ++c) acc += s.P[a * kLd + c] * s.S[c * kLd + j];
    s.G[a * kLd + j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int a = e / b, j = e - a * b;
    T acc = T(0);
    for (int c = 0; c < b; ++c) acc += s.S[c * kLd + a] * s.G[c * kLd + j];
    s.F[a * kLd + j] = acc;
  }
  __syncthreads();
  if (tid < 32) {
    col_scale_warp<T>(s.F, b, s.d);
    if (lane < b)
      for (int j = 0; j < b; ++j) s.F[lane * kLd + j] *= s.d[lane] * s.d[j];
    __syncwarp();
    chol_fast<T>(s.F, b, s.dead);
  }
  __syncthreads();
  // S <- S D R^-1: forward substitution against upper R, one row per thread
  if (tid < b) {
    T row[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) row[j] = j < b ? s.S[tid * kLd + j] : T(0);
    solve_row<T>(row, s.d, s.F, s.dead, b);
#pragma unroll
    for (int j = 0; j < kB; ++j)
      if (j < b) s.S[tid * kLd + j] = row[j];
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// M-length passes (all threads of a CTA, rows [i0, i1)).
// ----------------------------------------------------------------------------

// W[i, :ncols] = C[i, :] V[:, :ncols] for rows i in [i0, i1); warp per RPW
// rows, lane j per column j of V (coalesced rows of V, broadcast C).  The
// k loop keeps 8 independent partial sums per row so that 8 loads of C and
// V are in flight per lane (the operands may live in global memory).
template <typename T, int RPW>
__device__ void cv_rows(const T* C, int M, const T* V, int b, T* W, int ncols, int i0, int i1, int warp, int nwarps) {
  constexpr int KU = 8;
  const int lane = threadIdx.x & 31;
  for (int r0 = i0 + RPW * warp; r0 < i1; r0 += RPW * nwarps) {
    const int nr = min(RPW, i1 - r0);
    const T* crow[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) crow[q] = C + (size_t)(r0 + (q < nr ? q : 0)) * M;
    T acc[RPW][KU];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int u = 0; u < KU; ++u) acc[q][u] = T(0);
    if (lane < ncols) {
      const T* vc = V + lane;
      int k = 0;
      for (; k + KU <= M; k += KU) {
        T v[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) v[u] = vc[(size_t)(k + u) * b];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
          for (int u = 0; u < KU; ++u) acc[q][u] += crow[q][k + u] * v[u];
      }
      for (; k < M; ++k) {
        const T v = vc[(size_t)k * b];
#pragma unroll
        for (int q = 0; q < RPW; ++q) acc[q][0] += crow[q][k] * v;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        T t = T(0);
#pragma unroll
        for (int u = 0; u < KU; ++u) t += acc[q][u];
        if (q < nr) W[(size_t)(r0 + q) * b + lane] = t;
      }
    }
  }
}

// Out[i, j] = A[i, :K] B[:K, j]  (or Sub[i, j] - A[i, :K] B[:K, j] when Sub
// is given) for i < M, j < nc; all row-major with the given leading
// dimensions.  Each thread owns a 4 x 4 register tile of Out (16 FMAs per
// 8 loads); all threads of the CTA share the tiles.
template <typename T>
__device__ void tile_gemm(const T* A, int lda, const T* B, int ldb, int M, int K, int nc, T* Out, int ldo,
                          const T* Sub) {
  const int cg = (nc + 3) >> 2, rg = (M + 3) >> 2;
  for (int t = threadIdx.x; t < cg * rg; t += blockDim.x) {
    const int tr = t / cg, tc = t - tr * cg;
    const int i0 = tr << 2, j0 = tc << 2;
    const T* a[4];
    int jj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = A + (size_t)min(i0 + q, M - 1) * lda;
      jj[q] = min(j0 + q, nc - 1);
    }
    T acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q][u] = T(0);
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      T av[4], bv[4];
      const T* brow = B + (size_t)k * ldb;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        av[q] = a[q][k];
        bv[q] = brow[jj[q]];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[q][u] += av[q] * bv[u];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q;
      if (i >= M) break;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u;
        if (j < nc) Out[(size_t)i * ldo + j] = Sub ? Sub[(size_t)i * ldo + j] - acc[q][u] : acc[q][u];
      }
    }
  }
}

// Gram-type sums over rows [i0, i1): H = X^T Y, P = Y^T Y (when P != null);
// X, Y row-major with leading dimension ld.  Thread t owns entries t,
// t + blockDim.x, .. of the b x b results.
template <typename T>
__device__ void grams_rows(const T* X, const T* Y, int ld, int b, int i0, int i1, T* Hout, T* Pout, int ldo) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e - (e / b) * b;
    T h = T(0), g = T(0);
    for (int i = i0; i < i1; ++i) {
      const T yq = Y[(size_t)i * ld + q];
      h += X[(size_t)i * ld + p] * yq;
      if (Pout) g += Y[(size_t)i * ld + p] * yq;
    }
    Hout[p * ldo + q] = h;
    if (Pout) Pout[p * ldo + q] = g;
  }
}

// Out[i, :ncols] = X[i, :] S[:, :ncols] for rows [i0, i1) (S in shared memory, ld kLd).
template <typename T>
__device__ void apply_rows(const T* X, const T* S, int b, int ncols, T* Out, int ldout, int i0, int i1) {
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    T xr[kB];
#pragma unroll
    for (int k = 0; k < kB; ++k) xr[k] = k < b ? X[(size_t)i * b + k] : T(0);
    for (int j = 0; j < ncols; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < kB; ++k)
        if (k < b) acc += xr[k] * S[k * kLd + j];
      Out[(size_t)i * ldout + j] = acc;
    }
  }
}

// Final Rayleigh-Ritz of the leading r Ritz vectors in FP64: rr_refine in jacobi.cuh.

// The eigenvectors are U_r X: U_r (the leading r Ritz vectors, M x r in the
// path's precision) is written to Ur (row-major, ld r) and the FP64 rotation
// X (r x r, columns in descending order of lambda) to Xr, row-major; theta =
// the sorted lambda.  The product U_r X is formed by the factor kernel
// (launch_lsv_finish), which spreads its FP64 work over many CTAs.
template <typename T>
__device__ void rr_write(const T* U, int ld, int M, int r, const FinalRR& f, T* Ur, double* Xr, double* theta) {
  for (int e = threadIdx.x; e < M * r; e += blockDim.x) {
    const int i = e / r, j = e - (e / r) * r;
    Ur[e] = U[(size_t)i * ld + j];
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e / r, j = e - (e / r) * r;
    Xr[e] = f.X[k * kRl + f.perm[j]];
  }
  if (threadIdx.x < r) theta[threadIdx.x] = f.lam[f.perm[threadIdx.x]];
  __syncthreads();
}

// General form: H = U_r^T CU_r and G = U_r^T U_r by FP64 sums over the M
// rows (U, CU row-major with leading dimension ld), then refinement.
template <typename T>
__device__ void final_rr(const T* U, const T* CU, int M, int ld, int r, T* Ur, double* Xr, double* theta,
                         FinalRR& f) {
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - (e / r) * r;
    double h = 0.0, g = 0.0;
    for (int i = 0; i < M; ++i) {
      const double up = (double)U[(size_t)i * ld + p];
      h += up * (double)CU[(size_t)i * ld + q];
      g += up * (double)U[(size_t)i * ld + q];
    }
    f.T1[p * kRl + q] = h;
    f.G[p * kRl + q] = g;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int p = e / r, q = e - (e / r) * r;
    f.H[p * kRl + q] = 0.5 * (f.T1[p * kRl + q] + f.T1[q * kRl + p]);
  }
  __syncthreads();
  rr_refine(f, r, sizeof(T) == 4 ? 1e-5 : 1e-7);
  rr_write<T>(U, ld, M, r, f, Ur, Xr, theta);
}

// U_r of the fused path lives after X (r x r doubles) in the output area.
template <typename T>
__host__ __device__ inline T* eig_out_u(double* out, int r) {
  return reinterpret_cast<T*>(out + kMaxRank * kMaxRank);
}

template <typename T>
struct EigArgs {
  const T* C;          // M x M symmetric (row-major)
  int M, r, b;
  T* V;                // M x b start block (global); overwritten (split path)
  T* W;                // M x b scratch (global)
  T* U;                // M x b scratch (global)
  T* part;             // split path: partial b x b Grams, >= 3 * nblk * b * b
  double* Vout;        // output area: X (r x r FP64), then U_r (M x r, T)
  double* theta;       // r FP64 eigenvalues, descending
  int maxit;
  double tol;
  unsigned long long* stats;  // calls, iterations, unconverged
  T* basis_out;        // M x b final Ritz block (warm start of the next solve), or null
};

// ----------------------------------------------------------------------------
// Fused path: one CTA, M <= kEigSmallMax.
// ----------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kEigThreads) eig_fused_kernel(EigArgs<T> a, int smem_mode) {
#ifdef MACH_EIG_PHASES
  long long t_mark = clock64();
#endif
  extern __shared__ __align__(16) unsigned char eig_smem[];
  __shared__ BSpace<T> bs;
  __shared__ FinalRR frr;
  __shared__ double prev;
  const int M = a.M, b = a.b, r = a.r;
  // shared-memory copies use odd leading dimensions (conflict-free tiles)
  const int ld = smem_mode >= 1 ? (b | 1) : b;
  T* V = a.V;
  T* W = a.W;
  T* U = a.U;
  const T* C = a.C;
  int ldc = M;
  if (smem_mode >= 1) {
    V = reinterpret_cast<T*>(eig_smem);
    W = V + (size_t)M * ld;
    U = W + (size_t)M * ld;
    stage_rows<T>(V, ld, a.V, b, M, b);
  }
  if (smem_mode == 2) {
    T* Cs = U + (size_t)M * ld;
    ldc = M | 1;
    stage_rows<T>(Cs, ldc, a.C, M, M, M);
    C = Cs;
  }
  if (threadIdx.x == 0) prev = 1e300;
  __syncthreads();
  EIG_MARK(0);   // staging
  // orthonormalise the start block: P = V^T V, S from its scaled Cholesky
  grams_rows<T>(V, V, ld, b, 0, M, bs.P, nullptr, kLd);
  __syncthreads();
  EIG_MARK(8);   // start Gram
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    col_scale_warp<T>(bs.P, b, bs.d);
    if (lane < b)
      for (int j = 0; j < b; ++j) bs.G[lane * kLd + j] = bs.P[lane * kLd + j] * bs.d[lane] * bs.d[j];
    // A warm start block ([Y^T A_prev, previous Ritz directions]) can be
    // nearly orthonormal once its columns are scaled: with E = D P D - I and
    // ||E||_F small, S = D (I + E)^-1/2 = D (I - E/2 + 3/8 E^2) (the
    // omitted terms are below 5/16 ||E||_F^3: 3e-7 at the FP32 threshold
    // 1e-2, 3e-16 at the FP64 threshold 1e-5) takes one parallel product
    // instead of the step-by-step Cholesky below.
    T ef = T(0);
    for (int e = lane; e < b * b; e += 32) {
      const int i = e / b, j = e - (e / b) * b;
      const T x = bs.G[i * kLd + j] - (i == j ? T(1) : T(0));
      ef += x * x;
    }
    ef = warp_sum(ef);
    if (lane == 0) bs.conv = ef <= (sizeof(T) == 8 ? T(1e-10) : T(1e-4)) ? 1 : 0;   // conv is free until the first step
  }
  __syncthreads();
  if (bs.conv) {
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e - (e / b) * b;
      T e2 = T(0);
      for (int k = 0; k < b; ++k)
        e2 += (bs.G[i * kLd + k] - (i == k ? T(1) : T(0))) * (bs.G[k * kLd + j] - (k == j ? T(1) : T(0)));
      const T eij = bs.G[i * kLd + j] - (i == j ? T(1) : T(0));
      bs.S[i * kLd + j] = bs.d[i] * ((i == j ? T(1) : T(0)) - T(0.5) * eij + T(0.375) * e2);
    }
    __syncthreads();
  } else {
    chol_cta<T>(bs.G, b, bs.dead);
    apply_rinv_cta<T>(nullptr, bs.d, bs.G, bs.dead, b, bs.Q, bs.S);   // S = D R^-1
    __syncthreads();
  }
  EIG_MARK(9);   // start orthonormalising transform
  tile_gemm<T>(V, ld, bs.S, kLd, M, b, b, W, ld, nullptr);
  __syncthreads();
  {
    T* t = V;
    V = W;
    W = t;
  }

  int it = 0;
  bool conv = false;
  EIG_MARK(1);   // start orthonormalisation
  for (; it < a.maxit; ++it) {
    tile_gemm<T>(C, ldc, V, ld, M, M, b, W, ld, nullptr);        // W = C V
    __syncthreads();
    EIG_MARK(2);   // C V
    grams_rows<T>(V, W, ld, b, 0, M, bs.H, bs.P, kLd);           // H = V^T W, P = W^T W
    __syncthreads();
    tile_gemm<T>(V, ld, bs.H, kLd, M, b, b, U, ld, W);           // E = W - V H (U is free)
    __syncthreads();
    grams_rows<T>(U, U, ld, b, 0, M, bs.F, nullptr, kLd);        // F = E^T E
    __syncthreads();
    EIG_MARK(3);   // b x b sums and the residual block
    bspace_step<T>(bs, b, r, a.tol, &prev, true, it + 1 == a.maxit);
    EIG_MARK(4);   // b-space step
    if (bs.conv || it + 1 == a.maxit) {
      conv = bs.conv != 0;
      tile_gemm<T>(V, ld, bs.S, kLd, M, b, b, U, ld, nullptr);   // Ritz vectors
      __syncthreads();
      break;
    }
    tile_gemm<T>(W, ld, bs.S, kLd, M, b, b, U, ld, nullptr);     // next basis (into U, then swap)
    __syncthreads();
    T* t = V;
    V = U;
    U = t;
  }
  if (a.maxit <= 0) {
    for (int o = threadIdx.x; o < M * b; o += blockDim.x) {
      const int i = o / b, j = o - (o / b) * b;
      U[i * ld + j] = V[i * ld + j];
    }
    __syncthreads();
  }
  if (a.basis_out)
    for (int o = threadIdx.x; o < M * b; o += blockDim.x) {
      const int i = o / b, j = o - (o / b) * b;
      a.basis_out[o] = U[i * ld + j];
    }
  if (a.maxit > 0) {
    // projected matrix and Gram of U_r = V S_r from the last b-space step:
    // H_r = (S^T H S)[:r, :r] (the Jacobi-rotated H), G_r = S_r^T S_r
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int p = e / r, q = e - (e / r) * r;
      const int pp = bs.perm[p], pq = bs.perm[q];
      frr.H[p * kRl + q] = 0.5 * ((double)bs.H[pp * kLd + pq] + (double)bs.H[pq * kLd + pp]);
      double g = 0.0;
      for (int k = 0; k < b; ++k) g += (double)bs.S[k * kLd + p] * (double)bs.S[k * kLd + q];
      frr.G[p * kRl + q] = g;
    }
    __syncthreads();
    EIG_MARK(5);   // Ritz vectors and basis out
    rr_refine(frr, r, sizeof(T) == 4 ? 1e-5 : 1e-7);
    EIG_MARK(6);   // FP64 refinement
    rr_write<T>(U, ld, M, r, frr, eig_out_u<T>(a.Vout, r), a.Vout, a.theta);
    EIG_MARK(7);   // output
  } else {
    tile_gemm<T>(C, ldc, U, ld, M, M, r, W, ld, nullptr);        // C U_r
    __syncthreads();
    final_rr<T>(U, W, M, ld, r, eig_out_u<T>(a.Vout, r), a.Vout, a.theta, frr);
  }
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[0], 1ull);
    atomicAdd(&a.stats[1], (unsigned long long)min(it + 1, max(a.maxit, 0)));
    if (!conv) atomicAdd(&a.stats[2], 1ull);
  }
}

// ----------------------------------------------------------------------------
// Split path (large M): fixed iteration count, multi-CTA passes.
// ----------------------------------------------------------------------------
// Control words of the split path's early exit (device): [0] converged
// (the remaining iterations' launches return at once), [1] the iteration
// whose basis holds the Ritz vectors, [2] the previous residual (double bits).
__device__ __forceinline__ bool split_done(const unsigned long long* ctl) { return ctl && ctl[0] != 0ull; }

constexpr int kRowsPerCta = 32;
constexpr int kSplitCheck = 4;   // split path: Ritz residuals tested every 4 iterations
// W = C V (first nc columns): 64-row x 32-column output tiles with the k
// range split over gridDim.y (kCvSplit slices).  Tiles of C (stored
// transposed, so that a thread's 8 rows at one k are contiguous) and of V
// are staged in shared memory; thread (ty, tx) owns rows 8 ty .. 8 ty + 7 of
// column tx.  Slice ks writes its partial tile to P[ks] (M x kB); the
// slices are summed in ks order by cv_reduce_kernel (deterministic).
constexpr int kCvRows = 64, kCvK = 32, kCvSplit = 8;

template <typename T>
__global__ void __launch_bounds__(256) cv_tiled_kernel(const T* __restrict__ C, int M, const T* __restrict__ V, int b,
                                                       int nc, T* __restrict__ P, const unsigned long long* ctl) {
  if (split_done(ctl)) return;
  __shared__ __align__(16) T Ct[kCvK][kCvRows + 16 / sizeof(T)];
  __shared__ T Vs[kCvK][kB + 1];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int r0 = blockIdx.x * kCvRows;
  const int kper = (M + (int)gridDim.y - 1) / (int)gridDim.y;
  const int k0 = blockIdx.y * kper, k1 = min(M, k0 + kper);
  T acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = T(0);
  for (int kc = k0; kc < k1; kc += kCvK) {
#pragma unroll
    for (int u = 0; u < kCvRows * kCvK / 256; ++u) {
      const int e = tid + 256 * u;
      const int rr = e / kCvK, kk = e - (e / kCvK) * kCvK;
      const int gi = r0 + rr, gk = kc + kk;
      Ct[kk][rr] = (gi < M && gk < k1) ? C[(size_t)gi * M + gk] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kCvK * 32 / 256; ++u) {
      const int e = tid + 256 * u;
      const int kk = e >> 5, j = e & 31;
      const int gk = kc + kk;
      Vs[kk][j] = (gk < k1 && j < nc) ? V[(size_t)gk * b + j] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kCvK; ++kk) {
      const T v = Vs[kk][tx];
      const T* c = &Ct[kk][ty * 8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += c[q] * v;
    }
    __syncthreads();
  }
  T* Pk = P + (size_t)blockIdx.y * M * kB;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = r0 + ty * 8 + q;
    if (i < M && tx < nc) Pk[(size_t)i * kB + tx] = acc[q];
  }
}

template <typename T>
__global__ void cv_reduce_kernel(const T* __restrict__ P, int nsplit, int M, int nc, T* __restrict__ W, int ldw,
                                 const unsigned long long* ctl) {
  if (split_done(ctl)) return;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= M * nc) return;
  const int i = o / nc, j = o - (o / nc) * nc;
  T s = T(0);
  for (int k = 0; k < nsplit; ++k) s += P[(size_t)k * M * kB + (size_t)i * kB + j];
  W[(size_t)i * ldw + j] = s;
}

// partial Grams of a row block: part[blk][0] = V^T W, part[blk][1] = W^T W;
// with part64, also V^T V, V^T W and W^T W summed in FP64 (exact products of
// the stored values), from which the residual of the subspace is formed
// without cancellation in the path's precision
template <typename T>
__global__ void __launch_bounds__(256) split_grams_kernel(const T* V, const T* W, int M, int b, T* part,
                                                          double* part64, const unsigned long long* ctl) {
  if (split_done(ctl)) return;
  const int i0 = blockIdx.x * kRowsPerCta, i1 = min(M, i0 + kRowsPerCta);
  T* h = part + (size_t)blockIdx.x * 2 * b * b;
  grams_rows<T>(V, W, b, b, i0, i1, h, h + b * b, b);
  if (part64) {
    double* g = part64 + (size_t)blockIdx.x * 3 * b * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int p = e / b, q = e - (e / b) * b;
      double vv = 0.0, vw = 0.0, ww = 0.0;
      for (int i = i0; i < i1; ++i) {
        const double vp = (double)V[(size_t)i * b + p], vq = (double)V[(size_t)i * b + q];
        const double wp = (double)W[(size_t)i * b + p], wq = (double)W[(size_t)i * b + q];
        vv += vp * vq;
        vw += vp * wq;
        ww += wp * wq;
      }
      g[e] = vv;
      g[b * b + e] = vw;
      g[2 * b * b + e] = ww;
    }
  }
}

// partial start Gram V^T V of a row block
template <typename T>
__global__ void __launch_bounds__(256) split_gram_vv_kernel(const T* V, int M, int b, T* part) {
  const int i0 = blockIdx.x * kRowsPerCta;
  grams_rows<T>(V, V, b, b, i0, min(M, i0 + kRowsPerCta), part + (size_t)blockIdx.x * 2 * b * b, nullptr, b);
}

// one CTA: reduce partials (fixed order), b-space step; S to global (b x b)
template <typename T>
__global__ void __launch_bounds__(256) split_bspace_kernel(const T* part, int nblk, int b, int r, int mode,
                                                           T* S_out, double* rr_out, const double* part64,
                                                           unsigned long long* ctl, int it, double tol) {
  // mode 0: start block orthonormalisation (part holds V^T V)
  // mode 1: iteration (next basis, or the Ritz rotation once converged);
  // mode 2: final (Ritz rotation)
  if (mode != 0 && split_done(ctl)) return;
#ifdef MACH_EIG_PHASES
  long long t_mark = clock64();
#endif
  __shared__ BSpace<T> bs;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    T h = T(0), g = T(0);
    for (int k = 0; k < nblk; ++k) {
      h += part[(size_t)k * 2 * b * b + e];
      if (mode != 0) g += part[(size_t)k * 2 * b * b + b * b + e];
    }
    const int p = e / b, q = e - (e / b) * b;
    if (mode == 0) bs.P[p * kLd + q] = h;
    else {
      bs.H[p * kLd + q] = h;
      bs.P[p * kLd + q] = g;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (mode == 0) {
      col_scale_warp<T>(bs.P, b, bs.d);
      if (lane < b)
        for (int j = 0; j < b; ++j) bs.G[lane * kLd + j] = bs.P[lane * kLd + j] * bs.d[lane] * bs.d[j];
      __syncwarp();
    } else {
      // symmetrise H (rounding) before Jacobi
      if (lane < b)
        for (int j = lane + 1; j < b; ++j) {
          const T avg = T(0.5) * (bs.H[lane * kLd + j] + bs.H[j * kLd + lane]);
          bs.H[lane * kLd + j] = avg;
          bs.H[j * kLd + lane] = avg;
        }
      __syncwarp();
    }
  }
  __syncthreads();
  if (mode == 0) {
    chol_cta<T>(bs.G, b, bs.dead);
    apply_rinv_cta<T>(nullptr, bs.d, bs.G, bs.dead, b, bs.Q, bs.S);   // S = D R^-1
    __syncthreads();
  }
  EIG_MARK(10);   // split: partial sums (and the start Cholesky)
  bool final_rot = mode == 2;
  if (mode != 0) {
    __shared__ double prev;
    __shared__ double G64[kB * kLd], L64[kB * kLd], H64[kB * kLd];
    const bool check = part64 != nullptr;
    if (check) {
      // F = W^T (I - P_V) W = P - H^T G^-1 H from the FP64 sums, G = V^T V:
      // the part of C V outside span(V), exact to FP64 rounding even when V
      // is orthonormal only to the path's precision
      for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        double g = 0.0, h = 0.0, pp = 0.0;
        for (int k = 0; k < nblk; ++k) {
          const double* q = part64 + (size_t)k * 3 * b * b;
          g += q[e];
          h += q[b * b + e];
          pp += q[2 * b * b + e];
        }
        const int p = e / b, q2 = e - (e / b) * b;
        G64[p * kLd + q2] = g;
        H64[p * kLd + q2] = h;
        L64[p * kLd + q2] = pp;   // P until F is formed
      }
      __syncthreads();
      // G is the identity up to the path's rounding (V orthonormal to it):
      // G^-1 = I - E + E^2 with E = G - I (the first omitted term, E^3, is
      // below 1e-12 for max |E_ij| <= 1e-4), and with X = E H
      //   F = P - H^T H + H^T X - X^T X,
      // three parallel FP64 passes; otherwise the Cholesky G = L L^T.
      __shared__ double emax_w[8];
      {
        double em = 0.0;
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
          const int p = e / b, q2 = e - (e / b) * b;
          em = fmax(em, fabs(G64[p * kLd + q2] - (p == q2 ? 1.0 : 0.0)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
        if ((threadIdx.x & 31) == 0) emax_w[threadIdx.x >> 5] = em;
      }
      __syncthreads();
      double emax = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) emax = fmax(emax, emax_w[w]);
      if (emax <= 1e-4) {
        __shared__ double X64[kB * kLd];
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
          const int p = e / b, q2 = e - (e / b) * b;
          double x0 = 0.0, x1 = 0.0;
          int k = 0;
          for (; k + 1 < b; k += 2) {
            x0 += (G64[p * kLd + k] - (p == k ? 1.0 : 0.0)) * H64[k * kLd + q2];
            x1 += (G64[p * kLd + k + 1] - (p == k + 1 ? 1.0 : 0.0)) * H64[(k + 1) * kLd + q2];
          }
          if (k < b) x0 += (G64[p * kLd + k] - (p == k ? 1.0 : 0.0)) * H64[k * kLd + q2];
          X64[p * kLd + q2] = x0 + x1;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
          const int p = e / b, q2 = e - (e / b) * b;
          double f0 = L64[p * kLd + q2], f1 = 0.0;
          for (int k = 0; k < b; ++k) {
            f0 -= H64[k * kLd + p] * (H64[k * kLd + q2] - X64[k * kLd + q2]);
            f1 -= X64[k * kLd + p] * X64[k * kLd + q2];
          }
          bs.F[p * kLd + q2] = (T)(f0 + f1);
        }
      } else {
        if (threadIdx.x < 32) {
          // lower Cholesky G = L L^T in place (one warp)
          const int lane = threadIdx.x;
          for (int j = 0; j < b; ++j) {
            if (lane == 0) {
              double d = G64[j * kLd + j];
              for (int k = 0; k < j; ++k) d -= G64[j * kLd + k] * G64[j * kLd + k];
              G64[j * kLd + j] = d > 0.0 ? sqrt(d) : 1e-300;
            }
            __syncwarp();
            for (int i = j + 1 + lane; i < b; i += 32) {
              double v = G64[i * kLd + j];
              for (int k = 0; k < j; ++k) v -= G64[i * kLd + k] * G64[j * kLd + k];
              G64[i * kLd + j] = v / G64[j * kLd + j];
            }
            __syncwarp();
          }
          // Z = L^-1 H, column per lane (forward substitution), into H64
          for (int c = lane; c < b; c += 32) {
            for (int i = 0; i < b; ++i) {
              double v = H64[i * kLd + c];
              for (int k = 0; k < i; ++k) v -= G64[i * kLd + k] * H64[k * kLd + c];
              H64[i * kLd + c] = v / G64[i * kLd + i];
            }
          }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
          const int p = e / b, q2 = e - (e / b) * b;
          double f = L64[p * kLd + q2];
          for (int k = 0; k < b; ++k) f -= H64[k * kLd + p] * H64[k * kLd + q2];
          bs.F[p * kLd + q2] = (T)f;
        }
      }
      if (threadIdx.x == 0) prev = __longlong_as_double((long long)ctl[2]);
    } else if (threadIdx.x == 0) {
      prev = 1e300;
    }
    __syncthreads();
    EIG_MARK(11);   // split: FP64 residual block
    bspace_step<T>(bs, b, r, check ? tol : 0.0, &prev, check, mode == 2);
    EIG_MARK(12);   // split: b-space step
    if (check && bs.conv) final_rot = true;
    if (check && threadIdx.x == 0) ctl[2] = (unsigned long long)__double_as_longlong(prev);
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e - (e / b) * b;
    S_out[p * kB + q] = bs.S[p * kLd + q];
  }
  if (final_rot && ctl && threadIdx.x == 0) {
    ctl[1] = (unsigned long long)it;
    ctl[0] = 1ull;
  }
  if (final_rot) {
    // final FP64 Rayleigh-Ritz of U_r = V S_r from the b-space quantities:
    // H_r = (S^T H S)[:r, :r] (the Jacobi-rotated H), G_r = S_r^T S_r
    __shared__ FinalRR frr;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int p = e / r, q = e - (e / r) * r;
      const int pp = bs.perm[p], pq = bs.perm[q];
      frr.H[p * kRl + q] = 0.5 * ((double)bs.H[pp * kLd + pq] + (double)bs.H[pq * kLd + pp]);
      double g = 0.0;
      for (int k = 0; k < b; ++k) g += (double)bs.S[k * kLd + p] * (double)bs.S[k * kLd + q];
      frr.G[p * kRl + q] = g;
    }
    __syncthreads();
    rr_refine(frr, r, sizeof(T) == 4 ? 1e-5 : 1e-7);
    EIG_MARK(13);   // split: final FP64 Rayleigh-Ritz
    // rr_out: X (r x r, columns in descending order of lambda), then lambda
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int k = e / r, j = e - (e / r) * r;
      rr_out[e] = frr.X[k * kRl + frr.perm[j]];
    }
    if (threadIdx.x < r) rr_out[r * r + threadIdx.x] = frr.lam[frr.perm[threadIdx.x]];
  }
}

// theta from rr_out (its X stays there for the factor kernel); counts the solve.
__global__ void split_finish_kernel(int r, const double* __restrict__ rr_out, double* __restrict__ theta,
                                    unsigned long long* stats, int iters, const unsigned long long* ctl) {
  if (ctl) iters = (int)ctl[1] + 1;
  if (threadIdx.x < r) theta[threadIdx.x] = rr_out[r * r + threadIdx.x];
  if (threadIdx.x == 0 && stats) {
    atomicAdd(&stats[0], 1ull);
    atomicAdd(&stats[1], (unsigned long long)iters);
  }
}

__global__ void split_ctl_init(unsigned long long* ctl) {
  if (threadIdx.x < 2) ctl[threadIdx.x] = 0ull;
  if (threadIdx.x == 2) ctl[2] = (unsigned long long)__double_as_longlong(1e300);   // no previous residual
}

// Out = X S (rows of the CTA's block), S from global (b x b, ld kB).  With
// ctl: skipped once converged (sel == 0), or (sel == 1) X = X1 when the
// converged iteration ctl[1] is odd (the ping-pong of the bases).
template <typename T>
__global__ void __launch_bounds__(256) split_apply_kernel(const T* X, const T* S, int M, int b, T* Out,
                                                          const unsigned long long* ctl = nullptr, int sel = 0,
                                                          const T* X1 = nullptr) {
  if (sel == 0 && split_done(ctl)) return;
  if (sel == 1 && (ctl[1] & 1ull)) X = X1;
  __shared__ T Ss[kB * kLd];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int p = e / b, q = e - (e / b) * b;
    Ss[p * kLd + q] = S[p * kB + q];
  }
  __syncthreads();
  const int i0 = blockIdx.x * kRowsPerCta;
  apply_rows<T>(X, Ss, b, b, Out, b, i0, min(M, i0 + kRowsPerCta));
}


template <typename T>
__global__ void copy_kernel(const T* src, T* dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

int eig_split_threshold() { return kEigSmallMax; }

#ifdef MACH_EIG_PHASES
extern "C" int mach_debug_eig_phases(unsigned long long* out8, int reset) {
  if (cudaMemcpyFromSymbol(out8, g_eig_phase, sizeof(unsigned long long) * 16) != cudaSuccess) return 4;
  if (reset) {
    unsigned long long z[16] = {};
    if (cudaMemcpyToSymbol(g_eig_phase, z, sizeof(z)) != cudaSuccess) return 4;
  }
  return 0;
}
#endif

// split-path scratch: per-row-block partial Grams, the b x b transform S,
// and the k-split partial tiles of C V
size_t eig_part_elems(int M) {
  // T partials, S, the C V slices, then (16-byte aligned) the FP64 partials
  // of the convergence test, counted in 4-byte elements
  return (size_t)ceil_div(M, kRowsPerCta) * 2 * kB * kB + kB * kB + (size_t)kCvSplit * M * kB + 8 +
         (size_t)ceil_div(M, kRowsPerCta) * 3 * kB * kB * 2;
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
  a.part = static_cast<T*>(e.part);
  a.Vout = e.Vout;
  a.theta = e.theta;
  a.maxit = e.maxit;
  a.tol = e.tol;
  a.stats = e.stats;
  a.basis_out = static_cast<T*>(e.basis_out);
  const int M = e.M, b = e.b;
  if (M <= kEigSmallMax) {
    cudaFuncAttributes fa;
    MACH_CUDA_TRY(cudaFuncGetAttributes(&fa, eig_fused_kernel<T>));
    int dev = 0, optin = 0;
    MACH_CUDA_TRY(cudaGetDevice(&dev));
    MACH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t budget = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
    const size_t vwu = (size_t)3 * M * (b | 1) * sizeof(T), cb = (size_t)M * (M | 1) * sizeof(T);
    int mode = 0;
    size_t bytes = 0;
    if (vwu + cb <= budget) {
      mode = 2;
      bytes = vwu + cb;
    } else if (vwu <= budget) {
      mode = 1;
      bytes = vwu;
    }
    MACH_TRY(allow_max_dyn_smem(eig_fused_kernel<T>));
    eig_fused_kernel<T><<<1, kEigThreads, bytes, st>>>(a, mode);
    MACH_LAUNCH_CHECK();
    return MACH_OK;
  }
  // split path: V0 -> orthonormal V; iterations (FP32: with a convergence
  // test and an early exit on the device, every later launch returning at
  // once; FP64: a fixed count); final rotation and FP64 Rayleigh-Ritz
  const int nblk = (int)ceil_div(M, kRowsPerCta);
  T* part = a.part;
  T* S = part + (size_t)nblk * 2 * b * b;
  T* cvp = S + kB * kB;
  const bool check = sizeof(T) == 4 && e.ctl != nullptr;
  double* part64 = nullptr;
  if (check) {
    uintptr_t p64 = reinterpret_cast<uintptr_t>(cvp + (size_t)kCvSplit * M * kB);
    p64 = (p64 + 15) & ~(uintptr_t)15;
    part64 = reinterpret_cast<double*>(p64);
  }
  unsigned long long* ctl = check ? e.ctl : nullptr;
  const dim3 cv_grid((unsigned)ceil_div(M, kCvRows), kCvSplit);
  const unsigned red_grid = (unsigned)ceil_div((int64_t)M * b, 256);
  if (ctl) {
    split_ctl_init<<<1, 32, 0, st>>>(ctl);
    MACH_LAUNCH_CHECK();
  }
  split_gram_vv_kernel<T><<<nblk, 256, 0, st>>>(a.V, M, b, part);
  MACH_LAUNCH_CHECK();
  split_bspace_kernel<T><<<1, 256, 0, st>>>(part, nblk, b, e.r, 0, S, e.rr, nullptr, nullptr, 0, 0.0);
  MACH_LAUNCH_CHECK();
  split_apply_kernel<T><<<nblk, 256, 0, st>>>(a.V, S, M, b, a.U);
  MACH_LAUNCH_CHECK();
  T* Vb[2] = {a.U, a.V};   // the orthonormal start is in U; the bases alternate
  T* W = a.W;
  const int iters = std::max(1, e.maxit);
  for (int it = 0; it < iters; ++it) {
    T* Vc = Vb[it & 1];
    T* Vn = Vb[(it + 1) & 1];
    cv_tiled_kernel<T><<<cv_grid, 256, 0, st>>>(C, M, Vc, b, b, cvp, ctl);
    MACH_LAUNCH_CHECK();
    cv_reduce_kernel<T><<<red_grid, 256, 0, st>>>(cvp, kCvSplit, M, b, W, b, ctl);
    MACH_LAUNCH_CHECK();
    // the residual test (FP64 Grams) every kSplitCheck-th iteration
    const bool test = ctl && it % kSplitCheck == kSplitCheck - 1 && it + 1 < iters;
    split_grams_kernel<T><<<nblk, 256, 0, st>>>(Vc, W, M, b, part, test ? part64 : nullptr, ctl);
    MACH_LAUNCH_CHECK();
    const bool last = it + 1 == iters;
    split_bspace_kernel<T><<<1, 256, 0, st>>>(part, nblk, b, e.r, last ? 2 : 1, S, e.rr, test ? part64 : nullptr,
                                              ctl, it, e.tol);
    MACH_LAUNCH_CHECK();
    if (ctl) {
      split_apply_kernel<T><<<nblk, 256, 0, st>>>(W, S, M, b, Vn, ctl, 0);   // next basis, until converged
      MACH_LAUNCH_CHECK();
    } else if (!last) {
      split_apply_kernel<T><<<nblk, 256, 0, st>>>(W, S, M, b, Vn);
      MACH_LAUNCH_CHECK();
    }
  }
  // Ritz vectors of the converged (or last) iteration's basis, into W
  if (ctl)
    split_apply_kernel<T><<<nblk, 256, 0, st>>>(Vb[0], S, M, b, W, ctl, 1, Vb[1]);
  else
    split_apply_kernel<T><<<nblk, 256, 0, st>>>(Vb[(iters - 1) & 1], S, M, b, W);
  MACH_LAUNCH_CHECK();
  if (a.basis_out) {
    copy_kernel<T><<<(unsigned)std::min<int64_t>(ceil_div((int64_t)M * b, 256), 1024), 256, 0, st>>>(
        W, a.basis_out, (int64_t)M * b);
    MACH_LAUNCH_CHECK();
  }
  split_finish_kernel<<<1, 32, 0, st>>>(e.r, e.rr, a.theta, a.stats, iters, ctl);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename T>
EigResult<T> eig_result(const EigLaunch& e) {
  EigResult<T> out;
  if (e.M <= kEigSmallMax) {
    out.U = eig_out_u<T>(e.Vout, e.r);
    out.ldu = e.r;
    out.X = e.Vout;
  } else {
    out.U = static_cast<const T*>(e.W);   // the Ritz vectors of the split path
    out.ldu = e.b;
    out.X = e.rr;
  }
  out.theta = e.theta;
  return out;
}

size_t eig_out_bytes(int M) { return (size_t)kMaxRank * kMaxRank * sizeof(double) + (size_t)M * kMaxRank * 8; }

template EigResult<float> eig_result<float>(const EigLaunch&);
template EigResult<double> eig_result<double>(const EigLaunch&);
template mach_status launch_eig<float>(const float*, const EigLaunch&, cudaStream_t);
template mach_status launch_eig<double>(const double*, const EigLaunch&, cudaStream_t);

}  // namespace mach
