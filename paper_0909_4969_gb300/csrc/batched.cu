// Batched MACH-HOOI (Algorithm 2, the loop and the core) for many small
// 3-way tensors in ONE persistent launch.  Every CTA owns one decomposition
// at a time (grid-stride over the batch) and runs all of its sweeps and its
// core without leaving the kernel:
//
//   for each sweep, for n = 1..3 (Gauss-Seidel):
//     Y_(n) = X^ x_{k != n} A_k^T      fibre by fibre over the mode-n CSF
//                                      (Section 2.1 n-mode products)
//     C     = Y^T Y  (J_n < I_n)  or  Y Y^T  (I_n <= J_n);  M = min(I_n, J_n) <= 32
//     C     = Q diag(lambda) Q^T       cyclic Jacobi on one warp
//     A_n   = Y Q_r lambda_r^-1/2  (or Q_r), re-orthonormalised by a Cholesky
//             QR whose r x r Gram, factor and inverse are FP64
//   G = (1/p) A_3^T Y_(3)             (Algorithm 2's core, from the last Y)
//
// The arithmetic of the sweeps is FP32 (values as stored, factors FP32);
// the eigenvectors come from a full Jacobi of the small Gram, so there is no
// iteration tolerance.  Designed for the shapes of streamed monitoring
// windows: every J_n = prod_{k != n} r_k <= 32, leaf ranks <= 16.  Lane q of
// a warp owns column q of Y_(n); a warp owns whole rows, so every sum has a
// fixed order and the result does not depend on the grid.
#include "mach_internal.cuh"
#include "jacobi.cuh"

#include <algorithm>

namespace mach {

namespace {

constexpr int kBatWarps = 8;
constexpr int kBatThreads = 32 * kBatWarps;
constexpr int kBatMaxJ = 32;
constexpr int kBatLd = kBatMaxJ + 1;

struct BatShared {
  union {
    struct {
      float sz[kBatWarps][32][17];   // leaf-level fibre vectors of a batch of 32 fibres
      float sa[kBatWarps][32][17];   // the A_mid row of each of those fibres
    } t;
    float part[kBatWarps][kBatMaxJ][kBatLd];   // per-warp partial Grams
  } u;
  float C[kBatMaxJ * kBatLd];    // Gram, diagonalised in place
  float Q[kBatMaxJ * kBatLd];    // its eigenvectors (columns)
  float V[kBatMaxJ * kMaxRank];  // leading eigenvectors scaled by lambda^-1/2 (J x r)
  float Rf[kMaxRank * kMaxRank]; // R^-1 of the re-orthonormalisation (FP32 copy)
  double G[kMaxRank * kMaxRank]; // FP64 Gram of A, then its Cholesky factor
  double Ri[kMaxRank * kMaxRank];
  int perm[kBatMaxJ];
};

// Per-warp partial of X^T Y for R x n row-major X and Y (n <= 32), rows
// [warp, warp + 8, ..): lane q keeps column q in registers; the partials land
// in part[warp][k][q] = sum_i X[i][k] Y[i][q].  X == Y gives the Gram, with
// bitwise-symmetric entries.
__device__ __forceinline__ void cross_cols_partial(const float* X, const float* Y, int R, int n, int ld,
                                                   BatShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float c[kBatMaxJ];
#pragma unroll
  for (int k = 0; k < kBatMaxJ; ++k) c[k] = 0.f;
  for (int i = warp; i < R; i += kBatWarps) {
    const float x = lane < n ? X[(size_t)i * ld + lane] : 0.f;
    const float y = lane < n ? Y[(size_t)i * ld + lane] : 0.f;
#pragma unroll
    for (int k = 0; k < kBatMaxJ; ++k)
      if (k < n) c[k] += __shfl_sync(0xffffffffu, x, k) * y;
  }
#pragma unroll
  for (int k = 0; k < kBatMaxJ; ++k)
    if (k < n) sh.u.part[warp][k][lane] = c[k];
}

__device__ __forceinline__ void gram_cols_partial(const float* X, int R, int n, BatShared& sh) {
  cross_cols_partial(X, X, R, n, n, sh);
}

// Out (R x n) = X R^-1 for the Cholesky factor of X^T X (n <= 16; rows of
// X and Out at stride ld >= n): the FP32 Gram partials are summed in FP64,
// G = R^T R and R^-1 are FP64 (one warp), the product runs one thread per
// row.  Out may alias X.
__device__ void bat_orth(const float* X, int R, int n, int ld, float* Out, BatShared& sh, unsigned* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cross_cols_partial(X, X, R, n, ld, sh);
  __syncthreads();
  for (int e = tid; e < n * n; e += kBatThreads) {
    const int k = e / n, q = e - k * n;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kBatWarps; ++w) s += (double)sh.u.part[w][k][q];
    sh.G[e] = s;
  }
  __syncthreads();
  if (warp == 0) {
    double* G = sh.G;
    bool bad = false;
    for (int j = 0; j < n; ++j) {
      double djj = G[j * n + j];
      if (!(djj > 0.0)) {
        bad = true;
        djj = 1e-300;
      }
      djj = sqrt(djj);
      __syncwarp();
      if (lane == j) G[j * n + j] = djj;
      if (lane > j && lane < n) G[j * n + lane] /= djj;
      __syncwarp();
      if (lane > j && lane < n)
        for (int c = lane; c < n; ++c) G[lane * n + c] -= G[j * n + lane] * G[j * n + c];
      __syncwarp();
    }
    if (lane < n) {
      const int j = lane;
      for (int i = n - 1; i >= 0; --i) {
        double v = i == j ? 1.0 : 0.0;
        for (int k = i + 1; k <= j; ++k) v -= G[i * n + k] * sh.Ri[k * n + j];
        sh.Ri[i * n + j] = i > j ? 0.0 : v / G[i * n + i];
      }
    }
    __syncwarp();
    for (int e = lane; e < n * n; e += 32) sh.Rf[e] = (float)sh.Ri[e];
    if (lane == 0 && bad) atomicOr(err, DEV_NOTPD);
  }
  __syncthreads();
  for (int i = tid; i < R; i += kBatThreads) {
    float a[kMaxRank], o[kMaxRank];
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) {
      a[k] = k < n ? X[(size_t)i * ld + k] : 0.f;
      o[k] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kMaxRank; ++j)
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k)
        if (j < n && k < n && j <= k) o[k] += a[j] * sh.Rf[j * n + k];
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k)
      if (k < n) Out[(size_t)i * ld + k] = o[k];
  }
  __syncthreads();
}

// Y_(n) (I x J row-major) for mode n: warp per row, 32 fibres of the row per
// step: lane l forms the leaf-level vector z_f = sum_e x_e A_leaf[i_leaf(e), :]
// of its fibre and stages it with the fibre's A_mid row in shared memory;
// then lane q = (a, b) folds Y[i, q] += A_mid[i_mid(f), a] z_f[b] over the
// step's fibres in fibre order.
template <typename V, int RLM>
__device__ void bat_ttmc(const BatMode& m, int I, const float* Amid, int rm, const float* Aleaf, int rl, float* Y,
                         int J, BatShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const V* val = static_cast<const V*>(m.val);
  const int aq = lane / rl, bq = lane - aq * rl;   // column lane = aq * r_leaf + bq
  for (int i = warp; i < I; i += kBatWarps) {
    const uint32_t f0 = m.row_fib[i], f1 = m.row_fib[i + 1];
    float acc = 0.f;
    for (uint32_t fb = f0; fb < f1; fb += 32) {
      const uint32_t f = fb + lane;
      float z[RLM];
#pragma unroll
      for (int b = 0; b < RLM; ++b) z[b] = 0.f;
      if (f < f1) {
        const uint32_t e0 = m.fib_start[f], e1 = m.fib_start[f + 1];
#pragma unroll 4
        for (uint32_t e = e0; e < e1; ++e) {
          const float v = (float)val[e];
          const float* ar = Aleaf + (size_t)m.leaf[e] * rl;
#pragma unroll
          for (int b = 0; b < RLM; ++b)
            if (b < rl) z[b] += v * ar[b];
        }
        const float* am = Amid + (size_t)m.fib_mid[f] * rm;
#pragma unroll
        for (int a = 0; a < 16; ++a)
          if (a < rm) sh.u.t.sa[warp][lane][a] = am[a];
      }
#pragma unroll
      for (int b = 0; b < RLM; ++b) sh.u.t.sz[warp][lane][b] = z[b];
      __syncwarp();
      const int nv = (int)min(32u, f1 - fb);
      if (lane < J) {
#pragma unroll 8
        for (int j = 0; j < nv; ++j) acc += sh.u.t.sa[warp][j][aq] * sh.u.t.sz[warp][j][bq];
      }
      __syncwarp();
    }
    if (lane < J) Y[(size_t)i * J + lane] = acc;
  }
}

__device__ void bat_jacobi(BatShared& sh, int M) {
  const float tol = 1e-7f;
  if (M <= 8) jacobi_reg<float, 8>(sh.C, sh.Q, kBatLd, M, tol, 16);
  else if (M <= 16) jacobi_reg<float, 16>(sh.C, sh.Q, kBatLd, M, tol, 16);
  else if (M <= 24) jacobi_reg<float, 24>(sh.C, sh.Q, kBatLd, M, tol, 16);
  else jacobi_reg<float, 32>(sh.C, sh.Q, kBatLd, M, tol, 16);
}

// A_n (I x r, row-major FP32) = leading r left singular vectors of Y (I x J).
__device__ void bat_lsv(const float* Y, int I, int J, int r, float* A, BatShared& sh, unsigned* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool jroute = J < I;
  const int M = jroute ? J : I;
  // Gram of the smaller side
  if (jroute) {
    gram_cols_partial(Y, I, J, sh);
    __syncthreads();
    for (int e = tid; e < M * M; e += kBatThreads) {
      const int k = e / M, q = e - k * M;
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < kBatWarps; ++w) s += sh.u.part[w][k][q];
      sh.C[k * kBatLd + q] = s;
    }
  } else {
    for (int e = tid; e < M * M; e += kBatThreads) {
      const int i = e / M, k = e - i * M;
      float s = 0.f;
      for (int q = 0; q < J; ++q) s += Y[(size_t)i * J + q] * Y[(size_t)k * J + q];
      sh.C[i * kBatLd + k] = s;
    }
  }
  __syncthreads();
  // eigenvectors (one warp), descending eigenvalues
  if (warp == 0) {
    bat_jacobi(sh, M);
    if (lane < M) {
      const float v = sh.C[lane * kBatLd + lane];
      int rank = 0;
      for (int j = 0; j < M; ++j) {
        const float u = sh.C[j * kBatLd + j];
        rank += (u > v) || (u == v && j < lane);
      }
      sh.perm[rank] = lane;
    }
    __syncwarp();
  }
  __syncthreads();
  if (jroute) {
    // V = Q_r lambda_r^-1/2, then A = Y V (thread per row)
    for (int e = tid; e < J * r; e += kBatThreads) {
      const int q = e / r, k = e - q * r;
      const int pk = sh.perm[k];
      const float lam = sh.C[pk * kBatLd + pk];
      sh.V[q * kMaxRank + k] = lam > 0.f ? sh.Q[q * kBatLd + pk] * rsqrtf(lam) : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < I; i += kBatThreads) {
      float a[kMaxRank];
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k) a[k] = 0.f;
      for (int q = 0; q < J; ++q) {
        const float y = Y[(size_t)i * J + q];
#pragma unroll
        for (int k = 0; k < kMaxRank; ++k)
          if (k < r) a[k] += y * sh.V[q * kMaxRank + k];
      }
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k)
        if (k < r) A[(size_t)i * r + k] = a[k];
    }
  } else {
    for (int e = tid; e < I * r; e += kBatThreads) {
      const int i = e / r, k = e - i * r;
      A[(size_t)i * r + k] = sh.Q[i * kBatLd + sh.perm[k]];
    }
  }
  __syncthreads();
  // re-orthonormalise (FP64 r x r Gram, Cholesky factor and inverse)
  bat_orth(A, I, r, r, A, sh, err);
}

constexpr int kHosvdB = 16;     // block width of the HOSVD subspace iteration
constexpr int kHosvdIt = 40;    // its iteration cap (the start of the oracle is the exact HOSVD)
constexpr int kHosvdCheck = 4;  // Ritz residuals are tested every kHosvdCheck iterations
constexpr float kHosvdTol = 5e-7f;   // ... against this fraction of the largest Ritz value, or
                                     // 10x that once they stop halving (the FP32 floor)

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Uniform deviate in [-1/2, 1/2) from (seed, counter): a 64-bit
// finalising mix (splitmix64 constants of Steele, Lea and Flood, OOPSLA
// 2014); only the start block of the HOSVD iteration uses it.
__device__ __forceinline__ float start_deviate(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(uint32_t)(z >> 40) * (1.0f / 16777216.0f) - 0.5f;
}

// W = X^_(n) X^_(n)^T V for V (I x 16, row-major), through the fibres along
// mode n, i.e. the CSF `src` whose leaf index is i_n: X^_(n) X^_(n)^T =
// sum_f s_f s_f^T over those fibres, so each fibre gives t = s_f^T V and
// adds x_e t to row i_n(e) of W for each of its entries e (vector atomics).
template <typename V>
__device__ void bat_gram_apply(const BatMode& src, int rows_src, int I, const float* Vb, float* W) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < I * kHosvdB; e += kBatThreads) W[e] = 0.f;
  __syncthreads();
  const V* val = static_cast<const V*>(src.val);
  for (int row = warp; row < rows_src; row += kBatWarps) {
    const uint32_t f0 = src.row_fib[row], f1 = src.row_fib[row + 1];
    for (uint32_t f = f0 + lane; f < f1; f += 32) {
      const uint32_t e0 = src.fib_start[f], e1 = src.fib_start[f + 1];
      float t[kHosvdB];
#pragma unroll
      for (int c = 0; c < kHosvdB; ++c) t[c] = 0.f;
#pragma unroll 4
      for (uint32_t e = e0; e < e1; ++e) {
        const float x = (float)val[e];
        const float4* vr = reinterpret_cast<const float4*>(Vb + (size_t)src.leaf[e] * kHosvdB);
#pragma unroll
        for (int c4 = 0; c4 < kHosvdB / 4; ++c4) {
          const float4 v = vr[c4];
          t[4 * c4] += x * v.x;
          t[4 * c4 + 1] += x * v.y;
          t[4 * c4 + 2] += x * v.z;
          t[4 * c4 + 3] += x * v.w;
        }
      }
      for (uint32_t e = e0; e < e1; ++e) {
        const float x = (float)val[e];
        float* wr = W + (size_t)src.leaf[e] * kHosvdB;
#pragma unroll
        for (int c4 = 0; c4 < kHosvdB / 4; ++c4)
          red_add_v4(wr + 4 * c4, x * t[4 * c4], x * t[4 * c4 + 1], x * t[4 * c4 + 2], x * t[4 * c4 + 3]);
      }
    }
  }
  __threadfence();
  __syncthreads();
}

// Rayleigh-Ritz of the block: H = V^T W (W = C V, symmetrised) diagonalised
// by Jacobi on one warp; sh.C holds the Ritz values on its diagonal, sh.Q
// the rotation, sh.perm their descending order.  W is read through L2 (it
// is accumulated by atomics).
__device__ void bat_block_rr(const float* Vb, const float* W, int I, int bw, BatShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  cross_cols_partial(Vb, W, I, bw, kHosvdB, sh);
  __syncthreads();
  for (int e = tid; e < bw * bw; e += kBatThreads) {
    const int k = e / bw, q = e - k * bw;
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int w = 0; w < kBatWarps; ++w) {
      s1 += sh.u.part[w][k][q];
      s2 += sh.u.part[w][q][k];
    }
    sh.C[k * kBatLd + q] = 0.5f * (s1 + s2);
  }
  __syncthreads();
  if (warp == 0) {
    if (bw <= 8) jacobi_reg<float, 8>(sh.C, sh.Q, kBatLd, bw, 1e-7f, 16);
    else jacobi_reg<float, 16>(sh.C, sh.Q, kBatLd, bw, 1e-7f, 16);
    if (lane < bw) {
      const float v = sh.C[lane * kBatLd + lane];
      int rank = 0;
      for (int j = 0; j < bw; ++j) {
        const float u = sh.C[j * kBatLd + j];
        rank += (u > v) || (u == v && j < lane);
      }
      sh.perm[rank] = lane;
    }
    __syncwarp();
  }
  __syncthreads();
}

// Whether the leading r Ritz pairs of the last bat_block_rr have residuals
// ||W q_j - theta_j V q_j|| below kHosvdTol theta_1 (all threads return
// the same answer).
__device__ bool bat_ritz_converged(const float* Vb, const float* W, int I, int bw, int r, BatShared& sh,
                                   float* prev) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float res[kMaxRank];
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) res[k] = 0.f;
  for (int i = tid; i < I; i += kBatThreads) {
    float v[kHosvdB], w[kHosvdB];
#pragma unroll
    for (int c = 0; c < kHosvdB; ++c) {
      v[c] = Vb[(size_t)i * kHosvdB + c];
      w[c] = __ldcg(W + (size_t)i * kHosvdB + c);
    }
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) {
      if (k < r) {
        const int pk = sh.perm[k];
        const float th = sh.C[pk * kBatLd + pk];
        float e = 0.f;
#pragma unroll
        for (int c = 0; c < kHosvdB; ++c)
          if (c < bw) e += (w[c] - th * v[c]) * sh.Q[c * kBatLd + pk];
        res[k] += e * e;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) res[k] = warp_sum(res[k]);
  __shared__ float wres[kBatWarps][kMaxRank];
  __shared__ int conv;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) wres[warp][k] = res[k];
  __syncthreads();
  if (tid == 0) {
    const float th0 = sh.C[sh.perm[0] * kBatLd + sh.perm[0]];
    float worst = 0.f;
    for (int k = 0; k < r; ++k) {
      float t = 0.f;
      for (int w = 0; w < kBatWarps; ++w) t += wres[w][k];
      worst = fmaxf(worst, t);
    }
    const float rel = th0 > 0.f ? sqrtf(worst) / th0 : 0.f;
    conv = (th0 > 0.f && rel <= kHosvdTol) || (rel <= 10.f * kHosvdTol && rel > 0.5f * *prev) ? 1 : 0;
    *prev = rel;
  }
  __syncthreads();
  const bool out = conv != 0;
  __syncthreads();
  return out;
}

// HOSVD start of mode n (Algorithm 2's initialisation): A_n = leading r
// eigenvectors of X^_(n) X^_(n)^T by kHosvdIt block subspace iterations of
// width 16 from a seeded random block, then a Rayleigh-Ritz step on the last
// block (H = V^T C V, Jacobi, A = V Q_r).  Vb, W: I x 16 scratch (16-byte
// aligned); W is read through L2 only (it is accumulated by atomics).
template <typename V>
__device__ void bat_hosvd_mode(const BatMode& src, int rows_src, int I, int r, uint64_t seed, float* Vb, float* W,
                               float* A, BatShared& sh, unsigned* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // block width bw = min(16, I); rows of Vb and W have stride 16 (unused
  // columns are zero).  When I <= 16 the block is the identity, so one
  // product gives the whole Gram and the Rayleigh-Ritz step is exact.
  const int bw = min(kHosvdB, I);
  const bool exact = I <= kHosvdB;
  for (int e = tid; e < I * kHosvdB; e += kBatThreads) {
    const int i = e / kHosvdB, c = e - i * kHosvdB;
    Vb[e] = c >= bw ? 0.f : (exact ? (i == c ? 1.f : 0.f) : start_deviate(seed, (uint64_t)e));
  }
  __syncthreads();
  if (!exact) bat_orth(Vb, I, bw, kHosvdB, Vb, sh, err);
  bool have_rr = false;
  __shared__ float prev_res;
  if (tid == 0) prev_res = 3.0e38f;
  for (int it = 0;; ++it) {
    bat_gram_apply<V>(src, rows_src, I, Vb, W);
    if (exact || it + 1 == kHosvdIt) break;
    // every kHosvdCheck iterations: stop once the leading r Ritz pairs have
    // converged (the Rayleigh-Ritz step below is then the one just made)
    if (it % kHosvdCheck == kHosvdCheck - 1) {
      bat_block_rr(Vb, W, I, bw, sh);
      if (bat_ritz_converged(Vb, W, I, bw, r, sh, &prev_res)) {
        have_rr = true;
        break;
      }
    }
    // V <- orth(W): W is staged into V through L2 first
    for (int e = tid; e < I * kHosvdB; e += kBatThreads) Vb[e] = __ldcg(W + e);
    __syncthreads();
    bat_orth(Vb, I, bw, kHosvdB, Vb, sh, err);
  }
  // Rayleigh-Ritz: H = V^T W (symmetrised), eigenvectors Q, A = V Q_r
  if (!have_rr) bat_block_rr(Vb, W, I, bw, sh);
  for (int i = tid; i < I; i += kBatThreads) {
    float v[kHosvdB];
#pragma unroll
    for (int c = 0; c < kHosvdB; ++c) v[c] = Vb[(size_t)i * kHosvdB + c];
    for (int k = 0; k < r; ++k) {
      const int pk = sh.perm[k];
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < kHosvdB; ++c)
        if (c < bw) s += v[c] * sh.Q[c * kBatLd + pk];
      A[(size_t)i * r + k] = s;
    }
  }
  __syncthreads();
}

template <typename V, int RLM>
__global__ void __launch_bounds__(kBatThreads, 2) batched_hooi_kernel(BatArgs a) {
  __shared__ BatShared sh;
  const int tid = threadIdx.x;
  float* ws = a.ws + (size_t)blockIdx.x * a.ws_stride;
  __shared__ int claim;
  for (;;) {
    // items are claimed in order (the host sorts them largest first)
    if (tid == 0) claim = (int)atomicAdd(a.next, 1u);
    __syncthreads();
    const int bi = claim;
    if (bi >= a.B) break;
    const BatItem& it = a.items[bi];
    int I[3];
    float* A[3];
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
      I[k] = it.dims[k];
      A[k] = ws + off;
      off += ((size_t)I[k] * a.r[k] + 31) & ~(size_t)31;
    }
    float* Y = ws + off;
    if (a.warm) {
      // start factors: FP64 column-major -> FP32 row-major
      for (int k = 0; k < 3; ++k)
        for (int e = tid; e < I[k] * a.r[k]; e += kBatThreads) {
          const int i = e / a.r[k], c = e - i * a.r[k];
          A[k][e] = (float)it.fac[k][(size_t)c * I[k] + i];
        }
      __syncthreads();
    } else {
      // HOSVD start; Vb and W share the space of Y (I_n x 16 each)
      int imax = max(I[0], max(I[1], I[2]));
      float* Vb = Y;
      float* W = Y + (((size_t)imax * kHosvdB + 31) & ~(size_t)31);
      for (int n = 0; n < 3; ++n) {
        const int src = (n + 1) % 3;
        bat_hosvd_mode<V>(it.mode[src], I[src], I[n], a.r[n], it.seed ^ (0x5bd1e995ull * (uint64_t)(n + 1)), Vb, W,
                          A[n], sh, it.err);
      }
    }
    const int sweeps = a.sweeps;
    for (int sw = 0; sw < sweeps || (sw == 0 && it.core); ++sw) {
      for (int n = 0; n < 3; ++n) {
        if (sw >= sweeps && n < 2) continue;   // sweeps == 0: only the last mode's Y for the core
        const int mid = (n + 1) % 3, leaf = (n + 2) % 3;
        const int J = a.r[mid] * a.r[leaf];
        bat_ttmc<V, RLM>(it.mode[n], I[n], A[mid], a.r[mid], A[leaf], a.r[leaf], Y, J, sh);
        __syncthreads();
        if (sw < sweeps) bat_lsv(Y, I[n], J, a.r[n], A[n], sh, it.err);
      }
    }
    // core G = (1/p) A_3^T Y_(3): entry (c, k) at c * r_3 + k, C order r_1 x r_2 x r_3
    if (it.core) {
      const int J = a.r[0] * a.r[1], r3 = a.r[2];
      for (int e = tid; e < J * r3; e += kBatThreads) {
        const int c = e / r3, k = e - c * r3;
        double s = 0.0;
        for (int i0 = 0; i0 < I[2]; i0 += 64) {
          float t = 0.f;
          const int i1 = min(I[2], i0 + 64);
          for (int i = i0; i < i1; ++i) t += A[2][(size_t)i * r3 + k] * Y[(size_t)i * J + c];
          s += (double)t;
        }
        it.core[e] = s * it.inv_p;
      }
    }
    // factors out: FP32 row-major -> FP64 column-major
    for (int k = 0; k < 3; ++k)
      for (int e = tid; e < I[k] * a.r[k]; e += kBatThreads) {
        const int i = e / a.r[k], c = e - i * a.r[k];
        it.fac[k][(size_t)c * I[k] + i] = (double)A[k][e];
      }
    __syncthreads();
  }
}

template <typename V, int RLM>
mach_status launch_batched_vr(const BatArgs& a, int grid, cudaStream_t st) {
  batched_hooi_kernel<V, RLM><<<grid, kBatThreads, 0, st>>>(a);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template <typename V>
mach_status launch_batched_v(const BatArgs& a, int grid, int rlm, cudaStream_t st) {
  if (rlm <= 4) return launch_batched_vr<V, 4>(a, grid, st);
  if (rlm <= 8) return launch_batched_vr<V, 8>(a, grid, st);
  return launch_batched_vr<V, 16>(a, grid, st);
}

}  // namespace

int batched_max_j() { return kBatMaxJ; }

// floats of the HOSVD start's two I x 16 blocks (they share the space of Y)
int64_t batched_hosvd_scratch(int64_t max_dim) { return 2 * ((max_dim * kHosvdB + 31) & ~(int64_t)31); }

int batched_grid(int B) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_hooi_kernel<float, 16>, kBatThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return std::max(1, std::min(B, num_sms() * per_sm));
}

mach_status launch_batched_hooi(const BatArgs& a, mach_dtype dt, int grid, cudaStream_t st) {
  int rlm = 1;
  for (int n = 0; n < 3; ++n) rlm = std::max(rlm, a.r[(n + 2) % 3]);
  if (dt == MACH_F32) return launch_batched_v<float>(a, grid, rlm, st);
  return launch_batched_v<double>(a, grid, rlm, st);
}

}  // namespace mach
