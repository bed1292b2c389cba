// Small dense eigensolvers shared by the single-CTA eigensolver and the
// batched HOOI kernel: the register-resident cyclic Jacobi of one warp, and
// the FP64 iterative refinement of a few Ritz pairs (CTAs of 256 threads).
#pragma once

#include "mach_internal.cuh"

namespace mach {
namespace {

// Cyclic Jacobi (Golub & Van Loan, sym.schur2 rotations) in round-robin
// ("circle") pair order, register resident on one warp.  The matrix is kept
// in position order: lane a holds row a of H and the positions pair up as
// (k, NP-1-k) in every round; after each round positions 1..NP-1 shift by
// one (rows by a shuffle, columns by renaming registers), which walks
// through the circle pairings with every register index a compile-time
// constant.  After NP-1 rounds (one sweep) the order is the identity again.
// Lane i also holds row i of the accumulated rotation Q (columns =
// eigenvectors, in position order).  Padding to NP (a multiple of 8, <= 32)
// is zero and stays exactly zero.  H <- J^T H J until the off-diagonal mass
// is below rel_tol^2 of the diagonal's, or stalls at the rounding floor;
// the result goes back to H and Q (shared memory, leading dimension ldm).
template <typename T, int NP>
__device__ __noinline__ void jacobi_reg(T* Hs, T* Qs, int ldm, int n, T rel_tol, int max_sweeps) {
  const int lane = threadIdx.x & 31;
  const bool in_np = lane < NP;
  const int mate = in_np ? NP - 1 - lane : lane;                       // partner position
  const int src = lane == 0 || !in_np ? lane : (lane == NP - 1 ? 1 : lane + 1);  // row shift
  const int pair = lane < NP / 2 ? lane : NP - 1 - lane;
  const bool is_p = lane < NP / 2;
  T h[NP], q[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    h[j] = (lane < n && j < n) ? Hs[lane * ldm + j] : T(0);
    q[j] = lane == j ? T(1) : T(0);
  }
  T prev_off = T(-1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), dia = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const T v = h[j] * h[j];
      if (j == lane) dia += v; else off += v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (off <= rel_tol * rel_tol * dia) break;
    const T floor_rel = sizeof(T) == 8 ? T(1e-12) : T(1e-4);
    if (prev_off >= T(0) && off > T(0.25) * prev_off && off <= floor_rel * floor_rel * dia) break;
    prev_off = off;
#pragma unroll 1
    for (int round = 0; round < NP - 1; ++round) {
      // lane k < NP/2 takes (h_pp, h_qq, h_pq) of pair (k, NP-1-k)
      T pp = T(0), qq = T(0), pq = T(0);
#pragma unroll
      for (int k = 0; k < NP / 2; ++k) {
        const T vpp = __shfl_sync(0xffffffffu, h[k], k);
        const T vqq = __shfl_sync(0xffffffffu, h[NP - 1 - k], NP - 1 - k);
        const T vpq = __shfl_sync(0xffffffffu, h[NP - 1 - k], k);
        if (lane == k) {
          pp = vpp;
          qq = vqq;
          pq = vpq;
        }
      }
      T c = T(1), sn = T(0);
      if (pq != T(0)) {
        const T tau = (qq - pp) / (T(2) * pq);
        const T at = fabs(tau);
        const T t = at > T(1e15) ? T(0.5) / tau : (tau >= T(0) ? T(1) : T(-1)) / (at + sqrt(T(1) + tau * tau));
        c = T(1) / sqrt(T(1) + t * t);
        sn = t * c;
      }
      // H <- H J and Q <- Q J (columns k, NP-1-k of every lane's row)
#pragma unroll
      for (int k = 0; k < NP / 2; ++k) {
        const T ck = __shfl_sync(0xffffffffu, c, k), sk = __shfl_sync(0xffffffffu, sn, k);
        const T hp = h[k], hq = h[NP - 1 - k];
        h[k] = ck * hp - sk * hq;
        h[NP - 1 - k] = sk * hp + ck * hq;
        const T qp = q[k], qv = q[NP - 1 - k];
        q[k] = ck * qp - sk * qv;
        q[NP - 1 - k] = sk * qp + ck * qv;
      }
      // H <- J^T H: rows k and NP-1-k, exchanged between the pair's lanes
      T cm = __shfl_sync(0xffffffffu, c, pair), sm = __shfl_sync(0xffffffffu, sn, pair);
      if (!in_np) {
        cm = T(1);
        sm = T(0);
      }
      const T sg = is_p ? -sm : sm;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const T other = __shfl_sync(0xffffffffu, h[j], mate);
        h[j] = cm * h[j] + sg * other;
      }
      // next pairing: position a takes the contents of position src(a)
#pragma unroll
      for (int j = 0; j < NP; ++j) h[j] = __shfl_sync(0xffffffffu, h[j], src);
      const T h1 = h[1], q1 = q[1];
#pragma unroll
      for (int j = 1; j < NP - 1; ++j) {
        h[j] = h[j + 1];
        q[j] = q[j + 1];
      }
      h[NP - 1] = h1;
      q[NP - 1] = q1;
    }
  }
  if (lane < n) {
#pragma unroll
    for (int j = 0; j < NP; ++j)
      if (j < n) {
        Hs[lane * ldm + j] = h[j];
        Qs[lane * ldm + j] = q[j];
      }
  }
  __syncwarp();
}

// FP64, n <= 16, leading dimension ldm (fallback of the final Rayleigh-Ritz).
__device__ void jacobi_warp_small(double* H, double* Qm, int ldm, int n, double rel_tol, int max_sweeps) {
  if (n <= 8) jacobi_reg<double, 8>(H, Qm, ldm, n, rel_tol, max_sweeps);
  else if (n <= 12) jacobi_reg<double, 12>(H, Qm, ldm, n, rel_tol, max_sweeps);
  else jacobi_reg<double, 16>(H, Qm, ldm, n, rel_tol, max_sweeps);
}

constexpr int kRRWarps = 8;   // warps of the CTAs that call rr_refine (256 threads)
// ----------------------------------------------------------------------------
// Final Rayleigh-Ritz of the leading r Ritz vectors in FP64 (r <= 16).
// Given the projected matrix H = U_r^T C U_r and the Gram G = U_r^T U_r of
// the Ritz basis (orthonormal and diagonalising up to the b-space
// arithmetic), the eigenvectors of the pencil (H, G) are refined with the
// iterative refinement of Ogita and Aishima (Japan J. Indust. Appl. Math.
// 35, 2018): for the estimate X, S = X^T H X, R = I - X^T G X,
// lambda_i = S_ii / (1 - R_ii), E_ij = (S_ij + lambda_j R_ij) /
// (lambda_j - lambda_i) for pairs separated by more than
// delta = 2 (||offdiag S||_F + max|lambda| ||R||_F), R_ij / 2 otherwise,
// and X <- X (I + E).  The error is squared by every round, so from a
// start that is diagonal to FP32 precision one round reaches the FP32
// paths' accuracy and two reach FP64 precision; when four rounds do not
// converge, a cyclic FP64 Jacobi on H is used instead.  All threads of the CTA; one thread per entry.
// ----------------------------------------------------------------------------
constexpr int kRl = kMaxRank + 1;
struct FinalRR {
  double H[kMaxRank * kRl], G[kMaxRank * kRl], X[kMaxRank * kRl];
  double T1[kMaxRank * kRl], T2[kMaxRank * kRl];
  double lam[kMaxRank];
  double red[3][kRRWarps];
  double delta, emax;
  int perm[kMaxRank];
};

// `accept`: the round whose largest correction is below it is the last (the
// remaining error is of the order of its square times the eigenvalue spread
// over the smallest gap): 1e-5 for the FP32 paths, 1e-7 for FP64.
__device__ void rr_refine(FinalRR& f, int r, double accept) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const bool act = tid < r * r;
  const int i = act ? tid / r : 0, j = act ? tid - (tid / r) * r : 0;
  if (act) f.X[i * kRl + j] = i == j ? 1.0 : 0.0;
  __syncthreads();
  bool ok = false;
  for (int round = 0; round < 4 && !ok; ++round) {
    double sx = 0.0, rx = 0.0;
    if (round == 0) {
      // X = I: S = H and R = I - G, no products
      if (act) {
        sx = f.H[i * kRl + j];
        rx = (i == j ? 1.0 : 0.0) - f.G[i * kRl + j];
      }
    } else {
      // two partial sums per product: FP64 dependences are long on this part
      if (act) {
        double a0 = 0.0, a1 = 0.0, g0 = 0.0, g1 = 0.0;
        int k = 0;
        for (; k + 1 < r; k += 2) {
          const double x0 = f.X[k * kRl + j], x1 = f.X[(k + 1) * kRl + j];
          a0 += f.H[i * kRl + k] * x0;
          g0 += f.G[i * kRl + k] * x0;
          a1 += f.H[i * kRl + k + 1] * x1;
          g1 += f.G[i * kRl + k + 1] * x1;
        }
        if (k < r) {
          const double x0 = f.X[k * kRl + j];
          a0 += f.H[i * kRl + k] * x0;
          g0 += f.G[i * kRl + k] * x0;
        }
        f.T1[i * kRl + j] = a0 + a1;   // H X
        f.T2[i * kRl + j] = g0 + g1;   // G X
      }
      __syncthreads();
      if (act) {
        double s0 = 0.0, s1 = 0.0, r0 = 0.0, r1 = 0.0;
        int k = 0;
        for (; k + 1 < r; k += 2) {
          const double x0 = f.X[k * kRl + i], x1 = f.X[(k + 1) * kRl + i];
          s0 += x0 * f.T1[k * kRl + j];
          r0 += x0 * f.T2[k * kRl + j];
          s1 += x1 * f.T1[(k + 1) * kRl + j];
          r1 += x1 * f.T2[(k + 1) * kRl + j];
        }
        if (k < r) {
          const double x0 = f.X[k * kRl + i];
          s0 += x0 * f.T1[k * kRl + j];
          r0 += x0 * f.T2[k * kRl + j];
        }
        sx = s0 + s1;
        rx = (i == j ? 1.0 : 0.0) - (r0 + r1);
      }
    }
    __syncthreads();
    if (act) {
      f.T1[i * kRl + j] = sx;  // S
      f.T2[i * kRl + j] = rx;  // R
      if (i == j) f.lam[i] = sx / (1.0 - rx);
    }
    double o = (act && i != j) ? sx * sx : 0.0, q = act ? rx * rx : 0.0;
    o = warp_sum(o);
    q = warp_sum(q);
    if (lane == 0) {
      f.red[0][warp] = o;
      f.red[1][warp] = q;
    }
    __syncthreads();
    if (warp == 0) {
      // warp-parallel sums over the warps and maximum over lambda
      double so = lane < nw ? f.red[0][lane] : 0.0, sr = lane < nw ? f.red[1][lane] : 0.0;
      double lm = lane < r ? fabs(f.lam[lane]) : 0.0;
      so = warp_sum(so);
      sr = warp_sum(sr);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, d));
      if (lane == 0) f.delta = 2.0 * (sqrt(so) + lm * sqrt(sr));
    }
    __syncthreads();
    double e = 0.0;
    if (act) {
      if (i == j) {
        e = 0.5 * rx;
      } else {
        const double li = f.lam[i], lj = f.lam[j];
        e = fabs(lj - li) > f.delta ? (sx + lj * rx) / (lj - li) : 0.5 * rx;
      }
    }
    double em = act ? fabs(e) : 0.0;
    if (em != em) em = 1e300;   // NaN: never converged
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) em = fmax(em, __shfl_xor_sync(0xffffffffu, em, d));
    if (lane == 0) f.red[2][warp] = em;
    __syncthreads();
    if (act) f.T1[i * kRl + j] = e;   // E (S no longer needed)
    if (warp == 0) {
      double m = lane < nw ? f.red[2][lane] : 0.0;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
      if (lane == 0) f.emax = m;
    }
    __syncthreads();
    double xn = 0.0;
    if (act) {
      double x0 = f.X[i * kRl + j], x1 = 0.0;
      int k = 0;
      for (; k + 1 < r; k += 2) {
        x0 += f.X[i * kRl + k] * f.T1[k * kRl + j];
        x1 += f.X[i * kRl + k + 1] * f.T1[(k + 1) * kRl + j];
      }
      if (k < r) x0 += f.X[i * kRl + k] * f.T1[k * kRl + j];
      xn = x0 + x1;
    }
    __syncthreads();
    if (act) f.X[i * kRl + j] = xn;
    ok = f.emax < accept;
    __syncthreads();
  }
  if (!ok) {
    if (tid < 32) {
      jacobi_warp_small(f.H, f.X, kRl, r, 1e-15, 12);
      if (tid < r) f.lam[tid] = f.H[tid * kRl + tid];
    }
    __syncthreads();
  }
  // descending order of lambda (ties: lower index first)
  if (tid < r) {
    const double v = f.lam[tid];
    int rank = 0;
    for (int k = 0; k < r; ++k) {
      const double u = f.lam[k];
      rank += (u > v) || (u == v && k < tid);
    }
    f.perm[rank] = tid;
  }
  __syncthreads();
}

}  // namespace
}  // namespace mach
