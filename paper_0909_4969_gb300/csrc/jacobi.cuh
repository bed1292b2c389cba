// Register-resident cyclic Jacobi eigensolver for a small symmetric matrix
// on one warp (shared by the single-CTA eigensolver and the batched HOOI
// kernel).
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

}  // namespace
}  // namespace mach
