// Accuracy measure of Section 4 ("Speedups & Synthetic Experiment"):
//   ||X - G x_1 A_1 ... x_d A_d|| / ||X||  against the original dense X.
// With orthonormal factors ||G x A|| = ||G||, so
//   ||X - X~||^2 = ||X||^2 - 2 <X, X~> + ||G||^2,
//   <X, X~> = sum over fibres f along the last mode of
//             sum_k (sum_i x_{f,i} A_d[i,k]) * P_f[k],
//   P_f[k] = sum_{r_1..r_{d-1}} G[r_1..r_{d-1}, k] prod_{j<d} A_j[i_j(f), r_j].
// One streaming pass over X; one warp per fibre (coalesced reads along the
// contiguous last mode); FP64 accumulation of the per-fibre terms.
#include "mach_internal.cuh"

namespace mach {

namespace {

template <typename V>
__global__ void error_kernel(const V* __restrict__ X, int d, int64_t nfib, int I_last, int r_last, int Jlead,
                             Decoder lead_dec, const double* __restrict__ A0, const double* __restrict__ A1,
                             const double* __restrict__ A2, const double* __restrict__ Alast, int I0, int I1, int I2,
                             int r0, int r1, int r2, const double* __restrict__ G, double* __restrict__ acc) {
  using T = V;  // accumulate along the fibre in the input precision
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double sx2 = 0.0, sxy = 0.0;
  for (int64_t f = gw; f < nfib; f += nw) {
    const V* xf = X + f * I_last;
    T t[kMaxRank];
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) t[k] = T(0);
    double x2 = 0.0;
    for (int i = lane; i < I_last; i += 32) {
      const T x = xf[i];
      x2 += (double)x * (double)x;
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k)
        if (k < r_last) t[k] += x * (T)Alast[(size_t)k * I_last + i];
    }
    // leading coordinates of the fibre
    uint32_t c[kMaxModes] = {0, 0, 0, 0};
    decode(lead_dec, (uint64_t)f, c);
    double P[kMaxRank];
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) P[k] = 0.0;
    for (int j = lane; j < Jlead; j += 32) {
      // j = C-order over (r_0 .. r_{d-2})
      double kron = 1.0;
      int rem = j;
      if (d == 4) {
        const int a2 = rem % r2;
        rem /= r2;
        kron *= A2[(size_t)a2 * I2 + c[2]];
      }
      if (d >= 3) {
        const int a1 = rem % r1;
        rem /= r1;
        kron *= A1[(size_t)a1 * I1 + c[1]];
      }
      kron *= A0[(size_t)rem * I0 + c[0]];
#pragma unroll
      for (int k = 0; k < kMaxRank; ++k)
        if (k < r_last) P[k] += G[(size_t)j * r_last + k] * kron;
    }
    double dot = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) {
      if (k < r_last) {
        const double tk = warp_sum((double)t[k]);
        const double pk = warp_sum(P[k]);
        dot += tk * pk;
      }
    }
    x2 = warp_sum(x2);
    if (lane == 0) {
      sx2 += x2;
      sxy += dot;
    }
  }
  if (lane == 0) {
    atomicAdd(&acc[0], sx2);
    atomicAdd(&acc[1], sxy);
  }
}

}  // namespace

mach_status launch_error(const void* x, mach_dtype dt, int d, const int64_t* dims, const int* ranks,
                         double* const* factors, const double* core, double* acc, cudaStream_t st) {
  MACH_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  const int I_last = (int)dims[d - 1];
  int64_t nfib = 1;
  for (int k = 0; k < d - 1; ++k) nfib *= dims[k];
  int Jlead = 1;
  for (int k = 0; k < d - 1; ++k) Jlead *= ranks[k];
  Decoder lead = make_decoder(d - 1, dims);
  const double* A[3] = {nullptr, nullptr, nullptr};
  int I[3] = {1, 1, 1}, r[3] = {1, 1, 1};
  for (int k = 0; k < d - 1; ++k) {
    A[k] = factors[k];
    I[k] = (int)dims[k];
    r[k] = ranks[k];
  }
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nfib * 32, threads), num_sms() * 16));
  if (dt == MACH_F32) {
    error_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(static_cast<const float*>(x), d, nfib, I_last,
                                                               ranks[d - 1], Jlead, lead, A[0], A[1], A[2],
                                                               factors[d - 1], I[0], I[1], I[2], r[0], r[1], r[2],
                                                               core, acc);
  } else {
    error_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(static_cast<const double*>(x), d, nfib, I_last,
                                                                ranks[d - 1], Jlead, lead, A[0], A[1], A[2],
                                                                factors[d - 1], I[0], I[1], I[2], r[0], r[1],
                                                                r[2], core, acc);
  }
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

}  // namespace mach
