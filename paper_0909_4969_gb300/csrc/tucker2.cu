// Tucker2 of a 3-way tensor (Section 2.1, the Tucker family: compressing n
// of the d modes is a Tucker-n decomposition; Section 4 uses a Tucker2 of
// the sensor tensor, leaving the time mode uncompressed).  Mode c is kept
// whole; for each compressed mode n the other compressed mode m is the only
// one contracted:
//   Y_(n)[i_n, (beta, i_c)] = sum_{i_m} X^[i_n, i_m, i_c] A_m[i_m, beta],
// i.e. one vector per fibre along mode m, which is the leaf level of the
// CSF whose leaf index is i_m (rows and mids = i_n and i_c in some order).
// The core is G = X^ x_a A_a^T x_b A_b^T, of size r_a x r_b x I_c (modes in
// their natural order).
#include "mach_internal.cuh"

namespace mach {

namespace {

constexpr int kT2Warps = 8;

// Y (I_n x (r_m * I_c), row-major, zero beforehand): warp per row of the
// source CSF, lane per fibre; z_f = sum_e x_e A_m[i_m(e), :] goes to
// Y[i_n][beta * I_c + i_c] (each (i_n, i_c) pair is one fibre).
template <typename V, typename T, int RLM>
__global__ void __launch_bounds__(32 * kT2Warps) tucker2_leaf_kernel(const V* __restrict__ val,
                                                                     const uint16_t* __restrict__ leaf,
                                                                     const uint32_t* __restrict__ fib_start,
                                                                     const uint32_t* __restrict__ fib_mid,
                                                                     const uint32_t* __restrict__ row_fib, int rows,
                                                                     const T* __restrict__ Am, int rm, int row_is_n,
                                                                     int I_c, T* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kT2Warps + (threadIdx.x >> 5);
  const int nw = gridDim.x * kT2Warps;
  const int64_t ld = (int64_t)rm * I_c;
  for (int row = gw; row < rows; row += nw) {
    const uint32_t f0 = row_fib[row], f1 = row_fib[row + 1];
    for (uint32_t f = f0 + lane; f < f1; f += 32) {
      T z[RLM];
#pragma unroll
      for (int b = 0; b < RLM; ++b) z[b] = T(0);
      const uint32_t e1 = fib_start[f + 1];
      for (uint32_t e = fib_start[f]; e < e1; ++e) {
        const T x = (T)val[e];
        const T* ar = Am + (size_t)leaf[e] * rm;
#pragma unroll
        for (int b = 0; b < RLM; ++b)
          if (b < rm) z[b] += x * ar[b];
      }
      const int mid = (int)fib_mid[f];
      const int i_n = row_is_n ? row : mid, i_c = row_is_n ? mid : row;
      T* y = Y + (size_t)i_n * ld + i_c;
#pragma unroll
      for (int b = 0; b < RLM; ++b)
        if (b < rm) y[(size_t)b * I_c] = z[b];
    }
  }
}

// G (C order over the modes (0, 1, 2) with sizes (r'_0, r'_1, r'_2), r'_c =
// I_c) from the last compressed mode L: G[.., k at L, beta at O, i_c at c]
// = scale * sum_i A_L[i, k] Y_(L)[i][beta * I_c + i_c].  One warp per output,
// FP64 sums.
template <typename T>
__global__ void tucker2_core_kernel(const T* __restrict__ Y, const double* __restrict__ A, int I_L, int r_L, int r_O,
                                    int I_c, int L, int O, int c, double scale, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nout = (int64_t)r_L * r_O * I_c;
  if (gw >= nout) return;
  const int k = (int)(gw / ((int64_t)r_O * I_c));
  const int64_t rest = gw - (int64_t)k * r_O * I_c;
  const int beta = (int)(rest / I_c), ic = (int)(rest - (int64_t)beta * I_c);
  const int64_t ld = (int64_t)r_O * I_c;
  double s = 0.0;
  for (int i = lane; i < I_L; i += 32) s += A[(size_t)k * I_L + i] * (double)Y[(size_t)i * ld + (size_t)beta * I_c + ic];
  s = warp_sum(s);
  if (lane == 0) {
    int g[3], size[3];
    g[L] = k;
    g[O] = beta;
    g[c] = ic;
    size[L] = r_L;
    size[O] = r_O;
    size[c] = I_c;
    G[((int64_t)g[0] * size[1] + g[1]) * size[2] + g[2]] = s * scale;
  }
}

__global__ void identity_colmajor_kernel(double* A, int n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    A[e] = (e % (n + 1)) == 0 ? 1.0 : 0.0;
}

template <typename V, typename T>
mach_status launch_leaf_vt(const Tucker2Leaf& a, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a.rows, kT2Warps), (int64_t)num_sms() * 8));
  const V* val = static_cast<const V*>(a.val);
  const T* Am = static_cast<const T*>(a.Am);
  T* Y = static_cast<T*>(a.Y);
  if (a.rm <= 4)
    tucker2_leaf_kernel<V, T, 4><<<grid, 32 * kT2Warps, 0, st>>>(val, a.leaf, a.fib_start, a.fib_mid, a.row_fib,
                                                                 a.rows, Am, a.rm, a.row_is_n, a.I_c, Y);
  else if (a.rm <= 8)
    tucker2_leaf_kernel<V, T, 8><<<grid, 32 * kT2Warps, 0, st>>>(val, a.leaf, a.fib_start, a.fib_mid, a.row_fib,
                                                                 a.rows, Am, a.rm, a.row_is_n, a.I_c, Y);
  else
    tucker2_leaf_kernel<V, T, 16><<<grid, 32 * kT2Warps, 0, st>>>(val, a.leaf, a.fib_start, a.fib_mid, a.row_fib,
                                                                  a.rows, Am, a.rm, a.row_is_n, a.I_c, Y);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

}  // namespace

template <typename T>
mach_status launch_tucker2_leaf(const Tucker2Leaf& a, mach_dtype vdt, cudaStream_t st) {
  if (a.rm < 1 || a.rm > kMaxRank) return MACH_EINVAL;
  MACH_CUDA_TRY(cudaMemsetAsync(a.Y, 0, (size_t)a.I_n * a.rm * a.I_c * sizeof(T), st));
  return vdt == MACH_F32 ? launch_leaf_vt<float, T>(a, st) : launch_leaf_vt<double, T>(a, st);
}

template <typename T>
mach_status launch_tucker2_core(const T* Y, const double* A_L, int I_L, int r_L, int r_O, int I_c, int L, int O,
                                int c, double scale, double* G, cudaStream_t st) {
  const int64_t nout = (int64_t)r_L * r_O * I_c;
  const int64_t threads = nout * 32;
  tucker2_core_kernel<T><<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(Y, A_L, I_L, r_L, r_O, I_c, L, O, c,
                                                                           scale, G);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

mach_status launch_identity_colmajor(double* A, int n, cudaStream_t st) {
  identity_colmajor_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)n * n, 256), 1024)),
                             256, 0, st>>>(A, n);
  MACH_LAUNCH_CHECK();
  return MACH_OK;
}

template mach_status launch_tucker2_leaf<float>(const Tucker2Leaf&, mach_dtype, cudaStream_t);
template mach_status launch_tucker2_leaf<double>(const Tucker2Leaf&, mach_dtype, cudaStream_t);
template mach_status launch_tucker2_core<float>(const float*, const double*, int, int, int, int, int, int, int, double,
                                                double*, cudaStream_t);
template mach_status launch_tucker2_core<double>(const double*, const double*, int, int, int, int, int, int, int,
                                                 double, double*, cudaStream_t);

}  // namespace mach
