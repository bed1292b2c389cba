// Self-check of the bounded device-side wait that every kernel of libmach
// uses on its mbarriers (mach_check_bounded_wait in include/mach.h): one
// CTA waits on an mbarrier phase with a caller-given iteration limit.  With
// `arrive` set, the CTA's own thread arrives first and the wait completes;
// without it nothing ever arrives, so the wait runs out of iterations,
// records DEV_TIMEOUT in the status word and the kernel returns normally.
// No asynchronous copy is attached to the barrier, so nothing is left in
// flight when the kernel ends.
#include "mach_internal.cuh"

namespace mach {

namespace {

__global__ void bounded_wait_kernel(long long limit, int arrive, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit)) atomicOr(status, DEV_TIMEOUT);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar)) : "memory");
}

}  // namespace

mach_status run_bounded_wait_check(long long limit, int arrive, cudaStream_t st) {
  unsigned* d_status = nullptr;
  DevBuf buf;
  MACH_TRY(dev_alloc(buf, sizeof(unsigned), st));
  d_status = static_cast<unsigned*>(buf.ptr);
  unsigned h = 0;
  mach_status s = MACH_OK;
  if (cudaMemsetAsync(d_status, 0, sizeof(unsigned), st) != cudaSuccess) s = MACH_ECUDA;
  if (s == MACH_OK) {
    bounded_wait_kernel<<<1, 32, 0, st>>>(limit, arrive, d_status);
    count_launch();
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_last_error("bounded-wait check: %s", cudaGetErrorString(cudaGetLastError()));
      s = MACH_ECUDA;
    }
  }
  dev_free(buf, st);
  cudaStreamSynchronize(st);
  if (s != MACH_OK) return s;
  return (h & DEV_TIMEOUT) ? MACH_ETIMEOUT : MACH_OK;
}

}  // namespace mach
