// wp_selftest_bounded_wait: exercises the library's bounded device-side waits
// on a barrier that nothing ever completes, so that their expiry path (status
// word set to WP_ERR_TIMEOUT, kernel returns normally) can be tested on a GPU
// without a fault.  Nothing is in flight when the wait gives up: no TMA copy,
// no MMA and no remote store targets the barrier.

#include "common.cuh"
#include "jacobi_block.cuh"
#include "tc_ptx.cuh"

namespace wp {

// which = 0: ptx::mbar_wait (the tensor-core kernels' CTA-scope waits);
// which = 1: jblock::wait_peers (the Jacobi kernels' cluster-scope waits).
__global__ void __launch_bounds__(32) bounded_wait_kernel(int which, uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);   // one arrival expected; none is ever made
    ptx::fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  if (which == 0) ptx::mbar_wait(&bar, 0, status, limit_ns);
  else jblock::wait_peers(ptx::smem_u32(&bar), 0, status, limit_ns);
}

}  // namespace wp

extern "C" int wp_selftest_bounded_wait(int which, int64_t limit_ns, void* stream) {
  if (which != 0 && which != 1) return WP_ERR_SHAPE;
  if (limit_ns < 1000 || limit_ns > 100000000) return WP_ERR_SHAPE;
  cudaStream_t st = wp::as_stream(stream);
  WP_PROFILE("bounded_wait_selftest", st);
  wp::bounded_wait_kernel<<<1, 32, 0, st>>>(which, uint64_t(limit_ns), wp::device_status_ptr());
  return wp::launch_status();
}
