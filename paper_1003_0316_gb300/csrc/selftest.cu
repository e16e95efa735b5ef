// Diagnostic (no counterpart in the paper): exercises the bounded-wait machinery that every
// pipelined kernel of the library relies on. One thread waits on an mbarrier that nothing
// arrives on, with a wall-time limit; when the limit expires it records ST_ETIMEOUT in the
// status word and returns, so gw_check reports GW_ETIMEOUT and the context stays usable.
#include "gw_internal.cuh"
#include "tc_ptx.cuh"

namespace gw {

namespace {

__global__ void k_wait_selftest(uint64_t limit_ns, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int never;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    never = 0;
  }
  __syncthreads();
  // phase 0 of a fresh barrier completes only after one arrival, which never comes
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, &never, limit_ns))
    raise_status(status, ST_ETIMEOUT);
}

}  // namespace

int selftest_bounded_wait(double limit_ms, cudaStream_t s, const DeviceCtx& ctx) {
  k_wait_selftest<<<1, 32, 0, s>>>(uint64_t(limit_ms * 1e6), ctx.status);
  GW_LAUNCH_CHECK("k_wait_selftest");
  return GW_OK;
}

}  // namespace gw
