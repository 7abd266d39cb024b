// Failure-path self-test: a kernel whose bounded wait runs out.
//
// Every kernel of the library that waits (on an mbarrier phase: bulk-copy
// completion, tensor-core commits, arrivals of other warps) gives up after a
// bounded number of SM clocks, writes DEV_TIMEOUT to the handle's error word,
// drains what it has in flight and returns, and the entry point turns the
// word into KRR_ERR_TIMEOUT.  No input makes a healthy product or solve wait
// that long, so this entry point provides a wait that cannot complete: one
// thread initialises an mbarrier that expects one arrival, nothing ever
// arrives, and the thread waits with the same bounded routine the products
// use (with a short, caller-given limit).  No bulk copy, MMA or other warp is
// outstanding on the barrier, so giving up leaves nothing in flight.  The
// host then reads the error word exactly as after a product.
#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

__global__ void wait_timeout_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  if (!mbar_wait_for(&bar, 0, limit)) atomicExch(err, DEV_TIMEOUT);
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" krr_status krr_selftest_wait_timeout(krr_handle h, long long limit_clocks, void* stream) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  if (limit_clocks < 1 || limit_clocks > WAIT_LIMIT_CLOCKS)
    return set_error(c, KRR_ERR_INVALID_ARG, "krr_selftest_wait_timeout: limit %lld out of [1, %lld]",
                     limit_clocks, WAIT_LIMIT_CLOCKS);
  cudaStream_t st = (cudaStream_t)stream;
  wait_timeout_kernel<<<1, 32, 0, st>>>(c.d_err, limit_clocks); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e) return cuda_error(c, e, "krr_selftest_wait_timeout");
  return read_device_error(c, st, "krr_selftest_wait_timeout");
}
