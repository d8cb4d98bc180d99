// Check of the bounded device waits every pipeline kernel uses: a consumer waits on an
// mbarrier phase that a producer publishes only if the host asks it to.  Unpublished, the
// wait gives up after the limit, raises the abort flag and the call returns
// PHOEBE_GPU_ERR_TIMEOUT with the context still usable.
#include "pipeline.h"
#include "tc_ptx.cuh"

namespace phx {

using namespace tc;

__global__ void k_wait_check(int publish, unsigned long long limit_ns, int* __restrict__ err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 32 && publish) mbar_arrive(&bar);  // the producer of the phase
  if (threadIdx.x == 0) {
    if (!mbar_wait_limit(&bar, 0u, &abort_flag, limit_ns)) atomicOr(err, 1);
  }
  __syncthreads();
}

}  // namespace phx

using namespace phx;

extern "C" int phoebe_gpu_selftest_wait(phoebe_gpu_ctx* c, int publish, int64_t limit_us) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (limit_us < 1 || limit_us > 10000000) return fail(c, PHOEBE_GPU_ERR_ARG, "selftest_wait: limit in 1..1e7 us");
  int st;
  int* err = (int*)ensure(c, "selftest_err", 64, &st);
  if (!err) return st;
  CK(c, cudaMemsetAsync(err, 0, 64, c->stream));
  k_wait_check<<<1, 64, 0, c->stream>>>(publish ? 1 : 0, (unsigned long long)limit_us * 1000ull, err);
  c->launches++;
  CK(c, cudaGetLastError());
  int h = 0;
  CK(c, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (h) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a bounded device wait ran out after %lld us", (long long)limit_us);
  return PHOEBE_GPU_OK;
}
