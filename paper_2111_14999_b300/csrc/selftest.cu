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

// FP32 FMA rate: every thread runs 8 independent chains x <- x a + b (a < 1, so the values stay
// finite), iters steps each; the one store at the end, guarded by a test the data never passes,
// keeps the chains live.
__global__ void __launch_bounds__(256) k_fma_rate(int iters, float a, float b, float* __restrict__ sink) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) t += x[j];
  if (t == -1.0f) sink[blockIdx.x] = t;
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

extern "C" int phoebe_gpu_selftest_fp32_rate(phoebe_gpu_ctx* c, double* tflops, double* ms) {
  if (!c || !tflops) return PHOEBE_GPU_ERR_ARG;
  int st, sms = 0;
  CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  float* sink = (float*)ensure(c, "selftest_sink", sizeof(float) * 64 * sms, &st);
  if (!sink) return st;
  const int blocks = 8 * sms, threads = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  double best = 0.0, best_ms = 0.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up, the fastest of the rest counts
    cudaEventRecord(e0, c->stream);
    k_fma_rate<<<blocks, threads, 0, c->stream>>>(iters, 0.999f, 1e-4f, sink);
    cudaEventRecord(e1, c->stream);
    c->launches++;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(c, PHOEBE_GPU_ERR_CUDA, "the FP32 rate probe failed");
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    if (rep > 0 && t > 0.f && flops / (t * 1e-3) / 1e12 > best) {
      best = flops / (t * 1e-3) / 1e12;
      best_ms = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  if (ms) *ms = best_ms;
  return PHOEBE_GPU_OK;
}
