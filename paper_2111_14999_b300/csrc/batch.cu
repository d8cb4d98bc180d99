// Linewidths of many materials in one call.  Phase 1 runs, per material on its own
// context, everything up to the stage-2 operands (grid bands, phonons, window, stage 1,
// packing, epilogue tables) and records the material's stage-2 launches with tile shapes
// chosen by timing the candidates (autotuner); a pool of host threads plans several
// materials at once, each on its material's stream, so that small materials, host-side
// planning and synchronisations of one material overlap the kernels of others.  Phase 2
// captures every recorded launch of every material into one CUDA graph, materials spread over
// parallel branches, and launches it once; the first item's context keeps the executable graph,
// which a later call with a graph of the same shape updates in place instead of instantiating.  Phase 3 averages degenerate bands and copies each material's outputs.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "pipeline.h"

using namespace phx;

namespace {

struct StreamSet {
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> e;
  ~StreamSet() {
    for (auto x : s) cudaStreamDestroy(x);
    for (auto x : e) cudaEventDestroy(x);
  }
};

int end_capture_discard(cudaStream_t cs) {
  cudaGraph_t g = nullptr;
  cudaStreamEndCapture(cs, &g);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return PHOEBE_GPU_ERR_CUDA;
}

}  // namespace

extern "C" void phoebe_gpu_batch_opts_default(phoebe_gpu_batch_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->autotune = 1;
  o->n_streams = 4;
  o->g_chunk_bytes = (int64_t)128 << 20;
  o->plan_threads = 1;
}

extern "C" int phoebe_gpu_linewidths_rta_batch(phoebe_gpu_batch_item* items, int n, phoebe_gpu_batch_opts* opts) {
  if (!items || n < 1) return PHOEBE_GPU_ERR_ARG;
  phoebe_gpu_batch_opts dflt;
  phoebe_gpu_batch_opts_default(&dflt);
  phoebe_gpu_batch_opts* o = opts ? opts : &dflt;
  if (o->n_streams < 1 || o->n_streams > 64 || o->g_chunk_bytes < ((int64_t)1 << 20)) return PHOEBE_GPU_ERR_ARG;
  if (o->plan_threads < 0 || o->plan_threads > 64) return PHOEBE_GPU_ERR_ARG;
  for (int i = 0; i < 2; ++i)
    if (o->reserved[i]) return PHOEBE_GPU_ERR_ARG;
  o->graph_reused = 0;
  bool count_only = false;
  for (int i = 0; i < n; ++i) {
    if (!items[i].ctx || !items[i].params) return PHOEBE_GPU_ERR_ARG;
    for (int j = 0; j < i; ++j)  // phase 1 plans materials concurrently: one context per item
      if (items[j].ctx == items[i].ctx)
        return fail(items[i].ctx, PHOEBE_GPU_ERR_ARG, "batch items %d and %d share a context", j, i);
    if (items[i].ctx->device != items[0].ctx->device) {
      return fail(items[i].ctx, PHOEBE_GPU_ERR_ARG, "batch item %d is on device %d, item 0 on device %d", i,
                  items[i].ctx->device, items[0].ctx->device);
    }
    if (!items[i].gamma_eV) count_only = true;
  }
  if (count_only) {
    for (int i = 0; i < n; ++i) {
      phoebe_gpu_rta_params p = *items[i].params;
      p.sampler = PHOEBE_SAMPLER_FULL;
      int cnt = 0;
      TRY(linewidths(items[i].ctx, &p, &cnt, nullptr, nullptr, nullptr, false));
      items[i].n_states = cnt;
    }
    return PHOEBE_GPU_OK;
  }
  if (cudaSetDevice(items[0].ctx->device) != cudaSuccess) return PHOEBE_GPU_ERR_CUDA;
  // ---- phase 1: per material, record stage 2
  auto wall = [] {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t.tv_sec * 1e3 + t.tv_nsec * 1e-6;
  };
  double t0 = wall();
  std::vector<Deferred> D(n);
  for (int i = 0; i < n; ++i)
    if (items[i].params->sampler != PHOEBE_SAMPLER_FULL)
      return fail(items[i].ctx, PHOEBE_GPU_ERR_UNSUPPORTED, "batched linewidths use the full q sum");
  std::atomic<int> next(0), first_err(PHOEBE_GPU_OK);
  const int device = items[0].ctx->device;
  auto plan = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      int ok = PHOEBE_GPU_OK;
      first_err.compare_exchange_strong(ok, PHOEBE_GPU_ERR_CUDA);
      return;
    }
    for (int i = next++; i < n && first_err.load() == PHOEBE_GPU_OK; i = next++) {
      phoebe_gpu_ctx* c = items[i].ctx;
      D[i].autotune = o->autotune != 0;
      D[i].g_budget = o->g_chunk_bytes;
      c->defer = &D[i];
      int cap = items[i].n_states;
      int r = linewidths(c, items[i].params, &cap, nullptr, nullptr, items[i].gamma_eV, false);
      c->defer = nullptr;
      if (r == PHOEBE_GPU_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        r = fail(c, PHOEBE_GPU_ERR_CUDA, "phase 1 of material %d failed on the device", i);
      }
      if (r != PHOEBE_GPU_OK) {
        int ok = PHOEBE_GPU_OK;
        first_err.compare_exchange_strong(ok, r);
        return;
      }
      items[i].n_states = cap;
    }
  };
  const int nthreads = std::max(1, std::min(o->plan_threads > 0 ? o->plan_threads : 1, n));
  if (nthreads == 1) {
    plan();
  } else {
    std::vector<std::thread> pool;
    for (int w = 0; w < nthreads; ++w) pool.emplace_back(plan);
    for (auto& th : pool) th.join();
  }
  if (first_err.load() != PHOEBE_GPU_OK) return first_err.load();
  if (cudaSetDevice(device) != cudaSuccess) return PHOEBE_GPU_ERR_CUDA;
  o->plan_ms = wall() - t0;
  // ---- phase 2: one graph holding every material's stage 2
  phoebe_gpu_ctx* c0 = items[0].ctx;
  cudaStream_t cs = nullptr;
  CK(c0, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  StreamSet ss;
  ss.s.push_back(cs);
  const int nb = o->n_streams;
  for (int w = 0; w < nb; ++w) {
    cudaStream_t s;
    CK(c0, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ss.s.push_back(s);
  }
  for (int w = 0; w < nb + 3; ++w) {
    cudaEvent_t e;
    CK(c0, cudaEventCreateWithFlags(&e, w < nb + 1 ? cudaEventDisableTiming : cudaEventDefault));
    ss.e.push_back(e);
  }
  cudaEvent_t fork = ss.e[0], ta = ss.e[nb + 1], tb = ss.e[nb + 2];
  CK(c0, cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  if (cudaEventRecord(fork, cs) != cudaSuccess) return end_capture_discard(cs);
  for (int w = 0; w < nb; ++w)
    if (cudaStreamWaitEvent(ss.s[1 + w], fork, 0) != cudaSuccess) return end_capture_discard(cs);
  int64_t ops = 0;
  for (int i = 0; i < n; ++i) {
    phoebe_gpu_ctx* c = items[i].ctx;
    cudaStream_t saved = c->stream;
    c->stream = ss.s[1 + i % nb];
    for (auto& op : D[i].ops) {
      const int r = op();
      if (r != PHOEBE_GPU_OK) {
        c->stream = saved;
        end_capture_discard(cs);
        return r;
      }
      ++ops;
    }
    c->stream = saved;
  }
  for (int w = 0; w < nb; ++w) {
    if (cudaEventRecord(ss.e[1 + w], ss.s[1 + w]) != cudaSuccess) return end_capture_discard(cs);
    if (cudaStreamWaitEvent(cs, ss.e[1 + w], 0) != cudaSuccess) return end_capture_discard(cs);
  }
  cudaGraph_t graph = nullptr;
  CK(c0, cudaStreamEndCapture(cs, &graph));
  // the executable graph kept on c0 by an earlier call, updated in place when this graph has its
  // shape (same nodes and edges; kernel arguments and launch shapes may differ), else a new one
  cudaGraphExec_t exec = c0->batch_exec;
  cudaError_t ge = cudaErrorUnknown;
  if (exec) {
    cudaGraphExecUpdateResultInfo ui;
    ge = cudaGraphExecUpdate(exec, graph, &ui);
    if (ge != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(exec);
      c0->batch_exec = exec = nullptr;
    } else {
      o->graph_reused = 1;
    }
  }
  if (!exec) {
    ge = cudaGraphInstantiate(&exec, graph, 0);
    if (ge == cudaSuccess) c0->batch_exec = exec;
  }
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  cudaGraphDestroy(graph);
  if (ge != cudaSuccess) {
    cudaGetLastError();
    return fail(c0, PHOEBE_GPU_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ge));
  }
  cudaError_t le = cudaEventRecord(ta, cs);
  if (le == cudaSuccess) le = cudaGraphLaunch(exec, cs);
  if (le == cudaSuccess) le = cudaEventRecord(tb, cs);
  if (le == cudaSuccess) le = cudaStreamSynchronize(cs);
  if (le != cudaSuccess) {
    cudaGraphExecDestroy(exec);
    c0->batch_exec = nullptr;
    cudaGetLastError();
    return fail(c0, PHOEBE_GPU_ERR_CUDA, "batch graph launch failed: %s", cudaGetErrorString(le));
  }
  float gms = 0.f;
  cudaEventElapsedTime(&gms, ta, tb);
  o->graph_ms = gms;
  o->graph_nodes = (int64_t)nodes;
  o->recorded_launches = ops;
  // ---- phase 3: wait flags, degenerate averaging, outputs
  t0 = wall();
  for (int i = 0; i < n; ++i) {
    phoebe_gpu_ctx* c = items[i].ctx;
    auto it = c->bufs.find("tc_err");
    if (it != c->bufs.end() && it->second.p) {
      int herr = 0;
      CK(c, cudaMemcpy(&herr, it->second.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a tensor-core pipeline wait ran out; results discarded");
    }
    c->defer = &D[i];
    const int r = linewidths_finish(c, items[i].k_index, items[i].band, items[i].gamma_eV, false);
    c->defer = nullptr;
    if (r != PHOEBE_GPU_OK) return r;
    items[i].tile_n = D[i].bn;
    items[i].tile_kb = D[i].kb;
  }
  o->finish_ms = wall() - t0;
  return PHOEBE_GPU_OK;
}
