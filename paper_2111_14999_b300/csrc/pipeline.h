// Host-side context and orchestration interfaces of the phoebe_gpu library.
#pragma once

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "kernels.cuh"

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct TcState;  // tensor-core path state (tc_gemm.cu)

struct phoebe_gpu_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int cc = 0;
  std::string err;
  int64_t mem_cap = 0, mem_used = 0;
  bool profiling = false;
  int64_t launches = 0;
  phoebe_gpu_stats stats{};
  std::map<std::string, DBuf> bufs;
  // inputs
  bool have_H = false, have_Phi = false, have_g = false;
  int nw = 0, nRH = 0;
  int na = 0, nRf = 0;
  int nRe = 0, nRp = 0, g_nw = 0, g_na = 0;
  double we_max = 1.0, wp_max = 1.0;  // max |weight| of the R_e / R_p sets
  // tensor-core operands derived from g (invalidated by set_*)
  bool tc_g_valid = false;
  TcState* tc = nullptr;
  // learned q proposal: FP32 master parameters and Adam state live in bufs "mlp_*"
  bool have_mlp = false;
  int64_t adam_t = 0;
  // set by the sampler entry points for the duration of one pipeline call
  struct IsRequest* isreq = nullptr;
  // set by the batch entry point: stage 2 is recorded instead of launched
  struct Deferred* defer = nullptr;
  // phonon-electron rates requested by phoebe_gpu_phonon_rates_elph: accumulation [Nq][3na] and
  // the finished rates (device), nullptr otherwise
  double* prate_acc = nullptr;
  double* prate_out = nullptr;
  // primitive lattice vectors (rows, Cartesian, A), set by phoebe_gpu_set_lattice
  bool have_lattice = false;
  double lattice[9] = {0};
  // polar long-range coupling, set by phoebe_gpu_set_polar
  // third-order force constants, set by phoebe_gpu_set_force_constants3 (device buffers ph3_*)
  bool have_phi3 = false;
  int ph3_na = 0, ph3_nrp = 0;
  std::vector<int> ph3_rp;  // [ph3_nrp][3] the distinct R' (lattice coordinates), host copy
  // the autotuner's stage-2 tile choice (tile width, K blocks per partial) per GEMM problem
  // (operand format, parts, products, K, columns, q rows, q rows per chunk), kept for later calls
  std::map<std::vector<int64_t>, std::pair<int, int>> tuned_tiles;
  // the executable graph of the last batch call that named this context first (batch.cu)
  cudaGraphExec_t batch_exec = nullptr;
  bool have_polar = false;
  std::vector<double> zstar;  // [na][3][3]
  double eps_inf[9] = {0};
  double polar_alpha = 0.0;
};

// Stage-2 work of one material recorded for later issue (batch.cu): each op launches
// on the context's stream at the time it is called, so a caller can capture it.
struct Deferred {
  std::vector<std::function<int()>> ops;
  bool autotune = true;
  int bn = 0, kb = 0;              // stage-2 tile columns and K blocks per TMEM partial (0: default)
  int64_t g_budget = (int64_t)128 << 20;  // bytes of the G buffer per q chunk
  double tune_ms[6] = {0, 0, 0, 0, 0, 0};  // candidates (bn, kb) in {128, 256} x {1, 2, 4}
  // what the finishing step needs
  int64_t ns = 0;
  phx::GridMap gm{};
  double degen_tol = 0.0;
};

// What the sampled q sums of one pipeline call must produce (sampler.cu).
struct IsRequest {
  int mode = 0;             // 1: importance-sampled Gamma into the raw accumulator; 2: c_nk(q) of every q
  float* c_out = nullptr;   // mode 2: device [n_states][N_q]
  float* feat_out = nullptr;  // optional: device [n_states][4] (eps - mu, v)
  float* lphi_out = nullptr;  // mode 2, optional: device [n_states][N_q] log of the shell factor
};

namespace phx {

int fail(phoebe_gpu_ctx* c, int code, const char* fmt, ...);
int cuda_fail(phoebe_gpu_ctx* c, cudaError_t e, const char* what, int line);

#define CK(ctx, call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) {                                \
      cudaGetLastError();                                   \
      return phx::cuda_fail((ctx), e_, #call, __LINE__);    \
    }                                                       \
  } while (0)

#define TRY(...)                 \
  do {                           \
    int st_ = (__VA_ARGS__);     \
    if (st_ != PHOEBE_GPU_OK) return st_; \
  } while (0)

void* ensure(phoebe_gpu_ctx* c, const char* name, size_t bytes, int* status);
void release(phoebe_gpu_ctx* c, const char* name);
int upload(phoebe_gpu_ctx* c, const char* name, const void* host, size_t bytes, void** dev);

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  void begin(phoebe_gpu_ctx* c);
  void end(phoebe_gpu_ctx* c, double* acc);
};

GridPhase make_phase(const int n[3]);
int cis_table(phoebe_gpu_ctx* c, const GridPhase& gp, const char* name, cplx** out);
int electron_grid(phoebe_gpu_ctx* c, const int n[3], double** eps, cplx** U);
int velocity_grid(phoebe_gpu_ctx* c, const int n[3], const cplx* U, float4** vel);
int three_phonon(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, double* out_host);
int phonon_modes(phoebe_gpu_ctx* c, const int n[3], const double* qpts_dev, int64_t Q, double T,
                 double omega_cut, double** omega, double** nB, cplx** Z, const char* tag);

int linewidths(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int* n_states, int32_t* k_index,
               int32_t* band, double* gamma, bool device_out);
// Degenerate averaging of the raw accumulator of the last (deferred) linewidths call and the
// copy of its outputs.
int linewidths_finish(phoebe_gpu_ctx* c, int32_t* k_index, int32_t* band, double* gamma, bool device_out);
int interpolate_pairs(phoebe_gpu_ctx* c, int n_pairs, const double* k, const double* q, int precision,
                      double* g2, double* eps_k, double* eps_kq, double* omega_q);

// tensor-core path (tc_gemm.cu)
void destroy_tc_state(phoebe_gpu_ctx* c);

}  // namespace phx
