// Importance-sampled q sums with a learned proposal (sampler.cu): the interface the
// tensor-core linewidth path calls once per stage-1 batch.
#pragma once

#include <vector>

#include "pipeline.h"

namespace phx {

// One stage-1 batch of initial states, as the tensor-core path holds it.
struct IsBatch {
  int S = 0;                      // states in the batch
  int nkb = 0;                    // distinct initial k in the batch
  int64_t s_base = 0;             // offset of the batch in the call's state list
  const int* st_k = nullptr;      // device [S] k-grid index per state
  const int* st_b = nullptr;      // device [S] band per state
  const int* st_kb = nullptr;     // device [S] batch-local k index per state
  const int* kb = nullptr;        // device [nkb] k-grid index per batch k
  const std::vector<int>* st_kb_host = nullptr;
  const std::vector<int>* kb_host = nullptr;
  const float2* T = nullptr;      // device [S][nRp][3na][nw]: sum_Re w e^{ik.Re} g(Re,Rp) U_k, FP32 complex
};

// FP32 tables of the epilogue (fine grid for electrons, q grid for phonons) and FP64 inputs.
struct IsTables {
  const double* epsF = nullptr;   // [NF][nw]
  const double* fF = nullptr;     // [NF][nw] Fermi-Dirac occupations
  const cplx* UF = nullptr;       // [NF][nw][nw]
  const float2* eps2 = nullptr;   // [NF][nw] (hi, lo)
  const float* f32 = nullptr;     // [NF][nw]
  const float2* UH = nullptr;     // [NF][nw(m')][nw(m)] conj(U[m][m'])
  const double* omega = nullptr;  // [Nq][3na]
  const double* nB = nullptr;     // [Nq][3na]
  const cplx* Zq = nullptr;       // [Nq][3na][3na]
  double omega_max = 0.0;
};

template <int NW, int NM>
int is_batch(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, const IsBatch& b,
             const IsTables& t, double* raw);

}  // namespace phx
