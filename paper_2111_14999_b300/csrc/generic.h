// Stage-2 epilogue for any (nw, 3na) (generic.cu) and the power-of-two operand scaling
// shared with the tensor-core path.
#pragma once

#include <math.h>

#include "kernels.cuh"

namespace phx {

// Power-of-two factor that brings max|x| just below 2^14 (keeps FP16 parts in range; exact).
__host__ __device__ inline float pow2_scale(float maxabs) {
  if (!(maxabs > 0.f)) return 1.f;
  int e;
  frexpf(maxabs, &e);
  return ldexpf(1.f, 14 - e);
}
__device__ __forceinline__ float generic_pow2_scale(float maxabs) { return pow2_scale(maxabs); }

constexpr int kGenericMaxModes = kMaxModes;
constexpr int kGenericStatesPerBlock = 128;  // states per block of the generic epilogue

struct ElphGenericArgs {
  const float* G;          // [rows][ldg] stage-2 result of this q chunk, state s at columns s*2*nw*nm
  int64_t ldg;
  const int* q_of_row;     // q index of each A-operand row (-1: padding)
  int64_t row0;            // first A-operand row of the chunk
  int S;                   // states in the batch
  const int* st_k;         // [S] k-grid index
  const int* st_b;         // [S] band
  const double* epsF;      // [NF][nw]
  GridMap gm;
  int nw, nm;
  const float2* eps2;      // [NF][nw] (hi, lo)
  const float* f32;        // [NF][nw]
  const float2* UH;        // [NF][nw(m')][nw(m)] conj(U[m][m'])
  const float2* Zf;        // [Nq][nm][nm]
  const float* omf;        // [Nq][nm]
  const float* nBf;        // [Nq][nm]
  float reach, inv_sigma, cut2;
  double scale_base;       // (2 pi / N_q) / (sqrt(pi) sigma) / s_A^2
  const unsigned* tmax;    // max |T| of the batch (float bits): B operand scale pow2_scale(tmax)
  double* gamma;
  int64_t s_base;
};

size_t elph_generic_smem(int nw, int nm);
int launch_elph_generic(cudaStream_t s, const ElphGenericArgs& a, int64_t rows);

}  // namespace phx
