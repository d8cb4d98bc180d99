// Tensor-core inference of the learned q proposal (mlp_tc.cu).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

namespace phx {

// Offsets of the parameter blob (float32): W1[128][7], b1, W2[128][128], b2, W3[128][128], b3, w4, b4.
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + 128 * 7;
constexpr int kMlpOffW2 = kMlpOffB1 + 128;
constexpr int kMlpOffB2 = kMlpOffW2 + 128 * 128;
constexpr int kMlpOffW3 = kMlpOffB2 + 128;
constexpr int kMlpOffB3 = kMlpOffW3 + 128 * 128;
constexpr int kMlpOffW4 = kMlpOffB3 + 128;
constexpr int kMlpOffB4 = kMlpOffW4 + 128;

struct MlpTcArgs {
  const __half* W2h;       // [128][128] layer-2 weights in FP16
  const __half* W3h;       // [128][128]
  const float* P;          // parameter blob, BF16-rounded values
  const float* qt;         // [Nq][3] wrapped q
  const float* feat;       // [S][4] the state features (eps - mu, hbar v)
  int64_t Nq;
  int64_t tiles_per_state; // ceil(Nq / 128)
  int64_t ntiles;          // S * tiles_per_state
  float* z;                // [S][Nq] scores
  int* err;                // set to 1 if a bounded wait ran out
  // optional row list: rows[r] = (state, q) for r < *nrows (device count); the kernel then walks
  // ceil(*nrows / 128) tiles (ntiles is only the grid's upper bound) and writes z[state][q] of
  // those rows alone
  const int2* rows = nullptr;
  const unsigned long long* nrows = nullptr;
};

size_t mlp_tc_smem_bytes();
int mlp_tc_params(cudaStream_t s, const float* P, __half* W2h, __half* W3h);
int mlp_tc_launch(cudaStream_t s, int num_sms, const MlpTcArgs& a);

}  // namespace phx
