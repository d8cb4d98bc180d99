// Stage 2 on grid q points as a separable DFT over the R_p box (dft.cu).
#pragma once

#include "kernels.cuh"

namespace phx {

#ifndef PHX_DFT_LINES
#define PHX_DFT_LINES 4
#endif
#ifndef PHX_DFT_MINB
#define PHX_DFT_MINB 1
#endif
constexpr int kDftLines = PHX_DFT_LINES;  // (jy, jz) lines per block of the x-sum kernel
constexpr int kDftMaxThreads = 512;   // Nx * kDftLines <= 512 (Nx <= 64)

struct DftYzArgs {
  const float2* T;       // [S][nR][E] stage-1 output (E = 3na * nw, column c = sa*nw + m)
  const float* w;        // [nR] R_p weights
  int nR, E;
  int Bx, By, Bz;        // residues of R_p mod N per axis
  int Ny, Nz;
  const int* plane_off;  // [Bx+1] entries of each rx residue
  int ne_max;            // most entries of one rx residue
  const int* ent_ay;     // per entry (sorted by rx residue, then ry residue): ry residue index
  const int* ent_az;     //   rz residue index
  const int* ent_r;      //   R_p index
  const float2* Ey;      // [Ny][By] e^{2 pi i jy ry / Ny}
  const float2* Ez;      // [Nz][Bz]
  float2* Y;             // [S][Bx][Ny][Nz][E]
};

struct DftXArgs {
  const float2* Y;
  int Bx, Nx, Ny, Nz;
  const float2* Ex;      // [Nx][Bx]
  const int* st_k;       // [S]
  const int* st_b;       // [S]
  const double* epsF;    // [NF][nw]
  GridMap gm;
  const float2* eps2;    // [NF][nw] (hi, lo)
  const float* f32;      // [NF][nw]
  const float2* UH;      // [NF][nw][nw] conj(U[m][m'])
  const float2* Zf;      // [Nq][nm][nm]
  const float* omf;      // [Nq][nm]
  const float* nBf;      // [Nq][nm]
  float reach, inv_sigma, cut2;
  double scale;          // (2 pi / N_q) / (sqrt(pi) sigma)
  double* gamma;
  int64_t s_base;
};

// Launches both kernels for S states; -1 on a launch error, -2 for a (nw, 3na) without a kernel.
int dft_launch(cudaStream_t st, const DftYzArgs& yz, const DftXArgs& x, int S, int nw, int nm);
size_t dft_smem_bytes(int Bx, int E, int threads, int nw, int Nx);
size_t dft_yz_smem_bytes(int ne_max, int Ny, int By, int Nz, int Bz);
int dft_table(cudaStream_t st, const int* res, int B, int N, float2* E);

}  // namespace phx
