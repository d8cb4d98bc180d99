// Shared device helpers of the phoebe_gpu library (complex FP64 arithmetic,
// grid phases, small utilities).  Only the CUDA library includes this file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/phoebe_gpu.h"

namespace phx {

// Physical constants (CODATA 2018 derived).
constexpr double kBoltzmannEV = 8.617333262e-5;            // eV/K
constexpr double kHbarOmegaEV = 0.06465415130134121;       // hbar*sqrt(eV/(A^2 amu)) / eV
constexpr double kHbar2AmuEvA2 = 0.004180159280496722;     // hbar^2/(amu eV A^2)
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kCoulombEVA = 14.399645478425668;  // e^2 / (4 pi eps0), eV A

constexpr int kMaxNw = 32;      // Wannier functions
constexpr int kMaxModes = 30;   // 3 * atoms (10 atoms)

// ------------------------------------------------------------------ complex FP64
struct cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
__host__ __device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// acc += a*b
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a)*b
__host__ __device__ __forceinline__ void cfma_conja(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }

// Lets `kernel` take as much dynamic shared memory as the device allows beside its static shared
// memory.  The limit is one value per kernel for the whole process: setting each launch's own size
// would let host threads that launch the same kernel with different sizes (concurrent planning of a
// batch) lower it under one another's launches.  One value for every caller removes that race; how
// much shared memory a block gets is still the launch's own size.
template <typename K>
inline cudaError_t allow_dynamic_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

__device__ __forceinline__ cplx ldc(const cplx* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// ------------------------------------------------------------------ grids
// Gamma-centred grid n[3]; point index (i1*N2 + i2)*N3 + i3 (z fastest).
struct Grid {
  int n[3];
  int64_t size() const { return (int64_t)n[0] * n[1] * n[2]; }
};

__host__ __device__ __forceinline__ void grid_coords(int64_t idx, const int n[3], int c[3]) {
  c[2] = (int)(idx % n[2]);
  int64_t t = idx / n[2];
  c[1] = (int)(t % n[1]);
  c[0] = (int)(t / n[1]);
}

__host__ __device__ __forceinline__ int64_t grid_flat(const int c[3], const int n[3]) {
  return ((int64_t)c[0] * n[1] + c[1]) * n[2] + c[2];
}

// Exact phase index of k.R on a grid: k_i = j_i / N_i, so k.R = r / L with
// L = lcm(N1,N2,N3) and r = sum_i j_i n_i (L/N_i) mod L.
__host__ __device__ __forceinline__ int phase_index(const int j[3], const int R[3], const int mult[3], int L) {
  int64_t r = (int64_t)j[0] * R[0] * mult[0] + (int64_t)j[1] * R[1] * mult[1] +
              (int64_t)j[2] * R[2] * mult[2];
  int64_t m = r % L;
  if (m < 0) m += L;
  return (int)m;
}

}  // namespace phx
