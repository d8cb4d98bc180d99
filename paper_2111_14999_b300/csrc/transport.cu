// RTA transport coefficients from the linewidths (Sec. 4.2 charge and energy fluxes J, Q and
// the Onsager coefficients; Sec. 4.3.2 relaxation-time approximation):
//   L_n[a][b] = 1/(N_k V) sum_kb tau v_a v_b (eps - mu)^n (-df/deps),   tau = hbar / Gamma,
//   sigma = e^2 L_0,  S = -(1/(e T)) L_0^{-1} L_1,  kappa_el = (1/T)(L_2 - L_1 L_0^{-1} L_1),
// with hbar v the k-derivative of Eq. 10 (Sec. 3.3) in Cartesian axes.
#include <math.h>

#include "pipeline.h"

namespace phx {

constexpr double kHbarEvS = 6.582119569e-16;  // hbar, eV s
constexpr double kECharge = 1.602176634e-19;  // elementary charge, C

// One block per active state: hbar v (eV A, Cartesian) from -sum_R w_R R_cart Im(e^{ik.R} u^dag H(R) u),
// then its terms of L_0, L_1, L_2 (SI) added into L[3][3][3].
__global__ void k_transport_terms(const int* __restrict__ st_k, const int* __restrict__ st_b,
                                  const double* __restrict__ gamma, GridMap gm, GridPhase gf,
                                  const cplx* __restrict__ cis_f, const cplx* __restrict__ H,
                                  const int* __restrict__ RH, const double* __restrict__ wH, int nR, int nw,
                                  const double* __restrict__ epsF, const cplx* __restrict__ UF, double mu,
                                  double T, double3 a0, double3 a1, double3 a2, double inv_nkv,
                                  double* __restrict__ L) {
  __shared__ cplx u[kMaxNw];
  __shared__ double red[3][32];
  const int s = blockIdx.x;
  const double G = gamma[s];
  if (!(G > 0.0)) return;  // uniform over the block: no scattering partner, no lifetime
  const int64_t f = gm.k_to_fine(st_k[s]);
  const int b = st_b[s];
  int fc[3];
  grid_coords(f, gm.nf, fc);
  for (int m = threadIdx.x; m < nw; m += blockDim.x) u[m] = UF[(f * nw + m) * nw + b];
  __syncthreads();
  double v[3] = {0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < nR; r += blockDim.x) {
    const int Rv[3] = {RH[3 * r], RH[3 * r + 1], RH[3 * r + 2]};
    const cplx ph = cis_f[phase_index(fc, Rv, gf.mult, gf.L)];
    const cplx* h = H + (int64_t)r * nw * nw;
    cplx sr = {0.0, 0.0};
    for (int n = 0; n < nw; ++n) {
      cplx hu = {0.0, 0.0};
      for (int m = 0; m < nw; ++m) cfma(hu, h[n * nw + m], u[m]);
      cfma_conja(sr, u[n], hu);
    }
    const double e = -wH[r] * cmul(ph, sr).im;
    const double rc[3] = {Rv[0] * a0.x + Rv[1] * a1.x + Rv[2] * a2.x, Rv[0] * a0.y + Rv[1] * a1.y + Rv[2] * a2.y,
                          Rv[0] * a0.z + Rv[1] * a1.z + Rv[2] * a2.z};
    for (int i = 0; i < 3; ++i) v[i] += e * rc[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = 0; i < 3; ++i) {
    double x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[i][w] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double vs[3];
  for (int i = 0; i < 3; ++i) {
    double x = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) x += red[i][j];
    vs[i] = x * 1e-10 / kHbarEvS;  // (eV A) / (eV s) -> m/s
  }
  const double eps = epsF[f * nw + b];
  const double kT = kBoltzmannEV * T;
  const double fd = 1.0 / (exp((eps - mu) / kT) + 1.0);
  const double mdf = fd * (1.0 - fd) / kT / kECharge;  // -df/deps in 1/J
  const double tau = kHbarEvS / G;
  const double de = (eps - mu) * kECharge;
  double wn = tau * mdf * inv_nkv;
  for (int n = 0; n < 3; ++n, wn *= de)
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y < 3; ++y) atomicAdd(L + n * 9 + x * 3 + y, wn * vs[x] * vs[y]);
}

// sigma, S, kappa from L (one thread; 3x3 inverse by cofactors).
__global__ void k_transport_finish(const double* __restrict__ L, double T, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* L0 = L;
  const double* L1 = L + 9;
  const double* L2 = L + 18;
  double inv[9];
  const double det = L0[0] * (L0[4] * L0[8] - L0[5] * L0[7]) - L0[1] * (L0[3] * L0[8] - L0[5] * L0[6]) +
                     L0[2] * (L0[3] * L0[7] - L0[4] * L0[6]);
  inv[0] = (L0[4] * L0[8] - L0[5] * L0[7]) / det;
  inv[1] = (L0[2] * L0[7] - L0[1] * L0[8]) / det;
  inv[2] = (L0[1] * L0[5] - L0[2] * L0[4]) / det;
  inv[3] = (L0[5] * L0[6] - L0[3] * L0[8]) / det;
  inv[4] = (L0[0] * L0[8] - L0[2] * L0[6]) / det;
  inv[5] = (L0[2] * L0[3] - L0[0] * L0[5]) / det;
  inv[6] = (L0[3] * L0[7] - L0[4] * L0[6]) / det;
  inv[7] = (L0[1] * L0[6] - L0[0] * L0[7]) / det;
  inv[8] = (L0[0] * L0[4] - L0[1] * L0[3]) / det;
  double* sigma = out;
  double* seebeck = out + 9;
  double* kappa = out + 18;
  for (int i = 0; i < 9; ++i) sigma[i] = kECharge * kECharge * L0[i];
  double iL1[9];  // L0^{-1} L1
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double x = 0.0;
      for (int k = 0; k < 3; ++k) x += inv[i * 3 + k] * L1[k * 3 + j];
      iL1[i * 3 + j] = x;
      seebeck[i * 3 + j] = -x / (kECharge * T);
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double x = 0.0;
      for (int k = 0; k < 3; ++k) x += L1[i * 3 + k] * iL1[k * 3 + j];
      kappa[i * 3 + j] = (L2[i * 3 + j] - x) / T;
    }
}

}  // namespace phx

using namespace phx;

extern "C" int phoebe_gpu_transport_rta(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const double lattice[9],
                                        double sigma[9], double seebeck[9], double kappa[9]) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!p || !lattice || !sigma || !seebeck || !kappa) return fail(c, PHOEBE_GPU_ERR_ARG, "transport_rta: NULL argument");
  const double vol = fabs(lattice[0] * (lattice[4] * lattice[8] - lattice[5] * lattice[7]) -
                          lattice[1] * (lattice[3] * lattice[8] - lattice[5] * lattice[6]) +
                          lattice[2] * (lattice[3] * lattice[7] - lattice[4] * lattice[6]));
  if (!(vol > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "transport_rta: the lattice vectors are degenerate");
  int n = 0;
  TRY(linewidths(c, p, &n, nullptr, nullptr, nullptr, false));
  int st;
  const int nn = n > 0 ? n : 1;
  double* g = (double*)ensure(c, "trp_gamma", sizeof(double) * nn, &st);
  if (!g) return st;
  int* kd = (int*)ensure(c, "trp_k", sizeof(int) * nn, &st);
  if (!kd) return st;
  int* bd = (int*)ensure(c, "trp_b", sizeof(int) * nn, &st);
  if (!bd) return st;
  double* L = (double*)ensure(c, "trp_L", sizeof(double) * 27, &st);
  if (!L) return st;
  double* out = (double*)ensure(c, "trp_out", sizeof(double) * 27, &st);
  if (!out) return st;
  int cap = n;
  TRY(linewidths(c, p, &cap, kd, bd, g, true));
  GridMap gm;
  for (int i = 0; i < 3; ++i) {
    gm.nk[i] = p->nk[i];
    gm.nq[i] = p->nq[i];
    gm.nf[i] = p->nk[i] > p->nq[i] ? p->nk[i] : p->nq[i];
    gm.sk[i] = gm.nf[i] / p->nk[i];
    gm.sq[i] = gm.nf[i] / p->nq[i];
  }
  GridPhase gf = make_phase(gm.nf);
  cplx* cis_f;
  TRY(cis_table(c, gf, "cis_el", &cis_f));
  CK(c, cudaMemsetAsync(L, 0, sizeof(double) * 27, c->stream));
  const double nkv = (double)p->nk[0] * p->nk[1] * p->nk[2] * vol * 1e-30;
  if (n > 0) {
    k_transport_terms<<<n, 128, 0, c->stream>>>(
        kd, bd, g, gm, gf, cis_f, (const cplx*)c->bufs["H"].p, (const int*)c->bufs["RH"].p,
        (const double*)c->bufs["wH"].p, c->nRH, c->nw, (const double*)c->bufs["epsF"].p,
        (const cplx*)c->bufs["UF"].p, p->mu_eV, p->T_K, make_double3(lattice[0], lattice[1], lattice[2]),
        make_double3(lattice[3], lattice[4], lattice[5]), make_double3(lattice[6], lattice[7], lattice[8]),
        1.0 / nkv, L);
  }
  k_transport_finish<<<1, 32, 0, c->stream>>>(L, p->T_K, out);
  c->launches += 2;
  CK(c, cudaGetLastError());
  double h[27];
  CK(c, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 9; ++i) {
    sigma[i] = h[i];
    seebeck[i] = h[9 + i];
    kappa[i] = h[18 + i];
  }
  return PHOEBE_GPU_OK;
}
