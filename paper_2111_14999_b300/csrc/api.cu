// C ABI of the phoebe_gpu library: context, input upload, argument checks and
// the orchestration of the linewidth path.  Declarations and the contract of
// every entry point are in include/phoebe_gpu.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "pipeline.h"

using namespace phx;

// ------------------------------------------------------------------ errors
int phx::fail(phoebe_gpu_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int phx::cuda_fail(phoebe_gpu_ctx* c, cudaError_t e, const char* what, int line) {
  return fail(c, PHOEBE_GPU_ERR_CUDA, "CUDA error in %s (line %d): %s", what, line, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ device memory
void* phx::ensure(phoebe_gpu_ctx* c, const char* name, size_t bytes, int* status) {
  *status = PHOEBE_GPU_OK;
  DBuf& b = c->bufs[name];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.p;
  if (b.p) {
    cudaFree(b.p);
    c->mem_used -= (int64_t)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  if (c->mem_cap > 0 && c->mem_used + (int64_t)bytes > c->mem_cap) {
    *status = fail(c, PHOEBE_GPU_ERR_NOMEM, "buffer '%s' of %zu bytes exceeds the memory cap (%lld used of %lld)",
                   name, bytes, (long long)c->mem_used, (long long)c->mem_cap);
    return nullptr;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *status = fail(c, PHOEBE_GPU_ERR_NOMEM, "cudaMalloc of %zu bytes for '%s' failed: %s", bytes, name,
                   cudaGetErrorString(e));
    return nullptr;
  }
  b.p = p;
  b.bytes = bytes;
  c->mem_used += (int64_t)bytes;
  return p;
}

void phx::release(phoebe_gpu_ctx* c, const char* name) {
  auto it = c->bufs.find(name);
  if (it == c->bufs.end()) return;
  if (it->second.p) {
    cudaFree(it->second.p);
    c->mem_used -= (int64_t)it->second.bytes;
  }
  c->bufs.erase(it);
}

int phx::upload(phoebe_gpu_ctx* c, const char* name, const void* host, size_t bytes, void** dev) {
  int st;
  void* p = ensure(c, name, bytes, &st);
  if (!p) return st;
  CK(c, cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  *dev = p;
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ timing
void phx::Timer::begin(phoebe_gpu_ctx* c) {
  if (!c->profiling) return;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, c->stream);
  on = true;
}
void phx::Timer::end(phoebe_gpu_ctx* c, double* acc) {
  if (!on) return;
  cudaEventRecord(b, c->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  *acc += ms;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  on = false;
}

// ------------------------------------------------------------------ grid helpers
static int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }
static int lcm_i(int a, int b) { return a / gcd_i(a, b) * b; }

GridPhase phx::make_phase(const int n[3]) {
  GridPhase g;
  int L = lcm_i(lcm_i(n[0], n[1]), n[2]);
  for (int i = 0; i < 3; ++i) {
    g.n[i] = n[i];
    g.mult[i] = L / n[i];
  }
  g.L = L;
  return g;
}

int phx::cis_table(phoebe_gpu_ctx* c, const GridPhase& gp, const char* name, cplx** out) {
  int st;
  cplx* p = (cplx*)ensure(c, name, sizeof(cplx) * gp.L, &st);
  if (!p) return st;
  k_cis_table<<<(gp.L + 255) / 256, 256, 0, c->stream>>>(p, gp.L);
  c->launches++;
  CK(c, cudaGetLastError());
  *out = p;
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ band structures
// out[e][p] = sum_R w_R e^{2 pi i k_p.R} in[R][e] on the grid n, evaluated separably over the
// residue box of the R set (k_sep_* in bands.cu).
static int fourier_grid_sep(phoebe_gpu_ctx* c, const cplx* in, const int* R_dev, const double* w_dev, int nR, int E,
                            const int n[3], cplx* out) {
  std::vector<int> R((size_t)3 * nR);
  CK(c, cudaMemcpyAsync(R.data(), R_dev, sizeof(int) * 3 * nR, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  std::vector<int> res[3], idx((size_t)3 * nR);
  for (int d = 0; d < 3; ++d) {
    std::vector<int> r(nR);
    for (int i = 0; i < nR; ++i) r[i] = ((R[3 * i + d] % n[d]) + n[d]) % n[d];
    res[d] = r;
    std::sort(res[d].begin(), res[d].end());
    res[d].erase(std::unique(res[d].begin(), res[d].end()), res[d].end());
    for (int i = 0; i < nR; ++i)
      idx[3 * i + d] = (int)(std::lower_bound(res[d].begin(), res[d].end(), r[i]) - res[d].begin());
  }
  const int B0 = (int)res[0].size(), B1 = (int)res[1].size(), B2 = (int)res[2].size();
  std::vector<int> order(nR);
  for (int i = 0; i < nR; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    for (int d = 0; d < 3; ++d)
      if (idx[3 * a + d] != idx[3 * b + d]) return idx[3 * a + d] < idx[3 * b + d];
    return a < b;
  });
  std::vector<int> plane_off(B0 + 1, 0), pair_off, pair_b, ent_c(nR), ent_r(nR);
  for (int e = 0; e < nR; ++e) {
    const int r = order[e];
    ent_c[e] = idx[3 * r + 2];
    ent_r[e] = r;
    if (e == 0 || idx[3 * r] != idx[3 * order[e - 1]] || idx[3 * r + 1] != idx[3 * order[e - 1] + 1]) {
      pair_off.push_back(e);
      pair_b.push_back(idx[3 * r + 1]);
    }
    plane_off[idx[3 * r] + 1] = (int)pair_off.size();
  }
  const int npair = (int)pair_b.size();
  pair_off.push_back(nR);
  for (int a = 1; a <= B0; ++a) plane_off[a] = std::max(plane_off[a], plane_off[a - 1]);
  int st;
  void *d_res0, *d_res1, *d_res2, *d_po, *d_pb, *d_plo, *d_ec, *d_er;
  TRY(upload(c, "sep_res0", res[0].data(), sizeof(int) * B0, &d_res0));
  TRY(upload(c, "sep_res1", res[1].data(), sizeof(int) * B1, &d_res1));
  TRY(upload(c, "sep_res2", res[2].data(), sizeof(int) * B2, &d_res2));
  TRY(upload(c, "sep_pair_off", pair_off.data(), sizeof(int) * (npair + 1), &d_po));
  TRY(upload(c, "sep_pair_b", pair_b.data(), sizeof(int) * npair, &d_pb));
  TRY(upload(c, "sep_plane_off", plane_off.data(), sizeof(int) * (B0 + 1), &d_plo));
  TRY(upload(c, "sep_ent_c", ent_c.data(), sizeof(int) * nR, &d_ec));
  TRY(upload(c, "sep_ent_r", ent_r.data(), sizeof(int) * nR, &d_er));
  cplx* E0 = (cplx*)ensure(c, "sep_E0", sizeof(cplx) * n[0] * B0, &st);
  if (!E0) return st;
  cplx* E1 = (cplx*)ensure(c, "sep_E1", sizeof(cplx) * n[1] * B1, &st);
  if (!E1) return st;
  cplx* E2 = (cplx*)ensure(c, "sep_E2", sizeof(cplx) * n[2] * B2, &st);
  if (!E2) return st;
  const int64_t nz = (int64_t)npair * E * n[2], ny = (int64_t)B0 * E * n[1] * n[2];
  const int64_t nx = (int64_t)E * n[0] * n[1] * n[2];
  cplx* Zs = (cplx*)ensure(c, "sep_Zs", sizeof(cplx) * nz, &st);
  if (!Zs) return st;
  cplx* Y = (cplx*)ensure(c, "sep_Y", sizeof(cplx) * ny, &st);
  if (!Y) return st;
  k_sep_table<<<(n[0] * B0 + 127) / 128, 128, 0, c->stream>>>((const int*)d_res0, B0, n[0], E0);
  k_sep_table<<<(n[1] * B1 + 127) / 128, 128, 0, c->stream>>>((const int*)d_res1, B1, n[1], E1);
  k_sep_table<<<(n[2] * B2 + 127) / 128, 128, 0, c->stream>>>((const int*)d_res2, B2, n[2], E2);
  k_sep_z<<<(unsigned)((nz + 255) / 256), 256, 0, c->stream>>>(in, w_dev, E, npair, (const int*)d_po,
                                                                (const int*)d_ec, (const int*)d_er, E2, n[2], B2, Zs);
  k_sep_y<<<(unsigned)((ny + 255) / 256), 256, 0, c->stream>>>(Zs, E, B0, (const int*)d_plo, (const int*)d_pb, E1,
                                                                n[1], B1, n[2], Y);
  k_sep_x<<<(unsigned)((nx + 255) / 256), 256, 0, c->stream>>>(Y, E, B0, E0, n[0], n[1], n[2], out);
  c->launches += 6;
  CK(c, cudaGetLastError());
  return PHOEBE_GPU_OK;
}

// hbar v [P][nw] (eV A, Cartesian, FP32 (vx, vy, vz, 0)) on the grid n from its eigenvectors U.
int phx::velocity_grid(phoebe_gpu_ctx* c, const int n[3], const cplx* U, float4** vel_out) {
  if (!c->have_lattice) return fail(c, PHOEBE_GPU_ERR_ORDER, "band velocities need set_lattice first");
  const int64_t P = (int64_t)n[0] * n[1] * n[2];
  const int nw = c->nw, E = nw * nw, nR = c->nRH;
  int st;
  cplx* in = (cplx*)ensure(c, "vel_in", sizeof(cplx) * (size_t)nR * 3 * E, &st);
  if (!in) return st;
  cplx* dH = (cplx*)ensure(c, "vel_dH", sizeof(cplx) * (size_t)3 * E * P, &st);
  if (!dH) return st;
  float4* vel = (float4*)ensure(c, "vel_grid", sizeof(float4) * (size_t)P * nw, &st);
  if (!vel) return st;
  Lat9 lat;
  for (int i = 0; i < 9; ++i) lat.a[i] = c->lattice[i];
  const int64_t ni = (int64_t)nR * 3 * E;
  k_vel_input<<<(unsigned)((ni + 255) / 256), 256, 0, c->stream>>>((const cplx*)c->bufs["H"].p,
                                                                     (const int*)c->bufs["RH"].p, lat, nR, E, in);
  c->launches++;
  CK(c, cudaGetLastError());
  TRY(fourier_grid_sep(c, in, (const int*)c->bufs["RH"].p, (const double*)c->bufs["wH"].p, nR, 3 * E, n, dH));
  k_band_velocity<<<(unsigned)((P * nw + 127) / 128), 128, 0, c->stream>>>(dH, U, P, nw, vel);
  c->launches++;
  CK(c, cudaGetLastError());
  *vel_out = vel;
  return PHOEBE_GPU_OK;
}

// eps[P][nw], U[P][nw][nw] (columns = eigenvectors) on the grid n.
int phx::electron_grid(phoebe_gpu_ctx* c, const int n[3], double** eps, cplx** U) {
  int64_t P = (int64_t)n[0] * n[1] * n[2];
  int nw = c->nw, E = nw * nw, st;
  cplx* A = (cplx*)ensure(c, "jac_A", sizeof(cplx) * P * E, &st);
  if (!A) return st;
  cplx* V = (cplx*)ensure(c, "jac_V", sizeof(cplx) * P * E, &st);
  if (!V) return st;
  double* e = (double*)ensure(c, "epsF", sizeof(double) * P * nw, &st);
  if (!e) return st;
  cplx* u = (cplx*)ensure(c, "UF", sizeof(cplx) * P * E, &st);
  if (!u) return st;
  int* status = (int*)ensure(c, "status", 64, &st);
  if (!status) return st;
  CK(c, cudaMemsetAsync(status, 0, 64, c->stream));
  TRY(fourier_grid_sep(c, (const cplx*)c->bufs["H"].p, (const int*)c->bufs["RH"].p,
                       (const double*)c->bufs["wH"].p, c->nRH, E, n, A));
  if (eigh_launch(c->stream, A, V, nw, P, e, u, status)) return fail(c, PHOEBE_GPU_ERR_CUDA, "eigensolver launch failed");
  c->launches += 1;
  int hs = 0;
  CK(c, cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (hs) return fail(c, PHOEBE_GPU_ERR_NOTCONVERGED, "eigensolve of H(k) did not converge in %d QR steps", 30 * nw);
  *eps = e;
  *U = u;
  return PHOEBE_GPU_OK;
}

// omega, nB [Q][nm], Z [Q][nm][nm] on the grid n (or at explicit points qpts_dev if non-NULL).
int phx::phonon_modes(phoebe_gpu_ctx* c, const int n[3], const double* qpts_dev, int64_t Q, double T,
                      double omega_cut, double** omega, double** nB, cplx** Z, const char* tag) {
  GridPhase gp = make_phase(n);
  int nm = 3 * c->na, E = nm * nm, st;
  cplx* cis = nullptr;
  if (!qpts_dev)
    if ((st = cis_table(c, gp, "cis_ph", &cis))) return st;
  std::string t(tag);
  cplx* A = (cplx*)ensure(c, (t + "_jA").c_str(), sizeof(cplx) * Q * E, &st);
  if (!A) return st;
  cplx* V = (cplx*)ensure(c, (t + "_jV").c_str(), sizeof(cplx) * Q * E, &st);
  if (!V) return st;
  double* lam = (double*)ensure(c, (t + "_lam").c_str(), sizeof(double) * Q * nm, &st);
  if (!lam) return st;
  cplx* z = (cplx*)ensure(c, (t + "_z").c_str(), sizeof(cplx) * Q * E, &st);
  if (!z) return st;
  double* om = (double*)ensure(c, (t + "_omega").c_str(), sizeof(double) * Q * nm, &st);
  if (!om) return st;
  double* nb = (double*)ensure(c, (t + "_nB").c_str(), sizeof(double) * Q * nm, &st);
  if (!nb) return st;
  cplx* Zq = (cplx*)ensure(c, (t + "_Z").c_str(), sizeof(cplx) * Q * E, &st);
  if (!Zq) return st;
  int* status = (int*)ensure(c, "status", 64, &st);
  if (!status) return st;
  CK(c, cudaMemsetAsync(status, 0, 64, c->stream));
  dim3 g((unsigned)((Q + 127) / 128), (unsigned)E);
  k_dynmat_grid<<<g, 128, 0, c->stream>>>((const double*)c->bufs["Phi"].p, (const int*)c->bufs["Rf"].p,
                                            (const double*)c->bufs["wf"].p, c->nRf, nm,
                                            (const double*)c->bufs["inv_sqrt_m"].p, gp, cis, qpts_dev, Q, A);
  if (eigh_launch(c->stream, A, V, nm, Q, lam, z, status)) return fail(c, PHOEBE_GPU_ERR_CUDA, "eigensolver launch failed");
  k_phonon_factors<<<(unsigned)((Q * nm + 127) / 128), 128, 0, c->stream>>>(
      lam, z, nm, Q, (const double*)c->bufs["mass_of_row"].p, T, omega_cut, om, nb, Zq);
  c->launches += 3;
  CK(c, cudaGetLastError());
  int hs = 0;
  CK(c, cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (hs) return fail(c, PHOEBE_GPU_ERR_NOTCONVERGED, "eigensolve of D(q) did not converge in %d QR steps", 30 * nm);
  *omega = om;
  *nB = nb;
  *Z = Zq;
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* phoebe_gpu_version(void) { return "phoebe_gpu 0.1 (sm_103a)"; }

void phoebe_gpu_constants(double out[3]) {
  if (!out) return;
  out[0] = kBoltzmannEV;
  out[1] = kHbarOmegaEV;
  out[2] = kHbar2AmuEvA2;
}

void phoebe_gpu_rta_params_default(phoebe_gpu_rta_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  for (int i = 0; i < 3; ++i) p->nk[i] = p->nq[i] = 8;
  p->T_K = 300.0;
  p->sigma_eV = 0.05;
  p->delta_cut_sigmas = 6.0;
  p->omega_cut_eV = 1e-4;
  p->degen_tol_eV = 1e-6;
  p->precision = PHOEBE_PREC_FP64;
  p->sampler = PHOEBE_SAMPLER_FULL;
  p->sample_fraction = 0.05;
  p->mix_alpha = 0.1;
  p->sigma_min_eV = 1e-3;
}

int phoebe_gpu_set_force_constants3(phoebe_gpu_ctx* c, int n, const int32_t* R, const int32_t* Rp, const double* w,
                                    const double* Phi3) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (!c->have_Phi) return fail(c, PHOEBE_GPU_ERR_ORDER, "set_force_constants3 needs set_force_constants first");
  if (n <= 0 || !R || !Rp || !Phi3) return fail(c, PHOEBE_GPU_ERR_ARG, "n, R, Rp and Phi3 are required");
  const int nm = 3 * c->na;
  const int64_t blk = (int64_t)nm * nm * nm;
  std::map<std::array<int, 3>, int> rp_index;  // distinct R', sorted
  for (int i = 0; i < n; ++i) rp_index[{Rp[3 * i], Rp[3 * i + 1], Rp[3 * i + 2]}] = 0;
  int k = 0;
  std::vector<int> rpd;
  for (auto& kv : rp_index) {
    kv.second = k++;
    rpd.insert(rpd.end(), kv.first.begin(), kv.first.end());
  }
  const int NRp = k;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto rpi = [&](int i) { return rp_index[{Rp[3 * i], Rp[3 * i + 1], Rp[3 * i + 2]}]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rpi(a) < rpi(b); });
  std::vector<int> Rs((size_t)3 * n), off(NRp + 1, 0);
  std::vector<double> ws(n), phs((size_t)n * blk);
  for (int i = 0; i < n; ++i) {
    const int o = order[i];
    for (int d = 0; d < 3; ++d) Rs[3 * i + d] = R[3 * o + d];
    ws[i] = w ? w[o] : 1.0;
    for (int64_t e = 0; e < blk; ++e) phs[(size_t)i * blk + e] = Phi3[(size_t)o * blk + e];
    off[rpi(o) + 1] = i + 1;
  }
  for (int r = 1; r <= NRp; ++r) off[r] = std::max(off[r], off[r - 1]);
  void* d;
  int st;
  if ((st = upload(c, "ph3_R", Rs.data(), sizeof(int) * 3 * n, &d))) return st;
  if ((st = upload(c, "ph3_w", ws.data(), sizeof(double) * n, &d))) return st;
  if ((st = upload(c, "ph3_phi", phs.data(), sizeof(double) * n * blk, &d))) return st;
  if ((st = upload(c, "ph3_off", off.data(), sizeof(int) * (NRp + 1), &d))) return st;
  if ((st = upload(c, "ph3_Rpd", rpd.data(), sizeof(int) * 3 * NRp, &d))) return st;
  c->ph3_nrp = NRp;
  c->ph3_rp = rpd;
  c->ph3_na = c->na;
  c->have_phi3 = true;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_three_phonon_rates(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int64_t n_values, double* A_eV) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (!p || !A_eV) return fail(c, PHOEBE_GPU_ERR_ARG, "params or A_eV is NULL");
  if (!c->have_phi3 || c->ph3_na != c->na)
    return fail(c, PHOEBE_GPU_ERR_ORDER, "three_phonon_rates needs set_force_constants3 for the current atoms");
  for (int i = 0; i < 3; ++i)
    if (p->nq[i] < 1 || p->nq[i] > 4096) return fail(c, PHOEBE_GPU_ERR_ARG, "grid sizes must be in 1..4096");
  if (!(p->T_K > 0.0) || !(p->sigma_eV > 0.0) || !(p->delta_cut_sigmas > 0.0) || !(p->omega_cut_eV >= 0.0) ||
      !(p->degen_tol_eV >= 0.0))
    return fail(c, PHOEBE_GPU_ERR_ARG, "T_K, sigma_eV, delta_cut_sigmas must be > 0, omega_cut and degen_tol >= 0");
  const int64_t Q = (int64_t)p->nq[0] * p->nq[1] * p->nq[2];
  if (n_values != Q * 3 * c->na)
    return fail(c, PHOEBE_GPU_ERR_ARG, "A needs N_q * 3 n_at = %lld values", (long long)(Q * 3 * c->na));
  return three_phonon(c, p, A_eV);
}

int phoebe_gpu_set_polar(phoebe_gpu_ctx* c, const double* Zstar, const double* eps_inf, double alpha) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!Zstar) {
    c->have_polar = false;
    return PHOEBE_GPU_OK;
  }
  if (!c->have_Phi) return fail(c, PHOEBE_GPU_ERR_ORDER, "set_polar needs set_force_constants first");
  if (!eps_inf || !(alpha > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "eps_inf must be given and alpha > 0");
  const double* e = eps_inf;
  const double det = e[0] * (e[4] * e[8] - e[5] * e[7]) - e[1] * (e[3] * e[8] - e[5] * e[6]) +
                     e[2] * (e[3] * e[7] - e[4] * e[6]);
  const double m2 = e[0] * e[4] - e[1] * e[3];
  if (!(e[0] > 0.0 && m2 > 0.0 && det > 0.0) || fabs(e[1] - e[3]) > 1e-12 || fabs(e[2] - e[6]) > 1e-12 ||
      fabs(e[5] - e[7]) > 1e-12)
    return fail(c, PHOEBE_GPU_ERR_ARG, "eps_inf must be symmetric positive definite");
  c->zstar.assign(Zstar, Zstar + 9 * c->na);
  for (int i = 0; i < 9; ++i) c->eps_inf[i] = e[i];
  c->polar_alpha = alpha;
  c->have_polar = true;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_set_lattice(phoebe_gpu_ctx* c, const double* lattice) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!lattice) return fail(c, PHOEBE_GPU_ERR_ARG, "lattice is NULL");
  const double* A = lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(fabs(det) > 1e-12)) return fail(c, PHOEBE_GPU_ERR_ARG, "lattice vectors are singular");
  for (int i = 0; i < 9; ++i) c->lattice[i] = A[i];
  c->have_lattice = true;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_create(phoebe_gpu_ctx** out, int device, void* cuda_stream) {
  if (!out) return PHOEBE_GPU_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return PHOEBE_GPU_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return PHOEBE_GPU_ERR_CUDA;
  phoebe_gpu_ctx* c = new phoebe_gpu_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return PHOEBE_GPU_ERR_CUDA;
    }
    c->own_stream = true;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  c->cc = major * 10 + minor;
  *out = c;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_destroy(phoebe_gpu_ctx* c) {
  if (!c) return PHOEBE_GPU_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  c->bufs.clear();
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  destroy_tc_state(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return PHOEBE_GPU_OK;
}

const char* phoebe_gpu_last_error(const phoebe_gpu_ctx* c) { return c ? c->err.c_str() : "no context"; }

int phoebe_gpu_set_profiling(phoebe_gpu_ctx* c, int on) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  c->profiling = on != 0;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_get_stats(const phoebe_gpu_ctx* c, phoebe_gpu_stats* out) {
  if (!c || !out) return PHOEBE_GPU_ERR_ARG;
  *out = c->stats;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_set_memory_cap(phoebe_gpu_ctx* c, int64_t bytes) {
  if (!c || bytes < 0) return PHOEBE_GPU_ERR_ARG;
  c->mem_cap = bytes;
  return PHOEBE_GPU_OK;
}

static bool closed_under_minus(int n, const int32_t* R, std::vector<int>* minus) {
  std::map<std::tuple<int, int, int>, int> idx;
  for (int i = 0; i < n; ++i) idx[std::make_tuple(R[3 * i], R[3 * i + 1], R[3 * i + 2])] = i;
  if (minus) minus->assign(n, -1);
  for (int i = 0; i < n; ++i) {
    auto it = idx.find(std::make_tuple(-R[3 * i], -R[3 * i + 1], -R[3 * i + 2]));
    if (it == idx.end()) return false;
    if (minus) (*minus)[i] = it->second;
  }
  return true;
}

static std::vector<double> weights_or_ones(int n, const double* w) {
  std::vector<double> v(n, 1.0);
  if (w) v.assign(w, w + n);
  return v;
}

int phoebe_gpu_set_hamiltonian(phoebe_gpu_ctx* c, int nw, int n_R, const int32_t* R, const double* w,
                               const double* H) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (nw < 1 || nw > kMaxNw) return fail(c, PHOEBE_GPU_ERR_ARG, "nw=%d outside 1..%d", nw, kMaxNw);
  if (n_R < 1 || !R || !H) return fail(c, PHOEBE_GPU_ERR_ARG, "set_hamiltonian: n_R < 1 or NULL array");
  std::vector<int> minus;
  if (!closed_under_minus(n_R, R, &minus))
    return fail(c, PHOEBE_GPU_ERR_ARG, "set_hamiltonian: the R set is not closed under -R");
  std::vector<double> wv = weights_or_ones(n_R, w);
  double hmax = 0.0, herr = 0.0;
  for (int r = 0; r < n_R; ++r) {
    int rm = minus[r];
    if (fabs(wv[r] - wv[rm]) > 1e-12) return fail(c, PHOEBE_GPU_ERR_ARG, "set_hamiltonian: w(R) != w(-R)");
    for (int i = 0; i < nw; ++i)
      for (int j = 0; j < nw; ++j) {
        const double* a = H + 2 * (((int64_t)r * nw + i) * nw + j);
        const double* b = H + 2 * (((int64_t)rm * nw + j) * nw + i);
        hmax = fmax(hmax, fabs(a[0]) + fabs(a[1]));
        herr = fmax(herr, fabs(a[0] - b[0]) + fabs(a[1] + b[1]));
      }
  }
  if (herr > 1e-10 * fmax(hmax, 1e-300))
    return fail(c, PHOEBE_GPU_ERR_ARG, "set_hamiltonian: H(-R) != H(R)^dagger (max deviation %g)", herr);
  void* d;
  int st;
  if ((st = upload(c, "RH", R, sizeof(int32_t) * 3 * n_R, &d))) return st;
  if ((st = upload(c, "wH", wv.data(), sizeof(double) * n_R, &d))) return st;
  if ((st = upload(c, "H", H, sizeof(double) * 2 * (size_t)n_R * nw * nw, &d))) return st;
  if (c->have_g && c->nw != nw) c->have_g = false;  // stale couplings of another size
  c->nw = nw;
  c->nRH = n_R;
  c->have_H = true;
  c->tc_g_valid = false;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_set_force_constants(phoebe_gpu_ctx* c, int na, const double* mass_amu, int n_R,
                                   const int32_t* R, const double* w, const double* Phi) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (na < 1 || 3 * na > kMaxModes) return fail(c, PHOEBE_GPU_ERR_ARG, "na=%d outside 1..%d", na, kMaxModes / 3);
  if (!mass_amu || n_R < 1 || !R || !Phi) return fail(c, PHOEBE_GPU_ERR_ARG, "set_force_constants: bad arguments");
  for (int i = 0; i < na; ++i)
    if (!(mass_amu[i] > 0.0)) return fail(c, PHOEBE_GPU_ERR_ARG, "set_force_constants: mass[%d] <= 0", i);
  if (!closed_under_minus(n_R, R, nullptr))
    return fail(c, PHOEBE_GPU_ERR_ARG, "set_force_constants: the R set is not closed under -R");
  std::vector<double> wv = weights_or_ones(n_R, w);
  std::vector<double> inv(3 * na), mrow(3 * na);
  for (int i = 0; i < 3 * na; ++i) {
    mrow[i] = mass_amu[i / 3];
    inv[i] = 1.0 / sqrt(mass_amu[i / 3]);
  }
  void* d;
  int st;
  int nm = 3 * na;
  if ((st = upload(c, "Rf", R, sizeof(int32_t) * 3 * n_R, &d))) return st;
  if ((st = upload(c, "wf", wv.data(), sizeof(double) * n_R, &d))) return st;
  if ((st = upload(c, "Phi", Phi, sizeof(double) * (size_t)n_R * nm * nm, &d))) return st;
  if ((st = upload(c, "inv_sqrt_m", inv.data(), sizeof(double) * nm, &d))) return st;
  if ((st = upload(c, "mass_of_row", mrow.data(), sizeof(double) * nm, &d))) return st;
  if (c->have_g && c->na != na) c->have_g = false;
  c->na = na;
  c->nRf = n_R;
  c->have_Phi = true;
  c->tc_g_valid = false;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_set_elph_wannier(phoebe_gpu_ctx* c, int n_Re, const int32_t* Re, const double* we, int n_Rp,
                                const int32_t* Rp, const double* wp, const double* g) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (!c->have_H || !c->have_Phi)
    return fail(c, PHOEBE_GPU_ERR_ORDER, "set_elph_wannier needs set_hamiltonian and set_force_constants first");
  if (n_Re < 1 || n_Rp < 1 || !Re || !Rp || !g) return fail(c, PHOEBE_GPU_ERR_ARG, "set_elph_wannier: bad arguments");
  std::vector<double> wev = weights_or_ones(n_Re, we), wpv = weights_or_ones(n_Rp, wp);
  void* d;
  int st;
  size_t gbytes = sizeof(double) * 2 * (size_t)n_Re * n_Rp * c->nw * c->nw * 3 * c->na;
  if ((st = upload(c, "Re", Re, sizeof(int32_t) * 3 * n_Re, &d))) return st;
  if ((st = upload(c, "we", wev.data(), sizeof(double) * n_Re, &d))) return st;
  if ((st = upload(c, "Rp", Rp, sizeof(int32_t) * 3 * n_Rp, &d))) return st;
  if ((st = upload(c, "wp", wpv.data(), sizeof(double) * n_Rp, &d))) return st;
  if ((st = upload(c, "g", g, gbytes, &d))) return st;
  c->nRe = n_Re;
  c->nRp = n_Rp;
  c->we_max = 0.0;
  c->wp_max = 0.0;
  for (double v : wev) c->we_max = fmax(c->we_max, fabs(v));
  for (double v : wpv) c->wp_max = fmax(c->wp_max, fabs(v));
  c->g_nw = c->nw;
  c->g_na = c->na;
  c->have_g = true;
  c->tc_g_valid = false;
  return PHOEBE_GPU_OK;
}

int phoebe_gpu_interpolate_couplings(phoebe_gpu_ctx* c, int n_pairs, const double* k, const double* q,
                                     int precision, double* g2, double* eps_k, double* eps_kq, double* omega_q) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  return interpolate_pairs(c, n_pairs, k, q, precision, g2, eps_k, eps_kq, omega_q);
}

int phoebe_gpu_linewidths_rta(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int* n_states, int32_t* k_index,
                              int32_t* band, double* gamma_eV) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  return linewidths(c, p, n_states, k_index, band, gamma_eV, false);
}

int phoebe_gpu_linewidths_rta_dev(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int* n_states,
                                  int32_t* k_index_dev, int32_t* band_dev, double* gamma_dev) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  return linewidths(c, p, n_states, k_index_dev, band_dev, gamma_dev, true);
}

int phoebe_gpu_phonon_rates_elph(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, int64_t n_values,
                                 double* P_eV) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  cudaSetDevice(c->device);
  if (!p || !P_eV) return fail(c, PHOEBE_GPU_ERR_ARG, "params or P_eV is NULL");
  if (p->precision != PHOEBE_PREC_FP32_DFT)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "phonon-electron rates are evaluated by the grid-DFT stage 2 (precision 7)");
  if (p->sampler != PHOEBE_SAMPLER_FULL)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "phonon-electron rates need the full q sum");
  if (p->nq[0] <= 0 || p->nq[1] <= 0 || p->nq[2] <= 0 || p->nk[0] <= 0 || p->nk[1] <= 0 || p->nk[2] <= 0)
    return fail(c, PHOEBE_GPU_ERR_ARG, "grid sizes must be positive");
  if (!c->have_H || !c->have_Phi || !c->have_g)
    return fail(c, PHOEBE_GPU_ERR_ORDER, "phonon_rates_elph needs all three set_* calls first");
  const int64_t Nq = (int64_t)p->nq[0] * p->nq[1] * p->nq[2];
  const int nm = 3 * c->na;
  if (n_values != Nq * nm)
    return fail(c, PHOEBE_GPU_ERR_ARG, "P needs N_q * 3 n_at = %lld values, got %lld", (long long)(Nq * nm),
                (long long)n_values);
  int st;
  double* acc = (double*)ensure(c, "prate_acc", sizeof(double) * Nq * nm, &st);
  if (!acc) return st;
  double* out = (double*)ensure(c, "prate_out", sizeof(double) * Nq * nm, &st);
  if (!out) return st;
  const int64_t cap = (int64_t)p->nk[0] * p->nk[1] * p->nk[2] * c->nw;  // every (k, band) at most
  if (cap > INT32_MAX) return fail(c, PHOEBE_GPU_ERR_ARG, "k grid too large");
  int32_t* kd = (int32_t*)ensure(c, "prate_k", sizeof(int32_t) * cap, &st);
  if (!kd) return st;
  int32_t* bd = (int32_t*)ensure(c, "prate_b", sizeof(int32_t) * cap, &st);
  if (!bd) return st;
  double* gd = (double*)ensure(c, "prate_g", sizeof(double) * cap, &st);
  if (!gd) return st;
  CK(c, cudaMemsetAsync(acc, 0, sizeof(double) * Nq * nm, c->stream));
  CK(c, cudaMemsetAsync(out, 0, sizeof(double) * Nq * nm, c->stream));
  c->prate_acc = acc;
  c->prate_out = out;
  int n = (int)cap;
  st = linewidths(c, p, &n, kd, bd, gd, true);
  c->prate_acc = nullptr;
  c->prate_out = nullptr;
  if (st) return st;
  CK(c, cudaMemcpyAsync(P_eV, out, sizeof(double) * Nq * nm, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

}  // extern "C"
