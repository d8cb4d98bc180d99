// Three-phonon coupling (Sec. 3.1, Eq. 3PhCouplingInterpolation) on a q grid and the three-phonon
// part of the diagonal of the phonon scattering matrix A (Sec. 4.3):
//   V3(q nu, q' nu', q'' nu'') = sum_{R R'} w e^{-i(q.R + q'.R')} Phi3(s a R, s' b R', s'' c 0)
//                                conj(Z_q[s a,nu]) conj(Z_q'[s' b,nu']) conj(Z_q''[s'' c,nu'']),
//   A_{q nu} = (2 pi / N_q) sum_{q~ nu' nu''} |W|^2 [n n' (n''+1) d(w + w' - w'')
//                                                   + (1/2) n (n'+1)(n''+1) d(w - w' - w'')],
// W = V3(q nu, q~ nu', -(q + q~) nu''), Z the mode factors of Eq. 7.  The same two-stage form as
// the el-ph couplings: stage 1 sums over R and the first mode at fixed q (FP64, stored FP32),
// stage 2 sums over R' for every q~ of the grid, applies the other two modes and the delta weights
// (FP32, partial sums of non-negative terms, FP64 atomics per (q, nu)).  On the grid the phase of
// the R' sum factorises per axis, e^{-2 pi i q~.R'} = Ex[jx][rx] Ey[jy][ry] Ez[jz][rz] with
// r = R' mod N, so stage 2 forms, per (jx, jy) line of q~, XY[rz] = sum over the R' of each rz of
// Ex Ey A[R'] once, and each q~ of the line sums over the rz residues only.
#include <algorithm>
#include <vector>

#include "pipeline.h"

namespace phx {

struct Ph3S1Args {
  const double* phi;   // [n][nm][nm*nm] pairs sorted by R' index
  const int* R;        // [n][3]
  const double* w;     // [n]
  const int* off;      // [NRp+1] pairs of each R'
  const cplx* Zq;      // [Q][nm][nm]
  float2* A;           // [Q][NRp][nm][nm*nm]
  int64_t Q;
  int NRp, nm, N[3];
};

// A[q][r'][nu][c] = sum_{pairs p of R' r'} w_p e^{-2 pi i q.R_p} sum_{s a} Phi3[p][s a][c] conj(Z_q[s a][nu]);
// thread per (q, r', nu, c), exact integer reduction of the phase.
__global__ void k_ph3_stage1(Ph3S1Args a) {
  const int nm = a.nm, nc = nm * nm;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.Q * a.NRp * nm * nc) return;
  const int c = (int)(t % nc);
  const int nu = (int)((t / nc) % nm);
  const int r = (int)((t / ((int64_t)nc * nm)) % a.NRp);
  const int64_t q = t / ((int64_t)nc * nm * a.NRp);
  const int j[3] = {(int)(q / ((int64_t)a.N[1] * a.N[2])), (int)((q / a.N[2]) % a.N[1]), (int)(q % a.N[2])};
  double re = 0.0, im = 0.0;
  for (int p = a.off[r]; p < a.off[r + 1]; ++p) {
    double frac = 0.0;  // q.R mod 1 from integer residues
    for (int d = 0; d < 3; ++d) {
      const int m = (int)((((int64_t)j[d] * a.R[3 * p + d]) % a.N[d] + a.N[d]) % a.N[d]);
      frac += (double)m / a.N[d];
    }
    double sn, cs;
    sincospi(-2.0 * frac, &sn, &cs);
    double sr = 0.0, si = 0.0;  // sum_{s a} Phi3 conj(Z)
    for (int sa = 0; sa < nm; ++sa) {
      const double ph = a.phi[((int64_t)p * nm + sa) * nc + c];
      const cplx z = a.Zq[(q * nm + sa) * nm + nu];
      sr += ph * z.re;
      si -= ph * z.im;
    }
    const double wr = a.w[p];
    re += wr * (cs * sr - sn * si);
    im += wr * (cs * si + sn * sr);
  }
  a.A[t] = make_float2((float)re, (float)im);
}

struct Ph3S2Args {
  const float2* A;     // [Q][NRp][nm][nm*nm]
  const float2* Ex;    // [N0][Bx] e^{-2 pi i jx rx / N0} of the R' residues along x (likewise y, z)
  const float2* Ey;    // [N1][By]
  const float2* Ez;    // [N2][Bz]
  const int4* rres;    // [NRp] (x, y, z) residue indices of each R'
  const int* zr_off;   // [Bz+1] R' of each z residue in zr_list
  const int* zr_list;  // [NRp] the R' grouped by z residue
  const float2* Zf;    // [Q][nm][nm]
  const float2* onb;   // [Q][nm] (hbar w, n), hbar w < 0 for dead modes
  int64_t Q;
  int NRp, N[3], Bx, By, Bz;
  int L, Zc;           // (jx, jy) lines of q~ per block and jz per block (L Zc <= 32)
  float inv_sigma, cut2;
  double scale;        // 2 pi / (N_q sqrt(pi) sigma)
  double* acc;         // [Q][nm]
};

// One block per (L consecutive (jx, jy) lines of q~, chunk of Zc jz, q); thread (q~ of the block, nu).  The q row of
// stage 1 is staged in shared memory; the block forms XY[line][rz][nu][c] = sum over the R' of each
// rz residue of Ex Ey A[R'][nu][c], then each thread sums B[s' b][s'' c] = sum_rz Ez XY, rotates by
// the two other modes and adds the coalescence and decay weights of every (nu', nu'').
template <int NM>
__global__ void __launch_bounds__(32 * NM) k_ph3_stage2(Ph3S2Args a) {
  constexpr int NC = NM * NM;
  extern __shared__ __align__(16) unsigned char smem[];
  const int N2 = a.N[2], L = a.L, Bz = a.Bz, Zc = a.Zc;
  const int nzc = (N2 + Zc - 1) / Zc;
  float2* As = reinterpret_cast<float2*>(smem);        // [NRp][NM][NC]
  float2* XY = As + (size_t)a.NRp * NM * NC;           // [L][Bz][NM][NC]
  float2* pxy = XY + (size_t)L * Bz * NM * NC;         // [L][NRp] Ex Ey of each line and R'
  const int T = L * Zc;                                  // q~ per block
  float2* Zs1 = pxy + (size_t)L * a.NRp;                 // [T][NC] Z of each q~ of the block
  float2* Zs2 = Zs1 + (size_t)T * NC;                    // [T][NC] Z of its -q''
  float2* ons = Zs2 + (size_t)T * NC;                    // [T][3][NM] (hbar w, n) at q~, q'', -q''
  __shared__ float red[NM];
  const int64_t q = blockIdx.y;
  const int line0 = (blockIdx.x / nzc) * L;             // line = jx N1 + jy
  const int jz0 = (blockIdx.x % nzc) * Zc;
  const int nlines = min(L, a.N[0] * a.N[1] - line0);
  const float2* Ag = a.A + q * a.NRp * NM * NC;
  // q~ of tile position t (line l, jz), q'' = q + q~ and -q'' on the grid; false past the grid
  const int jq[3] = {(int)(q / ((int64_t)a.N[1] * a.N[2])), (int)((q / a.N[2]) % a.N[1]), (int)(q % a.N[2])};
  auto tile_q = [&](int t, int64_t& tq, int64_t& i2, int64_t& im) -> bool {
    const int l = t / Zc, jz = jz0 + t - l * Zc;
    if (l >= nlines || jz >= N2) return false;
    const int line = line0 + l, jx = line / a.N[1], jy = line - jx * a.N[1];
    tq = (int64_t)line * N2 + jz;
    const int jt[3] = {jx, jy, jz};
    int j2[3], jm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      j2[d] = (jq[d] + jt[d]) % a.N[d];
      jm[d] = (a.N[d] - j2[d]) % a.N[d];
    }
    i2 = ((int64_t)j2[0] * a.N[1] + j2[1]) * a.N[2] + j2[2];
    im = ((int64_t)jm[0] * a.N[1] + jm[1]) * a.N[2] + jm[2];
    return true;
  };
  for (int i = threadIdx.x; i < a.NRp * NM * NC; i += blockDim.x) As[i] = Ag[i];
  for (int i = threadIdx.x; i < T * NC; i += blockDim.x) {
    int64_t tq, i2, im;
    const int t = i / NC, e = i - t * NC;
    if (tile_q(t, tq, i2, im)) {
      Zs1[i] = a.Zf[tq * NC + e];
      Zs2[i] = a.Zf[im * NC + e];
    }
  }
  for (int i = threadIdx.x; i < T * NM; i += blockDim.x) {
    int64_t tq, i2, im;
    const int t = i / NM, v = i - t * NM;
    if (tile_q(t, tq, i2, im)) {
      ons[(t * 3) * NM + v] = a.onb[tq * NM + v];
      ons[(t * 3 + 1) * NM + v] = a.onb[i2 * NM + v];
      ons[(t * 3 + 2) * NM + v] = a.onb[im * NM + v];
    }
  }
  for (int i = threadIdx.x; i < nlines * a.NRp; i += blockDim.x) {
    const int l = i / a.NRp, r = i - l * a.NRp;
    const int line = line0 + l, jx = line / a.N[1], jy = line - jx * a.N[1];
    const int4 ri = a.rres[r];
    const float2 ex = a.Ex[jx * a.Bx + ri.x], ey = a.Ey[jy * a.By + ri.y];
    pxy[i] = make_float2(ex.x * ey.x - ex.y * ey.y, ex.x * ey.y + ex.y * ey.x);
  }
  if (threadIdx.x < NM) red[threadIdx.x] = 0.f;
  __syncthreads();
  {  // XY of every line of the block: the R' of each z residue with their Ex Ey
    const int per_line = Bz * NM * NC;
    for (int o = threadIdx.x; o < nlines * per_line; o += blockDim.x) {
      const int l = o / per_line, rem = o - l * per_line;
      const int b = rem / (NM * NC), e = rem - b * (NM * NC);
      float2 s = make_float2(0.f, 0.f);
      for (int i = a.zr_off[b]; i < a.zr_off[b + 1]; ++i) {
        const int r = a.zr_list[i];
        const float2 p = pxy[l * a.NRp + r], v = As[(size_t)r * NM * NC + e];
        s.x = fmaf(p.x, v.x, fmaf(-p.y, v.y, s.x));
        s.y = fmaf(p.x, v.y, fmaf(p.y, v.x, s.y));
      }
      XY[o] = s;
    }
  }
  __syncthreads();
  const int lt = threadIdx.x / NM, nu = threadIdx.x % NM;
  const int l = lt / Zc, jz = jz0 + lt - l * Zc;
  float acc = 0.f;  // every term is non-negative
  const float2 on0 = a.onb[q * NM + nu];
  if (l < nlines && jz < N2 && on0.x >= 0.f) {
    float2 B[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) B[c] = make_float2(0.f, 0.f);
    for (int b = 0; b < Bz; ++b) {
      const float2 p = a.Ez[jz * Bz + b];
      const float2* xr = XY + ((size_t)(l * Bz + b) * NM + nu) * NC;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 v = xr[c];
        B[c].x = fmaf(p.x, v.x, fmaf(-p.y, v.y, B[c].x));
        B[c].y = fmaf(p.x, v.y, fmaf(p.y, v.x, B[c].y));
      }
    }
    // the q~, q'' and -q'' tables staged above
    const float2* Z1 = Zs1 + (size_t)lt * NC;
    const float2* Z2 = Zs2 + (size_t)lt * NC;
    const float2* o1 = ons + (size_t)(lt * 3) * NM;
    for (int n1 = 0; n1 < NM; ++n1) {
      const float2 on1 = o1[n1];
      if (on1.x < 0.f) continue;
      float2 tt[NM];  // sum_{s' b} B[s' b][s'' c] conj(Z_q~[s' b][nu'])
#pragma unroll
      for (int k = 0; k < NM; ++k) tt[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < NM; ++b) {
        const float2 z = Z1[b * NM + n1];
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          const float2 v = B[b * NM + k];
          tt[k].x = fmaf(v.x, z.x, fmaf(v.y, z.y, tt[k].x));
          tt[k].y = fmaf(v.y, z.x, fmaf(-v.x, z.y, tt[k].y));
        }
      }
      for (int n2 = 0; n2 < NM; ++n2) {
        const float2 on2 = o1[NM + n2];
        if (on2.x < 0.f || o1[2 * NM + n2].x < 0.f) continue;
        float2 W = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          const float2 z = Z2[k * NM + n2];
          W.x = fmaf(tt[k].x, z.x, fmaf(tt[k].y, z.y, W.x));
          W.y = fmaf(tt[k].y, z.x, fmaf(-tt[k].x, z.y, W.y));
        }
        const float x1 = (on0.x + on1.x - on2.x) * a.inv_sigma;
        const float x2 = (on0.x - on1.x - on2.x) * a.inv_sigma;
        float wt = 0.f;
        if (x1 * x1 < a.cut2) wt += on0.y * on1.y * (on2.y + 1.f) * expf(-x1 * x1);
        if (x2 * x2 < a.cut2) wt += 0.5f * on0.y * (on1.y + 1.f) * (on2.y + 1.f) * expf(-x2 * x2);
        acc = fmaf(W.x * W.x + W.y * W.y, wt, acc);
      }
    }
  }
  if (acc != 0.f) atomicAdd(&red[nu], acc);
  __syncthreads();
  if (threadIdx.x < NM && red[threadIdx.x] != 0.f)
    atomicAdd(a.acc + q * NM + threadIdx.x, (double)red[threadIdx.x] * a.scale);
}

// Mode factors and (hbar w, n) as FP32 tables; dead modes get hbar w = -1.
__global__ void k_ph3_tables(const cplx* __restrict__ Zq, const double* __restrict__ om, const double* __restrict__ nB,
                             int64_t Q, int nm, double omega_cut, float2* __restrict__ Zf, float2* __restrict__ onb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < Q * nm * nm) Zf[t] = make_float2((float)Zq[t].re, (float)Zq[t].im);
  if (t < Q * nm) onb[t] = om[t] >= omega_cut ? make_float2((float)om[t], (float)nB[t]) : make_float2(-1.f, 0.f);
}

// Average over the modes degenerate within tol at the same q.
__global__ void k_ph3_degenerate(const double* __restrict__ acc, const double* __restrict__ om, int64_t Q, int nm,
                                 double tol, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Q * nm) return;
  const int64_t q = t / nm;
  const int nu = (int)(t % nm);
  double s = 0.0;
  int c = 0;
  for (int u = 0; u < nm; ++u)
    if (fabs(om[q * nm + u] - om[q * nm + nu]) < tol) {
      s += acc[q * nm + u];
      ++c;
    }
  out[t] = s / c;
}

template <int NM>
static int launch_s2(cudaStream_t st, const Ph3S2Args& a) {
  const size_t T = (size_t)a.L * a.Zc;
  const size_t smem = sizeof(float2) * ((size_t)a.NRp * NM * NM * NM + (size_t)a.L * a.Bz * NM * NM * NM +
                                        (size_t)a.L * a.NRp + 2 * T * NM * NM + 3 * T * NM);
  if (smem > 227 * 1024) return -2;
  if (allow_dynamic_smem(k_ph3_stage2<NM>) != cudaSuccess)
    return -1;
  const int lines = a.N[0] * a.N[1], nzc = (a.N[2] + a.Zc - 1) / a.Zc;
  dim3 grid((unsigned)((lines + a.L - 1) / a.L * nzc), (unsigned)a.Q);
  k_ph3_stage2<NM><<<grid, a.L * a.Zc * NM, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int three_phonon(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, double* out_host) {
  const int nm = 3 * c->na;
  const int N[3] = {p->nq[0], p->nq[1], p->nq[2]};
  const int64_t Q = (int64_t)N[0] * N[1] * N[2];
  if (Q > 65535) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the three-phonon path takes q grids of at most 65535 points");
  int st;
  c->stats = phoebe_gpu_stats{};
  c->launches = 0;
  Timer total;
  total.begin(c);
  double *omega, *nB;
  cplx* Zq;
  TRY(phonon_modes(c, N, nullptr, Q, p->T_K, p->omega_cut_eV, &omega, &nB, &Zq, "ph3q"));
  float2* Zf = (float2*)ensure(c, "ph3_Zf", sizeof(float2) * Q * nm * nm, &st);
  if (!Zf) return st;
  float2* onb = (float2*)ensure(c, "ph3_onb", sizeof(float2) * Q * nm, &st);
  if (!onb) return st;
  k_ph3_tables<<<(unsigned)((Q * nm * nm + 255) / 256), 256, 0, c->stream>>>(Zq, omega, nB, Q, nm, p->omega_cut_eV, Zf,
                                                                               onb);
  const int NRp = c->ph3_nrp;
  // the R' residues r = R' mod N per axis, each R''s residue indices, and the per-axis phase tables
  // e^{-2 pi i j r / N} (j r reduced modulo N in integers)
  std::vector<int> res[3];
  std::vector<int> rres((size_t)4 * NRp, 0);
  for (int d = 0; d < 3; ++d) {
    for (int r = 0; r < NRp; ++r) res[d].push_back(((c->ph3_rp[3 * r + d] % N[d]) + N[d]) % N[d]);
    std::sort(res[d].begin(), res[d].end());
    res[d].erase(std::unique(res[d].begin(), res[d].end()), res[d].end());
    for (int r = 0; r < NRp; ++r) {
      const int v = ((c->ph3_rp[3 * r + d] % N[d]) + N[d]) % N[d];
      rres[4 * r + d] = (int)(std::lower_bound(res[d].begin(), res[d].end(), v) - res[d].begin());
    }
  }
  void* d_tab[3];
  for (int d = 0; d < 3; ++d) {
    const int B = (int)res[d].size();
    std::vector<float2> tab((size_t)N[d] * B);
    for (int j = 0; j < N[d]; ++j)
      for (int b = 0; b < B; ++b) {
        const int64_t m = ((int64_t)j * res[d][b]) % N[d];
        double sn, cs;
        sincospi(-2.0 * (double)m / N[d], &sn, &cs);
        tab[(size_t)j * B + b] = make_float2((float)cs, (float)sn);
      }
    const char* name[3] = {"ph3_Ex", "ph3_Ey", "ph3_Ez"};
    TRY(upload(c, name[d], tab.data(), sizeof(float2) * tab.size(), &d_tab[d]));
  }
  std::vector<int> zr((size_t)res[2].size() + 1 + NRp, 0);  // offsets by z residue, then the R'
  for (int r = 0; r < NRp; ++r) ++zr[rres[4 * r + 2] + 1];
  for (size_t b = 1; b <= res[2].size(); ++b) zr[b] += zr[b - 1];
  {
    std::vector<int> fill(zr.begin(), zr.begin() + res[2].size());
    for (int r = 0; r < NRp; ++r) zr[res[2].size() + 1 + fill[rres[4 * r + 2]]++] = r;
  }
  void *d_rres, *d_zr;
  TRY(upload(c, "ph3_rres", rres.data(), sizeof(int) * rres.size(), &d_rres));
  TRY(upload(c, "ph3_zr", zr.data(), sizeof(int) * zr.size(), &d_zr));
  const int Zc = std::min(N[2], 32), L = std::max(1, 32 / Zc);  // L Zc <= 32 q~ per block
  float2* A = (float2*)ensure(c, "ph3_A", sizeof(float2) * Q * NRp * nm * nm * nm, &st);
  if (!A) return st;
  Ph3S1Args s1;
  s1.phi = (const double*)c->bufs["ph3_phi"].p;
  s1.R = (const int*)c->bufs["ph3_R"].p;
  s1.w = (const double*)c->bufs["ph3_w"].p;
  s1.off = (const int*)c->bufs["ph3_off"].p;
  s1.Zq = Zq;
  s1.A = A;
  s1.Q = Q;
  s1.NRp = NRp;
  s1.nm = nm;
  for (int d = 0; d < 3; ++d) s1.N[d] = N[d];
  const int64_t n1 = Q * NRp * nm * nm * nm;
  k_ph3_stage1<<<(unsigned)((n1 + 255) / 256), 256, 0, c->stream>>>(s1);
  double* acc = (double*)ensure(c, "ph3_acc", sizeof(double) * Q * nm, &st);
  if (!acc) return st;
  double* out = (double*)ensure(c, "ph3_out", sizeof(double) * Q * nm, &st);
  if (!out) return st;
  CK(c, cudaMemsetAsync(acc, 0, sizeof(double) * Q * nm, c->stream));
  c->launches += 3;
  CK(c, cudaGetLastError());
  Ph3S2Args s2;
  s2.A = A;
  s2.Ex = (const float2*)d_tab[0];
  s2.Ey = (const float2*)d_tab[1];
  s2.Ez = (const float2*)d_tab[2];
  s2.rres = (const int4*)d_rres;
  s2.zr_off = (const int*)d_zr;
  s2.zr_list = (const int*)d_zr + res[2].size() + 1;
  s2.Bx = (int)res[0].size();
  s2.By = (int)res[1].size();
  s2.Bz = (int)res[2].size();
  s2.L = L;
  s2.Zc = Zc;
  s2.Zf = Zf;
  s2.onb = onb;
  s2.Q = Q;
  s2.NRp = NRp;
  for (int d = 0; d < 3; ++d) s2.N[d] = N[d];
  s2.inv_sigma = (float)(1.0 / p->sigma_eV);
  s2.cut2 = (float)(p->delta_cut_sigmas * p->delta_cut_sigmas);
  s2.scale = 2.0 * kPi / ((double)Q * kSqrtPi * p->sigma_eV);
  s2.acc = acc;
  Timer t2;
  t2.begin(c);
  const int r = nm == 6 ? launch_s2<6>(c->stream, s2) : nm == 3 ? launch_s2<3>(c->stream, s2) : -3;
  if (r == -3) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "the three-phonon path is built for one or two atoms");
  if (r == -2) return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "too many distinct R' for the stage-2 tile");
  if (r != 0) {
    cudaGetLastError();
    return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the three-phonon stage 2 failed");
  }
  t2.end(c, &c->stats.stage2_ms);
  k_ph3_degenerate<<<(unsigned)((Q * nm + 255) / 256), 256, 0, c->stream>>>(acc, omega, Q, nm, p->degen_tol_eV, out);
  c->launches += 2;
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(out_host, out, sizeof(double) * Q * nm, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->stats.stage2_launches = 1;
  c->stats.kernel_launches = c->launches;
  c->stats.n_q = Q;
  // per q: the XY sums of every (jx, jy) line (one complex MAC per R' and element), then per (q~, nu)
  // the rz sum and the two mode rotations
  c->stats.stage2_flops = 8.0 * (double)Q *
                          ((double)N[0] * N[1] * NRp * nm * nm * nm +
                           (double)Q * nm * ((double)s2.Bz * nm * nm + 2.0 * nm * nm * nm));
  total.end(c, &c->stats.total_ms);
  return PHOEBE_GPU_OK;
}

}  // namespace phx
