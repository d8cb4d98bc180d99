// Stage 1 on grid k points as a separable DFT over the R_e box (Sec. 5.5 Eq. 71, its R_e sum
// evaluated exactly in another order).  With k = (kx/Nx, ky/Ny, kz/Nz) on the k grid,
//   X_k[c] = sum_Re w_e e^{2 pi i k.R_e} g(R_e)[c]
//          = sum_rz Ez[kz][rz] sum_ry Ey[ky][ry] sum_rx Ex[kx][rx] w g(rx, ry, rz)[c],
// r = R_e mod N per axis.  One block per (kx plane of the batch, chunk of element columns): the
// rx sum into W1[(ry, rz) pair] (g streamed once per plane), then per ky line of the plane the
// ry sum into W2(rz) by the y groups {r, -r} (the rows of a group replaced by their sum and
// difference once per plane, as for z below), then the rz sum for every k of the batch on that
// line by the z groups {r, -r}:
// with P = W2(r) + W2(-r), M = W2(r) - W2(-r) and Ez = c + i s, Ez(r) W2(r) + Ez(-r) W2(-r) =
// c P + i s M; the k (kz) and (-kz) of one line share A = sum c P and B = sum i s M, X = A +- B.
// X rows are written in the layout the tensor-core GEMM writes (unscaled).
// FP32 on the CUDA cores.
#include <stdint.h>

#include "dft.h"

namespace phx {

// GZ <= 8: exactly GZ z groups; GZ = 16: up to 16.  Element columns and X row strides below 2^31.
template <int GZ>
__global__ void __launch_bounds__(256) k_s1_dft(S1Args a) {
  constexpr int CW = kS1Cols, TPC = 256 / CW;  // threads per column
  constexpr bool EX = GZ <= 8;
  extern __shared__ __align__(16) unsigned char smem[];
  const int Pe = a.Pe, nRe = a.nRe, G = EX ? GZ : a.Gz, By = a.By;
  const int C32 = (int)a.C, ldx32 = (int)a.ldx;
  float2* W1 = reinterpret_cast<float2*>(smem);          // [Pe][CW]
  float2* exw = W1 + (size_t)Pe * CW;                    // [nRe] w Ex[kx][rx] per entry
  float2* Eyk = exw + nRe;                               // [nky][By]
  float2* Ezg = Eyk + (size_t)a.nky * By;                // [nkz][G]
  int2* zg = reinterpret_cast<int2*>(Ezg + (size_t)a.nkz * G);  // [G]
  int* peo = reinterpret_cast<int*>(zg + G);             // [Pe+1]
  int* erow = peo + Pe + 1;                              // [nRe]
  int2* yg = reinterpret_cast<int2*>(erow + nRe + ((Pe + 1 + nRe) & 1));  // [Gy] (pair, partner pair), 8-byte aligned
  int* yay = reinterpret_cast<int*>(yg + a.Gy);         // [Gy]
  int* rzg = yay + a.Gy;                                 // [Bz+1]
  int* line_ctr = rzg + a.Bz + 1;                        // [CW / 32] lines taken per column half
  const int pl = blockIdx.y, kx = a.plane_kx[pl];
  const int64_t c0 = (int64_t)blockIdx.x * CW;
  const int col = threadIdx.x % CW, t4 = threadIdx.x / CW;
  const bool live = c0 + col < a.C;
  const float2* gcol = a.g + c0 + col;  // this column of g and of the X rows
  float* Xcol = a.X + 2 * (c0 + col);
  for (int i = threadIdx.x; i < nRe; i += blockDim.x) {
    const float2 e = a.Ex[kx * a.Bx + a.ent_ax[i]];
    const float w = a.ent_w[i];
    exw[i] = make_float2(w * e.x, w * e.y);
    erow[i] = a.ent_row[i];
  }
  for (int i = threadIdx.x; i < a.nky * By; i += blockDim.x) Eyk[i] = a.Ey[i];
  for (int i = threadIdx.x; i < a.nkz * G; i += blockDim.x) Ezg[i] = a.Ezg[i];
  for (int i = threadIdx.x; i < G; i += blockDim.x) zg[i] = a.zgrp[i];
  for (int i = threadIdx.x; i <= Pe; i += blockDim.x) peo[i] = a.pair_ent_off[i];
  for (int i = threadIdx.x; i < a.Gy; i += blockDim.x) {
    yg[i] = a.ygrp[i];
    yay[i] = a.ygrp_ay[i];
  }
  for (int i = threadIdx.x; i <= a.Bz; i += blockDim.x) rzg[i] = a.rz_grp_off[i];
  for (int i = threadIdx.x; i < CW / 32; i += blockDim.x) line_ctr[i] = 0;
  for (int i = threadIdx.x; i < Pe * CW; i += blockDim.x) W1[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // rx sum: W1[p][col] = sum over the entries of pair p of w Ex g.  Each of the TPC threads of a
  // column takes a contiguous chunk of the entries (sorted by pair) with 8 loads in flight, and adds
  // its running pair sum into W1 when the pair changes (pairs split between chunks get two adds).
  {
    constexpr int U = 8;
    const int per = (nRe + TPC - 1) / TPC;
    const int e0 = t4 * per, e1 = min(nRe, e0 + per);
    int p = 0;
    while (p + 1 < Pe && peo[p + 1] <= e0) ++p;
    int pend = peo[p + 1];  // first entry past pair p
    float2 acc = make_float2(0.f, 0.f);
    for (int eb = e0; eb < e1; eb += U) {
      float2 gv[U];
#pragma unroll
      for (int i = 0; i < U; ++i)
        gv[i] = (live && eb + i < e1) ? __ldg(gcol + (int64_t)erow[eb + i] * C32) : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = eb + i;
        if (e >= e1) break;
        if (e >= pend) {  // next pair: flush the running sum
          atomicAdd(&W1[p * CW + col].x, acc.x);
          atomicAdd(&W1[p * CW + col].y, acc.y);
          acc = make_float2(0.f, 0.f);
          while (e >= peo[p + 1]) ++p;
          pend = peo[p + 1];
        }
        const float2 x = exw[e];
        acc.x = fmaf(x.x, gv[i].x, fmaf(-x.y, gv[i].y, acc.x));
        acc.y = fmaf(x.x, gv[i].y, fmaf(x.y, gv[i].x, acc.y));
      }
    }
    if (e1 > e0) {
      atomicAdd(&W1[p * CW + col].x, acc.x);
      atomicAdd(&W1[p * CW + col].y, acc.y);
    }
  }
  __syncthreads();
  // the rows of each y group {r, -r}: W1(r), W1(-r) -> P = W1(r) + W1(-r), M = W1(r) - W1(-r)
  for (int gi = t4; gi < a.Gy; gi += TPC) {
    const int2 pp = yg[gi];
    if (pp.y != pp.x) {
      const float2 u = W1[pp.x * CW + col], v = W1[pp.y * CW + col];
      W1[pp.x * CW + col] = make_float2(u.x + v.x, u.y + v.y);
      W1[pp.y * CW + col] = make_float2(u.x - v.x, u.y - v.y);
    }
  }
  __syncthreads();
  // Per ky line of the plane: the ry sums W2(rz) and the rz sums for the batch's k on the line.  A
  // warp takes whole lines from its column half's counter; every value it needs after the rx sum is
  // its own column's, so no barrier follows.  With Ez = c + i s, a z group {r, -r} adds
  // c P + i s M with P = W2(r) + W2(-r), M = W2(r) - W2(-r); W2(r) sums over the y groups of rz = r
  // as in the rx rows (c P' + i s M' with the group's Ey = c + i s).
  const int lb = a.plane_line_off[pl], le = a.plane_line_off[pl + 1];
  int* lctr = line_ctr + (threadIdx.x >> 5) % (CW / 32);  // this warp's column half
  auto ry_sum = [&](const float2* ey, int r) {
    float2 w = make_float2(0.f, 0.f);
    const int g1 = rzg[r + 1];
    for (int gi = rzg[r]; gi < g1; ++gi) {
      const int2 pp = yg[gi];
      const float2 e = ey[yay[gi]], v = W1[pp.x * CW + col], m = W1[pp.y * CW + col];
      w.x = fmaf(e.x, v.x, fmaf(-e.y, m.y, w.x));
      w.y = fmaf(e.x, v.y, fmaf(e.y, m.x, w.y));
    }
    return w;
  };
  for (;;) {
    int li = 0;
    if ((threadIdx.x & 31) == 0) li = lb + atomicAdd(lctr, 1);
    li = __shfl_sync(0xffffffffu, li, 0);
    if (li >= le) break;
    const float2* ey = Eyk + (size_t)a.line_ky[li] * By;
    float2 P[GZ], M[GZ];
#pragma unroll
    for (int g = 0; g < GZ; ++g) {
      P[g] = M[g] = make_float2(0.f, 0.f);
      if (EX || g < G) {
        const int2 z = zg[g];
        const float2 u = ry_sum(ey, z.x), v = z.y >= 0 ? ry_sum(ey, z.y) : make_float2(0.f, 0.f);
        P[g] = make_float2(u.x + v.x, u.y + v.y);
        M[g] = make_float2(u.x - v.x, u.y - v.y);
      }
    }
    const int i0 = a.line_k_off[li], i1 = a.line_k_off[li + 1];
    int4 kn = i0 < i1 ? __ldg(a.kent + i0) : make_int4(0, 0, 0, 0);  // the next k's entry, one ahead
    for (int i = i0; i < i1; ++i) {
      const int4 kr = kn;  // (kz, X row of kz, X row of -kz or -1)
      if (i + 1 < i1) kn = __ldg(a.kent + i + 1);
      const float2* ez = Ezg + (size_t)kr.x * G;
      float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
#pragma unroll
      for (int g = 0; g < GZ; ++g) {
        if (!EX && g >= G) break;
        const float2 e = ez[g];
        A.x = fmaf(e.x, P[g].x, A.x);
        A.y = fmaf(e.x, P[g].y, A.y);
        B.x = fmaf(-e.y, M[g].y, B.x);
        B.y = fmaf(e.y, M[g].x, B.y);
      }
      if (live) {
        *reinterpret_cast<float2*>(Xcol + (int64_t)kr.y * ldx32) = make_float2(A.x + B.x, A.y + B.y);
        if (kr.z >= 0) *reinterpret_cast<float2*>(Xcol + (int64_t)kr.z * ldx32) = make_float2(A.x - B.x, A.y - B.y);
      }
    }
  }
}

size_t s1_smem_bytes(int nRe, int Pe, int Bz, int Gz, int nky, int By, int nkz, int Gy) {
  return sizeof(float2) * ((size_t)Pe * kS1Cols + nRe + (size_t)nky * By + (size_t)nkz * Gz) + sizeof(int2) * (size_t)Gz +
         sizeof(int) * ((size_t)Pe + 1 + nRe + ((Pe + 1 + nRe) & 1)) + sizeof(int2) * (size_t)Gy +
         sizeof(int) * ((size_t)Gy + Bz + 1 + kS1Cols / 32);
}

template <int GZ>
static int s1_launch_t(cudaStream_t st, const S1Args& a, int planes) {
  const size_t smem = s1_smem_bytes(a.nRe, a.Pe, a.Bz, a.Gz, a.nky, a.By, a.nkz, a.Gy);
  if (allow_dynamic_smem(k_s1_dft<GZ>) != cudaSuccess)
    return -1;
  dim3 grid((unsigned)((a.C + kS1Cols - 1) / kS1Cols), (unsigned)planes);
  k_s1_dft<GZ><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int s1_launch(cudaStream_t st, const S1Args& a, int planes) {
  if (planes <= 0) return 0;
  if (a.C > INT32_MAX || a.ldx > INT32_MAX) return -2;
  switch (a.Gz) {
    case 1: return s1_launch_t<1>(st, a, planes);
    case 2: return s1_launch_t<2>(st, a, planes);
    case 3: return s1_launch_t<3>(st, a, planes);
    case 4: return s1_launch_t<4>(st, a, planes);
    case 5: return s1_launch_t<5>(st, a, planes);
    case 6: return s1_launch_t<6>(st, a, planes);
    case 7: return s1_launch_t<7>(st, a, planes);
    case 8: return s1_launch_t<8>(st, a, planes);
    default: return a.Gz <= 16 ? s1_launch_t<16>(st, a, planes) : -2;
  }
}

__global__ void k_s1_g32(const cplx* __restrict__ g, int64_t n, float2* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) out[t] = make_float2((float)g[t].re, (float)g[t].im);
}

int s1_convert_g(cudaStream_t st, const cplx* g, int64_t n, float2* out) {
  k_s1_g32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace phx
