// Stage 2 on grid q points as a separable DFT over the R_p box (Sec. 5.5 Eq. 70 evaluated
// exactly in another order).  With q = (jx/Nx, jy/Ny, jz/Nz) the phase of Eq. 13 factorises,
// e^{2 pi i q.R} = e^{2 pi i jx rx/Nx} e^{2 pi i jy ry/Ny} e^{2 pi i jz rz/Nz} with r = R mod N,
// so for every state
//   G(q)[c] = sum_rx Ex[jx][rx] sum_ry Ey[jy][ry] sum_rz Ez[jz][rz] T~[rx][ry][rz][c],
// T~ the stage-1 output T summed over the R_p of equal residue (weights folded in).  The y/z
// sums run first (k_dft_yz, into Y[s][rx][jy][jz][c]); k_dft_x_elph finishes the x sum for one
// q per thread and applies U_{k+q}^dagger, Z_q and the delta weights of Eq. 29 (Sec. 4.7 Eq. 61)
// like the fused tensor-core epilogue.  FP32 on the CUDA cores.
#include "dft.h"

namespace phx {

// One block per (column chunk of 16, rx residue, state); thread (jz, column).  For each chunk
// of 16 jy: acc[jy] = sum_ry Ey[jy][ry] (sum_{R in (rx, ry)} Ez[jz][rz(R)] w_R T[s][R][c]).
// The plane's weighted T columns and the phase tables are staged in shared memory.
__global__ void __launch_bounds__(1024) k_dft_yz(DftYzArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p0 = a.plane_off[blockIdx.y], p1 = a.plane_off[blockIdx.y + 1];
  const int ne = p1 - p0;
  float2* Ts = reinterpret_cast<float2*>(smem);  // [ne][16]
  float2* Eys = Ts + (size_t)ne * 16;            // [Ny][By]
  float2* Ezs = Eys + (size_t)a.Ny * a.By;       // [Nz][Bz]
  int* ays = reinterpret_cast<int*>(Ezs + (size_t)a.Nz * a.Bz);  // [ne]
  int* azs = ays + ne;                                           // [ne]
  const int s = blockIdx.z, ax = blockIdx.y, c0 = blockIdx.x * 16;
  const float2* T = a.T + (int64_t)s * a.nR * a.E;
  for (int i = threadIdx.x; i < ne * 16; i += blockDim.x) {
    const int e = p0 + i / 16, cc = c0 + (i & 15);
    const int r = a.ent_r[e];
    float2 t = make_float2(0.f, 0.f);
    if (cc < a.E) {
      t = T[(int64_t)r * a.E + cc];
      const float w = a.w[r];
      t.x *= w;
      t.y *= w;
    }
    Ts[i] = t;
  }
  for (int i = threadIdx.x; i < a.Ny * a.By; i += blockDim.x) Eys[i] = a.Ey[i];
  for (int i = threadIdx.x; i < a.Nz * a.Bz; i += blockDim.x) Ezs[i] = a.Ez[i];
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    ays[i] = a.ent_ay[p0 + i];
    azs[i] = a.ent_az[p0 + i];
  }
  __syncthreads();
  const int cl = threadIdx.x & 15;
  const int c = c0 + cl;
  const int jz = threadIdx.x >> 4;
  if (jz >= a.Nz || c >= a.E) return;
  float2* Y = a.Y + (((int64_t)s * a.Bx + ax) * a.Ny) * a.Nz * a.E;
  const float2* ez_row = Ezs + jz * a.Bz;
  for (int jy0 = 0; jy0 < a.Ny; jy0 += 16) {
    float2 acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = make_float2(0.f, 0.f);
    int e = 0;
    while (e < ne) {
      const int ay = ays[e];
      float2 yz = make_float2(0.f, 0.f);
      for (; e < ne && ays[e] == ay; ++e) {
        const float2 ez = ez_row[azs[e]];
        const float2 t = Ts[e * 16 + cl];
        yz.x = fmaf(ez.x, t.x, fmaf(-ez.y, t.y, yz.x));
        yz.y = fmaf(ez.x, t.y, fmaf(ez.y, t.x, yz.y));
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (jy0 + i < a.Ny) {
          const float2 ey = Eys[(jy0 + i) * a.By + ay];
          acc[i].x = fmaf(ey.x, yz.x, fmaf(-ey.y, yz.y, acc[i].x));
          acc[i].y = fmaf(ey.x, yz.y, fmaf(ey.y, yz.x, acc[i].y));
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (jy0 + i < a.Ny) Y[((int64_t)(jy0 + i) * a.Nz + jz) * a.E + c] = acc[i];
  }
}

// One block per (group of kDftLines (jy, jz) lines, state); thread (jx, line).  Phase 1: each
// thread sums over rx for its q (G in registers, then its own slot of shared memory) and marks the
// final bands m' that can reach the delta window.  Phase 2: the warp compacts its (q, m') items
// and every lane takes items in turn, so a band is rotated only for the q that need it.
template <int NW, int NM>
__global__ void __launch_bounds__(kDftMaxThreads / PHX_DFT_MINB, PHX_DFT_MINB) k_dft_x_elph(DftXArgs a) {
  constexpr int E = NW * NM;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* Ys = reinterpret_cast<float2*>(smem);                       // [Bx][kDftLines][E]
  float2* Gs = Ys + (size_t)a.Bx * kDftLines * E;                      // [E][threads] (element-major)
  float2* Exs = Gs + (size_t)blockDim.x * E;                           // [Nx][Bx]
  int* items = reinterpret_cast<int*>(Exs + (size_t)a.Nx * a.Bx);      // [warps][32 * NW]
  int* qkq = items + (blockDim.x >> 5) * 32 * NW;                      // [threads][2]: q, k+q
  const int s = blockIdx.y;
  const int line0 = blockIdx.x * kDftLines;
  const int nlines = a.Ny * a.Nz;
  const float2* Yg = a.Y + (int64_t)s * a.Bx * nlines * E;
  for (int i = threadIdx.x; i < a.Bx * kDftLines * E; i += blockDim.x) {
    const int ax = i / (kDftLines * E), rem = i % (kDftLines * E);
    const int l = rem / E, cc = rem % E;
    Ys[i] = line0 + l < nlines ? Yg[((int64_t)ax * nlines + line0 + l) * E + cc] : make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < a.Nx * a.Bx; i += blockDim.x) Exs[i] = a.Ex[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jx = threadIdx.x % a.Nx, l = threadIdx.x / a.Nx;
  const int line = line0 + l;
  const int64_t kf = a.gm.k_to_fine(a.st_k[s]);
  const double e_n = a.epsF[kf * NW + a.st_b[s]];
  const float en_hi = (float)e_n, en_lo = (float)(e_n - (double)en_hi);
  unsigned need = 0;
  if (l < kDftLines && line < nlines) {
    float2 G[E];
#pragma unroll
    for (int e = 0; e < E; ++e) G[e] = make_float2(0.f, 0.f);
    for (int ax = 0; ax < a.Bx; ++ax) {
      const float2 ex = Exs[jx * a.Bx + ax];
      const float2* y = Ys + (ax * kDftLines + l) * E;
      if constexpr (E % 2 == 0) {  // two complex values per 16-byte load
#pragma unroll
        for (int e = 0; e < E; e += 2) {
          const float4 v = reinterpret_cast<const float4*>(y)[e / 2];
          G[e].x = fmaf(ex.x, v.x, fmaf(-ex.y, v.y, G[e].x));
          G[e].y = fmaf(ex.x, v.y, fmaf(ex.y, v.x, G[e].y));
          G[e + 1].x = fmaf(ex.x, v.z, fmaf(-ex.y, v.w, G[e + 1].x));
          G[e + 1].y = fmaf(ex.x, v.w, fmaf(ex.y, v.z, G[e + 1].y));
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const float2 v = y[e];
          G[e].x = fmaf(ex.x, v.x, fmaf(-ex.y, v.y, G[e].x));
          G[e].y = fmaf(ex.x, v.y, fmaf(ex.y, v.x, G[e].y));
        }
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) Gs[(size_t)e * blockDim.x + threadIdx.x] = G[e];
    const int jy = line / a.Nz, jz = line % a.Nz;
    const int q = (jx * a.Ny + jy) * a.Nz + jz;
    int kc[3];
    grid_coords(kf, a.gm.nf, kc);
    const int qc[3] = {jx, jy, jz};
    int fc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) fc[d] = (kc[d] + qc[d] * a.gm.sq[d]) % a.gm.nf[d];
    const int kq = (int)grid_flat(fc, a.gm.nf);
    qkq[2 * threadIdx.x] = q;
    qkq[2 * threadIdx.x + 1] = kq;
#pragma unroll
    for (int mp = 0; mp < NW; ++mp) {
      const float2 ee = a.eps2[(int64_t)kq * NW + mp];
      const float dm = (en_hi - ee.x) + (en_lo - ee.y);
      if (fabsf(dm) < a.reach) need |= 1u << mp;
    }
  }
  // compact the warp's (thread, m') items
  const int cnt = __popc(need);
  int off = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, off, o);
    if (lane >= o) off += t;
  }
  const int total = __shfl_sync(0xffffffffu, off, 31);
  off -= cnt;
  int* wl = items + warp * 32 * NW;
  for (unsigned m = need; m; m &= m - 1) wl[off++] = (threadIdx.x << 4) | (__ffs(m) - 1);
  __syncwarp();
  double acc = 0.0;
  for (int it = lane; it < total; it += 32) {
    const int src = wl[it] >> 4, mp = wl[it] & 15;
    const int q = qkq[2 * src], kq = qkq[2 * src + 1];
    const float2* gs = Gs + src;  // element e at gs[e * blockDim.x]
    const float2 ee = a.eps2[(int64_t)kq * NW + mp];
    const float dm = (en_hi - ee.x) + (en_lo - ee.y);
    const float2* uh = a.UH + ((int64_t)kq * NW + mp) * NW;
    float2 u[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) u[m] = uh[m];
    float2 t[NM];
#pragma unroll
    for (int sa = 0; sa < NM; ++sa) {
      t[sa] = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < NW; ++m) {
        const float2 gv = gs[(size_t)(sa * NW + m) * blockDim.x];
        t[sa].x = fmaf(u[m].x, gv.x, fmaf(-u[m].y, gv.y, t[sa].x));
        t[sa].y = fmaf(u[m].x, gv.y, fmaf(u[m].y, gv.x, t[sa].y));
      }
    }
    const float f = a.f32[(int64_t)kq * NW + mp];
    const float2* zq = a.Zf + (int64_t)q * NM * NM;
    float part = 0.f;
#pragma unroll
    for (int v = 0; v < NM; ++v) {
      float2 g = make_float2(0.f, 0.f);
#pragma unroll
      for (int sa = 0; sa < NM; ++sa) {
        const float2 zz = zq[sa * NM + v];
        g.x = fmaf(t[sa].x, zz.x, fmaf(-t[sa].y, zz.y, g.x));
        g.y = fmaf(t[sa].x, zz.y, fmaf(t[sa].y, zz.x, g.y));
      }
      const float om = a.omf[(int64_t)q * NM + v], nb = a.nBf[(int64_t)q * NM + v];
      const float t1 = (dm - om) * a.inv_sigma;
      const float t2 = (dm + om) * a.inv_sigma;
      float w = 0.f;
      if (t1 * t1 < a.cut2) w += (nb + 1.f - f) * expf(-t1 * t1);
      if (t2 * t2 < a.cut2) w += (nb + f) * expf(-t2 * t2);
      part = fmaf(g.x * g.x + g.y * g.y, w, part);
    }
    acc += (double)part * a.scale;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += red[i];
    if (sum != 0.0) atomicAdd(a.gamma + a.s_base + s, sum);
  }
}

template <int NW, int NM>
static int launch_x(cudaStream_t st, const DftXArgs& a, int S) {
  const int threads = (a.Nx * kDftLines + 31) / 32 * 32;  // whole warps for the compaction and reduction
  const size_t smem = dft_smem_bytes(a.Bx, NW * NM, threads, NW, a.Nx);
  if (cudaFuncSetAttribute(k_dft_x_elph<NW, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return -1;
  const int lines = a.Ny * a.Nz;
  dim3 grid((unsigned)((lines + kDftLines - 1) / kDftLines), (unsigned)S);
  k_dft_x_elph<NW, NM><<<grid, threads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int dft_launch(cudaStream_t st, const DftYzArgs& yz, const DftXArgs& x, int S, int nw, int nm) {
  dim3 g1((unsigned)((yz.E + 15) / 16), (unsigned)yz.Bx, (unsigned)S);
  const size_t sm1 = dft_yz_smem_bytes(yz.ne_max, yz.Ny, yz.By, yz.Nz, yz.Bz);
  if (cudaFuncSetAttribute(k_dft_yz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1) != cudaSuccess) return -1;
  k_dft_yz<<<g1, yz.Nz * 16, sm1, st>>>(yz);
  if (cudaGetLastError() != cudaSuccess) return -1;
  if (nw == 8 && nm == 6) return launch_x<8, 6>(st, x, S);
  if (nw == 2 && nm == 3) return launch_x<2, 3>(st, x, S);
  if (nw == 1 && nm == 3) return launch_x<1, 3>(st, x, S);
  return -2;
}

size_t dft_smem_bytes(int Bx, int E, int threads, int nw, int Nx) {
  return sizeof(float2) * ((size_t)Bx * kDftLines * E + (size_t)threads * E + (size_t)Nx * Bx) +
         sizeof(int) * ((size_t)(threads / 32) * 32 * nw + 2 * (size_t)threads);
}

size_t dft_yz_smem_bytes(int ne_max, int Ny, int By, int Nz, int Bz) {
  return sizeof(float2) * ((size_t)ne_max * 16 + (size_t)Ny * By + (size_t)Nz * Bz) + sizeof(int) * 2 * (size_t)ne_max;
}

// E[j][a] = e^{2 pi i j r_a / N} for residues r_a (exact integer argument reduction, sincospi).
__global__ void k_dft_table(const int* __restrict__ res, int B, int N, float2* __restrict__ E) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * B) return;
  const int j = t / B, a = t % B;
  const int r = (int)(((int64_t)j * res[a]) % N);
  double sv, cv;
  sincospi(2.0 * (double)r / (double)N, &sv, &cv);
  E[t] = make_float2((float)cv, (float)sv);
}

int dft_table(cudaStream_t st, const int* res, int B, int N, float2* E) {
  k_dft_table<<<(N * B + 127) / 128, 128, 0, st>>>(res, B, N, E);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace phx
