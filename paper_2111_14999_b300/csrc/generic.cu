// Band and mode rotations plus the delta weights of Eq. 29 for any Wannier count and
// any number of modes (Sec. 3.2 Eqs. 7 and 13, Sec. 4.2 Eq. 29, Sec. 4.7 Eq. 61), applied to
// a stage-2 result G_s(q)[sa][m] = sum_Rp w e^{iq.Rp} T_s[Rp][sa][m] that the tensor-core
// GEMM wrote to HBM.  The fused stage-2 epilogue covers the (nw, 3na) shapes it is built
// for; this kernel serves every other shape.
#include "kernels.cuh"
#include "generic.h"

namespace phx {

// One block per (q row, group of kGenericStatesPerBlock states); each warp takes every 8th
// state of the group, one (q, state) pair at a time: lane = final band m' for the window test,
// then the whole warp on each final band in reach (lane = mode row sa for the U_{k+q}^dagger
// rotation, lane = mode v for the Z_q rotation and the delta weights).  MAXNM: instantiations
// below kGenericMaxModes are launched only for nm == MAXNM.
template <int MAXNM>
__global__ void __launch_bounds__(256) k_elph_generic(ElphGenericArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // instantiations below kGenericMaxModes are launched only for nm == MAXNM
  const int nw = a.nw, nm = MAXNM < kGenericMaxModes ? MAXNM : a.nm;
  const int cps = 2 * nw * nm;
  float2* zs = reinterpret_cast<float2*>(smem);                 // [nm][nm] mode factors of this q
  const int gstride = 2 * nw + 1;  // floats per mode row of a staged G row (odd: lanes sa hit distinct banks)
  float* gs = reinterpret_cast<float*>(zs + nm * nm) + warp * nm * gstride;  // this warp's G row [sa][m][re, im]
  float* oms = reinterpret_cast<float*>(zs + nm * nm) + 8 * nm * gstride;     // [nm] omega, then [nm] n_B
  float* nbs = oms + nm;
  const int64_t r = blockIdx.x;  // row of the chunk
  const int q = a.q_of_row[a.row0 + r];
  if (q < 0) return;  // padding row (uniform over the block)
  for (int i = threadIdx.x; i < nm * nm; i += blockDim.x) zs[i] = a.Zf[(int64_t)q * nm * nm + i];
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    oms[i] = a.omf[(int64_t)q * nm + i];
    nbs[i] = a.nBf[(int64_t)q * nm + i];
  }
  __syncthreads();
  int qc[3];
  grid_coords(q, a.gm.nq, qc);
  const int s_end = min(a.S, (int)(blockIdx.y + 1) * kGenericStatesPerBlock);
  for (int s = blockIdx.y * kGenericStatesPerBlock + warp; s < s_end; s += 8) {
    const int64_t kf = a.gm.k_to_fine(a.st_k[s]);
    int kc[3];
    grid_coords(kf, a.gm.nf, kc);
    int fc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) fc[d] = (kc[d] + qc[d] * a.gm.sq[d]) % a.gm.nf[d];
    const int64_t kq = grid_flat(fc, a.gm.nf);
    const double e_n = a.epsF[kf * nw + a.st_b[s]];
    const float en_hi = (float)e_n, en_lo = (float)(e_n - (double)en_hi);
    float part = 0.f;
    const int mp = lane;
    bool need = false;
    float dm = 0.f;
    if (mp < nw) {
      const float2 e = a.eps2[kq * nw + mp];
      dm = (en_hi - e.x) + (en_lo - e.y);
      need = fabsf(dm) < a.reach;
    }
    // a pair none of whose final bands reaches the delta window contributes nothing: its G row
    // is not read
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (!mask) continue;
    {  // stage the warp's G row (FP32 pairs) in shared memory
      const float* grow = a.G + r * a.ldg + (int64_t)s * cps;
      __syncwarp();
      for (int i = lane; i < cps; i += 32) {
        const int sa = i / (2 * nw);
        gs[i + sa] = grow[i];  // = gs[sa * gstride + i - sa * 2 nw]
      }
      __syncwarp();
    }
    // each final band in reach in turn, the whole warp on it: lane sa forms
    // t[sa] = sum_m conj(U_{k+q}[m][m']) G[sa][m], lane v then g_v = sum_sa t[sa] Z_q[sa][v]
    for (unsigned mm = mask; mm; mm &= mm - 1) {
      const int mpb = __ffs(mm) - 1;
      const float dmb = __shfl_sync(0xffffffffu, dm, mpb);
      float2 t = make_float2(0.f, 0.f);
      if (lane < nm) {
        const float2* uh = a.UH + (kq * nw + mpb) * nw;
        const float* gl = gs + lane * gstride;
        for (int m = 0; m < nw; ++m) {
          const float2 u = uh[m];
          const float gr = gl[2 * m], gi = gl[2 * m + 1];
          t.x = fmaf(u.x, gr, fmaf(-u.y, gi, t.x));
          t.y = fmaf(u.x, gi, fmaf(u.y, gr, t.y));
        }
      }
      const float f = a.f32[kq * nw + mpb];
      float2 g = make_float2(0.f, 0.f);
      for (int sa = 0; sa < nm; ++sa) {
        const float tx = __shfl_sync(0xffffffffu, t.x, sa), ty = __shfl_sync(0xffffffffu, t.y, sa);
        if (lane < nm) {
          const float2 z = zs[sa * nm + lane];
          g.x = fmaf(tx, z.x, fmaf(-ty, z.y, g.x));
          g.y = fmaf(tx, z.y, fmaf(ty, z.x, g.y));
        }
      }
      if (lane < nm) {
        const float t1 = (dmb - oms[lane]) * a.inv_sigma;
        const float t2 = (dmb + oms[lane]) * a.inv_sigma;
        float w = 0.f;
        if (t1 * t1 < a.cut2) w += (nbs[lane] + 1.f - f) * expf(-t1 * t1);
        if (t2 * t2 < a.cut2) w += (nbs[lane] + f) * expf(-t2 * t2);
        part = fmaf(g.x * g.x + g.y * g.y, w, part);
      }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0 && part != 0.f) {
      const float sT = generic_pow2_scale(__uint_as_float(*a.tmax));
      atomicAdd(a.gamma + a.s_base + s, (double)part * (a.scale_base / ((double)sT * (double)sT)));
    }
  }
}

size_t elph_generic_smem(int nw, int nm) {
  return sizeof(float2) * nm * nm + sizeof(float) * (8 * (size_t)nm * (2 * nw + 1) + 2 * nm);
}

template <int MAXNM>
static int launch_nm(cudaStream_t s, const ElphGenericArgs& a, int64_t rows) {
  const size_t smem = elph_generic_smem(a.nw, a.nm);
  if (allow_dynamic_smem(k_elph_generic<MAXNM>) !=
      cudaSuccess)
    return -1;
  dim3 grid((unsigned)rows, (unsigned)((a.S + kGenericStatesPerBlock - 1) / kGenericStatesPerBlock));
  k_elph_generic<MAXNM><<<grid, 256, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_elph_generic(cudaStream_t s, const ElphGenericArgs& a, int64_t rows) {
  switch (a.nm) {  // 3 modes per atom: exact unrolling for 1..6 atoms
    case 3: return launch_nm<3>(s, a, rows);
    case 6: return launch_nm<6>(s, a, rows);
    case 9: return launch_nm<9>(s, a, rows);
    case 12: return launch_nm<12>(s, a, rows);
    case 15: return launch_nm<15>(s, a, rows);
    case 18: return launch_nm<18>(s, a, rows);
    default: return launch_nm<kGenericMaxModes>(s, a, rows);
  }
}

}  // namespace phx
