// Scores of the learned q proposal for every (state, q) row on the tensor cores (inference
// only; training runs on the CUDA-core kernels of sampler.cu).  The network is
// z = w4 . silu(W3 silu(W2 silu(W1 x + b1) + b2) + b3) + b4, x = (q~, eps - mu, v); the three
// hidden layers run as tcgen05 MMAs (M = 128 rows, N = 128 neurons) with FP16 operands (the
// BF16-rounded parameters are exact in FP16 apart from values below 2^-14, which lose low bits)
// and FP32 accumulation in TMEM.  The 7-input layer is one MMA with K = 16: the row
// (q~, eps - mu, v, 1, 0 ...) against (W1, b1, 0 ...), so its bias comes from the constant input.
// SiLU, the other biases and the head run on the CUDA cores.
//
// One persistent CTA per SM: two groups of 4 warps (thread = row of a 128-row tile) work on
// alternate tiles so that one group's SiLU overlaps the other's MMAs; warp 8 issues the MMAs.
// Per tile and group: X -> smem, MMA layer 1 -> TMEM slot a, H1 -> smem, MMA layer 2 -> slot b,
// H2 -> smem, MMA layer 3 -> slot a, head.
// Every wait is bounded (2 s); on expiry the kernel raises an error flag and unwinds.
#include <cuda_fp16.h>

#include "common.cuh"
#include "mlp_tc.h"
#include "tc_ptx.cuh"

namespace phx {

using namespace tc;

namespace {

constexpr int kThreads = 288;
constexpr uint32_t kOpBytes = 128 * 256;  // one 128 x 128 FP16 operand, two 128-byte swizzle atoms
constexpr uint32_t kAtomBytes = 128 * 128;

// byte offset of element (row, k) of a 128 x 128 FP16 operand in the K-major 128-byte swizzled layout
__device__ __forceinline__ uint32_t sw_offset(int row, int chunk) {  // chunk = k / 8
  const int atom = chunk >> 3, cc = chunk & 7;
  return (uint32_t)(atom * kAtomBytes + (row >> 3) * 1024 + (row & 7) * 128 + ((cc ^ (row & 7)) << 4));
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// silu of two values in FP16: x sigmoid(x) = 0.5 x (1 + tanh(0.5 x)), inputs clamped to the FP16 range
__device__ __forceinline__ uint32_t silu2(float x0, float x1) {
  __half2 h = __floats2half2_rn(x0, x1);
  const __half2 lim = __float2half2_rn(65504.f);
  h = __hmin2(__hmax2(h, __hneg2(lim)), lim);
  const __half2 hh = __hmul2(h, __float2half2_rn(0.5f));
  uint32_t t;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h2_bits(hh)));
  const __half2 r = __hfma2(hh, *reinterpret_cast<__half2*>(&t), hh);
  return h2_bits(r);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(MlpTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* W2s = smem;
  uint8_t* W3s = smem + kOpBytes;
  uint8_t* Hs = smem + 2 * kOpBytes;  // two operands, one per group
  uint8_t* W1s = smem + 4 * kOpBytes;  // one swizzle atom: K chunks 0 and 1 of each neuron row
  float* b2 = reinterpret_cast<float*>(smem + 4 * kOpBytes + kAtomBytes);  // 16-byte aligned
  float* b3 = b2 + 128;
  float* w4 = b3 + 128;
  float* b4 = w4 + 128;
  uint64_t* hready = reinterpret_cast<uint64_t*>(b4 + 4);  // [2], 128 arrivals each
  uint64_t* dready = hready + 2;                           // [2]
  uint64_t* drain = dready + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // weights into the swizzled operand layout, small parameters as FP32
  for (int idx = tid; idx < 128 * 16; idx += kThreads) {
    const int row = idx >> 4, chunk = idx & 15;
    const uint4 v2 = reinterpret_cast<const uint4*>(a.W2h)[idx];
    const uint4 v3 = reinterpret_cast<const uint4*>(a.W3h)[idx];
    *reinterpret_cast<uint4*>(W2s + sw_offset(row, chunk)) = v2;
    *reinterpret_cast<uint4*>(W3s + sw_offset(row, chunk)) = v3;
  }
  for (int j = tid; j < 128; j += kThreads) {  // W1 row j: (W1[j][0..6], b1[j]) then 8 zeros
    const float* wj = a.P + kMlpOffW1 + j * 7;
    const uint4 c0 = make_uint4(h2_bits(__floats2half2_rn(wj[0], wj[1])), h2_bits(__floats2half2_rn(wj[2], wj[3])),
                                h2_bits(__floats2half2_rn(wj[4], wj[5])),
                                h2_bits(__floats2half2_rn(wj[6], a.P[kMlpOffB1 + j])));
    *reinterpret_cast<uint4*>(W1s + sw_offset(j, 0)) = c0;
    *reinterpret_cast<uint4*>(W1s + sw_offset(j, 1)) = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int i = tid; i < 128; i += kThreads) {
    b2[i] = a.P[kMlpOffB2 + i];
    b3[i] = a.P[kMlpOffB3 + i];
    w4[i] = a.P[kMlpOffW4 + i];
  }
  if (tid == 0) {
    b4[0] = a.P[kMlpOffB4];
    mbar_init(hready, 128);
    mbar_init(hready + 1, 128);
    mbar_init(dready, 1);
    mbar_init(dready + 1, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 8) {
    tmem_alloc(tslot, 512);
    tmem_relinquish();
  }
  fence_async_smem();  // weight operands written by the threads, read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tslot;
  const int64_t nrows = a.rows ? (int64_t)*a.nrows : 0;  // row-list mode: the listed rows only
  const int64_t ntiles = a.rows ? (nrows + 127) / 128 : a.ntiles;
  const int64_t n_local = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 8) {
    if (lane == 0) {
      // ---------------- MMA issuer: L2 of tile i, then L3 of tile i-1
      const uint32_t idesc = idesc_m128(128u, 0u);  // FP16 A and B, FP32 accumulate
      uint32_t hph[2] = {0u, 0u};
      bool ok = true;
      // layer l of tile i: l = 0 the 7-input layer (one K = 16 step) into slot a, l = 1 layer 2 into
      // slot b, l = 2 layer 3 into slot a again (its layer-1 result was read before H1 was published)
      auto layer = [&](int64_t i, int l) -> bool {
        const int g = (int)(i & 1);
        if (!mbar_wait(hready + g, hph[g] & 1u, abort_flag)) return false;
        ++hph[g];
        tc_fence_after();
        const uint32_t abase = smem_u32(Hs + g * kOpBytes);
        const uint32_t bbase = smem_u32(l == 0 ? W1s : l == 1 ? W2s : W3s);
        const uint32_t d = tmem_base + (uint32_t)(g * 2 + (l == 1 ? 1 : 0)) * 128u;
        const int nk = l == 0 ? 1 : 8;
        for (int kk = 0; kk < nk; ++kk) {
          const uint32_t off = (uint32_t)(kk >> 2) * kAtomBytes + (uint32_t)(kk & 3) * 32u;
          mma<0>(d, sdesc_k128(abase + off), sdesc_k128(bbase + off), idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(dready + g);
        return true;
      };
      // tiles in pairs, one per group, layer by layer: each group's three layers stay in order
      for (int64_t p0 = 0; p0 < n_local && ok; p0 += 2)
        for (int l = 0; l < 3 && ok; ++l)
          for (int64_t i = p0; i < p0 + 2 && i < n_local && ok; ++i) ok = layer(i, l);
      // no MMA may be in flight when TMEM is released
      mma_commit(drain);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain, 0)) {
        if (globaltimer() - t0 > kWaitLimitNs) {
          *abort_flag = 1;
          break;
        }
      }
    }
  } else {
    // ---------------- two groups of 4 warps; thread = row of the group's tile
    const int g = warp >> 2, wq = warp & 3;
    const int row = wq * 32 + lane;
    uint8_t* H = Hs + g * kOpBytes;
    uint32_t dph = 0;
    for (int64_t i = g; i < n_local; i += 2) {
      const int64_t t = blockIdx.x + i * gridDim.x;
      int s;
      int64_t q;
      bool valid;
      if (a.rows) {
        const int64_t r = t * 128 + row;
        valid = r < nrows;
        const int2 sq = valid ? a.rows[r] : make_int2(0, 0);
        s = sq.x;
        q = sq.y;
      } else {
        s = (int)(t / a.tiles_per_state);
        q = (t % a.tiles_per_state) * 128 + row;
        valid = q < a.Nq;
      }
      float qv[3] = {0.f, 0.f, 0.f}, fv[4] = {0.f, 0.f, 0.f, 0.f};
      if (valid) {
#pragma unroll
        for (int d = 0; d < 3; ++d) qv[d] = a.qt[q * 3 + d];
#pragma unroll
        for (int d = 0; d < 4; ++d) fv[d] = a.feat[(int64_t)s * 4 + d];
      }
      // the row of the 7-input layer's MMA: (q~, eps - mu, v, 1) in K chunk 0, zeros in chunk 1
      *reinterpret_cast<uint4*>(H + sw_offset(row, 0)) =
          make_uint4(h2_bits(__floats2half2_rn(qv[0], qv[1])), h2_bits(__floats2half2_rn(qv[2], fv[0])),
                     h2_bits(__floats2half2_rn(fv[1], fv[2])), h2_bits(__floats2half2_rn(fv[3], 1.f)));
      *reinterpret_cast<uint4*>(H + sw_offset(row, 1)) = make_uint4(0u, 0u, 0u, 0u);
      fence_async_smem();
      mbar_arrive(hready + g);
      bool ok = true;
      float z = 0.f;
#pragma unroll 1
      for (int l = 0; l < 3 && ok; ++l) {  // layer-1, layer-2 and layer-3 results
        int wv = 1;
        if (lane == 0) wv = mbar_wait(dready + g, dph & 1u, abort_flag) ? 1 : 0;
        wv = __shfl_sync(0xffffffffu, wv, 0);
        ++dph;
        if (!wv) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)(g * 2 + (l == 1 ? 1 : 0)) * 128u;
        const float* bias = l == 1 ? b2 : b3;  // layer 1 has its bias from the constant input
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {
          float v[32];
          tmem_ld32(taddr + c0, v);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int j0 = c0 + cc * 8;
            const float4 bA = l == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(bias + j0)[0];
            const float4 bB = l == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(bias + j0)[1];
            const float bv[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
            uint32_t w[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) w[p] = silu2(v[cc * 8 + p * 2] + bv[p * 2], v[cc * 8 + p * 2 + 1] + bv[p * 2 + 1]);
            if (l < 2) {
              *reinterpret_cast<uint4*>(H + sw_offset(row, (c0 >> 3) + cc)) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
              const float4 wA = reinterpret_cast<const float4*>(w4 + j0)[0];
              const float4 wB = reinterpret_cast<const float4*>(w4 + j0)[1];
              const float wv[8] = {wA.x, wA.y, wA.z, wA.w, wB.x, wB.y, wB.z, wB.w};
#pragma unroll
              for (int p = 0; p < 4; ++p) {
                const float2 hv = __half22float2(*reinterpret_cast<__half2*>(&w[p]));
                z = fmaf(hv.x, wv[p * 2], z);
                z = fmaf(hv.y, wv[p * 2 + 1], z);
              }
            }
          }
        }
        tc_fence_before();
        if (l < 2) {
          fence_async_smem();
          mbar_arrive(hready + g);
        }
      }
      if (!ok) break;
      if (valid) a.z[(int64_t)s * a.Nq + q] = z + b4[0];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
  if (tid == 0 && *abort_flag) atomicOr(a.err, 1);
}

__global__ void k_params_half(const float* __restrict__ P, __half* __restrict__ W2h, __half* __restrict__ W3h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 128 * 128) return;
  W2h[i] = __float2half_rn(P[kMlpOffW2 + i]);
  W3h[i] = __float2half_rn(P[kMlpOffW3 + i]);
}

size_t mlp_tc_smem_bytes() {
  return 1024 + 4 * kOpBytes + kAtomBytes + sizeof(float) * (3 * 128 + 4) + 8 * 6 + 16;
}

int mlp_tc_launch(cudaStream_t s, int num_sms, const MlpTcArgs& a) {
  if (a.ntiles <= 0) return 0;
  const size_t smem = mlp_tc_smem_bytes();
  if (allow_dynamic_smem(k_mlp_tc) != cudaSuccess)
    return -1;
  const int64_t grid = std::min<int64_t>(a.ntiles, num_sms > 0 ? num_sms : 148);
  k_mlp_tc<<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mlp_tc_params(cudaStream_t s, const float* P, __half* W2h, __half* W3h) {
  k_params_half<<<(128 * 128 + 255) / 256, 256, 0, s>>>(P, W2h, W3h);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace phx
