// Importance-sampled q sums of Eq. 29 with a learned proposal.  The paper has no
// counterpart: it sums every q of the grid (Sec. 4.2).  Write c_nk(q) for N_q times the
// q term of Eq. 29, so Gamma_nk = (1/N_q) sum_q c_nk(q).  Per initial k this file
//   * scores every q for each active band with a small network z_nk(q) (7 -> 128 -> 128 ->
//     128 -> 1, SiLU, BF16-rounded parameters, FP32 activations),
//   * weights every q by the shell factor phi_nk(q), the bracket of Eq. 29 with |g|^2 replaced by
//     1/(hbar w_q nu) (zero exactly where every Gaussian of the q term is cut, so zero wherever
//     c_nk(q) is), computed from the band and phonon tables alone,
//   * forms p_k(q) = (1 - alpha) mean_n softmax_q (z_nk(q) + log phi_nk(q)) + alpha mean_n phi_nk(q) /
//     sum_q phi_nk over the active bands with some phi > 0 (the shell proposal alone: phi / sum phi;
//     the uniform proposal: 1/N_q) and its FP64 running sum in q-index order,
//   * draws S q points i.i.d. by inverse CDF from Philox4x32-10 uniforms,
//   * evaluates c_nk(q_j) at the drawn points only (R_p phase sum on the stage-1 output, band
//     and mode rotations, Gaussian deltas) and accumulates (1/S) sum_j c/(N_q p).
// It also trains the network: targets c_nk(q) / sum_q c_nk(q) from a full-grid run, loss the
// per-state cross entropy against softmax_q (z + log phi), gradients by hand-written backward
// kernels, Adam updates.  All arithmetic runs in the kernels below; the host only orders them.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <random>
#include <vector>

#include "mlp_tc.h"
#include "sampler.h"

namespace phx {

// ------------------------------------------------------------------ parameter layout
constexpr int kNin = 7, kNh = 128;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kNh * kNin;
constexpr int kOffW2 = kOffB1 + kNh;
constexpr int kOffB2 = kOffW2 + kNh * kNh;
constexpr int kOffW3 = kOffB2 + kNh;
constexpr int kOffB3 = kOffW3 + kNh * kNh;
constexpr int kOffW4 = kOffB3 + kNh;
constexpr int kOffB4 = kOffW4 + kNh;
constexpr int kNParam = kOffB4 + 1;
static_assert(kNParam == PHOEBE_GPU_MLP_NPARAM, "parameter blob layout");

constexpr int64_t kMaxRows = (int64_t)1 << 21;  // network rows per evaluation chunk
constexpr int kIsStream = 0x4953;                // third Philox counter word of the draws
constexpr int kDrawChunk = 2048;                 // draws per block of the sampled-pair kernel

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

static int launched(phoebe_gpu_ctx* c, int n) {
  c->launches += n;
  CK(c, cudaGetLastError());
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key advancing by (W0, W1) between rounds.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Uniform in [0,1) of draw j for k-grid index k: 53 bits of the first two output words.
__host__ __device__ __forceinline__ double is_uniform(uint64_t seed, uint32_t j, uint32_t k) {
  uint32_t c[4] = {j, k, (uint32_t)kIsStream, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t bits = ((((uint64_t)c[1]) << 32) | c[0]) >> 11;
  return (double)bits * 1.1102230246251565e-16;  // 2^-53
}

__global__ void k_is_uniforms(uint64_t seed, uint32_t k, int64_t n, double* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) out[j] = is_uniform(seed, (uint32_t)j, k);
}

// ------------------------------------------------------------------ network pieces
__device__ __forceinline__ float bf16_rne(float x) {
  uint32_t b = __float_as_uint(x);
  b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
  return __uint_as_float(b);
}
__device__ __forceinline__ float silu(float a) { return a / (1.f + expf(-a)); }
__device__ __forceinline__ float dsilu(float a) {
  const float s = 1.f / (1.f + expf(-a));
  return s * (1.f + a * (1.f - s));
}

__global__ void k_round_params(const float* __restrict__ w, int n, float* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = bf16_rne(w[i]);
}

// Network input of row r: explicit rows, or (q~(q), features of the row group's state).
struct RowX {
  const float* x = nullptr;      // [rows][7]
  const float* qt = nullptr;     // [Nq][3]
  const float* feat = nullptr;   // [states][4]
  const int* states = nullptr;   // group -> state (NULL: identity)
  int64_t Nq = 1;                // rows per group
  int64_t rows = 0;              // real rows; later rows are zero input
  __device__ __forceinline__ float get(int64_t r, int i) const {
    if (r >= rows) return 0.f;
    if (x) return x[r * kNin + i];
    const int64_t g = r / Nq, q = r - g * Nq;
    if (i < 3) return qt[q * 3 + i];
    const int64_t s = states ? states[g] : g;
    return feat[s * 4 + (i - 3)];
  }
};

// A1 = W1 x + b1 (optional), H1 = silu(A1); rows_pad x 128.
__global__ void k_layer1(const float* __restrict__ Wr, RowX X, int64_t rows_pad, float* __restrict__ A1,
                         float* __restrict__ H1) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r = t >> 7;
  const int j = (int)(t & 127);
  if (r >= rows_pad) return;
  float a = Wr[kOffB1 + j];
#pragma unroll
  for (int i = 0; i < kNin; ++i) a = fmaf(Wr[kOffW1 + j * kNin + i], X.get(r, i), a);
  if (A1) A1[t] = a;
  H1[t] = silu(a);
}

// z[r] = w4 . H3[r] + b4 (one warp per row).
__global__ void k_head(const float* __restrict__ H3, const float* __restrict__ Wr, int64_t rows,
                       float* __restrict__ z) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float4 h = reinterpret_cast<const float4*>(H3 + r * kNh)[lane];
  const float4 w = reinterpret_cast<const float4*>(Wr + kOffW4)[lane];
  float s = h.x * w.x + h.y * w.y + h.z * w.z + h.w * w.w;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) z[r] = s + Wr[kOffB4];
}

// Targets of row r of group g: explicit per row, or c[state][q] of the training grid; the same for
// the additive log prior of the softmax (log phi; none: 0).
struct RowT {
  const float* t = nullptr;
  const float* c = nullptr;
  const float* lp = nullptr;    // explicit prior per row
  const float* lpc = nullptr;   // prior [state][q] of the training grid
  const int* states = nullptr;
  int64_t Nq = 1;
  __device__ __forceinline__ float get(int g, int64_t r, int64_t off_g) const {
    if (t) return t[r];
    return c[(int64_t)states[g] * Nq + (r - off_g)];
  }
  __device__ __forceinline__ float prior(int g, int64_t r, int64_t off_g) const {
    if (lp) return lp[r];
    if (lpc) return lpc[(int64_t)states[g] * Nq + (r - off_g)];
    return 0.f;
  }
};

template <typename T>
__device__ __forceinline__ T block_reduce_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}
__device__ __forceinline__ float block_reduce_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float s = -INFINITY;
  for (int i = 0; i < nw; ++i) s = fmaxf(s, red[i]);
  return s;
}

// Per group, with y = z + prior (prior -inf where the target is 0): loss_g = lse(y) - sum t y / sum t
// over the rows with t > 0, dz = (softmax(y) - t / sum t) * inv_G.
__global__ void k_softmax_ce(const float* __restrict__ z, const int64_t* __restrict__ off, RowT T, float inv_G,
                             float* __restrict__ dz, double* __restrict__ loss) {
  __shared__ double redd[32];
  __shared__ float redf[32];
  const int g = blockIdx.x;
  const int64_t a = off[g], b = off[g + 1];
  float m = -INFINITY;
  for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) m = fmaxf(m, z[r] + T.prior(g, r, a));
  m = block_reduce_max(m, redf);
  if (m == -INFINITY) {  // no row carries weight: nothing to learn from this group
    for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) dz[r] = 0.f;
    return;
  }
  double se = 0.0, st = 0.0, stz = 0.0;
  for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) {
    const float yr = z[r] + T.prior(g, r, a), tr = T.get(g, r, a);
    se += (double)expf(yr - m);
    st += (double)tr;
    if (tr > 0.f) stz += (double)tr * (double)(yr - m);
  }
  se = block_reduce_sum(se, redd);
  st = block_reduce_sum(st, redd);
  stz = block_reduce_sum(stz, redd);
  if (!(st > 0.0)) {
    for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x) dz[r] = 0.f;
    return;
  }
  const double lse = log(se);  // relative to m
  const float lsef = (float)lse;
  const float inv_st = (float)(1.0 / st);
  for (int64_t r = a + threadIdx.x; r < b; r += blockDim.x)
    dz[r] = (expf(z[r] + T.prior(g, r, a) - m - lsef) - T.get(g, r, a) * inv_st) * inv_G;
  if (threadIdx.x == 0) atomicAdd(loss, (lse - stz / st) * (double)inv_G);
}

// dA3 = dz w4 silu'(A3); grad w4 += sum_r dz H3, grad b4 += sum_r dz.
__global__ void k_head_back(const float* __restrict__ dz, const float* __restrict__ H3, const float* __restrict__ A3,
                            const float* __restrict__ Wr, int64_t rows, int64_t rows_per_block,
                            float* __restrict__ dA3, float* __restrict__ grad) {
  const int j = threadIdx.x;
  const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  const float w4 = Wr[kOffW4 + j];
  float aw = 0.f, ab = 0.f;
  for (int64_t r = r0; r < r1; ++r) {
    const float d = dz[r];
    dA3[r * kNh + j] = d * w4 * dsilu(A3[r * kNh + j]);
    aw = fmaf(d, H3[r * kNh + j], aw);
    ab += d;
  }
  atomicAdd(grad + kOffW4 + j, aw);
  if (j == 0) atomicAdd(grad + kOffB4, ab);
}

// out[j] += sum_r D[r][j] (bias gradients).
__global__ void k_colsum(const float* __restrict__ D, int64_t rows, int64_t rows_per_block, float* __restrict__ out) {
  const int j = threadIdx.x;
  const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  float a = 0.f;
  for (int64_t r = r0; r < r1; ++r) a += D[r * kNh + j];
  atomicAdd(out + j, a);
}

// grad W1[j][i] += sum_r dA1[r][j] x_r[i], grad b1[j] += sum_r dA1[r][j].
__global__ void k_layer1_back(const float* __restrict__ dA1, RowX X, int64_t rows, int64_t rows_per_block,
                              float* __restrict__ grad) {
  const int j = threadIdx.x;
  const int64_t r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  float aw[kNin] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, ab = 0.f;
  for (int64_t r = r0; r < r1; ++r) {
    const float d = dA1[r * kNh + j];
#pragma unroll
    for (int i = 0; i < kNin; ++i) aw[i] = fmaf(d, X.get(r, i), aw[i]);
    ab += d;
  }
#pragma unroll
  for (int i = 0; i < kNin; ++i) atomicAdd(grad + kOffW1 + j * kNin + i, aw[i]);
  atomicAdd(grad + kOffB1 + j, ab);
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------------------ FP32 tiled GEMM (CUDA cores)
// C[M][N] = op(A)[M][K] op(B)[K][N], row-major.  TA: A stored [K][M]; TB: B stored [N][K].
// 128 x 128 tiles, 256 threads, 8 x 8 outputs per thread, K steps of 8 staged through shared
// memory with a register prefetch of the next step.  M, N multiples of 128, K of 8.
enum { kEpiStore = 0, kEpiBiasSilu = 1, kEpiDsilu = 2, kEpiAtomic = 3 };
struct GemmEpi {
  const float* bias = nullptr;  // kEpiBiasSilu: bias[n]
  float* pre = nullptr;         // kEpiBiasSilu: pre-activation output (optional)
  const float* aux = nullptr;   // kEpiDsilu: pre-activation whose silu' multiplies the product
};

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_sgemm(int64_t M, int N, int64_t K, const float* __restrict__ A, int64_t lda,
                                               const float* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                               int64_t ldc, GemmEpi e, int64_t k_per_split) {
  __shared__ __align__(16) float As[2][8][128];
  __shared__ __align__(16) float Bs[2][8][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int n0 = blockIdx.y * 128;
  const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
  const int64_t kend = min(K, kbeg + k_per_split);
  if (kbeg >= kend) return;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 ra, rb;
  auto gload = [&](int64_t k0) {
    if (!TA) ra = *reinterpret_cast<const float4*>(A + (m0 + (tid >> 1)) * lda + k0 + (tid & 1) * 4);
    else ra = *reinterpret_cast<const float4*>(A + (k0 + (tid >> 5)) * lda + m0 + (tid & 31) * 4);
    if (!TB) rb = *reinterpret_cast<const float4*>(B + (k0 + (tid >> 5)) * ldb + n0 + (tid & 31) * 4);
    else rb = *reinterpret_cast<const float4*>(B + (int64_t)(n0 + (tid >> 1)) * ldb + k0 + (tid & 1) * 4);
  };
  auto sstore = [&](int buf) {
    if (!TA) {
      const int mm = tid >> 1, kk = (tid & 1) * 4;
      As[buf][kk][mm] = ra.x;
      As[buf][kk + 1][mm] = ra.y;
      As[buf][kk + 2][mm] = ra.z;
      As[buf][kk + 3][mm] = ra.w;
    } else {
      *reinterpret_cast<float4*>(&As[buf][tid >> 5][(tid & 31) * 4]) = ra;
    }
    if (!TB) {
      *reinterpret_cast<float4*>(&Bs[buf][tid >> 5][(tid & 31) * 4]) = rb;
    } else {
      const int nn = tid >> 1, kk = (tid & 1) * 4;
      Bs[buf][kk][nn] = rb.x;
      Bs[buf][kk + 1][nn] = rb.y;
      Bs[buf][kk + 2][nn] = rb.z;
      Bs[buf][kk + 3][nn] = rb.w;
    }
  };
  gload(kbeg);
  sstore(0);
  __syncthreads();
  int cur = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += 8) {
    const bool more = k0 + 8 < kend;
    if (more) gload(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) sstore(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h * 64 + tx * 4;
      float v[4] = {acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]};
      float* cp = C + m * ldc + n;
      if (EPI == kEpiAtomic) {
#pragma unroll
        for (int u = 0; u < 4; ++u) atomicAdd(cp + u, v[u]);
      } else if (EPI == kEpiBiasSilu) {
        float a4[4], h4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a4[u] = v[u] + e.bias[n + u];
          h4[u] = silu(a4[u]);
        }
        if (e.pre) *reinterpret_cast<float4*>(e.pre + m * ldc + n) = make_float4(a4[0], a4[1], a4[2], a4[3]);
        *reinterpret_cast<float4*>(cp) = make_float4(h4[0], h4[1], h4[2], h4[3]);
      } else if (EPI == kEpiDsilu) {
        const float4 x = *reinterpret_cast<const float4*>(e.aux + m * ldc + n);
        *reinterpret_cast<float4*>(cp) =
            make_float4(v[0] * dsilu(x.x), v[1] * dsilu(x.y), v[2] * dsilu(x.z), v[3] * dsilu(x.w));
      } else {
        *reinterpret_cast<float4*>(cp) = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
  }
}

template <bool TA, bool TB, int EPI>
static int sgemm(phoebe_gpu_ctx* c, int64_t M, int N, int64_t K, const float* A, int64_t lda, const float* B,
                 int64_t ldb, float* C, int64_t ldc, GemmEpi e, int splits = 1) {
  if (M % 128 || N % 128 || K % 8 || K <= 0)
    return fail(c, PHOEBE_GPU_ERR_ARG, "internal GEMM shape %lld x %d x %lld not tile aligned", (long long)M, N,
                (long long)K);
  const int64_t kps = round_up((K + splits - 1) / splits, 8);
  splits = (int)((K + kps - 1) / kps);
  dim3 grid((unsigned)(M / 128), (unsigned)(N / 128), (unsigned)splits);
  k_sgemm<TA, TB, EPI><<<grid, 256, 0, c->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, e, kps);
  return launched(c, 1);
}

// ------------------------------------------------------------------ features
// q~ per q of the grid: q wrapped into [-1/2, 1/2) per axis.
__global__ void k_wrapped_q(int n0, int n1, int n2, int64_t Nq, float* __restrict__ qt) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= Nq) return;
  const int n[3] = {n0, n1, n2};
  int j[3];
  grid_coords(q, n, j);
#pragma unroll
  for (int i = 0; i < 3; ++i) qt[q * 3 + i] = (float)((double)(2 * j[i] >= n[i] ? j[i] - n[i] : j[i]) / n[i]);
}

// feat[s] = (eps - mu, v[3]) with v_i = Re <u_b| sum_R w_R i R_i e^{ik.R} H(R) |u_b>
// = -sum_R w_R R_i Im(e^{ik.R} u_b^dagger H(R) u_b)   (Hellmann-Feynman on Eq. 10).
__global__ void k_state_features(const int* __restrict__ st_k, const int* __restrict__ st_b, GridMap gm,
                                 GridPhase gf, const cplx* __restrict__ cis_f, const cplx* __restrict__ H,
                                 const int* __restrict__ RH, const double* __restrict__ wH, int nR, int nw,
                                 const double* __restrict__ epsF, const cplx* __restrict__ UF, double mu,
                                 float* __restrict__ feat) {
  __shared__ cplx u[kMaxNw];
  __shared__ double red[32];
  const int s = blockIdx.x;
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
    const cplx e = cmul(ph, sr);
    for (int i = 0; i < 3; ++i) v[i] -= wH[r] * Rv[i] * e.im;
  }
  for (int i = 0; i < 3; ++i) v[i] = block_reduce_sum(v[i], red);
  if (threadIdx.x == 0) {
    feat[(int64_t)s * 4] = (float)(epsF[f * nw + b] - mu);
    for (int i = 0; i < 3; ++i) feat[(int64_t)s * 4 + 1 + i] = (float)v[i];
  }
}

// ------------------------------------------------------------------ shell factor, proposal and draws
// lphi[s][q] = log phi_s(q), phi_s(q) = sum_{m'} sum_{nu: w >= omega_cut} [(n + 1 - f) D(e - w - e') +
// (n + f) D(e + w - e')] / w with D(x) = exp(-x^2/sigma^2) for |x| < cut sigma (0 beyond), e = eps_nk,
// e' = eps_m'k+q, f = f_m'k+q, (w, n) = (hbar w_q nu, n_q nu): the bracket of Eq. 29 with |g|^2 replaced by
// 1/(hbar w).  Which terms are present is decided as the FP64 evaluation of Eq. 29 decides it (a band
// with |e - e'| >= reach = omega_max + cut sigma has none): in FP32 where the value is more than
// 1e-6 eV from a cut, in FP64 within that margin.  The weights are FP32 (phi is only a proposal: its
// rounding changes the variance, never the expectation).  -inf where phi = 0.  Grid (q blocks, states).
__global__ void k_shell_log(const int* __restrict__ st_k, const int* __restrict__ st_b, GridMap gm, int64_t Nq,
                            const double* __restrict__ epsF, const float2* __restrict__ eps2,
                            const double* __restrict__ fF, const double* __restrict__ omega,
                            const float* __restrict__ omf, const float* __restrict__ nBf, int nw, int nm,
                            double omega_cut, double inv_sigma, double xcut, double reach,
                            float* __restrict__ lphi) {
  const int s = blockIdx.y;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= Nq) return;
  const int64_t k = st_k[s];
  const double e = epsF[gm.k_to_fine(k) * nw + st_b[s]];
  const int64_t kq = gm.kq_to_fine(k, q);
  const float fis = (float)inv_sigma;
  const float ef = (float)e, reach_f = (float)reach * 1.0001f;  // FP32 screen with a margin far above FP32 rounding
  // FP32 decisions with a margin: x = de -+ w and w are within 1e-7 eV of their FP64 values, so
  // only a value within 1e-6 eV of a cut is decided again in FP64
  constexpr float kTol = 1e-6f;
  const float xcut_f = (float)xcut, cut_f = (float)omega_cut;
  float phi = 0.f;
  for (int mp = 0; mp < nw; ++mp) {
    if (!(fabsf(ef - eps2[kq * nw + mp].x) < reach_f)) continue;  // no term of this band can be present
    const double de = e - epsF[kq * nw + mp];
    if (!(fabs(de) < reach)) continue;
    const float f = (float)fF[kq * nw + mp];
    const float de_f = (float)de;
    for (int v = 0; v < nm; ++v) {
      const float wf = omf[q * nm + v];
      bool alive = wf > cut_f + kTol;
      if (!alive && !(wf < cut_f - kTol)) alive = omega[q * nm + v] >= omega_cut;
      if (!alive) continue;
      const float n = nBf[q * nm + v];
      const float x1 = de_f - wf, x2 = de_f + wf;
      bool in1 = fabsf(x1) < xcut_f - kTol, in2 = fabsf(x2) < xcut_f - kTol;
      if (!in1 && !(fabsf(x1) > xcut_f + kTol)) in1 = fabs(de - omega[q * nm + v]) < xcut;
      if (!in2 && !(fabsf(x2) > xcut_f + kTol)) in2 = fabs(de + omega[q * nm + v]) < xcut;
      float d = 0.f;
      if (in1) {
        const float t = x1 * fis;
        d = fmaf(n + 1.f - f, __expf(-t * t), d);
      }
      if (in2) {
        const float t = x2 * fis;
        d = fmaf(n + f, __expf(-t * t), d);
      }
      phi = fmaf(d, 1.f / wf, phi);
    }
  }
  lphi[(int64_t)s * Nq + q] = phi > 0.f ? logf(phi) : -INFINITY;
}

// The (state, q) rows with phi > 0 of S states, appended in chunks to rows[] (order across chunks
// arbitrary); *nrows counts them.  One block per state.
__global__ void k_shell_rows(const float* __restrict__ lphi, int64_t Nq, int2* __restrict__ rows,
                             unsigned long long* __restrict__ nrows) {
  __shared__ int wcount[32];
  __shared__ unsigned long long base_s;
  const int s = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int64_t c0 = 0; c0 < Nq; c0 += blockDim.x) {
    const int64_t q = c0 + threadIdx.x;
    const bool live = q < Nq && lphi[(int64_t)s * Nq + q] != -INFINITY;
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    if (lane == 0) wcount[w] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int i = 0; i < nwarp; ++i) tot += wcount[i];
      base_s = tot ? atomicAdd(nrows, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    if (live) {
      int before = 0;
      for (int i = 0; i < w; ++i) before += wcount[i];
      rows[base_s + before + __popc(bal & ((1u << lane) - 1u))] = make_int2(s, (int)q);
    }
    __syncthreads();
  }
}

// Per state: ymax = max_q y, ysum = sum_q expf(y - ymax) (FP64 sum) for y = z + lphi (z may be NULL:
// y = lphi, or lphi NULL: y = z); ymax = -inf and ysum = 0 when every y is -inf.
__global__ void k_logit_stats(const float* __restrict__ z, const float* __restrict__ lphi, int64_t Nq,
                              float* __restrict__ ymax, double* __restrict__ ysum, float* __restrict__ yinv) {
  __shared__ double redd[32];
  __shared__ float redf[32];
  const int s = blockIdx.x;
  const float* zs = z ? z + (int64_t)s * Nq : nullptr;
  const float* ls = lphi ? lphi + (int64_t)s * Nq : nullptr;
  // where lphi is -inf the score is not read (the network may not have evaluated that q)
  auto y = [&](int64_t q) -> float {
    const float l = ls ? ls[q] : 0.f;
    return l == -INFINITY ? -INFINITY : (zs ? zs[q] : 0.f) + l;
  };
  float m = -INFINITY;
  for (int64_t q = threadIdx.x; q < Nq; q += blockDim.x) m = fmaxf(m, y(q));
  m = block_reduce_max(m, redf);
  double a = 0.0;
  if (m != -INFINITY)
    for (int64_t q = threadIdx.x; q < Nq; q += blockDim.x) a += (double)expf(y(q) - m);
  a = block_reduce_sum(a, redd);
  if (threadIdx.x == 0) {
    ymax[s] = m;
    ysum[s] = a;
    yinv[s] = a > 0.0 ? (float)(1.0 / a) : 0.f;
  }
}

struct Proposal {
  int mode = PHOEBE_SAMPLER_UNIFORM;  // LEARNED, UNIFORM or SHELL
  const float* z = nullptr;       // [S][Nq] network scores (LEARNED)
  const float* lp = nullptr;      // [S][Nq] log phi (LEARNED, SHELL)
  const float* zmax = nullptr;    // [S] stats of z + lp
  const double* zsum = nullptr;
  const float* zinv = nullptr;    // [S] 1 / zsum in FP32
  const float* pmax = nullptr;    // [S] stats of lp
  const double* psum = nullptr;
  const float* pinv = nullptr;    // [S] 1 / psum in FP32
  const int* kfirst = nullptr;    // [nkb + 1] first batch state of each batch k
  int64_t Nq = 1;
  double alpha = 1.0;
  // LEARNED: (1 - alpha) mean_s expf(z + lp - zmax_s) / zsum_s + alpha mean_s expf(lp - pmax_s) / psum_s,
  // SHELL: mean_s expf(lp - pmax_s) / psum_s, both over the states of k with psum > 0 (some phi > 0);
  // 1 / N_q when there is none, and for UNIFORM.  Evaluated in FP32 (the draws and their weights
  // use the same values, so the estimate stays unbiased); the running sums over q are FP64.
  __device__ __forceinline__ double value(int kb, int64_t q) const {
    if (mode == PHOEBE_SAMPLER_UNIFORM) return 1.0 / (double)Nq;
    const int s0 = kfirst[kb], s1 = kfirst[kb + 1];
    float an = 0.f, as = 0.f;
    int live = 0;
    for (int s = s0; s < s1; ++s) {
      if (!(psum[s] > 0.0)) continue;
      ++live;
      const float l = lp[(int64_t)s * Nq + q];
      if (l == -INFINITY) continue;  // phi = 0: no weight (the score is not read)
      as = fmaf(expf(l - pmax[s]), pinv[s], as);
      if (mode == PHOEBE_SAMPLER_LEARNED) an = fmaf(expf(z[(int64_t)s * Nq + q] + l - zmax[s]), zinv[s], an);
    }
    if (live == 0) return 1.0 / (double)Nq;
    if (mode == PHOEBE_SAMPLER_SHELL) return (double)as / (double)live;
    return ((1.0 - alpha) * (double)an + alpha * (double)as) / (double)live;
  }
};

// cdf[kb][q] = sum_{q' <= q} p_k(q') in FP64, one block per batch k; chunks of blockDim * 8 q in q
// order, 8 consecutive q per thread (a serial sum, then a block scan of the threads' totals).
__global__ void k_prop_cdf(Proposal P, double* __restrict__ cdf) {
  constexpr int V = 8;
  __shared__ double wsum[32];
  __shared__ double carry_s;
  const int kb = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) carry_s = 0.0;
  __syncthreads();
  double* out = cdf + (int64_t)kb * P.Nq;
  for (int64_t base = 0; base < P.Nq; base += (int64_t)blockDim.x * V) {
    const int64_t q0 = base + (int64_t)threadIdx.x * V;
    double loc[V];
    double run = 0.0;
#pragma unroll
    for (int i = 0; i < V; ++i) {
      run += q0 + i < P.Nq ? P.value(kb, q0 + i) : 0.0;
      loc[i] = run;
    }
    double v = run;  // inclusive warp scan of the threads' totals
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    double before = carry_s + (v - run);
    for (int i = 0; i < w; ++i) before += wsum[i];
#pragma unroll
    for (int i = 0; i < V; ++i)
      if (q0 + i < P.Nq) out[q0 + i] = before + loc[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < nwarp; ++i) t += wsum[i];
      carry_s += t;
    }
    __syncthreads();
  }
}

// Draw j of batch k: the smallest q with cdf[q] > u total; weight total / (N_q p_k(q)).
__global__ void k_draw(Proposal P, const double* __restrict__ cdf, const int* __restrict__ kb_grid, int nkb,
                       int ndraw, uint64_t seed, int* __restrict__ draw_q, double* __restrict__ draw_w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nkb * ndraw) return;
  const int kb = (int)(t / ndraw), j = (int)(t % ndraw);
  const double* cd = cdf + (int64_t)kb * P.Nq;
  const double total = cd[P.Nq - 1];
  const double target = is_uniform(seed, (uint32_t)j, (uint32_t)kb_grid[kb]) * total;
  int64_t lo = 0, hi = P.Nq - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cd[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  draw_q[t] = (int)lo;
  draw_w[t] = total / ((double)P.Nq * P.value(kb, lo));
}

// ------------------------------------------------------------------ c_nk(q) at drawn pairs
struct PairsArgs {
  const float2* T;          // [S][nRp][NM][NW]
  int nRp;
  const int* Rp;            // [nRp][3]
  const double* wp;         // [nRp]
  GridPhase gq;
  const cplx* cis_q;        // [L]
  const int* st_kb;         // [S]
  const int* st_k;          // [S]
  const int* st_b;          // [S]
  const double* epsF;       // [NF][NW]
  const int* draw_q;        // [nkb][ndraw] or NULL (q = j)
  const double* draw_w;     // [nkb][ndraw]
  int ndraw;
  GridMap gm;
  const float2* eps2;       // [NF][NW]
  const float* f32;         // [NF][NW]
  const float2* UH;         // [NF][NW][NW]
  const float2* Zf;         // [Nq][NM][NM]
  const float* omf;         // [Nq][NM]
  const float* nBf;         // [Nq][NM]
  float reach, inv_sigma, cut2, pref;
  float* c_out;             // [S][ndraw] or NULL
  double* gamma;            // accumulate (1/ndraw) sum_j c w, or NULL
  int64_t s_base;
  double inv_ndraw;
};

// One block per (state, chunk of draws); one thread per draw.  The state's T (stage-1 output)
// sits in shared memory and is read as a broadcast; each thread sums its q's phases against it,
// then rotates by U_{k+q}^dagger and Z_q and applies the delta weights like the full-grid epilogue.
template <int NW, int NM>
__global__ void __launch_bounds__(256, 1) k_pairs_sampled(PairsArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int E = NW * NM;
  float2* Ts = reinterpret_cast<float2*>(smem);
  float2* cs = Ts + (size_t)a.nRp * E;
  float* wps = reinterpret_cast<float*>(cs + a.gq.L);
  int* Rs = reinterpret_cast<int*>(wps + a.nRp);
  const int s = blockIdx.y;
  const float2* Tg = a.T + (int64_t)s * a.nRp * E;
  for (int i = threadIdx.x; i < a.nRp * E; i += blockDim.x) Ts[i] = Tg[i];
  for (int i = threadIdx.x; i < a.gq.L; i += blockDim.x) {
    const cplx v = a.cis_q[i];
    cs[i] = make_float2((float)v.re, (float)v.im);
  }
  for (int i = threadIdx.x; i < a.nRp; i += blockDim.x) {
    wps[i] = (float)a.wp[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) Rs[3 * i + d] = a.Rp[3 * i + d] * a.gq.mult[d];
  }
  __syncthreads();
  const int kb = a.st_kb[s];
  const int64_t kf = a.gm.k_to_fine(a.st_k[s]);
  int kc[3];
  grid_coords(kf, a.gm.nf, kc);
  const double e_n = a.epsF[kf * NW + a.st_b[s]];
  const float en_hi = (float)e_n, en_lo = (float)(e_n - (double)en_hi);
  const int L = a.gq.L;
  const int64_t j0 = (int64_t)blockIdx.x * kDrawChunk;
  const int64_t j1 = min(j0 + kDrawChunk, (int64_t)a.ndraw);
  double acc = 0.0;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int q = a.draw_q ? a.draw_q[(int64_t)kb * a.ndraw + j] : (int)j;
    int qc[3];
    grid_coords(q, a.gq.n, qc);
    float2 G[E];
#pragma unroll
    for (int e = 0; e < E; ++e) G[e] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int r = 0; r < a.nRp; ++r) {
      int x = (qc[0] * Rs[3 * r] + qc[1] * Rs[3 * r + 1] + qc[2] * Rs[3 * r + 2]) % L;
      x += x < 0 ? L : 0;
      float2 ph = cs[x];
      const float w = wps[r];
      ph.x *= w;
      ph.y *= w;
      const float2* tr = Ts + r * E;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const float2 tv = tr[e];
        G[e].x = fmaf(ph.x, tv.x, fmaf(-ph.y, tv.y, G[e].x));
        G[e].y = fmaf(ph.x, tv.y, fmaf(ph.y, tv.x, G[e].y));
      }
    }
    // k + q on the fine grid
    int fc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) fc[d] = (kc[d] + qc[d] * a.gm.sq[d]) % a.gm.nf[d];
    const int64_t kq = grid_flat(fc, a.gm.nf);
    float om[NM], nb[NM];
#pragma unroll
    for (int v = 0; v < NM; ++v) {
      om[v] = a.omf[(int64_t)q * NM + v];
      nb[v] = a.nBf[(int64_t)q * NM + v];
    }
    const float2* zq = a.Zf + (int64_t)q * NM * NM;
    float part = 0.f;
#pragma unroll 1
    for (int mp = 0; mp < NW; ++mp) {
      const float2 ee = a.eps2[kq * NW + mp];
      const float dm = (en_hi - ee.x) + (en_lo - ee.y);  // eps_n - eps_{m', k+q}
      if (!(fabsf(dm) < a.reach)) continue;
      const float2* uh = a.UH + (kq * NW + mp) * NW;
      float2 u[NW];
#pragma unroll
      for (int m = 0; m < NW; ++m) u[m] = uh[m];
      float2 t[NM];
#pragma unroll
      for (int sa = 0; sa < NM; ++sa) {
        t[sa] = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < NW; ++m) {
          const float2 gv = G[sa * NW + m];
          t[sa].x = fmaf(u[m].x, gv.x, fmaf(-u[m].y, gv.y, t[sa].x));
          t[sa].y = fmaf(u[m].x, gv.y, fmaf(u[m].y, gv.x, t[sa].y));
        }
      }
      const float f = a.f32[kq * NW + mp];
#pragma unroll
      for (int v = 0; v < NM; ++v) {
        float2 g = make_float2(0.f, 0.f);
#pragma unroll
        for (int sa = 0; sa < NM; ++sa) {
          const float2 zz = zq[sa * NM + v];
          g.x = fmaf(t[sa].x, zz.x, fmaf(-t[sa].y, zz.y, g.x));
          g.y = fmaf(t[sa].x, zz.y, fmaf(t[sa].y, zz.x, g.y));
        }
        const float t1 = (dm - om[v]) * a.inv_sigma;
        const float t2 = (dm + om[v]) * a.inv_sigma;
        float w = 0.f;
        if (t1 * t1 < a.cut2) w += (nb[v] + 1.f - f) * expf(-t1 * t1);
        if (t2 * t2 < a.cut2) w += (nb[v] + f) * expf(-t2 * t2);
        part = fmaf(g.x * g.x + g.y * g.y, w, part);
      }
    }
    const float cval = part * a.pref;
    if (a.c_out) a.c_out[(int64_t)s * a.ndraw + j] = cval;
    if (a.gamma) acc += (double)cval * a.draw_w[(int64_t)kb * a.ndraw + j];
  }
  if (a.gamma) {
    __shared__ double red[32];
    acc = block_reduce_sum(acc, red);
    if (threadIdx.x == 0 && acc != 0.0) atomicAdd(a.gamma + a.s_base + s, acc * a.inv_ndraw);
  }
}

__global__ void k_is_tables_ph(const cplx* __restrict__ Z, const double* __restrict__ om,
                               const double* __restrict__ nB, int64_t Q, int nm, float2* __restrict__ Zf,
                               float* __restrict__ omf, float* __restrict__ nBf) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Q * nm * nm) return;
  Zf[t] = make_float2((float)Z[t].re, (float)Z[t].im);
  if (t < Q * nm) {
    omf[t] = (float)om[t];
    nBf[t] = (float)nB[t];
  }
}

// Row sums of c (FP64), one block per state.
__global__ void k_row_sums(const float* __restrict__ c, int64_t Nq, double* __restrict__ out) {
  __shared__ double red[32];
  const float* cs = c + (int64_t)blockIdx.x * Nq;
  double a = 0.0;
  for (int64_t q = threadIdx.x; q < Nq; q += blockDim.x) a += (double)cs[q];
  a = block_reduce_sum(a, red);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

// ------------------------------------------------------------------ host: network passes
struct Acts {
  float *A1 = nullptr, *H1 = nullptr, *A2 = nullptr, *H2 = nullptr, *A3 = nullptr, *H3 = nullptr;
  float *D1 = nullptr, *D2 = nullptr;  // backward scratch
};

static int round_params(phoebe_gpu_ctx* c, float** Wr) {
  int st;
  float* w = (float*)c->bufs["mlp_w"].p;
  float* r = (float*)ensure(c, "mlp_r", sizeof(float) * kNParam, &st);
  if (!r) return st;
  k_round_params<<<(kNParam + 255) / 256, 256, 0, c->stream>>>(w, kNParam, r);
  TRY(launched(c, 1));
  *Wr = r;
  return PHOEBE_GPU_OK;
}

// Forward pass over rows (padded to 128): logits z[rows].  With `keep`, pre-activations and
// activations stay in the Acts buffers for a backward pass.
static int mlp_forward(phoebe_gpu_ctx* c, const float* Wr, const RowX& X, int64_t rows, float* z, bool keep,
                       Acts* act) {
  int st;
  const int64_t rp = round_up(std::max<int64_t>(rows, 1), 128);
  const size_t bytes = sizeof(float) * (size_t)rp * kNh;
  Acts a;
  a.H1 = (float*)ensure(c, "mlp_H1", bytes, &st);
  if (!a.H1) return st;
  a.H2 = (float*)ensure(c, "mlp_H2", bytes, &st);
  if (!a.H2) return st;
  if (keep) {
    a.A1 = (float*)ensure(c, "mlp_A1", bytes, &st);
    if (!a.A1) return st;
    a.A2 = (float*)ensure(c, "mlp_A2", bytes, &st);
    if (!a.A2) return st;
    a.A3 = (float*)ensure(c, "mlp_A3", bytes, &st);
    if (!a.A3) return st;
    a.H3 = (float*)ensure(c, "mlp_H3", bytes, &st);
    if (!a.H3) return st;
  } else {
    a.H3 = a.H1;  // layer 3 output overwrites layer 1's, which is no longer needed
  }
  k_layer1<<<(unsigned)((rp * kNh + 255) / 256), 256, 0, c->stream>>>(Wr, X, rp, a.A1, a.H1);
  TRY(launched(c, 1));
  GemmEpi e2;
  e2.bias = Wr + kOffB2;
  e2.pre = a.A2;
  TRY((sgemm<false, true, kEpiBiasSilu>(c, rp, kNh, kNh, a.H1, kNh, Wr + kOffW2, kNh, a.H2, kNh, e2)));
  GemmEpi e3;
  e3.bias = Wr + kOffB3;
  e3.pre = a.A3;
  TRY((sgemm<false, true, kEpiBiasSilu>(c, rp, kNh, kNh, a.H2, kNh, Wr + kOffW3, kNh, a.H3, kNh, e3)));
  k_head<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, c->stream>>>(a.H3, Wr, rows, z);
  TRY(launched(c, 1));
  if (act) *act = a;
  return PHOEBE_GPU_OK;
}

// Backward pass from dz (zero on padded rows) through the kept activations; adds into grad.
static int mlp_backward(phoebe_gpu_ctx* c, const float* Wr, const RowX& X, int64_t rows, const float* dz,
                        const Acts& a0, float* grad) {
  int st;
  const int64_t rp = round_up(std::max<int64_t>(rows, 1), 128);
  const size_t bytes = sizeof(float) * (size_t)rp * kNh;
  Acts a = a0;
  a.D1 = (float*)ensure(c, "mlp_D1", bytes, &st);
  if (!a.D1) return st;
  a.D2 = (float*)ensure(c, "mlp_D2", bytes, &st);
  if (!a.D2) return st;
  CK(c, cudaMemsetAsync(a.D1, 0, bytes, c->stream));
  const int64_t rpb = 512;
  const unsigned nblk = (unsigned)((rows + rpb - 1) / rpb);
  const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(2 * c->num_sms, rp / 512));
  // layer 4 and dA3 (rows beyond `rows` stay zero)
  k_head_back<<<nblk, kNh, 0, c->stream>>>(dz, a.H3, a.A3, Wr, rows, rpb, a.D1, grad);
  TRY(launched(c, 1));
  // layer 3: grad W3 += dA3^T H2, grad b3 += colsum dA3, dA2 = (dA3 W3) silu'(A2)
  TRY((sgemm<true, false, kEpiAtomic>(c, kNh, kNh, rp, a.D1, kNh, a.H2, kNh, grad + kOffW3, kNh, GemmEpi{}, splits)));
  k_colsum<<<nblk, kNh, 0, c->stream>>>(a.D1, rows, rpb, grad + kOffB3);
  TRY(launched(c, 1));
  GemmEpi d2;
  d2.aux = a.A2;
  TRY((sgemm<false, false, kEpiDsilu>(c, rp, kNh, kNh, a.D1, kNh, Wr + kOffW3, kNh, a.D2, kNh, d2)));
  // layer 2: grad W2 += dA2^T H1, grad b2, dA1 = (dA2 W2) silu'(A1)
  TRY((sgemm<true, false, kEpiAtomic>(c, kNh, kNh, rp, a.D2, kNh, a.H1, kNh, grad + kOffW2, kNh, GemmEpi{}, splits)));
  k_colsum<<<nblk, kNh, 0, c->stream>>>(a.D2, rows, rpb, grad + kOffB2);
  TRY(launched(c, 1));
  GemmEpi d1;
  d1.aux = a.A1;
  TRY((sgemm<false, false, kEpiDsilu>(c, rp, kNh, kNh, a.D2, kNh, Wr + kOffW2, kNh, a.D1, kNh, d1)));
  // layer 1
  k_layer1_back<<<nblk, kNh, 0, c->stream>>>(a.D1, X, rows, rpb, grad);
  TRY(launched(c, 1));
  return PHOEBE_GPU_OK;
}

// Scores z[s][q] of S states over every q of a grid: tcgen05 kernel (FP16 operands, FP32
// accumulation) or the CUDA-core forward pass (FP32 activations) in row chunks.  With a row list
// (device rows[r] = (s, q), r < *nrows) the tensor-core kernel scores those rows only; the
// CUDA-core pass scores every q regardless.
static int network_scores(phoebe_gpu_ctx* c, const float* qt, const float* feat, int S, int64_t Nq, bool tensor_cores,
                          float* z, const int2* rows = nullptr, const unsigned long long* nrows = nullptr) {
  int st;
  float* Wr;
  TRY(round_params(c, &Wr));
  if (tensor_cores) {
    __half* W2h = (__half*)ensure(c, "mlp_w2h", sizeof(__half) * kNh * kNh, &st);
    if (!W2h) return st;
    __half* W3h = (__half*)ensure(c, "mlp_w3h", sizeof(__half) * kNh * kNh, &st);
    if (!W3h) return st;
    int* err = (int*)ensure(c, "mlp_err", 64, &st);
    if (!err) return st;
    CK(c, cudaMemsetAsync(err, 0, 64, c->stream));
    if (mlp_tc_params(c->stream, Wr, W2h, W3h) != 0) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "parameter conversion for the tensor-core network failed");
    }
    MlpTcArgs ma;
    ma.W2h = W2h;
    ma.W3h = W3h;
    ma.P = Wr;
    ma.qt = qt;
    ma.feat = feat;
    ma.Nq = Nq;
    ma.tiles_per_state = (Nq + 127) / 128;
    ma.ntiles = (int64_t)S * ma.tiles_per_state;
    ma.z = z;
    ma.err = err;
    ma.rows = rows;
    ma.nrows = nrows;
    if (mlp_tc_launch(c->stream, c->num_sms, ma) != 0) {
      cudaGetLastError();
      return fail(c, PHOEBE_GPU_ERR_CUDA, "launch of the tensor-core network failed");
    }
    c->launches += 2;
    int herr = 0;
    CK(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (herr) return fail(c, PHOEBE_GPU_ERR_TIMEOUT, "a tensor-core network wait ran out; results discarded");
    return PHOEBE_GPU_OK;
  }
  const int64_t spc = std::max<int64_t>(1, kMaxRows / Nq);  // states per network chunk
  for (int64_t s0 = 0; s0 < S; s0 += spc) {
    const int64_t ns = std::min<int64_t>(spc, S - s0);
    RowX X;
    X.qt = qt;
    X.feat = feat + s0 * 4;
    X.Nq = Nq;
    X.rows = ns * Nq;
    TRY(mlp_forward(c, Wr, X, X.rows, z + s0 * Nq, false, nullptr));
  }
  return PHOEBE_GPU_OK;
}

// ------------------------------------------------------------------ host: one batch of states
template <int NW, int NM>
int is_batch(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, const IsBatch& b,
             const IsTables& t, double* raw) {
  IsRequest* rq = c->isreq;
  const int nRp = c->nRp;
  const int64_t Nq = (int64_t)gm.nq[0] * gm.nq[1] * gm.nq[2];
  const int S = b.S;
  int st;
  const bool learned = rq->mode == 1 && p->sampler == PHOEBE_SAMPLER_LEARNED;
  const bool shell = rq->mode == 1 && (p->sampler == PHOEBE_SAMPLER_LEARNED || p->sampler == PHOEBE_SAMPLER_SHELL);
  Timer tm;
  tm.begin(c);
  // per-state features
  float* feat = nullptr;
  if (rq->feat_out || learned) {
    feat = rq->feat_out ? rq->feat_out + b.s_base * 4 : (float*)ensure(c, "is_feat", sizeof(float) * S * 4, &st);
    if (!feat) return st;
    GridPhase gf = make_phase(gm.nf);
    cplx* cis_f;
    TRY(cis_table(c, gf, "cis_el", &cis_f));
    k_state_features<<<S, 128, 0, c->stream>>>(b.st_k, b.st_b, gm, gf, cis_f, (const cplx*)c->bufs["H"].p,
                                               (const int*)c->bufs["RH"].p, (const double*)c->bufs["wH"].p,
                                               c->nRH, c->nw, t.epsF, t.UF, p->mu_eV, feat);
    TRY(launched(c, 1));
  }
  // phonon tables by q (FP32)
  float2* Zf = (float2*)ensure(c, "is_Zf", sizeof(float2) * Nq * NM * NM, &st);
  if (!Zf) return st;
  float* omf = (float*)ensure(c, "is_omf", sizeof(float) * Nq * NM, &st);
  if (!omf) return st;
  float* nBf = (float*)ensure(c, "is_nBf", sizeof(float) * Nq * NM, &st);
  if (!nBf) return st;
  k_is_tables_ph<<<(unsigned)((Nq * NM * NM + 255) / 256), 256, 0, c->stream>>>(t.Zq, t.omega, t.nB, Nq, NM, Zf,
                                                                                 omf, nBf);
  TRY(launched(c, 1));

  PairsArgs a{};
  a.T = b.T;
  a.nRp = nRp;
  a.Rp = (const int*)c->bufs["Rp"].p;
  a.wp = (const double*)c->bufs["wp"].p;
  a.gq = make_phase(gm.nq);
  cplx* cis_q;
  TRY(cis_table(c, a.gq, "cis_q", &cis_q));
  a.cis_q = cis_q;
  a.st_kb = b.st_kb;
  a.st_k = b.st_k;
  a.st_b = b.st_b;
  a.epsF = t.epsF;
  a.gm = gm;
  a.eps2 = t.eps2;
  a.f32 = t.f32;
  a.UH = t.UH;
  a.Zf = Zf;
  a.omf = omf;
  a.nBf = nBf;
  a.reach = (float)(t.omega_max + p->delta_cut_sigmas * p->sigma_eV) * 1.0001f;
  a.inv_sigma = (float)(1.0 / p->sigma_eV);
  a.cut2 = (float)(p->delta_cut_sigmas * p->delta_cut_sigmas);
  a.pref = (float)(2.0 * kPi / (kSqrtPi * p->sigma_eV));
  a.s_base = b.s_base;

  // log of the shell factor of every q for every state of the batch (proposal, or requested output)
  float* lphi = nullptr;
  if (shell || (rq->mode == 2 && rq->lphi_out)) {
    lphi = rq->mode == 2 ? rq->lphi_out + b.s_base * Nq : (float*)ensure(c, "is_lphi", sizeof(float) * S * Nq, &st);
    if (!lphi) return st;
    dim3 g((unsigned)((Nq + 255) / 256), (unsigned)S);
    const double xcut = p->delta_cut_sigmas * p->sigma_eV;
    k_shell_log<<<g, 256, 0, c->stream>>>(b.st_k, b.st_b, gm, Nq, t.epsF, t.eps2, t.fF, t.omega, omf, nBf, NW,
                                          NM, p->omega_cut_eV, 1.0 / p->sigma_eV, xcut,
                                          (t.omega_max + xcut) * (1.0 + 1e-12), lphi);
    TRY(launched(c, 1));
  }
  if (rq->mode == 2) {
    a.draw_q = nullptr;
    a.draw_w = nullptr;
    a.ndraw = (int)Nq;
    a.c_out = rq->c_out + b.s_base * Nq;
    a.gamma = nullptr;
    a.inv_ndraw = 1.0 / (double)Nq;
  } else {
    const int ndraw = (int)std::ceil(p->sample_fraction * (double)Nq - 1e-9);
    // scores of every q for every state of the batch
    Proposal P;
    P.mode = p->sampler;
    P.Nq = Nq;
    P.alpha = learned ? p->mix_alpha : 1.0;
    std::vector<int> kfirst(b.nkb + 1, 0);
    for (int s = 0; s < S; ++s) kfirst[(*b.st_kb_host)[s] + 1] = s + 1;
    for (int k = 1; k <= b.nkb; ++k) kfirst[k] = std::max(kfirst[k], kfirst[k - 1]);
    void* d_kfirst;
    TRY(upload(c, "is_kfirst", kfirst.data(), sizeof(int) * (b.nkb + 1), &d_kfirst));
    P.kfirst = (const int*)d_kfirst;
    if (learned) {
      float* z = (float*)ensure(c, "is_z", sizeof(float) * S * Nq, &st);
      if (!z) return st;
      float* zmax = (float*)ensure(c, "is_zmax", sizeof(float) * S, &st);
      if (!zmax) return st;
      float* zinv = (float*)ensure(c, "is_zinv", sizeof(float) * S, &st);
      if (!zinv) return st;
      double* zsum = (double*)ensure(c, "is_zsum", sizeof(double) * S, &st);
      if (!zsum) return st;
      float* qt = (float*)ensure(c, "is_qt", sizeof(float) * Nq * 3, &st);
      if (!qt) return st;
      k_wrapped_q<<<(unsigned)((Nq + 255) / 256), 256, 0, c->stream>>>(gm.nq[0], gm.nq[1], gm.nq[2], Nq, qt);
      TRY(launched(c, 1));
      // the network runs on the rows with phi > 0 only (elsewhere the proposal is 0)
      int2* rows = (int2*)ensure(c, "is_rows", sizeof(int2) * S * Nq, &st);
      if (!rows) return st;
      unsigned long long* nrows = (unsigned long long*)ensure(c, "is_nrows", 64, &st);
      if (!nrows) return st;
      CK(c, cudaMemsetAsync(nrows, 0, sizeof(unsigned long long), c->stream));
      k_shell_rows<<<S, 1024, 0, c->stream>>>(lphi, Nq, rows, nrows);
      TRY(launched(c, 1));
      TRY(network_scores(c, qt, feat, S, Nq, c->cc >= 100 && !p->sampler_fp32_network, z, rows, nrows));
      k_logit_stats<<<S, 256, 0, c->stream>>>(z, lphi, Nq, zmax, zsum, zinv);
      TRY(launched(c, 1));
      P.z = z;
      P.zmax = zmax;
      P.zsum = zsum;
      P.zinv = zinv;
    }
    if (shell) {
      float* pmax = (float*)ensure(c, "is_pmax", sizeof(float) * S, &st);
      if (!pmax) return st;
      double* psum = (double*)ensure(c, "is_psum", sizeof(double) * S, &st);
      if (!psum) return st;
      float* pinv = (float*)ensure(c, "is_pinv", sizeof(float) * S, &st);
      if (!pinv) return st;
      k_logit_stats<<<S, 256, 0, c->stream>>>(nullptr, lphi, Nq, pmax, psum, pinv);
      TRY(launched(c, 1));
      P.lp = lphi;
      P.pmax = pmax;
      P.psum = psum;
      P.pinv = pinv;
    }
    double* cdf = (double*)ensure(c, "is_cdf", sizeof(double) * b.nkb * Nq, &st);
    if (!cdf) return st;
    k_prop_cdf<<<b.nkb, 512, 0, c->stream>>>(P, cdf);
    int* dq = (int*)ensure(c, "is_dq", sizeof(int) * b.nkb * (int64_t)ndraw, &st);
    if (!dq) return st;
    double* dw = (double*)ensure(c, "is_dw", sizeof(double) * b.nkb * (int64_t)ndraw, &st);
    if (!dw) return st;
    const int64_t nd = (int64_t)b.nkb * ndraw;
    k_draw<<<(unsigned)((nd + 255) / 256), 256, 0, c->stream>>>(P, cdf, b.kb, b.nkb, ndraw, p->seed, dq, dw);
    TRY(launched(c, 2));
    a.draw_q = dq;
    a.draw_w = dw;
    a.ndraw = ndraw;
    a.c_out = nullptr;
    a.gamma = raw;
    a.inv_ndraw = 1.0 / (double)ndraw;
  }
  tm.end(c, &c->stats.sampler_ms);

  const size_t smem = sizeof(float2) * ((size_t)nRp * NW * NM + a.gq.L) + sizeof(float) * nRp + sizeof(int) * 3 * nRp;
  if (smem > 227 * 1024)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED,
                "sampled q sums keep one state's R_p sum in shared memory: %zu bytes needed, 227 KB available", smem);
  CK(c, allow_dynamic_smem(k_pairs_sampled<NW, NM>));
  tm.begin(c);
  dim3 grid((unsigned)((a.ndraw + kDrawChunk - 1) / kDrawChunk), (unsigned)S);
  k_pairs_sampled<NW, NM><<<grid, 256, smem, c->stream>>>(a);
  TRY(launched(c, 1));
  tm.end(c, &c->stats.stage2_ms);
  c->stats.stage2_launches++;
  c->stats.pairs_executed += (int64_t)S * a.ndraw;
  c->stats.stage2_flops += 8.0 * (double)S * a.ndraw * nRp * NW * NM;
  return PHOEBE_GPU_OK;
}

template int is_batch<8, 6>(phoebe_gpu_ctx*, const phoebe_gpu_rta_params*, const GridMap&, const IsBatch&,
                            const IsTables&, double*);
template int is_batch<2, 3>(phoebe_gpu_ctx*, const phoebe_gpu_rta_params*, const GridMap&, const IsBatch&,
                            const IsTables&, double*);
template int is_batch<1, 3>(phoebe_gpu_ctx*, const phoebe_gpu_rta_params*, const GridMap&, const IsBatch&,
                            const IsTables&, double*);

// ------------------------------------------------------------------ host: helpers of the entry points
static int mlp_buffers(phoebe_gpu_ctx* c) {
  int st;
  const size_t n = sizeof(float) * kNParam;
  for (const char* name : {"mlp_w", "mlp_m", "mlp_v", "mlp_g"})
    if (!ensure(c, name, n, &st)) return st;
  return PHOEBE_GPU_OK;
}

static int reset_optimiser(phoebe_gpu_ctx* c) {
  CK(c, cudaMemsetAsync(c->bufs["mlp_m"].p, 0, sizeof(float) * kNParam, c->stream));
  CK(c, cudaMemsetAsync(c->bufs["mlp_v"].p, 0, sizeof(float) * kNParam, c->stream));
  c->adam_t = 0;
  return PHOEBE_GPU_OK;
}

// Full-grid pass producing c_nk(q), the log shell factor and the features of every active state of
// `grid` into device buffers "isc_c" [n][Nq], "isc_lphi" [n][Nq] and "isc_feat" [n][4]; host copies of
// k and band.
static int contributions_dev(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* grid, int* n_out,
                             std::vector<int>* hk, std::vector<int>* hb, float** cdev, float** fdev,
                             float** ldev) {
  phoebe_gpu_rta_params p2 = *grid;
  p2.sampler = PHOEBE_SAMPLER_FULL;
  if (p2.precision == PHOEBE_PREC_FP64)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "q-resolved contributions need a tensor-core precision (1..6)");
  int n = 0;
  TRY(linewidths(c, &p2, &n, nullptr, nullptr, nullptr, false));
  const int64_t Nq = (int64_t)p2.nq[0] * p2.nq[1] * p2.nq[2];
  int st;
  const int64_t nn = std::max(n, 1);
  float* cd = (float*)ensure(c, "isc_c", sizeof(float) * nn * Nq, &st);
  if (!cd) return st;
  float* fd = (float*)ensure(c, "isc_feat", sizeof(float) * nn * 4, &st);
  if (!fd) return st;
  float* ld = (float*)ensure(c, "isc_lphi", sizeof(float) * nn * Nq, &st);
  if (!ld) return st;
  double* gd = (double*)ensure(c, "isc_gamma", sizeof(double) * nn, &st);
  if (!gd) return st;
  int* kd = (int*)ensure(c, "isc_k", sizeof(int) * nn, &st);
  if (!kd) return st;
  int* bd = (int*)ensure(c, "isc_b", sizeof(int) * nn, &st);
  if (!bd) return st;
  CK(c, cudaMemsetAsync(cd, 0, sizeof(float) * nn * Nq, c->stream));
  IsRequest req;
  req.mode = 2;
  req.c_out = cd;
  req.feat_out = fd;
  req.lphi_out = ld;
  c->isreq = &req;
  int cap = n;
  const int r = linewidths(c, &p2, &cap, kd, bd, gd, true);
  c->isreq = nullptr;
  TRY(r);
  hk->resize(n);
  hb->resize(n);
  if (n > 0) {
    CK(c, cudaMemcpyAsync(hk->data(), kd, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(hb->data(), bd, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  *n_out = n;
  *cdev = cd;
  *fdev = fd;
  *ldev = ld;
  return PHOEBE_GPU_OK;
}

// One Adam step on groups of rows (explicit rows, or training states x every q); loss added to *loss_dev.
static int train_step(phoebe_gpu_ctx* c, const RowX& X, int64_t rows, const int64_t* off_dev, int G, const RowT& T,
                      double* loss_dev, const phoebe_gpu_train_opts* o) {
  int st;
  float* Wr;
  TRY(round_params(c, &Wr));
  float* grad = (float*)c->bufs["mlp_g"].p;
  CK(c, cudaMemsetAsync(grad, 0, sizeof(float) * kNParam, c->stream));
  const int64_t rp = round_up(std::max<int64_t>(rows, 1), 128);
  float* z = (float*)ensure(c, "mlp_z", sizeof(float) * rp, &st);
  if (!z) return st;
  float* dz = (float*)ensure(c, "mlp_dz", sizeof(float) * rp, &st);
  if (!dz) return st;
  CK(c, cudaMemsetAsync(dz, 0, sizeof(float) * rp, c->stream));
  Acts a;
  TRY(mlp_forward(c, Wr, X, rows, z, true, &a));
  k_softmax_ce<<<G, 256, 0, c->stream>>>(z, off_dev, T, 1.0f / (float)G, dz, loss_dev);
  TRY(launched(c, 1));
  TRY(mlp_backward(c, Wr, X, rows, dz, a, grad));
  if (o) {
    c->adam_t++;
    const float bc1 = (float)(1.0 - std::pow(o->beta1, (double)c->adam_t));
    const float bc2 = (float)(1.0 - std::pow(o->beta2, (double)c->adam_t));
    k_adam<<<(kNParam + 255) / 256, 256, 0, c->stream>>>((float*)c->bufs["mlp_w"].p, (float*)c->bufs["mlp_m"].p,
                                                         (float*)c->bufs["mlp_v"].p, grad, kNParam, (float)o->lr,
                                                         (float)o->beta1, (float)o->beta2, (float)o->eps, bc1, bc2);
    TRY(launched(c, 1));
  }
  return PHOEBE_GPU_OK;
}

}  // namespace phx

using namespace phx;

// ------------------------------------------------------------------ C ABI
extern "C" int phoebe_gpu_sampler_init(phoebe_gpu_ctx* c, uint64_t seed) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  TRY(mlp_buffers(c));
  std::vector<float> w(kNParam, 0.f);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  auto fill = [&](int off, int n, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (int i = 0; i < n; ++i) w[off + i] = (float)(a * U(rng));
  };
  fill(kOffW1, kNh * kNin, kNin);
  fill(kOffW2, kNh * kNh, kNh);
  fill(kOffW3, kNh * kNh, kNh);
  fill(kOffW4, kNh, kNh);
  CK(c, cudaMemcpyAsync(c->bufs["mlp_w"].p, w.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, c->stream));
  TRY(reset_optimiser(c));
  CK(c, cudaStreamSynchronize(c->stream));
  c->have_mlp = true;
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_sampler_load(phoebe_gpu_ctx* c, const float* params, int64_t n) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!params || n != kNParam)
    return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_load: need %d parameters, got %lld", kNParam, (long long)n);
  TRY(mlp_buffers(c));
  CK(c, cudaMemcpyAsync(c->bufs["mlp_w"].p, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice, c->stream));
  TRY(reset_optimiser(c));
  CK(c, cudaStreamSynchronize(c->stream));
  c->have_mlp = true;
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_sampler_save(phoebe_gpu_ctx* c, float* params, int64_t n) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!params || n != kNParam)
    return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_save: need room for %d parameters, got %lld", kNParam, (long long)n);
  if (!c->have_mlp) return fail(c, PHOEBE_GPU_ERR_ORDER, "sampler_save: no parameters (init, load or train first)");
  CK(c, cudaMemcpyAsync(params, c->bufs["mlp_w"].p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

extern "C" void phoebe_gpu_train_opts_default(phoebe_gpu_train_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->epochs = 60;
  o->states_per_step = 64;
  o->lr = 3e-3;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->eps = 1e-8;
}

extern "C" int phoebe_gpu_sampler_train(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* grid,
                                        const phoebe_gpu_train_opts* o, double* loss_per_epoch) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  c->launches = 0;
  if (!grid || !o) return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_train: NULL params or options");
  if (o->epochs < 1 || o->states_per_step < 1 || !(o->lr > 0.0) || !(o->beta1 >= 0.0 && o->beta1 < 1.0) ||
      !(o->beta2 >= 0.0 && o->beta2 < 1.0) || !(o->eps > 0.0))
    return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_train: bad options");
  for (int i = 0; i < 4; ++i)
    if (o->reserved[i]) return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_train: reserved fields must be zero");
  if (!c->have_mlp) return fail(c, PHOEBE_GPU_ERR_ORDER, "sampler_train: call sampler_init or sampler_load first");
  int n = 0;
  std::vector<int> hk, hb;
  float *cd, *fd, *ld;
  TRY(contributions_dev(c, grid, &n, &hk, &hb, &cd, &fd, &ld));
  const int64_t Nq = (int64_t)grid->nq[0] * grid->nq[1] * grid->nq[2];
  int st;
  // states with a non-zero sum are the training set
  double* sums = (double*)ensure(c, "tr_sums", sizeof(double) * std::max(n, 1), &st);
  if (!sums) return st;
  if (n > 0) {
    k_row_sums<<<n, 256, 0, c->stream>>>(cd, Nq, sums);
    TRY(launched(c, 1));
  }
  std::vector<double> hs(n);
  if (n > 0) CK(c, cudaMemcpyAsync(hs.data(), sums, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  std::vector<int> train;
  for (int i = 0; i < n; ++i)
    if (hs[i] > 0.0) train.push_back(i);
  if (train.empty()) return fail(c, PHOEBE_GPU_ERR_ARG, "sampler_train: no state of the grid has a non-zero Gamma");
  float* qt = (float*)ensure(c, "tr_qt", sizeof(float) * Nq * 3, &st);
  if (!qt) return st;
  k_wrapped_q<<<(unsigned)((Nq + 255) / 256), 256, 0, c->stream>>>(grid->nq[0], grid->nq[1], grid->nq[2], Nq, qt);
  TRY(launched(c, 1));
  const int B = std::max(1, (int)std::min<int64_t>(o->states_per_step, std::max<int64_t>(1, kMaxRows / Nq)));
  std::vector<int64_t> off(B + 1);
  for (int g = 0; g <= B; ++g) off[g] = (int64_t)g * Nq;
  void* d_off;
  TRY(upload(c, "tr_off", off.data(), sizeof(int64_t) * (B + 1), &d_off));
  double* loss_dev = (double*)ensure(c, "tr_loss", sizeof(double), &st);
  if (!loss_dev) return st;
  std::mt19937_64 rng(o->seed);
  for (int ep = 0; ep < o->epochs; ++ep) {
    std::shuffle(train.begin(), train.end(), rng);
    CK(c, cudaMemsetAsync(loss_dev, 0, sizeof(double), c->stream));
    int steps = 0;
    for (size_t i0 = 0; i0 < train.size(); i0 += B) {
      const int G = (int)std::min<size_t>(B, train.size() - i0);
      void* d_states;
      TRY(upload(c, "tr_states", train.data() + i0, sizeof(int) * G, &d_states));
      RowX X;
      X.qt = qt;
      X.feat = fd;
      X.states = (const int*)d_states;
      X.Nq = Nq;
      X.rows = (int64_t)G * Nq;
      RowT T;
      T.c = cd;
      T.lpc = ld;
      T.states = (const int*)d_states;
      T.Nq = Nq;
      TRY(train_step(c, X, X.rows, (const int64_t*)d_off, G, T, loss_dev, o));
      ++steps;
    }
    double l = 0.0;
    CK(c, cudaMemcpyAsync(&l, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (loss_per_epoch) loss_per_epoch[ep] = l / std::max(steps, 1);
  }
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_q_contributions(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* params, int* n_states,
                                          int32_t* k_index, int32_t* band, float* cq, float* features,
                                          float* log_shell) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (!n_states) return fail(c, PHOEBE_GPU_ERR_ARG, "n_states is NULL");
  if (!params) return fail(c, PHOEBE_GPU_ERR_ARG, "params is NULL");
  if (!cq) {
    phoebe_gpu_rta_params p2 = *params;
    p2.sampler = PHOEBE_SAMPLER_FULL;
    return linewidths(c, &p2, n_states, nullptr, nullptr, nullptr, false);
  }
  const int cap = *n_states;
  int n = 0;
  std::vector<int> hk, hb;
  float *cd, *fd, *ld;
  TRY(contributions_dev(c, params, &n, &hk, &hb, &cd, &fd, &ld));
  if (cap < n) return fail(c, PHOEBE_GPU_ERR_ARG, "output capacity %d is below the %d active states", cap, n);
  const int64_t Nq = (int64_t)params->nq[0] * params->nq[1] * params->nq[2];
  if (n > 0) {
    CK(c, cudaMemcpyAsync(cq, cd, sizeof(float) * (size_t)n * Nq, cudaMemcpyDeviceToHost, c->stream));
    if (features) CK(c, cudaMemcpyAsync(features, fd, sizeof(float) * n * 4, cudaMemcpyDeviceToHost, c->stream));
    if (log_shell)
      CK(c, cudaMemcpyAsync(log_shell, ld, sizeof(float) * (size_t)n * Nq, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  if (k_index) memcpy(k_index, hk.data(), sizeof(int) * n);
  if (band) memcpy(band, hb.data(), sizeof(int) * n);
  *n_states = n;
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_mlp_loss_grad(phoebe_gpu_ctx* c, int64_t n_rows, const float* x, int n_groups,
                                        const int64_t* group_off, const float* target, const float* log_prior,
                                        float* logits, double* loss, float* grad) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  c->launches = 0;
  if (n_rows < 1 || !x || n_rows > kMaxRows) return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_loss_grad: n_rows in 1..%lld",
                                                         (long long)kMaxRows);
  if (!c->have_mlp) return fail(c, PHOEBE_GPU_ERR_ORDER, "mlp_loss_grad: no parameters (init, load or train first)");
  if (target) {
    if (n_groups < 1 || !group_off) return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_loss_grad: groups missing");
    if (group_off[0] != 0 || group_off[n_groups] != n_rows)
      return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_loss_grad: group offsets must run from 0 to n_rows");
    for (int g = 0; g < n_groups; ++g)
      if (group_off[g + 1] <= group_off[g])
        return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_loss_grad: group offsets must increase");
  }
  int st;
  void *dx, *dt = nullptr, *doff = nullptr;
  TRY(upload(c, "lg_x", x, sizeof(float) * n_rows * kNin, &dx));
  RowX X;
  X.x = (const float*)dx;
  X.rows = n_rows;
  const int64_t rp = round_up(n_rows, 128);
  float* z = (float*)ensure(c, "mlp_z", sizeof(float) * rp, &st);
  if (!z) return st;
  if (!target) {
    float* Wr;
    TRY(round_params(c, &Wr));
    TRY(mlp_forward(c, Wr, X, n_rows, z, false, nullptr));
  } else {
    TRY(upload(c, "lg_t", target, sizeof(float) * n_rows, &dt));
    TRY(upload(c, "lg_off", group_off, sizeof(int64_t) * (n_groups + 1), &doff));
    double* loss_dev = (double*)ensure(c, "lg_loss", sizeof(double), &st);
    if (!loss_dev) return st;
    CK(c, cudaMemsetAsync(loss_dev, 0, sizeof(double), c->stream));
    RowT T;
    T.t = (const float*)dt;
    if (log_prior) {
      void* dlp;
      TRY(upload(c, "lg_lp", log_prior, sizeof(float) * n_rows, &dlp));
      T.lp = (const float*)dlp;
    }
    TRY(train_step(c, X, n_rows, (const int64_t*)doff, n_groups, T, loss_dev, nullptr));
    if (loss) CK(c, cudaMemcpyAsync(loss, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad)
      CK(c, cudaMemcpyAsync(grad, c->bufs["mlp_g"].p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c->stream));
  }
  if (logits) CK(c, cudaMemcpyAsync(logits, z, sizeof(float) * n_rows, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_is_uniforms(phoebe_gpu_ctx* c, uint64_t seed, int32_t k, int64_t n, double* u) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  if (n < 1 || !u || k < 0 || n > ((int64_t)1 << 31)) return fail(c, PHOEBE_GPU_ERR_ARG, "is_uniforms: bad arguments");
  int st;
  double* d = (double*)ensure(c, "isu", sizeof(double) * n, &st);
  if (!d) return st;
  k_is_uniforms<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(seed, (uint32_t)k, n, d);
  c->launches++;
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(u, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}

extern "C" int phoebe_gpu_mlp_scores(phoebe_gpu_ctx* c, int n_states, const float* features, const int32_t nq[3],
                                     int tensor_cores, float* z) {
  if (!c) return PHOEBE_GPU_ERR_ARG;
  c->launches = 0;
  if (n_states < 1 || !features || !nq || !z) return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_scores: bad arguments");
  for (int i = 0; i < 3; ++i)
    if (nq[i] < 1 || nq[i] > 4096) return fail(c, PHOEBE_GPU_ERR_ARG, "mlp_scores: grid sizes must be in 1..4096");
  if (!c->have_mlp) return fail(c, PHOEBE_GPU_ERR_ORDER, "mlp_scores: no parameters (init, load or train first)");
  if (tensor_cores && c->cc < 100)
    return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "tensor-core network scores need an sm_10x GPU");
  const int64_t Nq = (int64_t)nq[0] * nq[1] * nq[2];
  int st;
  void* dfeat;
  TRY(upload(c, "ms_feat", features, sizeof(float) * 4 * n_states, &dfeat));
  float* qt = (float*)ensure(c, "ms_qt", sizeof(float) * Nq * 3, &st);
  if (!qt) return st;
  float* zd = (float*)ensure(c, "ms_z", sizeof(float) * Nq * n_states, &st);
  if (!zd) return st;
  k_wrapped_q<<<(unsigned)((Nq + 255) / 256), 256, 0, c->stream>>>(nq[0], nq[1], nq[2], Nq, qt);
  TRY(launched(c, 1));
  c->stats.sampler_ms = 0.0;  // with profiling on: the device time of the scoring alone
  Timer tm;
  tm.begin(c);
  TRY(network_scores(c, qt, (const float*)dfeat, n_states, Nq, tensor_cores != 0, zd));
  tm.end(c, &c->stats.sampler_ms);
  CK(c, cudaMemcpyAsync(z, zd, sizeof(float) * Nq * n_states, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return PHOEBE_GPU_OK;
}
