// Allocation-free band energies: Wannier-interpolated H(k) at explicit k points
// and its Hermitian eigensolve, with the eigensolver's work arrays in a
// file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: host programs that share the GPU with a framework which has
// already reserved almost all device memory for its own pool (a cudaMalloc
// would fail there), and latency-sensitive callers that cannot accept the
// device-wide synchronisation cudaMalloc/cudaFree may imply.  They pass their
// own input and output buffers; the only scratch is the static array below.
#include <mutex>

#include "kernels.cuh"

namespace {

// Work arrays of the eigensolver (two complex n_k x nw x nw arrays) plus
// a convergence word at the end.  Every GPU that loads the library keeps this
// allocation until the process exits.
constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes + 256];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

}  // namespace

extern "C" int phoebe_gpu_bands_noalloc(int nw, int n_R, const int32_t* R, const double* w, const double* H,
                                        int n_k, const double* k, double* eps, double* U, void* cuda_stream) {
  using namespace phx;
  if (nw < 1 || nw > kMaxNw || n_R < 1 || n_k < 1 || !R || !w || !H || !k || !eps) return PHOEBE_GPU_ERR_ARG;
  const size_t per = (size_t)n_k * nw * nw;
  if (2 * per * sizeof(cplx) > kNoallocScratchBytes) return PHOEBE_GPU_ERR_NOMEM;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return PHOEBE_GPU_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // every call ends with a read-back and a stream synchronisation, which a stream capture
  // does not allow: refuse before anything is enqueued, so the caller's capture stays valid
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) return PHOEBE_GPU_ERR_ARG;
  void* base = nullptr;
  {
    // one-time set-up per device, with that device current: device address of the scratch array
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return PHOEBE_GPU_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  cplx* A = reinterpret_cast<cplx*>(base);
  cplx* V = A + per;
  int* status = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kNoallocScratchBytes);
  // the array keeps the previous call's contents: the convergence word must start at zero
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  const int E = nw * nw;
  dim3 g((unsigned)((n_k + 127) / 128), (unsigned)E);
  k_fourier_points_c<<<g, 128, 0, s>>>(reinterpret_cast<const cplx*>(H), R, w, n_R, E, k, n_k, A);
  if (eigh_launch(s, A, V, nw, n_k, eps, reinterpret_cast<cplx*>(U), status)) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  int hs = 0;
  if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return PHOEBE_GPU_ERR_CUDA;
  }
  return hs ? PHOEBE_GPU_ERR_NOTCONVERGED : PHOEBE_GPU_OK;
}
