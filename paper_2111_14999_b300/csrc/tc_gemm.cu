// Reduced-precision linewidth path on tcgen05 tensor cores.
#include "tc.h"

struct TcState {};

namespace phx {

void destroy_tc_state(phoebe_gpu_ctx* c) {
  delete c->tc;
  c->tc = nullptr;
}

int run_tc(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
           const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF, const cplx* UF,
           const double* fF, const double* omega, const double* nB, const cplx* Zq, double* raw) {
  return fail(c, PHOEBE_GPU_ERR_UNSUPPORTED, "precision %d is not implemented yet", p->precision);
}

}  // namespace phx
