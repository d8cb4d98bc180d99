// Reduced-precision (tensor-core) linewidth path interface.
#pragma once

#include <vector>

#include "pipeline.h"

namespace phx {

int run_tc(phoebe_gpu_ctx* c, const phoebe_gpu_rta_params* p, const GridMap& gm, int64_t ns,
           const std::vector<int>& hk, const int* st_k, const int* st_b, const double* epsF, const cplx* UF,
           const double* fF, const double* omega, const double* nB, const cplx* Zq, double* raw);

}  // namespace phx
