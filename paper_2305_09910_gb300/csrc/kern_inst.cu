// kern_inst.cu -- instantiates the kernels and launchers for one (stencil, precision) pair.
// Compiled once per pair with -DLBM_Q=19|27 and -DLBM_S=float|__half|__nv_bfloat16.
#include "lbm_launch.cuh"

#ifndef LBM_Q
#error "LBM_Q must be defined"
#endif
#ifndef LBM_S
#error "LBM_S must be defined"
#endif

namespace lbm {

template <int Q, class S>
cudaError_t launch_step(const KParams& p, int closure, int parity, const Launch& L) {
  if (parity == 0) {
    if (closure == CL_NONE) k_step<Q, S, CL_NONE, 0><<<L.grid, L.block, 0, L.stream>>>(p);
    else if (closure == CL_SMAG) k_step<Q, S, CL_SMAG, 0><<<L.grid, L.block, 0, L.stream>>>(p);
    else k_step<Q, S, CL_MLP, 0><<<L.grid, L.block, 0, L.stream>>>(p);
  } else {
    if (closure == CL_NONE) k_step<Q, S, CL_NONE, 1><<<L.grid, L.block, 0, L.stream>>>(p);
    else if (closure == CL_SMAG) k_step<Q, S, CL_SMAG, 1><<<L.grid, L.block, 0, L.stream>>>(p);
    else k_step<Q, S, CL_MLP, 1><<<L.grid, L.block, 0, L.stream>>>(p);
  }
  return cudaGetLastError();
}

template <int Q, class S, int PAR>
static void export_par(const KParams& p, int mode, const ExportArgs& a, const Launch& L) {
  switch (mode) {
    case EX_POP: k_export<Q, S, PAR, EX_POP><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
    case EX_MOM: k_export<Q, S, PAR, EX_MOM><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
    case EX_SUM: k_export<Q, S, PAR, EX_SUM><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
    default: k_export<Q, S, PAR, EX_STATS><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
  }
}

template <int Q, class S>
cudaError_t launch_export(const KParams& p, int parity, int mode, const ExportArgs& a, const Launch& L) {
  if (parity == 0) export_par<Q, S, 0>(p, mode, a, L);
  else export_par<Q, S, 1>(p, mode, a, L);
  return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_init_eq(const KParams& p, const float* rho, const float* u, const Launch& L) {
  k_init_eq<Q, S><<<L.grid, L.block, 0, L.stream>>>(p, rho, u);
  return cudaGetLastError();
}

template <int Q, class S>
cudaError_t launch_set_pop(const KParams& p, const float* df, const Launch& L) {
  k_set_pop<Q, S><<<L.grid, L.block, 0, L.stream>>>(p, df);
  return cudaGetLastError();
}

template cudaError_t launch_step<LBM_Q, LBM_S>(const KParams&, int, int, const Launch&);
template cudaError_t launch_export<LBM_Q, LBM_S>(const KParams&, int, int, const ExportArgs&, const Launch&);
template cudaError_t launch_init_eq<LBM_Q, LBM_S>(const KParams&, const float*, const float*, const Launch&);
template cudaError_t launch_set_pop<LBM_Q, LBM_S>(const KParams&, const float*, const Launch&);

}  // namespace lbm
