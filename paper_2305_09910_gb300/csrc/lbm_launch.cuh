// lbm_launch.cuh -- host launchers of the templated kernels, one instantiation per
// (stencil, storage precision) translation unit (kern_inst.cu built with -DLBM_Q, -DLBM_S).
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_h2.cuh"
#include "lbm_mlp.cuh"

namespace lbm {

struct Launch {
  dim3 grid, block;
  cudaStream_t stream;
};

template <int Q, class S>
cudaError_t launch_step(const KParams& p, int closure, int parity, const Launch& L, bool stats = false,
                        int* nws = nullptr, int coll = 0);
template <int Q, class S>
cudaError_t launch_step_mlp(const KParams& p, int mode, cudaStream_t stream, int nsm);
template <int Q, class S>
cudaError_t launch_export(const KParams& p, int parity, int mode, const ExportArgs& a, const Launch& L);
template <int Q, class S>
cudaError_t launch_init_eq(const KParams& p, const float* rho, const float* u, const Launch& L);
template <int Q, class S>
cudaError_t launch_set_pop(const KParams& p, const float* df, const Launch& L);
template <int Q, class S>
cudaError_t launch_step_multi(const KParams& p0, const KParams& p1, int closure, int coll, bool aa, int odd0,
                              int nsteps, cudaStream_t stream, int nsm);

#define LBM_DECLARE_INSTANCE(Q, S)                                                                 \
  extern template cudaError_t launch_step<Q, S>(const KParams&, int, int, const Launch&, bool, int*, int); \
  extern template cudaError_t launch_step_mlp<Q, S>(const KParams&, int, cudaStream_t, int);      \
  extern template cudaError_t launch_export<Q, S>(const KParams&, int, int, const ExportArgs&,     \
                                                  const Launch&);                                  \
  extern template cudaError_t launch_init_eq<Q, S>(const KParams&, const float*, const float*,     \
                                                   const Launch&);                                 \
  extern template cudaError_t launch_set_pop<Q, S>(const KParams&, const float*, const Launch&);     \
  extern template cudaError_t launch_step_multi<Q, S>(const KParams&, const KParams&, int, int, bool, int, \
                                                      int, cudaStream_t, int);

LBM_DECLARE_INSTANCE(19, float)
LBM_DECLARE_INSTANCE(19, __half)
LBM_DECLARE_INSTANCE(19, __nv_bfloat16)
LBM_DECLARE_INSTANCE(27, float)
LBM_DECLARE_INSTANCE(27, __half)
LBM_DECLARE_INSTANCE(27, __nv_bfloat16)

}  // namespace lbm
