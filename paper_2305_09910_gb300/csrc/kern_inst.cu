// kern_inst.cu -- instantiates the kernels and launchers for one (stencil, precision) pair.
// Compiled once per pair with -DLBM_Q=19|27 and -DLBM_S=float|__half|__nv_bfloat16.
#include <algorithm>
#include <type_traits>

#include "lbm_launch.cuh"

#ifndef LBM_Q
#error "LBM_Q must be defined"
#endif
#ifndef LBM_S
#error "LBM_S must be defined"
#endif

namespace lbm {

// stats: also write the warp-slot plane statistics of the starting state (p.stats_w); *nws
// receives the number of warp slots per row.  coll: 0 TRT, 1 MRT (D3Q19, one cell per thread),
// 2 regularised (one cell per thread).
// listed cells up to which a split step runs them in its x-pair grid
#ifndef LBM_LIST_FUSE_MAX
#define LBM_LIST_FUSE_MAX (1ll << 18)
#endif

template <int Q, class S, int LOAD, int STORE, bool STATS>
static void step_mode_s(const KParams& p, int closure, const Launch& L, int coll, int* nws) {
  if constexpr (Q == 19) {
    if (coll == 1) {
      if (nws) *nws = p.nxp / 32;
      if (closure == CL_NONE) k_step<Q, S, CL_NONE, LOAD, STORE, STATS, 1><<<L.grid, L.block, 0, L.stream>>>(p);
      else k_step<Q, S, CL_SMAG, LOAD, STORE, STATS, 1><<<L.grid, L.block, 0, L.stream>>>(p);
      return;
    }
  }
  if (coll == 2) {  // regularised collision: one cell per thread, every stencil and storage
    if (nws) *nws = p.nxp / 32;
    if (closure == CL_NONE) k_step<Q, S, CL_NONE, LOAD, STORE, STATS, 2><<<L.grid, L.block, 0, L.stream>>>(p);
    else k_step<Q, S, CL_SMAG, LOAD, STORE, STATS, 2><<<L.grid, L.block, 0, L.stream>>>(p);
    return;
  }
  // half storage, gather step of two-grid pull without statistics (both stencils; D3Q19 unless
  // built with LBM_SPLIT19=0): the x-pair step over the interior cells (populations packed in
  // registers through the collision for D3Q27) and the cells the handle listed (rules, wraps):
  // a short list in extra z slices of the pair grid (no launch of its own: the 2:1 refined box's
  // small FP16 lattices 69.5 -> 71.9 % of the copy bandwidth), a long one as k_step_list at its
  // own occupancy (the D3Q27 bluff body's 1.5 M listed cells: 74.6 % against 73.0 % in the pair
  // grid, whose 95 registers leave fewer warps for the latency-bound list).  The other D3Q27
  // half steps take the one-cell kernel.
  if constexpr (sizeof(S) == 2 && (Q == 27 || LBM_SPLIT19) && LOAD == 2 && STORE == 2 && !STATS) {
    if (p.split && coll == 0) {
      dim3 g = L.grid;
      g.x = (p.nxp + 63) / 64;
      const long long per = 128ll * g.x * g.y;  // listed cells per extra z slice
      const long long extra = (p.nblist + per - 1) / per;
      const bool fused = p.nblist <= LBM_LIST_FUSE_MAX && g.z + extra <= 65535;
      if (fused) g.z += (unsigned)extra;
      if (closure == CL_NONE) k_step_h2<Q, S, CL_NONE, 2, 2, false, true><<<g, L.block, 0, L.stream>>>(p);
      else k_step_h2<Q, S, CL_SMAG, 2, 2, false, true><<<g, L.block, 0, L.stream>>>(p);
      if (!fused) {
        const unsigned nb = (unsigned)((p.nblist + 127) / 128);
        if (closure == CL_NONE) k_step_list<Q, S, CL_NONE><<<nb, 128, 0, L.stream>>>(p);
        else k_step_list<Q, S, CL_SMAG><<<nb, 128, 0, L.stream>>>(p);
      }
      return;
    }
  }
  // half storage, D3Q19: x-pairs, 64 x per warp
  if constexpr (sizeof(S) == 2 && Q == 19) {
    dim3 g = L.grid;
    g.x = (p.nxp + 63) / 64;
    if (nws) *nws = (int)g.x;
    if (closure == CL_NONE) k_step_h2<Q, S, CL_NONE, LOAD, STORE, STATS><<<g, L.block, 0, L.stream>>>(p);
    else k_step_h2<Q, S, CL_SMAG, LOAD, STORE, STATS><<<g, L.block, 0, L.stream>>>(p);
    return;
  }
  if (nws) *nws = p.nxp / 32;
  if (closure == CL_NONE) k_step<Q, S, CL_NONE, LOAD, STORE, STATS><<<L.grid, L.block, 0, L.stream>>>(p);
  else k_step<Q, S, CL_SMAG, LOAD, STORE, STATS><<<L.grid, L.block, 0, L.stream>>>(p);
}

template <int Q, class S, int LOAD, int STORE>
static void step_mode(const KParams& p, int closure, const Launch& L, bool stats, int coll, int* nws) {
  if (stats) step_mode_s<Q, S, LOAD, STORE, true>(p, closure, L, coll, nws);
  else step_mode_s<Q, S, LOAD, STORE, false>(p, closure, L, coll, nws);
}

// mode: 0 AA even, 1 AA odd, 2 first pull step after an import, 3 pull step
template <int Q, class S>
cudaError_t launch_step(const KParams& p, int closure, int mode, const Launch& L, bool stats, int* nws, int coll) {
  switch (mode) {
    case 0: step_mode<Q, S, 0, 0>(p, closure, L, stats, coll, nws); break;
    case 1: step_mode<Q, S, 1, 1>(p, closure, L, stats, coll, nws); break;
    case 2: step_mode<Q, S, 0, 2>(p, closure, L, stats, coll, nws); break;
    default: step_mode<Q, S, 2, 2>(p, closure, L, stats, coll, nws); break;
  }
  return cudaGetLastError();
}

// nsteps plain steps in one cooperative launch (k_step_multi): pull alternates p0 and p1, AA
// alternates the even and odd forms on p0 starting with `odd0`.  The grid is what fits on
// the device at once (a cooperative launch refuses more, it never waits).
template <int Q, class S, int CL, int COLL, bool AA>
static cudaError_t multi_one(const KParams2& pp, int nsteps, int odd0, cudaStream_t stream, int nsm) {
  auto kern = k_step_multi<Q, S, CL, COLL, AA>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const KParams& p = pp.p[0];
  const long long ntiles = (long long)(p.nxp / 32) * ((p.ny + 3) / 4) * p.nz;
  const int blocks = (int)std::min<long long>(ntiles, (long long)per_sm * nsm);
  void* args[] = {(void*)&pp, (void*)&nsteps, (void*)&odd0};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(32, 4), args, 0, stream);
}

template <int Q, class S, int COLL, bool AA>
static cudaError_t multi_cl(const KParams2& pp, int closure, int nsteps, int odd0, cudaStream_t st, int nsm) {
  return closure == CL_NONE ? multi_one<Q, S, CL_NONE, COLL, AA>(pp, nsteps, odd0, st, nsm)
                            : multi_one<Q, S, CL_SMAG, COLL, AA>(pp, nsteps, odd0, st, nsm);
}

template <int Q, class S, bool AA>
static cudaError_t multi_coll(const KParams2& pp, int closure, int coll, int nsteps, int odd0, cudaStream_t st,
                              int nsm) {
  if constexpr (Q == 19) {
    if (coll == 1) return multi_cl<Q, S, 1, AA>(pp, closure, nsteps, odd0, st, nsm);
  }
  if (coll == 2) return multi_cl<Q, S, 2, AA>(pp, closure, nsteps, odd0, st, nsm);
  return multi_cl<Q, S, 0, AA>(pp, closure, nsteps, odd0, st, nsm);
}

template <int Q, class S>
cudaError_t launch_step_multi(const KParams& p0, const KParams& p1, int closure, int coll, bool aa, int odd0,
                              int nsteps, cudaStream_t stream, int nsm) {
  KParams2 pp;
  pp.p[0] = p0;
  pp.p[1] = p1;
  return aa ? multi_coll<Q, S, true>(pp, closure, coll, nsteps, odd0, stream, nsm)
            : multi_coll<Q, S, false>(pp, closure, coll, nsteps, odd0, stream, nsm);
}

template <int Q, class S, int LOAD, int STORE>
static cudaError_t mlp_one(const KParams& p, cudaStream_t stream, int nsm) {
  constexpr int smem = (int)sizeof(MlpSmem);
  auto kern = k_step_mlp<Q, S, LOAD, STORE>;
  static int blocks_per_sm = 0;  // per instantiation, found once (one: the kernel allocates TMEM)
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 128 * MLP_NG, smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const long long ntiles = (long long)(p.nxp / 32) * ((p.ny + 3) / 4) * p.nz;
  if (ntiles >= (1ll << 31)) return cudaErrorInvalidValue;  // tile indices are 32-bit in the kernel
  const long long groups = (ntiles + MLP_NG - 1) / MLP_NG;
  const long long grid = std::min<long long>(groups, (long long)nsm * blocks_per_sm);
  kern<<<(unsigned)grid, dim3(32, 4 * MLP_NG, 1), smem, stream>>>(p, ntiles);
  return cudaGetLastError();
}

// The step with the learned closure (tensor-core hidden layer); mode as in launch_step.
template <int Q, class S>
cudaError_t launch_step_mlp(const KParams& p, int mode, cudaStream_t stream, int nsm) {
  switch (mode) {
    case 0: return mlp_one<Q, S, 0, 0>(p, stream, nsm);
    case 1: return mlp_one<Q, S, 1, 1>(p, stream, nsm);
    case 2: return mlp_one<Q, S, 0, 2>(p, stream, nsm);
    default: return mlp_one<Q, S, 2, 2>(p, stream, nsm);
  }
}

template <int Q, class S, int PAR>
static void export_par(const KParams& p, int mode, const ExportArgs& a, const Launch& L) {
  const dim3 rows((unsigned)p.ny, (unsigned)p.nz);
  switch (mode) {
    case EX_POP: k_export<Q, S, PAR, EX_POP><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
    case EX_MOM: k_export<Q, S, PAR, EX_MOM><<<L.grid, L.block, 0, L.stream>>>(p, a); break;
    case EX_SUM:
      k_row_sums<Q, S, PAR, EX_SUM><<<rows, ROW_THREADS, 0, L.stream>>>(p, a.partial);
      k_row_total<EX_SUM><<<1, 256, 0, L.stream>>>(a.partial, p.ny, p.nz, a.sums);
      break;
    default:
      k_row_sums<Q, S, PAR, EX_STATS><<<rows, ROW_THREADS, 0, L.stream>>>(p, a.partial);
      k_row_total<EX_STATS><<<(unsigned)p.ny, 256, 0, L.stream>>>(a.partial, p.ny, p.nz, a.sums);
      break;
  }
}

template <int Q, class S>
cudaError_t launch_export(const KParams& p, int parity, int mode, const ExportArgs& a, const Launch& L) {
  if (parity == 0) export_par<Q, S, 0>(p, mode, a, L);
  else if (parity == 1) export_par<Q, S, 1>(p, mode, a, L);
  else export_par<Q, S, 2>(p, mode, a, L);
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

template cudaError_t launch_step<LBM_Q, LBM_S>(const KParams&, int, int, const Launch&, bool, int*, int);
template cudaError_t launch_step_mlp<LBM_Q, LBM_S>(const KParams&, int, cudaStream_t, int);
template cudaError_t launch_export<LBM_Q, LBM_S>(const KParams&, int, int, const ExportArgs&, const Launch&);
template cudaError_t launch_init_eq<LBM_Q, LBM_S>(const KParams&, const float*, const float*, const Launch&);
template cudaError_t launch_set_pop<LBM_Q, LBM_S>(const KParams&, const float*, const Launch&);
template cudaError_t launch_step_multi<LBM_Q, LBM_S>(const KParams&, const KParams&, int, int, bool, int, int,
                                                     cudaStream_t, int);

}  // namespace lbm
