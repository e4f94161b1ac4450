// lbm_async.cuh -- the AA / pull step with its loads staged in shared memory by per-lane
// asynchronous copies (cp.async), a few cells ahead of the arithmetic.
//
// Why: the direct kernels are latency-bound.  A thread there holds its Q loaded values in
// registers, so the bytes a multiprocessor keeps in flight are capped by its register file
// and by the share of warps that are in their load phase.  Here a thread walks ZC cells along
// z; while it collides cell z it already has the copies of cells z+1 .. z+NST-1 in flight
// into shared memory, which costs no registers.  Each lane copies exactly the 4-byte values
// it will read (its own gather addresses), so there is no halo and no block barrier: a
// thread only ever reads its own copies, after cp.async.wait_group.
//
// Which cells take the staged path: the even AA launch stages every cell (own slots).  The
// gathering launches stage cells of rows away from the y and z faces, where the gather
// address of an interior cell is base + cell (with the periodic x wrap of the row ends);
// cells of the face rows and every non-interior cell load directly, as in the direct kernel.
//
// Hazards: in the AA launches each slot is read and written by its one owning cell (the
// boundary rules are involutions), so staging the loads of later cells of the same thread
// cannot observe a write of this launch to a slot those cells use.  Staged values of cells
// that then load directly are discarded.  The two-grid pull reads one array and writes the
// other.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ void cp_async4(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// True when the cell's gather addresses are the interior ones (no y or z face crossed).
__device__ __forceinline__ bool inner_row(const KParams& p, int y, int z) {
  return y > 0 && y < p.ny - 1 && z > 0 && z < p.nz - 1;
}

// Issues the staged copies of cell (x, y, z) into stage buffer `st` ([Q][128] floats, this
// thread's column t) and commits them as one group (an empty group when nothing is staged).
template <int Q, int PAR>
__device__ __forceinline__ void stage_cell(const KParams& p, int x, int y, int z, unsigned st, int t) {
  if (x < p.nx && (PAR == 0 || inner_row(p, y, z))) {
    const int cell = cidx(p, x, y, z);
    if (PAR == 0) {
#pragma unroll
      for (int i = 0; i < Q; i++) cp_async4(st + (i * 128 + t) * 4, plane_ptr<float>(p, i) + cell);
    } else {
      const int cp = cell + (x == 0 ? p.nx : 0);
      const int cm = cell - (x == p.nx - 1 ? p.nx : 0);
#pragma unroll
      for (int i = 0; i < Q; i++) {
        const float* base = static_cast<const float*>(PAR == 2 ? p.gb[i] : p.ga[i]);
        cp_async4(st + (i * 128 + t) * 4, base + (cx(i) > 0 ? cp : cx(i) < 0 ? cm : cell));
      }
    }
  }
  cp_async_commit();
}

#ifndef LBM_ASYNC_MINB
#define LBM_ASYNC_MINB 8
#endif

// LOAD / STORE modes as in k_step.  Block (32, 4); grid (nxp/32, ceil(ny/4), ceil(nz/ZC)).
// FP32 storage only (the copies are 4 bytes, one population each).
template <int Q, int CL, int LOAD, int STORE, int ZC, int NST>
__global__ void __launch_bounds__(128, LBM_ASYNC_MINB) k_step_async(const __grid_constant__ KParams p) {
  extern __shared__ __align__(16) float sbuf[];  // [NST][Q][128]
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int t = threadIdx.y * 32 + threadIdx.x;
  const int z0 = blockIdx.z * ZC;
  if (y >= p.ny) return;  // whole warp; no block barrier follows
  const int zend = min(p.nz, z0 + ZC);
  const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(sbuf));
  constexpr unsigned SB = Q * 128 * 4;  // bytes per stage
#pragma unroll
  for (int s = 0; s < NST - 1; s++) {
    if (z0 + s < zend) stage_cell<Q, LOAD>(p, x, y, z0 + s, sbase + s * SB, t);
    else cp_async_commit();
  }
#pragma unroll 1
  for (int z = z0; z < zend; z++) {
    const int k = z - z0;
    const int zn = z + NST - 1;
    if (zn < zend) stage_cell<Q, LOAD>(p, x, y, zn, sbase + ((k + NST - 1) % NST) * SB, t);
    else cp_async_commit();
    cp_async_wait<NST - 1>();  // the group of cell z is complete
    const int cell = cidx(p, x, y, z);
    const int cls = x < p.nx ? cls_at(p, cell) : CLS_SKIP;
    float f[Q];
    unsigned outmask = 0;
    const bool staged = LOAD == 0 ? (cls == CLS_INTERIOR || cls == CLS_WRAP) : (cls == CLS_INTERIOR && inner_row(p, y, z));
    if (staged) {
      const float* row = sbuf + (k % NST) * (Q * 128) + t;
#pragma unroll
      for (int i = 0; i < Q; i++) f[i] = row[i * 128];
    } else {
      load_state<Q, float, LOAD>(p, x, y, z, cell, cls, f, outmask);
    }
    outflow_fix<Q>(p, x, f, outmask);
    if (cls == CLS_SKIP) continue;
    const float rho = collide<Q, CL, float>(p, f);
    if (!(rho > 0.f && rho < 3.0e38f)) atomicOr(p.status, 1);
    store_state<Q, float, STORE>(p, x, y, z, cell, cls, f);
  }
  cp_async_wait<0>();
}

}  // namespace lbm
