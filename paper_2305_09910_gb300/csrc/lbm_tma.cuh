// lbm_tma.cuh -- the AA step with its loads staged through shared memory by the Tensor
// Memory Accelerator (1-D bulk copies, cp.async.bulk) in a multi-stage mbarrier pipeline.
//
// Why: the direct-load kernels are latency-bound (ncu: long-scoreboard stalls dominate, 64
// registers allow ~43 % of the warp slots, the odd launch's x-shifted pulls reach under half
// of the DRAM bandwidth).  Here each persistent CTA walks a list of tiles (one 128-cell row
// segment of one (y, z) row); one thread issues, per tile, one bulk copy per direction (the
// row segment the tile needs, plus a 16-byte halo on each side for the odd launch's x-shifted
// pulls) and one for the cell classes, STAGES tiles ahead of the computing warps.  The warps
// read their 19/27 values from shared memory at fixed offsets and write results directly.
//
// Hazards: in both AA launches every slot a tile reads is written only by that tile (the
// pull and the write-back of the odd launch touch the same slots), so prefetching later
// tiles cannot observe a write of this launch to a slot it uses; halo bytes of neighbouring
// tiles are copied but never used.  Every mbarrier wait is bounded; on a timeout the kernel
// sets status bit 1, waits (bounded) for its own copies in flight and returns.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int TMA_TX = 128;      // cells per tile (4 warps x 32)
constexpr int TMA_STAGES = 3;    // tiles in flight per CTA

template <class S>
struct TmaGeom {
  static constexpr int H = 16 / (int)sizeof(S);  // halo elements (16 bytes)
  template <int PAR>
  __host__ __device__ static constexpr int rowlen() { return PAR ? TMA_TX + 2 * H : TMA_TX; }
  template <int Q, int PAR>
  __host__ __device__ static constexpr int stage_bytes() {
    return Q * rowlen<PAR>() * (int)sizeof(S) + TMA_TX;  // rows + class bytes
  }
  template <int Q, int PAR>
  __host__ __device__ static constexpr int smem_bytes() {
    return TMA_STAGES * stage_bytes<Q, PAR>() + TMA_STAGES * 8;
  }
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity (about a second of spinning at most).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < (1 << 22); it++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

struct TileIdx {
  int x0, y, z, txr;
};

__device__ __forceinline__ TileIdx tile_of(const KParams& p, long long t) {
  const int nseg = (p.nxp + TMA_TX - 1) / TMA_TX;
  TileIdx ti;
  const int seg = (int)(t % nseg);
  const long long r = t / nseg;
  ti.y = (int)(r % p.ny);
  ti.z = (int)(r / p.ny);
  ti.x0 = seg * TMA_TX;
  ti.txr = min(TMA_TX, p.nxp - ti.x0);
  return ti;
}

// Source row of direction i for the odd launch (x - c_i), or -1 when it lies across a
// non-periodic face (cells that need it take the boundary path).
__device__ __forceinline__ int src_row(const KParams& p, int y, int z, int i) {
  int ys = y - cy(i), zs = z - cz(i);
  if (ys < 0 || ys >= p.ny) {
    if (p.face[2] != FACE_PERIODIC) return -1;
    ys = ys < 0 ? ys + p.ny : ys - p.ny;
  }
  if (zs < 0 || zs >= p.nz) {
    if (p.face[4] != FACE_PERIODIC) return -1;
    zs = zs < 0 ? zs + p.nz : zs - p.nz;
  }
  return (zs * p.ny + ys) * p.nxp;
}

// Producer (one thread): the copies of tile t into stage buffer `st`, completing on `bar`.
template <int Q, class S, int PAR>
__device__ __noinline__ void issue_tile(const KParams& p, long long t, unsigned char* st, unsigned bar) {
  using G = TmaGeom<S>;
  constexpr int RL = G::template rowlen<PAR>();
  const TileIdx ti = tile_of(p, t);
  const int base_row = (ti.z * p.ny + ti.y) * p.nxp;
  unsigned bytes = (unsigned)ti.txr;  // classes
  int xa = ti.x0, xb = ti.x0 + ti.txr;
  if (PAR) {
    xa = max(ti.x0 - G::H, 0);
    xb = min(ti.x0 + ti.txr + G::H, p.nxp);
  }
  int rows[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    rows[i] = PAR ? src_row(p, ti.y, ti.z, i) : base_row;
    if (rows[i] >= 0) bytes += (unsigned)((xb - xa) * (int)sizeof(S));
  }
  mbar_expect_tx(bar, bytes);
  bulk_g2s(smem_u32(st + Q * RL * (int)sizeof(S)), p.cls + base_row + ti.x0, (unsigned)ti.txr, bar);
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (rows[i] < 0) continue;
    const int plane = PAR ? opp(i) : i;
    const S* src = plane_ptr<S>(p, plane) + rows[i] + xa;
    const int off = PAR ? xa - (ti.x0 - G::H) : 0;
    bulk_g2s(smem_u32(st + (i * RL + off) * (int)sizeof(S)), src, (unsigned)((xb - xa) * (int)sizeof(S)), bar);
  }
}

template <int Q, class S, int CL, int PAR>
__global__ void __launch_bounds__(TMA_TX, 5) k_step_tma(const __grid_constant__ KParams p,
                                                                           long long ntiles) {
  using G = TmaGeom<S>;
  constexpr int RL = G::template rowlen<PAR>();
  constexpr int SB = G::template stage_bytes<Q, PAR>();
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stage0 = smem;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + TMA_STAGES * SB);
  const int t = threadIdx.x;
  if (t == 0) {
    for (int s = 0; s < TMA_STAGES; s++) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    for (int s = 0; s < TMA_STAGES; s++) {
      const long long tt = blockIdx.x + (long long)s * gridDim.x;
      if (tt < ntiles) issue_tile<Q, S, PAR>(p, tt, stage0 + s * SB, smem_u32(bars + s));
    }
  }
  int j = 0;
  for (long long tt = blockIdx.x; tt < ntiles; tt += gridDim.x, j++) {
    const int s = j % TMA_STAGES;
    const unsigned parity = (unsigned)((j / TMA_STAGES) & 1);
    unsigned char* st = stage0 + s * SB;
    const int timed_out = !mbar_wait(smem_u32(bars + s), parity);
    if (__syncthreads_or(timed_out)) {  // CTA-uniform decision
      if (t == 0) atomicOr(p.status, 2);
      // drain this CTA's copies in flight (bounded) before leaving
      for (int k = 0; k < TMA_STAGES; k++) {
        const long long tk = tt + (long long)k * gridDim.x;
        if (tk < ntiles) mbar_wait(smem_u32(bars + (j + k) % TMA_STAGES), (unsigned)(((j + k) / TMA_STAGES) & 1));
      }
      return;
    }
    const TileIdx ti = tile_of(p, tt);
    const int x = ti.x0 + t, y = ti.y, z = ti.z;
    const int cell = cidx(p, x, y, z);
    const S* rows = reinterpret_cast<const S*>(st);
    int cls = CLS_SKIP;
    if (t < ti.txr && x < p.nx) cls = st[Q * RL * (int)sizeof(S) + t];
    float f[Q];
    unsigned outmask = 0;
    // cells on the periodic x seam pull across the row end: their sources are not in this
    // tile's rows, so they take the direct path like boundary cells
    const bool seam = PAR && (x == 0 || x >= p.nx - 1);
    if ((cls == CLS_INTERIOR || cls == CLS_WRAP) && !seam) {
      if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < Q; i++) f[i] = ld<S>(rows + i * RL + t);
      } else {
#pragma unroll
        for (int i = 0; i < Q; i++) f[i] = ld<S>(rows + i * RL + G::H + t - cx(i));
      }
    } else {
      load_state<Q, S, PAR>(p, x, y, z, cell, cls, f, outmask);
    }
    __syncthreads();  // every thread is done with stage s
    if (t == 0) {
      const long long tn = tt + (long long)TMA_STAGES * gridDim.x;
      if (tn < ntiles) issue_tile<Q, S, PAR>(p, tn, st, smem_u32(bars + s));
    }
    outflow_fix<Q>(p, x, f, outmask);
    if (cls == CLS_SKIP) continue;
    const float rho = collide<Q, CL, float, acc_form<S>>(p, f);
    if (!(rho > 0.f && rho < 3.0e38f)) atomicOr(p.status, 1);
    store_state<Q, S, PAR>(p, x, y, z, cell, cls, f);
  }
}

}  // namespace lbm
