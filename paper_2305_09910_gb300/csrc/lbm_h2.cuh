// lbm_h2.cuh -- the step for half-precision storage with two x-adjacent cells per thread.
//
// A lane owns cells (x, x+1), x even, so every slot the pair owns in a direction with
// c_x = 0 (and every own-cell slot) is one aligned 32-bit word holding both cells' 16-bit
// values: one load and one store move two populations.  Slots shifted in x by the odd AA
// gather (c_x != 0) straddle two words and move as two 16-bit accesses.  The loaded words
// stay packed (one register per direction for both cells) until the collision, which runs on
// both cells at once in the packed FP32x2 pipe (float2 operands: FFMA2/FADD2/FMUL2); the two
// results are rounded and packed into one word each.  This halves the memory instructions,
// the address arithmetic and the arithmetic instructions per cell and doubles the bytes a
// thread keeps in flight (LBM_H2_VEC=0 collides the two cells one after the other instead).
//
// Warps with any non-interior cell (boundary rules, periodic y/z wrap, skipped cells) take
// the one-cell code for each of their two cells instead; the zero-gradient outflow passes
// what cell x-1 receives from the lane that owns it (nx % 32 != 1 keeps x = nx-1 off lane 0).
// Block (32, 4) covers 64 x 4 cells of one z plane; grid (ceil(nxp/64), ceil(ny/4), nz).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class S> __device__ __forceinline__ float lo_of(uint32_t v);
template <class S> __device__ __forceinline__ float hi_of(uint32_t v);
template <> __device__ __forceinline__ float lo_of<__half>(uint32_t v) {
  return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
}
template <> __device__ __forceinline__ float hi_of<__half>(uint32_t v) {
  return __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}
template <> __device__ __forceinline__ float lo_of<__nv_bfloat16>(uint32_t v) { return __uint_as_float(v << 16); }
template <> __device__ __forceinline__ float hi_of<__nv_bfloat16>(uint32_t v) {
  return __uint_as_float(v & 0xffff0000u);
}

template <class S> __device__ __forceinline__ uint32_t pack2(float a, float b);  // a in the low half
template <> __device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 16-bit pattern of v rounded to the storage precision (round to nearest even)
template <class S> __device__ __forceinline__ uint32_t bits16(float v);
template <> __device__ __forceinline__ uint32_t bits16<__half>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <> __device__ __forceinline__ uint32_t bits16<__nv_bfloat16>(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Checked 32-bit (two cells) and 16-bit (one cell) population accesses.
__device__ __forceinline__ uint32_t ld32(const KParams& p, const void* a) {
  return chk(p, a, 4, CHK_POP) ? *static_cast<const uint32_t*>(a) : 0u;
}
__device__ __forceinline__ void st32(const KParams& p, void* a, uint32_t v) {
  if (chk(p, a, 4, CHK_POP)) *static_cast<uint32_t*>(a) = v;
}
__device__ __forceinline__ uint32_t ld16(const KParams& p, const void* a) {
  return chk(p, a, 2, CHK_POP) ? *static_cast<const unsigned short*>(a) : 0u;
}
__device__ __forceinline__ void st16(const KParams& p, void* a, uint32_t v) {
  if (chk(p, a, 2, CHK_POP)) *static_cast<unsigned short*>(a) = (unsigned short)v;
}

// Zero-gradient outflow for x-pairs: cell x-1 of lane t's first cell is lane t-1's second.
template <int Q>
__device__ __forceinline__ void outflow_fix2(const KParams& p, int x0, float (&fa)[Q], float (&fb)[Q],
                                             unsigned oa, unsigned ob) {
  if (!p.outflow) return;
  if (!(x0 <= p.nx - 1 && p.nx - 1 < x0 + 64)) return;  // warp-uniform
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (cx(i) != -1) continue;
    const float v = __shfl_up_sync(0xffffffffu, fb[i], 1);
    if (ob & (1u << i)) fb[i] = fa[i];  // x-1 is this lane's first cell (never itself an outflow cell)
    if (oa & (1u << i)) fa[i] = v;
  }
}

// Slot offsets of the two cells' sources in a direction with c_x != 0 (periodic x wrap).
__device__ __forceinline__ void xsrc(int c, const KParams& p, int x, int cell, int& ca, int& cb) {
  if (c > 0) {  // sources x-1, x
    ca = cell + (x == 0 ? p.nx : 0);
    cb = cell + 1;
  } else {       // sources x+1, x+2
    ca = cell;
    cb = cell + 1 - (x + 1 == p.nx - 1 ? p.nx : 0);
  }
}

// One-cell code for both cells of a lane (warps with a non-interior cell).  Kept out of
// line so that the rare path does not take registers from the fast one.
template <int Q, class S, int CL, int LOAD, int STORE, bool STATS>
__device__ __noinline__ void pair_fallback(const KParams& p, int x, int y, int z, int cell, int clsA, int clsB,
                                           float (&v)[NSTAT]) {
  float fa[Q], fb[Q];
  unsigned oa, ob;
  load_state<Q, S, LOAD>(p, x, y, z, cell, clsA, fa, oa);
  load_state<Q, S, LOAD>(p, x + 1, y, z, cell + 1, clsB, fb, ob);
  outflow_fix2<Q>(p, 64 * blockIdx.x, fa, fb, oa, ob);
  if (clsA != CLS_SKIP) {
    Macro<float> M;
    const float r = collide<Q, CL, float, false>(p, fa, STATS ? &M : nullptr);
    if (!(r > 0.f && r < 3.0e38f)) atomicOr(p.status, 1);
    store_state<Q, S, STORE>(p, x, y, z, cell, clsA, fa);
    if (STATS) stat_values(M, v);
  }
  if (clsB != CLS_SKIP) {
    Macro<float> M;
    const float r = collide<Q, CL, float, false>(p, fb, STATS ? &M : nullptr);
    if (!(r > 0.f && r < 3.0e38f)) atomicOr(p.status, 1);
    store_state<Q, S, STORE>(p, x + 1, y, z, cell + 1, clsB, fb);
    if (STATS) {
      float w[NSTAT];
      stat_values(M, w);
#pragma unroll
      for (int k = 0; k < NSTAT; k++) v[k] += w[k];
    }
  }
}

// ---- two-grid pull: every warp takes the pair path ---------------------------------------
// A lane whose cells are not both interior loads them with the boundary rules of the one-cell
// step (out of line, below); the collision and the own-cell stores are common to all lanes, a
// lane with a skipped (solid or padding) cell storing only its other cell's half.

// Both cells of a boundary lane with the one-cell loads (load_state), packed into hs (the
// loaded values are exact in the storage precision).  Out of line: the rule-by-rule loads are
// long, run for few lanes, and inlined they would crowd the instruction cache of every warp.
template <int Q, class S, int PAR>
__device__ __noinline__ void load_pair_rules(const KParams& p, int x, int y, int z, int cell, int clsA, int clsB,
                                             uint32_t* hs, unsigned* oa, unsigned* ob) {
  float f[Q];
  load_state<Q, S, PAR>(p, x, y, z, cell, clsA, f, *oa);
#pragma unroll
  for (int i = 0; i < Q; i++) hs[i] = bits16<S>(f[i]);
  load_state<Q, S, PAR>(p, x + 1, y, z, cell + 1, clsB, f, *ob);
#pragma unroll
  for (int i = 0; i < Q; i++) hs[i] |= bits16<S>(f[i]) << 16;
}

// Zero-gradient outflow on packed words: x = nx-1 takes what x-1 receives (the lane's own
// first cell, or the previous lane's second).  Warp-uniform condition, full-mask shuffles.
template <int Q>
__device__ __forceinline__ void outflow_fix_packed(const KParams& p, int x0, uint32_t (&h)[Q], unsigned oa,
                                                   unsigned ob) {
  if (!p.outflow) return;
  if (!(x0 <= p.nx - 1 && p.nx - 1 < x0 + 64)) return;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (cx(i) != -1) continue;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, h[i], 1);
    if (ob & (1u << i)) h[i] = (h[i] & 0xffffu) | (h[i] << 16);
    if (oa & (1u << i)) h[i] = (h[i] & 0xffff0000u) | (prev >> 16);
  }
}

#ifndef LBM_H2_PACKED19
#define LBM_H2_PACKED19 0
#endif
#ifndef LBM_H2_PACKED27
#define LBM_H2_PACKED27 1
#endif
#ifndef LBM_H2_MINB27
#define LBM_H2_MINB27 5
#endif
#ifndef LBM_H2_EARLY19
#define LBM_H2_EARLY19 0
#endif
#ifndef LBM_H2_EARLY27
#define LBM_H2_EARLY27 1
#endif

// The collision of both cells (float2 lanes).  PACKED: the populations stay packed and are
// unpacked at each use (fewer live registers); else they are unpacked once into float2 values.
template <int Q, class S, int CL, bool PACKED>
__device__ __forceinline__ float2 collide_pair(const KParams& p, uint32_t (&h)[Q], Macro<float2>* mout) {
  if constexpr (PACKED) {
    PackedPops<Q, S> a{h};
    const Macro<float2> M = macro_acc<Q, CL != CL_NONE, float2>(p, a);
    if (mout) *mout = M;
    float2 wp = vset<float2>(p.omega_p), wm = vset<float2>(p.omega_m);
    if (CL != CL_NONE) {
      les_rates(p, M.qn.x, M.inv.x, p.cs2, wp.x, wm.x);
      les_rates(p, M.qn.y, M.inv.y, p.cs2, wp.y, wm.y);
    }
    relax_lean<Q, float2>(p, a, M, wp, wm);
    return M.rho;
  } else {
    float2 f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = unpack2<S>(h[i]);
    const float2 rho = collide<Q, CL, float2, false>(p, f, mout);
#pragma unroll
    for (int i = 0; i < Q; i++) h[i] = pack2rn<S>(f[i]);
    return rho;
  }
}

// SPLIT (gather step of a handle with a cell list, no statistics): only the interior cells and
// the simple inflow/outflow face cells are updated here, the listed ones by k_step_list.  A lane with one interior cell loads both cells'
// words (the other cell's sources, one x further, stay inside the arrays) and stores one half.
// The packed loads of a lane whose two cells take the fast path.
template <int Q, class S, int LOAD>
__device__ __forceinline__ void pair_loads(const KParams& p, int x, int cell, uint32_t (&h)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (LOAD == 0) {
      h[i] = ld32(p, plane_ptr<S>(p, i) + cell);
    } else {
      const S* base = static_cast<const S*>(p.gb[i]);
      if (cx(i) == 0) {
        h[i] = chk(p, base + cell, 4, CHK_POP) ? ldh_u32(base + cell) : 0u;
      } else {
        int a, b;
        xsrc(cx(i), p, x, cell, a, b);
        const uint32_t lo = chk(p, base + a, 2, CHK_POP) ? ldh_u16(base + a) : 0u;
        const uint32_t hi = chk(p, base + b, 2, CHK_POP) ? ldh_u16(base + b) : 0u;
        h[i] = lo | (hi << 16);
      }
    }
  }
}

// early: the lane's pair is off the lattice faces and hpre holds its fast-path loads, issued
// before the class load (in bounds whatever the classes).
// The split step's inflow/outflow face cells (CLS_XFACE; their other sources are plain fluid
// neighbours, so the fast loads hold them): the directions crossing the face take the
// moving-wall value of the own cell (inflow, x = 0: always the lane's first cell) or what the
// upstream cell x - 1 receives (outflow; x - 1 is the lane's first cell or, for a first cell
// at x = nx - 1, a plain gather one cell back).
template <int Q, class S>
__device__ __forceinline__ void xface_fix(const KParams& p, int x, int cell, bool xfA, bool xfB, uint32_t (&h)[Q]) {
  if (xfA && x == 0) {
#pragma unroll
    for (int i = 0; i < Q; i++) {
      if (cx(i) != 1) continue;
      const float v = rnd<S>(ldp<S>(p, plane_ptr<S>(p, opp(i)) + cell) + p.inflow_term[i]);
      h[i] = (h[i] & 0xffff0000u) | bits16<S>(v);
    }
  } else if (xfA) {  // x = nx - 1
#pragma unroll
    for (int i = 0; i < Q; i++)
      if (cx(i) == -1) h[i] = (h[i] & 0xffff0000u) | ld16(p, static_cast<const S*>(p.gb[i]) + cell - 1);
  }
  if (xfB) {  // x + 1 = nx - 1
#pragma unroll
    for (int i = 0; i < Q; i++)
      if (cx(i) == -1) h[i] = (h[i] & 0xffffu) | (h[i] << 16);
  }
}

template <int Q, class S, int CL, int LOAD, bool STATS, bool SPLIT>
__device__ __forceinline__ void pair_pull(const KParams& p, int x, int y, int z, int cell, int clsA, int clsB,
                                          bool fast, float (&v)[NSTAT], bool early, const uint32_t (&hpre)[Q],
                                          bool xfA, bool xfB) {
  constexpr bool PACKED = Q == 27 ? LBM_H2_PACKED27 : LBM_H2_PACKED19;
  static_assert(!SPLIT || (LOAD == 2 && !STATS), "the split runs the gather step without statistics");
  uint32_t h[Q];
  unsigned oa = 0, ob = 0;
  if (SPLIT) {
    if (clsA != CLS_INTERIOR && clsB != CLS_INTERIOR && !xfA && !xfB) return;
    fast = true;
  }
  if (fast) {
    if (!early) pair_loads<Q, S, LOAD>(p, x, cell, h);
    else {
#pragma unroll
      for (int i = 0; i < Q; i++) h[i] = hpre[i];
    }
  } else {
    uint32_t hs[Q];
    load_pair_rules<Q, S, LOAD>(p, x, y, z, cell, clsA, clsB, hs, &oa, &ob);
#pragma unroll
    for (int i = 0; i < Q; i++) h[i] = hs[i];
  }
  if (!SPLIT) outflow_fix_packed<Q>(p, 64 * blockIdx.x, h, oa, ob);
  else if (xfA || xfB) xface_fix<Q, S>(p, x, cell, xfA, xfB, h);
  Macro<float2> M2;
  const float2 rho = collide_pair<Q, S, CL, PACKED>(p, h, STATS ? &M2 : nullptr);
  const bool liveA = SPLIT ? (clsA == CLS_INTERIOR || xfA) : clsA != CLS_SKIP;
  const bool liveB = SPLIT ? (clsB == CLS_INTERIOR || xfB) : clsB != CLS_SKIP;
  if ((liveA && !(rho.x > 0.f && rho.x < 3.0e38f)) || (liveB && !(rho.y > 0.f && rho.y < 3.0e38f)))
    atomicOr(p.status, 1);
  if (STATS) {
    float va[NSTAT], vb[NSTAT];
    Macro<float> Ma, Mb;
    Ma.ux = M2.ux.x; Ma.uy = M2.uy.x; Ma.uz = M2.uz.x;
    Mb.ux = M2.ux.y; Mb.uy = M2.uy.y; Mb.uz = M2.uz.y;
    stat_values(Ma, va);
    stat_values(Mb, vb);
#pragma unroll
    for (int k = 0; k < NSTAT; k++) v[k] = (liveA ? va[k] : 0.f) + (liveB ? vb[k] : 0.f);
  }
  if (liveA && liveB) {
#pragma unroll
    for (int i = 0; i < Q; i++) st32(p, static_cast<S*>(p.fq[i]) + cell, h[i]);
  } else if (liveA) {
#pragma unroll
    for (int i = 0; i < Q; i++) st16(p, static_cast<S*>(p.fq[i]) + cell, h[i] & 0xffffu);
  } else if (liveB) {
#pragma unroll
    for (int i = 0; i < Q; i++) st16(p, static_cast<S*>(p.fq[i]) + cell + 1, h[i] >> 16);
  }
}

template <int Q, class S, int CL>
__device__ __noinline__ void list_cell(const KParams& p, long long t);

#ifndef LBM_H2_VEC
#define LBM_H2_VEC 1
#endif
#ifndef LBM_H2_MINB
#define LBM_H2_MINB (LBM_H2_VEC ? 7 : 8)
#endif
// STATS: also write the plane statistics of the state this step starts from (warp slot
// blockIdx.x of each row, ceil(nxp/64) slots per row).
template <int Q, class S, int CL, int LOAD, int STORE, bool STATS = false, bool SPLIT = false>
__global__ void __launch_bounds__(128, Q == 27 ? LBM_H2_MINB27 : LBM_H2_MINB) k_step_h2(const __grid_constant__ KParams p) {
  static_assert(sizeof(S) == 2, "two 16-bit populations per word");
  if constexpr (SPLIT) {
    // blocks past the last z plane take the listed cells, 128 per block: they follow the pair
    // blocks in launch order and fill the SMs the pair grid's tail leaves idle
    if (blockIdx.z >= (unsigned)p.nz) {
      const long long b = ((long long)(blockIdx.z - p.nz) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      list_cell<Q, S, CL>(p, b * 128 + threadIdx.y * 32 + threadIdx.x);
      return;
    }
  }
  const int x = 2 * (blockIdx.x * 32 + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= p.ny) return;  // whole warp
  const int cell = cidx(p, x, y, z);
  // two-grid pull, lanes off the lattice faces: the fast-path loads go out with the class load
  // (D3Q27 split step; for D3Q19 pairs measured slower, 60.4k against 64.7k MLUPS)
  constexpr bool EARLY = Q == 27 ? LBM_H2_EARLY27 : LBM_H2_EARLY19;
  const bool early = EARLY && STORE == 2 && LOAD == 2 && x >= 1 && x + 1 < p.nx - 1 && y >= 1 && y < p.ny - 1 &&
                     z >= 1 && z < p.nz - 1;
  uint32_t hpre[Q];
  if (early) pair_loads<Q, S, LOAD>(p, x, cell, hpre);
  int ca_ = CLS_SKIP, cb_ = CLS_SKIP;
  if (x < p.nx) {
    const unsigned c2 = chk(p, p.cls + cell, 2, CHK_CLS) ? *reinterpret_cast<const unsigned short*>(p.cls + cell) : 0x0202u;
    ca_ = c2 & 0xff;
    cb_ = x + 1 < p.nx ? (int)(c2 >> 8) : CLS_SKIP;
  }
  const int clsA = ca_ & CLS_MASK, clsB = cb_ & CLS_MASK;
  const bool xfA = ca_ & CLS_XFACE, xfB = cb_ & CLS_XFACE;
  const bool fast = LOAD == 0 ? ((clsA == CLS_INTERIOR || clsA == CLS_WRAP) && (clsB == CLS_INTERIOR || clsB == CLS_WRAP))
                              : (clsA == CLS_INTERIOR && clsB == CLS_INTERIOR);
  float v[NSTAT];
#pragma unroll
  for (int k = 0; k < NSTAT; k++) v[k] = 0.f;
  if constexpr (STORE == 2) {
    pair_pull<Q, S, CL, LOAD, STATS, SPLIT>(p, x, y, z, cell, clsA, clsB, fast, v, early, hpre, xfA, xfB);
  } else if (__all_sync(0xffffffffu, fast)) {
    uint32_t h[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      if (LOAD == 0) {
        h[i] = ld32(p, plane_ptr<S>(p, i) + cell);
      } else {
        const S* base = static_cast<const S*>(LOAD == 2 ? p.gb[i] : p.ga[i]);
        if (cx(i) == 0) {
          h[i] = ld32(p, base + cell);
        } else {
          int a, b;
          xsrc(cx(i), p, x, cell, a, b);
          const uint32_t lo = ld16(p, base + a);
          const uint32_t hi = ld16(p, base + b);
          h[i] = lo | (hi << 16);
        }
      }
    }
#if LBM_H2_VEC
    // both cells at once in the packed FP32x2 pipe
    float2 f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = make_float2(lo_of<S>(h[i]), hi_of<S>(h[i]));
    Macro<float2> M2;
    const float2 rho = collide<Q, CL, float2, false>(p, f, STATS ? &M2 : nullptr);
    if (STATS) {
      float va[NSTAT], vb[NSTAT];
      Macro<float> Ma, Mb;
      Ma.ux = M2.ux.x; Ma.uy = M2.uy.x; Ma.uz = M2.uz.x;
      Mb.ux = M2.ux.y; Mb.uy = M2.uy.y; Mb.uz = M2.uz.y;
      stat_values(Ma, va);
      stat_values(Mb, vb);
#pragma unroll
      for (int k = 0; k < NSTAT; k++) v[k] = va[k] + vb[k];
    }
#pragma unroll
    for (int i = 0; i < Q; i++) h[i] = pack2<S>(f[i].x, f[i].y);
    const float ra = rho.x, rb = rho.y;
#else
    // first cell: unpack, collide, round back into the low halves
    float f[Q];
    Macro<float> Ma, Mb;
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = lo_of<S>(h[i]);
    const float ra = collide<Q, CL, float, false>(p, f, STATS ? &Ma : nullptr);
#pragma unroll
    for (int i = 0; i < Q; i++) h[i] = __byte_perm(h[i], bits16<S>(f[i]), 0x3254);
    // second cell: the high halves
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = hi_of<S>(h[i]);
    const float rb = collide<Q, CL, float, false>(p, f, STATS ? &Mb : nullptr);
    if (STATS) {
      float va[NSTAT], vb[NSTAT];
      stat_values(Ma, va);
      stat_values(Mb, vb);
#pragma unroll
      for (int k = 0; k < NSTAT; k++) v[k] = va[k] + vb[k];
    }
#pragma unroll
    for (int i = 0; i < Q; i++) h[i] = __byte_perm(h[i], bits16<S>(f[i]), 0x5410);
#endif
    if (!(ra > 0.f && ra < 3.0e38f) || !(rb > 0.f && rb < 3.0e38f)) atomicOr(p.status, 1);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      if (STORE == 0) {
        st32(p, plane_ptr<S>(p, opp(i)) + cell, h[i]);
      } else if (STORE == 2) {
        st32(p, static_cast<S*>(p.fq[i]) + cell, h[i]);
      } else {  // back into the slots the gather of direction i read: f*_opp(i)
        S* base = static_cast<S*>(p.ga[i]);
        const uint32_t w = h[opp(i)];
        if (cx(i) == 0) {
          st32(p, base + cell, w);
        } else {
          int a, b;
          xsrc(cx(i), p, x, cell, a, b);
          st16(p, base + a, w & 0xffffu);
          st16(p, base + b, w >> 16);
        }
      }
    }
  } else {
    pair_fallback<Q, S, CL, LOAD, STORE, STATS>(p, x, y, z, cell, clsA, clsB, v);
  }
  if (STATS) stat_warp_store(p, y, z, blockIdx.x, (p.nxp + 63) / 64, v);
}

// ---- the listed cells of a split pull step ---------------------------------------------------
// A listed cell reads each incoming population through a table built with the list: for
// direction i, the cell the value is read from and a code byte holding the plane (bits 0-4),
// LT_INFLOW (the moving-wall term is added and the sum rounded to the storage precision, as
// for a bounce-back from a moving wall) or LT_ZERO (the value is 0).  The entry is what
// load_state of the gather step and its zero-gradient outflow copy read.
constexpr int LT_INFLOW = 0x40, LT_ZERO = 0x80;

// The table entry of direction i of the cell at `cell` with class cls and rule word r; false
// (and no entry) for a zero-gradient outflow copy, which reads what the upstream cell receives.
__device__ inline bool list_source_at(const KParams& p, int x, int y, int z, int cell, int cls, unsigned long long r,
                                      int i, int& src, int& code) {
  src = cell;
  code = LT_ZERO;
  if (cls == CLS_SKIP) return true;  // the upstream cell of an outflow copy is not fluid: 0
  Nbr nb;
  nb.init(p, x, y, z);
  src = nb.src(p, i);
  code = i;
  if (cls == CLS_INTERIOR || cls == CLS_WRAP) return true;
  const int k = (int)((r >> (2 * i)) & 3);
  if (k == R_STREAM) return true;
  if (k == R_SPECIAL) {
    int pl, ce;
    if (resolve_special(p, x, y, z, i, pl, ce) == K_OUTCOPY) return false;
    src = ce;
    code = opp(pl);
    return true;
  }
  src = cell;  // bounce-back from the own cell (moving wall: plus the inflow term)
  code = opp(i) | (k == R_INFLOW ? LT_INFLOW : 0);
  return true;
}

// The table entry of direction i of a listed cell (set-up): an outflow copy takes the entry of
// the upstream cell x - 1, which is never an outflow cell itself.
__device__ inline void list_source(const KParams& p, int x, int y, int z, int cell, int cls, unsigned long long r,
                                   int i, int& src, int& code) {
  if (list_source_at(p, x, y, z, cell, cls, r, i, src, code)) return;
  const int cu = cidx(p, x - 1, y, z);
  const int cl = cls_at(p, cu);
  if (!list_source_at(p, x - 1, y, z, cu, cl, cl == CLS_BOUNDARY ? rule_at(p, cu) : 0ull, i, src, code)) {
    src = cell;  // not reached (x - 1 is off the outflow face)
    code = LT_ZERO;
  }
}

// Listed cell t: loads through the table, the collision of the storage precision's form,
// own-cell store (the one-cell gather step's bits).
template <int Q, class S, int CL>
__device__ __noinline__ void list_cell(const KParams& p, long long t) {
  if (t >= p.nblist) return;
  const int cell = p.blist[t];
  const S* base = plane_ptr<S>(p, 0);
  float f[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const long long e = i * p.nblist + t;
    const int src = p.bltab[e];
    const int code = p.blcode[e];
    float v = 0.f;
    if (!(code & LT_ZERO)) v = ldp<S>(p, base + (code & 31) * p.pstride + src);
    if (code & LT_INFLOW) v = rnd<S>(v + p.inflow_term[i]);
    f[i] = v;
  }
  const float rho = collide<Q, CL, float, acc_form<S>>(p, f, nullptr);
  if (!(rho > 0.f && rho < 3.0e38f)) atomicOr(p.status, 1);
  store_state<Q, S, 2>(p, 0, 0, 0, cell, CLS_BOUNDARY, f);
}

// The listed cells as a launch of their own (one per thread), for a long list: above 2^18 cells
// (it then runs at the list code's own occupancy rather than the x-pair kernel's), or too many
// blocks to follow the x-pair grid in its z dimension.
template <int Q, class S, int CL>
__global__ void __launch_bounds__(128) k_step_list(const __grid_constant__ KParams p) {
  list_cell<Q, S, CL>(p, blockIdx.x * 128ll + threadIdx.x);
}

}  // namespace lbm
