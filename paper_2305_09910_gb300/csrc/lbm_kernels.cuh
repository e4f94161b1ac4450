// lbm_kernels.cuh -- sm_103a kernels of the lattice Boltzmann stream-and-collide update.
//
// One thread per lattice cell, x-contiguous warps, SoA populations stored shifted
// (df_i = f_i - w_i) in float32, float16 or bfloat16, arithmetic in float32.
//
// Streaming uses the AA pattern (one population array, updated in place).  Let A[x][i]
// be the slot of direction i at cell x.
//   parity 0 ("natural"): A[x][i] holds the pre-collision f_i(x,t).  The even kernel
//     reads its own slots, collides and writes f*_i(x) into its own slot A[x][opp(i)].
//   parity 1 ("swapped"): A[x][opp(i)] holds the post-collision f*_i(x,t-1).  The odd
//     kernel gathers f_i(x,t) = f*_i(x - c_i) from A[x - c_i][opp(i)] (or from the slot
//     its boundary rule names), collides, and writes f*_opp(i)(x) back into the very slot
//     it read f_i from, which is where f_opp(i) of the receiving cell lives at t+1.
//   Every slot is read and written by exactly one thread per launch, so both kernels are
//   race-free in place (the boundary rules are involutions on (cell, direction) pairs).
// Two-grid pull streaming keeps the post-collision f*_i(x) in slot (x, i) of one array and
// writes the next step's into the other: its gather is the odd AA gather with every plane
// index replaced by its opposite, and its store is a plain own-cell store.
// Zero-gradient outflow (+x face) copies what the upstream cell x-1 receives; both cells
// sit in the same warp (nx % 32 != 1), which passes the value with a warp shuffle before
// any thread writes.
//
// Paper: Eq. LBCollision / Eq. LBStreaming (Sec. 2), stream-collide kernel limited by
// memory bandwidth (Sec. 3, Sec. 5.2 Eq. roofline), single PDF set in place (Sec. 5.2).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbm {

// ---- velocity set: published order, components packed 2 bits each (value + 1) ---------
__host__ __device__ constexpr int cx(int i) { return int((0x20889548889549ull >> (2 * i)) & 3) - 1; }
__host__ __device__ constexpr int cy(int i) { return int((0xa088895609495ull >> (2 * i)) & 3) - 1; }
__host__ __device__ constexpr int cz(int i) { return int((0x8a0a0a0954955ull >> (2 * i)) & 3) - 1; }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }

template <int Q>
__host__ __device__ constexpr float wgt(int i) {
  return Q == 19 ? (csq(i) == 0 ? 1.f / 3.f : csq(i) == 1 ? 1.f / 18.f : 1.f / 36.f)
                 : (csq(i) == 0 ? 8.f / 27.f
                                : csq(i) == 1 ? 2.f / 27.f : csq(i) == 2 ? 1.f / 54.f : 1.f / 216.f);
}

// ---- flags, faces, cell classes ------------------------------------------------------
enum : int { CELL_FLUID = 0, CELL_SOLID = 1, CELL_INFLOW = 2 };
// FACE_HALO: the cells beyond the face are ghost cells of a neighbouring slab (z faces)
enum : int { FACE_PERIODIC = 0, FACE_WALL = 1, FACE_FREESLIP = 2, FACE_INFLOW = 3, FACE_OUTFLOW = 4, FACE_HALO = 5 };
// cls: interior fluid (every source is a fluid cell reached by plain streaming, or by a
// periodic wrap in x), wrap fluid (as interior, but a source wraps across a periodic y or z
// face), boundary fluid (some source needs a rule), and everything that is not updated.
enum : int { CLS_INTERIOR = 0, CLS_BOUNDARY = 1, CLS_SKIP = 2, CLS_WRAP = 3 };
// Class byte = class | CLS_XFACE: a boundary cell on an inflow (-x) or outflow (+x) face whose
// only rules are those of the directions crossing that face (every other source a fluid cell
// inside the lattice).  The split half-storage pull step updates such cells in its x-pair
// kernel; everywhere else they are plain boundary cells (cls_at drops the bit).
constexpr int CLS_MASK = 0x0f, CLS_XFACE = 0x10;

// The split half-storage pull step (x-pair kernel over interior cells + k_step_list) for D3Q27
// always, for D3Q19 with LBM_SPLIT19 (on by default: the FP16 channel measured 77.4 % of the copy
// bandwidth split against 74.7 % with the boundary rows and planes in the pair kernel).
#ifndef LBM_SPLIT19
#define LBM_SPLIT19 1
#endif
enum : int { CL_NONE = 0, CL_SMAG = 1, CL_MLP = 2 };
enum : int { K_STREAM = 0, K_BB = 1, K_INFLOW = 2, K_OUTCOPY = 3 };
enum : int { R_STREAM = 0, R_BB = 1, R_INFLOW = 2, R_SPECIAL = 3 };

constexpr int MLP_NIN = 7, MLP_NH = 32;
constexpr int MLP_NPARAM = MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1;
// scaled features are clipped to [-8, 8] (training data are standardised, so this only keeps
// rare outliers, e.g. acoustic density transients, from extrapolating the network)
constexpr float MLP_XCLAMP = 8.f;

struct KParams {
  void* f;               // population array, q planes of `plane` elements
  void* fp[27];          // fp[i] = start of plane i (per-direction base pointers)
  void* fq[27];          // two-grid pull: planes of the destination array
  // gather bases of interior cells: the slot holding f_i(x) is ga[i] + cell (AA swapped
  // layout) or gb[i] + cell (post-collision natural layout), i.e. the plane pointer moved by
  // -(c_x + c_y nxp + c_z nxp ny) elements; x wraps are applied to `cell` before use
  void* ga[27];
  void* gb[27];
  const uint8_t* flags;  // raw cell flags, padded layout
  const uint8_t* cls;    // cell classes, padded layout
  // boundary cells: 2 bits per direction i (bits 2i, 2i+1) naming the rule of the incoming
  // population: R_STREAM (periodic-wrapped neighbour x - c_i), R_BB (bounce-back from the
  // own cell), R_INFLOW (moving-wall bounce-back), R_SPECIAL (free-slip reflection or
  // zero-gradient outflow copy, resolved from the geometry alone)
  const unsigned long long* rules;
  const float* mlp;      // MLP parameters (bf16 values widened to float), device
  // two-grid pull, half storage, D3Q27: the cells that need boundary rules or a periodic y/z
  // wrap (classes BOUNDARY and WRAP), padded cell indices in row order; the x-pair step then
  // updates the interior cells and k_step_list these (null: no split)
  const int* blist;
  // per direction i and listed cell t (index i nblist + t): the cell its incoming population
  // is read from, and a code byte: the plane (bits 0-4), LT_INFLOW, LT_ZERO (see k_step_list)
  const int* bltab;
  const uint8_t* blcode;
  long long nblist;
  long long pstride;     // elements from one population plane to the next
  int split;             // the pull gather step runs as the interior x-pair step + k_step_list
  int* status;           // bit 0: non-finite or non-positive density seen; bits 1, 2: a
                         // bounded wait of the learned-closure step gave up (once, twice)
  int wait_polls;        // polls of the closure step's first wait for each tile's MMA
  float* stats_w;        // sampling steps: per-warp plane sums, [(z ny + y) nws + ws][10]
  long long plane;       // nxp * ny * nz
  int nx, ny, nz, nxp;
  int outflow;           // +x face is an outflow
  int nat_valid;         // natural layout holds imported values in the outflow slots
  int face[6];
  float tau0, lambda, cs2, omega_p, omega_m;
  float F[3];
  float inflow_term[27];  // 6 w_i rho_w (c_i . u_w)
  float F3w[27];          // 3 w_i (c_i . F): antisymmetric Guo term
  float F9w[27];          // 9 w_i (c_i . F): symmetric Guo term, times c_i . u
  float mlp_scale[2];
  float cs2_min;          // lower bound on the learned C_s^2 (0: none)
  float mrt_s[5];         // MRT rates of the e, eps, q, pi and m moment groups
  // bounds-checked builds (LBM_BOUNDS_CHECK): byte ranges of the population arrays (0, 1),
  // flags (2), classes (3) and rules (4), and the word that records the first bad access
  const char* chk_lo[5];
  const char* chk_hi[5];
  int* chk_bad;
};

// ---- checked accesses --------------------------------------------------------------------
// With LBM_BOUNDS_CHECK every global access of the step, export and set-up kernels checks its
// address against the array it belongs to; an access outside is skipped (a load gives 0) and
// the first one is recorded in *chk_bad as 1 + the array index (lbm_sync reports it).  Without
// it the checks compile away.
enum : int { CHK_POP = 0, CHK_FLAGS = 2, CHK_CLS = 3, CHK_RULES = 4 };

__device__ __forceinline__ bool chk(const KParams& p, const void* a, int bytes, int kind) {
#ifdef LBM_BOUNDS_CHECK
  const char* c = static_cast<const char*>(a);
  bool ok;
  if (kind == CHK_POP)
    ok = (c >= p.chk_lo[0] && c + bytes <= p.chk_hi[0]) || (p.chk_lo[1] && c >= p.chk_lo[1] && c + bytes <= p.chk_hi[1]);
  else
    ok = c >= p.chk_lo[kind] && c + bytes <= p.chk_hi[kind];
  if (!ok) atomicCAS(p.chk_bad, 0, 1 + kind);
  return ok;
#else
  (void)p; (void)a; (void)bytes; (void)kind;
  return true;
#endif
}

__device__ __forceinline__ int cls_at(const KParams& p, long long cell) {
  return chk(p, p.cls + cell, 1, CHK_CLS) ? (p.cls[cell] & CLS_MASK) : CLS_SKIP;
}
__device__ __forceinline__ int flag_at(const KParams& p, long long cell) {
  return chk(p, p.flags + cell, 1, CHK_FLAGS) ? p.flags[cell] : CELL_SOLID;
}
__device__ __forceinline__ unsigned long long rule_at(const KParams& p, long long cell) {
  return chk(p, p.rules + cell, 8, CHK_RULES) ? p.rules[cell] : 0ull;
}

__device__ __forceinline__ int cidx(const KParams& p, int x, int y, int z) {
  return (z * p.ny + y) * p.nxp + x;
}

// ---- storage precisions -----------------------------------------------------------------
template <class S> __device__ __forceinline__ float ld(const S* a);
template <> __device__ __forceinline__ float ld<float>(const float* a) { return *a; }
template <> __device__ __forceinline__ float ld<__half>(const __half* a) { return __half2float(*a); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* a) {
  return __bfloat162float(*a);
}
template <class S> __device__ __forceinline__ void st(S* a, float v);
template <> __device__ __forceinline__ void st<float>(float* a, float v) { *a = v; }
template <> __device__ __forceinline__ void st<__half>(__half* a, float v) { *a = __float2half_rn(v); }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16* a, float v) {
  *a = __float2bfloat16_rn(v);
}

// Population accesses of global memory (checked in bounds-checked builds).
template <class S>
__device__ __forceinline__ float ldp(const KParams& p, const S* a) {
  return chk(p, a, (int)sizeof(S), CHK_POP) ? ld<S>(a) : 0.f;
}
// Gather loads of the step kernels with the 256-byte L2 prefetch size: the L2 fetches the
// aligned 256 bytes around a warp's 128-byte row segment of one direction, whose other half the
// neighbouring block in x reads next.  Measured 0.5-1.2 % faster than plain loads on the pull
// and AA steps (a 128-byte prefetch size gains nothing, the non-coherent path nothing more, and
// bypassing L1 costs up to 15 %: the shifted directions of x-neighbouring warps share lines).
__device__ __forceinline__ float ldh_f32(const float* a) {
  float v;
  asm volatile("ld.global.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(a));
  return v;
}
__device__ __forceinline__ uint32_t ldh_u32(const void* a) {
  uint32_t v;
  asm volatile("ld.global.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(a));
  return v;
}
__device__ __forceinline__ uint32_t ldh_u16(const void* a) {
  unsigned short v;
  asm volatile("ld.global.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(a));
  return v;
}
// A checked gather load (the hinted form for FP32 storage).
template <class S>
__device__ __forceinline__ float ldg_pop(const KParams& p, const S* a) {
  if constexpr (sizeof(S) == 4) return chk(p, a, 4, CHK_POP) ? ldh_f32(reinterpret_cast<const float*>(a)) : 0.f;
  else return ldp<S>(p, a);
}

template <class S>
__device__ __forceinline__ void stp(const KParams& p, S* a, float v) {
  if (chk(p, a, (int)sizeof(S), CHK_POP)) st<S>(a, v);
}

// Value after a round trip through the storage precision.
template <class S> __device__ __forceinline__ float rnd(float v);
template <> __device__ __forceinline__ float rnd<float>(float v) { return v; }
template <> __device__ __forceinline__ float rnd<__half>(float v) { return __half2float(__float2half_rn(v)); }
template <> __device__ __forceinline__ float rnd<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// ---- boundary rule of one (cell, direction): which slot holds the incoming value -------
__device__ __forceinline__ int face_rank(int t) {
  return t == FACE_WALL ? 4 : t == FACE_INFLOW ? 3 : t == FACE_OUTFLOW ? 2 : 1;
}

__device__ __forceinline__ int dir_index(int dx, int dy, int dz) {
  // inverse of (cx, cy, cz) over the 27 velocities
  for (int j = 0; j < 27; j++)
    if (cx(j) == dx && cy(j) == dy && cz(j) == dz) return j;
  return 0;
}

// Returns the rule for the incoming population i of fluid cell (x,y,z) and, except for
// K_OUTCOPY, the slot (plane, cell) that holds it in the swapped layout.
static __device__ __noinline__ int classify(const KParams& p, int x, int y, int z, int i,
                                            int& plane, int& cell) {
  const int c[3] = {cx(i), cy(i), cz(i)};
  const int xc[3] = {x, y, z};
  const int n[3] = {p.nx, p.ny, p.nz};
  int s[3], fc[3], rank = 0;
  for (int a = 0; a < 3; a++) {
    s[a] = xc[a] - c[a];
    fc[a] = s[a] < 0 ? 2 * a : (s[a] >= n[a] ? 2 * a + 1 : -1);
    if (fc[a] >= 0 && p.face[fc[a]] == FACE_HALO) fc[a] = -1;  // a ghost cell, not a face
    if (fc[a] >= 0) rank = max(rank, face_rank(p.face[fc[a]]));
  }
  plane = i;
  cell = cidx(p, x, y, z);
  if (rank == 4) return K_BB;
  if (rank == 3) return K_INFLOW;
  if (rank == 2) return flag_at(p, cidx(p, x - 1, y, z)) == CELL_FLUID ? K_OUTCOPY : K_BB;
  int d[3];
  for (int a = 0; a < 3; a++) {
    d[a] = c[a];
    if (fc[a] >= 0) {
      if (p.face[fc[a]] == FACE_PERIODIC) {
        s[a] = s[a] < 0 ? s[a] + n[a] : s[a] - n[a];
      } else {  // free-slip: stay in the plane, reflect the normal component
        s[a] = xc[a];
        d[a] = -d[a];
      }
    }
  }
  const int src = cidx(p, s[0], s[1], s[2]);
  const int fl = flag_at(p, src);
  if (fl == CELL_SOLID) return K_BB;
  if (fl == CELL_INFLOW) return K_INFLOW;
  plane = opp(dir_index(d[0], d[1], d[2]));
  cell = src;
  return K_STREAM;
}

// The 2-bit rule of (cell, direction) from classify's answer: plain streaming from the
// periodic-wrapped neighbour, bounce-back, moving-wall bounce-back, or special.
__device__ __forceinline__ int rule_of(const KParams& p, int x, int y, int z, int i) {
  int pl, ce;
  const int k = classify(p, x, y, z, i, pl, ce);
  if (k == K_BB) return R_BB;
  if (k == K_INFLOW) return R_INFLOW;
  if (k == K_OUTCOPY) return R_SPECIAL;
  return pl == opp(i) ? R_STREAM : R_SPECIAL;  // a free-slip reflection changes the plane
}

// classify() for a direction whose rule is R_SPECIAL, without reading flags: the outflow copy
// at x = nx-1 (c_x = -1), otherwise the free-slip reflection (with periodic wraps on other axes).
static __device__ __noinline__ int resolve_special(const KParams& p, int x, int y, int z, int i,
                                                   int& plane, int& cell) {
  if (p.outflow && x == p.nx - 1 && cx(i) == -1) return K_OUTCOPY;
  const int c[3] = {cx(i), cy(i), cz(i)};
  const int xc[3] = {x, y, z};
  const int n[3] = {p.nx, p.ny, p.nz};
  int s[3], d[3];
  for (int a = 0; a < 3; a++) {
    s[a] = xc[a] - c[a];
    d[a] = c[a];
    if (s[a] < 0 || s[a] >= n[a]) {
      const int ft = p.face[s[a] < 0 ? 2 * a : 2 * a + 1];
      if (ft == FACE_HALO) {
        // the ghost cell beyond the face
      } else if (ft == FACE_PERIODIC) {
        s[a] = s[a] < 0 ? s[a] + n[a] : s[a] - n[a];
      } else {
        s[a] = xc[a];
        d[a] = -d[a];
      }
    }
  }
  plane = opp(dir_index(d[0], d[1], d[2]));
  cell = cidx(p, s[0], s[1], s[2]);
  return K_STREAM;
}

template <class S>
__device__ __forceinline__ S* plane_ptr(const KParams& p, int i) {
  return static_cast<S*>(p.fp[i]);
}

// Interior cells: periodic-wrapped source of direction i (x - c_i).
struct Nbr {
  int xs[3], ys[3], zs[3];  // index c+1 -> coordinate of x - c
  // wraps only across periodic faces (a source across another face is either never read,
  // as its rule is not plain streaming, or a ghost cell beyond a halo face)
  __device__ __forceinline__ void init(const KParams& p, int x, int y, int z) {
    xs[1] = x; ys[1] = y; zs[1] = z;
    xs[2] = x == 0 ? p.nx - 1 : x - 1;  // c = +1
    xs[0] = x == p.nx - 1 ? 0 : x + 1;  // c = -1
    ys[2] = y == 0 ? p.ny - 1 : y - 1;
    ys[0] = y == p.ny - 1 ? 0 : y + 1;
    zs[2] = (z == 0 && p.face[4] == FACE_PERIODIC) ? p.nz - 1 : z - 1;
    zs[0] = (z == p.nz - 1 && p.face[5] == FACE_PERIODIC) ? 0 : z + 1;
  }
  __device__ __forceinline__ int src(const KParams& p, int i) const {
    return (zs[cz(i) + 1] * p.ny + ys[cy(i) + 1]) * p.nxp + xs[cx(i) + 1];
  }
};

// ---- loading the pre-collision populations of one cell ---------------------------------
// PAR 0: natural layout (own slots); 1: AA swapped layout (gather); 2: post-collision values
// in natural layout (two-grid pull, gather).
template <int Q, class S, int PAR>
__device__ __forceinline__ void load_state(const KParams& p, int x, int y, int z, int cell, int cls,
                                           float (&f)[Q], unsigned& outmask) {
  outmask = 0;
#pragma unroll
  for (int i = 0; i < Q; i++) f[i] = 0.f;
  if (cls == CLS_SKIP) return;
  if (PAR == 0) {
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = ldp<S>(p, plane_ptr<S>(p, i) + cell);
    // after a streaming step the outflow slots of x = nx-1 were not written (they are
    // copies of the upstream cell); after an import they hold the imported values
    if (cls == CLS_BOUNDARY && p.outflow && !p.nat_valid && x == p.nx - 1) {
      const unsigned long long r = rule_at(p, cell);
#pragma unroll
      for (int i = 0; i < Q; i++)
        if (cx(i) == -1 && ((r >> (2 * i)) & 3) == R_SPECIAL) outmask |= 1u << i;
    }
  } else if (cls == CLS_INTERIOR) {
    // periodic x wrap of the row ends, applied to the cell index once per sign of c_x
    const int cp = cell + (x == 0 ? p.nx : 0);       // sources x - 1
    const int cm = cell - (x == p.nx - 1 ? p.nx : 0);  // sources x + 1
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const S* base = static_cast<const S*>(PAR == 2 ? p.gb[i] : p.ga[i]);
      f[i] = ldp<S>(p, base + (cx(i) > 0 ? cp : cx(i) < 0 ? cm : cell));
    }
  } else if (cls == CLS_WRAP) {
    Nbr nb;
    nb.init(p, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = ldp<S>(p, plane_ptr<S>(p, PAR == 2 ? i : opp(i)) + nb.src(p, i));
  } else {
    // boundary cell: the precomputed rules make every load independent of the others
    const unsigned long long r = rule_at(p, cell);
    Nbr nb;
    nb.init(p, x, y, z);
    unsigned special = 0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const int k = (int)((r >> (2 * i)) & 3);
      if (k == R_SPECIAL) {
        special |= 1u << i;
        continue;
      }
      const S* a = k == R_STREAM ? plane_ptr<S>(p, PAR == 2 ? i : opp(i)) + nb.src(p, i)
                                 : plane_ptr<S>(p, PAR == 2 ? opp(i) : i) + cell;
      float v = ldp<S>(p, a);
      // moving-wall value rounded like the natural-layout slot that holds it
      if (k == R_INFLOW) v = rnd<S>(v + p.inflow_term[i]);
      f[i] = v;
    }
    if (special) {
#pragma unroll
      for (int i = 0; i < Q; i++) {
        if (!(special & (1u << i))) continue;
        int pl, ce;
        if (resolve_special(p, x, y, z, i, pl, ce) == K_OUTCOPY) outmask |= 1u << i;
        else f[i] = ldp<S>(p, plane_ptr<S>(p, PAR == 2 ? opp(pl) : pl) + ce);
      }
    }
  }
}

// A cell off every lattice face (1 <= x, y, z <= n-2): the gather of an interior cell reads
// inside the arrays whatever the cell's class, so the step kernels issue it together with the
// class load instead of after it, and keep it if the cell is interior.
__device__ __forceinline__ bool off_faces(const KParams& p, int x, int y, int z) {
  return x >= 1 && x < p.nx - 1 && y >= 1 && y < p.ny - 1 && z >= 1 && z < p.nz - 1;
}

// The interior-cell gather of load_state (PAR 1: AA swapped layout, 2: pull) for a cell off the
// faces (no x wrap there).
template <int Q, class S, int PAR>
__device__ __forceinline__ void gather_interior(const KParams& p, int cell, float (&f)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; i++) f[i] = ldg_pop<S>(p, static_cast<const S*>(PAR == 2 ? p.gb[i] : p.ga[i]) + cell);
}

// Zero-gradient outflow: lane x = nx-1 takes the incoming c_x = -1 populations of lane x-1.
// Called by every thread of the block (warp-uniform condition, full-mask shuffles).
template <int Q>
__device__ __forceinline__ void outflow_fix(const KParams& p, int x, float (&f)[Q],
                                            unsigned outmask) {
  if (!p.outflow) return;
  const int x0 = x & ~31;
  if (!(x0 <= p.nx - 1 && p.nx - 1 < x0 + 32)) return;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    if (cx(i) != -1) continue;
    const float v = __shfl_up_sync(0xffffffffu, f[i], 1);
    if (outmask & (1u << i)) f[i] = v;
  }
}

// ---- storing the post-collision populations -------------------------------------------
// PAR 0: own cell, swapped slots (AA even); 1: back into the gathered slots (AA odd);
// 2: own cell, natural slots of the destination array (two-grid pull).
template <int Q, class S, int PAR>
__device__ __forceinline__ void store_state(const KParams& p, int x, int y, int z, int cell, int cls,
                                            const float (&fs)[Q]) {
  if (PAR == 2) {
#pragma unroll
    for (int i = 0; i < Q; i++) stp<S>(p, static_cast<S*>(p.fq[i]) + cell, fs[i]);
  } else if (PAR == 0) {
#pragma unroll
    for (int i = 0; i < Q; i++) stp<S>(p, plane_ptr<S>(p, opp(i)) + cell, fs[i]);
  } else if (cls == CLS_INTERIOR) {
    const int cp = cell + (x == 0 ? p.nx : 0);
    const int cm = cell - (x == p.nx - 1 ? p.nx : 0);
#pragma unroll
    for (int i = 0; i < Q; i++)
      stp<S>(p, static_cast<S*>(p.ga[i]) + (cx(i) > 0 ? cp : cx(i) < 0 ? cm : cell), fs[opp(i)]);
  } else if (cls == CLS_WRAP) {
    Nbr nb;
    nb.init(p, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; i++) stp<S>(p, plane_ptr<S>(p, opp(i)) + nb.src(p, i), fs[opp(i)]);
  } else {
    const unsigned long long r = rule_at(p, cell);
    Nbr nb;
    nb.init(p, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const int k = (int)((r >> (2 * i)) & 3);
      int pl = opp(i), ce = nb.src(p, i);
      if (k == R_BB || k == R_INFLOW) {
        pl = i;
        ce = cell;
      } else if (k == R_SPECIAL) {
        if (resolve_special(p, x, y, z, i, pl, ce) == K_OUTCOPY) continue;
      }
      float v = fs[opp(i)];
      if (k == R_INFLOW) v = rnd<S>(v) + p.inflow_term[i];  // same rounding as the swapped path
      stp<S>(p, plane_ptr<S>(p, pl) + ce, v);
    }
  }
}

__device__ __forceinline__ float softplus_f(float y) { return fmaxf(y, 0.f) + log1pf(__expf(-fabsf(y))); }

// ---- moments and TRT collision (in place on shifted populations) -----------------------
template <int Q>
__host__ __device__ constexpr double wgt_d(int i) {
  return Q == 19 ? (csq(i) == 0 ? 1.0 / 3.0 : csq(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                 : (csq(i) == 0 ? 8.0 / 27.0
                                : csq(i) == 1 ? 2.0 / 27.0 : csq(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0);
}

template <int Q>
struct Mom {
  float drho, rho, jx, jy, jz, ux, uy, uz;  // j = sum c df + F/2 = rho u
};

// ---- arithmetic, written for a value type V (float: one cell, float2: two cells per thread) ---
// Every operation rounds once to nearest even and none is contracted by the compiler, so every
// kernel form (direct, staged, x-pair, closure) gives a cell the same bits.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// two cells in the packed FP32x2 pipe (sm_100 family): the same roundings per component
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so this is the correctly rounded difference
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class V> __device__ __forceinline__ V vset(float a);
template <> __device__ __forceinline__ float vset<float>(float a) { return a; }
template <> __device__ __forceinline__ float2 vset<float2>(float a) { return make_float2(a, a); }

template <class V> struct Lanes;
template <> struct Lanes<float> {
  static constexpr int n = 1;
  __device__ __forceinline__ static float get(float v, int) { return v; }
  __device__ __forceinline__ static void put(float& v, int, float a) { v = a; }
};
template <> struct Lanes<float2> {
  static constexpr int n = 2;
  __device__ __forceinline__ static float get(float2 v, int k) { return k ? v.y : v.x; }
  __device__ __forceinline__ static void put(float2& v, int k, float a) { (k ? v.y : v.x) = a; }
};

// ---- closure network: activation functions ------------------------------------------------
// erf by the rational approximation of Abramowitz & Stegun, formula 7.1.26 (after Hastings):
// erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p z) for
// z >= 0, erf(-z) = -erf(z); absolute error below 1.5e-7, about one float32 ulp of erf near 1.
// GELU in its erf form, x Phi(x) = x (1 + erf(x / sqrt 2)) / 2, written with m = q t e - 1
// = -(1 - erf|z|) as  GELU(x) = x / 2 - |x| m / 2, for one value or two (packed FP32x2).
__device__ __forceinline__ float ex2_approx(float v) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

template <class V>
__device__ __forceinline__ V gelu_v(V a) {
  using L = Lanes<V>;
  V az, t, e;
#pragma unroll
  for (int k = 0; k < L::n; k++) L::put(az, k, fabsf(L::get(a, k)) * 0.70710678118654752f);  // |z|
  const V den = vfma(az, vset<V>(0.3275911f), vset<V>(1.f));
#pragma unroll
  for (int k = 0; k < L::n; k++) L::put(t, k, __fdividef(1.f, L::get(den, k)));
  V q = vfma(vset<V>(1.061405429f), t, vset<V>(-1.453152027f));
  q = vfma(q, t, vset<V>(1.421413741f));
  q = vfma(q, t, vset<V>(-0.284496736f));
  q = vfma(q, t, vset<V>(0.254829592f));
  const V arg = vmul(az, vmul(az, vset<V>(-1.4426950408889634f)));  // -z^2 log2(e)
#pragma unroll
  for (int k = 0; k < L::n; k++) L::put(e, k, ex2_approx(L::get(arg, k)));
  const V m = vfma(vmul(q, t), e, vset<V>(-1.f));
  return vfma(vmul(az, vset<V>(-0.70710678118654752f)), m, vmul(a, vset<V>(0.5f)));
}

__device__ __forceinline__ float gelu_erf(float a) { return gelu_v<float>(a); }

// erf of the same approximation, for the derivative Phi(x) + x phi(x) of the GELU
__device__ __forceinline__ float erf_as(float z) {
  const float a = fabsf(z);
  const float t = __fdividef(1.f, fmaf(0.3275911f, a, 1.f));
  float q = fmaf(1.061405429f, t, -1.453152027f);
  q = fmaf(q, t, 1.421413741f);
  q = fmaf(q, t, -0.284496736f);
  q = fmaf(q, t, 0.254829592f);
  const float r = fmaf(-q * t, ex2_approx(-a * a * 1.4426950408889634f), 1.f);
  return copysignf(r, z);
}
__device__ __forceinline__ float gelu_grad_f(float a) {
  return 0.5f * (1.f + erf_as(a * 0.70710678118654752f)) + a * 0.39894228040143268f * __expf(-0.5f * a * a);
}

// Orientation of the +/- pair (I, I+1), I odd: the member whose first non-zero velocity
// component is positive is the primary one, so that c.u is a plain sum with a leading +.
__host__ __device__ constexpr int lead(int i) { return cx(i) ? cx(i) : cy(i) ? cy(i) : cz(i); }
__host__ __device__ constexpr int prim(int I) { return lead(I) > 0 ? I : I + 1; }

// c . v for a velocity with entries in {-1, 0, 1} and a positive leading entry
template <int X, int Y, int Z, class V>
__device__ __forceinline__ V cdot(V vx, V vy, V vz) {
  static_assert(X > 0 || (X == 0 && (Y > 0 || (Y == 0 && Z > 0))), "leading component must be positive");
  V r;
  if (X) r = vx;
  if (Y) r = X ? (Y > 0 ? vadd(r, vy) : vsub(r, vy)) : vy;
  if (Z) r = (X || Y) ? (Z > 0 ? vadd(r, vz) : vsub(r, vz)) : vz;
  return r;
}

// Moment accumulators m[k]: k = 0 sum df, 1..3 j (without F/2), 4..6 sum c_a^2 df,
// 7..9 sum c_x c_y df, c_x c_z df, c_y c_z df.  coef(k, i) is the factor of df_i in m[k].
__host__ __device__ constexpr int mcoef(int k, int i) {
  return k == 0 ? 1 : k == 1 ? cx(i) : k == 2 ? cy(i) : k == 3 ? cz(i) : k == 4 ? cx(i) * cx(i)
       : k == 5 ? cy(i) * cy(i) : k == 6 ? cz(i) * cz(i) : k == 7 ? cx(i) * cy(i) : k == 8 ? cx(i) * cz(i)
       : cy(i) * cz(i);
}
// first pair (odd I) that contributes to m[k]; the rest population opens m[0]
__host__ __device__ constexpr int mfirst(int k) {
  if (k == 0) return 0;
  for (int I = 1; I < 27; I += 2)
    if (mcoef(k, I) != 0) return I;
  return -1;
}

template <int K, int I, class V>
__device__ __forceinline__ void macc(V (&m)[10], V v, int sign) {
  if (mfirst(K) == I) m[K] = sign > 0 ? v : vsub(vset<V>(0.f), v);
  else m[K] = sign > 0 ? vadd(m[K], v) : vsub(m[K], v);
}

// Population accessors of the moment and lean collision code: an array of values (one cell
// per thread, or two as float2), or two cells' half-precision values packed in 32-bit words,
// unpacked at each use and packed (round to nearest even) at each store, so that only the
// packed words stay live.  Both run the same operations in the same order.
template <int Q, class V, class T = V>  // T = const V: read only
struct ArrPops {
  T (&f)[Q];
  template <int I> __device__ __forceinline__ V get() const { return f[I]; }
  template <int I> __device__ __forceinline__ void set(V v) { f[I] = v; }
};

template <class S> __device__ __forceinline__ float2 unpack2(uint32_t w);
template <> __device__ __forceinline__ float2 unpack2<__half>(uint32_t w) {
  return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <> __device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <class S> __device__ __forceinline__ uint32_t pack2rn(float2 v);
template <> __device__ __forceinline__ uint32_t pack2rn<__half>(float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2rn<__nv_bfloat16>(float2 v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int Q, class S>
struct PackedPops {
  uint32_t (&h)[Q];
  template <int I> __device__ __forceinline__ float2 get() const { return unpack2<S>(h[I]); }
  template <int I> __device__ __forceinline__ void set(float2 v) { h[I] = pack2rn<S>(v); }
};

// Sums over the pair (I, I+1): s = f_I + f_I+1, d = f_P - f_R (P primary, R its opposite).
template <int Q, int I, class V, class A>
__device__ __forceinline__ void pair_moments_acc(const A& a, V (&m)[10]) {
  constexpr int P = prim(I);
  const V fi = a.template get<I>(), fj = a.template get<I + 1>();
  const V s = vadd(fi, fj);
  const V d = P == I ? vsub(fi, fj) : vsub(fj, fi);
  macc<0, I>(m, s, 1);
#pragma unroll
  for (int k = 1; k <= 3; k++) {
    if (mcoef(k, P) == 0) continue;
    if (k == 1) macc<1, I>(m, d, mcoef(1, P));
    if (k == 2) macc<2, I>(m, d, mcoef(2, P));
    if (k == 3) macc<3, I>(m, d, mcoef(3, P));
  }
  if (mcoef(4, P)) macc<4, I>(m, s, 1);
  if (mcoef(5, P)) macc<5, I>(m, s, 1);
  if (mcoef(6, P)) macc<6, I>(m, s, 1);
  if (mcoef(7, P)) macc<7, I>(m, s, mcoef(7, P));
  if (mcoef(8, P)) macc<8, I>(m, s, mcoef(8, P));
  if (mcoef(9, P)) macc<9, I>(m, s, mcoef(9, P));
}

template <int Q, class V, class A, int... P>
__device__ __forceinline__ void all_pair_moments(const A& a, V (&m)[10], std::integer_sequence<int, P...>) {
  (pair_moments_acc<Q, 2 * P + 1, V>(a, m), ...);
}

template <class V>
struct CollCtx {
  V ux, uy, uz, jx, jy, jz;
  V A, B;          // symmetric equilibrium w (A + B (c.u)^2): A = drho - 1.5 rho u^2, B = 4.5 rho
  V nhwp, nhwm;    // -omega+/2, -omega-/2
  V gp, gm;        // 1 - omega+/2, 1 - omega-/2
  V gu3;           // (1 - omega+/2) 3 u.F
};

// One +/- pair of the TRT collision, written as f* = f + delta so that the only rounding at
// the magnitude of f is the final addition.  The antisymmetric equilibrium 3 w (c.j) is
// carried as an unevaluated sum eh + el (the FMA recovers the product's rounding error
// exactly; eln = -el).  With a = f_P - eh and b = f_R + eh (exact when the operands are
// within a factor two, as near equilibrium), the non-equilibrium parts of the pair are
//   n+ = (a + b) - 2 w (A + B (c.u)^2)   and   n- = (a - b) + 2 eln,
// a - b being exact as well.  This keeps the per-step momentum error at the level of one
// rounding of f, which matters at the small velocities of laminar runs.
template <int Q, int I, class V>
__device__ __forceinline__ void trt_pair(const KParams& p, V (&f)[Q], const CollCtx<V>& c) {
  constexpr int P = prim(I), R = P == I ? I + 1 : I;
  constexpr int X = cx(P), Y = cy(P), Z = cz(P);
  constexpr float w = (float)wgt_d<Q>(P);
  constexpr float khi = (float)(3.0 * wgt_d<Q>(P));
  constexpr float klo = (float)(3.0 * wgt_d<Q>(P) - (double)khi);
  const V cu = cdot<X, Y, Z>(c.ux, c.uy, c.uz);
  const V cj = cdot<X, Y, Z>(c.jx, c.jy, c.jz);
  const V eh = vmul(cj, vset<V>(khi));
  const V eln = vfma(cj, vset<V>(-klo), vfma(cj, vset<V>(-khi), eh));
  const V a = vsub(f[P], eh), b = vadd(f[R], eh);
  const V es2 = vmul(vset<V>(2.f * w), vfma(c.B, vmul(cu, cu), c.A));
  const V np = vsub(vadd(a, b), es2);
  const V nm = vfma(eln, vset<V>(2.f), vsub(a, b));
  // Guo terms: symmetric w (9 (c.u)(c.F) - 3 u.F), antisymmetric 3 w (c.F)
  const V fsym = vfma(vmul(c.gp, vset<V>(p.F9w[P])), cu, vmul(c.gu3, vset<V>(-w)));
  const V ds = vfma(c.nhwp, np, fsym);
  const V da = vfma(c.nhwm, nm, vmul(c.gm, vset<V>(p.F3w[P])));
  f[P] = vadd(f[P], vadd(ds, da));
  f[R] = vadd(f[R], vsub(ds, da));
}

template <int Q, class V, int... P>
__device__ __forceinline__ void trt_pairs(const KParams& p, V (&f)[Q], const CollCtx<V>& c,
                                          std::integer_sequence<int, P...>) {
  (trt_pair<Q, 2 * P + 1, V>(p, f, c), ...);
}

// The pair update for half-precision storage, where the rounding of the stored value (2^-11
// or 2^-8 relative) dominates.  With s = f_P + f_R and d = f_P - f_R the TRT update reads
//   f*_P = S + D, f*_R = S - D,
//   S = (1 - omega+) s / 2 + omega+ f^eq+ + F+,   D = (1 - omega-) d / 2 + omega- f^eq- + F-,
// f^eq+ = w (A + B (c.u)^2), f^eq- = 3 w rho (c.u), F+ = (1 - omega+/2) w (9 (c.u)(c.F) - 3 u.F),
// F- = (1 - omega-/2) 3 w (c.F).  Per weight class k: kb = omega+ w B, kc = omega+ w A - w gu3,
// kr = 3 omega- w rho; hp = (1 - omega+)/2, hm = (1 - omega-)/2.
template <class V>
struct LeanCtx {
  V ux, uy, uz, hp, hm, gp, gm;
  V kb[3], kc[3], kr[3];
};

template <int Q, int I, class V, class A>
__device__ __forceinline__ void trt_pair_lean(const KParams& p, A& a, const LeanCtx<V>& c) {
  constexpr int P = prim(I), R = P == I ? I + 1 : I;
  constexpr int X = cx(P), Y = cy(P), Z = cz(P), K = csq(P) - 1;
  const V cu = cdot<X, Y, Z>(c.ux, c.uy, c.uz);
  const V fP = a.template get<P>(), fR = a.template get<R>();
  const V s = vadd(fP, fR);
  const V d = vsub(fP, fR);
  const V S = vfma(c.hp, s, vfma(vmul(c.gp, vset<V>(p.F9w[P])), cu, vfma(c.kb[K], vmul(cu, cu), c.kc[K])));
  const V D = vfma(c.hm, d, vfma(c.kr[K], cu, vmul(c.gm, vset<V>(p.F3w[P]))));
  a.template set<P>(vadd(S, D));
  a.template set<R>(vsub(S, D));
}

template <int Q, class V, class A, int... P>
__device__ __forceinline__ void trt_pairs_lean(const KParams& p, A& a, const LeanCtx<V>& c,
                                               std::integer_sequence<int, P...>) {
  (trt_pair_lean<Q, 2 * P + 1, V>(p, a, c), ...);
}

// sqrt of a non-negative value from the hardware reciprocal square root (x = 0 gives 0).
__device__ __forceinline__ float fast_sqrt(float x) { return __fmul_rn(x, rsqrtf(fmaxf(x, 1e-37f))); }

// Relaxation rates of one cell from its stress invariant Q = Pi:Pi: tau_eff solves
// tau = tau0 + 3 C_s^2 |S|(tau) in closed form, omega- keeps the magic parameter Lambda.
__device__ __forceinline__ void les_rates(const KParams& p, float qn, float inv, float cs2, float& wp, float& wm) {
  const float t = __fmul_rn(__fmul_rn(25.455844122715711f, cs2), __fmul_rn(fast_sqrt(qn), inv));
  const float tau = __fmul_rn(0.5f, __fadd_rn(p.tau0, fast_sqrt(__fmaf_rn(p.tau0, p.tau0, t))));
  wp = __fdividef(1.f, tau);
  wm = __fdividef(1.f, __fadd_rn(__fdividef(p.lambda, __fsub_rn(tau, 0.5f)), 0.5f));
}

// ACC: the accurate pair update (float32 storage) or the lean one (half storage).
template <class S>
constexpr bool acc_form = std::is_same<S, float>::value;

// Macroscopic fields of a cell (or two): density, momentum j = sum c df + F/2, velocity and,
// when STRESS, the non-equilibrium stress Pi^neq and its invariant Q = Pi:Pi.
template <class V>
struct Macro {
  V drho, rho, jx, jy, jz, inv, ux, uy, uz;
  V pi[6], qn;
};

template <int Q, bool STRESS, class V, class A>
__device__ __forceinline__ Macro<V> macro_acc(const KParams& p, const A& a) {
  using Pairs = std::make_integer_sequence<int, (Q - 1) / 2>;
  using L = Lanes<V>;
  V m[10];
  m[0] = a.template get<0>();
  all_pair_moments<Q, V>(a, m, Pairs{});
  Macro<V> M;
  M.drho = m[0];
  M.rho = vadd(M.drho, vset<V>(1.f));
  M.jx = vadd(m[1], vset<V>(0.5f * p.F[0]));
  M.jy = vadd(m[2], vset<V>(0.5f * p.F[1]));
  M.jz = vadd(m[3], vset<V>(0.5f * p.F[2]));
#pragma unroll
  for (int k = 0; k < L::n; k++) L::put(M.inv, k, __fdividef(1.f, L::get(M.rho, k)));
  M.ux = vmul(M.jx, M.inv);
  M.uy = vmul(M.jy, M.inv);
  M.uz = vmul(M.jz, M.inv);
  if (STRESS) {
    // Pi^neq = sum_i c c df_i - (drho/3) I - j u   (shifted form of sum c c (f - feq))
    const V d3 = vmul(M.drho, vset<V>(1.f / 3.f));
    M.pi[0] = vsub(vsub(m[4], d3), vmul(M.jx, M.ux));
    M.pi[1] = vsub(vsub(m[5], d3), vmul(M.jy, M.uy));
    M.pi[2] = vsub(vsub(m[6], d3), vmul(M.jz, M.uz));
    M.pi[3] = vsub(m[7], vmul(M.jx, M.uy));
    M.pi[4] = vsub(m[8], vmul(M.jx, M.uz));
    M.pi[5] = vsub(m[9], vmul(M.jy, M.uz));
    V qn = vfma(M.pi[5], M.pi[5], vfma(M.pi[4], M.pi[4], vmul(M.pi[3], M.pi[3])));
    M.qn = vfma(M.pi[2], M.pi[2], vfma(M.pi[1], M.pi[1], vfma(M.pi[0], M.pi[0], vadd(qn, qn))));
  }
  return M;
}

template <int Q, bool STRESS, class V>
__device__ __forceinline__ Macro<V> macro(const KParams& p, const V (&f)[Q]) {
  return macro_acc<Q, STRESS, V>(p, ArrPops<Q, V, const V>{f});
}

// Moments of one cell for the exports: the collision's macroscopic fields, so an export and
// the statistics sampled inside a step see the same per-cell values.
template <int Q>
__device__ __forceinline__ Mom<Q> moments(const KParams& p, const float (&f)[Q]) {
  const Macro<float> M = macro<Q, false, float>(p, f);
  Mom<Q> m;
  m.drho = M.drho;
  m.rho = M.rho;
  m.jx = M.jx;
  m.jy = M.jy;
  m.jz = M.jz;
  m.ux = M.ux;
  m.uy = M.uy;
  m.uz = M.uz;
  return m;
}

// The lean TRT relaxation (half storage) of the populations behind accessor a, in place.
template <int Q, class V, class A>
__device__ __forceinline__ void relax_lean(const KParams& p, A& a, const Macro<V>& M, V wp, V wm) {
  using Pairs = std::make_integer_sequence<int, (Q - 1) / 2>;
  const V usq = vfma(M.uz, M.uz, vfma(M.uy, M.uy, vmul(M.ux, M.ux)));
  const V uF = vfma(M.uz, vset<V>(p.F[2]), vfma(M.uy, vset<V>(p.F[1]), vmul(M.ux, vset<V>(p.F[0]))));
  const V A_ = vfma(vmul(M.rho, vset<V>(-1.5f)), usq, M.drho);
  const V nhwp = vmul(wp, vset<V>(-0.5f));
  const V gp = vadd(nhwp, vset<V>(1.f)), gm = vadd(vmul(wm, vset<V>(-0.5f)), vset<V>(1.f));
  const V gu3 = vmul(gp, vmul(uF, vset<V>(3.f)));
  LeanCtx<V> c;
  c.ux = M.ux;
  c.uy = M.uy;
  c.uz = M.uz;
  c.gp = gp;
  c.gm = gm;
  c.hp = vfma(wp, vset<V>(-0.5f), vset<V>(0.5f));
  c.hm = vfma(wm, vset<V>(-0.5f), vset<V>(0.5f));
  const V wpA = vmul(wp, A_), wpB = vmul(wp, vmul(M.rho, vset<V>(4.5f))), wmr = vmul(wm, vmul(M.rho, vset<V>(3.f)));
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float w = (float)(k == 0 ? wgt_d<Q>(1) : k == 1 ? wgt_d<Q>(7) : wgt_d<Q>(19 % Q));
    c.kb[k] = vmul(wpB, vset<V>(w));
    c.kc[k] = vfma(wpA, vset<V>(w), vmul(gu3, vset<V>(-w)));
    c.kr[k] = vmul(wmr, vset<V>(w));
  }
  {
    constexpr float w0 = (float)wgt_d<Q>(0);
    a.template set<0>(vfma(vadd(c.hp, c.hp), a.template get<0>(), vfma(wpA, vset<V>(w0), vmul(gu3, vset<V>(-w0)))));
  }
  trt_pairs_lean<Q, V>(p, a, c, Pairs{});
}

// TRT relaxation with Guo forcing at the rates omega+ (wp) and omega- (wm), in place.
// ACC: the accurate pair update (float32 storage) or the lean one (half storage).
template <int Q, class V, bool ACC>
__device__ __forceinline__ void relax(const KParams& p, V (&f)[Q], const Macro<V>& M, V wp, V wm) {
  using Pairs = std::make_integer_sequence<int, (Q - 1) / 2>;
  const V usq = vfma(M.uz, M.uz, vfma(M.uy, M.uy, vmul(M.ux, M.ux)));
  const V uF = vfma(M.uz, vset<V>(p.F[2]), vfma(M.uy, vset<V>(p.F[1]), vmul(M.ux, vset<V>(p.F[0]))));
  const V A = vfma(vmul(M.rho, vset<V>(-1.5f)), usq, M.drho);
  const V nhwp = vmul(wp, vset<V>(-0.5f)), nhwm = vmul(wm, vset<V>(-0.5f));
  const V gp = vadd(nhwp, vset<V>(1.f)), gm = vadd(nhwm, vset<V>(1.f));
  const V gu3 = vmul(gp, vmul(uF, vset<V>(3.f)));
  if constexpr (ACC) {
    CollCtx<V> c;
    c.ux = M.ux;
    c.uy = M.uy;
    c.uz = M.uz;
    c.jx = M.jx;
    c.jy = M.jy;
    c.jz = M.jz;
    c.A = A;
    c.B = vmul(M.rho, vset<V>(4.5f));
    c.nhwp = nhwp;
    c.nhwm = nhwm;
    c.gp = gp;
    c.gm = gm;
    c.gu3 = gu3;
    {
      constexpr float w0 = (float)wgt_d<Q>(0);
      const V n0 = vfma(c.A, vset<V>(-w0), f[0]);
      f[0] = vadd(f[0], vfma(vadd(c.nhwp, c.nhwp), n0, vmul(c.gu3, vset<V>(-w0))));
    }
    trt_pairs<Q, V>(p, f, c, Pairs{});
  } else {
    ArrPops<Q, V> a{f};
    relax_lean<Q, V>(p, a, M, wp, wm);
  }
}

// ---- MRT collision (D3Q19) ---------------------------------------------------------------
// Multiple-relaxation-time operator in the orthogonal moment basis of d'Humieres, Ginzburg,
// Krafczyk, Lallemand & Luo (2002), the collision of the paper's LAGOON runs (Sec. 5.2):
// m_k = sum_i M_ki (f_i - f^eq_i) relaxes at rate s_k, Guo's force enters as (1 - s_k/2) M F,
// and f* = f + M^T diag(1/|M_k|^2) dm (the rows are orthogonal).  Rows, with c2 = |c_i|^2:
// rho, e = 19 c2 - 30, eps = (21 c2^2 - 53 c2 + 24)/2, j_a = c_a, q_a = (5 c2 - 9) c_a,
// 3p_xx = 3 c_x^2 - c2, 3pi_xx = (3 c2 - 5)(3 c_x^2 - c2), p_ww = c_y^2 - c_z^2,
// pi_ww = (3 c2 - 5)(c_y^2 - c_z^2), p_xy, p_yz, p_xz = c_a c_b, m_x = (c_y^2 - c_z^2) c_x,
// m_y = (c_z^2 - c_x^2) c_y, m_z = (c_x^2 - c_y^2) c_z (all integer-valued).
__host__ __device__ constexpr int mrt_row(int k, int i) {
  const int x = cx(i), y = cy(i), z = cz(i), c2 = x * x + y * y + z * z;
  return k == 0 ? 1 : k == 1 ? 19 * c2 - 30 : k == 2 ? (21 * c2 * c2 - 53 * c2 + 24) / 2
       : k == 3 ? x : k == 4 ? (5 * c2 - 9) * x : k == 5 ? y : k == 6 ? (5 * c2 - 9) * y
       : k == 7 ? z : k == 8 ? (5 * c2 - 9) * z : k == 9 ? 3 * x * x - c2
       : k == 10 ? (3 * c2 - 5) * (3 * x * x - c2) : k == 11 ? y * y - z * z
       : k == 12 ? (3 * c2 - 5) * (y * y - z * z) : k == 13 ? x * y : k == 14 ? y * z : k == 15 ? x * z
       : k == 16 ? (y * y - z * z) * x : k == 17 ? (z * z - x * x) * y : (x * x - y * y) * z;
}
__host__ __device__ constexpr int mrt_norm(int k) {
  int n = 0;
  for (int i = 0; i < 19; i++) n += mrt_row(k, i) * mrt_row(k, i);
  return n;
}
// rate group of moment k: -1 conserved (rate 1, the moment only carries the force),
// -2 stress (1/tau_eff), 0..4 = e, eps, q, pi, m
__host__ __device__ constexpr int mrt_group(int k) {
  return (k == 0 || k == 3 || k == 5 || k == 7) ? -1 : k == 1 ? 0 : k == 2 ? 1
       : (k == 4 || k == 6 || k == 8) ? 2 : (k == 10 || k == 12) ? 3 : k >= 16 ? 4 : -2;
}

// Moments of the populations from the +/- pair sums s_P = f_P + f_R and differences
// a_P = f_P - f_R (P the primary member of a pair): even rows (rho, e, eps, p, pi) take the
// same coefficient on both members, odd rows (j, q, m) opposite ones.
__host__ __device__ constexpr bool mrt_even(int k) { return !(k >= 3 && k <= 8) && k < 16; }

template <int K, int... P>
__device__ __forceinline__ float mrt_pair_moment(float f0, const float (&sp)[9], const float (&ap)[9],
                                                 std::integer_sequence<int, P...>) {
  float m = (mrt_even(K) && mrt_row(K, 0) != 0) ? f0 * (float)mrt_row(K, 0) : 0.f;
  ((m = mrt_row(K, prim(2 * P + 1)) != 0
            ? vfma(mrt_even(K) ? sp[P] : ap[P], (float)mrt_row(K, prim(2 * P + 1)), m)
            : m),
   ...);
  return m;
}

template <int... K>
__device__ __forceinline__ void mrt_pair_moments(float f0, const float (&sp)[9], const float (&ap)[9],
                                                 float (&m)[19], std::integer_sequence<int, K...>) {
  ((m[K] = mrt_pair_moment<K>(f0, sp, ap, std::make_integer_sequence<int, 9>{})), ...);
}

// The update of pair P from the scaled moment increments dm: even part E, odd part O.
template <int P>
__device__ __forceinline__ void mrt_pair_back(float (&f)[19], const float (&dm)[19]) {
  constexpr int I = 2 * P + 1, PP = prim(I), R = PP == I ? I + 1 : I;
  float e = 0.f, o = 0.f;
#pragma unroll
  for (int k = 0; k < 19; k++) {
    if (mrt_row(k, PP) == 0) continue;
    if (mrt_even(k)) e = vfma(dm[k], (float)mrt_row(k, PP), e);
    else o = vfma(dm[k], (float)mrt_row(k, PP), o);
  }
  f[PP] = vadd(f[PP], vadd(e, o));
  f[R] = vadd(f[R], vsub(e, o));
}

template <int... P>
__device__ __forceinline__ void mrt_pairs_back(float (&f)[19], const float (&dm)[19], std::integer_sequence<int, P...>) {
  (mrt_pair_back<P>(f, dm), ...);
}

// ---- regularised collision (projected regularisation, Latt & Chopard 2006) ---------------
// BGK with Guo forcing reads f* = f^eq + (1 - w) g + F_i/2 with g = f - f^eq + F_i/2; the
// regularised operator keeps only the part of g on the second-order Hermite polynomials
// H_i = c_i c_i - I/3:  f*_i = f^eq_i + F_i/2 + (1 - w) (9/2) w_i H_i : P  with
// P = sum_j H_j g_j = Pi^neq + (u F + F u)/2 (the second moment of Guo's term is u F + F u).
// Shifted values per pair (i, opp i) with c = c_i: the even part S is common, the odd part A
// flips sign,
//   S = w_i [drho - 1.5 j.u - 1.5 u.F + 4.5 (c.j)(c.u) + 4.5 (c.u)(c.F) + (1 - w) 4.5 H_i:P]
//   A = w_i [3 c.j + 1.5 c.F].
struct RegCtx {
  float B0, a, tr3, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
  float ux, uy, uz, jx, jy, jz, Fx, Fy, Fz;
};

template <int Q, int I>
__device__ __forceinline__ void reg_pair(float (&f)[Q], const RegCtx& r) {
  constexpr int P = prim(I), R = P == I ? I + 1 : I;
  constexpr int X = cx(P), Y = cy(P), Z = cz(P);
  constexpr float w = (float)wgt_d<Q>(P);
  const float cu = cdot<X, Y, Z>(r.ux, r.uy, r.uz);
  const float cj = cdot<X, Y, Z>(r.jx, r.jy, r.jz);
  const float cF = cdot<X, Y, Z>(r.Fx, r.Fy, r.Fz);
  float h = -r.tr3;
  if (X) h = vadd(h, r.Pxx);
  if (Y) h = vadd(h, r.Pyy);
  if (Z) h = vadd(h, r.Pzz);
  if (X && Y) h = vfma((float)(2 * X * Y), r.Pxy, h);
  if (X && Z) h = vfma((float)(2 * X * Z), r.Pxz, h);
  if (Y && Z) h = vfma((float)(2 * Y * Z), r.Pyz, h);
  const float S = vmul(w, vfma(r.a, h, vfma(vmul(4.5f, cu), vadd(cj, cF), r.B0)));
  const float A = vmul(w, vfma(3.f, cj, vmul(1.5f, cF)));
  f[P] = vadd(S, A);
  f[R] = vsub(S, A);
}

template <int Q, int... K>
__device__ __forceinline__ void reg_pairs(float (&f)[Q], const RegCtx& r, std::integer_sequence<int, K...>) {
  (reg_pair<Q, 2 * K + 1>(f, r), ...);
}

template <int Q>
__device__ __forceinline__ void relax_reg(const KParams& p, float (&f)[Q], const Macro<float>& M, float w) {
  RegCtx r;
  r.Fx = p.F[0];
  r.Fy = p.F[1];
  r.Fz = p.F[2];
  r.ux = M.ux;
  r.uy = M.uy;
  r.uz = M.uz;
  r.jx = M.jx;
  r.jy = M.jy;
  r.jz = M.jz;
  r.Pxx = vfma(M.ux, r.Fx, M.pi[0]);
  r.Pyy = vfma(M.uy, r.Fy, M.pi[1]);
  r.Pzz = vfma(M.uz, r.Fz, M.pi[2]);
  r.Pxy = vfma(0.5f, vfma(M.ux, r.Fy, vmul(M.uy, r.Fx)), M.pi[3]);
  r.Pxz = vfma(0.5f, vfma(M.ux, r.Fz, vmul(M.uz, r.Fx)), M.pi[4]);
  r.Pyz = vfma(0.5f, vfma(M.uy, r.Fz, vmul(M.uz, r.Fy)), M.pi[5]);
  r.tr3 = vmul(vadd(vadd(r.Pxx, r.Pyy), r.Pzz), 1.f / 3.f);
  r.a = vmul(vsub(1.f, w), 4.5f);
  const float ju = vfma(M.jz, M.uz, vfma(M.jy, M.uy, vmul(M.jx, M.ux)));
  const float uF = vfma(M.uz, r.Fz, vfma(M.uy, r.Fy, vmul(M.ux, r.Fx)));
  r.B0 = vfma(-1.5f, vadd(ju, uF), M.drho);
  f[0] = vmul((float)wgt_d<Q>(0), vfma(r.a, -r.tr3, r.B0));
  reg_pairs<Q>(f, r, std::make_integer_sequence<int, (Q - 1) / 2>{});
}

// With shifted populations df = f - w: m(df) = M f - M w, and the equilibrium and force
// moments in closed form (the polynomial equilibrium and Guo's force on this lattice):
//   rho: drho, 0;  e: -11 drho + 19 rho u^2, 38 u.F;  eps: 3 drho - 11/2 rho u^2, -11 u.F;
//   j: rho u, F;  q: -2/3 rho u, -2/3 F;  3p_xx: rho (3u_x^2 - u^2), 6 u_x F_x - 2 u.F;
//   3pi_xx: -1/2 of 3p_xx (both);  p_ww: rho (u_y^2 - u_z^2), 2 (u_y F_y - u_z F_z);
//   pi_ww: -1/2 of p_ww;  p_ab: rho u_a u_b, u_a F_b + u_b F_a;  m: 0, 0.
__device__ __forceinline__ void relax_mrt(const KParams& p, float (&f)[19], const Macro<float>& M, float wnu) {
  float sp[9], ap[9];
  {
    // pair sums in the primary orientation
    auto fill = [&](auto I_) {
      constexpr int I = decltype(I_)::value;
      constexpr int PP = prim(I), R = PP == I ? I + 1 : I;
      sp[(I - 1) / 2] = vadd(f[PP], f[R]);
      ap[(I - 1) / 2] = vsub(f[PP], f[R]);
    };
    fill(std::integral_constant<int, 1>{});
    fill(std::integral_constant<int, 3>{});
    fill(std::integral_constant<int, 5>{});
    fill(std::integral_constant<int, 7>{});
    fill(std::integral_constant<int, 9>{});
    fill(std::integral_constant<int, 11>{});
    fill(std::integral_constant<int, 13>{});
    fill(std::integral_constant<int, 15>{});
    fill(std::integral_constant<int, 17>{});
  }
  float m[19];
  mrt_pair_moments(f[0], sp, ap, m, std::make_integer_sequence<int, 19>{});
  const float ux = M.ux, uy = M.uy, uz = M.uz, rho = M.rho;
  const float Fx = p.F[0], Fy = p.F[1], Fz = p.F[2];
  const float u2 = vfma(uz, uz, vfma(uy, uy, vmul(ux, ux)));
  const float uF = vfma(uz, Fz, vfma(uy, Fy, vmul(ux, Fx)));
  const float ru2 = vmul(rho, u2);
  const float p3xx = vmul(rho, vfma(3.f * ux, ux, -u2)), pww = vmul(rho, vsub(vmul(uy, uy), vmul(uz, uz)));
  const float f3xx = vfma(6.f * ux, Fx, -2.f * uF), fww = 2.f * vsub(vmul(uy, Fy), vmul(uz, Fz));
  float meq[19], mf[19];
  meq[0] = M.drho;                         mf[0] = 0.f;
  meq[1] = vfma(19.f, ru2, -11.f * M.drho); mf[1] = 38.f * uF;
  meq[2] = vfma(-5.5f, ru2, 3.f * M.drho);  mf[2] = -11.f * uF;
  meq[3] = M.jx;                           mf[3] = Fx;
  meq[4] = (-2.f / 3.f) * M.jx;            mf[4] = (-2.f / 3.f) * Fx;
  meq[5] = M.jy;                           mf[5] = Fy;
  meq[6] = (-2.f / 3.f) * M.jy;            mf[6] = (-2.f / 3.f) * Fy;
  meq[7] = M.jz;                           mf[7] = Fz;
  meq[8] = (-2.f / 3.f) * M.jz;            mf[8] = (-2.f / 3.f) * Fz;
  meq[9] = p3xx;                           mf[9] = f3xx;
  meq[10] = -0.5f * p3xx;                  mf[10] = -0.5f * f3xx;
  meq[11] = pww;                           mf[11] = fww;
  meq[12] = -0.5f * pww;                   mf[12] = -0.5f * fww;
  meq[13] = vmul(M.jx, uy);                mf[13] = vfma(ux, Fy, vmul(uy, Fx));
  meq[14] = vmul(M.jy, uz);                mf[14] = vfma(uy, Fz, vmul(uz, Fy));
  meq[15] = vmul(M.jx, uz);                mf[15] = vfma(ux, Fz, vmul(uz, Fx));
  meq[16] = 0.f;                           mf[16] = 0.f;
  meq[17] = 0.f;                           mf[17] = 0.f;
  meq[18] = 0.f;                           mf[18] = 0.f;
#pragma unroll
  for (int k = 0; k < 19; k++) {
    const int g = mrt_group(k);
    const float s = g == -1 ? 1.f : g == -2 ? wnu : p.mrt_s[g];
    // (the momentum rows of df lack the half force of j: m_j(df) - j = -F/2)
    m[k] = vmul(vfma(-s, vsub(m[k], meq[k]), vmul(vfma(s, -0.5f, 1.f), mf[k])), 1.f / (float)mrt_norm(k));
  }
  {
    float e0 = 0.f;
#pragma unroll
    for (int k = 0; k < 19; k++)
      if (mrt_even(k) && mrt_row(k, 0) != 0) e0 = vfma(m[k], (float)mrt_row(k, 0), e0);
    f[0] = vadd(f[0], e0);
  }
  mrt_pairs_back(f, m, std::make_integer_sequence<int, 9>{});
}

// Stream-collide arithmetic of one cell (or two) without a learned closure: plain TRT or
// TRT with the Smagorinsky relaxation time.  Returns rho.
// COLL: 0 TRT, 1 MRT (D3Q19, one cell per thread).
template <int Q, int CL, class V, bool ACC = true, int COLL = 0>
__device__ __forceinline__ V collide(const KParams& p, V (&f)[Q], Macro<V>* mout = nullptr) {
  static_assert(CL != CL_MLP, "the learned closure has its own kernel");
  using L = Lanes<V>;
  const Macro<V> M = macro<Q, CL != CL_NONE || COLL == 2, V>(p, f);
  if (mout) *mout = M;
  V wp = vset<V>(p.omega_p), wm = vset<V>(p.omega_m);
  if (CL != CL_NONE) {
#pragma unroll
    for (int k = 0; k < L::n; k++) {
      float a, b;
      les_rates(p, L::get(M.qn, k), L::get(M.inv, k), p.cs2, a, b);
      L::put(wp, k, a);
      L::put(wm, k, b);
    }
  }
  if constexpr (COLL == 1) {
    static_assert(Q == 19 && std::is_same<V, float>::value, "MRT: D3Q19, one cell per thread");
    relax_mrt(p, f, M, wp);
  } else if constexpr (COLL == 2) {
    static_assert(std::is_same<V, float>::value, "regularised: one cell per thread");
    relax_reg<Q>(p, f, M, wp);
  } else {
    relax<Q, V, ACC>(p, f, M, wp, wm);
  }
  return M.rho;
}

// ---- kernels ------------------------------------------------------------------------------
// Block (32, 4): a warp is 32 consecutive x of one row; grid (nxp/32, ceil(ny/4), nz).
#define LBM_CELL_COORDS                                   \
  const int x = blockIdx.x * 32 + threadIdx.x;            \
  const int y = blockIdx.y * blockDim.y + threadIdx.y;    \
  const int z = blockIdx.z;                               \
  if (y >= p.ny) return; /* whole warp */                 \
  const int cell = cidx(p, x, y, z);                      \
  const int cls = x < p.nx ? cls_at(p, cell) : CLS_SKIP;

// LOAD / STORE modes as in load_state / store_state: AA even (0, 0), AA odd (1, 1), first
// pull step after an import (0, 2), pull step (2, 2).
// ---- turbulence statistics sampled inside a step ----------------------------------------
// The 10 per-cell values of the plane statistics (count, u, u_a u_b) of the state a step
// starts from: u = j / rho of its macroscopic fields, so they equal those of the export.
constexpr int NSTAT = 10;

__device__ __forceinline__ void stat_values(const Macro<float>& M, float (&v)[NSTAT]) {
  v[0] = 1.f;
  v[1] = M.ux;
  v[2] = M.uy;
  v[3] = M.uz;
  v[4] = M.ux * M.ux;
  v[5] = M.uy * M.uy;
  v[6] = M.uz * M.uz;
  v[7] = M.ux * M.uy;
  v[8] = M.ux * M.uz;
  v[9] = M.uy * M.uz;
}

// One round of a warp reduce-scatter: lanes with bit `bit` of their index set keep the upper
// half of the N values (and receive their partner's upper half), the others the lower half;
// N odd is padded with a zero.  Returns ceil(N / 2) partial sums.
template <int N, int M = (N + 1) / 2>
__device__ __forceinline__ void rs_round(const float (&in)[N], float (&out)[M], int bit) {
  const bool hi = (threadIdx.x >> bit) & 1;
#pragma unroll
  for (int k = 0; k < M; k++) {
    const float lo_v = in[k], hi_v = k + M < N ? in[k + M] : 0.f;
    const float keep = hi ? hi_v : lo_v, send = hi ? lo_v : hi_v;
    out[k] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
  }
}

// Sum of v over the warp (FP32), written to the warp's slot ws of row (y, z): a reduce-scatter
// over lane bits 4, 3, 2, 1 leaves statistic k = b1 + 2 b2 + 3 b3 + 5 b4 (b_i the lane's
// index bits; padding where that index is out of range) summed over the lane pairs (l, l^1),
// which the last exchange completes; the even lane of each pair writes it.
__device__ __forceinline__ void stat_warp_store(const KParams& p, int y, int z, int ws, int nws,
                                                float (&v)[NSTAT]) {
  static_assert(NSTAT == 10, "the scatter below is laid out for 10 statistics");
  float a[5], b[3], c[2], d[1];
  rs_round<10>(v, a, 4);
  rs_round<5>(a, b, 3);
  rs_round<3>(b, c, 2);
  rs_round<2>(c, d, 1);
  const float s = d[0] + __shfl_xor_sync(0xffffffffu, d[0], 1);
  const int lane = threadIdx.x & 31;
  const int b1 = (lane >> 1) & 1, b2 = (lane >> 2) & 1, b3 = (lane >> 3) & 1, b4 = (lane >> 4) & 1;
  const int j = b1 + 2 * b2;  // slot after the second exchange (3 values)
  const int k = j + 3 * b3;   // slot after the first exchange (5 values)
  if (!(lane & 1) && j < 3 && k < 5)
    p.stats_w[(((long long)z * p.ny + y) * nws + ws) * NSTAT + k + 5 * b4] = s;
}

// Plane sums of the sampled statistics: sums[y * 10 + k] += sum over z and the nws warp
// slots of each row (FP64).  One block per plane y.  A thread sums its slots in FP32 with the
// rounding error of every addition carried along (Knuth's TwoSum: hi + lo is the exact sum up
// to the rounding of lo, about 2^-48 of it), then widens hi and lo once: FP64 arithmetic, which
// is slow on this GPU, is left to the block's final reduction.
static __global__ void __launch_bounds__(256) k_stats_total(const float* stats_w, int ny, int nz, int nws, double* sums) {
  const int y = blockIdx.x;
  float hi[NSTAT], lo[NSTAT];
#pragma unroll
  for (int k = 0; k < NSTAT; k++) hi[k] = lo[k] = 0.f;
  const int n = nz * nws;  // below 2^31: a warp slot per 32 cells of a lattice under 2^31 cells
#pragma unroll 4
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int z = r / nws, ws = r - z * nws;
    const float* src = stats_w + (((long long)z * ny + y) * nws + ws) * NSTAT;
#pragma unroll
    for (int k = 0; k < NSTAT; k++) {
      const float v = src[k];
      const float s = __fadd_rn(hi[k], v);
      const float bp = __fsub_rn(s, hi[k]);
      const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bp)), __fsub_rn(v, bp));
      lo[k] = __fadd_rn(lo[k], err);
      hi[k] = s;
    }
  }
  double acc[NSTAT];
#pragma unroll
  for (int k = 0; k < NSTAT; k++) acc[k] = (double)hi[k] + (double)lo[k];
  __shared__ double red[NSTAT][8];
#pragma unroll
  for (int k = 0; k < NSTAT; k++) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < NSTAT) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[threadIdx.x][w];
    sums[y * NSTAT + threadIdx.x] += t;
  }
}

// Resident blocks per SM the step is compiled for (registers per thread = 65536 / (128 x
// this)): more resident warps keep more loads in flight.  D3Q19 TRT and regularised: 10 (48
// registers; the pull step spills nothing and measured 10 % faster than at 8); D3Q27: 9 (56
// registers, no spill; pull 5 % faster); MRT: 8, above which it spills.
#ifndef LBM_STEP_MINB19
#define LBM_STEP_MINB19 10
#endif
#ifndef LBM_STEP_MINB27
#define LBM_STEP_MINB27 9
#endif

// STATS: also write the plane statistics of the state this step starts from (warp slot
// blockIdx.x of each row, nxp/32 slots per row).
template <int Q, class S, int CL, int LOAD, int STORE, bool STATS = false, int COLL = 0>
__global__ void __launch_bounds__(128, Q == 19 ? (COLL == 1 ? 8 : LBM_STEP_MINB19) : LBM_STEP_MINB27)
    k_step(const __grid_constant__ KParams p) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= p.ny) return;  // whole warp
  const int cell = cidx(p, x, y, z);
  float f[Q];
  unsigned outmask = 0;
  const bool early = LOAD != 0 && off_faces(p, x, y, z);
  if (early) gather_interior<Q, S, LOAD>(p, cell, f);  // in flight with the class load below
  const int cls = x < p.nx ? cls_at(p, cell) : CLS_SKIP;
  if (!(early && cls == CLS_INTERIOR)) load_state<Q, S, LOAD>(p, x, y, z, cell, cls, f, outmask);
  outflow_fix<Q>(p, x, f, outmask);
  if (!STATS && cls == CLS_SKIP) return;
  float v[NSTAT];
#pragma unroll
  for (int k = 0; k < NSTAT; k++) v[k] = 0.f;
  if (cls != CLS_SKIP) {
    Macro<float> M;
    const float rho = collide<Q, CL, float, acc_form<S>, COLL>(p, f, STATS ? &M : nullptr);
    if (!(rho > 0.f && rho < 3.0e38f)) atomicOr(p.status, 1);
    store_state<Q, S, STORE>(p, x, y, z, cell, cls, f);
    if (STATS) stat_values(M, v);
  }
  if (STATS) stat_warp_store(p, y, z, blockIdx.x, p.nxp / 32, v);
}

// ---- several steps in one launch --------------------------------------------------------
// Small lattices are launch-bound: k_step_multi runs nsteps plain steps in one cooperative
// launch, the steps separated by grid-wide barriers (cooperative groups), each block taking
// the (32 x 4)-cell tiles of k_step's grid in turn.  Two-grid pull alternates the two arrays
// (pp.p[s & 1]); AA alternates the even and odd forms on one array, starting with the form
// `odd0`.  Every cell gets the bits of the single-launch step.
struct KParams2 {
  KParams p[2];
};

template <int Q, class S, int CL, int LOAD, int STORE, int COLL>
__device__ __forceinline__ void step_tile(const KParams& p, int tile) {
  const int tx = p.nxp / 32, ty = (p.ny + 3) / 4;
  const int bz = tile / (tx * ty);
  const int r = tile - bz * tx * ty;
  const int by = r / tx, bx = r - by * tx;
  const int x = bx * 32 + threadIdx.x;
  const int y = by * 4 + threadIdx.y;
  const int z = bz;
  if (y >= p.ny) return;  // whole warp
  const int cell = cidx(p, x, y, z);
  const int cls = x < p.nx ? cls_at(p, cell) : CLS_SKIP;
  float f[Q];
  unsigned outmask;
  load_state<Q, S, LOAD>(p, x, y, z, cell, cls, f, outmask);
  outflow_fix<Q>(p, x, f, outmask);
  if (cls == CLS_SKIP) return;
  const float rho = collide<Q, CL, float, acc_form<S>, COLL>(p, f, nullptr);
  if (!(rho > 0.f && rho < 3.0e38f)) atomicOr(p.status, 1);
  store_state<Q, S, STORE>(p, x, y, z, cell, cls, f);
}

template <int Q, class S, int CL, int COLL, bool AA>
__global__ void __launch_bounds__(128, Q == 19 ? 8 : 6) k_step_multi(const __grid_constant__ KParams2 pp, int nsteps, int odd0) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const KParams& p0 = pp.p[0];
  const int ntiles = (p0.nxp / 32) * ((p0.ny + 3) / 4) * p0.nz;
  for (int s = 0; s < nsteps; s++) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      if (AA) {
        if ((s + odd0) & 1) step_tile<Q, S, CL, 1, 1, COLL>(p0, t);
        else step_tile<Q, S, CL, 0, 0, COLL>(p0, t);
      } else {
        step_tile<Q, S, CL, 2, 2, COLL>(pp.p[s & 1], t);
      }
    }
    if (s + 1 < nsteps) grid.sync();
  }
}

// Exports of the current state (read-only): populations, moments, FP64 sums, statistics.
enum : int { EX_POP = 0, EX_MOM = 1, EX_SUM = 2, EX_STATS = 3 };

struct ExportArgs {
  float* df;       // EX_POP: [q][nz][ny][nx]
  float* rho;      // EX_MOM: [nz][ny][nx] (may be null)
  float* u;        // EX_MOM: [3][nz][ny][nx] (may be null)
  double* sums;    // EX_SUM: 4 doubles; EX_STATS: ny * 10 doubles (added to)
  double* partial; // EX_SUM / EX_STATS: nz * ny * 10 doubles of scratch (per-row sums)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int Q, class S, int PAR, int MODE>
__global__ void __launch_bounds__(128) k_export(const __grid_constant__ KParams p, ExportArgs a) {
  LBM_CELL_COORDS
  float f[Q];
  unsigned outmask;
  load_state<Q, S, PAR>(p, x, y, z, cell, cls, f, outmask);
  outflow_fix<Q>(p, x, f, outmask);
  const bool fluid = cls != CLS_SKIP;
  const long long dense = ((long long)z * p.ny + y) * p.nx + x;
  const long long N = (long long)p.nx * p.ny * p.nz;
  if (MODE == EX_POP) {
    if (x >= p.nx) return;
#pragma unroll
    for (int i = 0; i < Q; i++) a.df[i * N + dense] = fluid ? f[i] : 0.f;
    return;
  }
  Mom<Q> m = moments<Q>(p, f);
  if (!fluid) m.rho = m.ux = m.uy = m.uz = 0.f;
  if (MODE == EX_MOM) {
    if (x >= p.nx) return;
    if (a.rho) a.rho[dense] = m.rho;
    if (a.u) {
      a.u[dense] = m.ux;
      a.u[N + dense] = m.uy;
      a.u[2 * N + dense] = m.uz;
    }
    return;
  }
}

// Sums over fluid cells, in two passes.  k_row_sums: one block per (y, z) row; a thread adds
// the values of its few cells of the row in FP32, the block adds the threads' partials in
// FP64 and writes partial[(z ny + y) K + k].  k_row_total then adds the rows in FP64:
//   EX_SUM   (K = 5: count, drho, j_x, j_y, j_z) -> sums[0] = count + sum drho = sum rho,
//            sums[1..3] = sum j = sum rho u (j includes F/2, so u = j / rho);
//   EX_STATS (K = 10: count, u_x, u_y, u_z, u_x^2, u_y^2, u_z^2, u_x u_y, u_x u_z, u_y u_z)
//            -> sums[y * 10 + k] += sum over the x-z plane y.
template <int MODE>
__host__ __device__ constexpr int row_k() { return MODE == EX_SUM ? 5 : 10; }

constexpr int ROW_THREADS = 128;

template <int Q, class S, int PAR, int MODE>
__global__ void __launch_bounds__(ROW_THREADS) k_row_sums(const __grid_constant__ KParams p, double* partial) {
  constexpr int K = row_k<MODE>();
  constexpr int NW = ROW_THREADS / 32;
  const int y = blockIdx.x, z = blockIdx.y;
  const int warp = threadIdx.x >> 5;
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = 0.f;
  for (int xb = 0; xb < p.nxp; xb += ROW_THREADS) {
    if (xb + warp * 32 >= p.nxp) break;  // warp-uniform (nxp is a multiple of 32)
    const int x = xb + threadIdx.x;
    const int cell = cidx(p, x, y, z);
    const int cls = x < p.nx ? cls_at(p, cell) : CLS_SKIP;
    float f[Q];
    unsigned outmask;
    load_state<Q, S, PAR>(p, x, y, z, cell, cls, f, outmask);
    outflow_fix<Q>(p, x, f, outmask);
    if (cls == CLS_SKIP) continue;
    const Mom<Q> m = moments<Q>(p, f);
    if (MODE == EX_SUM) {
      const float v[5] = {1.f, m.drho, m.jx, m.jy, m.jz};
#pragma unroll
      for (int k = 0; k < K; k++) acc[k] += v[k];
    } else {
      const float v[10] = {1.f, m.ux, m.uy, m.uz, m.ux * m.ux, m.uy * m.uy, m.uz * m.uz,
                           m.ux * m.uy, m.ux * m.uz, m.uy * m.uz};
#pragma unroll
      for (int k = 0; k < K; k++) acc[k] += v[k];
    }
  }
  __shared__ double red[K][NW];
#pragma unroll
  for (int k = 0; k < K; k++) {
    const double v = warp_sum((double)acc[k]);
    if ((threadIdx.x & 31) == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    const int k = threadIdx.x;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; w++) t += red[k][w];
    partial[((long long)z * p.ny + y) * K + k] = t;
  }
}

// EX_STATS: one block per plane y (its nz rows); EX_SUM: one block for all rows.
template <int MODE>
__global__ void __launch_bounds__(256) k_row_total(const double* partial, int ny, int nz, double* sums) {
  constexpr int K = row_k<MODE>();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; k++) acc[k] = 0.0;
  if (MODE == EX_STATS) {
    const int y = blockIdx.x;
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
#pragma unroll
      for (int k = 0; k < K; k++) acc[k] += partial[((long long)z * ny + y) * K + k];
    }
  } else {
    const long long nrow = (long long)ny * nz;
    for (long long r = threadIdx.x; r < nrow; r += blockDim.x) {
#pragma unroll
      for (int k = 0; k < K; k++) acc[k] += partial[r * K + k];
    }
  }
  __shared__ double red[K][8];
#pragma unroll
  for (int k = 0; k < K; k++) {
    const double v = warp_sum(acc[k]);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    const int k = threadIdx.x;
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[k][w];
    if (MODE == EX_STATS) {
      sums[blockIdx.x * 10 + k] += t;
    } else if (k == 0) {
      double t1 = 0.0;
      for (int w = 0; w < 8; w++) t1 += red[1][w];
      sums[0] = t + t1;  // count + sum drho
    } else if (k >= 2) {
      sums[k - 1] = t;
    }
  }
}

// f = f^eq(rho, u) (shifted) on fluid cells, 0 elsewhere; natural layout.
template <int Q, class S>
__global__ void __launch_bounds__(128) k_init_eq(const __grid_constant__ KParams p, const float* rho_in,
                                                 const float* u_in) {
  LBM_CELL_COORDS
  if (x >= p.nx) return;
  const long long dense = ((long long)z * p.ny + y) * p.nx + x;
  const long long N = (long long)p.nx * p.ny * p.nz;
  const bool fluid = cls != CLS_SKIP;
  const float rho = rho_in ? rho_in[dense] : 1.f;
  const float drho = rho - 1.f;
  const float ux = u_in ? u_in[dense] : 0.f, uy = u_in ? u_in[N + dense] : 0.f,
              uz = u_in ? u_in[2 * N + dense] : 0.f;
  const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const float v = wgt<Q>(i) * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * usq));
    stp<S>(p, plane_ptr<S>(p, i) + cell, fluid ? v : 0.f);
  }
}

// Natural-layout state from dense shifted float32 populations.
template <int Q, class S>
__global__ void __launch_bounds__(128) k_set_pop(const __grid_constant__ KParams p, const float* df) {
  LBM_CELL_COORDS
  if (x >= p.nx) return;
  const long long dense = ((long long)z * p.ny + y) * p.nx + x;
  const long long N = (long long)p.nx * p.ny * p.nz;
  const bool fluid = cls != CLS_SKIP;
#pragma unroll
  for (int i = 0; i < Q; i++) stp<S>(p, plane_ptr<S>(p, i) + cell, fluid ? df[i * N + dense] : 0.f);
}

}  // namespace lbm
