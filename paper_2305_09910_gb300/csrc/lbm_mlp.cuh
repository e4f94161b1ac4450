// lbm_mlp.cuh -- the stream-collide step with the learned closure, its two hidden layers on
// the fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory).
//
// Per tile of 128 cells (one group: 4 warps, each 32 x-consecutive cells of one row) every
// thread loads its cell, forms the moments and the non-equilibrium stress, and writes its 7
// scaled features and a constant 1 (which carries the bias b1), rounded to TF32, as row t of
// a 128 x 8 operand tile in shared memory.  One thread issues tcgen05.mma.kind::tf32
// (M = 128, N = 32, K = 8) against [W1 | b1] into 32 columns of tensor memory and commits it
// to an mbarrier; each warp reads its 32 TMEM lanes with tcgen05.ld (lane t = cell t's 32
// pre-activations), applies the GELU and writes row t of the 128 x 40 layer-2 operand, again
// in TF32 (columns 32..39 hold a constant 1, carrying b2, and zeros, written once per CTA).
// Five more MMAs (K = 5 x 8) against [W2 | b2 | 0] overwrite the same TMEM columns; the
// epilogue (GELU, 32 -> 1 output layer, softplus) stays one thread per cell and the thread
// finishes the TRT update with the learned C_s^2.  Weights are bfloat16 values, exact
// in TF32.
//
// The CTA is persistent and holds MLP_NG independent groups of 128 threads (4 warps each),
// which keep several tiles in flight per SM.  Group g owns TMEM columns 32g .. 32g+31 (warp w
// of the CTA reads lanes 32 (w % 4) .. +31), its own operand tiles and mbarrier, and
// synchronises on named barrier 1 + g; TMEM (32 MLP_NG columns) is allocated once and the
// weights staged once per CTA.  Operand tiles use the no-swizzle K-major layout of 8-row x
// 16-byte core matrices: element (r, k) of a 4-byte-element tile of K columns at
// (r / 8) * 32 K + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4 bytes, i.e. leading-dimension
// byte offset 128 (K-adjacent core matrices) and stride byte offset 32 K (8-row groups).
// Every mbarrier wait is bounded.  When a thread's first wait for a tile's MMA gives up (after
// p.wait_polls polls), it sets status bit 1 and waits again with the full bound, so that the
// tensor core has finished with its accumulator and operand tiles before it reads them; the
// tile is then completed as usual.  Should that second wait give up too, status bit 2 records
// that the MMA may still be running: the launch's results and the tensor memory it held are
// then undefined.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int MLP_TILE = 128;                     // cells per tile (TMEM lanes, MMA M)
#ifndef LBM_MLP_NG
#define LBM_MLP_NG 7
#endif
constexpr int MLP_NG = LBM_MLP_NG;                // tile groups per CTA
constexpr unsigned MLP_TMEM_COLS = MLP_NG <= 1 ? 32 : MLP_NG <= 2 ? 64 : MLP_NG <= 4 ? 128 : 256;  // allocation: 32 per group, power of 2
// instruction descriptor of tcgen05.mma.kind::tf32: D f32 (bits 4-5 = 1), A and B tf32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t MLP_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t cta_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading byte offset 128, stride byte offset sbo
// (32 K bytes for a tile of K 4-byte columns), descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// offset (in floats) of element (r, k) of a tile of K columns in the core-matrix layout
template <int K>
__device__ __forceinline__ int core_off(int r, int k) {
  return (r >> 3) * (8 * K) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// one tcgen05.mma.kind::tf32 (M = 128, N = 32, K = 8): D (+)= A B^T, D in tensor memory
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t da, uint64_t db, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(da), "l"(db), "r"(MLP_IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init1(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// polls of a full mbarrier wait (each try_wait may itself suspend the thread for a while)
constexpr int MBAR_POLLS = 1 << 22;

__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, int polls) {
  for (int it = 0; it < polls; it++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

constexpr int MLP_K1 = 8;   // layer-1 operand columns: the 7 features and a constant 1
constexpr int MLP_K2 = 40;  // layer-2 operand columns: 32 hidden values, a constant 1 and 7 zeros

struct MlpSmem {
  float A[MLP_NG][MLP_TILE * MLP_K2];  // layer-2 operand per group (hidden layer 1, 1; TF32; 20 KB each)
  float X[MLP_NG][MLP_TILE * MLP_K1];  // layer-1 operand per group (features and 1, TF32; 4 KB each)
  float B[MLP_NH * MLP_K2];            // [W2 | b2 | 0] (5 KB)
  float B1[MLP_NH * MLP_K1];           // [W1 | b1] (1 KB)
  // the output layer as pairs of hidden units (j, j+1) for the packed FP32x2 pipe
  float2 W3[MLP_NH / 2];
  float b3;
  unsigned long long bar[MLP_NG];
  uint32_t tmem;
};

__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// LOAD / STORE modes as in k_step.  Grid: persistent CTAs whose groups walk tiles (bx, by, z)
// of (nxp/32) x ceil(ny/4) x nz; block (32, 4 MLP_NG).
template <int Q, class S, int LOAD, int STORE>
__global__ void __launch_bounds__(128 * MLP_NG, 1) k_step_mlp(const __grid_constant__ KParams p, long long ntiles) {
  extern __shared__ __align__(1024) unsigned char mlp_smem_raw[];
  MlpSmem& sm = *reinterpret_cast<MlpSmem*>(mlp_smem_raw);
  const int warp = threadIdx.y;              // 0 .. 4 MLP_NG - 1
  const int g = warp >> 2;                   // group
  const int t = (warp & 3) * 32 + threadIdx.x;  // row of the group's tile = TMEM lane
  const int tc = threadIdx.y * 32 + threadIdx.x;  // thread of the CTA
  {
    const float* W1 = p.mlp;
    const float* b1 = W1 + MLP_NH * MLP_NIN;
    const float* W2 = b1 + MLP_NH;
    const float* b2 = W2 + MLP_NH * MLP_NH;
    const float* W3 = b2 + MLP_NH;
    for (int k = tc; k < MLP_NH * MLP_K2; k += 128 * MLP_NG) {
      const int n = k / MLP_K2, kk = k % MLP_K2;  // output n, input kk (kk = 32: the bias)
      sm.B[core_off<MLP_K2>(n, kk)] = kk < MLP_NH ? W2[n * MLP_NH + kk] : kk == MLP_NH ? b2[n] : 0.f;
    }
    // the constant columns of every group's layer-2 operand: 1 (carrying b2), then zeros
    for (int k = tc; k < MLP_NG * MLP_TILE; k += 128 * MLP_NG) {
      float* A = sm.A[k / MLP_TILE];
      const int r = k % MLP_TILE;
      *reinterpret_cast<uint4*>(A + core_off<MLP_K2>(r, MLP_NH)) = make_uint4(__float_as_uint(1.f), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(A + core_off<MLP_K2>(r, MLP_NH + 4)) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int k = tc; k < MLP_NH * MLP_K1; k += 128 * MLP_NG) {
      const int n = k / MLP_K1, kk = k % MLP_K1;  // output n, input kk (kk = 7: the bias)
      sm.B1[core_off<MLP_K1>(n, kk)] = kk < MLP_NIN ? W1[n * MLP_NIN + kk] : b1[n];
    }
    if (tc < MLP_NH / 2) {
      sm.W3[tc] = make_float2(W3[2 * tc], W3[2 * tc + 1]);
    }
    if (tc == 0) {
      sm.b3 = W3[MLP_NH];
      for (int k = 0; k < MLP_NG; k++) mbar_init1(cta_addr(&sm.bar[k]));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cta_addr(&sm.tmem)),
                   "r"(MLP_TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // weight tiles -> tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  const uint32_t tmem = sm.tmem;
  const uint32_t dcol = tmem + 32u * g;                          // this group's accumulator
  const uint32_t tl = dcol + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
  const uint32_t bar = cta_addr(&sm.bar[g]);
  float* const A = sm.A[g];
  float* const X = sm.X[g];
  const uint32_t a0 = cta_addr(A), x0 = cta_addr(X), b0 = cta_addr(sm.B), b10 = cta_addr(sm.B1);
  const int nbx = p.nxp / 32, nby = (p.ny + 3) / 4;
  const int gbar = 1 + g;  // named barrier of the group (0 is __syncthreads)
  uint32_t phase = 0;
  // Waits for the group's MMA.  A thread whose first wait gives up records it (status bit 1)
  // and waits again with the full bound, so that the tensor core has finished with the
  // accumulator and operand tiles before the thread goes on; every thread then keeps the
  // group's barrier sequence (no thread leaves the loop on its own).  Should that wait give up
  // too, status bit 2 records that the MMA may still be running.
  auto wait_mma = [&]() {
    if (!mbar_wait_parity(bar, phase, p.wait_polls)) {
      atomicOr(p.status, 2);
      if (!mbar_wait_parity(bar, phase, MBAR_POLLS)) atomicOr(p.status, 4);
    }
    phase ^= 1u;
    tc_fence_after();
  };
  // Makes the group's shared-memory operand rows visible to the tensor core, then has thread 0
  // of the group issue the layer's MMAs and commit them to the group's mbarrier.
  auto issue = [&](bool layer1) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(gbar);
    if (t == 0) {
      tc_fence_after();
      if (layer1) {
        mma_tf32(dcol, umma_desc(x0, 32 * MLP_K1), umma_desc(b10, 32 * MLP_K1), 0);
      } else {
#pragma unroll
        for (int kk = 0; kk < MLP_K2 / 8; kk++)  // K = 8 per instruction: 2 core matrices = 256 B
          mma_tf32(dcol, umma_desc(a0 + kk * 256, 32 * MLP_K2), umma_desc(b0 + kk * 256, 32 * MLP_K2), kk);
      }
      mma_commit(bar);
    }
  };
  // tile coordinates in 32-bit unsigned arithmetic (the launcher keeps ntiles below 2^31): a
  // 64-bit division by a runtime value costs far more instructions
  const unsigned nt = (unsigned)ntiles, unbx = (unsigned)nbx, unby = (unsigned)nby;
  for (unsigned tile = blockIdx.x * MLP_NG + g; tile < nt; tile += gridDim.x * MLP_NG) {
    const unsigned r = tile / unbx;
    const int bx = (int)(tile - r * unbx);
    const unsigned zq = r / unby;
    const int by = (int)(r - zq * unby);
    const int z = (int)zq;
    const int x = bx * 32 + threadIdx.x;
    const int y = by * 4 + (warp & 3);
    const bool row = y < p.ny;  // warp-uniform
    const int cell = row ? cidx(p, x, y, z) : 0;
    float f[Q];
    unsigned outmask = 0;
    const bool early = LOAD != 0 && row && off_faces(p, x, y, z);
    if (early) gather_interior<Q, S, LOAD>(p, cell, f);  // in flight with the class load below
    const int cls = (row && x < p.nx) ? cls_at(p, cell) : CLS_SKIP;
    if (!(early && cls == CLS_INTERIOR)) load_state<Q, S, LOAD>(p, x, y, z, cell, cls, f, outmask);
    outflow_fix<Q>(p, x, f, outmask);
    const Macro<float> M = macro<Q, true, float>(p, f);
    // layer 1 on the tensor core: row t of the feature tile = the 7 clipped, scaled features
    // and 1 (the bias column), in TF32
    {
      float xin[MLP_NIN];
#pragma unroll
      for (int k = 0; k < 6; k++) xin[k] = fminf(fmaxf(p.mlp_scale[0] * M.pi[k], -MLP_XCLAMP), MLP_XCLAMP);
      xin[6] = fminf(fmaxf(p.mlp_scale[1] * M.drho, -MLP_XCLAMP), MLP_XCLAMP);
      *reinterpret_cast<uint4*>(X + core_off<MLP_K1>(t, 0)) =
          make_uint4(to_tf32(xin[0]), to_tf32(xin[1]), to_tf32(xin[2]), to_tf32(xin[3]));
      *reinterpret_cast<uint4*>(X + core_off<MLP_K1>(t, 4)) =
          make_uint4(to_tf32(xin[4]), to_tf32(xin[5]), to_tf32(xin[6]), __float_as_uint(1.f));
    }
    issue(true);
    wait_mma();
    // GELU of the 32 pre-activations (this thread's TMEM lane), TF32, row t of the layer-2 tile
#pragma unroll
    for (int half = 0; half < 2; half++) {
      float v[16];
      tmem_ld16(tl + 16 * half, v);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const float2 g01 = gelu_v(make_float2(v[4 * c], v[4 * c + 1]));
        const float2 g23 = gelu_v(make_float2(v[4 * c + 2], v[4 * c + 3]));
        *reinterpret_cast<uint4*>(A + core_off<MLP_K2>(t, 16 * half + 4 * c)) =
            make_uint4(to_tf32(g01.x), to_tf32(g01.y), to_tf32(g23.x), to_tf32(g23.y));
      }
    }
    issue(false);  // (its barrier also orders every lane's layer-1 reads before the overwrite)
    wait_mma();
    // epilogue: this thread's 32 accumulator columns (b2 included), GELU, output layer (pairs)
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int half = 0; half < 2; half++) {
      float v[16];
      tmem_ld16(tl + 16 * half, v);
#pragma unroll
      for (int pr = 0; pr < 8; pr++)
        acc = vfma(sm.W3[8 * half + pr], gelu_v(make_float2(v[2 * pr], v[2 * pr + 1])), acc);
    }
    const float yv = sm.b3 + (acc.x + acc.y);
    const float cs2 = fmaxf(softplus_f(yv) * p.cs2 * 1.4426950408889634f, p.cs2_min);  // / ln 2
    float wp, wm;
    les_rates(p, M.qn, M.inv, cs2, wp, wm);
    relax<Q, float, acc_form<S>>(p, f, M, wp, wm);
    if (cls != CLS_SKIP) {
      if (!(M.rho > 0.f && M.rho < 3.0e38f)) atomicOr(p.status, 1);
      store_state<Q, S, STORE>(p, x, y, z, cell, cls, f);
    }
    // the next tile's layer-1 MMA overwrites these TMEM columns: order this lane's reads first
    tc_fence_before();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MLP_TMEM_COLS) : "memory");
}

}  // namespace lbm
