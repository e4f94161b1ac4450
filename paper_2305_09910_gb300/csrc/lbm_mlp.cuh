// lbm_mlp.cuh -- the stream-collide step with the learned closure, its 32x32 hidden layer on
// the fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory).
//
// Per tile of 128 cells (one CTA: 4 warps, each 32 x-consecutive cells of one row) every
// thread loads its cell, forms the moments and the non-equilibrium stress, evaluates the
// first layer (7 -> 32, GELU) in FP32 and writes the 32 hidden values, rounded to TF32, as
// row t of a 128 x 32 operand tile in shared memory.  One thread issues four
// tcgen05.mma.kind::tf32 (M = 128, N = 32, K = 8 each) against W2 (bf16 values, exact in TF32)
// into 32 columns of tensor memory and commits them to an mbarrier.  Each warp then reads its
// 32 TMEM lanes with tcgen05.ld -- lane t of the accumulator is exactly cell t's 32 outputs,
// so the epilogue (bias, GELU, 32 -> 1 output layer, softplus) stays one thread per cell --
// and the thread finishes the TRT update with the learned C_s^2.
//
// The CTA is persistent and holds MLP_NG independent groups of 128 threads (4 warps each):
// the runtime schedules one CTA per multiprocessor for a kernel that allocates tensor memory,
// so the groups are what keeps several tiles in flight per SM.  Group g owns TMEM columns
// 32g .. 32g+31 (warp w of the CTA reads lanes 32 (w % 4) .. +31), its own operand tile and
// mbarrier, and synchronises on named barrier 1 + g; TMEM (32 MLP_NG columns) is allocated
// once and W2 staged once per CTA.  Operand
// tiles use the no-swizzle K-major layout of 8-row x 16-byte core matrices: element (r, k) of
// a 4-byte-element tile at (r / 8) * 1024 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4, i.e.
// leading-dimension byte offset 128 (K-adjacent core matrices), stride byte offset 1024
// (8-row groups).  Every mbarrier wait is bounded.  When a group's first wait for a tile's MMA
// gives up (after p.wait_polls polls), the group sets status bit 1, waits again with the full
// bound so that the tensor core has finished with its accumulator and operand tile, and leaves
// its tile loop; the CTA then frees its tensor memory and returns.  Should that second wait
// give up too, status bit 2 records that the MMA may still be running: the launch's results
// and the tensor memory it held are then undefined.
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

// shared-memory matrix descriptor: start, leading byte offset 128, stride byte offset 1024,
// descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ int core_off(int r, int k) {  // in floats
  return (r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
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

struct MlpSmem {
  float A[MLP_NG][MLP_TILE * MLP_NH];  // hidden layer 1 per group, TF32, core-matrix layout (16 KB each)
  float B[MLP_NH * MLP_NH];            // W2, core-matrix layout (4 KB)
  // layers 1 and 3 as pairs of hidden units (j, j+1) for the packed FP32x2 pipe
  float2 W1[MLP_NH / 2][MLP_NIN], b1[MLP_NH / 2], b2[MLP_NH / 2], W3[MLP_NH / 2];
  float b3;
  unsigned long long bar[MLP_NG];
  uint32_t tmem;
};

__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ __forceinline__ bool group_any(int id, bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, %2, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(r)
               : "r"((uint32_t)v), "r"(id)
               : "memory");
  return r != 0;
}

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
    for (int k = tc; k < MLP_NH * MLP_NH; k += 128 * MLP_NG) {
      const int n = k / MLP_NH, kk = k % MLP_NH;  // output n, input kk
      sm.B[core_off(n, kk)] = W2[k];
    }
    for (int k = tc; k < (MLP_NH / 2) * MLP_NIN; k += 128 * MLP_NG) {
      const int jp = k / MLP_NIN, i = k % MLP_NIN;
      sm.W1[jp][i] = make_float2(W1[(2 * jp) * MLP_NIN + i], W1[(2 * jp + 1) * MLP_NIN + i]);
    }
    if (tc < MLP_NH / 2) {
      sm.b1[tc] = make_float2(b1[2 * tc], b1[2 * tc + 1]);
      sm.b2[tc] = make_float2(b2[2 * tc], b2[2 * tc + 1]);
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
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W2 tile -> tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  const uint32_t tmem = sm.tmem;
  const uint32_t dcol = tmem + 32u * g;                          // this group's accumulator
  const uint32_t tl = dcol + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
  const uint32_t bar = cta_addr(&sm.bar[g]);
  float* const A = sm.A[g];
  const uint32_t a0 = cta_addr(A), b0 = cta_addr(sm.B);
  const int nbx = p.nxp / 32, nby = (p.ny + 3) / 4;
  const int gbar = 1 + g;  // named barrier of the group (0 is __syncthreads)
  uint32_t phase = 0;
  for (long long tile = (long long)blockIdx.x * MLP_NG + g; tile < ntiles; tile += (long long)gridDim.x * MLP_NG) {
    const int bx = (int)(tile % nbx);
    const long long r = tile / nbx;
    const int by = (int)(r % nby);
    const int z = (int)(r / nby);
    const int x = bx * 32 + threadIdx.x;
    const int y = by * 4 + (warp & 3);
    const bool row = y < p.ny;  // warp-uniform
    const int cell = row ? cidx(p, x, y, z) : 0;
    const int cls = (row && x < p.nx) ? cls_at(p, cell) : CLS_SKIP;
    float f[Q];
    unsigned outmask;
    load_state<Q, S, LOAD>(p, x, y, z, cell, cls, f, outmask);
    outflow_fix<Q>(p, x, f, outmask);
    const Macro<float> M = macro<Q, true, float>(p, f);
    // layer 1 (FP32, two hidden units per packed FP32x2 operation), GELU, TF32 rounding,
    // row t of the operand tile
    float xin[MLP_NIN];
#pragma unroll
    for (int k = 0; k < 6; k++) xin[k] = fminf(fmaxf(p.mlp_scale[0] * M.pi[k], -MLP_XCLAMP), MLP_XCLAMP);
    xin[6] = fminf(fmaxf(p.mlp_scale[1] * M.drho, -MLP_XCLAMP), MLP_XCLAMP);
#pragma unroll
    for (int c4 = 0; c4 < MLP_NH / 4; c4++) {
      float2 s01 = sm.b1[2 * c4], s23 = sm.b1[2 * c4 + 1];
#pragma unroll
      for (int k = 0; k < MLP_NIN; k++) {
        const float2 xk = make_float2(xin[k], xin[k]);
        s01 = vfma(sm.W1[2 * c4][k], xk, s01);
        s23 = vfma(sm.W1[2 * c4 + 1][k], xk, s23);
      }
      const float2 g01 = gelu_v(s01), g23 = gelu_v(s23);
      *reinterpret_cast<uint4*>(A + core_off(t, 4 * c4)) =
          make_uint4(to_tf32(g01.x), to_tf32(g01.y), to_tf32(g23.x), to_tf32(g23.y));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(gbar);
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < MLP_NH / 8; kk++) {  // K = 8 per instruction: 2 core matrices = 256 B
        const uint64_t da = umma_desc(a0 + kk * 256), db = umma_desc(b0 + kk * 256);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
            "l"(da), "l"(db), "r"(MLP_IDESC), "r"(kk)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
    }
    const bool timed_out = !mbar_wait_parity(bar, phase, p.wait_polls);
    if (group_any(gbar, timed_out)) {
      // give up on this launch, but only after the MMA has finished with the accumulator and
      // the operand tile (the commit still arrives on the barrier)
      if (t == 0) atomicOr(p.status, 2);
      if (!mbar_wait_parity(bar, phase, MBAR_POLLS)) atomicOr(p.status, 4);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    // epilogue: this thread's 32 accumulator columns, bias, GELU, output layer (pairs)
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int half = 0; half < 2; half++) {
      float v[16];
      tmem_ld16(tl + 16 * half, v);
#pragma unroll
      for (int pr = 0; pr < 8; pr++) {
        const float2 a2 = vadd(make_float2(v[2 * pr], v[2 * pr + 1]), sm.b2[8 * half + pr]);
        acc = vfma(sm.W3[8 * half + pr], gelu_v(a2), acc);
      }
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
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MLP_TMEM_COLS) : "memory");
}

}  // namespace lbm
