// lbm_closure.cu -- learned closure: training samples from a fine lattice (box filter of
// width 2), the 7 -> 32 -> 32 -> 1 GELU network's forward and backward passes, the
// eddy-viscosity loss, and the Adam optimiser, all as CUDA kernels behind C entry points.
//
// The network gives the Smagorinsky coefficient of each cell, C_s^2 = softplus(y) C_s0^2 /
// ln 2, from the cell's non-equilibrium stress and density; its inference runs inside the
// collide kernel (lbm_kernels.cuh, mlp_cs2).  Training pairs come from the solver itself:
// a fine lattice is filtered onto the coarse grid (half resolution), and the target is the
// eddy viscosity that best reproduces the filtered subgrid stress (least-squares
// projection on the coarse strain rate).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

void lbm_internal_set_error(const char* msg);

namespace lbm {

// ---- training samples -------------------------------------------------------------------
struct SampleArgs {
  float* x;        // nc * 7
  float* target;   // nc
  float* smag;     // nc, |S_c|
  float* weight;   // nc, |S_c|^2
  int ncx, ncy, ncz;
  float tau0_c, cs0sq, scale_pi, scale_rho;
  int smag_fine;   // the fine lattice uses the Smagorinsky closure
};

template <int Q, class S, int PAR>
__global__ void __launch_bounds__(128) k_closure_samples(const __grid_constant__ KParams p, SampleArgs a) {
  const long long nc = (long long)a.ncx * a.ncy * a.ncz;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  const int X = (int)(k % a.ncx), Y = (int)((k / a.ncx) % a.ncy), Z = (int)(k / ((long long)a.ncx * a.ncy));
  float rho_k[8], ux_k[8], uy_k[8], uz_k[8];
  float rho_s = 0.f, m_s[3] = {0.f, 0.f, 0.f}, S_s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float nS_s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  bool all_fluid = true;
#pragma unroll 1
  for (int n = 0; n < 8; n++) {
    const int fx = 2 * X + (n & 1), fy = 2 * Y + ((n >> 1) & 1), fz = 2 * Z + (n >> 2);
    const int cell = cidx(p, fx, fy, fz);
    const int cls = cls_at(p, cell);
    float f[Q];
    unsigned outmask;
    load_state<Q, S, PAR>(p, fx, fy, fz, cell, cls, f, outmask);
    if (cls == CLS_SKIP) {
      all_fluid = false;
      rho_k[n] = ux_k[n] = uy_k[n] = uz_k[n] = 0.f;
      continue;
    }
    const Mom<Q> m = moments<Q>(p, f);
    // non-equilibrium stress (shifted form), as in the collision
    float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      if (cx(i)) sxx += f[i];
      if (cy(i)) syy += f[i];
      if (cz(i)) szz += f[i];
      if (cx(i) * cy(i)) sxy += cx(i) * cy(i) > 0 ? f[i] : -f[i];
      if (cx(i) * cz(i)) sxz += cx(i) * cz(i) > 0 ? f[i] : -f[i];
      if (cy(i) * cz(i)) syz += cy(i) * cz(i) > 0 ? f[i] : -f[i];
    }
    const float d3 = m.drho * (1.f / 3.f);
    const float pi[6] = {sxx - d3 - m.jx * m.ux, syy - d3 - m.jy * m.uy, szz - d3 - m.jz * m.uz,
                         sxy - m.jx * m.uy, sxz - m.jx * m.uz, syz - m.jy * m.uz};
    const float qn = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] +
                     2.f * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]);
    float tau = p.tau0;
    if (a.smag_fine)
      tau = 0.5f * (p.tau0 + sqrtf(p.tau0 * p.tau0 + 25.455844122715711f * p.cs2 * sqrtf(qn) / m.rho));
    const float nut = (tau - p.tau0) * (1.f / 3.f);
    const float sfac = -3.f / (2.f * m.rho * tau);
    rho_k[n] = m.rho;
    ux_k[n] = m.ux;
    uy_k[n] = m.uy;
    uz_k[n] = m.uz;
    rho_s += m.rho;
    m_s[0] += m.jx;
    m_s[1] += m.jy;
    m_s[2] += m.jz;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      S_s[j] += sfac * pi[j];
      nS_s[j] += nut * sfac * pi[j];
    }
  }
  float* xo = a.x + k * 7;
  if (!all_fluid) {
    for (int j = 0; j < 7; j++) xo[j] = 0.f;
    a.target[k] = 0.f;
    a.smag[k] = 0.f;
    a.weight[k] = 0.f;
    return;
  }
  const float rb = rho_s * 0.125f;
  const float ub[3] = {m_s[0] / rho_s, m_s[1] / rho_s, m_s[2] / rho_s};
  // Favre variance from deviations (no cancellation): sum rho (u - u_bar)(u - u_bar) / sum rho
  float R[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int n = 0; n < 8; n++) {
    const float dx = ux_k[n] - ub[0], dy = uy_k[n] - ub[1], dz = uz_k[n] - ub[2];
    R[0] += rho_k[n] * dx * dx;
    R[1] += rho_k[n] * dy * dy;
    R[2] += rho_k[n] * dz * dz;
    R[3] += rho_k[n] * dx * dy;
    R[4] += rho_k[n] * dx * dz;
    R[5] += rho_k[n] * dy * dz;
  }
  float tsg[6], Sc[6];
#pragma unroll
  for (int j = 0; j < 6; j++) {
    tsg[j] = R[j] / rho_s - 2.f * nS_s[j] * 0.125f;
    Sc[j] = 2.f * S_s[j] * 0.125f;
  }
  const float tr = (tsg[0] + tsg[1] + tsg[2]) * (1.f / 3.f);
  float num = 0.f, den = 0.f;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    const float mult = j < 3 ? 1.f : 2.f;
    const float td = j < 3 ? tsg[j] - tr : tsg[j];
    num += mult * td * Sc[j];
    den += mult * Sc[j] * Sc[j];
  }
  const float Smag = sqrtf(2.f * den);
  float nu = Smag > 1e-10f ? -num / (2.f * den) : 0.f;
  nu = fmaxf(nu, 0.f);
  const float tauc = a.tau0_c + 3.f * a.cs0sq * Smag;
#pragma unroll
  for (int j = 0; j < 6; j++)
    xo[j] = fminf(fmaxf(a.scale_pi * (-(2.f * rb / 3.f) * tauc * Sc[j]), -MLP_XCLAMP), MLP_XCLAMP);
  xo[6] = fminf(fmaxf(a.scale_rho * (rb - 1.f), -MLP_XCLAMP), MLP_XCLAMP);
  a.target[k] = nu;
  a.smag[k] = Smag;
  a.weight[k] = Smag * Smag;
}

// Box filter of width 2: mean density and Favre velocity of each coarse cell's 8 fine cells.
template <int Q, class S, int PAR>
__global__ void __launch_bounds__(128) k_filter2(const __grid_constant__ KParams p, int ncx, int ncy, int ncz,
                                                 float* rho_bar, float* u_bar) {
  const long long nc = (long long)ncx * ncy * ncz;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  const int X = (int)(k % ncx), Y = (int)((k / ncx) % ncy), Z = (int)(k / ((long long)ncx * ncy));
  float rs = 0.f, ms[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int n = 0; n < 8; n++) {
    const int fx = 2 * X + (n & 1), fy = 2 * Y + ((n >> 1) & 1), fz = 2 * Z + (n >> 2);
    const int cell = cidx(p, fx, fy, fz);
    const int cls = cls_at(p, cell);
    if (cls == CLS_SKIP) continue;
    float f[Q];
    unsigned outmask;
    load_state<Q, S, PAR>(p, fx, fy, fz, cell, cls, f, outmask);
    const Mom<Q> m = moments<Q>(p, f);
    rs += m.rho;
    ms[0] += m.jx;
    ms[1] += m.jy;
    ms[2] += m.jz;
  }
  rho_bar[k] = rs * 0.125f;
  const float inv = rs > 0.f ? 1.f / rs : 0.f;
  u_bar[k] = ms[0] * inv;
  u_bar[nc + k] = ms[1] * inv;
  u_bar[2 * nc + k] = ms[2] * inv;
}

// ---- network -------------------------------------------------------------------------------
constexpr int TB = 128;  // samples per block in the training kernels

__device__ __forceinline__ float mlp_forward_one(const float* W, const float* x, float* h1, float* g1,
                                                 float* h2, float* g2) {
  const float* W1 = W;
  const float* b1 = W1 + MLP_NH * MLP_NIN;
  const float* W2 = b1 + MLP_NH;
  const float* b2 = W2 + MLP_NH * MLP_NH;
  const float* W3 = b2 + MLP_NH;
  const float* b3 = W3 + MLP_NH;
#pragma unroll 4
  for (int j = 0; j < MLP_NH; j++) {
    float s = b1[j];
#pragma unroll
    for (int k = 0; k < MLP_NIN; k++) s = fmaf(W1[j * MLP_NIN + k], x[k], s);
    h1[j] = gelu_erf(s);
    if (g1) g1[j] = gelu_grad_f(s);
  }
  float y = b3[0];
#pragma unroll 2
  for (int j = 0; j < MLP_NH; j++) {
    float s = b2[j];
#pragma unroll
    for (int k = 0; k < MLP_NH; k++) s = fmaf(W2[j * MLP_NH + k], h1[k], s);
    const float h = gelu_erf(s);
    if (h2) h2[j] = h;
    if (g2) g2[j] = gelu_grad_f(s);
    y = fmaf(W3[j], h, y);
  }
  return y;
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ x,
                                                     long long n, float* __restrict__ y) {
  __shared__ float W[MLP_NPARAM];
  for (int j = threadIdx.x; j < MLP_NPARAM; j += blockDim.x) W[j] = params[j];
  __syncthreads();
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float xs[MLP_NIN], h1[MLP_NH];
#pragma unroll
  for (int k = 0; k < MLP_NIN; k++) xs[k] = x[s * MLP_NIN + k];
  y[s] = mlp_forward_one(W, xs, h1, nullptr, nullptr, nullptr);
}

// Mode of the backward kernel: given dy per sample, or the eddy-viscosity loss.
enum : int { BW_DY = 0, BW_LOSS = 1 };

struct BackArgs {
  const float* params;
  const float* x;
  const float* dy;       // BW_DY
  const float* target;   // BW_LOSS
  const float* smag;
  const float* weight;
  long long n;           // samples in the batch
  long long offset, stride;  // sample s of the batch is offset + s * stride
  float k;               // C_s0^2 / ln 2
  float* grad;           // MLP_NPARAM, accumulated (FP32 atomics)
  double* sums;          // BW_LOSS: [sum w, sum w r^2]
};

// One block = TB samples, one thread per sample for the per-sample passes, then the
// parameter gradients summed over the block's samples in shared memory (block-level
// GEMM-shaped reductions) and added to the global gradient.
template <int MODE>
__global__ void __launch_bounds__(TB) k_mlp_backward(const __grid_constant__ BackArgs a) {
  extern __shared__ float sm[];
  float* W = sm;                          // MLP_NPARAM
  float* H1 = W + MLP_NPARAM + 3;         // [NH][TB]
  float* D1 = H1 + MLP_NH * TB;           // [NH][TB] gelu'(a1), then dA1
  float* H2 = D1 + MLP_NH * TB;           // [NH][TB]
  float* D2 = H2 + MLP_NH * TB;           // [NH][TB] dA2
  float* XS = D2 + MLP_NH * TB;           // [NIN][TB]
  float* DY = XS + MLP_NIN * TB;          // [TB]
  for (int j = threadIdx.x; j < MLP_NPARAM; j += TB) W[j] = a.params[j];
  __syncthreads();
  const float* W2 = W + MLP_NH * MLP_NIN + MLP_NH;
  const float* W3 = W2 + MLP_NH * MLP_NH + MLP_NH;
  const int t = threadIdx.x;
  const long long s = (long long)blockIdx.x * TB + t;
  const bool valid = s < a.n;
  float dy = 0.f;
  {
    float xs[MLP_NIN], h1[MLP_NH], g1[MLP_NH], h2[MLP_NH], g2[MLP_NH];
    const long long gs = a.offset + s * a.stride;
#pragma unroll
    for (int k = 0; k < MLP_NIN; k++) xs[k] = valid ? a.x[gs * MLP_NIN + k] : 0.f;
    const float y = mlp_forward_one(W, xs, h1, g1, h2, g2);
    if (valid) {
      if (MODE == BW_DY) {
        dy = a.dy[s];
      } else {
        const float S = a.smag[gs], w = a.weight[gs];
        const float sp = fmaxf(y, 0.f) + log1pf(expf(-fabsf(y)));
        const float sg = 1.f / (1.f + expf(-y));
        const float r = sp * a.k * S - a.target[gs];
        dy = 2.f * w * r * a.k * S * sg;  // unnormalised; scaled by 1 / sum w afterwards
        atomicAdd(a.sums + 0, (double)w);
        atomicAdd(a.sums + 1, (double)w * (double)r * (double)r);
      }
    }
#pragma unroll
    for (int k = 0; k < MLP_NIN; k++) XS[k * TB + t] = xs[k];
#pragma unroll
    for (int j = 0; j < MLP_NH; j++) {
      H1[j * TB + t] = h1[j];
      D1[j * TB + t] = g1[j];
      H2[j * TB + t] = h2[j];
      D2[j * TB + t] = dy * W3[j] * g2[j];
    }
    DY[t] = dy;
  }
  __syncthreads();
  // dA1 = (W2^T dA2) * gelu'(a1), per sample
  {
    float d1[MLP_NH];
#pragma unroll
    for (int k = 0; k < MLP_NH; k++) d1[k] = 0.f;
#pragma unroll 4
    for (int j = 0; j < MLP_NH; j++) {
      const float d2 = D2[j * TB + t];
#pragma unroll
      for (int k = 0; k < MLP_NH; k++) d1[k] = fmaf(W2[j * MLP_NH + k], d2, d1[k]);
    }
#pragma unroll
    for (int k = 0; k < MLP_NH; k++) D1[k * TB + t] *= d1[k];
  }
  __syncthreads();
  // parameter gradients: sums over the block's samples
  float* G = a.grad;
  for (int e = t; e < MLP_NPARAM; e += TB) {
    float acc = 0.f;
    if (e < MLP_NH * MLP_NIN) {                       // W1[j][k] += dA1[j] x[k]
      const int j = e / MLP_NIN, k = e % MLP_NIN;
      for (int q = 0; q < TB; q++) acc = fmaf(D1[j * TB + q], XS[k * TB + q], acc);
    } else if (e < MLP_NH * MLP_NIN + MLP_NH) {       // b1[j] += dA1[j]
      const int j = e - MLP_NH * MLP_NIN;
      for (int q = 0; q < TB; q++) acc += D1[j * TB + q];
    } else if (e < MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH) {  // W2[j][k] += dA2[j] h1[k]
      const int r = e - (MLP_NH * MLP_NIN + MLP_NH);
      const int j = r / MLP_NH, k = r % MLP_NH;
      for (int q = 0; q < TB; q++) acc = fmaf(D2[j * TB + q], H1[k * TB + q], acc);
    } else if (e < MLP_NH * MLP_NIN + 2 * MLP_NH + MLP_NH * MLP_NH) {  // b2[j] += dA2[j]
      const int j = e - (MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH);
      for (int q = 0; q < TB; q++) acc += D2[j * TB + q];
    } else if (e < MLP_NPARAM - 1) {                 // W3[k] += dy h2[k]
      const int k = e - (MLP_NH * MLP_NIN + 2 * MLP_NH + MLP_NH * MLP_NH);
      for (int q = 0; q < TB; q++) acc = fmaf(DY[q], H2[k * TB + q], acc);
    } else {                                          // b3 += dy
      for (int q = 0; q < TB; q++) acc += DY[q];
    }
    atomicAdd(G + e, acc);
  }
}

__global__ void k_scale_grad(float* grad, const double* sums, double* loss_out) {
  const double w = sums[0];
  const float inv = w > 0.0 ? (float)(1.0 / w) : 0.f;
  for (int j = threadIdx.x; j < MLP_NPARAM; j += blockDim.x) grad[j] *= inv;
  if (threadIdx.x == 0) loss_out[0] = w > 0.0 ? sums[1] / w : 0.0;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float gj = g[j];
  const float mj = b1 * m[j] + (1.f - b1) * gj;
  const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  p[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

}  // namespace lbm

using namespace lbm;

// ---- host side --------------------------------------------------------------------------------

struct lbm_s;
// accessors into the handle (defined with the rest of the ABI)
KParams lbm_internal_kparams(lbm_handle h);
int lbm_internal_info(lbm_handle h, int* q, int* precision, int* parity, int* closure, int* nx, int* ny,
                      int* nz, void** stream);
lbm_status lbm_internal_fail(lbm_handle h, lbm_status s, const char* msg);

template <int Q, class S>
static void launch_samples(const KParams& p, int parity, const SampleArgs& a, long long nc, cudaStream_t st) {
  const unsigned blocks = (unsigned)((nc + 127) / 128);
  if (parity == 0) k_closure_samples<Q, S, 0><<<blocks, 128, 0, st>>>(p, a);
  else if (parity == 1) k_closure_samples<Q, S, 1><<<blocks, 128, 0, st>>>(p, a);
  else k_closure_samples<Q, S, 2><<<blocks, 128, 0, st>>>(p, a);
}

template <int Q, class S>
static void launch_filter(const KParams& p, int parity, int ncx, int ncy, int ncz, float* rb, float* ub,
                          cudaStream_t st) {
  const long long nc = (long long)ncx * ncy * ncz;
  const unsigned blocks = (unsigned)((nc + 127) / 128);
  if (parity == 0) k_filter2<Q, S, 0><<<blocks, 128, 0, st>>>(p, ncx, ncy, ncz, rb, ub);
  else if (parity == 1) k_filter2<Q, S, 1><<<blocks, 128, 0, st>>>(p, ncx, ncy, ncz, rb, ub);
  else k_filter2<Q, S, 2><<<blocks, 128, 0, st>>>(p, ncx, ncy, ncz, rb, ub);
}

extern "C" {

lbm_status lbm_filter2(lbm_handle fine, float* rho_bar, float* u_bar) {
  if (!fine) return LBM_EINVAL;
  if (!rho_bar || !u_bar) return lbm_internal_fail(fine, LBM_EINVAL, "lbm_filter2: NULL output");
  int q, prec, parity, closure, nx, ny, nz;
  void* stream;
  lbm_internal_info(fine, &q, &prec, &parity, &closure, &nx, &ny, &nz, &stream);
  KParams p = lbm_internal_kparams(fine);
  if (p.outflow) return lbm_internal_fail(fine, LBM_EUNSUPPORTED, "lbm_filter2: lattices with an outflow face");
  if (nx % 2 || ny % 2 || nz % 2) return lbm_internal_fail(fine, LBM_EINVAL, "lbm_filter2: sizes must be even");
  const cudaStream_t st = (cudaStream_t)stream;
  if (q == 19) {
    if (prec == LBM_F32) launch_filter<19, float>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
    else if (prec == LBM_F16_SHIFTED) launch_filter<19, __half>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
    else launch_filter<19, __nv_bfloat16>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
  } else {
    if (prec == LBM_F32) launch_filter<27, float>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
    else if (prec == LBM_F16_SHIFTED) launch_filter<27, __half>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
    else launch_filter<27, __nv_bfloat16>(p, parity, nx / 2, ny / 2, nz / 2, rho_bar, u_bar, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lbm_internal_fail(fine, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_closure_samples(lbm_handle fine, double tau0_c, double cs0, const double scale[2], float* x,
                               float* target, float* smag, float* weight) {
  if (!fine) return LBM_EINVAL;
  if (!x || !target || !smag || !weight || !scale)
    return lbm_internal_fail(fine, LBM_EINVAL, "lbm_closure_samples: NULL output");
  int q, prec, parity, closure, nx, ny, nz;
  void* stream;
  lbm_internal_info(fine, &q, &prec, &parity, &closure, &nx, &ny, &nz, &stream);
  KParams p = lbm_internal_kparams(fine);
  if (p.outflow)
    return lbm_internal_fail(fine, LBM_EUNSUPPORTED, "lbm_closure_samples: lattices with an outflow face");
  if (nx % 2 || ny % 2 || nz % 2)
    return lbm_internal_fail(fine, LBM_EINVAL, "lbm_closure_samples: fine sizes must be even");
  SampleArgs a;
  a.x = x;
  a.target = target;
  a.smag = smag;
  a.weight = weight;
  a.ncx = nx / 2;
  a.ncy = ny / 2;
  a.ncz = nz / 2;
  a.tau0_c = (float)tau0_c;
  a.cs0sq = (float)(cs0 * cs0);
  a.scale_pi = (float)scale[0];
  a.scale_rho = (float)scale[1];
  a.smag_fine = closure == LBM_CLOSURE_SMAG;
  const long long nc = (long long)a.ncx * a.ncy * a.ncz;
  const cudaStream_t st = (cudaStream_t)stream;
  if (q == 19) {
    if (prec == LBM_F32) launch_samples<19, float>(p, parity, a, nc, st);
    else if (prec == LBM_F16_SHIFTED) launch_samples<19, __half>(p, parity, a, nc, st);
    else launch_samples<19, __nv_bfloat16>(p, parity, a, nc, st);
  } else {
    if (prec == LBM_F32) launch_samples<27, float>(p, parity, a, nc, st);
    else if (prec == LBM_F16_SHIFTED) launch_samples<27, __half>(p, parity, a, nc, st);
    else launch_samples<27, __nv_bfloat16>(p, parity, a, nc, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lbm_internal_fail(fine, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream) {
  if (!params || !x || !y || n < 0) {
    lbm_internal_set_error("lbm_mlp_forward: bad argument");
    return LBM_EINVAL;
  }
  if (n == 0) return LBM_OK;
  k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(params, x, n, y);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm_internal_set_error(cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

static size_t backward_smem() {
  return (size_t)(MLP_NPARAM + 3 + 4 * MLP_NH * TB + MLP_NIN * TB + TB) * sizeof(float);
}

static cudaError_t prepare_backward() {
  static bool done = false;
  cudaError_t e = cudaSuccess;
  if (!done) {
    e = cudaFuncSetAttribute(k_mlp_backward<BW_DY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)backward_smem());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_mlp_backward<BW_LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)backward_smem());
    if (e == cudaSuccess) done = true;
  }
  return e;
}

lbm_status lbm_mlp_backward(const float* params, const float* x, const float* dy, int64_t n, float* grad,
                            void* stream) {
  if (!params || !x || !dy || !grad || n < 0) {
    lbm_internal_set_error("lbm_mlp_backward: bad argument");
    return LBM_EINVAL;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prepare_backward();
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), st);
  if (e == cudaSuccess && n > 0) {
    BackArgs a{};
    a.params = params;
    a.x = x;
    a.dy = dy;
    a.n = n;
    a.offset = 0;
    a.stride = 1;
    a.grad = grad;
    k_mlp_backward<BW_DY><<<(unsigned)((n + TB - 1) / TB), TB, backward_smem(), st>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    lbm_internal_set_error(cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

lbm_status lbm_closure_loss_grad(const float* params, const float* x, const float* target, const float* smag,
                                 const float* weight, int64_t n, int64_t offset, int64_t stride, double cs0,
                                 float* grad, double* loss, void* stream) {
  if (!params || !x || !target || !smag || !weight || !grad || !loss || n < 0 || offset < 0 || stride < 1) {
    lbm_internal_set_error("lbm_closure_loss_grad: bad argument");
    return LBM_EINVAL;
  }
  const cudaStream_t st = (cudaStream_t)stream;
  double* sums = nullptr;
  cudaError_t e = prepare_backward();
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&sums, 3 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), st);
  if (e == cudaSuccess && n > 0) {
    BackArgs a{};
    a.params = params;
    a.x = x;
    a.target = target;
    a.smag = smag;
    a.weight = weight;
    a.n = n;
    a.offset = offset;
    a.stride = stride;
    a.k = (float)(cs0 * cs0 / std::log(2.0));
    a.grad = grad;
    a.sums = sums;
    k_mlp_backward<BW_LOSS><<<(unsigned)((n + TB - 1) / TB), TB, backward_smem(), st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_scale_grad<<<1, 256, 0, st>>>(grad, sums, sums + 2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, sums + 2, sizeof(double), cudaMemcpyDefault, st);
  if (sums) cudaFreeAsync(sums, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    lbm_internal_set_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
  }
  return LBM_OK;
}

lbm_status lbm_adam_step(float* params, const float* grad, float* m, float* v, int n, double lr, double beta1,
                         double beta2, double eps, int64_t t, void* stream) {
  if (!params || !grad || !m || !v || n < 0 || t < 1) {
    lbm_internal_set_error("lbm_adam_step: bad argument");
    return LBM_EINVAL;
  }
  if (n == 0) return LBM_OK;
  const float c1 = (float)(1.0 - std::pow(beta1, (double)t));
  const float c2 = (float)(1.0 - std::pow(beta2, (double)t));
  k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, (float)lr, (float)beta1,
                                                           (float)beta2, (float)eps, c1, c2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm_internal_set_error(cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

}  // extern "C"
