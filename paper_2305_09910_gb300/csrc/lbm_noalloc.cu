// lbm_noalloc.cu -- lbm_reduce_noalloc: the FP64 mass/momentum sums of lbm_reduce, computed
// from caller-provided populations without allocating any memory.
//
// Who needs it: a caller that is not allowed to allocate device memory at the point where it
// wants the sums -- for example an analysis hook running inside another application's time
// loop on a GPU whose free memory is owned by that application's caching allocator, or a
// process held to a fixed device-memory budget.  lbm_reduce needs a handle, and creating a
// handle allocates; this entry point needs only the caller's arrays.
//
// Scratch: a file-scope __device__ array (LBM_NOALLOC_MAX_PARTIALS blocks x 4 doubles of
// per-block partial sums, plus 4 doubles for the total), which every GPU that loads the
// library holds until the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it; that first call should come before any stream
// capture.  Every call shares the array: calls whose work overlaps on the GPU race with each
// other.  Each call overwrites every partial it reads, so nothing carries over between calls.
// Every call synchronises its stream before it returns (the sums are in out by then).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

// Records the message returned by lbm_last_error(NULL) (defined with the rest of the ABI).
void lbm_internal_set_error(const char* msg);

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 64;
constexpr long long kCellsPerBlock = (long long)kThreads * kCellsPerThread;  // 16384

static __device__ __align__(256) double g_noalloc_scratch[(LBM_NOALLOC_MAX_PARTIALS + 1) * 4];

#ifdef LBM_BOUNDS_CHECK
// bounds-checked build: 1 + the array (0 populations, 1 flags) of the first access that fell
// outside [pointer, pointer + the size the call declares); the access is skipped
static __device__ int g_noalloc_bad;
#endif

// Whether the access of `bytes` bytes at a lies inside [lo, hi) (always, unless bounds-checked).
__device__ __forceinline__ bool noalloc_chk(const void* a, int bytes, const void* lo, const void* hi, int which) {
#ifdef LBM_BOUNDS_CHECK
  const char* c = static_cast<const char*>(a);
  const bool ok = c >= static_cast<const char*>(lo) && c + bytes <= static_cast<const char*>(hi);
  if (!ok) atomicCAS(&g_noalloc_bad, 0, 1 + which);
  return ok;
#else
  (void)a; (void)bytes; (void)lo; (void)hi; (void)which;
  return true;
#endif
}

// Per-block FP64 sums over a contiguous chunk of cells (fixed order within a thread, fixed
// tree across threads: the result does not depend on scheduling).
template <int Q>
__global__ void __launch_bounds__(kThreads) k_sum_partials(const float* __restrict__ df,
                                                           const uint8_t* __restrict__ flags,
                                                           long long n, float hfx, float hfy, float hfz,
                                                           double* partials) {
  using namespace lbm;
  const long long first = (long long)blockIdx.x * kCellsPerBlock;
  const float* const df_end = df + (long long)Q * n;
  const uint8_t* const fl_end = flags ? flags + n : nullptr;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < kCellsPerThread; k++) {
    const long long c = first + (long long)k * kThreads + threadIdx.x;
    if (c >= n) break;
    if (flags && (!noalloc_chk(flags + c, 1, flags, fl_end, 1) || flags[c] != CELL_FLUID)) continue;
    float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const float* a = df + (long long)i * n + c;
      const float v = noalloc_chk(a, 4, df, df_end, 0) ? *a : 0.f;
      d += v;
      if (cx(i)) jx += cx(i) > 0 ? v : -v;
      if (cy(i)) jy += cy(i) > 0 ? v : -v;
      if (cz(i)) jz += cz(i) > 0 ? v : -v;
    }
    acc[0] += 1.0 + (double)d;           // rho
    acc[1] += (double)(jx + hfx);        // rho u = sum c f + F/2
    acc[2] += (double)(jy + hfy);
    acc[3] += (double)(jz + hfz);
  }
  __shared__ double red[4][kThreads / 32];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; w++) s += red[threadIdx.x][w];
    partials[(long long)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// Sums the block partials in block order into total[0..3].
__global__ void k_sum_total(const double* partials, int nblocks, double* total) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += partials[(long long)b * 4 + threadIdx.x];
    total[threadIdx.x] = s;
  }
}

std::mutex g_mutex;
double* g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_reduce_noalloc(const float* df, const uint8_t* flags, int nx, int ny, int nz,
                                         int stencil, const double force[3], double out[4], void* stream) {
  if (!df || !out) {
    lbm_internal_set_error("lbm_reduce_noalloc: df and out must not be NULL");
    return LBM_EINVAL;
  }
  if (nx < 1 || ny < 1 || nz < 1 || (stencil != 19 && stencil != 27)) {
    lbm_internal_set_error("lbm_reduce_noalloc: sizes must be >= 1 and the stencil 19 or 27");
    return LBM_EINVAL;
  }
  const long long n = (long long)nx * ny * nz;
  const long long nblocks = (n + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nblocks > LBM_NOALLOC_MAX_PARTIALS) {
    char msg[160];
    snprintf(msg, sizeof msg, "lbm_reduce_noalloc: %lld cells exceed the maximum of %lld", n,
             (long long)LBM_NOALLOC_MAX_PARTIALS * kCellsPerBlock);
    lbm_internal_set_error(msg);
    return LBM_EINVAL;
  }
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    lbm_internal_set_error("lbm_reduce_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return LBM_ECUDA;
  }
  double* partials = scratch;
  double* total = scratch + (long long)LBM_NOALLOC_MAX_PARTIALS * 4;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
#ifdef LBM_BOUNDS_CHECK
  {
    const int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_noalloc_bad, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      lbm_internal_set_error("lbm_reduce_noalloc: clearing the bounds-check word failed");
      return LBM_ECUDA;
    }
  }
#endif
  const float hf[3] = {force ? (float)(0.5 * force[0]) : 0.f, force ? (float)(0.5 * force[1]) : 0.f,
                       force ? (float)(0.5 * force[2]) : 0.f};
  if (stencil == 19)
    k_sum_partials<19><<<(unsigned)nblocks, kThreads, 0, st>>>(df, flags, n, hf[0], hf[1], hf[2], partials);
  else
    k_sum_partials<27><<<(unsigned)nblocks, kThreads, 0, st>>>(df, flags, n, hf[0], hf[1], hf[2], partials);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_sum_total<<<1, 32, 0, st>>>(partials, (int)nblocks, total);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, total, 4 * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof msg, "lbm_reduce_noalloc: %s", cudaGetErrorString(e));
    lbm_internal_set_error(msg);
    return LBM_ECUDA;
  }
#ifdef LBM_BOUNDS_CHECK
  int bad = 0;
  if (cudaMemcpyFromSymbol(&bad, g_noalloc_bad, sizeof bad) != cudaSuccess || bad) {
    lbm_internal_set_error(bad == 2 ? "lbm_reduce_noalloc: bounds check: an access outside the flags was skipped"
                                    : "lbm_reduce_noalloc: bounds check: an access outside the populations was skipped");
    return LBM_ECUDA;
  }
#endif
  return LBM_OK;
}
