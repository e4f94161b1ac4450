// lbm_api.cu -- the C ABI declared in include/lbm.h: handle lifetime, validation, state
// bookkeeping (AA parity, two-grid buffers), and dispatch to the (stencil, precision)
// kernel instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_launch.cuh"

using namespace lbm;

struct lbm_s {
  int nx = 0, ny = 0, nz = 0, nxp = 0, q = 0;
  int zg = 0;  // ghost z planes on each side (1 with a LBM_FACE_HALO z face)
  double tau = 0.0;
  lbm_params prm{};
  cudaStream_t stream = nullptr;
  void* f = nullptr;          // populations, q * plane elements of the storage type
  void* f2 = nullptr;         // second population array (two-grid pull only)
  int cur = 0;                // pull: which array holds the state (0: f, 1: f2)
  uint8_t* flags = nullptr;   // raw flags, padded layout
  uint8_t* cls = nullptr;     // cell classes, padded layout
  unsigned long long* rules = nullptr;  // per-direction rules of boundary cells, padded layout
  int* status = nullptr;      // device status word
  int* chk_bad = nullptr;     // first out-of-range access seen by a bounds-checked build
  int* status_host = nullptr; // pinned copy
  double* sums = nullptr;     // 4 doubles (lbm_reduce)
  double* partial = nullptr;  // nz * ny * 10 doubles: per-row sums of the reductions
  float* stats_w = nullptr;   // per-warp plane statistics of sampling steps (see ensure_stats_w)
  int* blist = nullptr;       // cells the x-pair step leaves to the list code (see uses_blist)
  void* blaux = nullptr;      // their source table: q x nblist cells (int32), then q x nblist codes
  long long nblist = 0;
  // CUDA graph of GRAPH_STEPS plain steps that lbm_step replays (captured on a private
  // stream, keyed by the kernel parameters of its first step and the streaming state)
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  KParams gkey{};
  int gkey_state[3] = {-1, -1, -1};  // parity, cur, nat_valid
  bool graphs_off = false;
  bool multi_off = false;     // cooperative multi-step launches unavailable (refused once)
  double* stats = nullptr;    // ny * LBM_STATS_K doubles
  float* mlp = nullptr;       // MLP parameters widened to float
  float mlp_scale[2] = {0.f, 0.f};
  double cs_min = 0.0;        // lower bound on the learned Smagorinsky constant
  bool mlp_set = false;
  int64_t nsamples = 0;
  double force[3] = {0.0, 0.0, 0.0};
  // layout of the state: 0 natural pre-collision (AA after an even number of steps, or any
  // import), 1 AA swapped post-collision (odd number of steps), 2 pull post-collision
  int parity = 0;
  int nat_valid = 1;          // natural layout came from an import (outflow slots hold values)
  int prev_post = 0;          // pull: the other array holds the post-collision state before the current one
  int nsm = 0;                // multiprocessors of the device (persistent grid size)
  int wait_polls = MBAR_POLLS; // polls of the closure step's first wait for each tile's MMA
  bool broken = false;        // a device wait gave up twice: results and device state undefined
  std::string err;
};

static std::string g_create_error;

void lbm_internal_set_error(const char* msg) { g_create_error = msg; }

static lbm_status fail(lbm_handle h, lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return s;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((h), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                          \
  } while (0)

static size_t store_bytes(int precision) { return precision == LBM_F32 ? 4 : 2; }

static long long plane_of(const lbm_s* h) { return (long long)h->nxp * h->ny * h->nz; }
// allocated elements per direction (ghost planes included) and the offset of z = 0
static long long plane_alloc(const lbm_s* h) { return (long long)h->nxp * h->ny * (h->nz + 2 * h->zg); }
static long long ghost_off(const lbm_s* h) { return (long long)h->nxp * h->ny * h->zg; }

static long long ncell(const lbm_s* h) { return (long long)h->nx * h->ny * h->nz; }

static Launch launch_cfg(const lbm_s* h) {
  Launch L;
  L.block = dim3(32, 4, 1);
  L.grid = dim3(h->nxp / 32, (h->ny + 3) / 4, h->nz);
  L.stream = h->stream;
  return L;
}

static KParams kparams(const lbm_s* h) {
  KParams p;
  std::memset(&p, 0, sizeof p);
  {
    void* a = h->cur ? h->f2 : h->f;  // the state
    void* b = h->cur ? h->f : h->f2;  // pull destination (null for AA)
    p.f = a;
    const size_t sb = store_bytes(h->prm.precision);
    for (int i = 0; i < 27; i++) {
      const size_t off = ((size_t)i * (size_t)plane_alloc(h) + (size_t)ghost_off(h)) * sb;
      p.fp[i] = i < h->q ? (void*)((char*)a + off) : nullptr;
      p.fq[i] = (i < h->q && b) ? (void*)((char*)b + off) : nullptr;
    }
    int c[81];
    lbm_stencil(27, c, nullptr);
    for (int i = 0; i < h->q; i++) {
      const long long off = c[3 * i] + (long long)c[3 * i + 1] * h->nxp + (long long)c[3 * i + 2] * h->nxp * h->ny;
      const int o = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
      p.ga[i] = (void*)((uintptr_t)p.fp[o] - (uintptr_t)(off * (long long)sb));
      p.gb[i] = (void*)((uintptr_t)p.fp[i] - (uintptr_t)(off * (long long)sb));
    }
  }
  p.nat_valid = h->nat_valid;
  p.flags = h->flags + ghost_off(h);
  p.cls = h->cls;
  p.rules = h->rules;
  p.stats_w = h->stats_w;
  p.blist = h->blist;
  p.bltab = static_cast<const int*>(h->blaux);
  p.blcode = h->blaux ? static_cast<const uint8_t*>(h->blaux) + 4 * (size_t)h->q * h->nblist : nullptr;
  p.nblist = h->nblist;
  p.pstride = plane_alloc(h);
  p.split = (h->q == 27 || LBM_SPLIT19) && h->prm.precision != LBM_F32 && h->prm.streaming == LBM_PULL &&
            h->prm.collision == LBM_COLL_TRT && h->prm.closure != LBM_CLOSURE_MLP;
  {
    const size_t fbytes = (size_t)plane_alloc(h) * h->q * store_bytes(h->prm.precision);
    p.chk_lo[0] = (const char*)h->f;
    p.chk_hi[0] = (const char*)h->f + fbytes;
    p.chk_lo[1] = (const char*)h->f2;
    p.chk_hi[1] = h->f2 ? (const char*)h->f2 + fbytes : nullptr;
    p.chk_lo[2] = (const char*)h->flags;
    p.chk_hi[2] = (const char*)h->flags + plane_alloc(h);
    p.chk_lo[3] = (const char*)h->cls;
    p.chk_hi[3] = (const char*)h->cls + plane_of(h);
    p.chk_lo[4] = (const char*)h->rules;
    p.chk_hi[4] = (const char*)h->rules + 8 * plane_of(h);
    p.chk_bad = h->chk_bad;
  }
  p.mlp = h->mlp;
  p.status = h->status;
  p.wait_polls = h->wait_polls;
  p.plane = plane_of(h);
  p.nx = h->nx;
  p.ny = h->ny;
  p.nz = h->nz;
  p.nxp = h->nxp;
  p.outflow = h->prm.face_bc[1] == LBM_FACE_OUTFLOW;
  for (int k = 0; k < 6; k++) p.face[k] = h->prm.face_bc[k];
  const double tau = h->tau, lam = h->prm.magic_lambda;
  p.tau0 = (float)tau;
  p.lambda = (float)lam;
  p.cs2 = (float)(h->prm.cs_smag * h->prm.cs_smag);
  p.omega_p = (float)(1.0 / tau);
  p.omega_m = (float)(1.0 / (lam / (tau - 0.5) + 0.5));
  for (int a = 0; a < 3; a++) p.F[a] = (float)h->force[a];
  double w[27];
  int c[81];
  lbm_stencil(h->q, c, w);
  for (int i = 0; i < h->q; i++) {
    const double cu = c[3 * i] * h->prm.u_inflow[0] + c[3 * i + 1] * h->prm.u_inflow[1] +
                      c[3 * i + 2] * h->prm.u_inflow[2];
    p.inflow_term[i] = (float)(6.0 * w[i] * h->prm.rho_inflow * cu);
    const double cF = c[3 * i] * h->force[0] + c[3 * i + 1] * h->force[1] + c[3 * i + 2] * h->force[2];
    p.F3w[i] = (float)(3.0 * w[i] * cF);
    p.F9w[i] = (float)(9.0 * w[i] * cF);
  }
  p.mlp_scale[0] = h->mlp_scale[0];
  p.mlp_scale[1] = h->mlp_scale[1];
  p.cs2_min = (float)(h->cs_min * h->cs_min);
  for (int k = 0; k < 5; k++) p.mrt_s[k] = (float)h->prm.mrt_rates[k];
  return p;
}

// True when the step kernel of this handle samples the statistics itself (every form but the
// learned closure, which samples them in a separate pass before the step).
static bool fused_stats(const lbm_s* h) { return h->prm.closure != LBM_CLOSURE_MLP; }

template <int Q>
static cudaError_t dispatch_step(const lbm_s* h, const KParams& p, int closure, int parity, bool stats = false,
                                 int* nws = nullptr) {
  // mode of the step kernels: 0 AA even, 1 AA odd, 2 first pull step after an import, 3 pull
  const int mode = h->prm.streaming == LBM_PULL ? (parity == 0 ? 2 : 3) : parity;
  if (closure == CL_MLP) {  // the tensor-core closure step
    switch (h->prm.precision) {
      case LBM_F32: return launch_step_mlp<Q, float>(p, mode, h->stream, h->nsm);
      case LBM_F16_SHIFTED: return launch_step_mlp<Q, __half>(p, mode, h->stream, h->nsm);
      default: return launch_step_mlp<Q, __nv_bfloat16>(p, mode, h->stream, h->nsm);
    }
  }
  const Launch L = launch_cfg(h);
  const int coll = h->prm.collision;
  switch (h->prm.precision) {
    case LBM_F32: return launch_step<Q, float>(p, closure, mode, L, stats, nws, coll);
    case LBM_F16_SHIFTED: return launch_step<Q, __half>(p, closure, mode, L, stats, nws, coll);
    default: return launch_step<Q, __nv_bfloat16>(p, closure, mode, L, stats, nws, coll);
  }
}

template <int Q>
static cudaError_t dispatch_export(const lbm_s* h, const KParams& p, int mode, const ExportArgs& a, int parity) {
  const Launch L = launch_cfg(h);
  switch (h->prm.precision) {
    case LBM_F32: return launch_export<Q, float>(p, parity, mode, a, L);
    case LBM_F16_SHIFTED: return launch_export<Q, __half>(p, parity, mode, a, L);
    default: return launch_export<Q, __nv_bfloat16>(p, parity, mode, a, L);
  }
}

template <int Q>
static cudaError_t dispatch_init(const lbm_s* h, const KParams& p, const float* rho, const float* u) {
  const Launch L = launch_cfg(h);
  switch (h->prm.precision) {
    case LBM_F32: return launch_init_eq<Q, float>(p, rho, u, L);
    case LBM_F16_SHIFTED: return launch_init_eq<Q, __half>(p, rho, u, L);
    default: return launch_init_eq<Q, __nv_bfloat16>(p, rho, u, L);
  }
}

template <int Q>
static cudaError_t dispatch_set_pop(const lbm_s* h, const KParams& p, const float* df) {
  const Launch L = launch_cfg(h);
  switch (h->prm.precision) {
    case LBM_F32: return launch_set_pop<Q, float>(p, df, L);
    case LBM_F16_SHIFTED: return launch_set_pop<Q, __half>(p, df, L);
    default: return launch_set_pop<Q, __nv_bfloat16>(p, df, L);
  }
}

// ---- small kernels of the set-up path -----------------------------------------------------

// Copies dense flags into the padded layout and counts values outside the cell enum.
__global__ void k_flags_in(const uint8_t* in, uint8_t* out, int nx, int ny, int nz, int nxp, int* bad) {
  const long long n = (long long)nx * ny * nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx);
    const long long r = k / nx;
    const uint8_t v = in[k];
    if (v > CELL_INFLOW) atomicAdd(bad, 1);
    out[r * nxp + x] = v > CELL_INFLOW ? (uint8_t)CELL_SOLID : v;
  }
}

// Cell classes: skip (non-fluid or padding), boundary (a source needs a rule), interior.
__global__ void k_classify(const __grid_constant__ KParams p, uint8_t* cls, unsigned long long* rules, int q) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= p.ny) return;
  const int cell = cidx(p, x, y, z);
  if (x >= p.nx || flag_at(p, cell) != CELL_FLUID) {
    cls[cell] = CLS_SKIP;
    return;
  }
  const int xc[3] = {x, y, z};
  const int n[3] = {p.nx, p.ny, p.nz};
  int c = CLS_INTERIOR;
  bool wrap_yz = false;
  for (int i = 1; i < q && c == CLS_INTERIOR; i++) {
    const int d[3] = {cx(i), cy(i), cz(i)};
    int s[3];
    for (int a = 0; a < 3; a++) {
      s[a] = xc[a] - d[a];
      if (s[a] < 0 || s[a] >= n[a]) {
        const int ft = p.face[s[a] < 0 ? 2 * a : 2 * a + 1];
        if (ft == FACE_HALO) continue;  // a ghost cell: plain streaming unless its flag says otherwise
        if (ft != FACE_PERIODIC) c = CLS_BOUNDARY;
        else if (a > 0) wrap_yz = true;
        s[a] = s[a] < 0 ? s[a] + n[a] : s[a] - n[a];
      }
    }
    if (c == CLS_INTERIOR && flag_at(p, cidx(p, s[0], s[1], s[2])) != CELL_FLUID) c = CLS_BOUNDARY;
  }
  if (c == CLS_INTERIOR && wrap_yz) c = CLS_WRAP;
  int xf = 0;
  if (c == CLS_BOUNDARY) {
    unsigned long long r = 0;
    for (int i = 1; i < q; i++) r |= (unsigned long long)rule_of(p, x, y, z, i) << (2 * i);
    rules[cell] = r;
    // an inflow or outflow face cell whose directions crossing the face are its only rules
    const bool in_face = x == 0 && p.face[0] == FACE_INFLOW;
    const bool out_face = x == p.nx - 1 && p.face[1] == FACE_OUTFLOW;
    if (p.nx >= 4 && (in_face || out_face)) {
      const int dc = in_face ? 1 : -1, want = in_face ? R_INFLOW : R_SPECIAL;
      bool simple = true;
      for (int i = 1; i < q; i++) {
        const int k = (int)((r >> (2 * i)) & 3);
        const int sy = y - cy(i), sz = z - cz(i);
        simple = simple && sy >= 0 && sy < p.ny && sz >= 0 && sz < p.nz && k == (cx(i) == dc ? want : R_STREAM);
      }
      if (simple) xf = CLS_XFACE;
    }
  }
  cls[cell] = (uint8_t)(c | xf);
}

// Cells of one (y, z) row that need boundary rules or a periodic y/z wrap, except the simple
// inflow/outflow face cells (CLS_XFACE, updated by the x-pair kernel): counted, then listed in
// x order at the row's offset (one thread per row; a set-up pass).
__device__ __forceinline__ bool listed_class(int c) { return c == CLS_BOUNDARY || c == CLS_WRAP; }  // x-face cells excluded

__global__ void k_list_count(const uint8_t* cls, int nx, long long rows, int nxp, int* counts) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int n = 0;
  for (int x = 0; x < nx; x++) n += listed_class(cls[r * nxp + x]);
  counts[r] = n;
}

__global__ void k_list_fill(const uint8_t* cls, int nx, long long rows, int nxp, const long long* offsets, int* list) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  long long o = offsets[r];
  for (int x = 0; x < nx; x++)
    if (listed_class(cls[r * nxp + x])) list[o++] = (int)(r * nxp + x);
}

// The source table of the listed cells (list_source for every direction; a set-up pass after
// the fill, one thread per listed cell).
__global__ void k_list_table(const __grid_constant__ KParams p, const int* list, long long n, int q, int* tab,
                             uint8_t* code) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int cell = list[t];
  const int x = cell % p.nxp, r = cell / p.nxp, y = r % p.ny, z = r / p.ny;
  const int cls = cls_at(p, cell);
  const unsigned long long rule = cls == CLS_BOUNDARY ? rule_at(p, cell) : 0ull;
  for (int i = 0; i < q; i++) {
    int src, c;
    list_source(p, x, y, z, cell, cls, rule, i, src, c);
    tab[i * n + t] = src;
    code[i * n + t] = (uint8_t)c;
  }
}

// ---- accessors used by the other translation units (closure training) -------------------------
KParams lbm_internal_kparams(lbm_handle h) { return kparams(h); }

int lbm_internal_info(lbm_handle h, int* q, int* precision, int* parity, int* closure, int* nx, int* ny,
                      int* nz, void** stream) {
  *q = h->q;
  *precision = h->prm.precision;
  *parity = h->parity;
  *closure = h->prm.closure;
  *nx = h->nx;
  *ny = h->ny;
  *nz = h->nz;
  *stream = (void*)h->stream;
  return 0;
}

lbm_status lbm_internal_fail(lbm_handle h, lbm_status s, const char* msg) { return fail(h, s, "%s", msg); }

// ---- C ABI ----------------------------------------------------------------------------------

// cooperative multi-step launch of k_step_multi for lbm_step (see run_multi)
template <int Q>
static cudaError_t dispatch_multi(const lbm_s* h, const KParams& p0, const KParams& p1, int nsteps) {
  const bool aa = h->prm.streaming != LBM_PULL;
  const int odd0 = aa ? h->parity : 0;
  const int cl = h->prm.closure, coll = h->prm.collision;
  switch (h->prm.precision) {
    case LBM_F32: return launch_step_multi<Q, float>(p0, p1, cl, coll, aa, odd0, nsteps, h->stream, h->nsm);
    case LBM_F16_SHIFTED: return launch_step_multi<Q, __half>(p0, p1, cl, coll, aa, odd0, nsteps, h->stream, h->nsm);
    default: return launch_step_multi<Q, __nv_bfloat16>(p0, p1, cl, coll, aa, odd0, nsteps, h->stream, h->nsm);
  }
}

// ---- refinement transfer kernels (2:1 across a z face; see lbm_refine_explode below) ----
struct RefPlanes {
  void* dst[9];        // destination plane of each transferred direction
  const void* src[9];  // source plane (explode: coarse state; coalesce: fine F*(t+1/2))
  const void* old[9];  // coalesce: fine F*(t)
  int cx[9], cy[9];
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <class E>
__global__ void __launch_bounds__(256) k_refine_explode(RefPlanes rp, int nd, int nxf, int nyf, int nxpf,
                                                        int nxpc, int s) {
  const long long plane = (long long)nyf * nxf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nd * plane;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t / plane);
    const int r = (int)(t - k * plane);
    const int y = r / nxf, x = r - y * nxf;
    const int xs = wrap1(x - s * rp.cx[k], nxf), ys = wrap1(y - s * rp.cy[k], nyf);
    static_cast<E*>(rp.dst[k])[(long long)y * nxpf + x] =
        static_cast<const E*>(rp.src[k])[(long long)(ys >> 1) * nxpc + (xs >> 1)];
  }
}

template <class S>
__global__ void __launch_bounds__(256) k_refine_coalesce(RefPlanes rp, int nd, int nxc, int nyc, int nxpc,
                                                         int nxpf) {
  const long long plane = (long long)nyc * nxc;
  const int nxf = 2 * nxc, nyf = 2 * nyc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nd * plane;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t / plane);
    const int r = (int)(t - k * plane);
    const int Y = r / nxc, X = r - Y * nxc;
    const int cx = rp.cx[k], cy = rp.cy[k];
    const int xv = 2 * wrap1(X + cx, nxc), yv = 2 * wrap1(Y + cy, nyc);  // the receiving cell's volume
    const S* a = static_cast<const S*>(rp.src[k]);
    const S* b = static_cast<const S*>(rp.old[k]);
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int xf = xv + (j & 1), yf = yv + (j >> 1);
      sum += ld<S>(a + (long long)wrap1(yf - cy, nyf) * nxpf + wrap1(xf - cx, nxf));
      sum += ld<S>(b + (long long)wrap1(yf - 2 * cy, nyf) * nxpf + wrap1(xf - 2 * cx, nxf));
    }
    st<S>(static_cast<S*>(rp.dst[k]) + (long long)Y * nxpc + X, sum * 0.125f);
  }
}

extern "C" {

void lbm_params_default(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->struct_size = sizeof(lbm_params);
  p->precision = LBM_F32;
  p->streaming = LBM_AA;
  p->closure = LBM_CLOSURE_NONE;
  p->magic_lambda = 3.0 / 16.0;
  p->cs_smag = 0.1;
  for (int k = 0; k < 6; k++) p->face_bc[k] = LBM_FACE_PERIODIC;
  p->rho_inflow = 1.0;
  p->stream = nullptr;
  p->pipeline = LBM_PIPE_DIRECT;
  p->collision = LBM_COLL_TRT;
  const double rates[5] = {1.19, 1.4, 1.2, 1.4, 1.98};
  for (int k = 0; k < 5; k++) p->mrt_rates[k] = rates[k];
}

int lbm_stencil(int q, int* c, double* w) {
  if (q != 19 && q != 27) return 0;
  for (int i = 0; i < q; i++) {
    if (c) {
      c[3 * i] = cx(i);
      c[3 * i + 1] = cy(i);
      c[3 * i + 2] = cz(i);
    }
    if (w) {
      const int n = csq(i);
      if (q == 19) w[i] = n == 0 ? 1.0 / 3.0 : n == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
      else w[i] = n == 0 ? 8.0 / 27.0 : n == 1 ? 2.0 / 27.0 : n == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    }
  }
  return q;
}

const char* lbm_last_error(lbm_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

// Handles whose pull step splits into the x-pair kernel over interior cells and the list code
// over the listed ones: half storage, two-grid pull, TRT without the learned closure, both
// stencils (the warps that hold a boundary lane would otherwise diverge through its boundary
// loads; D3Q27 bluff body 32.2k MLUPS one-cell, 30.0k unsplit pairs, 43.7k split; D3Q19 FP16
// channel 65.1k unsplit, 67.4k split).
static bool uses_blist(const lbm_s* h) { return kparams(h).split != 0; }

// The list of cells needing rules or a y/z wrap, in row order, and its source table (rebuilt
// with the classes).
static lbm_status build_blist(lbm_handle h) {
  if (h->blist) CUDA_TRY(h, cudaFreeAsync(h->blist, h->stream));
  if (h->blaux) CUDA_TRY(h, cudaFreeAsync(h->blaux, h->stream));
  h->blist = nullptr;
  h->blaux = nullptr;
  h->nblist = 0;
  const long long rows = (long long)h->ny * h->nz;
  long long* offsets = nullptr;
  CUDA_TRY(h, cudaMallocAsync((void**)&offsets, (size_t)rows * sizeof(long long), h->stream));
  int* counts = reinterpret_cast<int*>(offsets);  // counts first, then the offsets over them
  const unsigned blocks = (unsigned)((rows + 255) / 256);
  k_list_count<<<blocks, 256, 0, h->stream>>>(h->cls, h->nx, rows, h->nxp, counts);
  CUDA_TRY(h, cudaGetLastError());
  std::vector<int> hc((size_t)rows);
  std::vector<long long> ho((size_t)rows);
  CUDA_TRY(h, cudaMemcpyAsync(hc.data(), counts, (size_t)rows * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  long long total = 0;
  for (long long r = 0; r < rows; r++) {
    ho[(size_t)r] = total;
    total += hc[(size_t)r];
  }
  if (total > 0) {
    CUDA_TRY(h, cudaMemcpyAsync(offsets, ho.data(), (size_t)rows * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMallocAsync((void**)&h->blist, (size_t)total * sizeof(int), h->stream));
    CUDA_TRY(h, cudaMallocAsync(&h->blaux, (size_t)total * h->q * 5, h->stream));
    k_list_fill<<<blocks, 256, 0, h->stream>>>(h->cls, h->nx, rows, h->nxp, offsets, h->blist);
    CUDA_TRY(h, cudaGetLastError());
    int* tab = static_cast<int*>(h->blaux);
    KParams p = kparams(h);
    k_list_table<<<(unsigned)((total + 127) / 128), 128, 0, h->stream>>>(
        p, h->blist, total, h->q, tab, reinterpret_cast<uint8_t*>(tab + (size_t)h->q * total));
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // ho must outlive the copy
  }
  CUDA_TRY(h, cudaFreeAsync(offsets, h->stream));
  h->nblist = total;
  return LBM_OK;
}

static lbm_status launch_classify(lbm_handle h) {
  KParams p = kparams(h);
  Launch L = launch_cfg(h);
  k_classify<<<L.grid, L.block, 0, h->stream>>>(p, h->cls, h->rules, h->q);
  CUDA_TRY(h, cudaGetLastError());
  if (uses_blist(h)) return build_blist(h);
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_handle h) {
  if (!h) return LBM_OK;
  if (h->f) cudaFreeAsync(h->f, h->stream);
  if (h->f2) cudaFreeAsync(h->f2, h->stream);
  if (h->flags) cudaFreeAsync(h->flags, h->stream);
  if (h->cls) cudaFreeAsync(h->cls, h->stream);
  if (h->rules) cudaFreeAsync(h->rules, h->stream);
  if (h->status) cudaFreeAsync(h->status, h->stream);
  if (h->chk_bad) cudaFreeAsync(h->chk_bad, h->stream);
  if (h->sums) cudaFreeAsync(h->sums, h->stream);
  if (h->partial) cudaFreeAsync(h->partial, h->stream);
  if (h->stats_w) cudaFreeAsync(h->stats_w, h->stream);
  if (h->stats) cudaFreeAsync(h->stats, h->stream);
  if (h->mlp) cudaFreeAsync(h->mlp, h->stream);
  if (h->blist) cudaFreeAsync(h->blist, h->stream);
  if (h->blaux) cudaFreeAsync(h->blaux, h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->status_host) cudaFreeHost(h->status_host);
  delete h;
  return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, int nz, int stencil, double tau, const lbm_params* prm,
                      lbm_handle* out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  lbm_params p;
  lbm_params_default(&p);
  if (prm) {
    if (prm->struct_size != sizeof(lbm_params))
      return fail(nullptr, LBM_EINVAL, "lbm_params.struct_size %u != %zu", prm->struct_size,
                  sizeof(lbm_params));
    p = *prm;
  }
  if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "lattice size must be >= 1");
  if (stencil != 19 && stencil != 27) return fail(nullptr, LBM_EINVAL, "stencil must be 19 or 27");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, LBM_EINVAL, "tau must be > 1/2");
  if (!(p.magic_lambda > 0.0) || !std::isfinite(p.magic_lambda))
    return fail(nullptr, LBM_EINVAL, "magic_lambda must be > 0");
  if (p.precision < LBM_F32 || p.precision > LBM_BF16_SHIFTED)
    return fail(nullptr, LBM_EINVAL, "unknown precision %d", p.precision);
  if (p.closure < LBM_CLOSURE_NONE || p.closure > LBM_CLOSURE_MLP)
    return fail(nullptr, LBM_EINVAL, "unknown closure %d", p.closure);
  if (p.streaming != LBM_AA && p.streaming != LBM_PULL)
    return fail(nullptr, LBM_EINVAL, "unknown streaming %d", p.streaming);
  if (p.pipeline < LBM_PIPE_TMA || p.pipeline > LBM_PIPE_ASYNC)
    return fail(nullptr, LBM_EINVAL, "unknown pipeline %d", p.pipeline);
  if (p.pipeline != LBM_PIPE_DIRECT)
    return fail(nullptr, LBM_EUNSUPPORTED, "only the direct-load pipeline is built (pipeline %d)", p.pipeline);
  if (!(p.cs_smag >= 0.0)) return fail(nullptr, LBM_EINVAL, "cs_smag must be >= 0");
  if (p.collision != LBM_COLL_TRT && p.collision != LBM_COLL_MRT && p.collision != LBM_COLL_REG)
    return fail(nullptr, LBM_EINVAL, "unknown collision %d", p.collision);
  if (p.collision == LBM_COLL_REG && p.closure == LBM_CLOSURE_MLP)
    return fail(nullptr, LBM_EUNSUPPORTED, "the learned closure runs with the TRT collision");
  if (p.collision == LBM_COLL_MRT) {
    if (stencil != 19) return fail(nullptr, LBM_EUNSUPPORTED, "the MRT collision is defined for D3Q19");
    if (p.closure == LBM_CLOSURE_MLP)
      return fail(nullptr, LBM_EUNSUPPORTED, "the learned closure runs with the TRT collision");
    for (int k = 0; k < 5; k++)
      if (!(p.mrt_rates[k] > 0.0 && p.mrt_rates[k] < 2.0))
        return fail(nullptr, LBM_EINVAL, "MRT rates must lie in (0, 2)");
  }
  for (int k = 0; k < 6; k++)
    if (p.face_bc[k] < LBM_FACE_PERIODIC || p.face_bc[k] > LBM_FACE_HALO)
      return fail(nullptr, LBM_EINVAL, "unknown face type %d", p.face_bc[k]);
  for (int k = 0; k < 6; k++)
    if (p.face_bc[k] == LBM_FACE_HALO && (k < 4 || p.streaming != LBM_PULL))
      return fail(nullptr, LBM_EUNSUPPORTED, "halo faces are supported on the z faces of two-grid pull lattices");
  for (int a = 0; a < 3; a++)
    if ((p.face_bc[2 * a] == LBM_FACE_PERIODIC) != (p.face_bc[2 * a + 1] == LBM_FACE_PERIODIC))
      return fail(nullptr, LBM_EINVAL, "periodic faces must come in pairs (axis %d)", a);
  for (int k = 0; k < 6; k++)
    if (p.face_bc[k] == LBM_FACE_OUTFLOW && k != 1)
      return fail(nullptr, LBM_EUNSUPPORTED, "outflow is supported on the +x face only");
  if (p.face_bc[1] == LBM_FACE_OUTFLOW && (nx < 2 || nx % 32 == 1))
    return fail(nullptr, LBM_EUNSUPPORTED, "an outflow face needs nx >= 2 and nx %% 32 != 1");
  const int nxp = (nx + 31) / 32 * 32;
  if ((long long)nxp * ny * nz >= (1ll << 31))
    return fail(nullptr, LBM_EINVAL, "lattice too large (padded cells must be < 2^31)");
  if (ny > 65535 * 4 || nz > 65535) return fail(nullptr, LBM_EINVAL, "ny or nz too large for the grid");

  lbm_s* h = new (std::nothrow) lbm_s();
  if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->nxp = nxp;
  h->q = stencil;
  h->zg = (p.face_bc[4] == LBM_FACE_HALO || p.face_bc[5] == LBM_FACE_HALO) ? 1 : 0;
  h->tau = tau;
  h->prm = p;
  h->stream = (cudaStream_t)p.stream;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (h->nsm < 1) h->nsm = 1;
  }
  const long long plane = plane_of(h);
  const long long gplane = plane_alloc(h);  // with the ghost planes (populations, flags)
  const size_t fbytes = (size_t)gplane * stencil * store_bytes(p.precision);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMallocAsync(&h->f, fbytes, h->stream);
  if (e == cudaSuccess && p.streaming == LBM_PULL) e = cudaMallocAsync(&h->f2, fbytes, h->stream);
  if (e == cudaSuccess && h->f2) e = cudaMemsetAsync(h->f2, 0, fbytes, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->flags, (size_t)gplane, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->cls, (size_t)plane, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->rules, (size_t)plane * 8, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->status, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->chk_bad, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->chk_bad, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->sums, 4 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->partial, (size_t)ny * nz * 10 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&h->stats, (size_t)ny * LBM_STATS_K * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->status_host, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f, 0, fbytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, (size_t)gplane, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->stats, 0, (size_t)ny * LBM_STATS_K * sizeof(double), h->stream);
  if (e != cudaSuccess) {
    lbm_status s = fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                        "allocation of %zu population bytes failed: %s", fbytes, cudaGetErrorString(e));
    lbm_destroy(h);
    return s;
  }
  // padding columns are never fluid
  if (nxp != nx) {
    e = cudaMemset2DAsync(h->flags + nx, nxp, CELL_SOLID, nxp - nx, (size_t)ny * (nz + 2 * h->zg), h->stream);
    if (e != cudaSuccess) {
      lbm_status s = fail(nullptr, LBM_ECUDA, "flag padding: %s", cudaGetErrorString(e));
      lbm_destroy(h);
      return s;
    }
  }
  lbm_status s = launch_classify(h);
  if (s != LBM_OK) {
    g_create_error = h->err;
    lbm_destroy(h);
    return s;
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_set_flags(lbm_handle h, const uint8_t* flags, int on_device) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!flags) return fail(h, LBM_EINVAL, "flags is NULL");
  const long long n = (long long)h->nx * h->ny * (h->nz + 2 * h->zg);  // ghost planes included
  const uint8_t* src = flags;
  uint8_t* tmp = nullptr;
  if (!on_device) {
    CUDA_TRY(h, cudaMallocAsync((void**)&tmp, (size_t)n, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(tmp, flags, (size_t)n, cudaMemcpyHostToDevice, h->stream));
    src = tmp;
  }
  int* bad = nullptr;
  CUDA_TRY(h, cudaMallocAsync((void**)&bad, sizeof(int), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 32);
  k_flags_in<<<blocks, 256, 0, h->stream>>>(src, h->flags, h->nx, h->ny, h->nz + 2 * h->zg, h->nxp, bad);
  CUDA_TRY(h, cudaGetLastError());
  int nbad = 0;
  CUDA_TRY(h, cudaMemcpyAsync(h->status_host, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaFreeAsync(bad, h->stream));
  if (tmp) CUDA_TRY(h, cudaFreeAsync(tmp, h->stream));
  lbm_status s = launch_classify(h);
  if (s != LBM_OK) return s;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  nbad = *h->status_host;
  if (nbad) return fail(h, LBM_EINVAL, "%d flag values outside {0,1,2} (stored as solid)", nbad);
  return LBM_OK;
}

lbm_status lbm_set_force(lbm_handle h, double fx, double fy, double fz) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz))
    return fail(h, LBM_EINVAL, "force must be finite");
  h->force[0] = fx;
  h->force[1] = fy;
  h->force[2] = fz;
  return LBM_OK;
}

// Stages a host array on the device (or passes a device pointer through).
// The device address of host memory the GPU can reach directly (pinned or registered host
// memory, managed memory), else nullptr (pageable memory, which is staged through a copy).
static void* host_alias(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error state
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) return a.devicePointer;
  return nullptr;
}

static lbm_status stage_in(lbm_handle h, const float* src, size_t count, int on_device, const float** dev,
                           float** tmp) {
  *tmp = nullptr;
  *dev = src;
  if (!src || on_device) return LBM_OK;
  if (const void* alias = host_alias(src)) {  // pinned: the kernel reads it in place
    *dev = static_cast<const float*>(alias);
    return LBM_OK;
  }
  CUDA_TRY(h, cudaMallocAsync((void**)tmp, count * sizeof(float), h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(*tmp, src, count * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  *dev = *tmp;
  return LBM_OK;
}

static lbm_status reset_status(lbm_handle h) {
  CUDA_TRY(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_handle h, const float* rho, const float* u, int on_device) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  const long long n = ncell(h);
  const float *drho = nullptr, *du = nullptr;
  float *trho = nullptr, *tu = nullptr;
  lbm_status s = stage_in(h, rho, (size_t)n, on_device, &drho, &trho);
  if (s == LBM_OK) s = stage_in(h, u, (size_t)n * 3, on_device, &du, &tu);
  if (s != LBM_OK) return s;
  KParams p = kparams(h);
  cudaError_t e = h->q == 19 ? dispatch_init<19>(h, p, drho, du) : dispatch_init<27>(h, p, drho, du);
  if (trho) cudaFreeAsync(trho, h->stream);
  if (tu) cudaFreeAsync(tu, h->stream);
  CUDA_TRY(h, e);
  h->parity = 0;
  h->prev_post = 0;
  h->nat_valid = 1;
  return reset_status(h);
}

lbm_status lbm_set_populations(lbm_handle h, const float* df, int on_device) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!df) return fail(h, LBM_EINVAL, "df is NULL");
  const float* d = nullptr;
  float* t = nullptr;
  lbm_status s = stage_in(h, df, (size_t)ncell(h) * h->q, on_device, &d, &t);
  if (s != LBM_OK) return s;
  KParams p = kparams(h);
  cudaError_t e = h->q == 19 ? dispatch_set_pop<19>(h, p, d) : dispatch_set_pop<27>(h, p, d);
  if (t) cudaFreeAsync(t, h->stream);
  CUDA_TRY(h, e);
  h->parity = 0;
  h->prev_post = 0;
  h->nat_valid = 1;
  return reset_status(h);
}

static lbm_status run_export(lbm_handle h, int mode, const ExportArgs& a, bool raw = false);
static void advance_state(lbm_handle h);

// The per-warp scratch of sampling steps; lbm_stats_reset allocates it ahead of the steps (the
// first allocation from the stream-ordered pool maps memory, which takes a while).
static lbm_status ensure_stats_w(lbm_handle h) {
  if (!fused_stats(h) || h->stats_w) return LBM_OK;
  const size_t slots = (size_t)((h->nxp + 31) / 32) * h->ny * h->nz;
  CUDA_TRY(h, cudaMallocAsync((void**)&h->stats_w, slots * 10 * sizeof(float), h->stream));
  return LBM_OK;
}

// n steps; with every > 0 the plane statistics of the state each step k (k % every == 0)
// starts from are added to the accumulated sums, inside that step's kernel where it can.
static lbm_status run_steps(lbm_handle h, int64_t n, int64_t every) {
  if (h->prm.closure == LBM_CLOSURE_MLP && !h->mlp_set)
    return fail(h, LBM_ESTATE, "MLP closure selected but lbm_set_closure was not called");
  if (every > 0) {
    const lbm_status s = ensure_stats_w(h);
    if (s != LBM_OK) return s;
  }
  KParams p = kparams(h);
  for (int64_t k = 0; k < n; k++) {
    p.nat_valid = h->nat_valid;
    const bool sample = every > 0 && k % every == 0;
    bool fused = false;
    if (sample && !fused_stats(h)) {
      ExportArgs a{};
      a.sums = h->stats;
      a.partial = h->partial;
      lbm_status s = run_export(h, EX_STATS, a);
      if (s != LBM_OK) return s;
    } else if (sample) {
      fused = true;
    }
    int nws = 0;
    cudaError_t e = h->q == 19 ? dispatch_step<19>(h, p, h->prm.closure, h->parity, fused, &nws)
                               : dispatch_step<27>(h, p, h->prm.closure, h->parity, fused, &nws);
    CUDA_TRY(h, e);
    if (fused) {
      k_stats_total<<<(unsigned)h->ny, 256, 0, h->stream>>>(h->stats_w, h->ny, h->nz, nws, h->stats);
      CUDA_TRY(h, cudaGetLastError());
    }
    if (sample) h->nsamples++;
    advance_state(h);  // pull: the destination array holds the new state
    if (h->prm.streaming == LBM_PULL) p = kparams(h);
  }
  return LBM_OK;
}

// ---- CUDA graph of plain steps ---------------------------------------------------------------
// Small lattices are launch-bound: lbm_step replays a graph of GRAPH_STEPS steps (an even
// number, so the streaming state returns to where it started) when the state is steady (pull
// after its first step; AA once the outflow import state is settled) and the closure is not
// the learned one (its persistent tensor-core kernel is not captured).  The graph is captured on a private stream and re-captured whenever the kernel
// parameters of its first step differ (force, closure, flags, parity, arrays); replays give
// the bits of single launches.
constexpr int GRAPH_STEPS = 8;

static void advance_state(lbm_handle h) {
  if (h->prm.streaming == LBM_PULL) {
    h->prev_post = h->parity == 2;  // the array just read keeps the state it held
    h->cur ^= 1;
    h->parity = 2;
  } else {
    if (h->parity == 1) h->nat_valid = 0;  // an odd step leaves the outflow slots unwritten
    h->parity ^= 1;
  }
}

// Lattices above this many padded cells step as single launches: a step takes long enough there
// (0.1 ms at 2^22 cells) that a replay saves nothing, while a capture costs milliseconds.
#ifndef LBM_GRAPH_MAX_CELLS
#define LBM_GRAPH_MAX_CELLS (1ll << 22)
#endif

static bool graph_ready(lbm_handle h) {
  if (h->graphs_off || h->prm.closure == LBM_CLOSURE_MLP) return false;
  if ((long long)h->nxp * h->ny * h->nz > LBM_GRAPH_MAX_CELLS) return false;
  if (h->prm.streaming == LBM_PULL ? h->parity != 2 : (h->prm.face_bc[1] == LBM_FACE_OUTFLOW && h->nat_valid))
    return false;
  KParams p = kparams(h);
  p.nat_valid = h->nat_valid;
  const int state[3] = {h->parity, h->cur, h->nat_valid};
  if (h->gexec && std::memcmp(&p, &h->gkey, sizeof p) == 0 && std::memcmp(state, h->gkey_state, sizeof state) == 0)
    return true;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    h->graphs_off = true;
    return false;
  }
  const int saved[4] = {h->parity, h->cur, h->nat_valid, h->prev_post};
  cudaStream_t user = h->stream;
  h->stream = h->cap;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  for (int k = 0; ok && k < GRAPH_STEPS; k++) {
    KParams q = kparams(h);
    q.nat_valid = h->nat_valid;
    ok = (h->q == 19 ? dispatch_step<19>(h, q, h->prm.closure, h->parity)
                     : dispatch_step<27>(h, q, h->prm.closure, h->parity)) == cudaSuccess;
    advance_state(h);
  }
  const bool ended = cudaStreamEndCapture(h->cap, &graph) == cudaSuccess;
  h->stream = user;
  h->parity = saved[0];
  h->cur = saved[1];
  h->nat_valid = saved[2];
  h->prev_post = saved[3];
  ok = ok && ended && graph && cudaGraphInstantiate(&h->gexec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();  // a failed capture leaves no sticky error; fall back to launches
  if (!ok) {
    h->gexec = nullptr;
    h->graphs_off = true;
    return false;
  }
  h->gkey = p;
  std::memcpy(h->gkey_state, state, sizeof state);
  return true;
}

// ---- several steps per launch on small lattices ---------------------------------------------
// On small lattices the steps are launch-bound even as graph replays: lbm_step runs them as
// cooperative launches of k_step_multi, MULTI_CHUNK steps at most each, once the state is
// steady (as for the graphs).  Measured on GB300 (FP32 D3Q19, us per step, multi / graph):
// pull 32^3 3.8 / 6.7, 64x32x32 4.6 / 7.7, 64^3 11.1 / 11.3, 128x64x64 17.6 / 16.9; AA 32^3
// 5.1 / 5.6, 64x32x32 6.1 / 6.2, 64^3 14.2 / 10.0 (the AA graph keeps the one array in L2).
// Hence the limits in padded cells below.  A device that refuses the cooperative launch falls
// back to the graphs.
#ifndef LBM_MULTI_MAX_CELLS
#define LBM_MULTI_MAX_CELLS (1ll << 17)
#endif
#ifndef LBM_MULTI_MAX_CELLS_AA
#define LBM_MULTI_MAX_CELLS_AA (1ll << 15)
#endif
constexpr int64_t MULTI_CHUNK = 4096;

static bool steady_state(const lbm_s* h) {
  return h->prm.streaming == LBM_PULL ? h->parity == 2
                                      : !(h->prm.face_bc[1] == LBM_FACE_OUTFLOW && h->nat_valid);
}

// Runs what it can of n steps as multi-step launches; returns the steps left.
static int64_t run_multi(lbm_handle h, int64_t n) {
  while (n >= 2) {
    const int chunk = (int)std::min<int64_t>(n, MULTI_CHUNK);
    KParams p0 = kparams(h), p1 = p0;
    p0.nat_valid = p1.nat_valid = h->nat_valid;
    if (h->prm.streaming == LBM_PULL) {  // the second array's view
      h->cur ^= 1;
      p1 = kparams(h);
      h->cur ^= 1;
      p1.nat_valid = h->nat_valid;
    }
    const cudaError_t e = h->q == 19 ? dispatch_multi<19>(h, p0, p1, chunk) : dispatch_multi<27>(h, p0, p1, chunk);
    if (e != cudaSuccess) {  // refused before anything ran: use the graphs from now on
      cudaGetLastError();
      h->multi_off = true;
      return n;
    }
    for (int k = 0; k < chunk; k++) advance_state(h);
    n -= chunk;
  }
  return n;
}

static const char* const BROKEN_MSG =
    "the handle is unusable: a learned-closure step gave up waiting for the tensor core twice";

lbm_status lbm_step(lbm_handle h, int64_t n) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (h->broken) return fail(h, LBM_ECUDA, "%s", BROKEN_MSG);
  if (n < 0) return fail(h, LBM_EINVAL, "n must be >= 0");
  if (h->prm.closure == LBM_CLOSURE_MLP && !h->mlp_set)
    return fail(h, LBM_ESTATE, "MLP closure selected but lbm_set_closure was not called");
  const long long multi_max = h->prm.streaming == LBM_PULL ? LBM_MULTI_MAX_CELLS : LBM_MULTI_MAX_CELLS_AA;
  if (n >= 2 && !h->multi_off && h->prm.closure != LBM_CLOSURE_MLP &&
      (long long)h->nxp * h->ny * h->nz <= multi_max) {
    while (n > 0 && !steady_state(h)) {  // settle with single launches
      lbm_status s = run_steps(h, 1, 0);
      if (s != LBM_OK) return s;
      n--;
    }
    n = run_multi(h, n);
  }
  // settle the state with single launches first (the first pull step, the AA outflow import)
  while (n > 0 && n >= 2 * GRAPH_STEPS && !graph_ready(h) && !h->graphs_off &&
         (h->prm.streaming == LBM_PULL ? h->parity != 2 : h->nat_valid != 0) &&
         h->prm.closure != LBM_CLOSURE_MLP) {
    lbm_status s = run_steps(h, 1, 0);
    if (s != LBM_OK) return s;
    n--;
  }
  while (n >= GRAPH_STEPS && graph_ready(h)) {
    CUDA_TRY(h, cudaGraphLaunch(h->gexec, h->stream));
    for (int k = 0; k < GRAPH_STEPS; k++) advance_state(h);
    n -= GRAPH_STEPS;
  }
  return run_steps(h, n, 0);
}

lbm_status lbm_step_stats(lbm_handle h, int64_t n, int64_t every) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (h->broken) return fail(h, LBM_ECUDA, "%s", BROKEN_MSG);
  if (n < 0) return fail(h, LBM_EINVAL, "n must be >= 0");
  if (every < 1) return fail(h, LBM_EINVAL, "every must be >= 1");
  return run_steps(h, n, every);
}

// ---- halo exchange of z slabs -------------------------------------------------------------
// Directions that cross a z face: those with c_z = sign (+1 for the +z face when leaving).
static int halo_dirs(const lbm_s* h, int sign, int* dirs) {
  int c[81], n = 0;
  lbm_stencil(h->q, c, nullptr);
  for (int i = 0; i < h->q; i++)
    if (c[3 * i + 2] == sign) dirs[n++] = i;
  return n;
}

static lbm_status halo_check(lbm_handle h, int face) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (face != 4 && face != 5) return fail(h, LBM_EINVAL, "face must be 4 (-z) or 5 (+z)");
  if (h->prm.face_bc[face] != LBM_FACE_HALO) return fail(h, LBM_EINVAL, "face %d is not a halo face", face);
  if (h->parity != 2) return fail(h, LBM_ESTATE, "no post-collision state yet: step once after an import");
  return LBM_OK;
}

// One z plane of up to 9 directions between the population array and a packed buffer
// [k][ny][nxp], as 32-bit words (a plane row is a multiple of 32 elements).
struct HaloPlanes {
  uint32_t* plane[9];
};

__global__ void __launch_bounds__(256) k_halo_copy(HaloPlanes hp, int nd, long long words, uint32_t* buf, int pack) {
  const long long n = (long long)nd * words;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t / words);
    const long long w = t - (long long)k * words;
    if (pack) buf[t] = hp.plane[k][w];
    else hp.plane[k][w] = buf[t];
  }
}

static lbm_status halo_copy(lbm_handle h, int face, void* buf, bool pack) {
  lbm_status st = halo_check(h, face);
  if (st != LBM_OK) return st;
  if (!buf) return fail(h, LBM_EINVAL, "buf is NULL");
  if ((uintptr_t)buf % 4) return fail(h, LBM_EINVAL, "buf must be 4-byte aligned");
  // the kernel dereferences buf: device, managed or pinned (registered) host memory only
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, buf) != cudaSuccess || attr.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();  // clear the query's error state
    return fail(h, LBM_EINVAL, "buf must be device memory or pinned host memory");
  }
  if (attr.type == cudaMemoryTypeHost) buf = attr.devicePointer;
  int dirs[27];
  // pack: leaving directions (c_z = -1 through -z, +1 through +z); unpack: entering ones
  const int sign = pack ? (face == 5 ? 1 : -1) : (face == 4 ? 1 : -1);
  const int nd = halo_dirs(h, sign, dirs);
  const KParams p = kparams(h);
  const size_t sb = store_bytes(h->prm.precision);
  const size_t pb = (size_t)h->nxp * h->ny * sb;  // one z plane of one direction
  const long long z = pack ? (face == 5 ? h->nz - 1 : 0) : (face == 4 ? -1 : h->nz);
  HaloPlanes hp{};
  for (int k = 0; k < nd; k++) hp.plane[k] = (uint32_t*)((char*)p.fp[dirs[k]] + z * (long long)pb);
  const long long words = (long long)(pb / 4);
  const int blocks = (int)std::min<long long>((nd * words + 255) / 256, (long long)h->nsm * 8);
  k_halo_copy<<<blocks, 256, 0, h->stream>>>(hp, nd, words, (uint32_t*)buf, pack ? 1 : 0);
  CUDA_TRY(h, cudaGetLastError());
  return LBM_OK;
}

size_t lbm_halo_bytes(lbm_handle h, int face) {
  if (!h || (face != 4 && face != 5)) return 0;
  int dirs[27];
  return (size_t)halo_dirs(h, face == 5 ? 1 : -1, dirs) * h->nxp * h->ny * store_bytes(h->prm.precision);
}

lbm_status lbm_halo_pack(lbm_handle h, int face, void* buf) { return halo_copy(h, face, buf, true); }

lbm_status lbm_halo_unpack(lbm_handle h, int face, const void* buf) {
  return halo_copy(h, face, const_cast<void*>(buf), false);
}

// ---- 2:1 grid refinement across a z face ---------------------------------------------------
// Volumetric transfer of Rohde et al. (2006) in pull form.  A fine cell (x, y) of the slab's
// boundary plane pulls a population entering through the face from the ghost plane at
// (x - c_x, y - c_y); in the scheme's push form the fine ghost region is two fine planes deep,
// filled from the coarse interface cell whose volume each ghost cell lies in and streamed (not
// collided) with the fine cells, so the ghost value seen in fine substep s (0, 1) is the coarse
// population of the cell over (x - s c_x, y - s c_y).  Leaving the slab, the 8 fine values that
// end in a coarse cell's volume after both substeps are F*(t+1/2) of (x - c_x, y - c_y) and
// F*(t) of (x - 2 c_x, y - 2 c_y) for the 2x2 fine cells (x, y) above the coarse cell; their mean
// is what the coarse cell receives, i.e. what its pull reads from the coarse ghost cell one
// coarse step back along c_i.
// The pair (coarse face, fine face) of one interface: the coarse lattice's +z face meets the
// fine lattice's -z face or the other way round; both halo faces of two-grid pull lattices of
// the same stencil and precision, periodic in x and y, the fine one twice as wide and deep.
// Errors are recorded on the destination handle e (fine for explode, coarse for coalesce).
static lbm_status refine_check(lbm_handle coarse, int cface, lbm_handle fine, int fface, lbm_handle e) {
  if (!coarse || !fine) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (coarse == fine) return fail(e, LBM_EINVAL, "coarse and fine must be different lattices");
  if ((cface != 4 && cface != 5) || fface != 9 - cface)
    return fail(e, LBM_EINVAL, "faces must be (coarse 5, fine 4) or (coarse 4, fine 5)");
  if (coarse->prm.face_bc[cface] != LBM_FACE_HALO || fine->prm.face_bc[fface] != LBM_FACE_HALO)
    return fail(e, LBM_EINVAL, "both faces must be halo faces");
  if (coarse->q != fine->q || coarse->prm.precision != fine->prm.precision)
    return fail(e, LBM_EINVAL, "coarse and fine lattices need the same stencil and precision");
  if (fine->nx != 2 * coarse->nx || fine->ny != 2 * coarse->ny)
    return fail(e, LBM_EINVAL, "the fine lattice must be 2 nx x 2 ny of the coarse one");
  for (int f = 0; f < 4; f++)
    if (coarse->prm.face_bc[f] != LBM_FACE_PERIODIC || fine->prm.face_bc[f] != LBM_FACE_PERIODIC)
      return fail(e, LBM_EUNSUPPORTED, "refinement interfaces need periodic x and y faces");
  if (coarse->parity != 2 || fine->parity != 2)
    return fail(e, LBM_ESTATE, "both lattices must have stepped since their last import");
  return LBM_OK;
}

// Orders the transfer after the source handle's work and the destination handle's later
// work after the transfer when the two handles use different streams.
static lbm_status stream_join(lbm_handle from, lbm_handle to, lbm_handle err) {
  if (from->stream == to->stream) return LBM_OK;
  cudaEvent_t ev;
  CUDA_TRY(err, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, from->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to->stream, ev, 0);
  cudaEventDestroy(ev);
  CUDA_TRY(err, e);
  return LBM_OK;
}

static int refine_planes(lbm_handle dst_h, long long dst_z, lbm_handle src_h, long long src_z, int sign,
                         RefPlanes& rp) {
  int dirs[27], c[81];
  const int nd = halo_dirs(src_h, sign, dirs);
  lbm_stencil(src_h->q, c, nullptr);
  const KParams pd = kparams(dst_h), ps = kparams(src_h);
  const size_t sb = store_bytes(src_h->prm.precision);
  const size_t pbd = (size_t)dst_h->nxp * dst_h->ny * sb, pbs = (size_t)src_h->nxp * src_h->ny * sb;
  for (int k = 0; k < nd; k++) {
    const int i = dirs[k];
    rp.dst[k] = (char*)pd.fp[i] + dst_z * (long long)pbd;
    rp.src[k] = (const char*)ps.fp[i] + src_z * (long long)pbs;
    rp.old[k] = ps.fq[i] ? (const char*)ps.fq[i] + src_z * (long long)pbs : nullptr;
    rp.cx[k] = c[3 * i];
    rp.cy[k] = c[3 * i + 1];
  }
  return nd;
}

lbm_status lbm_refine_explode(lbm_handle coarse, int coarse_face, lbm_handle fine, int fine_face, int substep) {
  lbm_status st = refine_check(coarse, coarse_face, fine, fine_face, fine);
  if (st != LBM_OK) return st;
  if (substep != 0 && substep != 1) return fail(fine, LBM_EINVAL, "substep must be 0 or 1");
  // populations leaving the coarse lattice through its face = entering the fine one through its face
  RefPlanes rp{};
  const int sign = coarse_face == 5 ? 1 : -1;
  const int nd = refine_planes(fine, fine_face == 4 ? -1 : fine->nz, coarse, coarse_face == 5 ? coarse->nz - 1 : 0,
                               sign, rp);
  st = stream_join(coarse, fine, fine);
  if (st != LBM_OK) return st;
  const long long n = (long long)nd * fine->nx * fine->ny;
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)fine->nsm * 8);
  if (fine->prm.precision == LBM_F32)
    k_refine_explode<uint32_t><<<blocks, 256, 0, fine->stream>>>(rp, nd, fine->nx, fine->ny, fine->nxp, coarse->nxp, substep);
  else
    k_refine_explode<uint16_t><<<blocks, 256, 0, fine->stream>>>(rp, nd, fine->nx, fine->ny, fine->nxp, coarse->nxp, substep);
  CUDA_TRY(fine, cudaGetLastError());
  return stream_join(fine, coarse, fine);
}

lbm_status lbm_refine_coalesce(lbm_handle fine, int fine_face, lbm_handle coarse, int coarse_face) {
  lbm_status st = refine_check(coarse, coarse_face, fine, fine_face, coarse);
  if (st != LBM_OK) return st;
  if (!fine->prev_post)
    return fail(coarse, LBM_ESTATE, "the fine lattice needs two steps since its last import");
  RefPlanes rp{};
  const int sign = fine_face == 5 ? 1 : -1;  // leaving the fine lattice through its face
  const int nd = refine_planes(coarse, coarse_face == 4 ? -1 : coarse->nz, fine, fine_face == 5 ? fine->nz - 1 : 0,
                               sign, rp);
  st = stream_join(fine, coarse, coarse);
  if (st != LBM_OK) return st;
  const long long n = (long long)nd * coarse->nx * coarse->ny;
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)coarse->nsm * 8);
  switch (coarse->prm.precision) {
    case LBM_F32:
      k_refine_coalesce<float><<<blocks, 256, 0, coarse->stream>>>(rp, nd, coarse->nx, coarse->ny, coarse->nxp, fine->nxp);
      break;
    case LBM_F16_SHIFTED:
      k_refine_coalesce<__half><<<blocks, 256, 0, coarse->stream>>>(rp, nd, coarse->nx, coarse->ny, coarse->nxp, fine->nxp);
      break;
    default:
      k_refine_coalesce<__nv_bfloat16><<<blocks, 256, 0, coarse->stream>>>(rp, nd, coarse->nx, coarse->ny, coarse->nxp,
                                                                          fine->nxp);
      break;
  }
  CUDA_TRY(coarse, cudaGetLastError());
  return stream_join(coarse, fine, coarse);
}

lbm_status lbm_sync(lbm_handle h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  CUDA_TRY(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (*h->status_host & 4) {
    h->broken = true;
    return fail(h, LBM_ECUDA, "%s", BROKEN_MSG);
  }
  if (*h->status_host & 2)
    return fail(h, LBM_ECUDA,
                "a learned-closure step gave up waiting for its tensor-core result (then waited with the full bound)");
#ifdef LBM_BOUNDS_CHECK
  int bad = 0;
  CUDA_TRY(h, cudaMemcpy(&bad, h->chk_bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) {
    static const char* names[5] = {"populations", "populations", "flags", "classes", "rules"};
    return fail(h, LBM_ECUDA, "bounds check: an access outside the %s array was skipped", names[(bad - 1) % 5]);
  }
#endif
  if (*h->status_host & 1)
    return fail(h, LBM_EUNSTABLE, "a step produced a non-finite or non-positive density");
  return LBM_OK;
}

lbm_status lbm_debug_set_wait_polls(lbm_handle h, int64_t polls) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (polls < -1 || polls > MBAR_POLLS) return fail(h, LBM_EINVAL, "polls must lie in [-1, %d]", MBAR_POLLS);
  h->wait_polls = polls < 0 ? MBAR_POLLS : (int)polls;
  return LBM_OK;
}

// raw: the values stored in the state array's own slots (layout 0), whatever the state
static lbm_status run_export(lbm_handle h, int mode, const ExportArgs& a, bool raw) {
  KParams p = kparams(h);
  if (raw) p.nat_valid = 1;
  const int par = raw ? 0 : h->parity;
  cudaError_t e = h->q == 19 ? dispatch_export<19>(h, p, mode, a, par) : dispatch_export<27>(h, p, mode, a, par);
  CUDA_TRY(h, e);
  return LBM_OK;
}

lbm_status lbm_moments(lbm_handle h, float* rho, float* u, int on_device) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!rho && !u) return LBM_OK;
  const long long n = ncell(h);
  ExportArgs a{};
  float *trho = nullptr, *tu = nullptr;
  if (on_device) {
    a.rho = rho;
    a.u = u;
  } else {  // pinned host arrays are written in place, pageable ones through a device copy
    float* arho = rho ? static_cast<float*>(host_alias(rho)) : nullptr;
    float* au = u ? static_cast<float*>(host_alias(u)) : nullptr;
    if (rho && !arho) CUDA_TRY(h, cudaMallocAsync((void**)&trho, (size_t)n * sizeof(float), h->stream));
    if (u && !au) CUDA_TRY(h, cudaMallocAsync((void**)&tu, (size_t)n * 3 * sizeof(float), h->stream));
    a.rho = arho ? arho : trho;
    a.u = au ? au : tu;
  }
  lbm_status s = run_export(h, EX_MOM, a);
  if (s != LBM_OK) return s;
  if (!on_device) {
    if (trho) CUDA_TRY(h, cudaMemcpyAsync(rho, trho, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (tu) CUDA_TRY(h, cudaMemcpyAsync(u, tu, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (trho) cudaFreeAsync(trho, h->stream);
    if (tu) cudaFreeAsync(tu, h->stream);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

static lbm_status get_pop(lbm_handle h, float* df, int on_device, bool raw);

lbm_status lbm_get_populations(lbm_handle h, float* df, int on_device) {
  return get_pop(h, df, on_device, false);
}

lbm_status lbm_get_post_collision(lbm_handle h, float* df, int on_device) {
  if (h && (h->prm.streaming != LBM_PULL || h->parity != 2))
    return fail(h, LBM_ESTATE, "no post-collision state: a two-grid pull lattice that has stepped is needed");
  return get_pop(h, df, on_device, true);
}

static lbm_status get_pop(lbm_handle h, float* df, int on_device, bool raw) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!df) return fail(h, LBM_EINVAL, "df is NULL");
  const size_t count = (size_t)ncell(h) * h->q;
  ExportArgs a{};
  float* t = nullptr;
  if (on_device) {
    a.df = df;
  } else if (float* alias = static_cast<float*>(host_alias(df))) {  // pinned: written in place
    a.df = alias;
  } else {
    CUDA_TRY(h, cudaMallocAsync((void**)&t, count * sizeof(float), h->stream));
    a.df = t;
  }
  lbm_status s = run_export(h, EX_POP, a, raw);
  if (s != LBM_OK) return s;
  if (!on_device) {
    if (t) {
      CUDA_TRY(h, cudaMemcpyAsync(df, t, count * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      cudaFreeAsync(t, h->stream);
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

lbm_status lbm_reduce(lbm_handle h, double out[4]) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  ExportArgs a{};
  a.sums = h->sums;
  a.partial = h->partial;
  lbm_status s = run_export(h, EX_SUM, a);
  if (s != LBM_OK) return s;
  CUDA_TRY(h, cudaMemcpyAsync(out, h->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_stats_reset(lbm_handle h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  CUDA_TRY(h, cudaMemsetAsync(h->stats, 0, (size_t)h->ny * LBM_STATS_K * sizeof(double), h->stream));
  h->nsamples = 0;
  return ensure_stats_w(h);
}

lbm_status lbm_stats_sample(lbm_handle h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  ExportArgs a{};
  a.sums = h->stats;
  a.partial = h->partial;
  lbm_status s = run_export(h, EX_STATS, a);
  if (s != LBM_OK) return s;
  h->nsamples++;
  return LBM_OK;
}

lbm_status lbm_stats_get(lbm_handle h, double* out, int64_t* nsamples) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  CUDA_TRY(h, cudaMemcpyAsync(out, h->stats, (size_t)h->ny * LBM_STATS_K * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (nsamples) *nsamples = h->nsamples;
  return LBM_OK;
}

lbm_status lbm_set_closure(lbm_handle h, const uint16_t* bf16_params, int n, double scale_pi,
                           double scale_rho) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!bf16_params || n != LBM_MLP_NPARAM)
    return fail(h, LBM_EINVAL, "expected %d bfloat16 parameters", LBM_MLP_NPARAM);
  if (!std::isfinite(scale_pi) || !std::isfinite(scale_rho))
    return fail(h, LBM_EINVAL, "feature scales must be finite");
  float host[LBM_MLP_NPARAM];
  for (int k = 0; k < n; k++) {
    const uint32_t bits = (uint32_t)bf16_params[k] << 16;
    float v;
    std::memcpy(&v, &bits, sizeof v);
    if (!std::isfinite(v)) return fail(h, LBM_EINVAL, "non-finite MLP parameter %d", k);
    host[k] = v;
  }
  if (!h->mlp) CUDA_TRY(h, cudaMallocAsync((void**)&h->mlp, sizeof host, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->mlp, host, sizeof host, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // host buffer is on the stack
  h->mlp_scale[0] = (float)scale_pi;
  h->mlp_scale[1] = (float)scale_rho;
  h->mlp_set = true;
  return LBM_OK;
}

lbm_status lbm_set_closure_f32(lbm_handle h, const float* params, int on_device, double scale_pi,
                               double scale_rho) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!params) return fail(h, LBM_EINVAL, "params is NULL");
  float host[LBM_MLP_NPARAM];
  if (on_device) {
    CUDA_TRY(h, cudaMemcpyAsync(host, params, sizeof host, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else {
    std::memcpy(host, params, sizeof host);
  }
  uint16_t bf[LBM_MLP_NPARAM];
  for (int k = 0; k < LBM_MLP_NPARAM; k++) {
    if (!std::isfinite(host[k])) return fail(h, LBM_EINVAL, "non-finite MLP parameter %d", k);
    uint32_t bits;
    std::memcpy(&bits, &host[k], sizeof bits);
    bits += 0x7FFFu + ((bits >> 16) & 1u);  // round to nearest even on the upper 16 bits
    bf[k] = (uint16_t)(bits >> 16);
  }
  return lbm_set_closure(h, bf, LBM_MLP_NPARAM, scale_pi, scale_rho);
}

lbm_status lbm_set_closure_floor(lbm_handle h, double cs_min) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!(cs_min >= 0.0) || !std::isfinite(cs_min)) return fail(h, LBM_EINVAL, "cs_min must be >= 0");
  h->cs_min = cs_min;
  return LBM_OK;
}

lbm_status lbm_info(lbm_handle h, int* nxp, int* bytes_per_pop, double* bytes_per_update) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (nxp) *nxp = h->nxp;
  const int s = (int)store_bytes(h->prm.precision);
  if (bytes_per_pop) *bytes_per_pop = s;
  if (bytes_per_update) *bytes_per_update = 2.0 * h->q * s + 1.0;
  return LBM_OK;
}

}  // extern "C"
