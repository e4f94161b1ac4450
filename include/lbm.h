/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann stream-and-collide library.
 *
 * The library advances a D3Q19 or D3Q27 lattice with the lattice Boltzmann equation of
 * arXiv 2305.09910, Sec. 2 (Eq. LBCollision: f*_i = f_i^eq + (1 - Omega) f_i^neq, a local
 * collision; Eq. LBStreaming: f_i(x + c_i, t + 1) = f*_i(x, t), first-neighbour streaming).
 * Like the generated kernels of Sec. 3, every entry point is a plain C function taking raw
 * pointers, sizes and the remaining free parameters.
 *
 * Operators (the paper names the collision and boundary schemes without defining them;
 * these are the readings implemented):
 *   collision  two-relaxation-time (TRT): the symmetric part relaxes with omega+ = 1/tau_eff,
 *              the antisymmetric part with omega- given by the magic parameter
 *              Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) (default 3/16);
 *   forcing    Guo: F_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F, split into symmetric and
 *              antisymmetric parts scaled by (1 - omega+/2) and (1 - omega-/2);
 *              the velocity is u = (sum_i c_i f_i + F/2) / rho;
 *   LES        Smagorinsky: tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C_s^2 sqrt(Pi:Pi) / rho))/2,
 *              Pi the non-equilibrium second moment; or a per-cell MLP giving C_s^2(x);
 *   boundaries halfway bounce-back (SOLID cells, WALL faces), moving-wall bounce-back
 *              f_i = f*_opp(i) + 6 w_i rho_w (c_i . u_w) (INFLOW cells and faces),
 *              zero-gradient outflow on the +x face (the incoming populations of x = nx-1
 *              equal those its upstream neighbour x = nx-2 receives), specular free-slip
 *              faces, periodic faces.  A population whose source lies across several faces
 *              follows the rule of highest precedence wall > inflow > outflow >
 *              (free-slip, periodic); free-slip axes are reflected and periodic axes wrapped
 *              independently, and the flag of the resolved cell then selects streaming or
 *              (moving-wall) bounce-back.  These are the wind-tunnel boundaries of Sec. 5.2
 *              (inflow on the left, outflow on the right).
 *
 * Velocity set order (both stencils; D3Q19 is the first 19 of D3Q27; opp(i) = i+1 for odd
 * i, i-1 for even i > 0, opp(0) = 0):
 *    0 ( 0, 0, 0)
 *    1 ( 1, 0, 0)   2 (-1, 0, 0)   3 ( 0, 1, 0)   4 ( 0,-1, 0)   5 ( 0, 0, 1)   6 ( 0, 0,-1)
 *    7 ( 1, 1, 0)   8 (-1,-1, 0)   9 ( 1,-1, 0)  10 (-1, 1, 0)  11 ( 1, 0, 1)  12 (-1, 0,-1)
 *   13 ( 1, 0,-1)  14 (-1, 0, 1)  15 ( 0, 1, 1)  16 ( 0,-1,-1)  17 ( 0, 1,-1)  18 ( 0,-1, 1)
 *   19 ( 1, 1, 1)  20 (-1,-1,-1)  21 ( 1, 1,-1)  22 (-1,-1, 1)  23 ( 1,-1, 1)  24 (-1, 1,-1)
 *   25 (-1, 1, 1)  26 ( 1,-1,-1)
 * Weights: D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216 (by |c|^2 = 0, 1, 2, 3).
 *
 * Units and layouts: lattice units (dx = dt = 1, c_s^2 = 1/3).  Host or device arrays
 * passed in are dense, x fastest: a scalar field is [nz][ny][nx]; a vector field is
 * [3][nz][ny][nx]; populations are [q][nz][ny][nx] and hold SHIFTED values
 * df_i = f_i - w_i in float32.  Inside the library populations are stored shifted in the
 * chosen precision, SoA, [q][nz][ny][nxp] with x padded to nxp = a multiple of 32.
 *
 * Ownership and ordering: the library owns its device memory (populations, flags,
 * scratch), allocated on the handle's stream.  The caller owns every pointer it passes in.
 * All device work is ordered on the handle's stream (lbm_params.stream, a cudaStream_t;
 * NULL = legacy default stream).  Calls that return data to host memory synchronise that
 * stream before returning.  Host arrays (on_device = 0) in pinned (page-locked) or managed
 * memory are read or written by the kernels in place; an input array there must stay
 * unchanged until the stream has passed the call (as for any asynchronous copy from pinned
 * memory).  Pageable host arrays are staged through device copies.  A handle must not be
 * used from two threads at once.
 *
 * Errors: every call returns an lbm_status; lbm_last_error() gives a message for the last
 * failing call on a handle.  A status of LBM_EUNSTABLE (a non-finite or non-positive
 * density was seen by a step) leaves the state in place for inspection.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1

typedef struct lbm_s* lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,      /* bad argument or configuration */
  LBM_ENOMEM = -2,      /* device or pinned allocation failed */
  LBM_ECUDA = -3,       /* a CUDA runtime call failed */
  LBM_EUNSTABLE = -4,   /* a step produced a non-finite or non-positive density */
  LBM_ESTATE = -5,      /* call not valid in the current state (e.g. no state yet) */
  LBM_EUNSUPPORTED = -6 /* valid request this build does not implement */
} lbm_status;

/* storage precision of the populations (arithmetic is float32 in every case) */
enum { LBM_F32 = 0, LBM_F16_SHIFTED = 1, LBM_BF16_SHIFTED = 2 };
/* streaming pattern: AA in place (one population array) or two-grid pull (two arrays; each
 * step gathers the neighbours' post-collision values from one and writes the other) */
enum { LBM_AA = 0, LBM_PULL = 1 };
/* relaxation-time closure */
enum { LBM_CLOSURE_NONE = 0, LBM_CLOSURE_SMAG = 1, LBM_CLOSURE_MLP = 2 };
/* face types, indexed -x, +x, -y, +y, -z, +z */
enum {
  LBM_FACE_PERIODIC = 0,
  LBM_FACE_WALL = 1,
  LBM_FACE_FREESLIP = 2,
  LBM_FACE_INFLOW = 3,
  LBM_FACE_OUTFLOW = 4, /* +x only; needs nx >= 2 and nx % 32 != 1 */
  /* -z / +z only, two-grid pull only: the lattice is one z slab of a larger one; the cells
   * beyond the face live in a ghost plane (populations and flags) filled by
   * lbm_halo_unpack from the neighbouring slab after every step */
  LBM_FACE_HALO = 5
};
/* cell flags (uint8) */
enum { LBM_CELL_FLUID = 0, LBM_CELL_SOLID = 1, LBM_CELL_INFLOW = 2 };

/* MLP closure parameters: 7 -> 32 -> 32 -> 1, packed W1[32][7], b1[32], W2[32][32], b2[32],
 * W3[32], b3 (bfloat16 bit patterns).  Features: Pi^neq_{xx,yy,zz,xy,xz,yz} * scale_pi and
 * (rho - 1) * scale_rho, each clipped to [-8, 8].  C_s^2(x) = softplus(y) * cs_smag^2 / ln 2 (y = 0 gives cs_smag^2). */
#define LBM_MLP_NPARAM 1345

/* Number of doubles per y-plane in the turbulence statistics:
 * count, Su_x, Su_y, Su_z, Su_x^2, Su_y^2, Su_z^2, Su_xu_y, Su_xu_z, Su_yu_z. */
#define LBM_STATS_K 10

typedef struct {
  uint32_t struct_size; /* = sizeof(lbm_params); lets the ABI grow */
  int32_t precision;    /* LBM_F32 (default) | LBM_F16_SHIFTED | LBM_BF16_SHIFTED */
  int32_t streaming;    /* LBM_AA (default) | LBM_PULL */
  int32_t closure;      /* LBM_CLOSURE_NONE (default) | _SMAG | _MLP */
  double magic_lambda;  /* TRT Lambda, default 3/16 */
  double cs_smag;       /* Smagorinsky constant (or the MLP's reference C_s0), default 0.1 */
  int32_t face_bc[6];   /* LBM_FACE_*, default all periodic */
  double u_inflow[3];   /* velocity of INFLOW faces and cells, default 0 */
  double rho_inflow;    /* density used by moving-wall bounce-back, default 1 */
  void* stream;         /* cudaStream_t for all work, default NULL */
  int32_t pipeline;     /* load pipeline (LBM_PIPE_*): DIRECT, the default, is the only one built */
  int32_t collision;    /* LBM_COLL_TRT (default) | LBM_COLL_MRT (D3Q19) | LBM_COLL_REG;
                         * MRT and REG without the learned closure */
  double mrt_rates[5];  /* MRT rates of the moment groups e, eps, q, pi, m; default
                         * 1.19, 1.4, 1.2, 1.4, 1.98; the stress moments relax with 1/tau_eff */
} lbm_params;

/* collision operator.  TRT: two relaxation times (magic_lambda).  MRT: the D3Q19 multiple-
 * relaxation-time operator of d'Humieres, Ginzburg, Krafczyk, Lallemand & Luo (2002) in its
 * orthogonal moment basis (rho, e, eps, j, q, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m),
 * relaxing the moments of f - f^eq (the same second-order equilibrium) with Guo's force in
 * moment space; the collision of the paper's LAGOON runs (Sec. 5.2).  REG: projected
 * regularisation (Latt & Chopard 2006), the non-hybrid member of the family of LaBS's
 * D3Q19HRR scheme (Sec. 4 and 5.1 name it without a definition; its finite-difference
 * blend is not built): with g = f - f^eq + F_i/2,
 * f*_i = f^eq_i + F_i/2 + (1 - 1/tau_eff) (9/2) w_i H_i : sum_j H_j g_j, H_i = c_i c_i - I/3
 * (D3Q19 and D3Q27). */
enum { LBM_COLL_TRT = 0, LBM_COLL_MRT = 1, LBM_COLL_REG = 2 };

/* load pipeline of the step kernels.  DIRECT (the default and the only one built): every thread
 * loads its cell's populations straight from global memory.  The staged forms (TMA bulk copies
 * into shared memory, register prefetch along z, per-lane cp.async) were measured slower than
 * direct loads on GB300, whose loads already move exactly the algorithmic bytes; their values
 * stay reserved and lbm_create answers them with LBM_EUNSUPPORTED. */
enum { LBM_PIPE_TMA = 0, LBM_PIPE_DIRECT = 1, LBM_PIPE_PREFETCH = 2, LBM_PIPE_ASYNC = 3 };

/* Halo exchange of z slabs (Sec. 3: a block's communication kernels pack and unpack the
 * populations that cross a face; only the directions crossing it travel, 5 of 19 or 9 of 27).
 * face: 4 (-z) or 5 (+z), a LBM_FACE_HALO face of a two-grid pull lattice that has stepped
 * at least once since its last import (else LBM_ESTATE).
 *   lbm_halo_bytes: size of one face's buffer, n_dir * ny * nxp * (4 or 2) bytes.
 *   lbm_halo_pack: copies the post-collision populations of the plane next to the face
 *     (z = 0 for -z, z = nz-1 for +z) that leave through it (c_z = -1 resp. +1) into buf,
 *     layout [direction (ascending index)][ny][nxp] in the storage precision.
 *   lbm_halo_unpack: copies buf into the ghost plane beyond the face (z = -1 resp. nz), for
 *     the directions that enter through it (c_z = +1 resp. -1).
 * The pack of slab A's +z face is the unpack of slab B's -z face and vice versa.  buf is a
 * device pointer (or host memory the GPU can address: pinned or managed), 4-byte aligned,
 * owned by the caller; one kernel per call, stream-ordered on the handle's stream.  Exchange
 * after every step, before the next. */
size_t lbm_halo_bytes(lbm_handle h, int face);
lbm_status lbm_halo_pack(lbm_handle h, int face, void* buf);
lbm_status lbm_halo_unpack(lbm_handle h, int face, const void* buf);

/* 2:1 static grid refinement across a z face (Sec. 3 and Fig. 2: blocks of the forest are
 * refined 2:1, and interpolation kernels carry the populations across a coarse-fine
 * transition; Sec. 5.2 runs them between the levels).  The paper leaves the transfer
 * undefined; these calls implement the volumetric, mass-conserving scheme of Rohde, Kandhai,
 * Derksen and van den Akker (2006), used by waLBerla (Schornbaum and Ruede 2016), in pull form.
 * A refined z slab is its own fine lattice (2 nx x 2 ny x 2 nz_slab cells, relaxation time
 * tau_f = 1/2 + 2 (tau_c - 1/2), body force F_c / 2: acoustic scaling) beside coarse lattices
 * that end at the slab; the faces that meet are LBM_FACE_HALO faces, coarse +z with fine -z or
 * coarse -z with fine +z.  Both lattices: two-grid pull, same stencil and precision, periodic
 * x and y faces, stepped at least once since their last import (else LBM_ESTATE); other
 * mismatches give LBM_EINVAL (LBM_EUNSUPPORTED for non-periodic x or y faces).
 * One coarse step, from post-collision states C*(t) and F*(t):
 *   lbm_refine_explode(coarse, cf, fine, ff, 0); lbm_step(fine, 1);
 *   lbm_refine_coalesce(fine, ff, coarse, cf);
 *   lbm_refine_explode(coarse, cf, fine, ff, 1); lbm_step(fine, 1); lbm_step(coarse, 1);
 * (for every interface), which leaves C*(t+1) and F*(t+1).
 *   lbm_refine_explode: writes the fine ghost plane beyond face ff, for the directions entering
 *     the fine lattice, from the post-collision populations of the coarse plane next to face
 *     cf: fine cell (x, y) of the ghost plane gets coarse cell ((x - s c_x)/2, (y - s c_y)/2)
 *     (floor, periodic), s = substep (0 before the first fine step, 1 before the second).
 *   lbm_refine_coalesce: writes the coarse ghost plane beyond face cf, for the directions
 *     entering the coarse lattice, with the mean of the 8 fine populations that reach the
 *     receiving coarse cell's volume in the two fine steps just taken (post-collision states
 *     F*(t+1/2) and F*(t) of the fine plane next to face ff; float32 sum).  Needs two fine
 *     steps since the fine lattice's last import (LBM_ESTATE).
 * One kernel per call on the destination handle's stream; when the handles use different
 * streams the call waits for the source's queued work and the source's later work waits for
 * the kernel.  Pure copies for explode (bit-exact); round-to-nearest-even into the storage
 * precision for coalesce. */
lbm_status lbm_refine_explode(lbm_handle coarse, int coarse_face, lbm_handle fine, int fine_face, int substep);
lbm_status lbm_refine_coalesce(lbm_handle fine, int fine_face, lbm_handle coarse, int coarse_face);

/* Fills p with the defaults listed above.  The parameter block holds the free parameters that
 * Sec. 3 passes to every generated kernel beside its raw pointers and shapes. */
void lbm_params_default(lbm_params* p);

/* Host-only: the library's velocity set, the c_i of Eq. LBStreaming (Sec. 2): D3Q19, the
 * stencil of Sec. 4 and 5.2, or D3Q27 (the 27-velocity extension; the paper names only D3Q19).
 * c: q*3 ints, w: q doubles (either may be NULL).  Returns q, or 0 if q is not 19 or 27. */
int lbm_stencil(int q, int* c, double* w);

/* Creates a lattice of nx*ny*nz cells (all fluid, populations at rest equilibrium rho = 1)
 * with stencil 19 or 27 and molecular relaxation time tau (> 1/2; nu = (tau - 1/2)/3).
 * p may be NULL for the defaults.  Sec. 2 (the lattice Boltzmann equation on a lattice of
 * cells) and Sec. 3 (a kernel takes raw pointers, shapes and free parameters).  Errors: EINVAL
 * for bad sizes, stencil, tau, Lambda, face combination (periodic faces come in pairs) or an
 * unknown enum value; ENOMEM; EUNSUPPORTED for an outflow face the kernels cannot serve, a
 * collision/closure/stencil combination that is not built, or a pipeline other than DIRECT.
 * *out is NULL on every error. */
lbm_status lbm_create(int nx, int ny, int nz, int stencil, double tau, const lbm_params* p,
                      lbm_handle* out);

/* Frees all device memory of h (after its stream's work).  NULL is accepted.  Memory
 * management only: the paper has no counterpart. */
lbm_status lbm_destroy(lbm_handle h);

/* Cell flags, nx*ny*nz uint8 (LBM_CELL_*), x fastest; on_device != 0 if flags is a device
 * pointer.  The geometry that the boundary kernels of Sec. 3 act on: solid cells (halfway
 * bounce-back) and the moving-wall cells of an inflow (Sec. 5.2, the wind tunnel's inflow);
 * the boundary rules are precomputed here, once per call.  Other values give EINVAL.  Cells that become fluid keep whatever populations
 * they held; call lbm_init_equilibrium or lbm_set_populations afterwards.  With a
 * LBM_FACE_HALO z face the array holds nz + 2 planes, z = -1 .. nz: the ghost planes carry
 * the flags of the neighbouring slabs' cells (so bounce-back against a solid cell across the
 * face is resolved here). */
lbm_status lbm_set_flags(lbm_handle h, const uint8_t* flags, int on_device);

/* Constant body-force density F (lattice units), used by every later step: the pressure
 * gradient that drives the turbulent channel of Sec. 5.1, entering the collision of Eq.
 * LBCollision as Guo's forcing term. */
lbm_status lbm_set_force(lbm_handle h, double fx, double fy, double fz);

/* Sets every fluid cell to f_i^eq(rho, u) (second-order equilibrium, the f^eq of Eq.
 * LBCollision, Sec. 2).  rho: N floats or NULL (rho = 1); u: 3*N floats [3][nz][ny][nx] or
 * NULL (u = 0).  The reported velocity of the new state is u + F/(2 rho).  Clears the status
 * word (instability, closure wait).  Host arrays: see "Ownership" above. */
lbm_status lbm_init_equilibrium(lbm_handle h, const float* rho, const float* u, int on_device);

/* Advances n >= 0 time steps: Eq. LBCollision then Eq. LBStreaming (Sec. 2) with the boundary
 * rules, fused into one sweep over the lattice per step (the stream-collide kernel of Sec. 3
 * and 5.2, bounded by memory bandwidth).  Asynchronous: returns
 * after enqueuing; instability is reported by lbm_sync.  Once the state is steady, several
 * steps go into one launch: on small lattices (up to 2^17 padded cells for two-grid pull,
 * 2^15 for AA) cooperative launches of up to 4096 steps separated by grid-wide barriers,
 * above that, up to 2^22 padded cells, replays of a CUDA graph of 8 steps, and single
 * launches on larger lattices; the result has the bits of n single steps.
 * LBM_ECUDA on a handle that lbm_sync has declared unusable. */
lbm_status lbm_step(lbm_handle h, int64_t n);

/* Waits for the handle's stream and reports what the steps since the last state reset saw
 * (failure detection; the paper has no counterpart).  LBM_EUNSTABLE: a non-finite or
 * non-positive density (the state is kept for inspection).  LBM_ECUDA: a learned-closure step
 * gave up its bounded wait for a tile's tensor-core result (an event that should not occur;
 * the step then waited again, with a longer bound, for the tensor core to finish and completed
 * its tiles); or that second wait gave up as well, after which the tensor-core work may still
 * have been running when the results were read and the kernel left: the handle is then marked
 * unusable and every later step returns LBM_ECUDA; or, in a library built with
 * LBM_BOUNDS_CHECK (liblbm_check.so), a kernel skipped an access outside its array. */
lbm_status lbm_sync(lbm_handle h);

/* Diagnostic: the number of polls (each a try-wait that may suspend the thread) the learned-
 * closure step makes in its first wait for each tile's tensor-core result before it gives up;
 * default 2^22 (far longer than any MMA takes), polls = -1 restores it, 0 makes every first
 * wait give up at once, which drives the timeout path of lbm_sync without a device fault
 * (the step still waits, with the full bound, for the tensor core to finish before it reads
 * the results).  EINVAL outside [-1, 2^22].  Failure detection; the paper has no
 * counterpart. */
lbm_status lbm_debug_set_wait_polls(lbm_handle h, int64_t polls);

/* Moments of the current state: rho (N floats) and u (3*N floats, includes +F/(2 rho)), the
 * local fluid properties on which f^eq of Eq. LBCollision depends (Sec. 2).  Either pointer
 * may be NULL.  Non-fluid cells report 0.  Host arrays: synchronises before returning. */
lbm_status lbm_moments(lbm_handle h, float* rho, float* u, int on_device);

/* Current populations (the PDFs f_i of Sec. 2) as shifted float32 df_i = f_i - w_i,
 * [q][nz][ny][nx]; 0 on non-fluid cells.  Exact for F32 storage; exact widening for F16/BF16
 * storage.  For checkpoints and parity checks. */
lbm_status lbm_get_populations(lbm_handle h, float* df, int on_device);

/* The stored post-collision populations f*_i(x, t) (Eq. LBCollision, Sec. 2) of the last step
 * of a two-grid pull lattice (natural slots, not streamed), as shifted float32
 * [q][nz][ny][nx]; 0 on non-fluid cells.  The values the refinement transfers move between
 * levels.  LBM_ESTATE for an AA lattice or before the first step after an import. */
lbm_status lbm_get_post_collision(lbm_handle h, float* df, int on_device);

/* Replaces the state by the given shifted populations (the PDFs f_i of Sec. 2, rounded to the
 * storage precision with round-to-nearest-even); restarts from a checkpoint.  Clears the
 * status word. */
lbm_status lbm_set_populations(lbm_handle h, const float* df, int on_device);

/* FP64 sums over fluid cells: out[0] = sum rho, out[1..3] = sum rho u.  Synchronises.  Mass
 * conservation is what the channel of Sec. 5.1 assesses first. */
lbm_status lbm_reduce(lbm_handle h, double out[4]);

/* Turbulence statistics in FP64, per y plane (LBM_STATS_K values each, see above):
 * reset, add one sample of the current state, read ny*LBM_STATS_K doubles (host).  What the
 * turbulent channel of Sec. 5.1 assesses: the symmetry and regularity of the solution and the
 * shear stresses along the wall normal, i.e. mean and fluctuation profiles over the
 * homogeneous x-z planes.  Per-cell values are float32 (the moments of lbm_moments); sums are
 * FP64.  lbm_stats_reset also allocates, once per handle, the device scratch that the
 * sampling steps of lbm_step_stats write their per-warp partial sums to. */
lbm_status lbm_stats_reset(lbm_handle h);
lbm_status lbm_stats_sample(lbm_handle h);
lbm_status lbm_stats_get(lbm_handle h, double* out, int64_t* nsamples);

/* Advances n >= 0 steps like lbm_step (Sec. 2 equations) and adds one statistics sample (the
 * channel profiles of Sec. 5.1) of the state that each
 * step k = 0, every, 2 every, ... (k counted from this call, every >= 1) starts from, i.e.
 * ceil(n / every) samples.  Without the learned closure the sample is
 * taken by that step's own kernel (per-warp float32 sums of 32 or 64 cells, then FP64 plane
 * sums), so sampling adds no pass over the populations; with the learned closure a separate
 * pass runs before the step.  Per-warp partial sums live in a scratch array allocated on the first
 * call (10 floats per warp slot, about 1.25 bytes per cell).  EINVAL for n < 0 or every < 1. */
lbm_status lbm_step_stats(lbm_handle h, int64_t n, int64_t every);

/* MLP closure parameters (host, bfloat16 bit patterns, n == LBM_MLP_NPARAM) and feature
 * scales.  Needed before stepping with closure LBM_CLOSURE_MLP.  The learned closure has no
 * counterpart in the paper (whose LES closures, Sec. 4, are fixed models): a per-cell network
 * gives the Smagorinsky coefficient inside the collision of Eq. LBCollision. */
lbm_status lbm_set_closure(lbm_handle h, const uint16_t* bf16_params, int n, double scale_pi,
                           double scale_rho);

/* As lbm_set_closure, from float32 parameters (host or device), rounded to bfloat16 with
 * round-to-nearest-even.  No counterpart in the paper (learned closure). */
lbm_status lbm_set_closure_f32(lbm_handle h, const float* params, int on_device, double scale_pi,
                               double scale_rho);

/* Lower bound on the learned coefficient: C_s^2(x) = max(network value, cs_min^2) (default
 * cs_min = 0, no bound).  No counterpart in the paper (learned closure).  A safeguard for coarse runs near tau = 1/2, where a learned eddy
 * viscosity below the Smagorinsky one can leave too little dissipation. */
lbm_status lbm_set_closure_floor(lbm_handle h, double cs_min);

/* ---- learned-closure training (all array arguments are caller-owned DEVICE pointers) ----
 * No counterpart in the paper: it compares LES closures (Sec. 4) but trains none.  The
 * closure's network is trained on pairs the solver generates: a fine lattice is
 * box-filtered (width 2) onto the coarse grid.  Per coarse cell (8 fine cells) the fine
 * solver's density, momentum, rho u u, strain rate S_f = -3 Pi^neq / (2 rho tau_eff) and
 * Smagorinsky stress -2 nu_t S_f are averaged; the unresolved stress is
 * tau_sgs = <rho u u>/<rho> - u_bar u_bar - 2 <nu_t S_f>; the coarse strain rate is
 * S_c = 2 <S_f> (one coarse step spans two fine steps); the target eddy viscosity is
 * nu* = max(0, -(tau_sgs^d : S_c) / (2 S_c : S_c)) (0 where |S_c| <= 1e-10), and the
 * features are those the coarse solver sees: Pi_c = -(2 rho_bar/3) tau_c S_c with
 * tau_c = tau0_c + 3 cs0^2 |S_c|, scaled by scale[0], and (rho_bar - 1) * scale[1].
 * Outputs (nc = (nx/2)(ny/2)(nz/2) coarse cells, x fastest): x[nc][7], target[nc],
 * smag[nc] = |S_c| = sqrt(2 S_c:S_c), weight[nc] = |S_c|^2 (0 where a fine cell is not
 * fluid).  Needs even sizes and no outflow face (EUNSUPPORTED).  Asynchronous on the
 * fine handle's stream. */
lbm_status lbm_closure_samples(lbm_handle fine, double tau0_c, double cs0, const double scale[2],
                               float* x, float* target, float* smag, float* weight);

/* Box filter of width 2 of the fine state (device outputs, nc coarse cells as above); the
 * coarse-from-fine averaging of a 2:1 grid transition (Sec. 3, Fig. 2), here for the
 * closure's reference fields:
 * rho_bar = mean density of the 8 fine cells, u_bar = <rho u> / <rho> (Favre, [3][nc]).
 * Needs even sizes and no outflow face.  Asynchronous on the fine handle's stream. */
lbm_status lbm_filter2(lbm_handle fine, float* rho_bar, float* u_bar);

/* Network output y for n samples x[n][7] (parameters: LBM_MLP_NPARAM floats).  No counterpart
 * in the paper (learned closure). */
lbm_status lbm_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream);

/* grad = sum_s dy[s] d y_s / d params (overwritten).  No counterpart in the paper. */
lbm_status lbm_mlp_backward(const float* params, const float* x, const float* dy, int64_t n,
                            float* grad, void* stream);

/* Weighted mean-square error of the predicted eddy viscosity over the batch of samples
 * offset + s * stride (s < n):  nu = softplus(y) cs0^2/ln 2 * smag,
 * L = sum w (nu - target)^2 / sum w.  grad (overwritten) = dL/dparams; *loss (host or
 * device double) = L.  Synchronises the stream.  No counterpart in the paper. */
lbm_status lbm_closure_loss_grad(const float* params, const float* x, const float* target,
                                 const float* smag, const float* weight, int64_t n, int64_t offset,
                                 int64_t stride, double cs0, float* grad, double* loss, void* stream);

/* One Adam step (Kingma and Ba 2015) on n parameters; t is the 1-based step count.  No
 * counterpart in the paper. */
lbm_status lbm_adam_step(float* params, const float* grad, float* m, float* v, int n, double lr,
                         double beta1, double beta2, double eps, int64_t t, void* stream);

/* Sizes of the handle: padded row length nxp, bytes of one stored population, algorithmic
 * bytes moved per lattice update of the stepping kernel (2 q s + 1 class byte): the n_b of
 * Eq. roofline (Sec. 5.2, 304 bytes for D3Q19 in double precision there). */
lbm_status lbm_info(lbm_handle h, int* nxp, int* bytes_per_pop, double* bytes_per_update);

/* lbm_reduce_noalloc: the sums of lbm_reduce (out[0] = sum rho, out[1..3] = sum rho u over
 * fluid cells, FP64) computed from populations the caller already holds, without allocating
 * any host or device memory.  The paper has no counterpart: this exists for callers that may
 * not allocate device memory where they need the sums (e.g. an analysis hook inside another
 * application's time loop on a GPU whose free memory that application's allocator owns, or
 * a process held to a fixed device-memory budget), since creating a handle allocates.
 *   df      device pointer, shifted float32 populations [q][nz][ny][nx] (the layout
 *           lbm_get_populations writes); caller-owned, read only.
 *   flags   device pointer to nx*ny*nz uint8 cell flags, or NULL for all fluid.
 *   force   body-force density (3 doubles, host) used for rho u = sum c f + F/2, or NULL.
 *   out     4 doubles, host or device memory; written before the call returns.
 *   stream  cudaStream_t the work is ordered on (NULL = legacy default stream).  Every call
 *           synchronises this stream before it returns, so out holds the sums on return.
 * Scratch: a static device array of LBM_NOALLOC_MAX_PARTIALS * 4 + 4 doubles (512 KiB) that
 * every GPU loading the library keeps until exit.  Lattices of more than
 * LBM_NOALLOC_MAX_PARTIALS * 16384 cells (2^28) are rejected with LBM_EINVAL and a message in
 * lbm_last_error(NULL).  The first call on a device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.  All calls share
 * the array, so calls whose GPU work overlaps race with each other.  No cudaMalloc, cudaFree
 * or allocating library call is made.  The caller must pass arrays of the stated sizes: the
 * call can only trust the pointers (the Python binding checks sizes and devices). */
#define LBM_NOALLOC_MAX_PARTIALS 16384
lbm_status lbm_reduce_noalloc(const float* df, const uint8_t* flags, int nx, int ny, int nz,
                              int stencil, const double force[3], double out[4], void* stream);

/* Message for the last failing call on h (or on creation, and on calls without a handle, when
 * h is NULL).  Error reporting; the paper has no counterpart. */
const char* lbm_last_error(lbm_handle h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
