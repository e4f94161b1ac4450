/*
 * lbm_oracle.h -- FP64 CPU oracle of the lattice Boltzmann stream-and-collide update.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (arXiv 2305.09910, Sec. 2, Eq. LBCollision and Eq. LBStreaming):
 *   collision   f*_i(x,t)       = f_i^eq + (1 - Omega) f_i^neq           (per cell, local)
 *   streaming   f_i(x+c_i, t+1) = f*_i(x,t)                              (first neighbours)
 * The paper names the collision operator but does not define it; the reading used here
 * is the two-relaxation-time (TRT) operator with magic parameter Lambda, Guo body
 * forcing split into its symmetric/antisymmetric parts, and optional Smagorinsky LES or a
 * per-cell MLP closure acting on the symmetric relaxation time.  Boundary rules: halfway
 * bounce-back, moving-wall bounce-back for velocity inflow, zero-gradient outflow on the
 * +x face, specular free-slip and periodic faces (the wind-tunnel setup of Sec. 5.2).
 *
 * Storage: plain (unshifted) populations f[i][z][y][x], x fastest, no padding, FP64.
 * State convention: the array always holds the pre-collision populations f(x,t); one
 * step applies the collision everywhere and then streams (the order of the paper's two
 * equations).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_CELL_FLUID = 0, ORA_CELL_SOLID = 1, ORA_CELL_INFLOW = 2 };
enum {
  ORA_FACE_PERIODIC = 0,
  ORA_FACE_WALL = 1,
  ORA_FACE_FREESLIP = 2,
  ORA_FACE_INFLOW = 3,
  ORA_FACE_OUTFLOW = 4
};
enum { ORA_CLOSURE_NONE = 0, ORA_CLOSURE_SMAG = 1, ORA_CLOSURE_MLP = 2 };
/* collision operator: TRT, or D3Q19 multiple-relaxation-time (MRT) in the orthogonal moment
 * basis of d'Humieres, Ginzburg, Krafczyk, Lallemand & Luo (2002), the operator the paper's
 * LAGOON runs use (Sec. 5.2) */
/* or projected regularisation (Latt & Chopard 2006): the non-equilibrium part, with the half
 * force of the forcing scheme, is replaced by its projection on the second-order Hermite
 * polynomials before it relaxes with 1/tau_eff (D3Q19 and D3Q27) */
enum { ORA_COLL_TRT = 0, ORA_COLL_MRT = 1, ORA_COLL_REG = 2 };

/* MLP closure: 7 -> 32 -> 32 -> 1, parameters packed as
 * W1[32][7], b1[32], W2[32][32], b2[32], W3[32], b3[1]. */
#define ORA_MLP_NIN 7
#define ORA_MLP_NH 32
#define ORA_MLP_NPARAM (32 * 7 + 32 + 32 * 32 + 32 + 32 + 1)

typedef struct {
  int nx, ny, nz;
  int q;                /* 19 or 27 */
  double tau;           /* molecular relaxation time tau0 = 3 nu + 1/2 */
  double lambda;        /* TRT magic parameter */
  int closure;          /* ORA_CLOSURE_* */
  double cs;            /* Smagorinsky C_s (SMAG) or reference C_s0 (MLP) */
  int face[6];          /* -x,+x,-y,+y,-z,+z : ORA_FACE_* */
  double u_w[3];        /* inflow velocity (faces and INFLOW cells) */
  double rho_w;         /* inflow density */
  double force[3];      /* constant body-force density */
  const uint8_t* flags; /* nx*ny*nz cell flags, NULL = all fluid */
  const double* mlp;    /* ORA_MLP_NPARAM parameters (closure MLP) */
  double mlp_scale[2];  /* feature scales: stress components, density deviation */
  double mlp_cs_min;    /* lower bound on the learned C_s (0: none) */
  int collision;        /* ORA_COLL_TRT (default) or ORA_COLL_MRT (D3Q19 only) */
  /* MRT rates of the moment groups energy e, energy square eps, heat flux q, stress square
   * pi and third-order m; the stress moments (3p_xx, p_ww, p_xy, p_yz, p_xz) relax with
   * 1/tau_eff, the conserved density and momentum moments with rate 1 */
  double mrt_s[5];
} ora_cfg;

/* Direction table in the published order; returns q or 0 on a bad q. */
int ora_stencil(int q, int* c /* q*3 */, double* w /* q */, int* opp /* q */);

/* Second-order equilibrium of one cell. */
void ora_equilibrium(int q, double rho, const double u[3], double* feq);

/* Smagorinsky closed form: tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt2 cs2 sqrt(Qn)/rho))/2. */
double ora_smag_tau(double tau0, double cs2, double qn, double rho);

/* Row k of the D3Q19 MRT moment basis at direction i (k = 0..18: rho, e, eps, j_x, q_x, j_y,
 * q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z). */
double ora_mrt_row(int k, int i);

/* Collision of one cell (f -> f*).  tau_eff may be NULL. */
void ora_collide(const ora_cfg* cfg, const double* f, double* fstar, double* tau_eff);

/* Macroscopic moments of one cell: rho = sum f, u = (sum c f + F/2) / rho. */
void ora_moments_cell(const ora_cfg* cfg, const double* f, double* rho, double* u);

/* Post-collision value lookup used by the streaming rule: f*_dir at linear cell index. */
typedef double (*ora_fstar_fn)(void* ctx, int64_t cell, int dir);

/* Streamed value f_i(x, t+1) of a non-solid cell, from post-collision values at t. */
double ora_pull(const ora_cfg* cfg, int x, int y, int z, int i, ora_fstar_fn fs, void* ctx);

/* Checks a configuration: 0 if usable, negative otherwise. */
int ora_check(const ora_cfg* cfg);

/* Eq. LBStreaming alone: f = streamed fstar with the boundary rules (solid cells get w). */
int ora_stream(const ora_cfg* cfg, const double* fstar, double* f, int nthreads);

/* Eq. LBCollision alone on every fluid cell: fstar = collided f (0 on other cells). */
int ora_collide_all(const ora_cfg* cfg, const double* f, double* fstar, int nthreads);

/* nsteps full steps in place on f (q*N); work is a q*N scratch array. */
int ora_step(const ora_cfg* cfg, double* f, double* work, int64_t nsteps, int nthreads);

/* f = f^eq(rho, u) on non-solid cells, f = w on solid cells.  u is 3*N (SoA). */
void ora_init_equilibrium(const ora_cfg* cfg, const double* rho, const double* u, double* f);

/* rho, u (3*N SoA) of the state; solid cells report 0. */
void ora_moments(const ora_cfg* cfg, const double* f, double* rho, double* u);

/* out[0] = sum rho, out[1..3] = sum rho u over non-solid cells. */
void ora_mass_momentum(const ora_cfg* cfg, const double* f, double* out);

/* One step from f(t) = f^eq(rho_in, u_in), evaluated only at the listed cells.
 * rho_in is N floats, u_in 3*N floats (SoA).  out is n*q (cell-major). */
void ora_step_sampled(const ora_cfg* cfg, const float* rho_in, const float* u_in,
                      const int64_t* cells, int64_t n, double* out);

/* One step from f(t) = w + df, df the shifted float32 populations of every cell ([q][N], e.g.
 * a GPU state), evaluated only at the listed cells.  out is n*q (cell-major), plain f. */
void ora_step_sampled_pop(const ora_cfg* cfg, const float* df, const int64_t* cells, int64_t n, double* out);

/* Adds one sample of per-y-plane velocity sums to acc (ny*10):
 * count, Su_x, Su_y, Su_z, Su_x^2, Su_y^2, Su_z^2, Su_xu_y, Su_xu_z, Su_yu_z. */
void ora_stats_sample(const ora_cfg* cfg, const double* f, double* acc);

/* MLP closure, one sample: features x[7] -> output y; hidden activations optional. */
double ora_mlp_forward(const double* p, const double* x, double* a1, double* h1, double* a2,
                       double* h2);
/* Gradient of y with respect to all parameters (added into grad), times dy. */
void ora_mlp_backward(const double* p, const double* x, double dy, double* grad);
/* Closure features of one cell: scaled non-equilibrium stress and density deviation, each
 * clipped to [-8, 8]. */
void ora_mlp_features(const ora_cfg* cfg, const double* f, double* x);

/* ---- learned closure: training data, loss, optimiser ------------------------------------
 * Samples for the coarse grid (half the fine resolution in each axis) from one fine state,
 * by a box filter of width 2.  For each coarse cell (8 fine cells) the fine solver's local
 * quantities are averaged: density, momentum, rho u u, strain rate estimated from the
 * non-equilibrium stress S_f = -3 Pi_f / (2 rho tau_eff), and the fine Smagorinsky stress
 * -2 nu_t,f S_f.  The unresolved stress on the coarse grid is
 *   tau_sgs = <rho u u>/<rho> - u_bar u_bar - 2 <nu_t,f S_f>,
 * the coarse strain rate is S_c = 2 <S_f> (one coarse step = two fine steps, acoustic
 * scaling), and the target eddy viscosity is the least-squares projection of the
 * deviatoric tau_sgs on S_c, nu* = -(tau_sgs^d : S_c) / (2 S_c : S_c), clipped at 0
 * (and 0 where |S_c| <= 1e-10, below the round-off of the strain estimate).
 * Features are what the coarse solver sees: Pi_c = -(2 rho_bar / 3) tau_c S_c with the
 * coarse Smagorinsky relaxation time tau_c = tau0_c + 3 cs0^2 |S_c|, |S| = sqrt(2 S:S),
 * scaled like ora_mlp_features (and, like them, clipped to [-8, 8]).  Per sample: x[7], target nu*, |S_c|, weight |S_c|^2. */
void ora_closure_samples(const ora_cfg* fine, const double* f, double tau0_c, double cs0,
                         const double* scale, double* x /* nc*7 */, double* target,
                         double* smag /* |S_c| */, double* weight);

/* Box filter of width 2: per coarse cell the mean density and the Favre-averaged velocity
 * <rho u> / <rho> of its 8 fine cells (u including +F/2).  rho_bar nc, u_bar 3*nc (SoA). */
void ora_filter2(const ora_cfg* fine, const double* f, double* rho_bar, double* u_bar);

/* Weighted mean-square error of the predicted eddy viscosity and its gradient:
 *   nu = softplus(y) cs0^2 / ln 2 * |S|,  L = sum w (nu - nu*)^2 / sum w.
 * grad (ORA_MLP_NPARAM, overwritten) = dL/dparams.  Returns L. */
double ora_closure_loss(const double* p, const double* x, const double* target,
                        const double* smag, const double* weight, int64_t n, double cs0,
                        double* grad);

/* One Adam step (Kingma and Ba 2015) on n parameters; t is the 1-based step count. */
void ora_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr,
              double beta1, double beta2, double eps, int64_t t);

#ifdef __cplusplus
}
#endif
#endif
