/*
 * lbm_oracle.c -- FP64 CPU oracle of the lattice Boltzmann stream-and-collide update.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Plain loops in the order of the method:
 * every step first applies the collision (Sec. 2, Eq. LBCollision) to every non-solid
 * cell, then streams (Sec. 2, Eq. LBStreaming) with the boundary rules.  No blocking, no
 * fusion, no shifted storage: the populations are the plain f_i in double precision.
 *
 * Readings of the paper (which defines neither the collision operator nor the boundary
 * schemes) are those of the standard LBM literature the paper cites for the method:
 *   - D3Q19 / D3Q27 velocity sets with weights 1/3,1/18,1/36 and 8/27,2/27,1/54,1/216;
 *   - second-order polynomial equilibrium for both sets;
 *   - TRT collision: symmetric part relaxed with omega+ = 1/tau_eff, antisymmetric part
 *     with omega- fixed by the magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2);
 *   - Guo forcing F_i = w_i [3(c_i - u) + 9 (c_i.u) c_i] . F, split into symmetric and
 *     antisymmetric parts with factors (1 - omega+/2), (1 - omega-/2); u includes +F/2;
 *   - Smagorinsky LES: tau_eff = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_s^2 sqrt(Pi:Pi)/rho))/2
 *     with Pi the non-equilibrium second moment (closed form of Hou et al. 1996);
 *   - boundaries (wind-tunnel case of Sec. 5.2: inflow left, outflow right, other faces):
 *     halfway bounce-back, moving-wall bounce-back f_i = f*_opp(i) + 6 w_i rho_w (c_i.u_w),
 *     zero-gradient outflow on the +x face (incoming populations copied from the upstream
 *     neighbour x-1 after its own streaming), specular free-slip, periodic wrap.
 *     A source crossing several faces takes the rule of highest precedence:
 *     wall > inflow > outflow > (free-slip, periodic), each free-slip axis reflected and
 *     each periodic axis wrapped independently; the flag of the resolved cell then decides
 *     between streaming and (moving-wall) bounce-back.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- velocity sets (published order: rest, then +/- pairs) ---------------------------- */

static const int C27[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},   {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};

static double weight(int q, const int* c) {
  int n = abs(c[0]) + abs(c[1]) + abs(c[2]);
  if (q == 19) {
    if (n == 0) return 1.0 / 3.0;
    if (n == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
  }
  if (n == 0) return 8.0 / 27.0;
  if (n == 1) return 2.0 / 27.0;
  if (n == 2) return 1.0 / 54.0;
  return 1.0 / 216.0;
}

static int find_dir(int q, int cx, int cy, int cz) {
  for (int i = 0; i < q; i++)
    if (C27[i][0] == cx && C27[i][1] == cy && C27[i][2] == cz) return i;
  return -1;
}

static int opposite(int q, int i) { return find_dir(q, -C27[i][0], -C27[i][1], -C27[i][2]); }

/* Lookup tables derived once from C27 and weight(): opposite direction, weight, and the
 * index of a velocity vector (the searches above are too slow inside the cell loops). */
static int OPP[27];
static double WT[2][27];
static int DIR[3][3][3];

__attribute__((constructor)) static void init_tables(void) {
  for (int i = 0; i < 27; i++) {
    OPP[i] = opposite(27, i);
    WT[0][i] = weight(19, C27[i]);
    WT[1][i] = weight(27, C27[i]);
    DIR[C27[i][0] + 1][C27[i][1] + 1][C27[i][2] + 1] = i;
  }
}

#define W_(q, i) (WT[(q) == 27][i])

int ora_stencil(int q, int* c, double* w, int* opp) {
  if (q != 19 && q != 27) return 0;
  for (int i = 0; i < q; i++) {
    if (c)
      for (int a = 0; a < 3; a++) c[3 * i + a] = C27[i][a];
    if (w) w[i] = weight(q, C27[i]);
    if (opp) opp[i] = opposite(q, i);
  }
  return q;
}

/* ---- local collision ------------------------------------------------------------------ */

void ora_equilibrium(int q, double rho, const double u[3], double* feq) {
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < q; i++) {
    double cu = C27[i][0] * u[0] + C27[i][1] * u[1] + C27[i][2] * u[2];
    feq[i] = W_(q, i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  }
}

double ora_smag_tau(double tau0, double cs2, double qn, double rho) {
  return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * sqrt(2.0) * cs2 * sqrt(qn) / rho));
}

void ora_moments_cell(const ora_cfg* cfg, const double* f, double* rho, double* u) {
  double r = 0.0, m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < cfg->q; i++) {
    r += f[i];
    for (int a = 0; a < 3; a++) m[a] += C27[i][a] * f[i];
  }
  *rho = r;
  for (int a = 0; a < 3; a++) u[a] = (m[a] + 0.5 * cfg->force[a]) / r;
}

/* Non-equilibrium second moment Pi_ab = sum_i c_ia c_ib (f_i - feq_i), as xx,yy,zz,xy,xz,yz. */
static void noneq_stress(int q, const double* f, const double* feq, double* pi) {
  static const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; k++) {
    double s = 0.0;
    for (int i = 0; i < q; i++) s += C27[i][A[k]] * C27[i][B[k]] * (f[i] - feq[i]);
    pi[k] = s;
  }
}

static double gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }

static double gelu_grad(double a) {
  return 0.5 * (1.0 + erf(a / sqrt(2.0))) + a * exp(-0.5 * a * a) / sqrt(2.0 * M_PI);
}

static double softplus(double y) { return (y > 0.0 ? y : 0.0) + log1p(exp(-fabs(y))); }

/* scaled closure features are clipped to [-8, 8] */
static double xclamp(double v) { return v < -8.0 ? -8.0 : (v > 8.0 ? 8.0 : v); }

double ora_mlp_forward(const double* p, const double* x, double* a1, double* h1, double* a2,
                       double* h2) {
  const double* W1 = p;
  const double* b1 = W1 + ORA_MLP_NH * ORA_MLP_NIN;
  const double* W2 = b1 + ORA_MLP_NH;
  const double* b2 = W2 + ORA_MLP_NH * ORA_MLP_NH;
  const double* W3 = b2 + ORA_MLP_NH;
  const double* b3 = W3 + ORA_MLP_NH;
  double la1[ORA_MLP_NH], lh1[ORA_MLP_NH], la2[ORA_MLP_NH], lh2[ORA_MLP_NH];
  for (int j = 0; j < ORA_MLP_NH; j++) {
    double s = b1[j];
    for (int k = 0; k < ORA_MLP_NIN; k++) s += W1[j * ORA_MLP_NIN + k] * x[k];
    la1[j] = s;
    lh1[j] = gelu(s);
  }
  for (int j = 0; j < ORA_MLP_NH; j++) {
    double s = b2[j];
    for (int k = 0; k < ORA_MLP_NH; k++) s += W2[j * ORA_MLP_NH + k] * lh1[k];
    la2[j] = s;
    lh2[j] = gelu(s);
  }
  double y = b3[0];
  for (int k = 0; k < ORA_MLP_NH; k++) y += W3[k] * lh2[k];
  if (a1) memcpy(a1, la1, sizeof la1);
  if (h1) memcpy(h1, lh1, sizeof lh1);
  if (a2) memcpy(a2, la2, sizeof la2);
  if (h2) memcpy(h2, lh2, sizeof lh2);
  return y;
}

void ora_mlp_backward(const double* p, const double* x, double dy, double* grad) {
  const double* W2 = p + ORA_MLP_NH * ORA_MLP_NIN + ORA_MLP_NH;
  const double* W3 = W2 + ORA_MLP_NH * ORA_MLP_NH + ORA_MLP_NH;
  double* gW1 = grad;
  double* gb1 = gW1 + ORA_MLP_NH * ORA_MLP_NIN;
  double* gW2 = gb1 + ORA_MLP_NH;
  double* gb2 = gW2 + ORA_MLP_NH * ORA_MLP_NH;
  double* gW3 = gb2 + ORA_MLP_NH;
  double* gb3 = gW3 + ORA_MLP_NH;
  double a1[ORA_MLP_NH], h1[ORA_MLP_NH], a2[ORA_MLP_NH], h2[ORA_MLP_NH];
  ora_mlp_forward(p, x, a1, h1, a2, h2);
  /* output layer */
  gb3[0] += dy;
  double d2[ORA_MLP_NH];
  for (int k = 0; k < ORA_MLP_NH; k++) {
    gW3[k] += dy * h2[k];
    d2[k] = dy * W3[k] * gelu_grad(a2[k]);
  }
  /* second layer */
  double d1[ORA_MLP_NH];
  for (int k = 0; k < ORA_MLP_NH; k++) d1[k] = 0.0;
  for (int j = 0; j < ORA_MLP_NH; j++) {
    gb2[j] += d2[j];
    for (int k = 0; k < ORA_MLP_NH; k++) {
      gW2[j * ORA_MLP_NH + k] += d2[j] * h1[k];
      d1[k] += d2[j] * W2[j * ORA_MLP_NH + k];
    }
  }
  /* first layer */
  for (int j = 0; j < ORA_MLP_NH; j++) {
    double d = d1[j] * gelu_grad(a1[j]);
    gb1[j] += d;
    for (int k = 0; k < ORA_MLP_NIN; k++) gW1[j * ORA_MLP_NIN + k] += d * x[k];
  }
}

void ora_mlp_features(const ora_cfg* cfg, const double* f, double* x) {
  double rho, u[3], feq[27], pi[6];
  ora_moments_cell(cfg, f, &rho, u);
  ora_equilibrium(cfg->q, rho, u, feq);
  noneq_stress(cfg->q, f, feq, pi);
  for (int k = 0; k < 6; k++) x[k] = xclamp(cfg->mlp_scale[0] * pi[k]);
  x[6] = xclamp(cfg->mlp_scale[1] * (rho - 1.0));
}

/* ---- MRT collision (D3Q19) ----------------------------------------------------------------
 * d'Humieres, Ginzburg, Krafczyk, Lallemand & Luo, "Multiple-relaxation-time lattice Boltzmann
 * models in three dimensions", Phil. Trans. R. Soc. A 360 (2002) 437: moments m_k = sum_i M_ki f_i
 * with the orthogonal polynomial rows below (c2 = |c_i|^2), each relaxed toward the moment of
 * the equilibrium at its own rate s_k:
 *   f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M F,
 * Guo's force F_i written in moment space.  The rows are orthogonal, so M^-1 = M^T diag(1/|M_k|^2). */
double ora_mrt_row(int k, int i) {
  const double cx = C27[i][0], cy = C27[i][1], cz = C27[i][2];
  const double c2 = cx * cx + cy * cy + cz * cz;
  switch (k) {
    case 0: return 1.0;                                            /* rho */
    case 1: return 19.0 * c2 - 30.0;                               /* e */
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;      /* eps */
    case 3: return cx;                                             /* j_x */
    case 4: return (5.0 * c2 - 9.0) * cx;                          /* q_x */
    case 5: return cy;
    case 6: return (5.0 * c2 - 9.0) * cy;
    case 7: return cz;
    case 8: return (5.0 * c2 - 9.0) * cz;
    case 9: return 3.0 * cx * cx - c2;                             /* 3 p_xx */
    case 10: return (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);       /* 3 pi_xx */
    case 11: return cy * cy - cz * cz;                             /* p_ww */
    case 12: return (3.0 * c2 - 5.0) * (cy * cy - cz * cz);        /* pi_ww */
    case 13: return cx * cy;                                       /* p_xy */
    case 14: return cy * cz;                                       /* p_yz */
    case 15: return cx * cz;                                       /* p_xz */
    case 16: return (cy * cy - cz * cz) * cx;                      /* m_x */
    case 17: return (cz * cz - cx * cx) * cy;                      /* m_y */
    default: return (cx * cx - cy * cy) * cz;                      /* m_z */
  }
}

/* Rate of moment k: conserved moments 1 (they enter only through the force), stress moments
 * 1/tau_eff, the others from cfg->mrt_s (e, eps, q, pi, m). */
static double mrt_rate(const ora_cfg* cfg, int k, double tau) {
  switch (k) {
    case 0: case 3: case 5: case 7: return 1.0;
    case 1: return cfg->mrt_s[0];
    case 2: return cfg->mrt_s[1];
    case 4: case 6: case 8: return cfg->mrt_s[2];
    case 10: case 12: return cfg->mrt_s[3];
    case 16: case 17: case 18: return cfg->mrt_s[4];
    default: return 1.0 / tau; /* 9, 11, 13, 14, 15 */
  }
}

static void mrt_collide(const ora_cfg* cfg, const double* f, const double* feq, const double* fi, double tau,
                        double* fstar) {
  double dm[19];
  for (int k = 0; k < 19; k++) {
    double m = 0.0, meq = 0.0, mf = 0.0, norm = 0.0;
    for (int i = 0; i < 19; i++) {
      const double r = ora_mrt_row(k, i);
      m += r * f[i];
      meq += r * feq[i];
      mf += r * fi[i];
      norm += r * r;
    }
    const double s = mrt_rate(cfg, k, tau);
    dm[k] = (-s * (m - meq) + (1.0 - 0.5 * s) * mf) / norm;
  }
  for (int i = 0; i < 19; i++) {
    double d = 0.0;
    for (int k = 0; k < 19; k++) d += ora_mrt_row(k, i) * dm[k];
    fstar[i] = f[i] + d;
  }
}

void ora_collide(const ora_cfg* cfg, const double* f, double* fstar, double* tau_eff) {
  const int q = cfg->q;
  double rho, u[3], feq[27];
  ora_moments_cell(cfg, f, &rho, u);
  ora_equilibrium(q, rho, u, feq);

  double tau = cfg->tau;
  if (cfg->closure != ORA_CLOSURE_NONE) {
    double pi[6];
    noneq_stress(q, f, feq, pi);
    double qn = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] +
                2.0 * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]);
    double cs2;
    if (cfg->closure == ORA_CLOSURE_SMAG) {
      cs2 = cfg->cs * cfg->cs;
    } else {
      double x[ORA_MLP_NIN];
      for (int k = 0; k < 6; k++) x[k] = xclamp(cfg->mlp_scale[0] * pi[k]);
      x[6] = xclamp(cfg->mlp_scale[1] * (rho - 1.0));
      double y = ora_mlp_forward(cfg->mlp, x, NULL, NULL, NULL, NULL);
      cs2 = softplus(y) * cfg->cs * cfg->cs / log(2.0);
      if (cs2 < cfg->mlp_cs_min * cfg->mlp_cs_min) cs2 = cfg->mlp_cs_min * cfg->mlp_cs_min;
    }
    tau = ora_smag_tau(cfg->tau, cs2, qn, rho);
  }
  if (tau_eff) *tau_eff = tau;
  double wp = 1.0 / tau;
  double wm = 1.0 / (cfg->lambda / (tau - 0.5) + 0.5);

  /* Guo forcing term per direction. */
  double fi[27];
  double uF = u[0] * cfg->force[0] + u[1] * cfg->force[1] + u[2] * cfg->force[2];
  for (int i = 0; i < q; i++) {
    double cu = C27[i][0] * u[0] + C27[i][1] * u[1] + C27[i][2] * u[2];
    double cF = C27[i][0] * cfg->force[0] + C27[i][1] * cfg->force[1] + C27[i][2] * cfg->force[2];
    fi[i] = W_(q, i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
  }
  if (cfg->collision == ORA_COLL_MRT) {
    mrt_collide(cfg, f, feq, fi, tau, fstar);
    return;
  }
  if (cfg->collision == ORA_COLL_REG) {
    /* BGK with Guo forcing reads f* = f^eq + (1 - w) g + F_i/2 with g = f - f^eq + F_i/2;
     * the regularised operator keeps only the projection of g on the Hermite polynomials
     * H_i = c_i c_i - I/3: g_i -> (9/2) w_i H_i : P, P = sum_j c_j c_j g_j (sum_j g_j = 0) */
    double P[3][3] = {{0.0}};
    for (int i = 0; i < q; i++) {
      double g = f[i] - feq[i] + 0.5 * fi[i];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) P[a][b] += C27[i][a] * C27[i][b] * g;
    }
    double tr = P[0][0] + P[1][1] + P[2][2];
    for (int i = 0; i < q; i++) {
      double h = -tr / 3.0;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) h += C27[i][a] * C27[i][b] * P[a][b];
      fstar[i] = feq[i] + 0.5 * fi[i] + (1.0 - wp) * 4.5 * W_(q, i) * h;
    }
    return;
  }
  for (int i = 0; i < q; i++) {
    int j = OPP[i];
    double fp = 0.5 * (f[i] + f[j]), fm = 0.5 * (f[i] - f[j]);
    double ep = 0.5 * (feq[i] + feq[j]), em = 0.5 * (feq[i] - feq[j]);
    double Fp = 0.5 * (fi[i] + fi[j]), Fm = 0.5 * (fi[i] - fi[j]);
    fstar[i] = f[i] - wp * (fp - ep) - wm * (fm - em) + (1.0 - 0.5 * wp) * Fp +
               (1.0 - 0.5 * wm) * Fm;
  }
}

/* ---- streaming with boundary rules ---------------------------------------------------- */

static int64_t cell_index(const ora_cfg* cfg, int x, int y, int z) {
  return ((int64_t)z * cfg->ny + y) * cfg->nx + x;
}

static int cell_flag(const ora_cfg* cfg, int x, int y, int z) {
  return cfg->flags ? cfg->flags[cell_index(cfg, x, y, z)] : ORA_CELL_FLUID;
}

static int face_rank(int type) {
  switch (type) {
    case ORA_FACE_WALL: return 4;
    case ORA_FACE_INFLOW: return 3;
    case ORA_FACE_OUTFLOW: return 2;
    default: return 1; /* periodic, free-slip */
  }
}

static double inflow_term(const ora_cfg* cfg, int i) {
  double cu = C27[i][0] * cfg->u_w[0] + C27[i][1] * cfg->u_w[1] + C27[i][2] * cfg->u_w[2];
  return 6.0 * W_(cfg->q, i) * cfg->rho_w * cu;
}

double ora_pull(const ora_cfg* cfg, int x, int y, int z, int i, ora_fstar_fn fs, void* ctx) {
  const int n[3] = {cfg->nx, cfg->ny, cfg->nz};
  const int xc[3] = {x, y, z};
  const int self = OPP[i];
  const int64_t here = cell_index(cfg, x, y, z);
  int s[3], face[3], rank = 0;
  for (int a = 0; a < 3; a++) {
    s[a] = xc[a] - C27[i][a];
    face[a] = -1;
    if (s[a] < 0) face[a] = 2 * a;
    if (s[a] >= n[a]) face[a] = 2 * a + 1;
    if (face[a] >= 0) {
      int r = face_rank(cfg->face[face[a]]);
      if (r > rank) rank = r;
    }
  }
  if (rank == 4) return fs(ctx, here, self);
  if (rank == 3) return fs(ctx, here, self) + inflow_term(cfg, i);
  if (rank == 2) {
    /* zero-gradient outflow: the value the upstream neighbour x-1 receives */
    if (cell_flag(cfg, x - 1, y, z) != ORA_CELL_FLUID) return fs(ctx, here, self);
    return ora_pull(cfg, x - 1, y, z, i, fs, ctx);
  }
  int p[3], d[3];
  for (int a = 0; a < 3; a++) {
    p[a] = s[a];
    d[a] = C27[i][a];
    if (face[a] >= 0) {
      if (cfg->face[face[a]] == ORA_FACE_PERIODIC) {
        p[a] = (s[a] + n[a]) % n[a];
      } else { /* free-slip: stay in the plane, reflect the normal component */
        p[a] = xc[a];
        d[a] = -d[a];
      }
    }
  }
  int fl = cell_flag(cfg, p[0], p[1], p[2]);
  if (fl == ORA_CELL_SOLID) return fs(ctx, here, self);
  if (fl == ORA_CELL_INFLOW) return fs(ctx, here, self) + inflow_term(cfg, i);
  return fs(ctx, cell_index(cfg, p[0], p[1], p[2]), DIR[d[0] + 1][d[1] + 1][d[2] + 1]);
}

int ora_check(const ora_cfg* cfg) {
  if (cfg->q != 19 && cfg->q != 27) return -1;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return -2;
  if (!(cfg->tau > 0.5)) return -3;
  for (int a = 0; a < 3; a++)
    if ((cfg->face[2 * a] == ORA_FACE_PERIODIC) != (cfg->face[2 * a + 1] == ORA_FACE_PERIODIC))
      return -4;
  for (int k = 0; k < 6; k++) {
    if (cfg->face[k] < ORA_FACE_PERIODIC || cfg->face[k] > ORA_FACE_OUTFLOW) return -5;
    if (cfg->face[k] == ORA_FACE_OUTFLOW && k != 1) return -6;
  }
  if (cfg->face[1] == ORA_FACE_OUTFLOW && cfg->nx < 2) return -7;
  if (cfg->closure == ORA_CLOSURE_MLP && !cfg->mlp) return -8;
  if (cfg->collision != ORA_COLL_TRT && cfg->collision != ORA_COLL_MRT && cfg->collision != ORA_COLL_REG)
    return -9;
  if (cfg->collision == ORA_COLL_MRT) {
    if (cfg->q != 19) return -10;
    for (int k = 0; k < 5; k++)
      if (!(cfg->mrt_s[k] > 0.0 && cfg->mrt_s[k] < 2.0)) return -11;
  }
  return 0;
}

typedef struct {
  const double* fstar;
  int64_t ncell;
} array_ctx;

static double array_lookup(void* ctx, int64_t cell, int dir) {
  const array_ctx* a = (const array_ctx*)ctx;
  return a->fstar[(int64_t)dir * a->ncell + cell];
}

int ora_stream(const ora_cfg* cfg, const double* fstar, double* f, int nthreads) {
  if (ora_check(cfg) != 0) return -1;
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  if (nthreads < 1) nthreads = 1;
  array_ctx ctx = {fstar, N};
  /* Eq. LBStreaming with the boundary rules */
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int z = 0; z < cfg->nz; z++)
    for (int y = 0; y < cfg->ny; y++)
      for (int x = 0; x < cfg->nx; x++) {
        int64_t c = cell_index(cfg, x, y, z);
        if (cell_flag(cfg, x, y, z) != ORA_CELL_FLUID) {
          for (int i = 0; i < q; i++) f[i * N + c] = W_(q, i);
          continue;
        }
        for (int i = 0; i < q; i++) f[i * N + c] = ora_pull(cfg, x, y, z, i, array_lookup, &ctx);
      }
  return 0;
}

int ora_collide_all(const ora_cfg* cfg, const double* f, double* fstar, int nthreads) {
  if (ora_check(cfg) != 0) return -1;
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  if (nthreads < 1) nthreads = 1;
  /* Eq. LBCollision on every fluid cell */
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int z = 0; z < cfg->nz; z++)
    for (int y = 0; y < cfg->ny; y++)
      for (int x = 0; x < cfg->nx; x++) {
        int64_t c = cell_index(cfg, x, y, z);
        double fl[27], fs[27];
        if (cell_flag(cfg, x, y, z) != ORA_CELL_FLUID) {
          for (int i = 0; i < q; i++) fstar[i * N + c] = 0.0;
          continue;
        }
        for (int i = 0; i < q; i++) fl[i] = f[i * N + c];
        ora_collide(cfg, fl, fs, NULL);
        for (int i = 0; i < q; i++) fstar[i * N + c] = fs[i];
      }
  return 0;
}

int ora_step(const ora_cfg* cfg, double* f, double* work, int64_t nsteps, int nthreads) {
  if (ora_check(cfg) != 0) return -1;
  for (int64_t t = 0; t < nsteps; t++) {
    ora_collide_all(cfg, f, work, nthreads);
    ora_stream(cfg, work, f, nthreads);
  }
  return 0;
}

void ora_init_equilibrium(const ora_cfg* cfg, const double* rho, const double* u, double* f) {
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  for (int64_t c = 0; c < N; c++) {
    double feq[27];
    if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) {
      for (int i = 0; i < q; i++) f[i * N + c] = W_(q, i);
      continue;
    }
    double uc[3] = {u[c], u[N + c], u[2 * N + c]};
    ora_equilibrium(q, rho[c], uc, feq);
    for (int i = 0; i < q; i++) f[i * N + c] = feq[i];
  }
}

void ora_moments(const ora_cfg* cfg, const double* f, double* rho, double* u) {
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  for (int64_t c = 0; c < N; c++) {
    if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) {
      rho[c] = 0.0;
      u[c] = u[N + c] = u[2 * N + c] = 0.0;
      continue;
    }
    double fl[27], r, uc[3];
    for (int i = 0; i < q; i++) fl[i] = f[i * N + c];
    ora_moments_cell(cfg, fl, &r, uc);
    rho[c] = r;
    u[c] = uc[0];
    u[N + c] = uc[1];
    u[2 * N + c] = uc[2];
  }
}

void ora_mass_momentum(const ora_cfg* cfg, const double* f, double* out) {
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int64_t c = 0; c < N; c++) {
    if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) continue;
    double fl[27], r, uc[3];
    for (int i = 0; i < q; i++) fl[i] = f[i * N + c];
    ora_moments_cell(cfg, fl, &r, uc);
    out[0] += r;
    for (int a = 0; a < 3; a++) out[1 + a] += r * uc[a];
  }
}

/* On-demand post-collision values for ora_step_sampled: f(t) = f^eq(rho_in, u_in). */
typedef struct {
  const ora_cfg* cfg;
  const float* rho;
  const float* u;
  int64_t ncell;
  int64_t cached_cell;
  double cached[27];
} eq_ctx;

static double eq_lookup(void* vctx, int64_t cell, int dir) {
  eq_ctx* e = (eq_ctx*)vctx;
  if (e->cached_cell != cell) {
    double f[27], uc[3] = {e->u[cell], e->u[e->ncell + cell], e->u[2 * e->ncell + cell]};
    ora_equilibrium(e->cfg->q, (double)e->rho[cell], uc, f);
    ora_collide(e->cfg, f, e->cached, NULL);
    e->cached_cell = cell;
  }
  return e->cached[dir];
}

void ora_step_sampled(const ora_cfg* cfg, const float* rho_in, const float* u_in,
                      const int64_t* cells, int64_t n, double* out) {
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  for (int64_t k = 0; k < n; k++) {
    int64_t c = cells[k];
    int x = (int)(c % cfg->nx), y = (int)((c / cfg->nx) % cfg->ny), z = (int)(c / ((int64_t)cfg->nx * cfg->ny));
    eq_ctx e = {cfg, rho_in, u_in, N, -1, {0}};
    for (int i = 0; i < cfg->q; i++) {
      if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) {
        out[k * cfg->q + i] = 0.0;
        continue;
      }
      out[k * cfg->q + i] = ora_pull(cfg, x, y, z, i, eq_lookup, &e);
    }
  }
}

/* On-demand post-collision values for ora_step_sampled_pop: f(t) = w + df (shifted float32
 * populations given for every cell, [q][N]). */
typedef struct {
  const ora_cfg* cfg;
  const float* df;
  int64_t ncell;
  int64_t cached_cell;
  double cached[27];
} pop_ctx;

static double pop_lookup(void* vctx, int64_t cell, int dir) {
  pop_ctx* e = (pop_ctx*)vctx;
  if (e->cached_cell != cell) {
    double f[27];
    for (int i = 0; i < e->cfg->q; i++) f[i] = W_(e->cfg->q, i) + (double)e->df[(int64_t)i * e->ncell + cell];
    ora_collide(e->cfg, f, e->cached, NULL);
    e->cached_cell = cell;
  }
  return e->cached[dir];
}

void ora_step_sampled_pop(const ora_cfg* cfg, const float* df, const int64_t* cells, int64_t n, double* out) {
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  for (int64_t k = 0; k < n; k++) {
    int64_t c = cells[k];
    int x = (int)(c % cfg->nx), y = (int)((c / cfg->nx) % cfg->ny), z = (int)(c / ((int64_t)cfg->nx * cfg->ny));
    pop_ctx e = {cfg, df, N, -1, {0}};
    for (int i = 0; i < cfg->q; i++) {
      if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) {
        out[k * cfg->q + i] = 0.0;
        continue;
      }
      out[k * cfg->q + i] = ora_pull(cfg, x, y, z, i, pop_lookup, &e);
    }
  }
}

void ora_stats_sample(const ora_cfg* cfg, const double* f, double* acc) {
  const int q = cfg->q;
  const int64_t N = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  for (int z = 0; z < cfg->nz; z++)
    for (int y = 0; y < cfg->ny; y++)
      for (int x = 0; x < cfg->nx; x++) {
        int64_t c = cell_index(cfg, x, y, z);
        if (cfg->flags && cfg->flags[c] != ORA_CELL_FLUID) continue;
        double fl[27], r, u[3];
        for (int i = 0; i < q; i++) fl[i] = f[i * N + c];
        ora_moments_cell(cfg, fl, &r, u);
        double* a = acc + (int64_t)y * 10;
        a[0] += 1.0;
        a[1] += u[0];
        a[2] += u[1];
        a[3] += u[2];
        a[4] += u[0] * u[0];
        a[5] += u[1] * u[1];
        a[6] += u[2] * u[2];
        a[7] += u[0] * u[1];
        a[8] += u[0] * u[2];
        a[9] += u[1] * u[2];
      }
}

/* ---- learned closure ------------------------------------------------------------------- */

static double sigmoid(double y) { return 1.0 / (1.0 + exp(-y)); }

void ora_closure_samples(const ora_cfg* fine, const double* f, double tau0_c, double cs0,
                         const double* scale, double* x, double* target, double* smag,
                         double* weight) {
  const int q = fine->q;
  const int ncx = fine->nx / 2, ncy = fine->ny / 2, ncz = fine->nz / 2;
  const int64_t N = (int64_t)fine->nx * fine->ny * fine->nz;
  static const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  for (int Z = 0; Z < ncz; Z++)
    for (int Y = 0; Y < ncy; Y++)
      for (int X = 0; X < ncx; X++) {
        const int64_t k = ((int64_t)Z * ncy + Y) * ncx + X;
        double rho_s = 0.0, m_s[3] = {0, 0, 0}, ruu_s[6] = {0, 0, 0, 0, 0, 0};
        double S_s[6] = {0, 0, 0, 0, 0, 0}, nS_s[6] = {0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 2; c++)
          for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
              const int fx = 2 * X + a, fy = 2 * Y + b, fz = 2 * Z + c;
              const int64_t cell = ((int64_t)fz * fine->ny + fy) * fine->nx + fx;
              double fl[27], rho, u[3], feq[27], pi[6];
              for (int i = 0; i < q; i++) fl[i] = f[i * N + cell];
              ora_moments_cell(fine, fl, &rho, u);
              ora_equilibrium(q, rho, u, feq);
              noneq_stress(q, fl, feq, pi);
              double qn = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] +
                          2.0 * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]);
              double tau = fine->closure == ORA_CLOSURE_SMAG
                               ? ora_smag_tau(fine->tau, fine->cs * fine->cs, qn, rho)
                               : fine->tau;
              double nut = (tau - fine->tau) / 3.0;
              rho_s += rho;
              for (int d = 0; d < 3; d++) m_s[d] += rho * u[d];
              for (int j = 0; j < 6; j++) {
                const double S = -3.0 * pi[j] / (2.0 * rho * tau);
                ruu_s[j] += rho * u[A[j]] * u[B[j]];
                S_s[j] += S;
                nS_s[j] += nut * S;
              }
            }
        const double rb = rho_s / 8.0;
        double ub[3], tsg[6], Sc[6];
        for (int d = 0; d < 3; d++) ub[d] = m_s[d] / 8.0 / rb;
        for (int j = 0; j < 6; j++) {
          tsg[j] = ruu_s[j] / 8.0 / rb - ub[A[j]] * ub[B[j]] - 2.0 * nS_s[j] / 8.0;
          Sc[j] = 2.0 * S_s[j] / 8.0;
        }
        const double tr = (tsg[0] + tsg[1] + tsg[2]) / 3.0;
        double num = 0.0, den = 0.0;
        for (int j = 0; j < 6; j++) {
          const double mult = j < 3 ? 1.0 : 2.0;
          const double td = j < 3 ? tsg[j] - tr : tsg[j];
          num += mult * td * Sc[j];
          den += mult * Sc[j] * Sc[j];
        }
        const double Smag = sqrt(2.0 * den);
        /* no strain (below round-off level): the projection is undefined, take nu* = 0 */
        double nu = Smag > 1e-10 ? -num / (2.0 * den) : 0.0;
        if (nu < 0.0) nu = 0.0;
        const double tauc = tau0_c + 3.0 * cs0 * cs0 * Smag;
        for (int j = 0; j < 6; j++) x[k * 7 + j] = xclamp(scale[0] * (-(2.0 * rb / 3.0) * tauc * Sc[j]));
        x[k * 7 + 6] = xclamp(scale[1] * (rb - 1.0));
        target[k] = nu;
        smag[k] = Smag;
        weight[k] = Smag * Smag;
      }
}

double ora_closure_loss(const double* p, const double* x, const double* target,
                        const double* smag, const double* weight, int64_t n, double cs0,
                        double* grad) {
  const double k = cs0 * cs0 / log(2.0);
  double wsum = 0.0, loss = 0.0;
  for (int64_t s = 0; s < n; s++) wsum += weight[s];
  for (int j = 0; j < ORA_MLP_NPARAM; j++) grad[j] = 0.0;
  if (wsum <= 0.0) return 0.0;
  for (int64_t s = 0; s < n; s++) {
    const double y = ora_mlp_forward(p, x + s * 7, NULL, NULL, NULL, NULL);
    const double nu = softplus(y) * k * smag[s];
    const double r = nu - target[s];
    loss += weight[s] * r * r;
    const double dy = 2.0 * weight[s] * r * k * smag[s] * sigmoid(y) / wsum;
    ora_mlp_backward(p, x + s * 7, dy, grad);
  }
  return loss / wsum;
}

void ora_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr,
              double beta1, double beta2, double eps, int64_t t) {
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t j = 0; j < n; j++) {
    m[j] = beta1 * m[j] + (1.0 - beta1) * g[j];
    v[j] = beta2 * v[j] + (1.0 - beta2) * g[j] * g[j];
    const double mh = m[j] / c1, vh = v[j] / c2;
    p[j] -= lr * mh / (sqrt(vh) + eps);
  }
}

void ora_filter2(const ora_cfg* fine, const double* f, double* rho_bar, double* u_bar) {
  const int q = fine->q;
  const int ncx = fine->nx / 2, ncy = fine->ny / 2, ncz = fine->nz / 2;
  const int64_t N = (int64_t)fine->nx * fine->ny * fine->nz, nc = (int64_t)ncx * ncy * ncz;
  for (int Z = 0; Z < ncz; Z++)
    for (int Y = 0; Y < ncy; Y++)
      for (int X = 0; X < ncx; X++) {
        const int64_t k = ((int64_t)Z * ncy + Y) * ncx + X;
        double rs = 0.0, ms[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 8; c++) {
          const int64_t cell = ((int64_t)(2 * Z + (c >> 2)) * fine->ny + 2 * Y + ((c >> 1) & 1)) * fine->nx +
                               2 * X + (c & 1);
          if (fine->flags && fine->flags[cell] != ORA_CELL_FLUID) continue;
          double fl[27], rho, u[3];
          for (int i = 0; i < q; i++) fl[i] = f[i * N + cell];
          ora_moments_cell(fine, fl, &rho, u);
          rs += rho;
          for (int d = 0; d < 3; d++) ms[d] += rho * u[d];
        }
        rho_bar[k] = rs / 8.0;
        for (int d = 0; d < 3; d++) u_bar[d * nc + k] = rs > 0.0 ? ms[d] / rs : 0.0;
      }
}
