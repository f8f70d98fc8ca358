/*
 * FP64 CPU oracle: one time step of the double-MRT lattice Boltzmann model of
 * Liu & He (arXiv:1503.08406), written out plainly.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  It is not part of the product
 * path and shares nothing with the CUDA library.
 *
 * Order of one step n -> n+1 (Sec. 3, Sec. 4 preamble):
 *   1. T(x,n) = sum_i g_i                                        Eq. (33)
 *   2. flow lattice on liquid nodes: rho, v, u, F, m = M f, m^eq, S,
 *      m+ = m - Lambda (m - m^eq) + (I - Lambda/2) S, f+ = M^-1 m+,
 *      stream; links into solid or wall nodes bounce back halfway   Eq. (4)-(6), (16)-(28)
 *   3. thermal lattice: non-equilibrium extrapolation on wall nodes,
 *      n+ = n - Theta (n - n^eq) + S~, g+ = N^-1 n+, stream        Eq. (30)-(39)
 *   4. iterative enthalpy method for f_l(n+1), which S~ needs     Eq. (38), (40)-(42)
 *
 * Readings of the paper taken here (the CUDA path takes the same ones):
 *  - d_0 in Eq. (26) is l_0.
 *  - Lambda is diagonal in moment space, entries (1, s_e, s_eps, 1, s_q, 1, s_q, s_nu, s_nu).
 *  - the force correction in Eq. (17) uses rho_0, as Eq. (25) does.
 *  - Eq. (6) is evaluated at varphi = phi f_l; the input K is the fully liquid
 *    permeability, so K_eff = K f_l^3 ((1 - phi) / (1 - phi f_l))^2.
 *  - a node carries flow when it is not a wall node and f_l >= f_act; other
 *    nodes keep their populations unchanged and reflect incoming links.
 *  - wall nodes are the outer rows/columns of non-periodic sides; the thermal
 *    extrapolation is applied before collision, with the inward neighbour as
 *    the fluid node; an adiabatic wall takes the neighbour's temperature.
 *  - the enthalpy fixed point h = T + a f_l, f_l = clamp((h - T_s)/(dT~ + a)),
 *    a = phi dT / (sigma St), is reached by the plain iteration of Sec. 3.2.
 *  - varphi, K_eff, sigma and tau_T use f_l(n) for the whole step; only the
 *    source uses f_l(n+1).
 *  - with alpha_l != alpha_s (Sec. 4.1), tau_T = 1/2 + alpha_e/(sigma c_sT^2),
 *    alpha_e = alpha_l f_l + alpha_s (1 - f_l), per node; a wall node relaxes
 *    at the rate of the inward neighbour it extrapolates from.
 *  - flow walls (flow_walls = 1): the non-equilibrium extrapolation of Sec. 4
 *    for the no-slip walls.  A wall node whose inward neighbour carries flow
 *    is a boundary node: before collision its populations become
 *    f^eq(rho_f, 0) + f(x_f) - f^eq(rho_f, u_f), with rho_f, u_f and varphi of
 *    the inward node x_f; it then collides with x_f's T, f_l, phi and K and
 *    streams like a flow node; links into it are no longer reflected.  (The
 *    default, flow_walls = 0, reflects them halfway.)
 *  - flow front (flow_front = 1): the same extrapolation for the no-slip condition on
 *    the moving solid-liquid interface (Sec. 4).  A link from a flow node x into a
 *    non-flow lattice node x_s (not a wall) returns, instead of x's own reflected
 *    population, the one x_s would stream back as a boundary node extrapolated from x:
 *    f^eq(rho_x, 0) + f(x) - f^eq(rho_x, u_x) collided with x's T, f_l, phi and K.
 *    Each link takes its own flow node, so no choice among a solid node's neighbours
 *    is needed; x_s keeps its populations (flow only in the liquid).
 *  - with sigma_solid set, sigma follows Eq. (7), linear in f_l:
 *    sigma(f_l) = sigma_s + f_l (sigma_l - sigma_s), evaluated at f_l(n) per
 *    node for the step, in tau_T, in n^eq of Eq. (34) and in the latent
 *    coefficient a = phi dT / (sigma St) of Eq. (38); the given tau_T (or the
 *    one derived from lambda) belongs to the liquid, alpha_l = sigma_l c_sT^2
 *    (tau_T - 1/2).  A wall node takes its inward neighbour's sigma, as for
 *    tau_T.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- D2Q9 velocity set, Eq. (15): rest, E, N, W, S, NE, NW, SW, SE ---- */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* ---- transformation matrix M, Eq. (18) ---- */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* ---- D2Q5 velocity set, Eq. (31), and matrix N, Eq. (32) ---- */
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};
static const double N5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1}};

static const double CS2 = 1.0 / 3.0; /* c_s^2 of D2Q9 with c = 1 (Sec. 3.1) */

struct ora_ctx {
  ora_params p;
  int nx, ny, n;
  /* derived */
  double tau_nu, tau_T, nu_e, nu_l, alpha_e, g_beta, csT2, lat; /* lat = dT/(sigma St) */
  double Minv[9][9], Ninv[5][5];
  double lam[9];   /* diagonal of Lambda, Eq. (23) */
  double theta[5]; /* diagonal of Theta, Eq. (37) */
  double wt[5];    /* D2Q5 weights, Eq. (39) */
  /* fields */
  double *phi, *K, *wallTl;
  double *f, *fpost, *fnew; /* [9][n] */
  double *fext;             /* [9][n]: post-collision extrapolated boundary state (flow_front) */
  double *g, *gpre, *gpost, *gstar, *gtmp; /* [5][n] */
  double *fl, *fk, *fk1, *ux, *uy, *T, *Tk, *a; /* a: of the step under way */
  unsigned char *wall, *active;
  int sigma_var; /* sigma follows f_l (sigma_solid set and != sigma) */
  int64_t inner_total;
};

/* ------------------------------------------------------------------------ */
static int idx(const ora_ctx* c, int x, int y) { return y * c->nx + x; }

static int is_wall(const ora_ctx* c, int x, int y) {
  if (c->p.bc[ORA_SIDE_LEFT] != ORA_BC_PERIODIC && x == 0) return 1;
  if (c->p.bc[ORA_SIDE_RIGHT] != ORA_BC_PERIODIC && x == c->nx - 1) return 1;
  if (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC && y == 0) return 1;
  if (c->p.bc[ORA_SIDE_TOP] != ORA_BC_PERIODIC && y == c->ny - 1) return 1;
  return 0;
}

/* neighbour of (x,y) along (dx,dy): wraps on periodic axes, -1 outside the domain */
static int neighbour(const ora_ctx* c, int x, int y, int dx, int dy) {
  int xx = x + dx, yy = y + dy;
  if (xx < 0 || xx >= c->nx) {
    if (c->p.bc[ORA_SIDE_LEFT] != ORA_BC_PERIODIC) return -1;
    xx = (xx + c->nx) % c->nx;
  }
  if (yy < 0 || yy >= c->ny) {
    if (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC) return -1;
    yy = (yy + c->ny) % c->ny;
  }
  return idx(c, xx, yy);
}

static double clamp01(double v) { return v < 0 ? 0 : (v > 1 ? 1 : v); }

void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---- single-node pieces ------------------------------------------------ */

/* Eq. (29) */
void ora_feq(const ora_ctx* c, double rho, double ux, double uy, double varphi, double out[9]) {
  double rho0 = c->p.rho0;
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; ++i) {
    double eu = EX9[i] * ux + EY9[i] * uy;
    out[i] = W9[i] * (rho + rho0 * (eu / CS2 + eu * eu / (2 * CS2 * CS2 * varphi) -
                                    uu / (2 * CS2 * varphi)));
  }
}

/* Eq. (19) */
void ora_meq(const ora_ctx* c, double rho, double ux, double uy, double varphi, double out[9]) {
  double rho0 = c->p.rho0;
  double uu = ux * ux + uy * uy;
  out[0] = rho;
  out[1] = -2 * rho + 3 * rho0 * uu / varphi;
  out[2] = rho - 3 * rho0 * uu / varphi;
  out[3] = rho0 * ux;
  out[4] = -rho0 * ux;
  out[5] = rho0 * uy;
  out[6] = -rho0 * uy;
  out[7] = rho0 * (ux * ux - uy * uy) / varphi;
  out[8] = rho0 * ux * uy / varphi;
}

/* Eq. (22) */
void ora_force_moments(const ora_ctx* c, double ux, double uy, double Fx, double Fy,
                       double varphi, double out[9]) {
  double rho0 = c->p.rho0;
  double uF = ux * Fx + uy * Fy;
  out[0] = 0;
  out[1] = 6 * rho0 * uF / varphi;
  out[2] = -6 * rho0 * uF / varphi;
  out[3] = rho0 * Fx;
  out[4] = -rho0 * Fx;
  out[5] = rho0 * Fy;
  out[6] = -rho0 * Fy;
  out[7] = 2 * rho0 * (ux * Fx - uy * Fy) / varphi;
  out[8] = rho0 * (ux * Fy + uy * Fx) / varphi;
}

/* sigma of a node with liquid fraction fl: Eq. (7) is linear in f_l */
static double sigma_of(const ora_ctx* c, double fl) {
  if (!c->sigma_var) return c->p.sigma;
  return c->p.sigma_solid + fl * (c->p.sigma - c->p.sigma_solid);
}

/* Eq. (39), with the convective term switched by vartheta as in Eq. (34) */
static void geq_s(const ora_ctx* c, double T, double ux, double uy, double sig, double out[5]) {
  double th = c->p.flow ? 1.0 : 0.0;
  for (int i = 0; i < 5; ++i) {
    double eu = EX5[i] * ux + EY5[i] * uy;
    out[i] = c->wt[i] * T * (1 + th * eu / (sig * c->csT2));
  }
}
void ora_geq(const ora_ctx* c, double T, double ux, double uy, double out[5]) {
  geq_s(c, T, ux, uy, c->p.sigma, out);
}

/* Eq. (34) */
static void thermal_meq_s(const ora_ctx* c, double T, double ux, double uy, double sig,
                          double out[5]) {
  double th = c->p.flow ? 1.0 : 0.0;
  out[0] = T;
  out[1] = th * ux * T / sig;
  out[2] = th * uy * T / sig;
  out[3] = c->p.varpi * T;
  out[4] = 0;
}
void ora_thermal_meq(const ora_ctx* c, double T, double ux, double uy, double out[5]) {
  thermal_meq_s(c, T, ux, uy, c->p.sigma, out);
}

/* Permeability and inertial coefficient at varphi = phi f_l, Eq. (6). */
static void porous_coeffs(double fl, double phi, double K, double* Keff, double* CF) {
  double varphi = phi * fl;
  if (isinf(K)) {
    *Keff = INFINITY;
  } else {
    double r = (1 - phi) / (1 - varphi);
    *Keff = K * fl * fl * fl * r * r;
  }
  *CF = 1.75 / sqrt(175 * varphi * varphi * varphi);
}

/* Eq. (24)-(28) and (4)-(5): density, velocity and total body force. */
static void macro_flow(const ora_ctx* c, const double f[9], double T, double fl, double phi,
                       double K, double* rho, double* ux, double* uy, double* Fx, double* Fy) {
  double rho0 = c->p.rho0;
  double r = 0, jx = 0, jy = 0;
  for (int i = 0; i < 9; ++i) {
    r += f[i];
    jx += EX9[i] * f[i];
    jy += EY9[i] * f[i];
  }
  double varphi = phi * fl;
  double G = c->g_beta * (T - c->p.T_ref); /* Eq. (5), along +y */
  double Keff, CF;
  porous_coeffs(fl, phi, K, &Keff, &CF);
  double vx = jx / rho0;                   /* Eq. (27) */
  double vy = jy / rho0 + 0.5 * varphi * G;
  double l0 = 0.5 * (1 + varphi * 0.5 * c->nu_l / Keff); /* Eq. (28) */
  double l1 = varphi * 0.5 * CF / sqrt(Keff);
  double vmag = sqrt(vx * vx + vy * vy);
  double den = l0 + sqrt(l0 * l0 + l1 * vmag); /* Eq. (26) with d_0 = l_0 */
  double u_x = vx / den, u_y = vy / den;
  double umag = sqrt(u_x * u_x + u_y * u_y);
  /* Eq. (4) */
  *Fx = -varphi * c->nu_l / Keff * u_x - varphi * CF / sqrt(Keff) * umag * u_x;
  *Fy = -varphi * c->nu_l / Keff * u_y - varphi * CF / sqrt(Keff) * umag * u_y + varphi * G;
  *rho = r;
  *ux = u_x;
  *uy = u_y;
}

void ora_velocity(const ora_ctx* c, const double f[9], double T, double fl, double phi, double K,
                  double out[4]) {
  double rho;
  macro_flow(c, f, T, fl, phi, K, &rho, &out[0], &out[1], &out[2], &out[3]);
}

/* Eq. (16), (19)-(22): collision in moment space, back to velocity space. */
static void collide_flow(const ora_ctx* c, const double f[9], double T, double fl, double phi,
                         double K, double fpost[9], double* uxo, double* uyo) {
  double rho, ux, uy, Fx, Fy;
  macro_flow(c, f, T, fl, phi, K, &rho, &ux, &uy, &Fx, &Fy);
  double varphi = phi * fl;
  double m[9], meq[9], S[9], mp[9];
  for (int k = 0; k < 9; ++k) {
    m[k] = 0;
    for (int i = 0; i < 9; ++i) m[k] += M9[k][i] * f[i];
  }
  ora_meq(c, rho, ux, uy, varphi, meq);
  ora_force_moments(c, ux, uy, Fx, Fy, varphi, S);
  for (int k = 0; k < 9; ++k)
    mp[k] = m[k] - c->lam[k] * (m[k] - meq[k]) + (1 - 0.5 * c->lam[k]) * S[k];
  for (int i = 0; i < 9; ++i) {
    fpost[i] = 0;
    for (int k = 0; k < 9; ++k) fpost[i] += c->Minv[i][k] * mp[k];
  }
  if (uxo) *uxo = ux;
  if (uyo) *uyo = uy;
}

void ora_collide_flow(const ora_ctx* c, const double f[9], double T, double fl, double phi,
                      double K, double fpost[9]) {
  collide_flow(c, f, T, fl, phi, K, fpost, NULL, NULL);
}

/* Eq. (35), (38): collision with the latent source S~ = (S0, 0, 0, varpi S0, 0). */
double ora_theta_T(const ora_ctx* c, double fl) {
  const double r = c->p.alpha_ratio;
  const int two_alpha = (r > 0) && r != 1.0;
  if (!two_alpha && !c->sigma_var) return c->theta[1];
  /* alpha_e / alpha_l = fl + (1 - fl) alpha_s / alpha_l; tau_T - 1/2 =
   * alpha_e / (sigma(fl) c_sT^2) with alpha_l = sigma_l c_sT^2 (tau_T,l - 1/2) */
  const double ae = two_alpha ? fl + (1.0 - fl) / r : 1.0;
  if (!c->sigma_var) return 1.0 / (0.5 + (c->tau_T - 0.5) * ae);
  return 1.0 / (0.5 + (c->tau_T - 0.5) * ae * (c->p.sigma / sigma_of(c, fl)));
}

/* Eq. (35), (38) with the diffusivity rate za for the two flux moments and the
 * node's sigma in n^eq */
static void collide_thermal(const ora_ctx* c, const double g[5], double ux, double uy,
                            double src0, double za, double sig, double gpost[5]);

void ora_collide_thermal(const ora_ctx* c, const double g[5], double ux, double uy, double src0,
                         double gpost[5]) {
  collide_thermal(c, g, ux, uy, src0, c->theta[1], c->p.sigma, gpost);
}

static void collide_thermal(const ora_ctx* c, const double g[5], double ux, double uy,
                            double src0, double za, double sig, double gpost[5]) {
  double T = 0;
  for (int i = 0; i < 5; ++i) T += g[i];
  double n[5], neq[5], np[5];
  for (int k = 0; k < 5; ++k) {
    n[k] = 0;
    for (int i = 0; i < 5; ++i) n[k] += N5[k][i] * g[i];
  }
  thermal_meq_s(c, T, ux, uy, sig, neq);
  double St[5] = {src0, 0, 0, c->p.varpi * src0, 0};
  const double th[5] = {c->theta[0], za, za, c->theta[3], c->theta[4]};
  for (int k = 0; k < 5; ++k) np[k] = n[k] - th[k] * (n[k] - neq[k]) + St[k];
  for (int i = 0; i < 5; ++i) {
    gpost[i] = 0;
    for (int k = 0; k < 5; ++k) gpost[i] += c->Ninv[i][k] * np[k];
  }
}

void ora_matrices(double M[81], double Minv[81], double N[25], double Ninv[25]) {
  /* M^-1 = M^T (M M^T)^-1, P. 3.1 */
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < 9; ++k) {
      double d = 0;
      for (int j = 0; j < 9; ++j) d += M9[k][j] * M9[k][j];
      M[i * 9 + k] = M9[i][k];
      Minv[i * 9 + k] = M9[k][i] / d;
    }
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) {
      double d = 0;
      for (int j = 0; j < 5; ++j) d += N5[k][j] * N5[k][j];
      N[i * 5 + k] = N5[i][k];
      Ninv[i * 5 + k] = N5[k][i] / d;
    }
}

/* ---- context ----------------------------------------------------------- */

static int derive(ora_ctx* c) {
  ora_params* p = &c->p;
  if (p->H <= 0) p->H = p->ny;
  if (p->dT <= 0) p->dT = 1;
  if (p->rho0 <= 0) p->rho0 = 1;
  if (p->s_e <= 0) p->s_e = 1.1;
  if (p->s_eps <= 0) p->s_eps = 1.1;
  if (p->s_q <= 0) p->s_q = 1.2;
  if (p->zeta_e <= 0) p->zeta_e = 1.5;
  if (p->zeta_nu <= 0) p->zeta_nu = 1.5;
  if (p->J <= 0) p->J = 1;
  if (p->lambda_ <= 0) p->lambda_ = 1;
  if (p->sigma <= 0) return ORA_ERR_INVALID_ARG;
  if (p->sigma_solid < 0) return ORA_ERR_INVALID_ARG;
  c->sigma_var = p->sigma_solid > 0 && p->sigma_solid != p->sigma;
  if (p->St <= 0) return ORA_ERR_INVALID_ARG;
  if (!(p->varpi > -4 && p->varpi < 1)) return ORA_ERR_INVALID_ARG;
  c->csT2 = (4 + p->varpi) / 10.0; /* Eq. (39) */
  if (p->flow) {
    /* Sec. 4.3: tau_nu = 1/2 + Ma J H sqrt(3 Pr) / sqrt(Ra), nu_e = c_s^2 (tau_nu - 1/2) */
    if (p->tau_nu > 0)
      c->tau_nu = p->tau_nu;
    else if (p->Ra > 0 && p->Pr > 0 && p->Ma > 0)
      c->tau_nu = 0.5 + p->Ma * p->J * p->H * sqrt(3 * p->Pr) / sqrt(p->Ra);
    else
      return ORA_ERR_INVALID_ARG;
    c->nu_e = CS2 * (c->tau_nu - 0.5);
    c->nu_l = c->nu_e / p->J; /* J = nu_e / nu_l, Eq. (9) */
    double alpha_l = (p->Pr > 0) ? c->nu_l / p->Pr : 0;
    if (p->tau_T > 0) {
      c->tau_T = p->tau_T;
    } else {
      if (!(p->Pr > 0)) return ORA_ERR_INVALID_ARG;
      /* tau_T = 1/2 + lambda c_s^2 (tau_nu - 1/2) / (J sigma c_sT^2 Pr) */
      c->tau_T = 0.5 + p->lambda_ * CS2 * (c->tau_nu - 0.5) / (p->J * p->sigma * c->csT2 * p->Pr);
    }
    if (p->g_beta >= 0) {
      c->g_beta = p->g_beta;
    } else {
      if (!(p->Ra > 0)) return ORA_ERR_INVALID_ARG;
      /* Ra = g beta dT H^3 / (nu_l alpha_l), Eq. (9) */
      c->g_beta = p->Ra * c->nu_l * alpha_l / (p->dT * p->H * p->H * p->H);
    }
  } else {
    if (!(p->tau_T > 0)) return ORA_ERR_INVALID_ARG;
    c->tau_T = p->tau_T;
    c->tau_nu = 0;
    c->nu_e = c->nu_l = 0;
    c->g_beta = 0;
  }
  if (c->tau_T <= 0.5 || (p->flow && c->tau_nu <= 0.5)) return ORA_ERR_INVALID_ARG;
  /* alpha_e = sigma c_sT^2 (tau_T - 1/2), Eq. (39) */
  c->alpha_e = p->sigma * c->csT2 * (c->tau_T - 0.5);
  c->lat = p->dT / (p->sigma * p->St);
  double snu = 1.0 / c->tau_nu;
  double l9[9] = {1, p->s_e, p->s_eps, 1, p->s_q, 1, p->s_q, snu, snu}; /* Eq. (23) */
  memcpy(c->lam, l9, sizeof l9);
  double t5[5] = {1, 1.0 / c->tau_T, 1.0 / c->tau_T, p->zeta_e, p->zeta_nu}; /* Eq. (37) */
  memcpy(c->theta, t5, sizeof t5);
  c->wt[0] = (1 - p->varpi) / 5.0;
  for (int i = 1; i < 5; ++i) c->wt[i] = (4 + p->varpi) / 20.0;
  double M[81], Mi[81], N[25], Ni[25];
  ora_matrices(M, Mi, N, Ni);
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < 9; ++k) c->Minv[i][k] = Mi[i * 9 + k];
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 5; ++k) c->Ninv[i][k] = Ni[i * 5 + k];
  if (p->max_inner_iters <= 0) p->max_inner_iters = 1000;
  if (p->inner_tol <= 0) p->inner_tol = 1e-13;
  if (p->f_act <= 0) p->f_act = 1e-3;
  return ORA_OK;
}

int ora_create(const ora_params* p, ora_ctx** out) {
  if (!p || !out) return ORA_ERR_INVALID_ARG;
  *out = NULL;
  if (p->nx < 3 || p->ny < 3) return ORA_ERR_INVALID_ARG;
  if ((p->bc[0] == ORA_BC_PERIODIC) != (p->bc[1] == ORA_BC_PERIODIC)) return ORA_ERR_INVALID_ARG;
  if ((p->bc[2] == ORA_BC_PERIODIC) != (p->bc[3] == ORA_BC_PERIODIC)) return ORA_ERR_INVALID_ARG;
  ora_ctx* c = (ora_ctx*)calloc(1, sizeof(ora_ctx));
  if (!c) return ORA_ERR_OOM;
  c->p = *p;
  c->nx = p->nx;
  c->ny = p->ny;
  c->n = p->nx * p->ny;
  int rc = derive(c);
  if (rc) {
    free(c);
    return rc;
  }
  size_t n = (size_t)c->n;
  c->phi = calloc(n, sizeof(double));
  c->K = calloc(n, sizeof(double));
  c->wallTl = calloc((size_t)c->ny, sizeof(double));
  c->f = calloc(9 * n, sizeof(double));
  c->fpost = calloc(9 * n, sizeof(double));
  c->fnew = calloc(9 * n, sizeof(double));
  c->fext = calloc(9 * n, sizeof(double));
  c->g = calloc(5 * n, sizeof(double));
  c->gpre = calloc(5 * n, sizeof(double));
  c->gpost = calloc(5 * n, sizeof(double));
  c->gstar = calloc(5 * n, sizeof(double));
  c->gtmp = calloc(5 * n, sizeof(double));
  c->fl = calloc(n, sizeof(double));
  c->fk = calloc(n, sizeof(double));
  c->fk1 = calloc(n, sizeof(double));
  c->ux = calloc(n, sizeof(double));
  c->uy = calloc(n, sizeof(double));
  c->T = calloc(n, sizeof(double));
  c->Tk = calloc(n, sizeof(double));
  c->a = calloc(n, sizeof(double));
  c->wall = calloc(n, 1);
  c->active = calloc(n, 1);
  if (!c->phi || !c->K || !c->wallTl || !c->f || !c->fpost || !c->fnew || !c->fext || !c->g ||
      !c->gpre ||
      !c->gpost || !c->gstar || !c->gtmp || !c->fl || !c->fk || !c->fk1 || !c->ux || !c->uy ||
      !c->T || !c->Tk || !c->a || !c->wall || !c->active) {
    ora_destroy(c);
    return ORA_ERR_OOM;
  }
  for (int y = 0; y < c->ny; ++y) {
    c->wallTl[y] = p->T_bc[ORA_SIDE_LEFT];
    for (int x = 0; x < c->nx; ++x) c->wall[idx(c, x, y)] = (unsigned char)is_wall(c, x, y);
  }
  *out = c;
  return ORA_OK;
}

void ora_destroy(ora_ctx* c) {
  if (!c) return;
  free(c->phi); free(c->K); free(c->wallTl);
  free(c->f); free(c->fpost); free(c->fnew); free(c->fext);
  free(c->g); free(c->gpre); free(c->gpost); free(c->gstar); free(c->gtmp);
  free(c->fl); free(c->fk); free(c->fk1); free(c->ux); free(c->uy); free(c->T); free(c->Tk);
  free(c->a); free(c->wall); free(c->active);
  free(c);
}

void ora_get_derived(const ora_ctx* c, double out[8]) {
  out[0] = c->tau_nu; out[1] = c->tau_T; out[2] = c->nu_e; out[3] = c->nu_l;
  out[4] = c->alpha_e; out[5] = c->g_beta; out[6] = c->csT2; out[7] = c->lat;
}

int64_t ora_inner_iterations(const ora_ctx* c) { return c->inner_total; }

int ora_set_fields(ora_ctx* c, const double* phi, const double* K, const double* T0,
                   const double* fl0, const double* wall_T_left) {
  if (!c || !phi || !K || !T0 || !fl0) return ORA_ERR_INVALID_ARG;
  for (int s = 0; s < c->n; ++s) {
    if (!(phi[s] > 0 && phi[s] <= 1)) return ORA_ERR_INVALID_ARG;
    if (c->p.flow && !(phi[s] < 1)) return ORA_ERR_INVALID_ARG;
    if (!(K[s] > 0)) return ORA_ERR_INVALID_ARG;
    if (!(fl0[s] >= 0 && fl0[s] <= 1)) return ORA_ERR_INVALID_ARG;
    if (!isfinite(T0[s])) return ORA_ERR_INVALID_ARG;
  }
  if (wall_T_left)
    for (int y = 0; y < c->ny; ++y) c->wallTl[y] = wall_T_left[y];
  for (int s = 0; s < c->n; ++s) {
    c->phi[s] = phi[s];
    c->K[s] = K[s];
    c->fl[s] = fl0[s];
    c->a[s] = phi[s] * c->lat; /* a = phi L/(sigma c_pl), Eq. (38), in temperature units */
    if (c->sigma_var) c->a[s] = phi[s] * c->p.dT / (sigma_of(c, fl0[s]) * c->p.St);
    double feq[9], geq[5];
    ora_feq(c, c->p.rho0, 0, 0, 1, feq);
    ora_geq(c, T0[s], 0, 0, geq);
    for (int i = 0; i < 9; ++i) c->f[i * c->n + s] = feq[i];
    for (int i = 0; i < 5; ++i) c->g[i * c->n + s] = geq[i];
    c->ux[s] = c->uy[s] = 0;
  }
  c->inner_total = 0;
  return ORA_OK;
}

/* ---- walls ---------------------------------------------------------------- */

/* Which side a wall node belongs to (corners go to the vertical wall), and its
 * inward fluid neighbour for the extrapolation. */
static int wall_side(const ora_ctx* c, int x, int y) {
  if (c->p.bc[ORA_SIDE_LEFT] != ORA_BC_PERIODIC && x == 0) return ORA_SIDE_LEFT;
  if (c->p.bc[ORA_SIDE_RIGHT] != ORA_BC_PERIODIC && x == c->nx - 1) return ORA_SIDE_RIGHT;
  if (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC && y == 0) return ORA_SIDE_BOTTOM;
  return ORA_SIDE_TOP;
}

static int is_corner(const ora_ctx* c, int x, int y) {
  int vx = (c->p.bc[ORA_SIDE_LEFT] != ORA_BC_PERIODIC) && (x == 0 || x == c->nx - 1);
  int vy = (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC) && (y == 0 || y == c->ny - 1);
  return vx && vy;
}

/* Inward neighbour of a wall node: the normal neighbour for side nodes, the
 * diagonal neighbour for corners. */
static int inward(const ora_ctx* c, int x, int y) {
  if (is_corner(c, x, y)) {
    int xx = (x == 0) ? 1 : c->nx - 2;
    int yy = (y == 0) ? 1 : c->ny - 2;
    return idx(c, xx, yy);
  }
  switch (wall_side(c, x, y)) {
    case ORA_SIDE_LEFT: return idx(c, 1, y);
    case ORA_SIDE_RIGHT: return idx(c, c->nx - 2, y);
    case ORA_SIDE_BOTTOM: return idx(c, x, 1);
    default: return idx(c, x, c->ny - 2);
  }
}

static double sum5(const double* g, int n, int s) {
  double t = 0;
  for (int i = 0; i < 5; ++i) t += g[i * n + s];
  return t;
}

/* Wall temperature imposed at wall node (x,y), given T of its inward neighbour.
 * A corner takes the vertical wall's condition; if that wall is adiabatic it
 * takes the horizontal wall's Dirichlet value if there is one. */
static double wall_temperature(const ora_ctx* c, int x, int y, double Tf) {
  int side = wall_side(c, x, y);
  int bc = c->p.bc[side];
  if (bc == ORA_BC_DIRICHLET)
    return (side == ORA_SIDE_LEFT) ? c->wallTl[y] : c->p.T_bc[side];
  if (is_corner(c, x, y)) {
    int hs = (y == 0) ? ORA_SIDE_BOTTOM : ORA_SIDE_TOP;
    if (c->p.bc[hs] == ORA_BC_DIRICHLET) return c->p.T_bc[hs];
  }
  return Tf; /* adiabatic: zero normal gradient */
}

/* ---- one time step -------------------------------------------------------- */

static void flow_step(ora_ctx* c) {
  const int n = c->n, nx = c->nx, ny = c->ny;
  /* active: 1 flow node, 2 extrapolated wall node (flow_walls = 1), 0 none */
  for (int s = 0; s < n; ++s) c->active[s] = (!c->wall[s] && c->fl[s] >= c->p.f_act);
  if (c->p.flow_walls == 1)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int s = idx(c, x, y);
        if (c->wall[s] && c->active[inward(c, x, y)] == 1) c->active[s] = 2;
      }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      int s = idx(c, x, y);
      double fin[9], fout[9];
      for (int i = 0; i < 9; ++i) fin[i] = c->f[i * n + s];
      if (c->active[s] == 1) {
        collide_flow(c, fin, c->T[s], c->fl[s], c->phi[s], c->K[s], fout, &c->ux[s], &c->uy[s]);
        if (c->p.flow_front == 1) {
          /* the boundary state a non-flow neighbour extrapolates from this node */
          double rho, ufx, ufy, Fx, Fy, eqw[9], eqf[9], fb[9], fe[9], tx, ty;
          macro_flow(c, fin, c->T[s], c->fl[s], c->phi[s], c->K[s], &rho, &ufx, &ufy, &Fx, &Fy);
          const double vphi = c->phi[s] * c->fl[s];
          ora_feq(c, rho, 0, 0, vphi, eqw);
          ora_feq(c, rho, ufx, ufy, vphi, eqf);
          for (int i = 0; i < 9; ++i) fb[i] = eqw[i] + fin[i] - eqf[i];
          collide_flow(c, fb, c->T[s], c->fl[s], c->phi[s], c->K[s], fe, &tx, &ty);
          for (int i = 0; i < 9; ++i) c->fext[i * n + s] = fe[i];
        }
      } else if (c->active[s] == 2) {
        /* Sec. 4: equilibrium at the wall velocity (0) with the fluid node's
         * density plus the fluid node's non-equilibrium part */
        const int sf = inward(c, x, y);
        double ff[9], rho, ufx, ufy, Fx, Fy, eqw[9], eqf[9], tx, ty;
        for (int i = 0; i < 9; ++i) ff[i] = c->f[i * n + sf];
        macro_flow(c, ff, c->T[sf], c->fl[sf], c->phi[sf], c->K[sf], &rho, &ufx, &ufy, &Fx, &Fy);
        const double vphi = c->phi[sf] * c->fl[sf];
        ora_feq(c, rho, 0, 0, vphi, eqw);
        ora_feq(c, rho, ufx, ufy, vphi, eqf);
        for (int i = 0; i < 9; ++i) fin[i] = eqw[i] + ff[i] - eqf[i];
        collide_flow(c, fin, c->T[sf], c->fl[sf], c->phi[sf], c->K[sf], fout, &tx, &ty);
        c->ux[s] = c->uy[s] = 0;
      } else {
        for (int i = 0; i < 9; ++i) fout[i] = fin[i];
        c->ux[s] = c->uy[s] = 0;
      }
      for (int i = 0; i < 9; ++i) c->fpost[i * n + s] = fout[i];
    }
  }
  /* streaming, Eq. (21), with halfway bounce-back on links into non-flow nodes
   * (extrapolated wall nodes stream like flow nodes; what they would receive
   * from outside the lattice is reflected, and replaced before it is used) */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      int s = idx(c, x, y);
      if (!c->active[s]) {
        for (int i = 0; i < 9; ++i) c->fnew[i * n + s] = c->f[i * n + s];
        continue;
      }
      for (int i = 0; i < 9; ++i) {
        /* population i arriving at s comes from s - e_i, or is s's own
         * population in the opposite direction reflected at the link */
        int src = neighbour(c, x, y, -EX9[i], -EY9[i]);
        if (src >= 0 && c->active[src])
          c->fnew[i * n + s] = c->fpost[i * n + src];
        else if (c->p.flow_front == 1 && c->active[s] == 1 && src >= 0 && !c->wall[src])
          c->fnew[i * n + s] = c->fext[i * n + s];   /* from the front's boundary node */
        else
          c->fnew[i * n + s] = c->fpost[OPP9[i] * n + s];
      }
    }
  }
  double* t = c->f;
  c->f = c->fnew;
  c->fnew = t;
}

/* non-equilibrium extrapolation on wall nodes (before collision), into gpre */
static void thermal_walls(ora_ctx* c) {
  const int n = c->n, nx = c->nx, ny = c->ny;
  for (int pass = 0; pass < 2; ++pass) { /* side nodes first, then corners */
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int s = idx(c, x, y);
        if (!c->wall[s] || is_corner(c, x, y) != pass) continue;
        int sf = inward(c, x, y);
        double Tf = sum5(c->gpre, n, sf);
        double Tw = wall_temperature(c, x, y, Tf);
        double eqw[5], eqf[5];
        const double sig = sigma_of(c, c->fl[sf]);
        geq_s(c, Tw, 0, 0, sig, eqw);
        geq_s(c, Tf, c->ux[sf], c->uy[sf], sig, eqf);
        for (int i = 0; i < 5; ++i) c->gpre[i * n + s] = eqw[i] + c->gpre[i * n + sf] - eqf[i];
      }
  }
}

/* collide every node with source S~_0 = src[s] (NULL: none), stream into out */
static void thermal_collide_stream(ora_ctx* c, const double* src, double* out) {
  const int n = c->n, nx = c->nx, ny = c->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int s = idx(c, x, y);
      double gin[5], gout[5];
      for (int i = 0; i < 5; ++i) gin[i] = c->gpre[i * n + s];
      double ux = c->wall[s] ? 0 : c->ux[s];
      double uy = c->wall[s] ? 0 : c->uy[s];
      double s0 = (src && !c->wall[s]) ? src[s] : 0;
      /* tau_T from f_l(n); a wall node, whose populations the extrapolation
       * took from its inward neighbour, relaxes at that neighbour's rate */
      const double flt = c->wall[s] ? c->fl[inward(c, x, y)] : c->fl[s];
      collide_thermal(c, gin, ux, uy, s0, ora_theta_T(c, flt), sigma_of(c, flt), gout);
      for (int i = 0; i < 5; ++i) c->gpost[i * n + s] = gout[i];
    }
  /* streaming, Eq. (36); populations leaving the domain are dropped and the
   * slots of wall nodes that nothing streams into are set to zero (the
   * extrapolation rewrites wall nodes before they are used) */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int s = idx(c, x, y);
      for (int i = 0; i < 5; ++i) {
        int srcn = neighbour(c, x, y, -EX5[i], -EY5[i]);
        out[i * n + s] = (srcn >= 0) ? c->gpost[i * n + srcn] : 0.0;
      }
    }
}

static int thermal_step(ora_ctx* c, int literal) {
  const int n = c->n, nx = c->nx, ny = c->ny;
  if (c->sigma_var) /* a = phi dT / (sigma(f_l(n)) St) for this step, Eq. (38) */
    for (int s = 0; s < n; ++s)
      c->a[s] = c->phi[s] * c->p.dT / (sigma_of(c, c->fl[s]) * c->p.St);
  memcpy(c->gpre, c->g, sizeof(double) * 5 * (size_t)n);
  thermal_walls(c);
  /* source-free collision and streaming */
  thermal_collide_stream(c, NULL, c->gstar);

  /* iterative enthalpy method, Sec. 3.2: f^(0) = f_l(n); with f^(k) build
   * S~_0 = -a (f^(k) - f_l(n)), get T^(k) = sum g after collision with the
   * source and streaming, h^(k) = T^(k) + a f^(k),
   * f^(k+1) = clamp((h^(k) - T_s) / (T_l - T_s + a), 0, 1). */
  const double Ts = c->p.T_s, dTt = c->p.T_l - c->p.T_s;
  double* src = c->Tk;  /* per-node S~_0 */
  double* Tk = c->fk1;  /* T^(k) */
  double* fk = c->fk;   /* f^(k) */
  double* fnext = (double*)malloc(sizeof(double) * (size_t)n);
  if (!fnext) return ORA_ERR_OOM;
  memcpy(fk, c->fl, sizeof(double) * (size_t)n);
  int rc = ORA_OK, converged = 0;
  for (int k = 0; k < c->p.max_inner_iters; ++k) {
    for (int s = 0; s < n; ++s) src[s] = c->wall[s] ? 0.0 : -c->a[s] * (fk[s] - c->fl[s]);
    if (literal) {
      thermal_collide_stream(c, src, c->gtmp);
      for (int s = 0; s < n; ++s) Tk[s] = sum5(c->gtmp, n, s);
    } else {
      /* N^-1 S~ = S~_0 (w~_0, ..., w~_4), streamed like any population */
#pragma omp parallel for schedule(static)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int s = idx(c, x, y);
          double t = 0;
          for (int i = 0; i < 5; ++i) {
            int srcn = neighbour(c, x, y, -EX5[i], -EY5[i]);
            t += c->gstar[i * n + s];
            if (srcn >= 0) t += c->wt[i] * src[srcn];
          }
          Tk[s] = t;
        }
    }
    double diff = 0;
#pragma omp parallel for schedule(static) reduction(max : diff)
    for (int s = 0; s < n; ++s) {
      if (c->wall[s]) {
        fnext[s] = c->fl[s];
        continue;
      }
      double h = Tk[s] + c->a[s] * fk[s];
      fnext[s] = clamp01((h - Ts) / (dTt + c->a[s]));
      double d = fabs(fnext[s] - fk[s]);
      if (d > diff) diff = d;
    }
    memcpy(fk, fnext, sizeof(double) * (size_t)n);
    c->inner_total++;
    if (diff <= c->p.inner_tol) {
      converged = 1;
      break;
    }
  }
  if (!converged) rc = ORA_ERR_NOT_CONVERGED;
  /* final thermal populations with the source of f_l(n+1) = fk */
  for (int s = 0; s < n; ++s) src[s] = c->wall[s] ? 0.0 : -c->a[s] * (fk[s] - c->fl[s]);
  if (literal) {
    thermal_collide_stream(c, src, c->g);
  } else {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int s = idx(c, x, y);
        for (int i = 0; i < 5; ++i) {
          int srcn = neighbour(c, x, y, -EX5[i], -EY5[i]);
          double v = c->gstar[i * n + s];
          if (srcn >= 0) v += c->wt[i] * src[srcn];
          c->g[i * n + s] = v;
        }
      }
  }
  memcpy(c->fl, fk, sizeof(double) * (size_t)n);
  free(fnext);
  return rc;
}

int ora_step(ora_ctx* c, int64_t nsteps, int literal) {
  if (!c || nsteps < 0) return ORA_ERR_INVALID_ARG;
  int rc = ORA_OK;
  for (int64_t t = 0; t < nsteps; ++t) {
    for (int s = 0; s < c->n; ++s) c->T[s] = sum5(c->g, c->n, s);
    if (c->p.flow) {
      flow_step(c);
    } else {
      for (int s = 0; s < c->n; ++s) c->ux[s] = c->uy[s] = 0;
    }
    int r = thermal_step(c, literal);
    if (r == ORA_ERR_OOM) return r;
    if (r && !rc) rc = r;
  }
  return rc;
}

/* ---- outputs -------------------------------------------------------------- */

static double node_T(const ora_ctx* c, int x, int y) {
  int s = idx(c, x, y);
  if (!c->wall[s]) return sum5(c->g, c->n, s);
  int sf = inward(c, x, y);
  return wall_temperature(c, x, y, sum5(c->g, c->n, sf));
}

void ora_get_macros(const ora_ctx* c, double* ux, double* uy, double* rho, double* T, double* fl) {
  const int n = c->n;
  for (int y = 0; y < c->ny; ++y)
    for (int x = 0; x < c->nx; ++x) {
      int s = idx(c, x, y);
      double Tn = node_T(c, x, y);
      double f[9], r = 0;
      for (int i = 0; i < 9; ++i) {
        f[i] = c->f[i * n + s];
        r += f[i];
      }
      double vx = 0, vy = 0;
      if (c->p.flow && !c->wall[s] && c->fl[s] >= c->p.f_act) {
        double o[4];
        ora_velocity(c, f, Tn, c->fl[s], c->phi[s], c->K[s], o);
        vx = o[0];
        vy = o[1];
      }
      if (ux) ux[s] = vx;
      if (uy) uy[s] = vy;
      if (rho) rho[s] = r;
      if (T) T[s] = Tn;
      if (fl) fl[s] = c->fl[s];
    }
}

void ora_reduce(const ora_ctx* c, double out[4]) {
  const int n = c->n;
  double mass = 0, ent = 0, melt = 0;
  long cnt = 0;
  for (int s = 0; s < n; ++s) {
    if (c->wall[s]) continue;
    double T = sum5(c->g, n, s);
    for (int i = 0; i < 9; ++i) mass += c->f[i * n + s];
    const double a = c->sigma_var ? c->phi[s] * c->p.dT / (sigma_of(c, c->fl[s]) * c->p.St)
                                  : c->a[s];
    ent += T + a * c->fl[s];
    melt += c->fl[s];
    cnt++;
  }
  /* Nusselt number on the left wall: -H dT/dx / dT with the second-order
   * one-sided difference (-3 T0 + 4 T1 - T2) / 2, averaged over wall rows */
  double nu = 0;
  int rows = 0;
  if (c->p.bc[ORA_SIDE_LEFT] != ORA_BC_PERIODIC && c->nx >= 3) {
    int y0 = (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC) ? 1 : 0;
    int y1 = (c->p.bc[ORA_SIDE_BOTTOM] != ORA_BC_PERIODIC) ? c->ny - 1 : c->ny;
    for (int y = y0; y < y1; ++y) {
      double T0 = node_T(c, 0, y), T1 = node_T(c, 1, y), T2 = node_T(c, 2, y);
      nu += -(-3 * T0 + 4 * T1 - T2) / 2 * c->p.H / c->p.dT;
      rows++;
    }
  }
  out[0] = mass;
  out[1] = ent;
  out[2] = cnt ? melt / cnt : 0;
  out[3] = rows ? nu / rows : 0;
}

void ora_get_state(const ora_ctx* c, double* f, double* g, double* fl) {
  size_t n = (size_t)c->n;
  if (f) memcpy(f, c->f, sizeof(double) * 9 * n);
  if (g) memcpy(g, c->g, sizeof(double) * 5 * n);
  if (fl) memcpy(fl, c->fl, sizeof(double) * n);
}

void ora_set_state(ora_ctx* c, const double* f, const double* g, const double* fl) {
  size_t n = (size_t)c->n;
  if (f) memcpy(c->f, f, sizeof(double) * 9 * n);
  if (g) memcpy(c->g, g, sizeof(double) * 5 * n);
  if (fl) memcpy(c->fl, fl, sizeof(double) * n);
}
