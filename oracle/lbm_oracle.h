/*
 * FP64 CPU oracle for the double-MRT lattice Boltzmann model of solid-liquid
 * phase change in porous media (Liu & He, arXiv:1503.08406).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lbm_oracle.c are the plain,
 * slow reference that the CUDA path is checked against.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
 * load it.  It shares no code, header, table or constant with the CUDA
 * library in paper_1503_08406_gb300/csrc, and it does not include
 * include/lbm.h.
 *
 * Everything is double precision, two full population buffers per lattice
 * ("collide into a scratch copy, then stream"), and the latent-heat source
 * is applied inside the thermal collision exactly as Eq. (35) writes it.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BC_PERIODIC = 0, ORA_BC_DIRICHLET = 1, ORA_BC_ADIABATIC = 2 };
enum { ORA_SIDE_LEFT = 0, ORA_SIDE_RIGHT = 1, ORA_SIDE_BOTTOM = 2, ORA_SIDE_TOP = 3 };
enum {
  ORA_OK = 0,
  ORA_ERR_INVALID_ARG = -1,
  ORA_ERR_OOM = -2,
  ORA_ERR_NOT_CONVERGED = -3
};

/* Inputs.  Dimensionless groups follow Eq. (9); a negative tau_nu, tau_T or
 * g_beta asks the oracle to derive it from (Ra, Pr, Ma, J, lambda, sigma)
 * with the relations of Sec. 4.3; zero relaxation rates take the Sec. 4
 * values (s_e = s_eps = 1.1, s_q = 1.2, zeta_e = zeta_nu = 1.5). */
typedef struct {
  int32_t nx, ny;
  int32_t bc[4];        /* left, right, bottom, top: ORA_BC_* */
  double  T_bc[4];      /* Dirichlet wall temperatures, same order */
  int32_t flow;         /* 1: D2Q9 flow lattice on (vartheta = 1); 0: conduction (vartheta = 0) */
  double  Ra, Pr, Ma, J, lambda_, sigma, St, dT, H;
  double  T_ref;        /* T_0 of Eq. (5) */
  double  T_s, T_l;     /* solidus / liquidus of Eq. (41)-(42); equal = isothermal */
  double  varpi;        /* D2Q5 parameter of Eq. (34) */
  double  rho0;
  double  tau_nu, tau_T, g_beta;
  double  s_e, s_eps, s_q, zeta_e, zeta_nu;
  double  f_act;        /* liquid fraction at and above which a cell carries flow */
  int32_t max_inner_iters;
  double  inner_tol;
  double  alpha_ratio;  /* alpha_l / alpha_s (Sec. 4.1); 0 or 1: one diffusivity */
  double  sigma_solid;  /* sigma at f_l = 0, Eq. (7) (sigma above is its value at
                           f_l = 1); 0: sigma everywhere */
  int32_t flow_walls;   /* 0: halfway bounce-back on links into wall nodes;
                           1: non-equilibrium extrapolation on wall nodes (Sec. 4) */
  int32_t flow_front;   /* 0: halfway bounce-back on links into non-flow lattice nodes;
                           1: non-equilibrium extrapolation at the moving solid-liquid
                           interface (Sec. 4), from the flow node of each link */
} ora_params;

typedef struct ora_ctx ora_ctx;

/* Relaxation rate zeta_alpha = 1/tau_T of a node with liquid fraction fl (Sec. 4.1):
 * alpha_e = alpha_l fl + alpha_s (1 - fl), tau_T = 1/2 + alpha_e / (sigma c_sT^2),
 * sigma = sigma(fl) of Eq. (7) when sigma_solid is set. */
double ora_theta_T(const ora_ctx* c, double fl);

int  ora_create(const ora_params* p, ora_ctx** out);
void ora_destroy(ora_ctx* c);
void ora_set_threads(int n);

/* Derived lattice quantities, in this order:
 * tau_nu, tau_T, nu_e, nu_l, alpha_e, g_beta, csT2, latent coefficient dT/(sigma St). */
void ora_get_derived(const ora_ctx* c, double out[8]);

/* Row-major [ny][nx] arrays.  wall_T_left (ny values) may be NULL; when given it
 * replaces T_bc[LEFT] row by row on a Dirichlet left wall.  Populations start at
 * the rest equilibria: f = f^eq(rho0, 0) (Eq. 29), g = g^eq(T0, 0) (Eq. 39). */
int  ora_set_fields(ora_ctx* c, const double* phi, const double* K, const double* T0,
                    const double* fl0, const double* wall_T_left);

/* Advance nsteps.  literal = 1 re-runs the thermal collision and streaming for
 * every inner iteration; literal = 0 adds the streamed source to the source-free
 * post-stream field (the same numbers, by linearity of Eq. (35)-(36) in S~).
 * Returns ORA_ERR_NOT_CONVERGED when an inner iteration hit its cap (the step is
 * still completed with the last iterate). */
int  ora_step(ora_ctx* c, int64_t nsteps, int literal);
int64_t ora_inner_iterations(const ora_ctx* c);   /* total inner iterations so far */

/* Macroscopic fields at the current time: u from Eq. (26)-(28), rho from (24),
 * T from (33) (walls: the wall value the extrapolation imposes), f_l. */
void ora_get_macros(const ora_ctx* c, double* ux, double* uy, double* rho, double* T, double* fl);

/* mass = sum f over non-wall nodes, enthalpy = sum (T + a f_l) over non-wall
 * nodes, melt = mean f_l over non-wall nodes, nu_hot = mean left-wall Nusselt number. */
void ora_reduce(const ora_ctx* c, double out[4]);

/* Raw state in natural layout: f[9][ny][nx], g[5][ny][nx], fl[ny][nx]. */
void ora_get_state(const ora_ctx* c, double* f, double* g, double* fl);
void ora_set_state(ora_ctx* c, const double* f, const double* g, const double* fl);

/* Single-node pieces, exposed so tests can check them against the paper's identities. */
void ora_matrices(double M[81], double Minv[81], double N[25], double Ninv[25]);
void ora_feq(const ora_ctx* c, double rho, double ux, double uy, double varphi, double out[9]);
void ora_meq(const ora_ctx* c, double rho, double ux, double uy, double varphi, double out[9]);
void ora_force_moments(const ora_ctx* c, double ux, double uy, double Fx, double Fy,
                       double varphi, double out[9]);
void ora_geq(const ora_ctx* c, double T, double ux, double uy, double out[5]);
void ora_thermal_meq(const ora_ctx* c, double T, double ux, double uy, double out[5]);
/* velocity solve and total force at one node: out = (ux, uy, Fx, Fy) */
void ora_velocity(const ora_ctx* c, const double f[9], double T, double fl, double phi,
                  double K, double out[4]);
/* one flow collision at one node (no streaming) */
void ora_collide_flow(const ora_ctx* c, const double f[9], double T, double fl, double phi,
                      double K, double fpost[9]);
/* one thermal collision at one node with source S~_0 = src0 (no streaming) */
void ora_collide_thermal(const ora_ctx* c, const double g[5], double ux, double uy,
                         double src0, double gpost[5]);

#ifdef __cplusplus
}
#endif
#endif
