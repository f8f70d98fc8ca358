// Host emulation, in float64, of one reversed coupled step: the fixed point's
// adjoint on the band (a plain Jacobi solve, as the band kernel does it), then
// lbm::coupled_reverse_node over every node, the body the reverse-sweep kernel
// runs with one node per thread.  Test infrastructure: the CPU tests check it
// against autograd of the FP64 reference over several steps.
#include <math.h>
#include <string.h>

#include <vector>

#include "lbm_flow_adjoint.cuh"

// prm layout: flowprm[14] (rho0, nu_l, g_beta, T_ref, lam[9], eps), thprm[10]
// (sigma, csT2, varpi, theta[5], w0, w1), sc[4] = (f_act, T_s, T_l, lat),
// nuprm[8] = (nu_g1, nu_g2, nu_tw, ny0, ny1, tau_T,l (0: one diffusivity),
// alpha_s / alpha_l, flow lattice on).  State of the step: f0 [9][n],
// g0 [5][n], fl0, fl1 (f_l before / after).  Adjoints after the step in lf,
// lg, lfl (overwritten with those before it); lphi, lK and lTw accumulate.
// Returns the number of Jacobi sweeps.
extern "C" int coupled_reverse_step_f64(int nx, int ny, int per_x, int per_y, const int* bc,
                                        const double* flowprm, const double* thprm,
                                        const double* sc, const double* nuprm, const double* f0,
                                        const double* g0, const double* fl0, const double* fl1,
                                        const double* phi, const double* K, double* lf,
                                        double* lg, double* lfl, double* lphi, double* lK,
                                        double* lTw) {
  lbm::CoupledStep<double> A;
  A.geo = lbm::CoupledGeo{nx, ny, per_x, per_y, {bc[0], bc[1], bc[2], bc[3]}};
  const int n = nx * ny;
  A.n = n;
  A.fp.rho0 = flowprm[0];
  A.fp.nu_l = flowprm[1];
  A.fp.g_beta = flowprm[2];
  A.fp.T_ref = flowprm[3];
  for (int k = 0; k < 9; ++k) A.fp.lam[k] = flowprm[4 + k];
  A.fp.eps = flowprm[13];
  A.tp.sigma = thprm[0];
  A.tp.csT2 = thprm[1];
  A.tp.varpi = thprm[2];
  for (int k = 0; k < 5; ++k) A.tp.theta[k] = thprm[3 + k];
  A.tp.w0 = thprm[8];
  A.tp.w1 = thprm[9];
  A.f_act = sc[0];
  A.T_s = sc[1];
  A.T_l = sc[2];
  A.lat = sc[3];
  A.nu_g1 = nuprm[0];
  A.nu_g2 = nuprm[1];
  A.nu_tw = nuprm[2];
  A.ny0 = (int)nuprm[3];
  A.ny1 = (int)nuprm[4];
  A.alpha_var = nuprm[5] > 0;   // alpha_l / alpha_s != 1: nuprm[5] = tau_T,l, nuprm[6] = alpha_s/alpha_l
  A.tauT_l = nuprm[5];
  A.inv_aratio = nuprm[6];
  A.flow = nuprm[7] != 0;
  const double dTt = A.T_l - A.T_s, w0 = A.tp.w0, w1 = A.tp.w1;
  const int ex[5] = {0, 1, 0, -1, 0};
  const int ey[5] = {0, 0, 1, 0, -1};

  // the fixed point's adjoint on the band (0 < f_l(n+1) < 1, not a wall)
  std::vector<double> a(n), rhs(n, 0.0), mu(n, 0.0), mo(n, 0.0);
  std::vector<char> band(n);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      a[s] = phi[s] * A.lat;
      band[s] = !A.geo.wall(x, y) && lbm::adj_mushy(fl1[s]);
      if (!band[s]) continue;
      double L = 0;
      for (int i = 0; i < 5; ++i) {
        const int t = A.geo.nb(x, y, ex[i], ey[i]);
        if (t >= 0) L += (i == 0 ? w0 : w1) * lg[i * n + t];
      }
      rhs[s] = (lfl[s] - a[s] * L) / (1 - a[s] * (1 - w0) / (dTt + a[s]));
    }
  int sweeps = 0;
  for (; sweeps < 10000; ++sweeps) {
    double moved = 0;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int s = y * nx + x;
        if (!band[s]) continue;
        double nbs = 0;
        for (int i = 1; i < 5; ++i) {
          const int t = A.geo.nb(x, y, ex[i], ey[i]);
          if (t >= 0 && band[t]) nbs += mu[t] / (dTt + a[t]);
        }
        const double v = rhs[s] - a[s] * w1 / (1 - a[s] * (1 - w0) / (dTt + a[s])) * nbs;
        moved = fmax(moved, fabs(v - mu[s]) / fmax(fabs(v), 1e-300));
        mo[s] = v;
      }
    mu.swap(mo);
    if (moved < 1e-15) break;
  }
  std::vector<double> lg1(lg, lg + 5 * n);
  for (int s = 0; s < n; ++s)
    if (band[s])
      for (int i = 0; i < 5; ++i) lg1[i * n + s] += mu[s] / (dTt + a[s]);

  std::vector<double> lf0(9 * n), lg0(5 * n);
  std::vector<int> list(n);
  int count = 0;
  A.f0 = f0;
  for (int i = 0; i < 9; ++i) A.foff[i] = 0;
  A.g0 = g0;
  A.fl0 = fl0;
  A.fl1 = fl1;
  A.phi = phi;
  A.K = K;
  A.lf1 = lf;
  A.lg1 = lg1.data();
  A.lf0 = lf0.data();
  A.lg0 = lg0.data();
  A.lfl = lfl;
  A.lphi = lphi;
  A.lK = lK;
  A.lTw = lTw;
  A.next_list = list.data();
  A.next_count = &count;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) lbm::coupled_reverse_node(A, x, y);
  memcpy(lf, lf0.data(), sizeof(double) * 9 * n);
  memcpy(lg, lg0.data(), sizeof(double) * 5 * n);
  return sweeps;
}
