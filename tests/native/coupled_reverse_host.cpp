// Host emulation, in float64, of one reversed coupled step built from the node
// functions of lbm_flow_adjoint.cuh: each loop below is the body of a kernel
// (one node per thread, gathering from its neighbours) of the reverse sweep
// of the flow lattice.  Test infrastructure: the CPU tests check it against
// autograd of the FP64 reference over several steps.
#include <math.h>
#include <string.h>

#include <vector>

#include "lbm_flow_adjoint.cuh"

namespace {

const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
const int EX5[5] = {0, 1, 0, -1, 0};
const int EY5[5] = {0, 0, 1, 0, -1};

struct Geo {
  int nx, ny, n, per_x, per_y;
  int bc[4];
  int nb(int x, int y, int dx, int dy) const {
    int xx = x + dx, yy = y + dy;
    if (xx < 0 || xx >= nx) {
      if (!per_x) return -1;
      xx = (xx + nx) % nx;
    }
    if (yy < 0 || yy >= ny) {
      if (!per_y) return -1;
      yy = (yy + ny) % ny;
    }
    return yy * nx + xx;
  }
  bool vx(int x) const { return !per_x && (x == 0 || x == nx - 1); }
  bool vy(int y) const { return !per_y && (y == 0 || y == ny - 1); }
  bool wall(int x, int y) const { return vx(x) || vy(y); }
  int inward(int x, int y) const {   // the diagonal node at corners
    const bool cx = vx(x), cy = vy(y);
    const int xx = cx ? (x == 0 ? 1 : nx - 2) : x;
    const int yy = cy ? (y == 0 ? 1 : ny - 2) : y;
    return yy * nx + xx;
  }
  // 0 left, 1 right, 2 bottom, 3 top (corners go to the vertical wall)
  int side(int x, int y) const {
    if (vx(x)) return x == 0 ? 0 : 1;
    return y == 0 ? 2 : 3;
  }
};

}  // namespace

// prm layout: flowprm[14] (rho0, nu_l, g_beta, T_ref, lam[9], eps), thprm[10]
// (sigma, csT2, varpi, theta[5], w0, w1), sc[4] = (f_act, T_s, T_l, lat).
// State of the step: f0 [9][n], g0 [5][n], fl0, fl1 (f_l before / after).
// Adjoints after the step in lf, lg, lfl (overwritten with those before it);
// lphi, lK and lTw accumulate.  Returns the number of Jacobi sweeps.
extern "C" int coupled_reverse_step_f64(int nx, int ny, int per_x, int per_y, const int* bc,
                                        const double* flowprm, const double* thprm,
                                        const double* sc, const double* f0, const double* g0,
                                        const double* fl0, const double* fl1, const double* phi,
                                        const double* K, double* lf, double* lg, double* lfl,
                                        double* lphi, double* lK, double* lTw) {
  Geo G{nx, ny, nx * ny, per_x, per_y, {bc[0], bc[1], bc[2], bc[3]}};
  const int n = G.n;
  lbm::FlowNode<double> fp;
  fp.rho0 = flowprm[0];
  fp.nu_l = flowprm[1];
  fp.g_beta = flowprm[2];
  fp.T_ref = flowprm[3];
  for (int k = 0; k < 9; ++k) fp.lam[k] = flowprm[4 + k];
  fp.eps = flowprm[13];
  lbm::ThermalNode<double> tp;
  tp.sigma = thprm[0];
  tp.csT2 = thprm[1];
  tp.varpi = thprm[2];
  for (int k = 0; k < 5; ++k) tp.theta[k] = thprm[3 + k];
  tp.w0 = thprm[8];
  tp.w1 = thprm[9];
  const double f_act = sc[0], T_s = sc[1], T_l = sc[2], lat = sc[3];
  const double dTt = T_l - T_s;
  auto wt = [&](int i) { return i == 0 ? tp.w0 : tp.w1; };

  // forward quantities of the step: flow mask, T(n), velocity
  std::vector<char> act(n), wal(n);
  std::vector<double> T(n), ux(n, 0.0), uy(n, 0.0), a(n);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      wal[s] = G.wall(x, y);
      act[s] = !wal[s] && fl0[s] >= f_act;
      double t = 0;
      for (int i = 0; i < 5; ++i) t += g0[i * n + s];
      T[s] = t;
      a[s] = phi[s] * lat;
    }
  for (int s = 0; s < n; ++s) {
    if (!act[s]) continue;
    double f[9], fpost[9];
    for (int i = 0; i < 9; ++i) f[i] = f0[i * n + s];
    lbm::flow_node_collide(fp, f, T[s], fl0[s], phi[s], K[s], fpost, &ux[s], &uy[s]);
  }

  // thermal reverse, 1: the fixed point's adjoint on the band (0 < f_l(n+1) < 1)
  std::vector<double> nu(n, 0.0), rhs(n, 0.0), mu(n, 0.0), mo(n, 0.0);
  std::vector<char> band(n);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      band[s] = !wal[s] && fl1[s] > 0 && fl1[s] < 1;
      if (!band[s]) continue;
      double L = 0;
      for (int i = 0; i < 5; ++i) {
        const int t = G.nb(x, y, EX5[i], EY5[i]);
        if (t >= 0) L += wt(i) * lg[i * n + t];
      }
      const double c = 1.0 / (dTt + a[s]);
      rhs[s] = (lfl[s] - a[s] * L) / (1 - a[s] * (1 - tp.w0) * c);
    }
  int sweeps = 0;
  for (; sweeps < 10000; ++sweeps) {
    double moved = 0;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int s = y * nx + x;
        if (!band[s]) continue;
        const double c = 1.0 / (dTt + a[s]);
        double nbs = 0;
        for (int i = 1; i < 5; ++i) {
          const int t = G.nb(x, y, EX5[i], EY5[i]);
          if (t >= 0 && band[t]) nbs += mu[t] / (dTt + a[t]);
        }
        const double v = rhs[s] - a[s] * tp.w1 / (1 - a[s] * (1 - tp.w0) * c) * nbs;
        moved = fmax(moved, fabs(v - mu[s]) / fmax(fabs(v), 1e-300));
        mo[s] = v;
      }
    mu.swap(mo);
    if (moved < 1e-15) break;
  }
  for (int s = 0; s < n; ++s) nu[s] = band[s] ? mu[s] / (dTt + a[s]) : 0.0;

  // 2: per node, lam_g+ (streamed back, nu included), A(u)^T, the source's
  // adjoint S, f_l(n), a; lam_u from the collision
  std::vector<double> lgpre(5 * n, 0.0), lux(n, 0.0), luy(n, 0.0), lfl0(n), lgn(5 * n, 0.0);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      double lp[5], gin[5], lgin[5], S = 0;
      for (int i = 0; i < 5; ++i) {
        const int t = G.nb(x, y, EX5[i], EY5[i]);
        lp[i] = t >= 0 ? lg[i * n + t] + nu[t] : 0.0;
        S += wt(i) * lp[i];
      }
      // with u = 0 on wall nodes the collision is linear and its transpose does
      // not depend on the populations (the extrapolated ones on walls)
      const double uxc = wal[s] ? 0.0 : ux[s], uyc = wal[s] ? 0.0 : uy[s];
      for (int i = 0; i < 5; ++i) gin[i] = g0[i * n + s];
      double lx = 0, ly = 0;
      lbm::thermal_node_adjoint(tp, gin, uxc, uyc, lp, lgin, &lx, &ly);
      for (int i = 0; i < 5; ++i) lgpre[i * n + s] = lgin[i];
      if (!wal[s]) {
        lux[s] += lx;
        luy[s] += ly;
        lfl0[s] = a[s] * S;
        lphi[s] += -(fl1[s] - fl0[s]) * S * lat;
      } else {
        lfl0[s] = lfl[s];
      }
    }
  // 3: walls: fold the extrapolation's adjoint into the inward nodes
  for (int s = 0; s < n; ++s)
    if (!wal[s])
      for (int i = 0; i < 5; ++i) lgn[i * n + s] = lgpre[i * n + s];
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      if (!wal[s]) continue;
      const int sf = G.inward(x, y);
      double gf[5], lgb[5], lgf[5] = {0, 0, 0, 0, 0}, lTwv, lxf, lyf;
      for (int i = 0; i < 5; ++i) {
        gf[i] = g0[i * n + sf];
        lgb[i] = lgpre[i * n + s];
      }
      lbm::wall_extrapolation_adjoint(tp, gf, ux[sf], uy[sf], lgb, lgf, &lTwv, &lxf, &lyf);
      const int sd = G.side(x, y);
      int cond = G.bc[sd];   // 1 Dirichlet, 2 adiabatic
      bool corner_h = false;
      if (G.vx(x) && G.vy(y) && cond != 1) {
        const int hs = (y == 0) ? 2 : 3;
        if (G.bc[hs] == 1) corner_h = true;
      }
      if (cond == 1) {
        if (sd == 0) lTw[y] += lTwv;
      } else if (!corner_h) {
        for (int i = 0; i < 5; ++i) lgf[i] += lTwv;   // adiabatic: T_w = T_f
      }
      for (int i = 0; i < 5; ++i) lgn[i * n + sf] += lgf[i];
      if (act[sf]) {
        lux[sf] += lxf;
        luy[sf] += lyf;
      }
    }

  // flow reverse: streaming with bounce-back, then the collision's adjoint
  std::vector<double> lfn(9 * n, 0.0);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int s = y * nx + x;
      if (!act[s]) {
        for (int i = 0; i < 9; ++i) lfn[i * n + s] = lf[i * n + s];   // kept populations
        continue;
      }
      double lpost[9], f[9], lfin[9], lT, lflv, lphiv, lKv;
      for (int j = 0; j < 9; ++j) {
        const int t = G.nb(x, y, EX9[j], EY9[j]);
        lpost[j] = (t >= 0 && act[t]) ? lf[j * n + t] : lf[OPP9[j] * n + s];
        f[j] = f0[j * n + s];
      }
      lbm::flow_node_adjoint(fp, f, T[s], fl0[s], phi[s], K[s], lpost, lux[s], luy[s], lfin, &lT,
                             &lflv, &lphiv, &lKv);
      for (int i = 0; i < 9; ++i) lfn[i * n + s] = lfin[i];
      for (int i = 0; i < 5; ++i) lgn[i * n + s] += lT;   // T(n) = sum g(n)
      lfl0[s] += lflv;
      lphi[s] += lphiv;
      lK[s] += lKv;
    }
  memcpy(lf, lfn.data(), sizeof(double) * 9 * n);
  memcpy(lg, lgn.data(), sizeof(double) * 5 * n);
  memcpy(lfl, lfl0.data(), sizeof(double) * n);
  return sweeps;
}
