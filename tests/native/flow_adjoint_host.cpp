// Host build of the flow collision's adjoint (float64) for the CPU tests:
// the same header the reverse-sweep kernels include.
#include "lbm_flow_adjoint.cuh"

namespace {
lbm::FlowNode<double> node_params(const double* p) {
  lbm::FlowNode<double> n;
  n.rho0 = p[0];
  n.nu_l = p[1];
  n.g_beta = p[2];
  n.T_ref = p[3];
  for (int k = 0; k < 9; ++k) n.lam[k] = p[4 + k];
  n.eps = p[13];
  return n;
}
}  // namespace

// prm: rho0, nu_l, g_beta, T_ref, lam[9], eps; per node: f[9], T, fl, phi, K
extern "C" void flow_collide_f64(const double* prm, int count, const double* f, const double* T,
                                 const double* fl, const double* phi, const double* K,
                                 double* fpost, double* ux, double* uy) {
  const lbm::FlowNode<double> p = node_params(prm);
  for (int s = 0; s < count; ++s)
    lbm::flow_node_collide(p, f + 9 * s, T[s], fl[s], phi[s], K[s], fpost + 9 * s, ux + s, uy + s);
}

// lf[9], lux, luy per node in; lfin[9], lT, lfl, lphi, lK per node out
extern "C" void flow_adjoint_f64(const double* prm, int count, const double* f, const double* T,
                                 const double* fl, const double* phi, const double* K,
                                 const double* lf, const double* lux, const double* luy,
                                 double* lfin, double* lT, double* lfl, double* lphi,
                                 double* lK) {
  const lbm::FlowNode<double> p = node_params(prm);
  for (int s = 0; s < count; ++s)
    lbm::flow_node_adjoint(p, f + 9 * s, T[s], fl[s], phi[s], K[s], lf + 9 * s, lux[s], luy[s],
                           lfin + 9 * s, lT + s, lfl + s, lphi + s, lK + s);
}

namespace {
lbm::ThermalNode<double> thermal_params(const double* p) {
  lbm::ThermalNode<double> t;
  t.sigma = p[0];
  t.csT2 = p[1];
  t.varpi = p[2];
  for (int k = 0; k < 5; ++k) t.theta[k] = p[3 + k];
  t.w0 = p[8];
  t.w1 = p[9];
  return t;
}
}  // namespace

// prm: sigma, csT2, varpi, theta[5], w0, w1; per node g[5], ux, uy, lg[5]
extern "C" void thermal_collide_f64(const double* prm, int count, const double* g,
                                    const double* ux, const double* uy, double* gpost) {
  const lbm::ThermalNode<double> p = thermal_params(prm);
  for (int s = 0; s < count; ++s) lbm::thermal_node_collide(p, g + 5 * s, ux[s], uy[s], gpost + 5 * s);
}

extern "C" void thermal_adjoint_f64(const double* prm, int count, const double* g,
                                    const double* ux, const double* uy, const double* lg,
                                    double* lgin, double* lux, double* luy) {
  const lbm::ThermalNode<double> p = thermal_params(prm);
  for (int s = 0; s < count; ++s)
    lbm::thermal_node_adjoint(p, g + 5 * s, ux[s], uy[s], lg + 5 * s, lgin + 5 * s, lux + s,
                              luy + s);
}

// per node gf[5], uxf, uyf, lgb[5]; out lgf[5] (zeroed here), lTw, luxf, luyf
extern "C" void wall_adjoint_f64(const double* prm, int count, const double* gf,
                                 const double* uxf, const double* uyf, const double* lgb,
                                 double* lgf, double* lTw, double* luxf, double* luyf) {
  const lbm::ThermalNode<double> p = thermal_params(prm);
  for (int s = 0; s < count; ++s) {
    for (int i = 0; i < 5; ++i) lgf[5 * s + i] = 0;
    lbm::wall_extrapolation_adjoint(p, gf + 5 * s, uxf[s], uyf[s], lgb + 5 * s, lgf + 5 * s,
                                    lTw + s, luxf + s, luyf + s);
  }
}
