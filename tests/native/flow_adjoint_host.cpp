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
