// Adjoint of the flow collision at one node (Sec. 3.1), written out by hand for
// the reverse sweep of the coupled step: the vector-Jacobian product of the map
// (f, T, f_l, phi, K) -> (f+, u) of
//   rho = sum f, j = sum e f                                   Eq. (24)
//   varphi = phi f_l, G = g beta (T - T_0)                     Eq. (5)
//   K_eff = K f_l^3 ((1 - phi) / (1 - varphi))^2,
//   C_F = 1.75 / sqrt(175 varphi^3)                            Eq. (6), f_l-scaled
//   v = j / rho0 + varphi G e_y / 2                            Eq. (27)
//   l0 = (1 + varphi nu / (2 K_eff)) / 2, l1 = varphi C_F / (2 sqrt(K_eff))   Eq. (28)
//   u = v / (l0 + sqrt(l0^2 + l1 |v|))                        Eq. (26)
//   F = -varphi nu / K_eff u - varphi C_F / sqrt(K_eff) |u| u + varphi G e_y   Eq. (4)
//   m+ = m - Lambda (m - m^eq(rho, u, varphi)) + (I - Lambda/2) S(u, F, varphi),
//   m = M f, f+ = M^-1 m+                                      Eq. (16)-(23)
// Given the adjoints of f+ and of u (the velocity the thermal collision and
// the wall extrapolation use), it returns those of f, T, f_l, phi and K.
// Square roots of speeds carry a floor (FlowNode::eps) so that a node at rest
// has a finite derivative.  M has orthogonal rows: M^-1 = M^T D^-1 with
// D = diag(9, 36, 36, 6, 12, 6, 12, 4, 4).
//
// Header-only and templated on the real type; LBM_HD marks the functions for
// both the host (float64 checks) and the device.
#pragma once

#include <math.h>

#ifndef LBM_HD
#ifdef __CUDACC__
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif
#endif

namespace lbm {

// The reverse sweeps take the clamp of Eq. (42) as open at a node (the node
// mushy, its f_l a function of the step's temperature) where f_l after the
// step lies strictly inside (0, 1); at the bounds the one-sided derivative of
// the clamped side, 0, is taken.
template <typename R>
LBM_HD bool adj_mushy(R f) {
  return f > R(0) && f < R(1);
}

template <typename R>
struct FlowNode {
  R rho0, nu_l, g_beta, T_ref;
  R lam[9];   // diagonal of Lambda, Eq. (23)
  R eps;      // floor under the squared speeds
};

template <typename R>
LBM_HD void mrt_M(const R f[9], R m[9]) {
  const R c = f[5] + f[6] + f[7] + f[8];
  const R a = f[1] + f[2] + f[3] + f[4];
  m[0] = f[0] + a + c;
  m[1] = -4 * f[0] - a + 2 * c;
  m[2] = 4 * f[0] - 2 * a + c;
  m[3] = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  m[4] = -2 * f[1] + 2 * f[3] + f[5] - f[6] - f[7] + f[8];
  m[5] = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  m[6] = -2 * f[2] + 2 * f[4] + f[5] + f[6] - f[7] - f[8];
  m[7] = f[1] - f[2] + f[3] - f[4];
  m[8] = f[5] - f[6] + f[7] - f[8];
}

// out = M^T l
template <typename R>
LBM_HD void mrt_MT(const R l[9], R o[9]) {
  const R e = l[0] - l[1] - 2 * l[2], d = l[0] + 2 * l[1] + l[2];
  o[0] = l[0] - 4 * l[1] + 4 * l[2];
  o[1] = e + l[3] - 2 * l[4] + l[7];
  o[2] = e + l[5] - 2 * l[6] - l[7];
  o[3] = e - l[3] + 2 * l[4] + l[7];
  o[4] = e - l[5] + 2 * l[6] - l[7];
  o[5] = d + l[3] + l[4] + l[5] + l[6] + l[8];
  o[6] = d - l[3] - l[4] + l[5] + l[6] - l[8];
  o[7] = d - l[3] - l[4] - l[5] - l[6] + l[8];
  o[8] = d + l[3] + l[4] - l[5] - l[6] - l[8];
}

template <typename R>
LBM_HD R mrt_D(int k) {
  return k == 0 ? R(9) : (k == 1 || k == 2) ? R(36) : (k == 3 || k == 5) ? R(6)
         : (k == 4 || k == 6) ? R(12) : R(4);
}

// Forward intermediates of one node, kept for the reverse pass.
template <typename R>
struct FlowFwd {
  R rho, jx, jy, vp, G, q, r, Keff, CF, sK, vx, vy, l0, l1, vm, s2, den, ux, uy, um, a1, a2;
  R Fx, Fy, uu, uF;
};

template <typename R>
LBM_HD void flow_node_forward(const FlowNode<R>& p, const R f[9], R T, R fl, R phi, R K,
                              FlowFwd<R>& w) {
  w.rho = 0;
  w.jx = 0;
  w.jy = 0;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int i = 0; i < 9; ++i) {
    w.rho += f[i];
    w.jx += ex[i] * f[i];
    w.jy += ey[i] * f[i];
  }
  w.vp = phi * fl;
  w.G = p.g_beta * (T - p.T_ref);
  w.q = 1 - w.vp;
  w.r = (1 - phi) / w.q;
  w.Keff = K * fl * fl * fl * w.r * w.r;
  w.CF = R(1.75) / sqrt(R(175) * w.vp * w.vp * w.vp);
  w.sK = sqrt(w.Keff);
  w.vx = w.jx / p.rho0;
  w.vy = w.jy / p.rho0 + R(0.5) * w.vp * w.G;
  w.l0 = R(0.5) * (1 + w.vp * R(0.5) * p.nu_l / w.Keff);
  w.l1 = w.vp * R(0.5) * w.CF / w.sK;
  w.vm = sqrt(w.vx * w.vx + w.vy * w.vy + p.eps);
  w.s2 = sqrt(w.l0 * w.l0 + w.l1 * w.vm);
  w.den = w.l0 + w.s2;
  w.ux = w.vx / w.den;
  w.uy = w.vy / w.den;
  w.um = sqrt(w.ux * w.ux + w.uy * w.uy + p.eps);
  w.a1 = w.vp * p.nu_l / w.Keff;
  w.a2 = w.vp * w.CF / w.sK;
  w.Fx = -w.a1 * w.ux - w.a2 * w.um * w.ux;
  w.Fy = -w.a1 * w.uy - w.a2 * w.um * w.uy + w.vp * w.G;
  w.uu = w.ux * w.ux + w.uy * w.uy;
  w.uF = w.ux * w.Fx + w.uy * w.Fy;
}

// m^eq of Eq. (19) and S of Eq. (22) from the intermediates
template <typename R>
LBM_HD void flow_node_meq_S(const FlowNode<R>& p, const FlowFwd<R>& w, R meq[9], R S[9]) {
  const R r0 = p.rho0, vp = w.vp;
  meq[0] = w.rho;
  meq[1] = -2 * w.rho + 3 * r0 * w.uu / vp;
  meq[2] = w.rho - 3 * r0 * w.uu / vp;
  meq[3] = r0 * w.ux;
  meq[4] = -r0 * w.ux;
  meq[5] = r0 * w.uy;
  meq[6] = -r0 * w.uy;
  meq[7] = r0 * (w.ux * w.ux - w.uy * w.uy) / vp;
  meq[8] = r0 * w.ux * w.uy / vp;
  S[0] = 0;
  S[1] = 6 * r0 * w.uF / vp;
  S[2] = -6 * r0 * w.uF / vp;
  S[3] = r0 * w.Fx;
  S[4] = -r0 * w.Fx;
  S[5] = r0 * w.Fy;
  S[6] = -r0 * w.Fy;
  S[7] = 2 * r0 * (w.ux * w.Fx - w.uy * w.Fy) / vp;
  S[8] = r0 * (w.ux * w.Fy + w.uy * w.Fx) / vp;
}

// The collision itself (for checks of the forward map): f+ and u.
template <typename R>
LBM_HD void flow_node_collide(const FlowNode<R>& p, const R f[9], R T, R fl, R phi, R K,
                              R fpost[9], R* ux, R* uy) {
  FlowFwd<R> w;
  flow_node_forward(p, f, T, fl, phi, K, w);
  R m[9], meq[9], S[9], mp[9];
  mrt_M(f, m);
  flow_node_meq_S(p, w, meq, S);
  for (int k = 0; k < 9; ++k)
    mp[k] = (m[k] - p.lam[k] * (m[k] - meq[k]) + (1 - R(0.5) * p.lam[k]) * S[k]) / mrt_D<R>(k);
  mrt_MT(mp, fpost);
  *ux = w.ux;
  *uy = w.uy;
}

// The reverse of flow_node_collide: lf = adjoint of f+, (lux, luy) = adjoint
// of u; out: lfin = adjoint of f, and of T, f_l, phi and K.
template <typename R>
LBM_HD void flow_node_adjoint(const FlowNode<R>& p, const R f[9], R T, R fl, R phi, R K,
                              const R lf[9], R lux, R luy, R lfin[9], R* lT, R* lfl, R* lphi,
                              R* lK) {
  FlowFwd<R> w;
  flow_node_forward(p, f, T, fl, phi, K, w);
  const R r0 = p.rho0, vp = w.vp;
  // f+ = M^T D^-1 m+  ->  lm+ = D^-1 M lf
  R lmp[9];
  mrt_M(lf, lmp);
  for (int k = 0; k < 9; ++k) lmp[k] /= mrt_D<R>(k);
  R lm[9], lmeq[9], lS[9];
  for (int k = 0; k < 9; ++k) {
    lm[k] = (1 - p.lam[k]) * lmp[k];
    lmeq[k] = p.lam[k] * lmp[k];
    lS[k] = (1 - R(0.5) * p.lam[k]) * lmp[k];
  }
  mrt_MT(lm, lfin);   // m = M f
  R lrho = lmeq[0] - 2 * lmeq[1] + lmeq[2];
  R lvp = 0, lFx = 0, lFy = 0, lG = 0;
  // m^eq
  {
    const R W = 3 * r0 * (lmeq[1] - lmeq[2]);   // adjoint of uu / varphi
    lux += W * 2 * w.ux / vp + lmeq[7] * 2 * r0 * w.ux / vp + lmeq[8] * r0 * w.uy / vp +
           r0 * (lmeq[3] - lmeq[4]);
    luy += W * 2 * w.uy / vp - lmeq[7] * 2 * r0 * w.uy / vp + lmeq[8] * r0 * w.ux / vp +
           r0 * (lmeq[5] - lmeq[6]);
    lvp += -(W * w.uu + lmeq[7] * r0 * (w.ux * w.ux - w.uy * w.uy) +
             lmeq[8] * r0 * w.ux * w.uy) / (vp * vp);
  }
  // S
  {
    const R P = 6 * r0 * (lS[1] - lS[2]);   // adjoint of uF / varphi
    const R S7 = 2 * r0 * (w.ux * w.Fx - w.uy * w.Fy) / vp;
    const R S8 = r0 * (w.ux * w.Fy + w.uy * w.Fx) / vp;
    lux += (P * w.Fx + lS[7] * 2 * r0 * w.Fx + lS[8] * r0 * w.Fy) / vp;
    luy += (P * w.Fy - lS[7] * 2 * r0 * w.Fy + lS[8] * r0 * w.Fx) / vp;
    lFx += r0 * (lS[3] - lS[4]) + (P * w.ux + lS[7] * 2 * r0 * w.ux + lS[8] * r0 * w.uy) / vp;
    lFy += r0 * (lS[5] - lS[6]) + (P * w.uy - lS[7] * 2 * r0 * w.uy + lS[8] * r0 * w.ux) / vp;
    lvp += -(P * w.uF / vp + lS[7] * S7 + lS[8] * S8) / vp;
  }
  // F
  R la1, la2, lum;
  {
    const R t = lFx * w.ux + lFy * w.uy;
    la1 = -t;
    la2 = -w.um * t;
    lum = -w.a2 * t;
    lux += lFx * (-w.a1 - w.a2 * w.um);
    luy += lFy * (-w.a1 - w.a2 * w.um);
    lvp += lFy * w.G;
    lG += lFy * vp;
  }
  lux += lum * w.ux / w.um;
  luy += lum * w.uy / w.um;
  R lKeff = 0, lCF = 0, lsK = 0;
  lvp += la1 * p.nu_l / w.Keff;
  lKeff += -la1 * vp * p.nu_l / (w.Keff * w.Keff);
  lvp += la2 * w.CF / w.sK;
  lCF += la2 * vp / w.sK;
  lsK += -la2 * vp * w.CF / (w.sK * w.sK);
  // u = v / den
  R lvx = lux / w.den, lvy = luy / w.den;
  const R lden = -(lux * w.ux + luy * w.uy) / w.den;
  const R ll0 = lden * (1 + w.l0 / w.s2);
  const R ll1 = lden * w.vm / (2 * w.s2);
  const R lvm = lden * w.l1 / (2 * w.s2);
  lvx += lvm * w.vx / w.vm;
  lvy += lvm * w.vy / w.vm;
  // l1, l0
  lvp += ll1 * R(0.5) * w.CF / w.sK;
  lCF += ll1 * R(0.5) * vp / w.sK;
  lsK += -ll1 * R(0.5) * vp * w.CF / (w.sK * w.sK);
  lvp += ll0 * R(0.25) * p.nu_l / w.Keff;
  lKeff += -ll0 * R(0.25) * vp * p.nu_l / (w.Keff * w.Keff);
  // v
  const R ljx = lvx / r0, ljy = lvy / r0;
  lvp += lvy * R(0.5) * w.G;
  lG += lvy * R(0.5) * vp;
  // sqrt(K_eff), C_F, K_eff
  lKeff += lsK / (2 * w.sK);
  lvp += lCF * (R(-1.5) * w.CF / vp);
  *lK = lKeff * w.Keff / K;
  R lflv = lKeff * 3 * w.Keff / fl;
  const R lr = lKeff * 2 * w.Keff / w.r;
  R lphiv = -lr / w.q;
  lvp += lr * w.r / w.q;
  *lT = lG * p.g_beta;
  lphiv += lvp * fl;
  lflv += lvp * phi;
  *lfl = lflv;
  *lphi = lphiv;
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int i = 0; i < 9; ++i) lfin[i] += lrho + ex[i] * ljx + ey[i] * ljy;
}

// ---- the thermal collision and wall extrapolation with the flow's velocity ----
// D2Q5: N of Eq. (32) has orthogonal rows, N^-1 = N^T D5^-1, D5 = diag(5, 2, 2, 20, 4).

template <typename R>
struct ThermalNode {
  R sigma, csT2, varpi;
  R theta[5];   // diagonal of Theta, Eq. (37)
  R w0, w1;     // D2Q5 weights of Eq. (39)
};

template <typename R>
LBM_HD void d2q5_N(const R g[5], R n[5]) {
  n[0] = g[0] + g[1] + g[2] + g[3] + g[4];
  n[1] = g[1] - g[3];
  n[2] = g[2] - g[4];
  n[3] = -4 * g[0] + g[1] + g[2] + g[3] + g[4];
  n[4] = g[1] - g[2] + g[3] - g[4];
}

// out = N^T l
template <typename R>
LBM_HD void d2q5_NT(const R l[5], R o[5]) {
  o[0] = l[0] - 4 * l[3];
  o[1] = l[0] + l[1] + l[3] + l[4];
  o[2] = l[0] + l[2] + l[3] - l[4];
  o[3] = l[0] - l[1] + l[3] + l[4];
  o[4] = l[0] - l[2] + l[3] - l[4];
}

template <typename R>
LBM_HD R d2q5_D(int k) {
  return k == 0 ? R(5) : (k == 1 || k == 2) ? R(2) : k == 3 ? R(20) : R(4);
}

// g+ = N^-1 [n - Theta (n - n^eq)], n = N g, n^eq = (T, u_x T/sigma,
// u_y T/sigma, varpi T, 0) of Eq. (34), T = n_0
template <typename R>
LBM_HD void thermal_node_collide(const ThermalNode<R>& p, const R g[5], R ux, R uy, R gpost[5]) {
  R n[5], np[5];
  d2q5_N(g, n);
  const R T = n[0];
  const R neq[5] = {T, ux * T / p.sigma, uy * T / p.sigma, p.varpi * T, R(0)};
  for (int k = 0; k < 5; ++k) np[k] = (n[k] - p.theta[k] * (n[k] - neq[k])) / d2q5_D<R>(k);
  d2q5_NT(np, gpost);
}

// its reverse: lg = adjoint of g+; out: adjoint of g (lgin) and of u, and
// (lz non-null) of the flux moments' rate theta_1 = theta_2
template <typename R>
LBM_HD void thermal_node_adjoint(const ThermalNode<R>& p, const R g[5], R ux, R uy, const R lg[5],
                                 R lgin[5], R* lux, R* luy, R* lz = nullptr) {
  R n[5], lnp[5], ln[5];
  d2q5_N(g, n);
  const R T = n[0];
  d2q5_N(lg, lnp);
  for (int k = 0; k < 5; ++k) lnp[k] /= d2q5_D<R>(k);
  if (lz) *lz = -lnp[1] * (n[1] - ux * T / p.sigma) - lnp[2] * (n[2] - uy * T / p.sigma);
  R lneq[5];
  for (int k = 0; k < 5; ++k) {
    ln[k] = (1 - p.theta[k]) * lnp[k];
    lneq[k] = p.theta[k] * lnp[k];
  }
  ln[0] += lneq[0] + (lneq[1] * ux + lneq[2] * uy) / p.sigma + p.varpi * lneq[3];
  *lux = lneq[1] * T / p.sigma;
  *luy = lneq[2] * T / p.sigma;
  d2q5_NT(ln, lgin);
}

// Wall extrapolation g_b = g^eq(T_w, 0) + g_f - g^eq(T_f, u_f), T_f = sum g_f,
// g^eq_i(T, u) = w~_i T (1 + e_i . u / (sigma c_sT^2)) of Eq. (39): given the
// adjoint of g_b, adds that of g_f to lgf and returns those of T_w and u_f
// (an adiabatic wall, T_w = T_f, adds lTw to every lgf_i itself).
template <typename R>
LBM_HD void wall_extrapolation_adjoint(const ThermalNode<R>& p, const R gf[5], R uxf, R uyf,
                                       const R lgb[5], R lgf[5], R* lTw, R* luxf, R* luyf) {
  const int ex[5] = {0, 1, 0, -1, 0};
  const int ey[5] = {0, 0, 1, 0, -1};
  const R Tf = gf[0] + gf[1] + gf[2] + gf[3] + gf[4];
  const R c = p.sigma * p.csT2;
  R lTf = 0, lw = 0, lx = 0, ly = 0;
  for (int j = 0; j < 5; ++j) {
    const R wj = j == 0 ? p.w0 : p.w1;
    const R t = lgb[j] * wj;
    lw += t;
    lTf -= t * (1 + (ex[j] * uxf + ey[j] * uyf) / c);
    lx -= t * Tf * ex[j] / c;
    ly -= t * Tf * ey[j] / c;
  }
  for (int i = 0; i < 5; ++i) lgf[i] += lgb[i] + lTf;
  *lTw = lw;
  *luxf = lx;
  *luyf = ly;
}

// ---- one reversed coupled step at one node (gather form) ---------------------

LBM_HD int hd_fetch_add(int* p, int v) {
#ifdef __CUDA_ARCH__
  return atomicAdd(p, v);
#else
  const int o = *p;
  *p += v;
  return o;
#endif
}

// Lattice geometry of the oracle: an axis is periodic or walled on both sides;
// bc = left, right, bottom, top: 0 periodic, 1 Dirichlet, 2 adiabatic.
struct CoupledGeo {
  int nx, ny, per_x, per_y;
  int bc[4];
  LBM_HD int nb(int x, int y, int dx, int dy) const {
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
  LBM_HD bool vx(int x) const { return !per_x && (x == 0 || x == nx - 1); }
  LBM_HD bool vy(int y) const { return !per_y && (y == 0 || y == ny - 1); }
  LBM_HD bool wall(int x, int y) const { return vx(x) || vy(y); }
  // inward neighbour of a wall node (the diagonal one at corners)
  LBM_HD int inward(int x, int y) const {
    const int xx = vx(x) ? (x == 0 ? 1 : nx - 2) : x;
    const int yy = vy(y) ? (y == 0 ? 1 : ny - 2) : y;
    return yy * nx + xx;
  }
  // 0 left, 1 right, 2 bottom, 3 top (corners go to the vertical wall)
  LBM_HD int side(int x, int y) const { return vx(x) ? (x == 0 ? 0 : 1) : (y == 0 ? 2 : 3); }
};

// Everything one reversed step reads and writes (natural layout, planes of n).
template <typename R>
struct CoupledStep {
  CoupledGeo geo;
  long long n;
  FlowNode<R> fp;
  ThermalNode<R> tp;
  R f_act, T_s, T_l, lat;
  // alpha_l != alpha_s (Sec. 4.1): the flux moments' rate follows f_l(n),
  // 1 / (1/2 + (tauT_l - 1/2) (f_l + (1 - f_l) inv_aratio)); a wall node's
  // that of its inward node
  int alpha_var;
  R tauT_l, inv_aratio;
  int flow;                                  // the flow lattice is on
  // the objective's direct terms in the state before the step: all five
  // populations at x = 1 and x = 2 and the left wall value, rows [ny0, ny1)
  R nu_g1, nu_g2, nu_tw;
  int ny0, ny1;
  const R *f0, *g0, *fl0, *fl1, *phi, *K;   // the step's state: before it, and f_l after
  R foff[9];                                 // added to f0 (stored deviations: w_i rho0)
  const R* lf1;                              // adjoint of f after the step
  const R* lg1;                              // adjoint of g after it, nu added on the band
  R *lf0, *lg0;                              // adjoints before the step
  R* lfl;                                    // adjoint of f_l: after the step in, before it out
  R *lphi, *lK, *lTw;                        // accumulated
  int *next_list, *next_count;               // band of the state before the step
};

// the flux moments' rate at liquid fraction fl, and its derivative
template <typename R>
LBM_HD R coupled_rate(const CoupledStep<R>& A, R fl, R* dz) {
  if (!A.alpha_var) {
    *dz = 0;
    return A.tp.theta[1];
  }
  const R c = A.tauT_l - R(0.5);
  const R z = R(1) / (R(0.5) + c * (fl + (1 - fl) * A.inv_aratio));
  *dz = -z * z * c * (1 - A.inv_aratio);
  return z;
}

template <typename R>
LBM_HD bool coupled_active(const CoupledStep<R>& A, int s) {
  const int y = s / A.geo.nx, x = s - y * A.geo.nx;
  return A.flow && !A.geo.wall(x, y) && A.fl0[s] >= A.f_act;
}
// the same for node s at (x, y), known already (no division)
template <typename R>
LBM_HD bool coupled_active_xy(const CoupledStep<R>& A, int x, int y, int s) {
  return A.flow && !A.geo.wall(x, y) && A.fl0[s] >= A.f_act;
}

// lam_g+ of node (x, y) streamed back from lg1 (0 from outside the lattice)
template <typename R>
LBM_HD void coupled_lp(const CoupledStep<R>& A, int x, int y, R lp[5]) {
  const int ex[5] = {0, 1, 0, -1, 0};
  const int ey[5] = {0, 0, 1, 0, -1};
  for (int i = 0; i < 5; ++i) {
    const int t = A.geo.nb(x, y, ex[i], ey[i]);
    lp[i] = t >= 0 ? A.lg1[i * A.n + t] : R(0);
  }
}

template <typename R>
LBM_HD void coupled_reverse_node(const CoupledStep<R>& A, int x, int y) {
  const CoupledGeo& G = A.geo;
  const long long n = A.n;
  const int s = y * G.nx + x;
  const bool wall = G.wall(x, y);
  const bool act = coupled_active_xy(A, x, y, s);
  // a node two or more nodes away from every wall is nobody's inward node
  const bool near_wall = (!G.per_x && (x <= 1 || x >= G.nx - 2)) ||
                         (!G.per_y && (y <= 1 || y >= G.ny - 2));
  R g[5], T = 0;
  for (int i = 0; i < 5; ++i) T += (g[i] = A.g0[i * n + s]);
  R f[9], ux = 0, uy = 0;
  for (int i = 0; i < 9; ++i) f[i] = A.f0[i * n + s] + A.foff[i];
  if (act) {
    FlowFwd<R> w;
    flow_node_forward(A.fp, f, T, A.fl0[s], A.phi[s], A.K[s], w);
    ux = w.ux;
    uy = w.uy;
  }
  // thermal: this node's collision (u = 0 on walls and off flow), at the rate
  // of f_l(n) (a wall node's inward node's)
  R lp[5], lgin[5], lux = 0, luy = 0, S = 0, lz = 0;
  coupled_lp(A, x, y, lp);
  for (int i = 0; i < 5; ++i) S += (i == 0 ? A.tp.w0 : A.tp.w1) * lp[i];
  R dz;
  ThermalNode<R> tpn = A.tp;
  tpn.theta[1] = tpn.theta[2] =
      coupled_rate(A, wall ? A.fl0[G.inward(x, y)] : A.fl0[s], &dz);
  {
    R lx, ly;
    thermal_node_adjoint(tpn, g, wall ? R(0) : ux, wall ? R(0) : uy, lp, lgin, &lx, &ly,
                         A.alpha_var ? &lz : nullptr);
    if (act) {
      lux += lx;
      luy += ly;
    }
  }
  R lg[5];
  R lfl;
  const R a = A.phi[s] * A.lat;
  if (wall) {
    for (int i = 0; i < 5; ++i) lg[i] = 0;   // the extrapolation rewrites them
    lfl = A.lfl[s];                          // a wall node keeps f_l(n)
  } else {
    const bool r = y >= A.ny0 && y < A.ny1;
    const R src = r && x == 1 ? A.nu_g1 : r && x == 2 ? A.nu_g2 : R(0);
    for (int i = 0; i < 5; ++i) lg[i] = lgin[i] + src;
    lfl = a * S + lz * dz;
    const R df = A.fl1[s] - A.fl0[s];
    if (df != 0) A.lphi[s] += -df * S * A.lat;
    // the extrapolation of every wall node whose inward node this is
    const int ex9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int d = 1; d < 9 && near_wall; ++d) {
      const int bx = x + ex9[d], by = y + ey9[d];
      if (bx < 0 || bx >= G.nx || by < 0 || by >= G.ny) continue;
      if (!G.wall(bx, by) || G.inward(bx, by) != s) continue;
      R lpb[5], lgb[5], lx, ly, lTwv, lxf, lyf, lzb = 0, dzb;
      coupled_lp(A, bx, by, lpb);
      ThermalNode<R> tpb = A.tp;
      tpb.theta[1] = tpb.theta[2] = coupled_rate(A, A.fl0[s], &dzb);   // the wall's rate: ours
      // the wall node's populations before collision up to g^eq(T_w, 0), whose
      // flux moments are 0: enough for the rate's adjoint (u = 0 there)
      R gb[5];
      {
        const int ex5[5] = {0, 1, 0, -1, 0};
        const int ey5[5] = {0, 0, 1, 0, -1};
        const R c = A.tp.sigma * A.tp.csT2;
        for (int i = 0; i < 5; ++i)
          gb[i] = g[i] - (i == 0 ? A.tp.w0 : A.tp.w1) * T * (1 + (ex5[i] * ux + ey5[i] * uy) / c);
      }
      thermal_node_adjoint(tpb, gb, R(0), R(0), lpb, lgb, &lx, &ly, A.alpha_var ? &lzb : nullptr);
      lfl += lzb * dzb;
      R lgf[5] = {0, 0, 0, 0, 0};
      wall_extrapolation_adjoint(A.tp, g, ux, uy, lgb, lgf, &lTwv, &lxf, &lyf);
      const int sd = G.side(bx, by);
      bool fixed = G.bc[sd] == 1;   // Dirichlet: the imposed value
      if (!fixed && G.vx(bx) && G.vy(by) && G.bc[by == 0 ? 2 : 3] == 1) fixed = true;
      if (G.bc[sd] == 1 && sd == 0) {
        A.lTw[by] += lTwv;
        if (by >= A.ny0 && by < A.ny1) A.lTw[by] += A.nu_tw;
      } else if (!fixed) {
        for (int i = 0; i < 5; ++i) lgf[i] += lTwv;   // adiabatic: T_w = T_f
      }
      for (int i = 0; i < 5; ++i) lg[i] += lgf[i];
      if (act) {
        lux += lxf;
        luy += lyf;
      }
    }
  }
  // flow: streaming reversed (bounce-back links in place), then the collision
  const int ex9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  if (act) {
    R lpost[9], lfin[9], lT, lflv, lphiv, lKv;
    for (int j = 0; j < 9; ++j) {
      const int t = G.nb(x, y, ex9[j], ey9[j]);
      bool on = t >= 0;
      if (on) {
        // (x + e_j, y + e_j) wrapped, without dividing t by nx
        int tx = x + ex9[j], ty = y + ey9[j];
        tx = tx < 0 ? tx + G.nx : (tx >= G.nx ? tx - G.nx : tx);
        ty = ty < 0 ? ty + G.ny : (ty >= G.ny ? ty - G.ny : ty);
        on = coupled_active_xy(A, tx, ty, t);
      }
      lpost[j] = on ? A.lf1[j * n + t] : A.lf1[op9[j] * n + s];
    }
    flow_node_adjoint(A.fp, f, T, A.fl0[s], A.phi[s], A.K[s], lpost, lux, luy, lfin, &lT, &lflv,
                      &lphiv, &lKv);
    for (int i = 0; i < 9; ++i) A.lf0[i * n + s] = lfin[i];
    for (int i = 0; i < 5; ++i) lg[i] += lT;   // T(n) = sum g(n)
    lfl += lflv;
    A.lphi[s] += lphiv;
    A.lK[s] += lKv;
  } else {
    for (int i = 0; i < 9; ++i) A.lf0[i * n + s] = A.lf1[i * n + s];
  }
  for (int i = 0; i < 5; ++i) A.lg0[i * n + s] = lg[i];
  A.lfl[s] = lfl;
  const R fa = A.fl0[s];
  if (!wall && adj_mushy(fa)) A.next_list[hd_fetch_add(A.next_count, 1)] = s;
}

}  // namespace lbm
