// Fused stream-collide of both lattices for one time step (AA pattern, in place).
//
// Per non-wall node:
//   1. gather g (5 populations) and T = sum g, Eq. (33);
//   2. on a flow node: gather f (9), rho and j, Eq. (24), velocity Eq. (26)-(28),
//      force Eq. (4)-(6), relax in moment space, Eq. (20) with Eq. (19), (22),
//      (23), back to velocity space and scatter, Eq. (21), with halfway
//      bounce-back on links into nodes without flow;
//   3. relax g in moment space without the latent source, Eq. (35) with (34),
//      (37), scatter, Eq. (36);
//   4. next to a thermal wall: write the wall node's inward post-collision
//      population by non-equilibrium extrapolation (Sec. 4 preamble), in the
//      post-collision form g+(x_b) = g^eq(T_w, 0) + [g+(x_f) - g^eq(T_f, u_f)];
//   5. decide whether this node could change phase in this step (see below)
//      and list the enthalpy tiles that must be solved.
// The latent source of the step is added afterwards by the enthalpy kernels.
//
// Two kernels share that per-node update.  fused_step_kernel reads each
// node's inputs with ordinary loads (one node per thread, any lattice).
// In fused_tma_kernel each CTA takes a few 32x8 tiles, strided by the grid
// size, and, while its threads update one tile from shared memory, the tensor
// memory accelerator copies the next tile's boxes (all f planes, all g planes,
// f_l with a halo, phi, K) into a second buffer, so data in flight costs no
// registers and no load addressing.  CTAs are short-lived, so the enthalpy
// kernels that overlap the far-tile pass get SMs as they retire.
// It serves lattices walled on all four sides with nx a multiple of 4 (the
// tensor maps need 16-byte row strides and cannot wrap periodic halos).  Each
// CTA reads from its buffer only the slots of its own nodes' AA access sets,
// which no other CTA writes during the step, so prefetching is race-free.
//
// Phase-change screen.  The temperature a node y sees after streaming is
// T*(y) = sum_i g+_i(y - e_i).  If y and its four neighbours are all solid
// (f_l = 0) and every outgoing population satisfies g+_i <= w~_i T_s, then
// T*(y) <= T_s and y stays solid; likewise all liquid with g+_i >= w~_i T_l.
// Every node failing both tests puts the enthalpy tiles of its 3x3
// neighbourhood on the step's work list; only listed tiles run the enthalpy
// solve.  The tests allow a margin of 1e-7 of the temperature scale (and f_l
// within 1e-7 of 0 or 1): without it, the sub-1e-30 values that diffusion
// carries ahead of a front at the lattice speed would list every tile they
// reach.  A node skipped this way can lag the exact fixed point by at most
// that margin; the enthalpy sum is unaffected, and the node is solved as soon
// as it leaves the margin.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

// g populations: FP32 storage holds them as they are, 16-bit storage as
// deviations from w~_i T_m (r = w~_i T_m is added back on load, removed on store)
template <typename S>
__device__ __forceinline__ float gload(const S* p, float r) {
  if constexpr (std::is_same<S, float>::value) return *p;
  else return Pop<S>::ld(p) + r;
}
template <typename S>
__device__ __forceinline__ void gstore(S* p, float v, float r, unsigned& rnd) {
  if constexpr (std::is_same<S, float>::value) *p = v;
  else st_round(p, v - r, next_rand(rnd));
}
template <typename S>
__device__ __forceinline__ void fstore(S* p, float v, unsigned& rnd) {
  if constexpr (std::is_same<S, float>::value) *p = v;
  else st_round(p, v, next_rand(rnd));
}

// put enthalpy tile t on this step's work list (once), and stamp the tiles
// within one tile of it in this parity's near map
__device__ __forceinline__ void mark_tile(const Dev& d, int t, int par) {
  int* fl = d.flags + par * d.ntiles;
  if (fl[t] == 0 && atomicExch(&fl[t], 1) == 0) {
    const int i = atomicAdd(&d.lcount[par], 1);
    d.list[par * d.ntiles + i] = t;
    const int stamp = d.ctr[1 - par] + 1;   // this step's stamp
    const int tx = t % d.etx, ty = t / d.etx;
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = ty + dy;
      if (yy < 0 || yy >= d.ety) {
        if (!d.per_y) continue;
        yy = (yy + d.ety) % d.ety;
      }
      for (int dx = -1; dx <= 1; ++dx) {
        int xx = tx + dx;
        if (xx < 0 || xx >= d.etx) {
          if (!d.per_x) continue;
          xx = (xx + d.etx) % d.etx;
        }
        d.nearmap[par * d.ntiles + yy * d.etx + xx] = stamp;
      }
    }
  }
}

// Indices of a non-wall node's neighbours (one step away: one wrap at most)
// and which of them are wall nodes.  Directions: 0 rest, 1 E, 2 N, 3 W, 4 S,
// 5 NE, 6 NW, 7 SW, 8 SE.
struct Geo {
  int s, xm, xp, ym, yp;
  int nb[9];
  bool wl[9];
};

// lattices walled on all four sides: a non-wall node's neighbours never wrap
__device__ __forceinline__ Geo node_geo_walled(const Dev& d, int x, int y) {
  Geo q;
  const int nx = d.nx;
  q.s = y * nx + x;
  q.xm = x - 1;
  q.xp = x + 1;
  q.ym = y - 1;
  q.yp = y + 1;
  q.nb[0] = q.s;
  q.nb[1] = q.s + 1;
  q.nb[2] = q.s + nx;
  q.nb[3] = q.s - 1;
  q.nb[4] = q.s - nx;
  q.nb[5] = q.s + nx + 1;
  q.nb[6] = q.s + nx - 1;
  q.nb[7] = q.s - nx - 1;
  q.nb[8] = q.s - nx + 1;
  const bool cE = x == nx - 2, cW = x == 1, rN = y == d.ny - 2, rS = y == 1;
  q.wl[0] = false;
  q.wl[1] = cE;
  q.wl[2] = rN;
  q.wl[3] = cW;
  q.wl[4] = rS;
  q.wl[5] = cE || rN;
  q.wl[6] = cW || rN;
  q.wl[7] = cW || rS;
  q.wl[8] = cE || rS;
  return q;
}

__device__ __forceinline__ Geo node_geo(const Dev& d, int x, int y) {
  Geo q;
  const int nx = d.nx, ny = d.ny;
  q.s = y * nx + x;
  q.xm = (x == 0) ? nx - 1 : x - 1;
  q.xp = (x == nx - 1) ? 0 : x + 1;
  q.ym = (y == 0) ? ny - 1 : y - 1;
  q.yp = (y == ny - 1) ? 0 : y + 1;
  q.nb[0] = q.s;
  q.nb[1] = y * nx + q.xp;
  q.nb[2] = q.yp * nx + x;
  q.nb[3] = y * nx + q.xm;
  q.nb[4] = q.ym * nx + x;
  q.nb[5] = q.yp * nx + q.xp;
  q.nb[6] = q.yp * nx + q.xm;
  q.nb[7] = q.ym * nx + q.xm;
  q.nb[8] = q.ym * nx + q.xp;
  const bool cE = d.wall_r && q.xp == nx - 1, cW = d.wall_l && q.xm == 0;
  const bool rN = d.wall_t && q.yp == ny - 1, rS = d.wall_b && q.ym == 0;
  q.wl[0] = false;
  q.wl[1] = cE;
  q.wl[2] = rN;
  q.wl[3] = cW;
  q.wl[4] = rS;
  q.wl[5] = cE || rN;
  q.wl[6] = cW || rN;
  q.wl[7] = cW || rS;
  q.wl[8] = cE || rS;
  return q;
}

// The flow collision of one node, Eq. (16)-(28): f (nine populations as
// deviations f_i - w_i rho0) relaxed in moment space with the porous force and
// buoyancy at temperature T, liquid fraction flc, porosity phi and
// permeability K; fp gets the post-collision deviations, (ux, uy) the velocity.
__device__ __forceinline__ void flow_collide(const Dev& d, const float f[9], float T, float flc,
                                             float phi, float K, float fp[9], float& ux,
                                             float& uy) {
  // populations are stored as deviations from the rest equilibrium,
  // f_i - w_i rho0 (sum_i e_i w_i = 0, so j needs no correction)
  const float drho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const float jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const float jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  float Fx, Fy;
  velocity(jx, jy, T, flc, phi, K, d, ux, uy, Fx, Fy);
  const float varphi = phi * flc;
  const float ivp = 1.f / varphi;
  const float rho0 = d.rho0;
  // moments of the deviations, M (f - w rho0); M (w rho0) = (rho0, -2 rho0, rho0, 0, ..., 0)
  const float sa = f[1] + f[2] + f[3] + f[4];
  const float sd = f[5] + f[6] + f[7] + f[8];
  const float m1 = -4.f * f[0] - sa + 2.f * sd;
  const float m2 = 4.f * f[0] - 2.f * sa + sd;
  const float m4 = -2.f * f[1] + 2.f * f[3] + f[5] - f[6] - f[7] + f[8];
  const float m6 = -2.f * f[2] + 2.f * f[4] + f[5] + f[6] - f[7] - f[8];
  const float m7 = f[1] - f[2] + f[3] - f[4];
  const float m8 = f[5] - f[6] + f[7] - f[8];
  const float uu = ux * ux + uy * uy;
  // non-equilibrium parts m - m^eq of e and eps, Eq. (19), with rho = rho0 + drho
  const float ne1 = m1 + 2.f * drho - 3.f * rho0 * uu * ivp;
  const float ne2 = m2 - drho + 3.f * rho0 * uu * ivp;
  // forcing moments, Eq. (22)
  const float uF = ux * Fx + uy * Fy;
  const float S1 = 6.f * rho0 * uF * ivp;
  const float S7 = 2.f * rho0 * (ux * Fx - uy * Fy) * ivp;
  const float S8 = rho0 * (ux * Fy + uy * Fx) * ivp;
  // m+ - m = -Lambda (m - m^eq) + (I - Lambda/2) S, Eq. (20); for the
  // conserved moments this is 0 (rho) and rho0 F (momentum, with Eq. 25)
  const float d1 = -d.s_e * ne1 + (1.f - 0.5f * d.s_e) * S1;
  const float d2 = -d.s_eps * ne2 - (1.f - 0.5f * d.s_eps) * S1;
  const float d3 = rho0 * Fx;
  const float d4 = -d.s_q * (m4 + rho0 * ux) - (1.f - 0.5f * d.s_q) * rho0 * Fx;
  const float d5 = rho0 * Fy;
  const float d6 = -d.s_q * (m6 + rho0 * uy) - (1.f - 0.5f * d.s_q) * rho0 * Fy;
  const float d7 = -d.s_nu * (m7 - rho0 * (ux * ux - uy * uy) * ivp) + (1.f - 0.5f * d.s_nu) * S7;
  const float d8 = -d.s_nu * (m8 - rho0 * ux * uy * ivp) + (1.f - 0.5f * d.s_nu) * S8;
  // f+ = f + M^-1 (m+ - m), M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
  const float a1 = d1 * (1.f / 36.f), a2 = d2 * (1.f / 36.f);
  const float a3 = d3 * (1.f / 6.f), a4 = d4 * (1.f / 12.f);
  const float a5 = d5 * (1.f / 6.f), a6 = d6 * (1.f / 12.f);
  const float a7 = d7 * 0.25f, a8 = d8 * 0.25f;
  const float c_ax = -a1 - 2.f * a2;   // common part of the axis directions
  const float c_dg = 2.f * a1 + a2;    // common part of the diagonals
  fp[0] = f[0] - 4.f * a1 + 4.f * a2;
  fp[1] = f[1] + c_ax + a3 - 2.f * a4 + a7;
  fp[2] = f[2] + c_ax + a5 - 2.f * a6 - a7;
  fp[3] = f[3] + c_ax - a3 + 2.f * a4 + a7;
  fp[4] = f[4] + c_ax - a5 + 2.f * a6 - a7;
  fp[5] = f[5] + c_dg + a3 + a4 + a5 + a6 + a8;
  fp[6] = f[6] + c_dg - a3 - a4 + a5 + a6 - a8;
  fp[7] = f[7] + c_dg - a3 - a4 - a5 - a6 + a8;
  fp[8] = f[8] + c_dg + a3 + a4 - a5 - a6 - a8;
}

// Non-equilibrium extrapolation of Sec. 4 from a flow node: the boundary
// node's state f^eq(rho, 0) + f - f^eq(rho, u) (deviations: f minus the
// velocity part of f^eq at the node's rho and u), collided with the flow
// node's T, f_l, phi and K, into fe
static __device__ __noinline__ void extrapolated_post(const Dev& d, const float f[9], float T, float fl,
                                               float phi, float K, float ux, float uy,
                                               float fe[9]) {
  const float w9[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                       1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
  const float ivp = 1.f / (phi * fl);
  const float uu = ux * ux + uy * uy;
  float fb[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float eu = ex9(i) * ux + ey9(i) * uy;
    fb[i] = f[i] - w9[i] * d.rho0 * (3.f * eu + 4.5f * eu * eu * ivp - 1.5f * uu * ivp);
  }
  float ub, vb;
  flow_collide(d, fb, T, fl, phi, K, fe, ub, vb);
}

// The update of one non-wall node from its gathered inputs: fln = f_l of the
// 3x3 neighbourhood (-1 on walls), gin = its five thermal populations, f = its
// nine flow populations as streamed from the neighbours, fb = (odd steps) the
// populations reflected at each link, used where the neighbour carries no
// flow.  wact (flow walls only): bit i set when neighbour i is a wall node that
// carries flow (its inward node does), so that the link streams instead of
// reflecting.  Writes the post-collision populations to their AA slots and
// returns whether the node fails the phase-change screen.
template <typename S, int PAR, int FLOW, bool EDGE = true>
__device__ __forceinline__ bool node_update(const Dev& d, int x, int y, const Geo& q,
                                            const float fln[9], const float gin[5], float f[9],
                                            const float fb[9], float phi, float K,
                                            unsigned wact = 0u, unsigned seed = 0u) {
  const int nx = d.nx, ny = d.ny;
  const int n = (int)d.n;
  const int s = q.s;
  const int sE = q.nb[1], sN = q.nb[2], sW = q.nb[3], sS = q.nb[4];
  S* G = static_cast<S*>(d.g);
  S* F = static_cast<S*>(d.f);
  const float r0 = d.wt0 * d.g_ref, r1 = d.wt1 * d.g_ref;   // g storage reference
  // rounding bits of this node and step (16-bit storage only)
  unsigned rnd = 0u;
  if constexpr (!std::is_same<S, float>::value)
    rnd = mix32((unsigned)s ^ seed);
  const float flc = fln[0];
  const float g0 = gin[0], g1 = gin[1], g2 = gin[2], g3 = gin[3], g4 = gin[4];
  const float T = g0 + g1 + g2 + g3 + g4;

  // ---- flow lattice ------------------------------------------------------
  float ux = 0.f, uy = 0.f;
  if (FLOW && flc >= d.f_act) {
    const float fa = d.f_act;
    // neighbour flow activity, directions 1..8 (E, N, W, S, NE, NW, SW, SE)
    bool act[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) act[i] = fln[i] >= fa || ((wact >> i) & 1u);
    if (PAR == 1) {
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if (!act[opp9(i)]) f[i] = fb[i];
    }
    float fp[9];
    flow_collide(d, f, T, flc, phi, K, fp, ux, uy);
    if (FLOW == 2) {
      // links into non-flow lattice nodes (the front; walls keep their own
      // rule): what arrives from the solid node is its extrapolated population
      // in place of our reflected one, in the same slot
      unsigned fm = 0u;
#pragma unroll
      for (int i = 1; i < 9; ++i)
        if (!act[i] && !(EDGE && q.wl[i])) fm |= 1u << i;
      if (fm) {
        float fe[9];
        extrapolated_post(d, f, T, flc, phi, K, ux, uy, fe);
#pragma unroll
        for (int i = 1; i < 9; ++i)
          if ((fm >> i) & 1u) fp[i] = fe[opp9(i)];
      }
    }
    if (PAR == 0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) fstore(&F[opp9(i) * n + s], fp[i], rnd);
    } else {
      fstore(&F[s], fp[0], rnd);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        // into a node without flow: halfway bounce-back into our own slot
        const int off = act[i] ? i * n + q.nb[i] : opp9(i) * n + s;
        fstore(&F[off], fp[i], rnd);
      }
    }
  }

  // ---- thermal collision (no latent source) ------------------------------
  const float n1 = g1 - g3, n2 = g2 - g4;
  const float n3 = -4.f * g0 + g1 + g2 + g3 + g4;
  const float n4 = g1 - g2 + g3 - g4;
  // sigma_l / sigma(f_l(n)) (Eq. (7)); 1 with one sigma for both phases
  const float sr = sigma_ratio(d, flc);
  const float th = d.conv * d.csT2 * sr;   // vartheta / sigma
  // zeta_alpha = 1/tau_T = 1/(1/2 + alpha_e / (sigma c_sT^2)); alpha_e follows
  // f_l(n) with alpha_l != alpha_s (Sec. 4.1), sigma with sigma_s != sigma_l
  const float za =
      (d.alpha_var | d.sigma_var)
          ? 1.f / (0.5f + (d.tauT_l - 0.5f) * (d.alpha_var ? flc + (1.f - flc) * d.inv_aratio
                                                           : 1.f) * sr)
          : d.z_a;
  const float b1 = -0.5f * za * (n1 - th * ux * T);
  const float b2 = -0.5f * za * (n2 - th * uy * T);
  const float b3 = -0.05f * d.z_e * (n3 - d.varpi * T);
  const float b4 = -0.25f * d.z_nu * n4;
  const float gp0 = g0 - 4.f * b3;
  const float gp1 = g1 + b1 + b3 + b4;
  const float gp2 = g2 + b2 + b3 - b4;
  const float gp3 = g3 - b1 + b3 + b4;
  const float gp4 = g4 - b2 + b3 - b4;
  if (PAR == 0) {
    gstore(&G[s], gp0, r0, rnd);
    gstore(&G[3 * n + s], gp1, r1, rnd);
    gstore(&G[4 * n + s], gp2, r1, rnd);
    gstore(&G[n + s], gp3, r1, rnd);
    gstore(&G[2 * n + s], gp4, r1, rnd);
  } else {
    gstore(&G[s], gp0, r0, rnd);
    gstore(&G[n + sE], gp1, r1, rnd);
    gstore(&G[2 * n + sN], gp2, r1, rnd);
    gstore(&G[3 * n + sW], gp3, r1, rnd);
    gstore(&G[4 * n + sS], gp4, r1, rnd);
  }

  // ---- phase-change screen (own populations) -----------------------------
  bool cold = (flc <= d.scr_f), hot = (flc >= 1.f - d.scr_f);
  {
    const float nbv[4] = {fln[1], fln[2], fln[3], fln[4]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (nbv[k] >= 0.f) {
        cold = cold && (nbv[k] <= d.scr_f);
        hot = hot && (nbv[k] >= 1.f - d.scr_f);
      }
    }
    const float lo0 = d.wt0 * (d.T_s + d.scr_T), lo1 = d.wt1 * (d.T_s + d.scr_T);
    const float hi0 = d.wt0 * (d.T_l - d.scr_T), hi1 = d.wt1 * (d.T_l - d.scr_T);
    cold = cold && gp0 <= lo0 && gp1 <= lo1 && gp2 <= lo1 && gp3 <= lo1 && gp4 <= lo1;
    hot = hot && gp0 >= hi0 && gp1 >= hi1 && gp2 >= hi1 && gp3 >= hi1 && gp4 >= hi1;
  }

  // ---- thermal walls: inward population of adjacent wall nodes ------------
  // wall on side S at x_b = x - e_k, inward direction k; geq_k(T,u) = w~ T (1 + conv e_k.u)
  const float cv = d.conv * sr;
#define LBM_WALL_POP(COND, K, SB, TW, EU)                                         \
  if (COND) {                                                                     \
    const float gpk = (K == 1) ? gp1 : (K == 2) ? gp2 : (K == 3) ? gp3 : gp4;     \
    const float w = d.wt1 * (TW) + gpk - d.wt1 * T * (1.f + cv * (EU));           \
    if (PAR == 0) gstore(&G[opp5(K) * n + (SB)], w, r1, rnd);                     \
    else gstore(&G[(K) * n + s], w, r1, rnd);                                     \
    cold = cold && (w <= d.wt1 * (d.T_s + d.scr_T));                              \
    hot = hot && (w >= d.wt1 * (d.T_l - d.scr_T));                                \
  }
  if (EDGE) {   // (a node of an interior tile has no wall neighbour)
    LBM_WALL_POP(d.wall_l && x == 1, 1, sW, d.bc[0] == 1 ? d.wallTl[y] : T, ux)
    LBM_WALL_POP(d.wall_r && x == nx - 2, 3, sE, d.bc[1] == 1 ? d.Tbc[1] : T, -ux)
    LBM_WALL_POP(d.wall_b && y == 1, 2, sS, d.bc[2] == 1 ? d.Tbc[2] : T, uy)
    LBM_WALL_POP(d.wall_t && y == ny - 2, 4, sN, d.bc[3] == 1 ? d.Tbc[3] : T, -uy)
  }
#undef LBM_WALL_POP

  const bool unsafe = d.screen_off || !(cold || hot);
  if (unsafe) {
    // list the enthalpy tiles holding this node's 3x3 neighbourhood (other
    // than its own, which the caller lists with one vote per warp)
    const int cx = (unsigned)x / TE, cy = (unsigned)y / TE;
    const int txs[3] = {(int)((unsigned)q.xm / TE), cx, (int)((unsigned)q.xp / TE)};
    const int tys[3] = {(int)((unsigned)q.ym / TE), cy, (int)((unsigned)q.yp / TE)};
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (txs[i] != cx || tys[j] != cy) mark_tile(d, tys[j] * d.etx + txs[i], PAR);
  }
  return unsafe;
}

// Flow walls (Sec. 4): which wall neighbours of node (x, y) carry flow, as bits
// 1..8 of a mask; flat(dx, dy) gives f_l of the node at offset (dx, dy), and a
// wall neighbour's inward node is always within one node of (x, y).
template <typename FlAt>
__device__ __forceinline__ unsigned wall_activity(const Dev& d, int x, int y, const Geo& q,
                                                  FlAt flat) {
  unsigned m = 0u;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (!q.wl[i]) continue;
    int ix, iy;
    inward_of(d, x + ex9(i), y + ey9(i), ix, iy);
    if (flat(ix - x, iy - y) >= d.f_act) m |= 1u << i;
  }
  return m;
}

// Once per step (the near-tile launch runs after the previous step's enthalpy
// kernels, the last readers of the other list): stamp the step and empty the
// next step's list.
template <int PAR>
__device__ __forceinline__ void step_prologue(const Dev& d) {
  d.ctr[PAR] = d.ctr[1 - PAR] + 1;
  d.lcount[1 - PAR] = 0;
}

// Split steps: does this launch (MODE 1 far tiles, MODE 2 near tiles) take the
// tile whose enthalpy tile is et?  The previous step's near map carries its
// stamp on the tiles within one tile of its listed tiles.
template <int PAR, int MODE>
__device__ __forceinline__ bool takes_tile(const Dev& d, int et) {
  if (MODE == 0) return true;
  const bool nr = d.nearmap[(1 - PAR) * d.ntiles + et] == d.ctr[1 - PAR];
  return (MODE == 2) == nr;
}

// ---- flow walls (Sec. 4, non-equilibrium extrapolation) ---------------------
//
// With flow walls on, a wall node x_b whose inward node x_f carries flow takes,
// before collision, f^eq(rho_f, 0) + f(x_f) - f^eq(rho_f, u_f) (rho, u and
// varphi of x_f; the u-terms of Eq. (29) only, since f^eq's rho-term cancels),
// collides with x_f's T, f_l, phi and K, and streams like a flow node; the
// links from its neighbours into it stream instead of reflecting.  This kernel
// does that for the wall nodes, one thread each, before the step's
// stream-collide pass overwrites x_f's populations (in the AA pattern a node
// reads and writes the same slots, and x_b only writes slots that nobody else
// reads or writes in the step).  MODE 1 / 2 take the wall nodes whose x_f lies
// in a far / near enthalpy tile, as the split stream-collide passes do.
template <typename S, int PAR, int MODE>
__global__ void __launch_bounds__(256) flow_wall_kernel(Dev d) {
  const int nx = d.nx, ny = d.ny, n = (int)d.n;
  const int nbot = d.wall_b ? nx : 0, ntop = d.wall_t ? nx : 0;
  const int ylo = d.wall_b ? 1 : 0, yhi = d.wall_t ? ny - 1 : ny;
  const int nleft = d.wall_l ? yhi - ylo : 0, nright = d.wall_r ? yhi - ylo : 0;
  const int total = nbot + ntop + nleft + nright;
  S* F = static_cast<S*>(d.f);
  const S* G = static_cast<const S*>(d.g);
  const float r0 = d.wt0 * d.g_ref, r1 = d.wt1 * d.g_ref;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    int x, y, kk = k;
    if (kk < nbot) {
      x = kk;
      y = 0;
    } else if ((kk -= nbot) < ntop) {
      x = kk;
      y = ny - 1;
    } else if ((kk -= ntop) < nleft) {
      x = 0;
      y = ylo + kk;
    } else {
      x = nx - 1;
      y = ylo + kk - nleft;
    }
    int ix, iy;
    inward_of(d, x, y, ix, iy);
    if (is_wall(d, ix, iy)) continue;   // a lattice too narrow to have an inward node
    const int sf = iy * nx + ix;
    const float flf = d.fl[sf];
    if (flf < d.f_act) continue;   // the inward node carries no flow: the wall reflects
    if (MODE != 0 && !takes_tile<PAR, MODE>(d, (iy / TE) * d.etx + ix / TE)) continue;
    // x_f's populations before the step's collision, as its own update reads them
    float f[9], g[5];
    if (PAR == 0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = Pop<S>::ld(&F[i * n + sf]);
#pragma unroll
      for (int i = 0; i < 5; ++i) g[i] = gload(&G[i * n + sf], i ? r1 : r0);
    } else {
      f[0] = Pop<S>::ld(&F[sf]);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int sx = wrapx(d, ix - ex9(i)), sy = wrapy(d, iy - ey9(i));
        bool a;   // does the source node carry flow?
        if (is_wall(d, sx, sy)) {
          int jx, jy;
          inward_of(d, sx, sy, jx, jy);
          a = d.fl[jy * nx + jx] >= d.f_act;
        } else {
          a = d.fl[sy * nx + sx] >= d.f_act;
        }
        f[i] = a ? Pop<S>::ld(&F[opp9(i) * n + sy * nx + sx]) : Pop<S>::ld(&F[i * n + sf]);
      }
      g[0] = gload(&G[sf], r0);
#pragma unroll
      for (int i = 1; i < 5; ++i) {
        const int sx = wrapx(d, ix - ex9(i)), sy = wrapy(d, iy - ey9(i));
        g[i] = gload(&G[opp5(i) * n + sy * nx + sx], r1);
      }
    }
    const float T = g[0] + g[1] + g[2] + g[3] + g[4];
    const float phi = d.phi[sf], K = d.K[sf];
    const float jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const float jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    float ux, uy, Fx, Fy;
    velocity(jx, jy, T, flf, phi, K, d, ux, uy, Fx, Fy);
    float fp[9];
    extrapolated_post(d, f, T, flf, phi, K, ux, uy, fp);
    const int sb = y * nx + x;
    unsigned rnd = 0u;
    if constexpr (!std::is_same<S, float>::value)
      rnd = mix32((unsigned)sb ^ mix32((unsigned)d.ctr[1 - PAR]));
    if (PAR == 0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) fstore(&F[opp9(i) * n + sb], fp[i], rnd);
    } else {
      fstore(&F[sb], fp[0], rnd);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int zx = wrapx(d, x + ex9(i)), zy = wrapy(d, y + ey9(i));
        bool a = false;   // does the receiving node carry flow?
        if (zx >= 0 && zy >= 0) {
          if (is_wall(d, zx, zy)) {
            int jx2, jy2;
            inward_of(d, zx, zy, jx2, jy2);
            a = d.fl[jy2 * nx + jx2] >= d.f_act;
          } else {
            a = d.fl[zy * nx + zx] >= d.f_act;
          }
        }
        fstore(&F[a ? i * n + zy * nx + zx : opp9(i) * n + sb], fp[i], rnd);
      }
    }
  }
}

template <typename S>
static void launch_flow_walls_t(const Dev& d, int parity, int mode, cudaStream_t s) {
  const int total = 2 * (d.nx + d.ny);
  const int grid = (total + 255) / 256;
#define LBM_FW(P, M) flow_wall_kernel<S, P, M><<<grid, 256, 0, s>>>(d)
  if (parity == 0) {
    if (mode == 0) LBM_FW(0, 0);
    else if (mode == 1) LBM_FW(0, 1);
    else LBM_FW(0, 2);
  } else {
    if (mode == 0) LBM_FW(1, 0);
    else if (mode == 1) LBM_FW(1, 1);
    else LBM_FW(1, 2);
  }
#undef LBM_FW
}

// ---- ordinary-load kernel ----------------------------------------------------

template <typename S, int PAR, int FLOW, int MODE>
__global__ void __launch_bounds__(TX* TY, 4) fused_step_kernel(Dev d) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  if (MODE != 1 && blockIdx.x == 0 && blockIdx.y == 0 && lane == 0 && threadIdx.y == 0)
    step_prologue<PAR>(d);
  if (!takes_tile<PAR, MODE>(d, ((blockIdx.y * TY) / TE) * d.etx + (blockIdx.x * TX) / TE)) return;
  const int x = blockIdx.x * TX + lane, y = blockIdx.y * TY + threadIdx.y;
  const int nx = d.nx, ny = d.ny;
  if (y >= ny) return;  // whole warp: one warp is one row segment
  const bool node = x < nx && !is_wall(d, x, y);
  bool unsafe = false;
  if (node) {
    const Geo q = node_geo(d, x, y);
    const int n = (int)d.n;
    const int s = q.s;
    // all loads of the node are issued before any of them is used, so one
    // memory round trip covers the step: the populations are read whether or
    // not the node carries flow, and on odd steps both candidate slots of each
    // direction (streamed from the neighbour, or reflected at the link)
    float fln[9];
    fln[0] = d.fl[s];
#pragma unroll
    for (int i = 1; i < 9; ++i) fln[i] = q.wl[i] ? -1.f : d.fl[q.nb[i]];
    const S* G = static_cast<const S*>(d.g);
    const float r0 = d.wt0 * d.g_ref, r1 = d.wt1 * d.g_ref;
    float g[5];
    if (PAR == 0) {
#pragma unroll
      for (int i = 0; i < 5; ++i) g[i] = gload(&G[i * n + s], i ? r1 : r0);
    } else {
      g[0] = gload(&G[s], r0);
#pragma unroll
      for (int i = 1; i < 5; ++i) g[i] = gload(&G[opp5(i) * n + q.nb[opp5(i)]], r1);
    }
    float f[9], fb[9];
    float phi = 0.f, K = 1.f;
    if (FLOW) {
      const S* F = static_cast<const S*>(d.f);
      phi = d.phi[s];
      K = d.K[s];
      if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = Pop<S>::ld(&F[i * n + s]);
      } else {
        f[0] = Pop<S>::ld(&F[s]);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int o = opp9(i);
          f[i] = Pop<S>::ld(&F[o * n + q.nb[o]]);   // from the source node x - e_i
          fb[i] = Pop<S>::ld(&F[i * n + s]);        // reflected at the link x - e_i | x
        }
      }
    }
    unsigned wact = 0u;
    if (FLOW && d.flow_walls)
      wact = wall_activity(d, x, y, q, [&](int dx, int dy) {
        return d.fl[(long long)wrapy(d, y + dy) * nx + wrapx(d, x + dx)];
      });
    const unsigned seed = std::is_same<S, float>::value ? 0u : mix32((unsigned)d.ctr[1 - PAR]);
    unsafe = node_update<S, PAR, FLOW>(d, x, y, q, fln, g, f, fb, phi, K, wact, seed);
  }
  if (__any_sync(FULL, unsafe) && lane == 0)
    mark_tile(d, (y / TE) * d.etx + (blockIdx.x * TX) / TE, PAR);
}

// ---- TMA-staged kernel ----------------------------------------------

constexpr int HX = 4;            // halo columns each side (16-byte aligned box start)
constexpr int HY = 1;            // halo rows each side
constexpr int WX = TX + 2 * HX;  // 40
constexpr int WY = TY + 2 * HY;  // 10
constexpr int TMA_MIN_CTAS = 4;  // resident CTAs per SM the register budget allows
constexpr long long TMA_WAIT_NS = 200000000LL;   // bounded mbarrier waits: 0.2 s
constexpr int TMA_NBUF_EVEN = 2;
constexpr int TMA_NBUF_ODD = 2;

// shared-memory layout of one buffer (byte offsets, each 128-byte aligned);
// two buffers, then two mbarriers and the tile indices of the two buffers
template <int PAR, typename S>
struct TmaLayout {
  // population boxes: a halo only on odd steps, as wide as the 16-byte rule
  // needs for the storage type (4 columns of FP32, 8 of a 16-bit type)
  static constexpr int HS = 16 / (int)sizeof(S);
  static constexpr int PX = PAR ? TX + 2 * HS : TX;
  static constexpr int PY = PAR ? WY : TY;
  static constexpr int F_BYTES = 9 * PX * PY * (int)sizeof(S);
  static constexpr int G_BYTES = 5 * PX * PY * (int)sizeof(S);
  static constexpr int FL_BYTES = WX * WY * 4;
  static constexpr int M_BYTES = TX * TY * 4;
  static constexpr int al(int b) { return (b + 127) & ~127; }
  static constexpr int F_OFF = 0;
  static constexpr int G_OFF = F_OFF + al(F_BYTES);
  static constexpr int FL_OFF = G_OFF + al(G_BYTES);
  static constexpr int PHI_OFF = FL_OFF + al(FL_BYTES);
  static constexpr int K_OFF = PHI_OFF + al(M_BYTES);
  static constexpr int BYTES = K_OFF + al(M_BYTES);
  // buffers in the ring: NBUF - 1 tiles load while one is computed (a third
  // buffer for the even step's smaller boxes still fits four CTAs per SM, but
  // measured no faster on the 2048^2 cavity)
  static constexpr int NBUF = PAR ? TMA_NBUF_ODD : TMA_NBUF_EVEN;
  static constexpr int BAR_OFF = NBUF * BYTES;
  static constexpr int IDX_OFF = BAR_OFF + 8 * NBUF;
  static constexpr int SMEM = IDX_OFF + 16;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for phase `parity` of an mbarrier, giving up after limit_ns (and after
// 2^24 polls whatever the clock says); false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity,
                                          long long limit_ns = TMA_WAIT_NS) {
  long long t0 = 0;
  for (int it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > limit_ns || it > (1 << 24)) return false;
  }
}

// issue the copies of the tile at (x0, y0) into buffer `buf`, completing on `bar`;
// flows: some node of the tile carries flow (else its nodes read neither their
// flow populations nor phi and K, and those are not copied)
template <typename S, int PAR, int FLOW>
__device__ __forceinline__ void tma_issue(const TmaMaps& m, unsigned buf, unsigned bar, int x0,
                                          int y0, bool flows) {
  using L = TmaLayout<PAR, S>;
  const bool fc = FLOW && flows;
  const int bytes = (fc ? L::F_BYTES + 2 * L::M_BYTES : 0) + L::G_BYTES + L::FL_BYTES;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  // x0 is a multiple of 32 and HX of 4: every box starts on a 16-byte boundary
  const int px = PAR ? x0 - L::HS : x0, py = PAR ? y0 - HY : y0;
  if (fc) tma_load_3d(buf + L::F_OFF, PAR ? &m.f_odd : &m.f_even, px, py, 0, bar);
  tma_load_3d(buf + L::G_OFF, PAR ? &m.g_odd : &m.g_even, px, py, 0, bar);
  tma_load_2d(buf + L::FL_OFF, &m.fl, x0 - HX, y0 - HY, bar);
  if (fc) {
    tma_load_2d(buf + L::PHI_OFF, &m.phi, x0, y0, bar);
    tma_load_2d(buf + L::K_OFF, &m.K, x0, y0, bar);
  }
}

// The update of node (x0 + lane, y0 + ty) of a tile staged in buffer sb.
// EDGE = false: the tile has no wall node and no neighbour of a wall node.
template <typename S, int PAR, int FLOW, bool EDGE>
__device__ __forceinline__ bool tma_node(const Dev& d, const unsigned char* sb, int x0, int y0,
                                         int lane, int ty, unsigned seed) {
  using L = TmaLayout<PAR, S>;
  const int nx = d.nx, ny = d.ny;
  const int x = x0 + lane, y = y0 + ty;
  bool unsafe = false;
  if (!EDGE || (x < nx && y < ny && !is_wall(d, x, y))) {
      Geo q = node_geo_walled(d, x, y);
      if (!EDGE)
#pragma unroll
        for (int i = 0; i < 9; ++i) q.wl[i] = false;
      const S* sF = reinterpret_cast<const S*>(sb + L::F_OFF);
      const S* sG = reinterpret_cast<const S*>(sb + L::G_OFF);
      const float r0 = d.wt0 * d.g_ref, r1 = d.wt1 * d.g_ref;
      const float* sFL = reinterpret_cast<const float*>(sb + L::FL_OFF);
      // f_l of the 3x3 neighbourhood from the halo window (origin x0 - 4, y0 - 1);
      // all four sides are walls, so every neighbour of a non-wall node is in it
      const int c = (ty + HY) * WX + (lane + HX);
      float fln[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) fln[i] = q.wl[i] ? -1.f : sFL[c + ey9(i) * WX + ex9(i)];
      constexpr int PX = L::PX, PP = L::PX * L::PY;
      const int pc = PAR ? (ty + HY) * PX + (lane + L::HS) : ty * PX + lane;
      float g[5];
      if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = gload(&sG[i * PP + pc], i ? r1 : r0);
      } else {
        g[0] = gload(&sG[pc], r0);
#pragma unroll
        for (int i = 1; i < 5; ++i) {
          const int o = opp5(i);   // from the source node x - e_i = x + e_o, its slot o
          g[i] = gload(&sG[o * PP + pc + ey9(o) * PX + ex9(o)], r1);
        }
      }
      float f[9], fb[9];
      float phi = 0.f, K = 1.f;
      if (FLOW) {
        phi = reinterpret_cast<const float*>(sb + L::PHI_OFF)[ty * TX + lane];
        K = reinterpret_cast<const float*>(sb + L::K_OFF)[ty * TX + lane];
        if (PAR == 0) {
#pragma unroll
          for (int i = 0; i < 9; ++i) f[i] = Pop<S>::ld(&sF[i * PP + pc]);
        } else {
          f[0] = Pop<S>::ld(&sF[pc]);
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            const int o = opp9(i);
            f[i] = Pop<S>::ld(&sF[o * PP + pc + ey9(o) * PX + ex9(o)]);
            fb[i] = Pop<S>::ld(&sF[i * PP + pc]);
          }
        }
      }
      unsigned wact = 0u;
      if (FLOW && EDGE && d.flow_walls)
        wact = wall_activity(d, x, y, q, [&](int dx, int dy) { return sFL[c + dy * WX + dx]; });
      unsafe = node_update<S, PAR, FLOW, EDGE>(d, x, y, q, fln, g, f, fb, phi, K, wact, seed);
  }
  return unsafe;
}

// One CTA's share of the pass over one lattice: CTA bid of nblk (blockIdx.x
// and gridDim.x of a single lattice's launch; its range in a batched launch).
template <typename S, int PAR, int FLOW, int MODE>
__device__ __forceinline__ void fused_tma_body(const Dev& d, const TmaMaps& m, int bid,
                                               int nblk) {
  using L = TmaLayout<PAR, S>;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned* s_mask = reinterpret_cast<unsigned*>(smem + L::IDX_OFF);
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + lane;
  const int nx = d.nx, ny = d.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int ntile = tiles_x * ((ny + TY - 1) / TY);
  // this CTA's tiles: blockIdx.x + k gridDim.x, k < cnt <= 32 (the grid is sized for
  // it).  The CTAs resident at any moment so work on one band of tiles, which keeps
  // the DRAM traffic of a moment within a few rows of each plane (measured 4% faster
  // than runs of consecutive tiles per CTA).
  const int t0 = bid, dt = nblk;
  const int cnt = (ntile - t0 + dt - 1) / dt;
  const long long tr0 = trace_start(d);
  // 16-bit storage: the step's part of every node's rounding seed (this
  // launch does not change ctr[1 - PAR])
  const unsigned seed = std::is_same<S, float>::value ? 0u : mix32((unsigned)d.ctr[1 - PAR]);
  if (MODE != 1 && bid == 0 && tid == 0) step_prologue<PAR>(d);
  constexpr int NB = L::NBUF;
  const unsigned buf0 = smem_u32(smem);
  const unsigned bar0 = buf0 + L::BAR_OFF;   // mbarrier of buffer j: bar0 + 8 j
  if ((buf0 & 127) != 0) {   // bulk tensor copies need 128-byte aligned destinations
    if (tid == 0) atomicExch(&d.stats[4], 2);
    return;
  }
  // bit k: this CTA's tile k needs its flow populations (with d.tskip: it has a
  // node that carries flow, read once, one lane per tile, by the thread that
  // issues every copy)
  unsigned fmask = 0u;
  auto issue = [&](int k, int j) {   // tile k of this CTA into buffer j
    const int t = t0 + k * dt;
    tma_issue<S, PAR, FLOW>(m, buf0 + j * L::BYTES, bar0 + 8 * j, (t % tiles_x) * TX,
                            (t / tiles_x) * TY, (fmask >> k) & 1u);
  };
  if (ty == 0) {
    // which of this CTA's tiles this launch takes, one lane per tile
    const int t = t0 + lane * dt;
    const int et = ((t / tiles_x) * TY / TE) * d.etx + (t % tiles_x) * TX / TE;
    bool take = lane < cnt;
    if (take && MODE != 0) take = takes_tile<PAR, MODE>(d, et);
    fmask = !FLOW ? 0u : d.tskip ? __ballot_sync(FULL, take && d.tact[et]) : ~0u;
    const unsigned mask = __ballot_sync(FULL, take);
    if (lane == 0) {
      *s_mask = mask;
      if (mask) {
        for (int j = 0; j < NB; ++j)
          asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * j) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        unsigned rest = mask;   // the first NB tiles fill the ring
        for (int j = 0; j < NB && rest; ++j, rest &= rest - 1) issue(__ffs(rest) - 1, j);
      }
    }
  }
  __syncthreads();
  unsigned mask = *s_mask;   // tiles not yet processed (the same in every thread)
  // tile coordinates of this CTA's k-th tile, advanced tile by tile
  const int gq = dt / tiles_x, gr = dt - gq * tiles_x;
  int cur_k = 0, ctx = t0 % tiles_x, cty = t0 / tiles_x;
  unsigned phases = 0u;      // bit j: phase parity the next wait on buffer j expects
  bool failed = false;
  int b = 0;                 // buffer of the current tile (tiles take the buffers in turn)
  for (; mask; b = (b + 1 == NB) ? 0 : b + 1) {
    const int k = __ffs(mask) - 1;
    mask &= mask - 1;
    const unsigned bar = bar0 + 8 * b;
    const bool ok = mbar_wait(bar, (phases >> b) & 1u);
    if (__syncthreads_or(!ok)) {   // the whole CTA gives up together
      failed = true;
      break;
    }
    phases ^= 1u << b;
    const unsigned char* sb = smem + b * L::BYTES;
    for (; cur_k < k; ++cur_k) {
      ctx += gr;
      cty += gq;
      if (ctx >= tiles_x) {
        ctx -= tiles_x;
        ++cty;
      }
    }
    const int x0 = ctx * TX, y0 = cty * TY;
    const int y = y0 + ty;
    // interior tiles (no wall node and no wall neighbour in them) take a copy
    // of the update with the wall logic compiled out
    const bool edge = x0 < 2 || x0 + TX > nx - 2 || y0 < 2 || y0 + TY > ny - 2;
    const bool unsafe = edge ? tma_node<S, PAR, FLOW, true>(d, sb, x0, y0, lane, ty, seed)
                             : tma_node<S, PAR, FLOW, false>(d, sb, x0, y0, lane, ty, seed);
    if (__any_sync(FULL, unsafe) && lane == 0)
      mark_tile(d, ((unsigned)y / TE) * d.etx + (unsigned)x0 / TE, PAR);
    // every thread is done with buffer b before it is refilled with the tile
    // NB places further on
    __syncthreads();
    if (tid == 0) {
      unsigned nxt = mask;   // the next NB - 1 tiles are already in flight
      for (int j = 0; j < NB - 1 && nxt; ++j) nxt &= nxt - 1;
      if (nxt) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(__ffs(nxt) - 1, b);
      }
    }
  }
  if (failed) {
    // a copy did not arrive in time: report it, and give the copies still in
    // flight a bounded chance to land before the shared memory is released
    if (tid == 0) atomicExch(&d.stats[4], 1);
    unsigned pend = mask;
    mbar_wait(bar0 + 8 * b, (phases >> b) & 1u);
    for (int j = 1; j < NB && pend; ++j, pend &= pend - 1) {
      const int bj = (b + j) % NB;
      mbar_wait(bar0 + 8 * bj, (phases >> bj) & 1u);
    }
  }
  // (ctr[1 - PAR] + 1: the step this launch computes; no launch of the step changes it)
  if (tid == 0 && d.trace) trace_end(d, 100 * PAR + 10 + MODE, d.ctr[1 - PAR] + 1, tr0);
}

template <typename S, int PAR, int FLOW, int MODE>
__global__ void __launch_bounds__(TX* TY, TMA_MIN_CTAS)
    fused_tma_kernel(Dev d, const __grid_constant__ TmaMaps m) {
  fused_tma_body<S, PAR, FLOW, MODE>(d, m, (int)blockIdx.x, (int)gridDim.x);
}

// The same pass over every lattice of a batch in one launch: each lattice's
// CTAs are a range of the grid, its parameters one entry of the plan, its
// tensor maps one entry of a device array.
template <typename S, int PAR, int FLOW, int MODE>
__global__ void __launch_bounds__(TX* TY, TMA_MIN_CTAS)
    fused_tma_batch_kernel(const __grid_constant__ BatchPlan P, const TmaMaps* __restrict__ maps) {
  const int c = plan_lattice(P, (int)blockIdx.x);
  fused_tma_body<S, PAR, FLOW, MODE>(P.d[c], maps[c], (int)blockIdx.x - P.start[c],
                                     P.start[c + 1] - P.start[c]);
}

// ---- launches ------------------------------------------------------------------

// FLOW: 0 no flow lattice, 1 flow, 2 flow with the front extrapolation
template <typename S, int MODE>
static void launch_mode(const Dev& d, int parity, dim3 grid, dim3 block, cudaStream_t s) {
  if (d.flow && d.flow_front) {
    if (parity == 0) fused_step_kernel<S, 0, 2, MODE><<<grid, block, 0, s>>>(d);
    else fused_step_kernel<S, 1, 2, MODE><<<grid, block, 0, s>>>(d);
  } else if (d.flow) {
    if (parity == 0) fused_step_kernel<S, 0, 1, MODE><<<grid, block, 0, s>>>(d);
    else fused_step_kernel<S, 1, 1, MODE><<<grid, block, 0, s>>>(d);
  } else {
    if (parity == 0) fused_step_kernel<S, 0, 0, MODE><<<grid, block, 0, s>>>(d);
    else fused_step_kernel<S, 1, 0, MODE><<<grid, block, 0, s>>>(d);
  }
}

template <typename S, int PAR, int FLOW, int MODE>
static void launch_tma_one(const Dev& d, const TmaMaps& m, cudaStream_t s) {
  const size_t sm = TmaLayout<PAR, S>::SMEM;
  fused_tma_kernel<S, PAR, FLOW, MODE><<<d.tgrid, dim3(TX, TY), sm, s>>>(d, m);
}

template <typename S, int MODE>
static void launch_tma_mode(const Dev& d, const TmaMaps& m, int parity, cudaStream_t s) {
  if (d.flow && d.flow_front) {
    if (parity == 0) launch_tma_one<S, 0, 2, MODE>(d, m, s);
    else launch_tma_one<S, 1, 2, MODE>(d, m, s);
  } else if (d.flow) {
    if (parity == 0) launch_tma_one<S, 0, 1, MODE>(d, m, s);
    else launch_tma_one<S, 1, 1, MODE>(d, m, s);
  } else {
    if (parity == 0) launch_tma_one<S, 0, 0, MODE>(d, m, s);
    else launch_tma_one<S, 1, 0, MODE>(d, m, s);
  }
}

// the stream-collide launch for population storage S (see launch_fused)
template <typename S>
static void launch_fused_t(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  if (m) {
    if (mode == 0) launch_tma_mode<S, 0>(d, *m, parity, s);
    else if (mode == 1) launch_tma_mode<S, 1>(d, *m, parity, s);
    else launch_tma_mode<S, 2>(d, *m, parity, s);
    return;
  }
  dim3 block(TX, TY), grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY);
  if (mode == 0) launch_mode<S, 0>(d, parity, grid, block, s);
  else if (mode == 1) launch_mode<S, 1>(d, parity, grid, block, s);
  else launch_mode<S, 2>(d, parity, grid, block, s);
}

// encode one tiled tensor map over a [planes][ny][nx] array of esize-byte elements
bool tma_encode(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, int rank,
                int nx, int ny, int planes, int bx, int by);

// Fill *m with the tensor maps of this context's arrays (populations of
// storage S, tensor-map element type dt) and size the grid; false if the
// lattice does not qualify or encoding fails.
template <typename S>
static bool tma_setup_t(Dev& d, TmaMaps* m, CUtensorMapDataType dt) {
  constexpr int es = (int)sizeof(S);
  constexpr int WXS = TmaLayout<1, S>::PX;   // odd-step population box width
  // 16-byte row strides; every box no wider than the lattice
  if (d.per_x || d.per_y || (d.nx * es) % 16 != 0) return false;
  if (d.nx < WX || d.nx < WXS || d.ny < WY) return false;
  const bool ok = tma_encode(&m->f_even, d.f, dt, es, 3, d.nx, d.ny, 9, TX, TY) &&
                  tma_encode(&m->f_odd, d.f, dt, es, 3, d.nx, d.ny, 9, WXS, WY) &&
                  tma_encode(&m->g_even, d.g, dt, es, 3, d.nx, d.ny, 5, TX, TY) &&
                  tma_encode(&m->g_odd, d.g, dt, es, 3, d.nx, d.ny, 5, WXS, WY) &&
                  tma_encode(&m->fl, d.fl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d.nx, d.ny, 1,
                             WX, WY) &&
                  tma_encode(&m->phi, d.phi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d.nx, d.ny, 1,
                             TX, TY) &&
                  tma_encode(&m->K, d.K, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, 2, d.nx, d.ny, 1, TX,
                             TY);
  if (!ok) return false;
  const int s0 = TmaLayout<0, S>::SMEM, s1 = TmaLayout<1, S>::SMEM;
#define LBM_SMEM(P, FL, MO, SM)                                                      \
  cudaFuncSetAttribute(fused_tma_kernel<S, P, FL, MO>,                               \
                       cudaFuncAttributeMaxDynamicSharedMemorySize, SM)
  LBM_SMEM(0, 2, 0, s0); LBM_SMEM(0, 2, 1, s0); LBM_SMEM(0, 2, 2, s0);
  LBM_SMEM(0, 1, 0, s0); LBM_SMEM(0, 1, 1, s0); LBM_SMEM(0, 1, 2, s0);
  LBM_SMEM(0, 0, 0, s0); LBM_SMEM(0, 0, 1, s0); LBM_SMEM(0, 0, 2, s0);
  LBM_SMEM(1, 2, 0, s1); LBM_SMEM(1, 2, 1, s1); LBM_SMEM(1, 2, 2, s1);
  LBM_SMEM(1, 1, 0, s1); LBM_SMEM(1, 1, 1, s1); LBM_SMEM(1, 1, 2, s1);
  LBM_SMEM(1, 0, 0, s1); LBM_SMEM(1, 0, 1, s1); LBM_SMEM(1, 0, 2, s1);
#undef LBM_SMEM
  int per0 = 0, per1 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per0, fused_tma_kernel<S, 0, 1, 0>, TX * TY,
                                                s0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, fused_tma_kernel<S, 1, 1, 0>, TX * TY,
                                                s1);
  if (cudaGetLastError() != cudaSuccess || per0 <= 0 || per1 <= 0) return false;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return false;
  d.tslots = sms * (per0 < per1 ? per0 : per1);
  d.tgrid = tma_grid(d, TMA_TPC);
  return true;
}

}  // namespace lbm
