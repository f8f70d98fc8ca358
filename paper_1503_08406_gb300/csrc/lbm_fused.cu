// Fused stream-collide of both lattices for one time step (AA pattern, in place).
//
// One thread per node.  Per non-wall node:
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
//      and mark the enthalpy tiles that must be solved.
// The latent source of the step is added afterwards by the enthalpy kernels.
//
// Phase-change screen.  The temperature a node y sees after streaming is
// T*(y) = sum_i g+_i(y - e_i).  If y and its four neighbours are all solid
// (f_l = 0) and every outgoing population satisfies g+_i <= w~_i T_s, then
// T*(y) <= T_s and y stays solid; likewise all liquid with g+_i >= w~_i T_l.
// Every node failing both tests puts the enthalpy tiles of its 3x3
// neighbourhood on the step's work list; only listed tiles run the enthalpy
// solve.  The tests allow a
// margin of 1e-7 of the temperature scale (and f_l within 1e-7 of 0 or 1):
// without it, the sub-1e-30 values that diffusion carries ahead of a front at
// the lattice speed would mark every tile they reach.  A node skipped this way
// can lag the exact fixed point by at most that margin; the enthalpy sum is
// unaffected, and the node is solved as soon as it leaves the margin.
#include "lbm_internal.cuh"

namespace lbm {

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

template <int PAR, bool FLOW, int MODE>
__global__ void __launch_bounds__(TX* TY, 4) fused_step_kernel(Dev d) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  if (MODE != 1 && blockIdx.x == 0 && blockIdx.y == 0 && lane == 0 && threadIdx.y == 0) {
    // once per step (the near-tile launch runs after the previous step's
    // enthalpy kernels, the last readers of the other list): stamp the step
    // and empty the next step's list
    d.ctr[PAR] = d.ctr[1 - PAR] + 1;
    d.lcount[1 - PAR] = 0;
  }
  if (MODE != 0) {
    // split step: this launch takes the CTAs on one side of the previous
    // step's near map (entries carry the stamp of the step that set them)
    const int prev = d.ctr[1 - PAR];
    const int et = ((blockIdx.y * TY) / TE) * d.etx + (blockIdx.x * TX) / TE;
    const bool nr = d.nearmap[(1 - PAR) * d.ntiles + et] == prev;
    if ((MODE == 1) == nr) return;
  }
  const int x = blockIdx.x * TX + lane, y = blockIdx.y * TY + threadIdx.y;
  const int nx = d.nx, ny = d.ny;
  if (y >= ny) return;  // whole warp: one warp is one row segment
  const bool inside = x < nx;
  const bool node = inside && !is_wall(d, x, y);
  bool unsafe = false;
  if (node) {
    const int n = (int)d.n;
    const int s = y * nx + x;
    // neighbours of a non-wall node are one step away: one wrap at most
    const int xm = (x == 0) ? nx - 1 : x - 1, xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1, yp = (y == ny - 1) ? 0 : y + 1;
    const int sE = y * nx + xp, sW = y * nx + xm;
    const int sN = yp * nx + x, sS = ym * nx + x;
    const int nb[9] = {s, sE, sN, sW, sS, yp * nx + xp, yp * nx + xm, ym * nx + xm, ym * nx + xp};
    // which neighbours are wall nodes
    const bool cE = d.wall_r && xp == nx - 1, cW = d.wall_l && xm == 0;
    const bool rN = d.wall_t && yp == ny - 1, rS = d.wall_b && ym == 0;
    const bool wl[9] = {false, cE, rN, cW, rS, cE || rN, cW || rN, cW || rS, cE || rS};
    // f_l of the 3x3 neighbourhood (L1 hits for all but the node's own row);
    // -1 marks a wall
    const float* FL = d.fl;
    float fln[9];
    fln[0] = FL[s];
#pragma unroll
    for (int i = 1; i < 9; ++i) fln[i] = wl[i] ? -1.f : FL[nb[i]];
    const float c0 = fln[0], e0 = fln[1], cN = fln[2], w0 = fln[3], cS = fln[4];
    const float flc = c0;

    // ---- thermal gather -------------------------------------------------
    float* G = d.g;
    float g0, g1, g2, g3, g4;
    if (PAR == 0) {
      g0 = G[s]; g1 = G[n + s]; g2 = G[2 * n + s]; g3 = G[3 * n + s]; g4 = G[4 * n + s];
    } else {
      g0 = G[s];
      g1 = G[3 * n + sW];   // population E comes from the west neighbour's W slot
      g2 = G[4 * n + sS];
      g3 = G[1 * n + sE];
      g4 = G[2 * n + sN];
    }
    const float T = g0 + g1 + g2 + g3 + g4;

    // ---- flow lattice ----------------------------------------------------
    // All loads of the node are issued before any of them is used, so one
    // memory round trip covers the step: the populations are read whether or
    // not the node carries flow, and on odd steps both candidate slots of each
    // direction (streamed from the neighbour, or reflected at the link) are
    // read and chosen once the neighbours' activity is known.
    float ux = 0.f, uy = 0.f;
    float f[9], fb[9];
    float phi = 0.f, K = 1.f;
    float* F = d.f;
    if (FLOW) {
      phi = d.phi[s];
      K = d.K[s];
      if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = F[i * n + s];
      } else {
        f[0] = F[s];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int o = opp9(i);
          f[i] = F[o * n + nb[o]];   // from the source node x - e_i (direction opp(i) from x)
          fb[i] = F[i * n + s];      // reflected at the link x - e_i | x
        }
      }
    }
    if (FLOW && flc >= d.f_act) {
      const float fa = d.f_act;
      // neighbour flow activity, directions 1..8 (E, N, W, S, NE, NW, SW, SE)
      bool act[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) act[i] = fln[i] >= fa;
      if (PAR == 1) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          if (!act[opp9(i)]) f[i] = fb[i];
      }
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
      float fp[9];
      fp[0] = f[0] - 4.f * a1 + 4.f * a2;
      fp[1] = f[1] + c_ax + a3 - 2.f * a4 + a7;
      fp[2] = f[2] + c_ax + a5 - 2.f * a6 - a7;
      fp[3] = f[3] + c_ax - a3 + 2.f * a4 + a7;
      fp[4] = f[4] + c_ax - a5 + 2.f * a6 - a7;
      fp[5] = f[5] + c_dg + a3 + a4 + a5 + a6 + a8;
      fp[6] = f[6] + c_dg - a3 - a4 + a5 + a6 - a8;
      fp[7] = f[7] + c_dg - a3 - a4 - a5 - a6 + a8;
      fp[8] = f[8] + c_dg + a3 + a4 - a5 - a6 - a8;
      if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) F[opp9(i) * n + s] = fp[i];
      } else {
        F[s] = fp[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          // into a node without flow: halfway bounce-back into our own slot
          const int off = act[i] ? i * n + nb[i] : opp9(i) * n + s;
          F[off] = fp[i];
        }
      }
    }

    // ---- thermal collision (no latent source) ----------------------------
    const float n1 = g1 - g3, n2 = g2 - g4;
    const float n3 = -4.f * g0 + g1 + g2 + g3 + g4;
    const float n4 = g1 - g2 + g3 - g4;
    const float th = d.conv * d.csT2;   // vartheta / sigma
    const float b1 = -0.5f * d.z_a * (n1 - th * ux * T);
    const float b2 = -0.5f * d.z_a * (n2 - th * uy * T);
    const float b3 = -0.05f * d.z_e * (n3 - d.varpi * T);
    const float b4 = -0.25f * d.z_nu * n4;
    const float gp0 = g0 - 4.f * b3;
    const float gp1 = g1 + b1 + b3 + b4;
    const float gp2 = g2 + b2 + b3 - b4;
    const float gp3 = g3 - b1 + b3 + b4;
    const float gp4 = g4 - b2 + b3 - b4;
    if (PAR == 0) {
      G[s] = gp0; G[3 * n + s] = gp1; G[4 * n + s] = gp2; G[n + s] = gp3; G[2 * n + s] = gp4;
    } else {
      G[s] = gp0; G[n + sE] = gp1; G[2 * n + sN] = gp2; G[3 * n + sW] = gp3; G[4 * n + sS] = gp4;
    }

    // ---- phase-change screen (own populations) ---------------------------
    bool cold = (flc <= d.scr_f), hot = (flc >= 1.f - d.scr_f);
    {
      const float nbv[4] = {e0, cN, w0, cS};
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

    // ---- thermal walls: inward population of adjacent wall nodes ----------
    // wall on side S at x_b = x - e_k, inward direction k; geq_k(T,u) = w~ T (1 + conv e_k.u)
    const float cv = d.conv;
#define LBM_WALL_POP(COND, K, SB, TW, EU)                                         \
  if (COND) {                                                                     \
    const float gpk = (K == 1) ? gp1 : (K == 2) ? gp2 : (K == 3) ? gp3 : gp4;     \
    const float w = d.wt1 * (TW) + gpk - d.wt1 * T * (1.f + cv * (EU));           \
    if (PAR == 0) G[opp5(K) * n + (SB)] = w;                                      \
    else G[(K) * n + s] = w;                                                      \
    cold = cold && (w <= d.wt1 * (d.T_s + d.scr_T));                              \
    hot = hot && (w >= d.wt1 * (d.T_l - d.scr_T));                                \
  }
    LBM_WALL_POP(d.wall_l && x == 1, 1, sW, d.bc[0] == 1 ? d.wallTl[y] : T, ux)
    LBM_WALL_POP(d.wall_r && x == nx - 2, 3, sE, d.bc[1] == 1 ? d.Tbc[1] : T, -ux)
    LBM_WALL_POP(d.wall_b && y == 1, 2, sS, d.bc[2] == 1 ? d.Tbc[2] : T, uy)
    LBM_WALL_POP(d.wall_t && y == ny - 2, 4, sN, d.bc[3] == 1 ? d.Tbc[3] : T, -uy)
#undef LBM_WALL_POP

    unsafe = d.screen_off || !(cold || hot);
    if (unsafe) {
      // mark the enthalpy tiles holding this node's 3x3 neighbourhood (other
      // than its own, which the warp vote below marks)
      const int cx = x / TE, cy = y / TE;
      const int txs[3] = {xm / TE, cx, xp / TE};
      const int tys[3] = {ym / TE, cy, yp / TE};
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (txs[i] != cx || tys[j] != cy) mark_tile(d, tys[j] * d.etx + txs[i], PAR);
    }
  }
  if (__any_sync(FULL, unsafe) && lane == 0)
    mark_tile(d, (y / TE) * d.etx + (blockIdx.x * TX) / TE, PAR);
}

template <int MODE>
static void launch_mode(const Dev& d, int parity, dim3 grid, dim3 block, cudaStream_t s) {
  if (d.flow) {
    if (parity == 0) fused_step_kernel<0, true, MODE><<<grid, block, 0, s>>>(d);
    else fused_step_kernel<1, true, MODE><<<grid, block, 0, s>>>(d);
  } else {
    if (parity == 0) fused_step_kernel<0, false, MODE><<<grid, block, 0, s>>>(d);
    else fused_step_kernel<1, false, MODE><<<grid, block, 0, s>>>(d);
  }
}

void launch_fused(const Dev& d, int parity, int mode, cudaStream_t s) {
  dim3 block(TX, TY), grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY);
  if (mode == 0) launch_mode<0>(d, parity, grid, block, s);
  else if (mode == 1) launch_mode<1>(d, parity, grid, block, s);
  else launch_mode<2>(d, parity, grid, block, s);
}

}  // namespace lbm
