// Iterative enthalpy method for f_l(n+1) and the latent-heat source, Eq. (38),
// (40)-(42) and the inner iteration of Sec. 3.2.
//
// The fused kernel streamed the source-free thermal populations, so a node y
// sees T*(y) = sum_i g_i(y).  The latent source S~ = (S0, 0, 0, varpi S0, 0)
// of node x, S0 = -a(x) (f_l(n+1) - f_l(n)), a = phi dT / (sigma St), adds
// N^-1 S~ = S0 w~ to the post-collision populations of x, which stream to the
// neighbours: T(y) = T*(y) + sum_i w~_i S0(y - e_i).  With h = T + a f_l, the
// enthalpy relation f_l = clamp((h - T_s)/(T_l - T_s + a), 0, 1) is solved for
// f_l(n+1) as a fixed point.
//
// Work list.  The fused kernel appends every 32x32 tile that may hold a phase
// change this step to list[parity] (a tile flag de-duplicates).  Both kernels
// below run a fixed grid of CTAs that walk that list, so steps with no front
// cost almost nothing.  Per-tile status words carry a step stamp (a counter the
// fused kernel advances), so nothing needs clearing between steps.
//
// enthalpy_solve: per listed tile, load T*, f_l(n) and a on the tile plus an
// 8-node halo into shared memory and run red-black Gauss-Seidel sweeps; each
// node update solves its own term exactly,
//   f(x) = clamp((T*(x) + w~_0 a f_l(n) - T_s - w~_1 sum_{i>0} q(x - e_i)) / (T_l - T_s + w~_0 a), 0, 1),
//   q = a (f - f_l(n)),
// which has the same fixed point as the plain iteration (the map is monotone
// with slope < 1).  Sweeps stop when no node moves by more than about four
// float32 ulps of its value and of the terms it is computed from: Gauss-Seidel
// from f_l(n) approaches the fixed point from one side, so a looser stop would
// bias every step the same way, and a tighter one can chase a rounding cycle
// forever (at the melting threshold v is a small difference of two larger
// terms).  Two more sweeps follow the stop, which shrink what is left of the
// one-sided error down to rounding noise.  Nodes outside
// the halo keep f = f_l(n).  The tile's own results go to scratch as
// (f_l(n), f_l(n+1)).
//
// enthalpy_commit: per listed tile, store f_l(n+1), add the streamed source of
// every changed node to the five populations it reaches, and, before an odd
// step, swap the two slots of every flow link whose "both ends carry flow"
// state changed, so the AA layout matches the new flow mask.
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

// Over-relaxation factor of the projected SOR sweeps.  The Jacobi map of the
// self-solved update has spectral radius at most 4 w~_1 a / (T_l - T_s + w~_0 a),
// which is 2/3 with the paper's varpi = -2; red-black SOR on this diagonally
// dominant system converges for 0 < omega < 2, fastest near 2 / (1 + sqrt(1 - rho^2))
// (about 1.15 - 1.3).  The fixed point does not depend on omega.
constexpr float SOR_OMEGA = 1.15f;
constexpr int SOR_SWEEPS = 8;   // over-relaxed sweeps before plain Gauss-Seidel

__device__ __forceinline__ int stamp_of(const Dev& d, int par) { return d.ctr[par] & 0x0FFFFFFF; }
__device__ __forceinline__ bool solved(const Dev& d, int tile, int stamp) {
  return (d.proc[tile] >> 3) == stamp;
}

// T* at node (x, y) from the populations after the step, stored as S:
// natural layout (layout 0) or swapped (layout 1, population i of x sits in
// x - e_i).  Neighbours one step away (xm, xp, ym, yp) wrap once at most.
template <typename S>
__device__ __forceinline__ float tstar_t(const Dev& d, int s, int xm, int xp, int ym, int yp,
                                         int x, int y, int layout) {
  const int n = (int)d.n;
  const S* G = static_cast<const S*>(d.g);
  // the stored g deviations add up to T* - T_m (the weights sum to 1)
  const float ref = std::is_same<S, float>::value ? 0.f : d.g_ref;
  if (layout == 0)
    return Pop<S>::ld(G + s) + Pop<S>::ld(G + n + s) + Pop<S>::ld(G + 2 * n + s) +
           Pop<S>::ld(G + 3 * n + s) + Pop<S>::ld(G + 4 * n + s) + ref;
  return Pop<S>::ld(G + s) + Pop<S>::ld(G + 3 * n + y * d.nx + xm) +
         Pop<S>::ld(G + 4 * n + ym * d.nx + x) + Pop<S>::ld(G + n + y * d.nx + xp) +
         Pop<S>::ld(G + 2 * n + yp * d.nx + x) + ref;
}

// bar.sync / bar.red.or on named barrier 1 over the first `threads` threads
__device__ __forceinline__ void sub_sync(int threads) {
  asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}
__device__ __forceinline__ bool sub_sync_or(int threads, bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((unsigned)v), "r"(threads)
      : "memory");
  return r != 0;
}

// CTA bid of nblk (the whole grid of a single lattice's launch, a range of a
// batched one) takes listed tiles bid, bid + nblk, ...
template <int PAR, typename S, int EB>
__device__ __forceinline__ void enthalpy_solve_body(const Dev& d, int bid, int nblk) {
  const long long tr0 = trace_start(d);
  constexpr int LAYOUT = 1 - PAR;
  extern __shared__ float smem[];
  float* sbase = smem;               // T* + w~0 a f_l(n) - T_s
  float* sinv = sbase + RE * RE;     // 1 / (T_l - T_s + w~0 a); 0 on fixed nodes
  float* sa = sinv + RE * RE;        // a; 0 on walls and outside
  float* sfn = sa + RE * RE;         // f_l(n)
  float* sq = sfn + RE * RE;         // a (f - f_l(n))
  float* sf = sq + RE * RE;          // current iterate
  __shared__ int sbox[4];            // box of the nodes the sweeps update: x0, x1, y0, y1
  const int tid = threadIdx.x;
  const int cnt = d.lcount[PAR];
  const int stamp = stamp_of(d, PAR);
  const float w0 = d.wt0, w1 = d.wt1, Ts = d.T_s, dTt = d.dTt;
  for (int li = bid; li < cnt; li += nblk) {
    const int tile = d.list[PAR * d.ntiles + li];
    const int X0 = (tile % d.etx) * TE, Y0 = (tile / d.etx) * TE;
    // a region (tile and halo) inside the wall ring needs no wrapping and holds
    // no wall node: its loads go straight to their addresses
    const bool inner = X0 - RH >= 1 && X0 + TE + RH <= d.nx - 1 && Y0 - RH >= 1 &&
                       Y0 + TE + RH <= d.ny - 1;
    if (inner) {
      // every thread's nodes loaded in one go (all loads in flight together)
      constexpr int NK = (RE * RE + EB - 1) / EB;
      float fnv[NK], phv[NK], Tv[NK];
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        const int k = tid + j * EB;
        if (k < RE * RE) {
          const int ly = k / RE, lx = k - ly * RE;
          const int gx = X0 - RH + lx, gy = Y0 - RH + ly;
          const int s = gy * d.nx + gx;
          fnv[j] = d.fl[s];
          phv[j] = d.phi[s];
          Tv[j] = tstar_t<S>(d, s, gx - 1, gx + 1, gy - 1, gy + 1, gx, gy, LAYOUT);
        }
      }
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        const int k = tid + j * EB;
        if (k < RE * RE) {
          const float fn = fnv[j];
          const float a = phv[j] * d.lat * sigma_ratio(d, fn);   // phi dT / (sigma(f_l(n)) St)
          sbase[k] = Tv[j] + w0 * a * fn - Ts;
          sinv[k] = 1.f / (dTt + w0 * a);
          sa[k] = a;
          sfn[k] = fn;
          sq[k] = 0.f;
          sf[k] = fn;
        }
      }
    } else {
#pragma unroll 3
      for (int k = tid; k < RE * RE; k += EB) {
        const int ly = k / RE, lx = k - ly * RE;
        const int gx = wrapx(d, X0 - RH + lx), gy = wrapy(d, Y0 - RH + ly);
        float base = 0.f, inv = 0.f, a = 0.f, fn = 0.f;
        if (gx >= 0 && gy >= 0) {
          const int s = gy * d.nx + gx;
          fn = d.fl[s];
          if (!is_wall(d, gx, gy)) {
            a = d.phi[s] * d.lat * sigma_ratio(d, fn);   // phi dT / (sigma(f_l(n)) St)
            const int xm = (gx == 0) ? d.nx - 1 : gx - 1, xp = (gx == d.nx - 1) ? 0 : gx + 1;
            const int ym = (gy == 0) ? d.ny - 1 : gy - 1, yp = (gy == d.ny - 1) ? 0 : gy + 1;
            base = tstar_t<S>(d, s, xm, xp, ym, yp, gx, gy, LAYOUT) + w0 * a * fn - Ts;
            inv = 1.f / (dTt + w0 * a);
          }
        }
        sbase[k] = base;
        sinv[k] = inv;
        sa[k] = a;
        sfn[k] = fn;
        sq[k] = 0.f;
        sf[k] = fn;
      }
    }
    __syncthreads();
    // Nodes whose update is clamped whatever their neighbours do are fixed now
    // and left out of the sweeps: with q_j in [-a_j f_l(n)_j, a_j (1 - f_l(n)_j)],
    // the unclamped value (b - w~_1 sum_j q_j) inv stays <= 0 (or >= 1) when it
    // does so at the extreme sum.  The sweeps then cover only the bounding box of
    // the nodes left (a band along the front); the fixed point is unchanged.
    if (tid == 0) {
      sbox[0] = RE;
      sbox[1] = -1;
      sbox[2] = RE;
      sbox[3] = -1;
    }
    __syncthreads();
    {
      int bx0 = RE, bx1 = -1, by0 = RE, by1 = -1;
      for (int k = tid; k < RE * RE; k += EB) {
        const float inv = sinv[k];
        if (inv == 0.f) continue;
        const int ly = k / RE, lx = k - ly * RE;
        float nlo = 0.f, nhi = 0.f;   // extreme neighbour sums of q
        auto acc = [&](int j) {
          nlo -= sa[j] * sfn[j];
          nhi += sa[j] * (1.f - sfn[j]);
        };
        if (lx > 0) acc(k - 1);
        if (lx < RE - 1) acc(k + 1);
        if (ly > 0) acc(k - RE);
        if (ly < RE - 1) acc(k + RE);
        const float b = sbase[k];
        const float hi_raw = (b - w1 * nlo) * inv, lo_raw = (b - w1 * nhi) * inv;
        float v = -1.f;
        if (hi_raw < -1e-6f) v = 0.f;            // clamped to 0 for any neighbour values
        else if (lo_raw > 1.f + 1e-6f) v = 1.f;  // clamped to 1
        if (v >= 0.f) {
          sf[k] = v;
          sq[k] = sa[k] * (v - sfn[k]);
          sinv[k] = 0.f;
        } else {
          bx0 = min(bx0, lx);
          bx1 = max(bx1, lx);
          by0 = min(by0, ly);
          by1 = max(by1, ly);
        }
      }
      bx0 = __reduce_min_sync(0xffffffffu, bx0);
      bx1 = __reduce_max_sync(0xffffffffu, bx1);
      by0 = __reduce_min_sync(0xffffffffu, by0);
      by1 = __reduce_max_sync(0xffffffffu, by1);
      if ((tid & 31) == 0 && bx1 >= 0) {
        atomicMin(&sbox[0], bx0);
        atomicMax(&sbox[1], bx1);
        atomicMin(&sbox[2], by0);
        atomicMax(&sbox[3], by1);
      }
    }
    __syncthreads();
    const int lx0 = sbox[0], ly0 = sbox[2];
    const int ncol = sbox[1] >= lx0 ? (sbox[1] - lx0 + 2) >> 1 : 0;   // per colour and row
    const int nbox = ncol * (sbox[3] - ly0 + 1);
    const float inv_ncol = ncol ? 1.f / (float)ncol : 0.f;
    // the sweeps run on as many whole warps as one colour of the box needs;
    // the other warps wait at the barrier after them
    const int sw = min(EB, (nbox + 31) & ~31);
    int it = 0;
    bool more = sw > 0;   // (nothing left to sweep: solved by the fixing pass)
    int polish = more ? 2 : 0;   // extra sweeps after the stop test passes
    if (nbox <= EB) {
      // One node per colour and thread: each sweeping thread keeps its two
      // nodes' place (packed with which neighbours lie in the region),
      // coefficients and current value in registers, so that a sweep only
      // exchanges q through shared memory.
      int kk[2];
      float cb[2], cinv[2], ca[2], cfn[2], cf[2];
#pragma unroll
      for (int color = 0; color < 2; ++color) {
        int k = -1;
        if (tid < nbox) {
          // (row, column pair) of the box; exact for j < 2^16 and ncol <= 24
          const int r = (int)(((float)tid + 0.5f) * inv_ncol);
          const int ly = ly0 + r;
          const int lx = lx0 + ((lx0 + ly + color) & 1) + 2 * (tid - r * ncol);
          if (lx < RE) {
            k = ly * RE + lx;
            if (sinv[k] == 0.f) k = -1;   // wall, outside, or fixed above
            else
              k |= ((lx > 0) | ((lx < RE - 1) << 1) | ((ly > 0) << 2) | ((ly < RE - 1) << 3)) << 16;
          }
        }
        const int q = k & 0xffff;
        const float inv = k >= 0 ? sinv[q] : 0.f;
        kk[color] = k;
        cb[color] = k >= 0 ? sbase[q] : 0.f;
        cinv[color] = inv;
        ca[color] = k >= 0 ? sa[q] : 0.f;
        cfn[color] = k >= 0 ? sfn[q] : 0.f;
        cf[color] = k >= 0 ? sf[q] : 0.f;
      }
      if (tid < sw)
        for (; it < d.max_inner && (more || polish > 0); ++it) {
          if (!more) --polish;
          // over-relaxed for the first sweeps, then plain Gauss-Seidel: at the last
          // few ulps over-relaxation can cycle instead of meeting the stop test
          const float om = (more && it < SOR_SWEEPS) ? SOR_OMEGA : 1.f;
          bool changed = false;
#pragma unroll
          for (int color = 0; color < 2; ++color) {
            const int k = kk[color];
            if (k >= 0) {
              const int q = k & 0xffff;
              const int m = k >> 16;
              float nb = 0.f;
              if (m & 1) nb += sq[q - 1];
              if (m & 2) nb += sq[q + 1];
              if (m & 4) nb += sq[q - RE];
              if (m & 8) nb += sq[q + RE];
              const float fo = cf[color];
              const float raw = (cb[color] - w1 * nb) * cinv[color];
              float v = (om == 1.f) ? raw : fo + om * (raw - fo);
              v = fminf(fmaxf(v, 0.f), 1.f);
              // converged at about four ulps of v and of the terms that make it
              const float tol =
                  4.8e-7f * (v + (fabsf(cb[color]) + w1 * fabsf(nb)) * cinv[color]);
              if (fabsf(v - fo) > tol) changed = true;
              cf[color] = v;
              // (a (v - f_l(n)) is exactly 0 on a node that does not move: a
              // spurious source there would cost a rounding of its neighbours'
              // 16-bit populations in the commit)
              sq[q] = ca[color] * (v - cfn[color]);
            }
            // the second colour's barrier also collects the convergence vote
            if (color == 0) sub_sync(sw);
          }
          const bool c = sub_sync_or(sw, changed);
          if (more) more = c;
        }
#pragma unroll
      for (int color = 0; color < 2; ++color)
        if (kk[color] >= 0) sf[kk[color] & 0xffff] = cf[color];
    } else if (tid < sw) {
      for (; it < d.max_inner && (more || polish > 0); ++it) {
        if (!more) --polish;
        const float om = (more && it < SOR_SWEEPS) ? SOR_OMEGA : 1.f;
        bool changed = false;
#pragma unroll
        for (int color = 0; color < 2; ++color) {
          for (int j = tid; j < nbox; j += EB) {
            const int r = (int)(((float)j + 0.5f) * inv_ncol);
            const int ly = ly0 + r;
            const int lx = lx0 + ((lx0 + ly + color) & 1) + 2 * (j - r * ncol);
            if (lx >= RE) continue;
            const int k = ly * RE + lx;
            const float inv = sinv[k];
            if (inv == 0.f) continue;   // wall, outside, or fixed above
            const float a = sa[k];
            float nb = 0.f;
            if (lx > 0) nb += sq[k - 1];
            if (lx < RE - 1) nb += sq[k + 1];
            if (ly > 0) nb += sq[k - RE];
            if (ly < RE - 1) nb += sq[k + RE];
            const float b = sbase[k];
            const float fo = sf[k];
            const float raw = (b - w1 * nb) * inv;
            float v = (om == 1.f) ? raw : fo + om * (raw - fo);
            v = fminf(fmaxf(v, 0.f), 1.f);
            const float tol = 4.8e-7f * (v + (fabsf(b) + w1 * fabsf(nb)) * inv);
            if (fabsf(v - fo) > tol) changed = true;
            sf[k] = v;
            sq[k] = a * (v - sfn[k]);
          }
          if (color == 0) sub_sync(sw);
        }
        const bool c = sub_sync_or(sw, changed);
        if (more) more = c;
      }
    }
    __syncthreads();
    bool fchg = false, achg = false;
    for (int k = tid; k < TE * TE; k += EB) {
      const int ly = k / TE, lx = k - ly * TE;
      const int gx = X0 + lx, gy = Y0 + ly;
      if (gx >= d.nx || gy >= d.ny) continue;
      const int r = (ly + RH) * RE + (lx + RH);
      const float fo = sfn[r], fnw = sf[r];
      d.scr[gy * d.nx + gx] = make_float2(fo, fnw);
      if (fnw != fo) {
        fchg = true;
        if ((fo >= d.f_act) != (fnw >= d.f_act)) achg = true;
      }
    }
    const int bits = 1 | (__syncthreads_or(fchg) ? 2 : 0) | (__syncthreads_or(achg) ? 4 : 0);
    if (tid == 0) {
      if (more) {
        atomicExch(&d.stats[0], 1);
        d.stats[3] = tile;
      }
      atomicAdd(&d.stats[1], 1);
      atomicMax(&d.stats[2], it);
      d.proc[tile] = (stamp << 3) | bits;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && d.trace) trace_end(d, 100 * PAR + 20, d.ctr[PAR], tr0);
}

template <int PAR, typename S, int EB>
__global__ void __launch_bounds__(EB) enthalpy_solve_kernel(Dev d) {
  enthalpy_solve_body<PAR, S, EB>(d, (int)blockIdx.x, (int)gridDim.x);
}

// (three CTAs a SM: a batch lists many small tiles at once)
template <int PAR, typename S, int EB>
__global__ void __launch_bounds__(EB, 3) enthalpy_solve_batch_kernel(const __grid_constant__ BatchPlan P) {
  const int c = plan_lattice(P, (int)blockIdx.x);
  enthalpy_solve_body<PAR, S, EB>(P.d[c], (int)blockIdx.x - P.start[c], P.start[c + 1] - P.start[c]);
}

// x changed flow activity and is the inward node of a flow wall w next to it:
// w's links to its other lattice neighbours x' change state with x.  Those x'
// that kept their activity leave the link to x (a changed x' takes it itself).
template <int PAR>
__device__ __noinline__ void wall_links(const Dev& d, int x, int y, bool ao, bool an,
                                        int stamp) {
  const int n = (int)d.n;
  for (int j = 1; j < 9; ++j) {
    const int wx = wrapx(d, x + ex9(j)), wy = wrapy(d, y + ey9(j));
    if (wx < 0 || wy < 0 || !is_wall(d, wx, wy)) continue;
    int ix, iy;
    inward_of(d, wx, wy, ix, iy);
    if (ix != x || iy != y) continue;
    for (int k = 1; k < 9; ++k) {
      const int px = wrapx(d, wx + ex9(k)), py = wrapy(d, wy + ey9(k));
      if (px < 0 || py < 0 || is_wall(d, px, py) || (px == x && py == y)) continue;
      const int ps = py * d.nx + px;
      const bool vs = solved(d, (py / TE) * d.etx + (px / TE), stamp);
      const float fo = vs ? d.scr[ps].x : d.fl[ps], fnw = vs ? d.scr[ps].y : fo;
      const bool xo = fo >= d.f_act, xn = fnw >= d.f_act;
      if (xo != xn || (xo && ao) == (xn && an)) continue;
      // the pair (x', w): population opp(k) at w, population k at x'
      const long long A = (long long)opp9(k) * n + (wy * d.nx + wx);
      const long long B = (long long)k * n + ps;
      const float t = ld_pop(d, d.f, A);
      st_pop(d, d.f, A, ld_pop(d, d.f, B));
      st_pop(d, d.f, B, t);
    }
  }
}

template <int PAR, bool WALLS>
__device__ __forceinline__ void enthalpy_commit_body(const Dev& d, int bid, int nblk) {
  const long long tr0 = trace_start(d);
  constexpr int LAYOUT = 1 - PAR;
  constexpr int RW = TE + 2;              // tile plus a one-node ring
  __shared__ float2 sp[RW * RW];          // (f_l(n), f_l(n+1)); (-1,-1) on walls / outside
  __shared__ unsigned char ssolved[RW * RW];
  __shared__ int links;
  const int tid = threadIdx.x;
  const int cnt = d.lcount[PAR];
  const int stamp = stamp_of(d, PAR);
  const int n = (int)d.n;
  for (int li = bid; li < cnt; li += nblk) {
    const int tile = d.list[PAR * d.ntiles + li];
    const int tx0 = tile % d.etx, ty0 = tile / d.etx;
    const int X0 = tx0 * TE, Y0 = ty0 * TE;
    const int pb = d.proc[tile] & 7;
    if (tid == 0) {
      d.flags[PAR * d.ntiles + tile] = 0;   // this step's fused pass is done with it
      // flow links need attention only around tiles where a node's activity changed
      int l = 0;
      if (d.flow && LAYOUT == 1) {
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int tx = tx0 + dx, ty = ty0 + dy;
            if (tx < 0 || tx >= d.etx) {
              if (!d.per_x) continue;
              tx = (tx + d.etx) % d.etx;
            }
            if (ty < 0 || ty >= d.ety) {
              if (!d.per_y) continue;
              ty = (ty + d.ety) % d.ety;
            }
            const int t = ty * d.etx + tx;
            if (solved(d, t, stamp) && (d.proc[t] & 4)) l = 1;
          }
      }
      links = l;
    }
    __syncthreads();
    const bool lk = links != 0;
    if ((pb & 2) || lk) {
      if (lk) {
        // old/new liquid fraction of the tile and its ring: scratch in tiles
        // solved this step, the (unchanged) stored value elsewhere
#pragma unroll 2
        for (int k = tid; k < RW * RW; k += CB) {
          const int ly = k / RW, lx = k - ly * RW;
          const int gx = wrapx(d, X0 - 1 + lx), gy = wrapy(d, Y0 - 1 + ly);
          float2 v = make_float2(-1.f, -1.f);
          unsigned char sol = 0;
          if (gx >= 0 && gy >= 0) {
            const bool wall = is_wall(d, gx, gy);
            // a flow wall node carries flow with its inward node (marked 2)
            int vx = gx, vy = gy;
            if (WALLS && wall) inward_of(d, gx, gy, vx, vy);
            if (!wall || WALLS) {
              const int gs = vy * d.nx + vx;
              const bool vs = solved(d, (vy / TE) * d.etx + (vx / TE), stamp);
              sol = wall ? 2 : vs ? 1 : 0;
              if (vs) {
                v = d.scr[gs];
              } else {
                const float f = d.fl[gs];
                v = make_float2(f, f);
              }
            }
          }
          sp[k] = v;
          ssolved[k] = sol;
        }
        __syncthreads();
      }
      int flows = 0;   // a node of the tile carries flow after the step
#pragma unroll 4
      for (int k = tid; k < TE * TE; k += CB) {
        const int ly = k / TE, lx = k - ly * TE;
        const int x = X0 + lx, y = Y0 + ly;
        if (x >= d.nx || y >= d.ny || is_wall(d, x, y)) continue;
        const int s = y * d.nx + x;
        const float2 p = d.scr[s];
        const float fn = p.x, fnew = p.y;
        flows |= fnew >= d.f_act;
        if (fnew != fn) {
          d.fl[s] = fnew;
          const float S0 = -d.phi[s] * d.lat * sigma_ratio(d, fn) * (fnew - fn);
          // N^-1 S~ = S0 w~, streamed: population i of node x + e_i gains w~_i S0
#pragma unroll
          for (int i = 0; i < 5; ++i) {
            const int rx = wrapx(d, x + ex9(i)), ry = wrapy(d, y + ey9(i));
            if (rx < 0 || ry < 0 || is_wall(d, rx, ry)) continue;
            const float w = (i == 0) ? d.wt0 : d.wt1;
            const int slot = (LAYOUT == 1) ? opp5(i) * n + s : i * n + ry * d.nx + rx;
            // (16-bit storage: rounded stochastically, or every small source
            // would be lost to rounding in the same direction)
            st_pop_round(d, d.g, slot, ld_pop(d, d.g, slot) + w * S0,
                         mix32((unsigned)slot ^ mix32((unsigned)stamp)));
          }
        }
        if (lk) {
          const bool ao = fn >= d.f_act, an = fnew >= d.f_act;
          const int c = (ly + 1) * RW + (lx + 1);
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            const int q = c + ey9(i) * RW + ex9(i);
            const float2 pp = sp[q];
            const bool po = pp.x >= d.f_act, pn = pp.y >= d.f_act;
            if ((ao && po) == (an && pn)) continue;
            // link (x, x + e_i) belongs to x for E, N, NE, NW, otherwise to the
            // partner; a partner in a tile not solved this step cannot handle it.
            // A link to a flow wall belongs to x when x changed, else to the
            // wall's inward node (below).
            const bool own = (i == 1 || i == 2 || i == 5 || i == 6);
            if (ssolved[q] == 2 ? ao == an : (!own && ssolved[q])) continue;
            const int px = wrapx(d, x + ex9(i)), py = wrapy(d, y + ey9(i));
            const long long A = (long long)i * n + (py * d.nx + px);
            const long long B = (long long)opp9(i) * n + s;
            const float t = ld_pop(d, d.f, A);   // exact for every storage type
            st_pop(d, d.f, A, ld_pop(d, d.f, B));
            st_pop(d, d.f, B, t);
          }
        }
      }
      // links of flow walls whose inward node changed (tiles along the walls)
      if (WALLS && lk &&
          (X0 == 0 || Y0 == 0 || X0 + TE >= d.nx - 1 || Y0 + TE >= d.ny - 1)) {
        for (int k = tid; k < TE * TE; k += CB) {
          const int ly = k / TE, lx = k - ly * TE;
          const int x = X0 + lx, y = Y0 + ly;
          if (x >= d.nx || y >= d.ny || is_wall(d, x, y)) continue;
          int ix, iy;
          bool inw = false;
          for (int j = 1; j < 9 && !inw; ++j) {
            const int wx = wrapx(d, x + ex9(j)), wy = wrapy(d, y + ey9(j));
            if (wx < 0 || wy < 0 || !is_wall(d, wx, wy)) continue;
            inward_of(d, wx, wy, ix, iy);
            inw = ix == x && iy == y;
          }
          if (!inw) continue;
          const float2 p = d.scr[y * d.nx + x];
          const bool ao = p.x >= d.f_act, an = p.y >= d.f_act;
          if (ao != an) wall_links<PAR>(d, x, y, ao, an, stamp);
        }
      }
      // (the stream-collide pass copies a tile's flow populations only when
      // this is set; no fused pass reads it while the commit runs on its tile)
      if (pb & 2) {
        flows = __syncthreads_or(flows);
        if (tid == 0) d.tact[tile] = (unsigned char)(flows ? 1 : 0);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && d.trace) trace_end(d, 100 * PAR + 30, d.ctr[PAR], tr0);
}

template <int PAR, bool WALLS>
__global__ void __launch_bounds__(CB, 2) enthalpy_commit_kernel(Dev d) {
  enthalpy_commit_body<PAR, WALLS>(d, (int)blockIdx.x, (int)gridDim.x);
}

template <int PAR>
__global__ void __launch_bounds__(CB, 2) enthalpy_commit_batch_kernel(const __grid_constant__ BatchPlan P) {
  const int c = plan_lattice(P, (int)blockIdx.x);
  enthalpy_commit_body<PAR, false>(P.d[c], (int)blockIdx.x - P.start[c], P.start[c + 1] - P.start[c]);
}

size_t enthalpy_solve_smem() { return 6 * RE * RE * sizeof(float); }

template <typename S>
static void solve_setup_t(int bytes) {
  cudaFuncSetAttribute(enthalpy_solve_kernel<0, S, EB_WIDE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(enthalpy_solve_kernel<1, S, EB_WIDE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(enthalpy_solve_kernel<0, S, EB_NARROW>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(enthalpy_solve_kernel<1, S, EB_NARROW>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void enthalpy_setup() {
  const int bytes = (int)enthalpy_solve_smem();
  solve_setup_t<float>(bytes);
  solve_setup_t<__half>(bytes);
  solve_setup_t<__nv_bfloat16>(bytes);
}

// A large lattice's solve runs beside a long far-tile pass, whose SMs it shares:
// narrow CTAs (fewer registers held) cost that pass less.  On a small lattice
// the far-tile pass hides under the solve, whose latency is then the step
// time: wide CTAs finish sooner.
template <typename S>
static void launch_solve_t(const Dev& d, int parity, cudaStream_t s) {
  const size_t sm = enthalpy_solve_smem();
  if (d.ntiles >= SOLVE_NARROW_TILES) {
    if (parity == 0) enthalpy_solve_kernel<0, S, EB_NARROW><<<d.egrid, EB_NARROW, sm, s>>>(d);
    else enthalpy_solve_kernel<1, S, EB_NARROW><<<d.egrid, EB_NARROW, sm, s>>>(d);
  } else {
    if (parity == 0) enthalpy_solve_kernel<0, S, EB_WIDE><<<d.egrid, EB_WIDE, sm, s>>>(d);
    else enthalpy_solve_kernel<1, S, EB_WIDE><<<d.egrid, EB_WIDE, sm, s>>>(d);
  }
}

void launch_enthalpy_solve(const Dev& d, int parity, cudaStream_t s) {
  if (d.storage == 1) launch_solve_t<__half>(d, parity, s);
  else if (d.storage == 2) launch_solve_t<__nv_bfloat16>(d, parity, s);
  else launch_solve_t<float>(d, parity, s);
}

void fused_batch_setup();   // lbm_fused_f32.cu

void batch_setup() {
  fused_batch_setup();
  const int bytes = (int)enthalpy_solve_smem();
  cudaFuncSetAttribute(enthalpy_solve_batch_kernel<0, float, EB_WIDE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(enthalpy_solve_batch_kernel<1, float, EB_WIDE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// the lattices of a batch are small: the wide CTAs, which finish a tile sooner
void launch_enthalpy_solve_batch(const BatchPlan& P, int parity, cudaStream_t s) {
  const size_t sm = enthalpy_solve_smem();
  const int grid = P.start[P.count];
  if (grid <= 0) return;
  if (parity == 0) enthalpy_solve_batch_kernel<0, float, EB_WIDE><<<grid, EB_WIDE, sm, s>>>(P);
  else enthalpy_solve_batch_kernel<1, float, EB_WIDE><<<grid, EB_WIDE, sm, s>>>(P);
}

void launch_enthalpy_commit_batch(const BatchPlan& P, int parity, cudaStream_t s) {
  const int grid = P.start[P.count];
  if (grid <= 0) return;
  if (parity == 0) enthalpy_commit_batch_kernel<0><<<grid, CB, 0, s>>>(P);
  else enthalpy_commit_batch_kernel<1><<<grid, CB, 0, s>>>(P);
}

void launch_enthalpy_commit(const Dev& d, int parity, cudaStream_t s) {
  // flow walls add their links to the re-pairing (a variant of its own, which
  // leaves the common one's registers alone)
  if (d.flow && d.flow_walls) {
    if (parity == 0) enthalpy_commit_kernel<0, true><<<d.cgrid, CB, 0, s>>>(d);
    else enthalpy_commit_kernel<1, true><<<d.cgrid, CB, 0, s>>>(d);
  } else {
    if (parity == 0) enthalpy_commit_kernel<0, false><<<d.cgrid, CB, 0, s>>>(d);
    else enthalpy_commit_kernel<1, false><<<d.cgrid, CB, 0, s>>>(d);
  }
}

}  // namespace lbm
