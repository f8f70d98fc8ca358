// Internal declarations shared by the liblbm translation units.
//
// Device state layout (structure of arrays, x fastest, plane stride n = nx*ny):
//   f[9][n]   D2Q9 populations as deviations f_i - w_i rho0 from the rest
//             equilibrium (keeps FP32 resolution for small velocities), AA in place
//   g[5][n]   D2Q5 populations, in place with the AA pattern; with 16-bit
//             storage as deviations g_i - w~_i T_m (g_ref below)
// Populations are FP32, FP16 or BF16 in memory (storage); all arithmetic is FP32.
//   fl[n]     liquid fraction f_l
//   phi[n]    porosity, K[n] fully liquid permeability
// Velocity order, Eq. (15) and (31): 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
//
// AA pattern.  Even steps read population i of node x from slot (x, i) and
// write the post-collision value to slot (x, opp(i)) of the same node.  Odd
// steps read population i from slot (x - e_i, opp(i)) and write it to slot
// (x + e_i, i).  After an odd step every population sits in its own node's
// slot ("natural" layout); after an even step population i of node x sits in
// node x - e_i ("swapped" layout).  A flow link into a node without flow is
// resolved on the odd step: the population reflected at the link is read
// from (x, i) and written to (x, opp(i)).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

constexpr int TX = 32;       // fused kernel tile (threads x)
constexpr int TY = 8;        // fused kernel tile (threads y)
constexpr int TE = 32;       // enthalpy tile edge
constexpr int RH = 8;        // enthalpy halo width
constexpr int RE = TE + 2 * RH;
// enthalpy solve block sizes: narrow CTAs on large lattices (they share SMs with
// the far-tile pass), wide ones on small lattices (the solve's latency is the step)
constexpr int EB_NARROW = 256;
constexpr int EB_WIDE = 512;
constexpr int SOLVE_NARROW_TILES = 1024;   // enthalpy tiles from which the narrow form runs
constexpr int CB = 1024;     // enthalpy commit block size (one thread per node of a tile:
                             // narrower CTAs measured slower beside the far-tile pass)
constexpr int RB = 256;      // reduction block size
// default tiles per CTA of the TMA-staged kernel: few enough that CTAs retire
// often (the enthalpy kernels overlapping the far-tile pass need SMs), enough
// to hide the first copy of each CTA (2048^2 cavity: 4-5 best, 2-3 and 6-12
// slower); lbm_autotune picks per lattice
constexpr int TMA_TPC = 5;

struct Dev {
  int nx, ny;
  long long n;               // nodes per plane
  int per_x, per_y;          // periodic axes
  int wall_l, wall_r, wall_b, wall_t;
  int bc[4];
  float Tbc[4];
  int flow;                  // vartheta
  float rho0, inv_rho0;
  float nu_l, g_beta, T_ref;
  float s_e, s_eps, s_q, s_nu;
  float z_a, z_e, z_nu;      // 1/tau_T, zeta_e, zeta_nu
  int alpha_var;             // tau_T depends on f_l (alpha_l != alpha_s)
  float tauT_l, inv_aratio;  // liquid tau_T, alpha_s / alpha_l
  int flow_walls;            // 1: flow walls by non-equilibrium extrapolation (Sec. 4): a wall
                             // node whose inward node carries flow collides and streams
  int sigma_var;             // sigma follows f_l, Eq. (7): sigma_s + f_l (sigma - sigma_s)
  float sigma_s;             // its solid value (sigma is the liquid one)
  float varpi, csT2, sigma;
  float conv;                // vartheta / (sigma c_sT^2)
  float wt0, wt1;            // D2Q5 weights of Eq. (39)
  float lat;                 // dT / (sigma St)
  float T_s, T_l, dTt;
  float f_act;
  float scr_T;               // phase-change screen margin in temperature (1e-7 of the scale)
  float scr_f;               // liquid fraction treated as 0 / 1 by the screen
  int screen_off;            // 1: every enthalpy tile is solved every step
  float H_over_dT;
  int etx, ety;              // enthalpy tiles
  int ntiles;                // etx * ety
  int egrid, cgrid;          // CTAs of the enthalpy solve / commit kernels (they walk the tile list)
  int tgrid;                 // CTAs of the TMA-staged fused kernel
  int tslots;                // its CTAs resident at once (SMs x CTAs per SM)
  int max_inner;
  float tol;
  void* f;                   // 9 planes of the storage type
  void* g;                   // 5 planes of the storage type
  int storage;               // 0 FP32, 1 FP16, 2 BF16
  float g_ref;               // T_m of the stored g deviations (0 for FP32 storage)
  float* fl;
  const float* phi;
  const float* K;
  const float* wallTl;
  int* flags;                // [2][ntiles]: 1 once listed in that parity's step (cleared by the solve)
  int* list;                 // [2][ntiles]: tiles to solve, one list per step parity
  int* lcount;               // [2]: entries in each list
  int* ctr;                  // [2]: step stamp per parity (the fused pass sets ctr[p] = ctr[1-p] + 1)
  int* nearmap;              // [2][ntiles]: per parity, the stamp of the step that listed a tile
                             // within one tile of this one
  int* proc;                 // per enthalpy tile: (stamp << 3) | bits, bit 0 solved, bit 1
                             // some f_l changed, bit 2 some node's flow activity changed
  float2* scr;               // per node of solved tiles: (f_l(n), f_l(n+1))
  int flow_front;            // 1: links from a flow node into a non-flow lattice node take
                             // the extrapolated boundary population (Sec. 4, moving front)
  int tskip;                 // 1: the TMA-staged pass copies flow populations, phi and K
                             // only for tiles with tact set (batch members: mostly solid
                             // lattices); 0: for every tile
  unsigned char* tact;       // per enthalpy tile: 1 if a non-wall node of it carries flow
                             // (f_l >= f_act); kept by the commit kernel and by
                             // launch_tile_activity wherever f_l is loaded
  // kernel trace (lbm_trace): per CTA, at its end, (kind, step stamp, start
  // and end in ns of %globaltimer) appended at trace[4 k], k = trace_n[0]++,
  // while k < trace_cap; null: off
  long long* trace;
  unsigned* trace_n;
  unsigned trace_cap;
  int* stats;                // [0] inner cap hit, [1] tiles solved, [2] max sweeps,
                             // [3] last tile that hit the cap, [4] a bounded wait gave up,
                             // [5] the sentinel found a non-finite value
};

__device__ __forceinline__ long long trace_now() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// start time of a traced CTA (0 when tracing is off)
__device__ __forceinline__ long long trace_start(const Dev& d) {
  return d.trace ? trace_now() : 0;
}
// one record for the calling CTA (call from one thread, at the CTA's end)
__device__ __forceinline__ void trace_end(const Dev& d, int kind, int stamp, long long t0) {
  if (!d.trace) return;
  const unsigned k = atomicAdd(d.trace_n, 1u);
  if (k >= d.trace_cap) return;
  long long* r = d.trace + 4ll * k;
  r[0] = kind;
  r[1] = stamp;
  r[2] = t0;
  r[3] = trace_now();
}

// Tensor maps of the TMA-staged fused kernel (passed as a __grid_constant__
// kernel parameter): population boxes without halo for even steps and with a
// 4-column, 1-row halo for odd steps, f_l with the halo, phi and K without.
struct TmaMaps {
  CUtensorMap f_even, f_odd, g_even, g_odd, fl, phi, K;
};

// A batched launch runs one kernel over several lattices: lattice i takes the
// CTAs [start[i], start[i + 1]) of the grid, with its own parameters d[i].
// Passed as a __grid_constant__ kernel parameter (25 KB, within the 32 KB
// parameter limit), so a CTA reads its lattice's fields from the constant
// bank as a single lattice's launch does.
constexpr int BATCH_MAX = 64;
struct BatchPlan {
  int count;
  int start[BATCH_MAX + 1];
  Dev d[BATCH_MAX];
};
// the lattice whose range holds CTA b (binary search over the starts)
__device__ __forceinline__ int plan_lattice(const BatchPlan& P, int b) {
  int lo = 0, hi = P.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// conversions between a stored population and FP32 (round to nearest on store)
template <typename S>
struct Pop;
template <>
struct Pop<float> {
  __device__ static __forceinline__ float ld(const float* p) { return *p; }
  __device__ static __forceinline__ void st(float* p, float v) { *p = v; }
};
// FP16 holds populations scaled by 2^10: the small deviations of slow flow and
// of temperatures near T_m then stay clear of FP16's subnormal range (below
// 6.1e-5), where its resolution is absolute, not relative.  Limit: stored
// magnitudes up to 65504 / 1024 = 64 (|T - T_m| up to ~100 with w~_0 = 0.6).
constexpr float HALF_SCALE = 1024.f;
template <>
struct Pop<__half> {
  __device__ static __forceinline__ float ld(const __half* p) {
    return __half2float(*p) * (1.f / HALF_SCALE);
  }
  __device__ static __forceinline__ void st(__half* p, float v) {
    *p = __float2half_rn(v * HALF_SCALE);
  }
};
template <>
struct Pop<__nv_bfloat16> {
  __device__ static __forceinline__ float ld(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
  }
  __device__ static __forceinline__ void st(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
  }
};

// Stores into 16-bit storage round stochastically: up with probability
// (v - down) / (up - down), so that the expected stored value is v.  Rounding
// to nearest loses every increment below half an ulp, every time: the small
// latent-heat sources and the slow relaxation of a nearly converged field
// then drift systematically.  r: 32 random bits (the top 24 are used).
constexpr bool STOCHASTIC_ROUNDING = true;

// MurmurHash3's 32-bit finaliser (Appleby), used as a counter-based mixer
__device__ __forceinline__ unsigned mix32(unsigned h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
// next random word of a per-node sequence (a linear congruential step; only
// its high bits are used)
__device__ __forceinline__ unsigned next_rand(unsigned& r) {
  r = r * 1664525u + 1013904223u;
  return r;
}

// Blackwell converts with stochastic rounding in hardware (cvt.rs): the value
// goes into the low half of a packed pair (the high half, from 0, is dropped)
constexpr bool HW_STOCHASTIC = true;

template <typename S>
__device__ __forceinline__ void st_round(S* p, float v, unsigned r) {
  if constexpr (sizeof(S) == 4 || !STOCHASTIC_ROUNDING) {
    Pop<S>::st(p, v);
  } else if constexpr (HW_STOCHASTIC) {
    unsigned pair;
    if constexpr (std::is_same<S, __half>::value)
      asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(pair) : "f"(0.f), "f"(v * HALF_SCALE), "r"(r));
    else
      asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(pair) : "f"(0.f), "f"(v), "r"(r));
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)(pair & 0xffffu);
  } else {
    S lo, hi;
    float flo, fhi;
    if constexpr (std::is_same<S, __half>::value) {
      v *= HALF_SCALE;   // exact (a power of two)
      lo = __float2half_rd(v);
      hi = __float2half_ru(v);
      flo = __half2float(lo);
      fhi = __half2float(hi);
    } else {
      lo = __float2bfloat16_rd(v);
      hi = __float2bfloat16_ru(v);
      flo = __bfloat162float(lo);
      fhi = __bfloat162float(hi);
    }
    const float u = (float)(r >> 8) * 5.9604645e-8f;   // uniform in [0, 1), 2^-24 steps
    *p = (u * (fhi - flo) < v - flo) ? hi : lo;
  }
}

// Population access with the storage chosen at run time (kernels off the
// stream-collide path): element i of array base, as FP32.
__device__ __forceinline__ float ld_pop(const Dev& d, const void* base, long long i) {
  if (d.storage == 1) return Pop<__half>::ld(static_cast<const __half*>(base) + i);
  if (d.storage == 2) return Pop<__nv_bfloat16>::ld(static_cast<const __nv_bfloat16*>(base) + i);
  return static_cast<const float*>(base)[i];
}
__device__ __forceinline__ void st_pop(const Dev& d, void* base, long long i, float v) {
  if (d.storage == 1) Pop<__half>::st(static_cast<__half*>(base) + i, v);
  else if (d.storage == 2) Pop<__nv_bfloat16>::st(static_cast<__nv_bfloat16*>(base) + i, v);
  else static_cast<float*>(base)[i] = v;
}
__device__ __forceinline__ void st_pop_round(const Dev& d, void* base, long long i, float v,
                                             unsigned r) {
  if (d.storage == 1) st_round(static_cast<__half*>(base) + i, v, r);
  else if (d.storage == 2) st_round(static_cast<__nv_bfloat16*>(base) + i, v, r);
  else static_cast<float*>(base)[i] = v;
}
// f plane k at node s (stored as deviations in every storage)
__device__ __forceinline__ float ld_f(const Dev& d, int k, long long s) {
  return ld_pop(d, d.f, k * d.n + s);
}
__device__ __forceinline__ void st_f(const Dev& d, int k, long long s, float v) {
  st_pop(d, d.f, k * d.n + s, v);
}
// g plane k at node s: the stored deviation plus w~_k T_m for 16-bit storage
__device__ __forceinline__ float ld_g(const Dev& d, int k, long long s) {
  const float v = ld_pop(d, d.g, k * d.n + s);
  if (d.storage == 0) return v;
  return v + (k == 0 ? d.wt0 : d.wt1) * d.g_ref;
}
__device__ __forceinline__ void st_g(const Dev& d, int k, long long s, float v) {
  if (d.storage != 0) v -= (k == 0 ? d.wt0 : d.wt1) * d.g_ref;
  st_pop(d, d.g, k * d.n + s, v);
}

__host__ __device__ inline int opp9(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__host__ __device__ inline int opp5(int i) { return i == 0 ? 0 : ((i + 1) & 3) + 1; }

__device__ __forceinline__ int ex9(int i) {
  const int e[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  return e[i];
}
__device__ __forceinline__ int ey9(int i) {
  const int e[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  return e[i];
}

// wrapped coordinate (any number of periods: an enthalpy halo can be wider
// than a narrow periodic lattice), or -1 outside a non-periodic domain
__device__ __forceinline__ int wrapx(const Dev& d, int x) {
  if (x >= 0 && x < d.nx) return x;
  if (!d.per_x) return -1;
  x %= d.nx;
  return x < 0 ? x + d.nx : x;
}
__device__ __forceinline__ int wrapy(const Dev& d, int y) {
  if (y >= 0 && y < d.ny) return y;
  if (!d.per_y) return -1;
  y %= d.ny;
  return y < 0 ? y + d.ny : y;
}
__device__ __forceinline__ bool is_wall(const Dev& d, int x, int y) {
  return (d.wall_l && x == 0) || (d.wall_r && x == d.nx - 1) || (d.wall_b && y == 0) ||
         (d.wall_t && y == d.ny - 1);
}
// inward neighbour of wall node (x, y): one node into the lattice from each wall
// it lies on (the diagonal neighbour at a corner)
__device__ __forceinline__ void inward_of(const Dev& d, int x, int y, int& ix, int& iy) {
  ix = (d.wall_l && x == 0) ? 1 : (d.wall_r && x == d.nx - 1) ? d.nx - 2 : x;
  iy = (d.wall_b && y == 0) ? 1 : (d.wall_t && y == d.ny - 1) ? d.ny - 2 : y;
}

// sigma_l / sigma(f_l) with the heat-capacity ratio of Eq. (7) linear in f_l
// (1 when sigma does not follow f_l)
__host__ __device__ __forceinline__ float sigma_ratio(const Dev& d, float fl) {
  return d.sigma_var ? d.sigma / (d.sigma_s + fl * (d.sigma - d.sigma_s)) : 1.f;
}

// Permeability and inertial coefficient at varphi = phi f_l, Eq. (6); the
// input K is the fully liquid permeability (K_eff(f_l = 1) = K).
__device__ __forceinline__ void porous(float fl, float phi, float K, float& nuK, float& cfK,
                                       const Dev& d) {
  float varphi = phi * fl;
  float r = (1.f - phi) / (1.f - varphi);
  float Keff = K * fl * fl * fl * r * r;   // +inf stays +inf
  float cf = 1.75f * rsqrtf(175.f * varphi * varphi * varphi);
  nuK = d.nu_l / Keff;                     // nu_l / K_eff
  cfK = cf * rsqrtf(Keff);                 // C_F / sqrt(K_eff)
}

// Velocity from Eq. (26)-(28) and total force of Eq. (4)-(5) at one node.
__device__ __forceinline__ void velocity(float jx, float jy, float T, float fl, float phi,
                                         float K, const Dev& d, float& ux, float& uy,
                                         float& Fx, float& Fy) {
  float varphi = phi * fl;
  float G = d.g_beta * (T - d.T_ref);
  float nuK, cfK;
  porous(fl, phi, K, nuK, cfK, d);
  float vx = jx * d.inv_rho0;
  float vy = jy * d.inv_rho0 + 0.5f * varphi * G;
  float l0 = 0.5f * (1.f + 0.5f * varphi * nuK);
  float l1 = 0.5f * varphi * cfK;
  float vm = sqrtf(vx * vx + vy * vy);
  float inv = 1.f / (l0 + sqrtf(l0 * l0 + l1 * vm));
  ux = vx * inv;
  uy = vy * inv;
  float um = sqrtf(ux * ux + uy * uy);
  float drag = varphi * (nuK + cfK * um);
  Fx = -drag * ux;
  Fy = -drag * uy + varphi * G;
}

// Kernel entry points (defined in the .cu files)
// fused kernel over all tiles (mode 0), only tiles away from the last step's
// front (mode 1) or only tiles near it (mode 2); the TMA-staged kernel
// when m is non-null (maps filled by tma_setup, which also sets tgrid)
void launch_fused(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s);
bool tma_setup(Dev& d, TmaMaps* m);
// CTAs of the TMA-staged kernel for about tpc tiles per CTA, in whole waves of
// the resident CTAs (d.tslots), at most 32 tiles per CTA
int tma_grid(const Dev& d, int tpc);
void launch_enthalpy_solve(const Dev& d, int parity, cudaStream_t s);
void launch_enthalpy_commit(const Dev& d, int parity, cudaStream_t s);
// Batched launches (FP32 storage, TMA-staged stream-collide, no flow walls):
// one launch runs the pass for every lattice of the plan, lattice i on the
// CTAs [P.start[i], P.start[i + 1]); maps: device array of the lattices'
// tensor maps.  batch_setup sets the kernels' shared-memory limits (call it
// before capturing them).
void batch_setup();
void launch_fused_batch(const BatchPlan& P, const TmaMaps* maps, int parity, int mode, bool flow,
                        cudaStream_t s);
void launch_enthalpy_solve_batch(const BatchPlan& P, int parity, cudaStream_t s);
void launch_enthalpy_commit_batch(const BatchPlan& P, int parity, cudaStream_t s);
void enthalpy_setup();
size_t enthalpy_solve_smem();
void launch_init(const Dev& d, const float* T0, cudaStream_t s);
void launch_macros(const Dev& d, int parity, float* ux, float* uy, float* rho, float* T,
                   float* fl, cudaStream_t s);
void launch_reduce(const Dev& d, int parity, double* partials, double* out, int nblocks,
                   cudaStream_t s);
int reduce_blocks(const Dev& d);
void launch_get_state(const Dev& d, int parity, float* f, float* g, cudaStream_t s);
void launch_set_state(const Dev& d, const float* f, const float* g, cudaStream_t s);
// the whole state (f, g, f_l: 15 n floats, natural layout) into base, or into
// base + ctr[0] 15 n and then ctr[0]++ when ctr is non-null (ctr[1] must be 0)
void launch_keep_state(const Dev& d, int layout, float* base, unsigned* ctr, cudaStream_t s);
// d.tact from d.fl, every tile (after f_l is loaded from outside the step)
void launch_tile_activity(const Dev& d, cudaStream_t s);
// NaN/Inf sentinel over the whole state (sets stats[5])
void launch_nonfinite(const Dev& d, int nblocks, cudaStream_t s);
// one CTA waiting, with a limit of limit_ns, on an mbarrier nothing completes
// (sets stats[4] when the wait gives up, as a timed-out bulk copy does)
void launch_wait_probe(const Dev& d, long long limit_ns, cudaStream_t s);
// the wall nodes' flow update when flow walls are on (mode as for launch_fused,
// by the enthalpy tile of each wall node's inward node); runs before the
// stream-collide pass of the same step and mode
void launch_flow_walls(const Dev& d, int parity, int mode, cudaStream_t s);
void launch_validate(const Dev& d, const float* phi, const float* K, const float* T0,
                     const float* fl0, int* bad, cudaStream_t s);

}  // namespace lbm
