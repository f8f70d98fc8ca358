// Utility kernels: initial equilibria, macroscopic outputs, FP64 reductions,
// checkpoint gather/scatter and input validation.
#include "lbm_adjoint.cuh"

namespace lbm {

// ---- population gathers for any node, any layout --------------------------

__device__ __forceinline__ bool flow_active(const Dev& d, int x, int y) {
  if (is_wall(d, x, y)) {
    if (!d.flow_walls) return false;
    int ix, iy;   // an extrapolated wall node carries flow with its inward node
    inward_of(d, x, y, ix, iy);
    return d.fl[(long long)iy * d.nx + ix] >= d.f_act;
  }
  return d.fl[(long long)y * d.nx + x] >= d.f_act;
}

// g_i of non-wall node (x, y) in the given layout
__device__ __forceinline__ void gather_g(const Dev& d, int x, int y, int layout, float g[5]) {
  const long long n = d.n, s = (long long)y * d.nx + x;
  (void)n;
  g[0] = ld_g(d, 0, s);
  for (int i = 1; i < 5; ++i) {
    if (layout == 0) {
      g[i] = ld_g(d, i, s);
    } else {
      const int sx = wrapx(d, x - ex9(i)), sy = wrapy(d, y - ey9(i));
      g[i] = ld_g(d, opp5(i), (long long)sy * d.nx + sx);
    }
  }
}

// f_i of node (x, y): nodes without flow hold theirs in their own slots
__device__ __forceinline__ void gather_f(const Dev& d, int x, int y, int layout, float f[9]) {
  const long long n = d.n, s = (long long)y * d.nx + x;
  const bool self = flow_active(d, x, y);
  (void)n;
  f[0] = ld_f(d, 0, s);
  for (int i = 1; i < 9; ++i) {
    if (layout == 0 || !self) {
      f[i] = ld_f(d, i, s);
    } else {
      const int sx = wrapx(d, x - ex9(i)), sy = wrapy(d, y - ey9(i));
      if (flow_active(d, sx, sy)) f[i] = ld_f(d, opp9(i), (long long)sy * d.nx + sx);
      else f[i] = ld_f(d, i, s);
    }
  }
}

__device__ float node_T(const Dev& d, int x, int y, int layout);

// temperature of a non-wall node
__device__ __forceinline__ float interior_T(const Dev& d, int x, int y, int layout) {
  float g[5];
  gather_g(d, x, y, layout, g);
  return g[0] + g[1] + g[2] + g[3] + g[4];
}

// temperature of any node; wall nodes report the temperature their wall
// imposes (Dirichlet value, or the inward neighbour's for an adiabatic wall;
// a corner follows its vertical wall, then its horizontal wall's Dirichlet
// value, then its diagonal neighbour)
__device__ float node_T(const Dev& d, int x, int y, int layout) {
  if (!is_wall(d, x, y)) return interior_T(d, x, y, layout);
  int side;
  if (d.wall_l && x == 0) side = 0;
  else if (d.wall_r && x == d.nx - 1) side = 1;
  else if (d.wall_b && y == 0) side = 2;
  else side = 3;
  if (d.bc[side] == 1) return side == 0 ? d.wallTl[y] : d.Tbc[side];
  const bool vx = (d.wall_l || d.wall_r) && (x == 0 || x == d.nx - 1);
  const bool vy = (d.wall_b || d.wall_t) && (y == 0 || y == d.ny - 1);
  if (vx && vy) {
    const int hs = (y == 0) ? 2 : 3;
    if (d.bc[hs] == 1) return d.Tbc[hs];
    return interior_T(d, x == 0 ? 1 : d.nx - 2, y == 0 ? 1 : d.ny - 2, layout);
  }
  switch (side) {
    case 0: return interior_T(d, 1, y, layout);
    case 1: return interior_T(d, d.nx - 2, y, layout);
    case 2: return interior_T(d, x, 1, layout);
    default: return interior_T(d, x, d.ny - 2, layout);
  }
}

// ---- kernels ----------------------------------------------------------------

__global__ void init_kernel(Dev d, const float* T0) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= d.n) return;
  // f^eq(rho0, u = 0) = w_i rho0, Eq. (29); stored as the deviation f - w_i rho0 = 0
  for (int i = 0; i < 9; ++i) st_f(d, i, s, 0.f);
  // g^eq(T0, u = 0), Eq. (39): w~_i T0
  const float T = T0[s];
  st_g(d, 0, s, d.wt0 * T);
  for (int i = 1; i < 5; ++i) st_g(d, i, s, d.wt1 * T);
}

__global__ void macros_kernel(Dev d, int layout, float* ux, float* uy, float* rho, float* T,
                              float* fl) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= d.n) return;
  const int y = (int)(s / d.nx), x = (int)(s - (long long)y * d.nx);
  const float Tn = node_T(d, x, y, layout);
  const bool wall = is_wall(d, x, y);
  float f[9];
  if (wall) {
    for (int i = 0; i < 9; ++i) f[i] = ld_f(d, i, s);
  } else {
    gather_f(d, x, y, layout, f);
  }
  float dr = 0.f;
  for (int i = 0; i < 9; ++i) dr += f[i];
  const float r = d.rho0 + dr;   // stored populations are f_i - w_i rho0
  float vx = 0.f, vy = 0.f;
  if (d.flow && !wall && flow_active(d, x, y)) {   // a wall's velocity is the wall's, 0
    const float jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const float jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    float Fx, Fy;
    velocity(jx, jy, Tn, d.fl[s], d.phi[s], d.K[s], d, vx, vy, Fx, Fy);
  }
  if (ux) ux[s] = vx;
  if (uy) uy[s] = vy;
  if (rho) rho[s] = r;
  if (T) T[s] = Tn;
  if (fl) fl[s] = d.fl[s];
}

// per-block FP64 partial sums in a fixed order:
// [0] mass, [1] enthalpy, [2] sum f_l, [3] non-wall count, [4] Nusselt sum, [5] Nusselt rows
__global__ void __launch_bounds__(RB) reduce_kernel(Dev d, int layout, double* partials) {
  __shared__ double sh[6][RB];
  const int tid = threadIdx.x;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long s = blockIdx.x * (long long)RB + tid; s < d.n; s += (long long)gridDim.x * RB) {
    const int y = (int)(s / d.nx), x = (int)(s - (long long)y * d.nx);
    if (!is_wall(d, x, y)) {
      float f[9];
      gather_f(d, x, y, layout, f);
      double m = (double)d.rho0;   // stored populations are f_i - w_i rho0
      for (int i = 0; i < 9; ++i) m += (double)f[i];
      const double T = (double)interior_T(d, x, y, layout);
      const double fl = (double)d.fl[s];
      acc[0] += m;
      // a = phi dT / (sigma(f_l) St), Eq. (38) with Eq. (7)
      const double sr = d.sigma_var ? (double)d.sigma / ((double)d.sigma_s +
                                                         fl * ((double)d.sigma - d.sigma_s))
                                    : 1.0;
      acc[1] += T + (double)d.phi[s] * (double)d.lat * sr * fl;
      acc[2] += fl;
      acc[3] += 1.0;
    }
    if (d.wall_l && x == 0 && d.nx >= 3 && (!d.wall_b || (y > 0 && y < d.ny - 1))) {
      const double T0 = node_T(d, 0, y, layout), T1 = node_T(d, 1, y, layout),
                   T2 = node_T(d, 2, y, layout);
      acc[4] += -(-3.0 * T0 + 4.0 * T1 - T2) * 0.5 * (double)d.H_over_dT;
      acc[5] += 1.0;
    }
  }
  for (int k = 0; k < 6; ++k) sh[k][tid] = acc[k];
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int k = 0; k < 6; ++k) sh[k][tid] += sh[k][tid + w];
    __syncthreads();
  }
  if (tid == 0)
    for (int k = 0; k < 6; ++k) partials[blockIdx.x * 6 + k] = sh[k][0];
}

// The left-wall Nusselt number of the current state (the rows and the
// formula of reduce_kernel), added to acc[0]; one block, fixed summation order.
__global__ void __launch_bounds__(RB) wall_nusselt_kernel(Dev d, int layout, double* acc) {
  __shared__ double sh[RB];
  const int tid = threadIdx.x;
  const int y0 = d.wall_b ? 1 : 0, y1 = d.wall_t ? d.ny - 1 : d.ny;
  double v = 0.0;
  if (d.wall_l && d.nx >= 3)
    for (int y = y0 + tid; y < y1; y += RB) {
      const double T0 = node_T(d, 0, y, layout), T1 = node_T(d, 1, y, layout),
                   T2 = node_T(d, 2, y, layout);
      v += -(-3.0 * T0 + 4.0 * T1 - T2) * 0.5 * (double)d.H_over_dT;
    }
  sh[tid] = v;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  if (tid == 0 && d.wall_l && d.nx >= 3 && y1 > y0) acc[0] += sh[0] / (double)(y1 - y0);
}

__global__ void reduce_final_kernel(const double* partials, int nblocks, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < 6; ++k) t[k] += partials[b * 6 + k];
  out[0] = t[0];
  out[1] = t[1];
  out[2] = t[3] > 0 ? t[2] / t[3] : 0.0;
  out[3] = t[5] > 0 ? t[4] / t[5] : 0.0;
}

// f (9 planes) and g (5 planes) in the natural layout; each output is optional
__global__ void get_state_kernel(Dev d, int layout, float* f, float* g) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= d.n) return;
  const int y = (int)(s / d.nx), x = (int)(s - (long long)y * d.nx);
  const long long n = d.n;
  const bool wall = is_wall(d, x, y);
  if (f) {
    float fv[9];
    if (wall)
      for (int i = 0; i < 9; ++i) fv[i] = ld_f(d, i, s);
    else
      gather_f(d, x, y, layout, fv);
    for (int i = 0; i < 9; ++i) f[i * n + s] = fv[i];
  }
  if (g) {
    float gv[5];
    if (wall)
      for (int i = 0; i < 5; ++i) gv[i] = ld_g(d, i, s);
    else
      gather_g(d, x, y, layout, gv);
    for (int i = 0; i < 5; ++i) g[i * n + s] = gv[i];
  }
}

__global__ void set_state_kernel(Dev d, const float* f, const float* g) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= d.n) return;
  const long long n = d.n;
  if (f)
    for (int i = 0; i < 9; ++i) st_f(d, i, s, f[i * n + s]);
  if (g)
    for (int i = 0; i < 5; ++i) st_g(d, i, s, g[i * n + s]);
}

__global__ void validate_kernel(Dev d, const float* phi, const float* K, const float* T0,
                                const float* fl0, int* bad) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= d.n) return;
  const float p = phi[s], k = K[s], t = T0[s], l = fl0[s];
  bool ok = (p > 0.f && p <= 1.f) && (!d.flow || p < 1.f) && (k > 0.f) && isfinite(t) &&
            (l >= 0.f && l <= 1.f);
  if (!ok) atomicExch(bad, 1);
}

// The whole state in natural layout (f as deviations, 9 planes; g, 5 planes;
// f_l) into dst, 15 n floats; with ctr non-null into base + ctr[0] 15 n, after
// which ctr[0] advances (ctr[1]: 0, scratch), so one captured launch serves
// every replay of a graph.
__global__ void keep_state_kernel(Dev d, int layout, float* base, unsigned* ctr) {
  const long long n = d.n;
  float* dst = base + (ctr ? (long long)ctr[0] * 15 * n : 0LL);
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(s / d.nx), x = (int)(s - (long long)y * d.nx);
    const bool wall = is_wall(d, x, y);
    const float fls = d.fl[s];
    // every load is issued before any value is chosen (gather_f / gather_g
    // with the candidates of both layouts loaded up front)
    float own[9], str[9], gown[5], gstr[5];
    bool act[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) own[i] = ld_f(d, i, s);
#pragma unroll
    for (int i = 0; i < 5; ++i) gown[i] = ld_g(d, i, s);
    const bool swapped = layout == 1 && !wall;
    if (swapped) {
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int sx = wrapx(d, x - ex9(i)), sy = wrapy(d, y - ey9(i));
        const long long t = (long long)sy * d.nx + sx;
        act[i] = flow_active(d, sx, sy);
        str[i] = ld_f(d, opp9(i), t);
        if (i < 5) gstr[i] = ld_g(d, opp5(i), t);
      }
    }
    const bool self = !wall && fls >= d.f_act;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float v = (swapped && self && i > 0 && act[i]) ? str[i] : own[i];
      dst[i * n + s] = v;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) dst[(9 + i) * n + s] = (swapped && i > 0) ? gstr[i] : gown[i];
    dst[14 * n + s] = fls;
  }
  if (ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
        ctr[1] = 0;
        ctr[0] = ctr[0] + 1;
      }
    }
  }
}

// Sentinel: every population and f_l of every node, flag stats[5] on the first
// value that is not finite (NaN or Inf).
__global__ void nonfinite_kernel(Dev d) {
  bool bad = false;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < d.n;
       s += (long long)gridDim.x * blockDim.x) {
    bool ok = isfinite(d.fl[s]);
    for (int i = 0; i < 9; ++i) ok = ok && isfinite(ld_pop(d, d.f, i * d.n + s));
    for (int i = 0; i < 5; ++i) ok = ok && isfinite(ld_pop(d, d.g, i * d.n + s));
    bad = bad || !ok;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&d.stats[5], 1);
}

static unsigned grid1(long long n, int b) { return (unsigned)((n + b - 1) / b); }

void launch_init(const Dev& d, const float* T0, cudaStream_t s) {
  init_kernel<<<grid1(d.n, 256), 256, 0, s>>>(d, T0);
}
// one CTA per enthalpy tile: does a non-wall node of it carry flow?
__global__ void __launch_bounds__(256) tile_activity_kernel(Dev d) {
  const int tile = blockIdx.x;
  const int X0 = (tile % d.etx) * TE, Y0 = (tile / d.etx) * TE;
  int any = 0;
  for (int k = threadIdx.x; k < TE * TE; k += blockDim.x) {
    const int x = X0 + k % TE, y = Y0 + k / TE;
    if (x < d.nx && y < d.ny && !is_wall(d, x, y) && d.fl[(long long)y * d.nx + x] >= d.f_act)
      any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) d.tact[tile] = (unsigned char)(any ? 1 : 0);
}

void launch_tile_activity(const Dev& d, cudaStream_t s) {
  if (d.ntiles > 0) tile_activity_kernel<<<d.ntiles, 256, 0, s>>>(d);
}

void launch_macros(const Dev& d, int layout, float* ux, float* uy, float* rho, float* T,
                   float* fl, cudaStream_t s) {
  macros_kernel<<<grid1(d.n, 256), 256, 0, s>>>(d, layout, ux, uy, rho, T, fl);
}
int reduce_blocks(const Dev& d) {
  long long b = (d.n + RB - 1) / RB;
  return (int)(b < 1024 ? b : 1024);
}
void launch_reduce(const Dev& d, int layout, double* partials, double* out, int nblocks,
                   cudaStream_t s) {
  reduce_kernel<<<nblocks, RB, 0, s>>>(d, layout, partials);
  reduce_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out);
}
void launch_wall_nusselt(const Dev& d, int layout, double* acc, cudaStream_t s) {
  wall_nusselt_kernel<<<1, RB, 0, s>>>(d, layout, acc);
}
void launch_get_state(const Dev& d, int layout, float* f, float* g, cudaStream_t s) {
  get_state_kernel<<<grid1(d.n, 256), 256, 0, s>>>(d, layout, f, g);
}
void launch_set_state(const Dev& d, const float* f, const float* g, cudaStream_t s) {
  set_state_kernel<<<grid1(d.n, 256), 256, 0, s>>>(d, f, g);
}
void launch_keep_state(const Dev& d, int layout, float* base, unsigned* ctr, cudaStream_t s) {
  long long nb = (d.n + 255) / 256;
  if (nb > 8 * 152) nb = 8 * 152;
  keep_state_kernel<<<(unsigned)nb, 256, 0, s>>>(d, layout, base, ctr);
}
void launch_nonfinite(const Dev& d, int nblocks, cudaStream_t s) {
  nonfinite_kernel<<<nblocks, 256, 0, s>>>(d);
}
void launch_validate(const Dev& d, const float* phi, const float* K, const float* T0,
                     const float* fl0, int* bad, cudaStream_t s) {
  validate_kernel<<<grid1(d.n, 256), 256, 0, s>>>(d, phi, K, T0, fl0, bad);
}

}  // namespace lbm
