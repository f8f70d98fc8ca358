// lbm_reduce_state_noalloc: the FP64 state reduction of lbm_reduce, for callers
// that cannot allocate device memory.
//
// Who needs it: code that holds a checkpoint of the lattice (the natural-layout
// FP32 arrays lbm_get_state writes, whatever the context's population storage)
// in device memory it already owns, and wants the conservation sums without
// creating a context, which allocates a workspace.  Typical cases are a
// framework whose caching allocator owns all device memory and forbids side
// allocations, and monitoring code that runs inside a fixed memory budget and
// must not take device memory from the job it watches.
//
// The call is synchronous: it queues two kernels on the caller's stream, copies
// the four sums to host memory and synchronises that stream before returning.
//
// Scratch lives in a file-scope __device__ array (one FP64 partial per lattice
// row and quantity), so the call allocates nothing.  Every GPU that loads the
// library holds it until the process exits.  Its device address is looked up
// with cudaGetSymbolAddress the first time the function runs on a device, with
// that device current; make that first call before any stream capture.  All
// calls share the array: every element a call reads it writes first in the same
// call, but two calls whose kernels overlap on the GPU (different streams, no
// ordering) race on it and may return wrong sums.
#include <math.h>
#include <mutex>
#include <string.h>

#include "lbm.h"

namespace {

constexpr int NQ = 6;          // mass, enthalpy, sum f_l, node count, Nusselt sum, Nusselt rows
constexpr int RED_THREADS = 256;
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) double g_noalloc_rows[LBM_NOALLOC_MAX_ROWS * NQ];
__device__ __align__(256) double g_noalloc_total[8];

struct Geo {
  int nx, ny;
  int wl, wr, wb, wt;          // wall on side
  int bc[4];
  float Tbc[4];
  float rho0, lat, H_over_dT;
  int sigma_var;               // sigma linear in f_l (Eq. 7): sigma_s + f_l (sigma_l - sigma_s)
  float sigma_l, sigma_s;
  float f_act;
};

__device__ bool wall_node(const Geo& q, int x, int y) {
  return (q.wl && x == 0) || (q.wr && x == q.nx - 1) || (q.wb && y == 0) || (q.wt && y == q.ny - 1);
}

__device__ float sum_g(const float* g, long long n, long long s) {
  return g[s] + g[n + s] + g[2 * n + s] + g[3 * n + s] + g[4 * n + s];
}

// temperature of a node: sum g inside; on a wall node the temperature the wall
// imposes (Dirichlet value; adiabatic: inward neighbour; a corner follows its
// vertical wall, then its horizontal wall's Dirichlet value, then the diagonal)
__device__ float node_temp(const Geo& q, const float* g, const float* wallTl, int x, int y) {
  const long long n = (long long)q.nx * q.ny;
  if (!wall_node(q, x, y)) return sum_g(g, n, (long long)y * q.nx + x);
  int side;
  if (q.wl && x == 0) side = LBM_SIDE_LEFT;
  else if (q.wr && x == q.nx - 1) side = LBM_SIDE_RIGHT;
  else if (q.wb && y == 0) side = LBM_SIDE_BOTTOM;
  else side = LBM_SIDE_TOP;
  if (q.bc[side] == LBM_BC_DIRICHLET)
    return (side == LBM_SIDE_LEFT && wallTl) ? wallTl[y] : q.Tbc[side];
  const bool cx = (q.wl || q.wr) && (x == 0 || x == q.nx - 1);
  const bool cy = (q.wb || q.wt) && (y == 0 || y == q.ny - 1);
  int ix = x, iy = y;
  if (cx && cy) {
    const int hs = (y == 0) ? LBM_SIDE_BOTTOM : LBM_SIDE_TOP;
    if (q.bc[hs] == LBM_BC_DIRICHLET) return q.Tbc[hs];
    ix = (x == 0) ? 1 : q.nx - 2;
    iy = (y == 0) ? 1 : q.ny - 2;
  } else if (side == LBM_SIDE_LEFT) {
    ix = 1;
  } else if (side == LBM_SIDE_RIGHT) {
    ix = q.nx - 2;
  } else if (side == LBM_SIDE_BOTTOM) {
    iy = 1;
  } else {
    iy = q.ny - 2;
  }
  return sum_g(g, n, (long long)iy * q.nx + ix);
}

// one CTA per row: FP64 row sums in a fixed order into scratch[row]
__global__ void __launch_bounds__(RED_THREADS) rows_kernel(Geo q, const float* f, const float* g,
                                                          const float* fl, const float* phi,
                                                          const float* wallTl, double* rows) {
  __shared__ double sh[NQ][RED_THREADS];
  const int y = blockIdx.x, tid = threadIdx.x;
  const long long n = (long long)q.nx * q.ny;
  double acc[NQ] = {0, 0, 0, 0, 0, 0};
  for (int x = tid; x < q.nx; x += RED_THREADS) {
    if (wall_node(q, x, y)) continue;
    const long long s = (long long)y * q.nx + x;
    double m = (double)q.rho0;   // f holds deviations f_i - w_i rho0
    for (int i = 0; i < 9; ++i) m += (double)f[i * n + s];
    const double T = (double)sum_g(g, n, s);
    const double l = (double)fl[s];
    acc[0] += m;
    const double sr = q.sigma_var ? (double)q.sigma_l / ((double)q.sigma_s +
                                                         l * ((double)q.sigma_l - q.sigma_s))
                                  : 1.0;
    acc[1] += T + (double)phi[s] * (double)q.lat * sr * l;
    acc[2] += l;
    acc[3] += 1.0;
  }
  if (tid == 0 && q.wl && q.nx >= 3 && (!q.wb || (y > 0 && y < q.ny - 1))) {
    const double T0 = node_temp(q, g, wallTl, 0, y), T1 = node_temp(q, g, wallTl, 1, y),
                 T2 = node_temp(q, g, wallTl, 2, y);
    acc[4] = -(-3.0 * T0 + 4.0 * T1 - T2) * 0.5 * (double)q.H_over_dT;
    acc[5] = 1.0;
  }
  for (int k = 0; k < NQ; ++k) sh[k][tid] = acc[k];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int k = 0; k < NQ; ++k) sh[k][tid] += sh[k][tid + w];
    __syncthreads();
  }
  if (tid == 0)
    for (int k = 0; k < NQ; ++k) rows[(long long)y * NQ + k] = sh[k][0];
}

__global__ void total_kernel(int ny, const double* rows, double* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[NQ] = {0, 0, 0, 0, 0, 0};
  for (int y = 0; y < ny; ++y)
    for (int k = 0; k < NQ; ++k) t[k] += rows[(long long)y * NQ + k];
  total[0] = t[0];
  total[1] = t[1];
  total[2] = t[3] > 0 ? t[2] / t[3] : 0.0;
  total[3] = t[5] > 0 ? t[4] / t[5] : 0.0;
}

std::mutex g_setup_mu;
double* g_rows_ptr[MAX_DEVICES];
double* g_total_ptr[MAX_DEVICES];

// device addresses of the scratch arrays on the current device (looked up once)
int scratch_for_current_device(double** rows, double** total) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return LBM_ERR_NO_DEVICE;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_rows_ptr[dev]) {
    void* pr = nullptr;
    void* pt = nullptr;
    if (cudaGetSymbolAddress(&pr, g_noalloc_rows) != cudaSuccess ||
        cudaGetSymbolAddress(&pt, g_noalloc_total) != cudaSuccess || !pr || !pt) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    g_rows_ptr[dev] = (double*)pr;
    g_total_ptr[dev] = (double*)pt;
  }
  *rows = g_rows_ptr[dev];
  *total = g_total_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_state_noalloc(const lbm_params* p, const float* f, const float* g,
                                        const float* fl, const float* phi,
                                        const float* wall_T_left, void* stream, double out[4]) {
  if (!p || !f || !g || !fl || !phi || !out) return LBM_ERR_INVALID_ARG;
  if (p->nx < 3 || p->ny < 3) return LBM_ERR_INVALID_ARG;
  if (p->ny > LBM_NOALLOC_MAX_ROWS) return LBM_ERR_INVALID_ARG;  // scratch holds one row each
  if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC)) return LBM_ERR_INVALID_ARG;
  if ((p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) return LBM_ERR_INVALID_ARG;
  if (!(p->sigma > 0) || !(p->St > 0)) return LBM_ERR_INVALID_ARG;
  double* rows = nullptr;
  double* total = nullptr;
  const int rc = scratch_for_current_device(&rows, &total);
  if (rc != LBM_OK) return rc;
  Geo q;
  memset(&q, 0, sizeof q);
  q.nx = p->nx;
  q.ny = p->ny;
  q.wl = q.wr = p->bc[0] != LBM_BC_PERIODIC;
  q.wb = q.wt = p->bc[2] != LBM_BC_PERIODIC;
  for (int k = 0; k < 4; ++k) {
    q.bc[k] = p->bc[k];
    q.Tbc[k] = (float)p->T_bc[k];
  }
  const double dT = p->dT > 0 ? p->dT : 1.0;
  const double H = p->H > 0 ? p->H : (double)p->ny;
  q.rho0 = (float)(p->rho0 > 0 ? p->rho0 : 1.0);
  q.lat = (float)(dT / (p->sigma * p->St));
  q.sigma_var = p->sigma_solid > 0 && p->sigma_solid != p->sigma;
  q.sigma_l = (float)p->sigma;
  q.sigma_s = (float)(q.sigma_var ? p->sigma_solid : p->sigma);
  q.H_over_dT = (float)(H / dT);
  cudaStream_t s = (cudaStream_t)stream;
  rows_kernel<<<p->ny, RED_THREADS, 0, s>>>(q, f, g, fl, phi, wall_T_left, rows);
  total_kernel<<<1, 32, 0, s>>>(p->ny, rows, total);
  double h[4];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h, total, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  memcpy(out, h, sizeof h);
  for (int k = 0; k < 4; ++k)
    if (!isfinite(h[k])) return LBM_ERR_NONFINITE;
  return LBM_OK;
}
