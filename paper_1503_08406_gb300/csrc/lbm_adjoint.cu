// Adjoint of the conduction step (flow lattice off): the reverse sweep of one
// time step for the gradient of an objective of the final liquid fraction.
//
// Forward map of one step, natural layout (population i of node x at slot
// (x, i)), written as the composition the adjoint reverses:
//   A  wall columns x_b (x = 0, nx - 1), from the inward node x_f (Sec. 4):
//      g(x_b) = w~ T_w + g(x_f) - w~ T(x_f)  (Dirichlet; adiabatic: g(x_f));
//   B  collision, linear with u = 0: g+ = N^-1 [n - Theta (n - n^eq)], n = N g,
//      n^eq = (T, 0, 0, varpi T, 0), Eq. (32)-(37);
//   C  streaming g*_i(x) = g+_i(x - e_i), periodic in y, nothing from beyond
//      the wall columns, Eq. (36);
//   E  enthalpy fixed point f = clamp(z), z(x) = (T*(x) + sum_i w~_i s(x - e_i)
//      + a(x) f(x) - T_s) / (T_l - T_s + a(x)), s = -a (f - f_l(n)) on
//      non-wall nodes, Eq. (38), (40)-(42); wall nodes keep f_l(n);
//   F  g(n+1)_i(x) = g*_i(x) + w~_i s(x - e_i).
// The fixed point's adjoint follows from the implicit function theorem on the
// nodes where 0 < z < 1 (elsewhere the clamp's derivative is 0): with
// c = 1/(T_l - T_s + a) on those nodes and 0 elsewhere, the adjoint mu solves
//   mu(y) = lam_f(y) + a(y) c(y) mu(y) - a(y) sum_i w~_i (c mu)(y + e_i),
// solved here by Jacobi sweeps over those nodes only, with the self term exact
// (a contraction: the row sums of the coupling are at most
// 4 w~_1 a / (T_l - T_s + w~_0 a) <= 2/3).
// At the fixed point z = f on those nodes, which removes the direct term of
// d z / d a.
#include "lbm_internal.cuh"

namespace lbm {

constexpr int AB = 256;   // block size of the adjoint kernels

__device__ __forceinline__ int adj_nb(const Dev& d, int x, int y, int dx, int dy) {
  const int xx = x + dx;
  if (xx < 0 || xx >= d.nx) return -1;
  int yy = y + dy;
  if (yy < 0) yy += d.ny;
  if (yy >= d.ny) yy -= d.ny;
  return yy * d.nx + xx;
}

__device__ __forceinline__ float wt(const Dev& d, int i) { return i == 0 ? d.wt0 : d.wt1; }

// Each reversed step is two kernels.  adj_full_kernel passes over the whole
// lattice once and takes every term that does not involve the fixed point's
// adjoint; adj_band_kernel (one CTA) solves that adjoint on the unclamped
// nodes, a band along the front, adds its share to the nodes next to the band
// and folds the wall columns.  With Ls(y) = sum_i w~_i lam_g'_i(y + e_i) (the
// source adjoint of step F) and nu = c mu:
//   lam_gpre = A^T lam_g+,  lam_g+_i(x) = lam_g'_i(x + e_i) + nu(x + e_i)
//   lam_f(n)(y) = a(y) (Ls(y) + sum_i w~_i nu(y + e_i))     (wall: lam_f')
//   lam_a(y) += -(f(n+1) - f(n))(y) (Ls(y) + sum_i w~_i nu(y + e_i))
//   walls: lam_g(x_f) += lam_gpre(x_b) - (sum_i w~_i lam_gpre_i(x_b)), and the
//          Dirichlet value's adjoint is sum_i w~_i lam_gpre_i(x_b)
// The first kernel writes the terms without nu; the second adds the nu terms,
// which are nonzero only at the band and its neighbours.

// Whole lattice: the terms without nu, the clamp state (c, from z evaluated on
// the state after the step) and the list of unclamped nodes with their
// lam_f(y) = lam_f'(y) - a(y) Ls(y), the right-hand side of mu's equation.
__global__ void adj_full_kernel(Dev d, AdjBuffers b, const float* T1, const float* f0,
                                const float* f1) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  const int y = s / d.nx, x = s - y * d.nx;
  const int n = (int)d.n;
  const bool wall = (x == 0 || x == d.nx - 1);
  float lp[5];
  float L = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = adj_nb(d, x, y, ex9(i), ey9(i));
    lp[i] = (t >= 0) ? b.lamg[i * n + t] : 0.f;
    L += wt(d, i) * lp[i];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) v += b.At[k * 5 + i] * lp[i];
    b.lamgpre[k * n + s] = v;
  }
  float c = 0.f;
  if (!wall) {
    const float as = b.a[s], fa = f1[s];
    const float inv = 1.f / (d.dTt + as);
    const float z = (T1[s] + as * fa - d.T_s) * inv;
    const float lf = b.lamf[s];
    if (z > 0.f && z < 1.f) {
      c = inv;
      b.lamf_tot[s] = lf - as * L;
      b.list[atomicAdd(b.count, 1)] = s;
    }
    b.lamf[s] = as * L;
    b.lama[s] += -(fa - f0[s]) * L;
  }
  b.cinv[s] = c;
}

// The fixed point's adjoint on the band: Jacobi sweeps with the self term
// exact, from mu = 0, until no node changes by more than MU_RTOL of its value
// or after max_sweeps.  Up to BAND_CAP band nodes sweep in shared memory (each
// node's coefficients and its neighbours' places in the list staged once);
// a wider band sweeps in global memory.  Jacobi makes the result independent
// of the list's order.
constexpr float MU_RTOL = 4e-7f;
constexpr int BAND_CAP = 4096;
constexpr int BAND_THREADS = 1024;
constexpr int BAND_SMEM = BAND_CAP * (int)(sizeof(float4) + sizeof(ushort4) + 5 * sizeof(float));

__device__ __forceinline__ bool in_band(const AdjBuffers& b, int t) {
  return t >= 0 && b.cinv[t] != 0.f;
}

__global__ void __launch_bounds__(BAND_THREADS) adj_band_kernel(Dev d, AdjBuffers b,
                                                                const float* f0, const float* f1,
                                                                int max_sweeps) {
  extern __shared__ float4 band_smem[];
  const int cnt = *b.count;
  const int n = (int)d.n;
  if (cnt <= BAND_CAP) {
    float4* ct = band_smem;                                    // c of the 4 neighbours
    ushort4* ix = reinterpret_cast<ushort4*>(ct + BAND_CAP);   // their places in the list
    float* rhs = reinterpret_cast<float*>(ix + BAND_CAP);
    float* kk = rhs + BAND_CAP;                                // a w~_1
    float* dd = kk + BAND_CAP;                                 // 1 - a (1 - w~_0) c
    float* mu = dd + BAND_CAP;
    float* mo = mu + BAND_CAP;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) b.pos[b.list[j]] = j;
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = b.list[j];
      const int y = s / d.nx, x = s - y * d.nx;
      float c4[4];
      unsigned short i4[4];
#pragma unroll
      for (int i = 1; i < 5; ++i) {
        const int t = adj_nb(d, x, y, ex9(i), ey9(i));
        const bool on = in_band(b, t);
        c4[i - 1] = on ? b.cinv[t] : 0.f;
        i4[i - 1] = (unsigned short)(on ? b.pos[t] : j);
      }
      ct[j] = make_float4(c4[0], c4[1], c4[2], c4[3]);
      ix[j] = make_ushort4(i4[0], i4[1], i4[2], i4[3]);
      const float as = b.a[s];
      rhs[j] = b.lamf_tot[s];
      kk[j] = as * d.wt1;
      dd[j] = 1.f - as * (1.f - d.wt0) * b.cinv[s];
      mu[j] = 0.f;
    }
    __syncthreads();
    for (int k = 0; k < max_sweeps; ++k) {
      int moved = 0;
      for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const float4 c = ct[j];
        const ushort4 q = ix[j];
        const float nb = c.x * mu[q.x] + c.y * mu[q.y] + c.z * mu[q.z] + c.w * mu[q.w];
        const float v = (rhs[j] - kk[j] * nb) / dd[j];
        moved |= fabsf(v - mu[j]) > MU_RTOL * fabsf(v);
        mo[j] = v;
      }
      moved = __syncthreads_or(moved);
      float* t = mu;
      mu = mo;
      mo = t;
      if (!moved) break;
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = b.list[j];
      b.nu[s] = b.cinv[s] * mu[j];
    }
  } else {
    float* mu = b.mu0;
    float* mo = b.mu1;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) mu[b.list[j]] = 0.f;
    __syncthreads();
    for (int k = 0; k < max_sweeps; ++k) {
      int moved = 0;
      for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int s = b.list[j];
        const int y = s / d.nx, x = s - y * d.nx;
        float nb = 0.f;
#pragma unroll
        for (int i = 1; i < 5; ++i) {
          const int t = adj_nb(d, x, y, ex9(i), ey9(i));
          nb += in_band(b, t) ? b.cinv[t] * mu[t] : 0.f;
        }
        const float as = b.a[s];
        const float v = (b.lamf_tot[s] - as * d.wt1 * nb) / (1.f - as * (1.f - d.wt0) * b.cinv[s]);
        moved |= fabsf(v - mu[s]) > MU_RTOL * fabsf(v);
        mo[s] = v;
      }
      moved = __syncthreads_or(moved);
      float* t = mu;
      mu = mo;
      mo = t;
      if (!moved) break;
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = b.list[j];
      b.nu[s] = b.cinv[s] * mu[s];
    }
  }
  __syncthreads();
  // the nu terms at every node y with a band node among y + e_i: each such y
  // is taken by the band node y + e_i of smallest i, so once
  for (int q = threadIdx.x; q < 5 * cnt; q += blockDim.x) {
    const int j = q / 5, i = q - 5 * j;
    const int t = b.list[j];
    const int ty = t / d.nx, tx = t - ty * d.nx;
    const int s = adj_nb(d, tx, ty, -ex9(i), -ey9(i));
    if (s < 0) continue;
    const int y = s / d.nx, x = s - y * d.nx;
    bool first = true;
    for (int m = 0; m < i; ++m) first = first && !in_band(b, adj_nb(d, x, y, ex9(m), ey9(m)));
    if (!first) continue;
    float nv[5];
    float sn = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const int u = adj_nb(d, x, y, ex9(m), ey9(m));
      nv[m] = in_band(b, u) ? b.nu[u] : 0.f;
      sn += wt(d, m) * nv[m];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float v = 0.f;
#pragma unroll
      for (int m = 0; m < 5; ++m) v += b.At[k * 5 + m] * nv[m];
      b.lamgpre[k * n + s] += v;
    }
    if (x != 0 && x != d.nx - 1) {
      b.lamf[s] += b.a[s] * sn;
      b.lama[s] += -(f1[s] - f0[s]) * sn;
    }
  }
  __syncthreads();
  // wall columns: fold the extrapolation's adjoint into the inward column and
  // the left wall profile; the wall nodes' own populations do not reach the
  // next step (the extrapolation rewrites them)
  for (int y = threadIdx.x; y < d.ny; y += blockDim.x) {
    for (int side = 0; side < 2; ++side) {
      const int xb = side ? d.nx - 1 : 0, xf = side ? d.nx - 2 : 1;
      const int bn = y * d.nx + xb, fn = y * d.nx + xf;
      float wl = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) wl += wt(d, i) * b.lamgpre[i * n + bn];
      const bool dirichlet = d.bc[side] == 1;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        b.lamgpre[i * n + fn] += b.lamgpre[i * n + bn] - (dirichlet ? wl : 0.f);
        b.lamgpre[i * n + bn] = 0.f;
      }
      if (dirichlet && side == 0) b.lamtw[y] += wl;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *b.count = 0;
}

// J = mean f_l over non-wall nodes (FP64 partial sums, one block)
constexpr int OB = 1024;
__global__ void __launch_bounds__(OB) adj_objective_kernel(Dev d, const float* fl, double* out) {
  __shared__ double sh[OB];
  double acc = 0.0;
  for (int y = 0; y < d.ny; ++y)
    for (int x = 1 + threadIdx.x; x < d.nx - 1; x += OB) acc += fl[(long long)y * d.nx + x];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = OB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / ((double)(d.nx - 2) * d.ny);
}

__global__ void adj_seed_kernel(Dev d, float* lamf, float* lamg) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  const int x = s % d.nx;
  lamf[s] = (x != 0 && x != d.nx - 1) ? 1.f / ((float)(d.nx - 2) * d.ny) : 0.f;
  for (int i = 0; i < 5; ++i) lamg[i * (int)d.n + s] = 0.f;
}

__global__ void adj_a_kernel(Dev d, float* a) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  a[s] = d.phi[s] * d.lat;
}

static unsigned blocks(long long n) { return (unsigned)((n + AB - 1) / AB); }

void adj_seed(const Dev& d, float* lamf, float* lamg, float* a, cudaStream_t s) {
  adj_seed_kernel<<<blocks(d.n), AB, 0, s>>>(d, lamf, lamg);
  adj_a_kernel<<<blocks(d.n), AB, 0, s>>>(d, a);
}

void adj_objective(const Dev& d, const float* fl, double* out, cudaStream_t s) {
  adj_objective_kernel<<<1, OB, 0, s>>>(d, fl, out);
}

bool adj_init() {
  return cudaFuncSetAttribute(adj_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BAND_SMEM) == cudaSuccess;
}

void adj_step(const Dev& d, const AdjBuffers& b, const float* T1, const float* f0, const float* f1,
              int mu_sweeps, cudaStream_t s) {
  adj_full_kernel<<<blocks(d.n), AB, 0, s>>>(d, b, T1, f0, f1);
  adj_band_kernel<<<1, BAND_THREADS, BAND_SMEM, s>>>(d, b, f0, f1, mu_sweeps);
}

}  // namespace lbm
