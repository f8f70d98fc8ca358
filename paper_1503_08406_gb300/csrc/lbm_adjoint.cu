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

// Per node: the source adjoint of step F and the clamp state of step E.
//   Ls(y) = sum_i w~_i lam_g'_i(y + e_i)
//   lam_f(y) = lam_f'(y) - a(y) Ls(y)           (non-wall; wall: lam_f')
//   c(y) = 1/(T_l - T_s + a) where 0 < z < 1, z from the state after the step
__global__ void adj_prep_kernel(Dev d, const float* g1, const float* f0, const float* f1,
                                const float* a, const float* lamg, const float* lamf_in,
                                float* lamf, float* ls, float* cinv, int* list, int* count) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  const int y = s / d.nx, x = s - y * d.nx;
  const int n = (int)d.n;
  const bool wall = (x == 0 || x == d.nx - 1);
  float L = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = adj_nb(d, x, y, ex9(i), ey9(i));
    if (t >= 0) L += wt(d, i) * lamg[i * n + t];
  }
  ls[s] = wall ? 0.f : L;
  float c = 0.f;
  if (!wall) {
    float T1 = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) T1 += g1[i * n + s];
    const float inv = 1.f / (d.dTt + a[s]);
    const float z = (T1 + a[s] * f1[s] - d.T_s) * inv;
    if (z > 0.f && z < 1.f) {
      c = inv;
      list[atomicAdd(count, 1)] = s;   // the fixed point's adjoint couples these nodes only
    }
    lamf[s] = lamf_in[s] - a[s] * L;
  } else {
    lamf[s] = lamf_in[s];
  }
  cinv[s] = c;
  (void)f0;
}

// The fixed point's adjoint on the unclamped nodes (elsewhere c mu = 0, and
// only c mu is used further on): Jacobi sweeps with the self term exact, from
// mu = 0, in one CTA (the unclamped nodes are a band along the front), until
// no node changes by more than MU_RTOL of its value or after max_sweeps; the
// result is left in mu0.  Leaves the list count at zero for the next step.
constexpr float MU_RTOL = 4e-7f;

__global__ void __launch_bounds__(1024) adj_mu_kernel(Dev d, const float* a, const float* cinv,
                                                      const float* lamf, const int* list,
                                                      int* count, float* mu0, float* mu1,
                                                      int max_sweeps) {
  const int cnt = *count;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) mu0[list[j]] = 0.f;
  __syncthreads();
  float* mu = mu0;
  float* mo = mu1;
  for (int k = 0; k < max_sweeps; ++k) {
    int moved = 0;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = list[j];
      const int y = s / d.nx, x = s - y * d.nx;
      float nb = 0.f;
#pragma unroll
      for (int i = 1; i < 5; ++i) {
        const int t = adj_nb(d, x, y, ex9(i), ey9(i));
        if (t >= 0) {
          const float ct = cinv[t];
          if (ct != 0.f) nb += ct * mu[t];
        }
      }
      const float as = a[s], cs = cinv[s];
      const float v = (lamf[s] - as * d.wt1 * nb) / (1.f - as * (1.f - d.wt0) * cs);
      moved |= fabsf(v - mu[s]) > MU_RTOL * fabsf(v);
      mo[s] = v;
    }
    moved = __syncthreads_or(moved);
    float* t = mu;
    mu = mo;
    mo = t;
    if (!moved) break;
  }
  if (mu != mu0)
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) mu0[list[j]] = mu[list[j]];
  __syncthreads();
  if (threadIdx.x == 0) *count = 0;
}

// The rest of the step's adjoint: from nu = c mu, the adjoint of the
// source-free streamed populations, streaming, collision and the wall
// extrapolation; the adjoints of f_l(n), a and the left wall profile.
//   lam_g*_i(x) = lam_g'_i(x) + nu(x)
//   lam_g+_i(x) = lam_g*_i(x + e_i)
//   lam_gpre = A^T lam_g+ per node
//   walls: lam_g(x_f) += lam_gpre(x_b) - (sum_i w~_i lam_gpre_i(x_b)), and the
//          Dirichlet value's adjoint is sum_i w~_i lam_gpre_i(x_b)
// This kernel writes lam_gpre; adj_walls_kernel folds the walls in.
__global__ void adj_back_kernel(Dev d, const float* f0, const float* f1, const float* a,
                                const float* cinv, const float* mu, const float* ls,
                                const float* lamg, const float* lamf, const float* At,
                                float* lamgpre, float* lamf0, float* lama) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  const int y = s / d.nx, x = s - y * d.nx;
  const int n = (int)d.n;
  const bool wall = (x == 0 || x == d.nx - 1);
  // streamed populations' adjoint at the downstream nodes, then A^T
  float lp[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = adj_nb(d, x, y, ex9(i), ey9(i));
    lp[i] = (t >= 0) ? lamg[i * n + t] + (cinv[t] != 0.f ? cinv[t] * mu[t] : 0.f) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) v += At[k * 5 + i] * lp[i];
    lamgpre[k * n + s] = v;
  }
  if (wall) {
    lamf0[s] = lamf[s];   // a wall node keeps f_l(n)
    return;
  }
  // sum_i w~_i nu(y + e_i) from the fixed point, plus the source term of step F
  float sn = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = adj_nb(d, x, y, ex9(i), ey9(i));
    if (t >= 0 && cinv[t] != 0.f) sn += wt(d, i) * cinv[t] * mu[t];
  }
  const float tot = ls[s] + sn;
  lamf0[s] = a[s] * tot;
  lama[s] += -(f1[s] - f0[s]) * tot;
}

// Wall columns: fold the extrapolation's adjoint into the inward column and
// the left wall profile; the wall nodes' own populations do not reach the
// next step (the extrapolation rewrites them).
__global__ void adj_walls_kernel(Dev d, float* lamgpre, float* lamtw) {
  const int y = blockIdx.x * AB + threadIdx.x;
  if (y >= d.ny) return;
  const int n = (int)d.n;
  for (int side = 0; side < 2; ++side) {
    const int xb = side ? d.nx - 1 : 0, xf = side ? d.nx - 2 : 1;
    const int b = y * d.nx + xb, f = y * d.nx + xf;
    float wl = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) wl += wt(d, i) * lamgpre[i * n + b];
    const bool dirichlet = d.bc[side] == 1;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      lamgpre[i * n + f] += lamgpre[i * n + b] - (dirichlet ? wl : 0.f);
      lamgpre[i * n + b] = 0.f;
    }
    if (dirichlet && side == 0) lamtw[y] += wl;
  }
}

// J = mean f_l over non-wall nodes (FP64 partial sums, one block)
__global__ void adj_objective_kernel(Dev d, const float* fl, double* out) {
  __shared__ double sh[AB];
  double acc = 0.0;
  for (int s = threadIdx.x; s < (int)d.n; s += AB) {
    const int x = s % d.nx;
    if (x != 0 && x != d.nx - 1) acc += fl[s];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = AB / 2; w > 0; w >>= 1) {
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
  adj_objective_kernel<<<1, AB, 0, s>>>(d, fl, out);
}

void adj_step(const Dev& d, const AdjBuffers& b, const float* g1, const float* f0, const float* f1,
              int mu_sweeps, cudaStream_t s) {
  const unsigned nb = blocks(d.n);
  adj_prep_kernel<<<nb, AB, 0, s>>>(d, g1, f0, f1, b.a, b.lamg, b.lamf, b.lamf_tot, b.ls, b.cinv,
                                    b.list, b.count);
  adj_mu_kernel<<<1, 1024, 0, s>>>(d, b.a, b.cinv, b.lamf_tot, b.list, b.count, b.mu0, b.mu1,
                                   mu_sweeps);
  adj_back_kernel<<<nb, AB, 0, s>>>(d, f0, f1, b.a, b.cinv, b.mu0, b.ls, b.lamg, b.lamf_tot, b.At,
                                    b.lamgpre, b.lamf, b.lama);
  adj_walls_kernel<<<blocks(d.ny), AB, 0, s>>>(d, b.lamgpre, b.lamtw);
}

}  // namespace lbm
