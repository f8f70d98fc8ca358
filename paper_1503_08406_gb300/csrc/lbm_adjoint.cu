// Adjoint of the conduction step (flow lattice off): the reverse sweep of one
// time step for the gradient of an objective (the final melted fraction, or
// the left-wall Nusselt number averaged over the steps) with respect to the
// porosity field and the left wall's temperature profile.
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
#include "lbm_adjoint.cuh"
#include "lbm_flow_adjoint.cuh"

namespace lbm {

constexpr int AB = 256;   // block size of the adjoint kernels

// neighbour (x + dx, y + dy): wraps on periodic axes, -1 beyond a wall side
__device__ __forceinline__ int adj_nb(const Dev& d, int x, int y, int dx, int dy) {
  int xx = x + dx, yy = y + dy;
  if (xx < 0 || xx >= d.nx) {
    if (!d.per_x) return -1;
    xx = xx < 0 ? xx + d.nx : xx - d.nx;
  }
  if (yy < 0 || yy >= d.ny) {
    if (!d.per_y) return -1;
    yy = yy < 0 ? yy + d.ny : yy - d.ny;
  }
  return yy * d.nx + xx;
}

__device__ __forceinline__ float wt(const Dev& d, int i) { return i == 0 ? d.wt0 : d.wt1; }

// Each reversed step is two kernels.  adj_band_kernel (one CTA) solves the
// fixed point's adjoint on the unclamped nodes, a band along the front, and
// adds nu = c mu there to lam_g' (nu is 0 elsewhere).  adj_full_kernel passes
// over the whole lattice once: with lam_g+_i(x) = lam_g'_i(x + e_i) + nu(x + e_i) and
// S(y) = sum_i w~_i lam_g+_i(y) (the source adjoint of step F, the fixed
// point's share included),
//   lam_gpre = A^T lam_g+ per node
//   lam_f(n)(y) = a(y) S(y)                       (wall: lam_f')
//   lam_a(y) += -(f(n+1) - f(n))(y) S(y)
//   plus the objective's direct terms in the state before the step (the
//   Nusselt number's T_1, T_2 and T_w)
//   walls: lam_g(x_f) += lam_gpre(x_b) - (sum_i w~_i lam_gpre_i(x_b)), and the
//          Dirichlet value's adjoint is sum_i w~_i lam_gpre_i(x_b); the wall
//          nodes' own populations do not reach the next step (the
//          extrapolation rewrites them).
// The unclamped nodes of a step are the non-wall nodes with 0 < f_l < 1 after
// it (the solver converges to f = z there, and clamps elsewhere); the full
// pass of one reversed step lists them for the next (its f(n) is the next
// one's f(n+1)).

__device__ __forceinline__ bool band_node(const Dev& d, const float* f, int t) {
  if (t < 0) return false;
  const int y = t / d.nx, x = t - y * d.nx;
  const float v = f[t];
  return !is_wall(d, x, y) && adj_mushy(v);
}

// the band of the state with liquid fraction f, appended at list[*count]
__global__ void adj_list_kernel(Dev d, const float* f, int* list, int* count) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  if (band_node(d, f, s)) list[atomicAdd(count, 1)] = s;
}

// The fixed point's adjoint on the band: right-hand side
// lam_f'(y) - a(y) sum_i w~_i lam_g'_i(y + e_i), then red-black sweeps with the
// self term exact, from mu = 0: nodes with x + y even, then odd (a node's four
// neighbours have the other colour, so each colour updates in place, in any
// order), over-relaxed by MU_OMEGA for the first MU_SOR sweeps, until no node
// changes by more than MU_RTOL of its value or after max_sweeps.  The result
// does not depend on the list's order.  Up to BAND_CAP band nodes sweep in
// shared memory (each node's coefficients and its neighbours' places in the
// list staged once); a wider band sweeps in global memory.  Empties the
// previous band's list (old_count) for the full pass to refill.
constexpr float MU_RTOL = 4e-7f;
// The Jacobi map's spectral radius is at most 2/3 here, so red-black SOR
// converges fastest near omega = 2 / (1 + sqrt(1 - 4/9)) = 1.146
constexpr float MU_OMEGA = 1.15f;
constexpr int MU_SOR = 6;
constexpr int BAND_CAP = 4096;
constexpr int BAND_THREADS = 1024;
constexpr int BAND_SMEM = BAND_CAP * (int)(sizeof(float4) + sizeof(ushort4) + 4 * sizeof(float) + 1);

// right-hand side of mu's equation at band node s
__device__ __forceinline__ float band_rhs(const Dev& d, const AdjBuffers& b, int s) {
  const int y = s / d.nx, x = s - y * d.nx;
  const int n = (int)d.n;
  float L = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int t = adj_nb(d, x, y, ex9(i), ey9(i));
    L += wt(d, i) * ((t >= 0) ? b.lamg[i * n + t] : 0.f);
  }
  return b.lamf[s] - b.a[s] * L;
}

// nu = c mu at band node s joins every lam_g'_i there (lam_g+_i(x) takes
// lam_g'_i + nu at x + e_i; nothing else reads lam_g' after this kernel)
__device__ __forceinline__ void add_nu(const Dev& d, const AdjBuffers& b, int s, float v) {
#pragma unroll
  for (int i = 0; i < 5; ++i) b.lamg[i * (long long)d.n + s] += v;
}

__global__ void __launch_bounds__(BAND_THREADS) adj_band_kernel(Dev d, AdjBuffers b,
                                                                const float* f1, const int* list,
                                                                const int* count, int* old_count,
                                                                int max_sweeps) {
  extern __shared__ float4 band_smem[];
  const int cnt = *count;
  if (cnt <= BAND_CAP) {
    float4* ct = band_smem;                                    // c of the 4 neighbours
    ushort4* ix = reinterpret_cast<ushort4*>(ct + BAND_CAP);   // their places in the list
    float* rhs = reinterpret_cast<float*>(ix + BAND_CAP);      // divided by dd
    float* kk = rhs + BAND_CAP;                                // a w~_1, divided by dd
    float* dd = kk + BAND_CAP;                                 // 1 - a (1 - w~_0) c
    float* mu = dd + BAND_CAP;
    unsigned char* col = reinterpret_cast<unsigned char*>(mu + BAND_CAP);   // x + y parity
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) b.pos[list[j]] = j;
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = list[j];
      const int y = s / d.nx, x = s - y * d.nx;
      float c4[4];
      unsigned short i4[4];
#pragma unroll
      for (int i = 1; i < 5; ++i) {
        const int t = adj_nb(d, x, y, ex9(i), ey9(i));
        const bool on = band_node(d, f1, t);
        c4[i - 1] = on ? 1.f / (d.dTt + b.a[t]) : 0.f;
        i4[i - 1] = (unsigned short)(on ? b.pos[t] : j);
      }
      ct[j] = make_float4(c4[0], c4[1], c4[2], c4[3]);
      ix[j] = make_ushort4(i4[0], i4[1], i4[2], i4[3]);
      const float as = b.a[s];
      const float den = 1.f - as * (1.f - d.wt0) / (d.dTt + as);
      rhs[j] = band_rhs(d, b, s) / den;
      kk[j] = as * d.wt1 / den;
      mu[j] = 0.f;
      col[j] = (unsigned char)((x + y) & 1);
    }
    __syncthreads();
    bool more = true;
    for (int k = 0; k < max_sweeps && more; ++k) {
      const float om = k < MU_SOR ? MU_OMEGA : 1.f;
      int moved = 0;
      for (int c0 = 0; c0 < 2; ++c0) {
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
          if (col[j] != c0) continue;
          const float4 c = ct[j];
          const ushort4 q = ix[j];
          const float nb = c.x * mu[q.x] + c.y * mu[q.y] + c.z * mu[q.z] + c.w * mu[q.w];
          const float raw = rhs[j] - kk[j] * nb;
          const float o = mu[j];
          const float v = o + om * (raw - o);
          moved |= fabsf(v - o) > MU_RTOL * fabsf(v);
          mu[j] = v;
        }
        if (c0 == 0) __syncthreads();
      }
      more = __syncthreads_or(moved);
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = list[j];
      add_nu(d, b, s, mu[j] / (d.dTt + b.a[s]));
    }
  } else {
    float* mu = b.mu0;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = list[j];
      const float as = b.a[s];
      b.rhs[s] = band_rhs(d, b, s) / (1.f - as * (1.f - d.wt0) / (d.dTt + as));
      mu[s] = 0.f;
    }
    __syncthreads();
    bool more = true;
    for (int k = 0; k < max_sweeps && more; ++k) {
      const float om = k < MU_SOR ? MU_OMEGA : 1.f;
      int moved = 0;
      for (int c0 = 0; c0 < 2; ++c0) {
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
          const int s = list[j];
          const int y = s / d.nx, x = s - y * d.nx;
          if (((x + y) & 1) != c0) continue;
          float nb = 0.f;
#pragma unroll
          for (int i = 1; i < 5; ++i) {
            const int t = adj_nb(d, x, y, ex9(i), ey9(i));
            nb += band_node(d, f1, t) ? mu[t] / (d.dTt + b.a[t]) : 0.f;
          }
          const float as = b.a[s];
          const float raw = b.rhs[s] - as * d.wt1 / (1.f - as * (1.f - d.wt0) / (d.dTt + as)) * nb;
          const float o = mu[s];
          const float v = o + om * (raw - o);
          moved |= fabsf(v - o) > MU_RTOL * fabsf(v);
          mu[s] = v;
        }
        if (c0 == 0) __syncthreads();
      }
      more = __syncthreads_or(moved);
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const int s = list[j];
      add_nu(d, b, s, mu[s] / (d.dTt + b.a[s]));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *old_count = 0;
}

// lam_g+ of node (x, y) (rows yu = y + 1, yd = y - 1, periodic) and A^T of it
__device__ __forceinline__ void pre_pops(const Dev& d, const AdjBuffers& b, const Mat5& At, int x,
                                         int y, int yu, int yd, float lp[5], float out[5]) {
  const int n = (int)d.n;
  const int s = y * d.nx + x;
  const int t[5] = {s, x + 1 < d.nx ? s + 1 : -1, yu * d.nx + x, x > 0 ? s - 1 : -1,
                    yd * d.nx + x};
#pragma unroll
  for (int i = 0; i < 5; ++i)
    lp[i] = (t[i] >= 0) ? __ldg(b.lamg + i * n + t[i]) : 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) v += At.m[k * 5 + i] * lp[i];
    out[k] = v;
  }
}

// one row segment per block (x along threads, y = blockIdx.y + k gridDim.y)
__global__ void __launch_bounds__(AB) adj_full_kernel(Dev d, AdjBuffers b, Mat5 At, NuSrc nu,
                                                      const float* __restrict__ f0,
                                                      const float* __restrict__ f1,
                                                      int* next_list, int* next_count) {
  const int x = blockIdx.x * AB + threadIdx.x;
  if (x >= d.nx) return;
  const int n = (int)d.n;
  for (int y = blockIdx.y; y < d.ny; y += gridDim.y) {
    const int yu = y + 1 == d.ny ? 0 : y + 1, yd = y == 0 ? d.ny - 1 : y - 1;
    const int s = y * d.nx + x;
    float lp[5], pre[5];
    pre_pops(d, b, At, x, y, yu, yd, lp, pre);
    if (x == 0 || x == d.nx - 1) {
      if (x == 0 && d.bc[0] == 1) {
        float wl = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) wl += wt(d, i) * pre[i];
        b.lamtw[y] += wl + nu.tw;
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) b.lamgpre[k * n + s] = 0.f;
      continue;   // a wall node keeps f_l(n): lam_f unchanged, no share of a
    }
    // an inward column also takes its wall node's adjoint
    for (int side = 0; side < 2; ++side) {
      if (x != (side ? d.nx - 2 : 1)) continue;
      float lw[5], pw[5];
      pre_pops(d, b, At, side ? d.nx - 1 : 0, y, yu, yd, lw, pw);
      float wl = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) wl += wt(d, i) * pw[i];
      if (d.bc[side] != 1) wl = 0.f;
#pragma unroll
      for (int k = 0; k < 5; ++k) pre[k] += pw[k] - wl;
    }
    const float src = x == 1 ? nu.g1 : x == 2 ? nu.g2 : 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) b.lamgpre[k * n + s] = pre[k] + src;
    float S = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) S += wt(d, i) * lp[i];
    const float fa = f0[s], fb = f1[s];
    b.lamf[s] = __ldg(b.a + s) * S;
    if (fb != fa) b.lama[s] += -(fb - fa) * S;   // (adds 0 elsewhere)
    if (adj_mushy(fa)) next_list[atomicAdd(next_count, 1)] = s;
  }
}

// Forward runs that keep every step's f_l: copies d.fl to base + k n, k the
// counter at *ctr, which the last block to finish advances (no block waits).
__global__ void adj_save_kernel(Dev d, float* base, unsigned* ctr, unsigned* done) {
  const unsigned k = *ctr;
  const long long n = d.n;
  float* dst = base + (long long)k * n;
  for (long long s = blockIdx.x * (long long)AB + threadIdx.x; s < n; s += (long long)gridDim.x * AB)
    dst[s] = d.fl[s];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      *done = 0;
      *ctr = k + 1;
    }
  }
}

// J = mean f_l over non-wall nodes: FP64 partial sums per row block, then
// their sum in a fixed order
constexpr int OB = 256, OBLOCKS = 128;
__global__ void __launch_bounds__(OB) adj_partial_kernel(Dev d, const float* fl, double* part) {
  __shared__ double sh[OB];
  double acc = 0.0;
  for (int y = blockIdx.x; y < d.ny; y += gridDim.x)
    for (int x = 1 + threadIdx.x; x < d.nx - 1; x += OB) acc += fl[(long long)y * d.nx + x];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = OB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void adj_objective_kernel(Dev d, const double* part, int nparts, double* out) {
  if (threadIdx.x != 0) return;
  double acc = 0.0;
  for (int k = 0; k < nparts; ++k) acc += part[k];
  *out = acc / ((double)(d.nx - 2) * d.ny);
}

__global__ void adj_seed_kernel(Dev d, float* lamf, float* lamg, bool melt, NuSrc nu) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  const int x = s % d.nx;
  lamf[s] = (melt && x != 0 && x != d.nx - 1) ? 1.f / ((float)(d.nx - 2) * d.ny) : 0.f;
  const float src = x == 1 ? nu.g1 : x == 2 ? nu.g2 : 0.f;
  for (int i = 0; i < 5; ++i) lamg[i * (int)d.n + s] = src;
}

__global__ void adj_scale_kernel(long long n, float* v, float k) {
  const long long s = blockIdx.x * (long long)AB + threadIdx.x;
  if (s < n) v[s] *= k;
}

__global__ void adj_a_kernel(Dev d, float* a) {
  const int s = blockIdx.x * AB + threadIdx.x;
  if (s >= (int)d.n) return;
  a[s] = d.phi[s] * d.lat;
}

static unsigned blocks(long long n) { return (unsigned)((n + AB - 1) / AB); }

void adj_seed(const Dev& d, float* lamf, float* lamg, float* a, bool melt, NuSrc nu,
              cudaStream_t s) {
  adj_seed_kernel<<<blocks(d.n), AB, 0, s>>>(d, lamf, lamg, melt, nu);
  adj_a_kernel<<<blocks(d.n), AB, 0, s>>>(d, a);
}

__global__ void adj_mul_kernel(long long n, float* v, const float* w) {
  const long long s = blockIdx.x * (long long)AB + threadIdx.x;
  if (s < n) v[s] *= w[s];
}

void adj_mul(long long n, float* v, const float* w, cudaStream_t s) {
  adj_mul_kernel<<<(unsigned)((n + AB - 1) / AB), AB, 0, s>>>(n, v, w);
}

void adj_a(const Dev& d, float* a, cudaStream_t s) {
  adj_a_kernel<<<blocks(d.n), AB, 0, s>>>(d, a);
}

void adj_scale(long long n, float* v, float k, cudaStream_t s) {
  adj_scale_kernel<<<(unsigned)((n + AB - 1) / AB), AB, 0, s>>>(n, v, k);
}

void adj_objective(const Dev& d, const float* fl, double* out, cudaStream_t s) {
  const int nb = d.ny < OBLOCKS ? d.ny : OBLOCKS;
  adj_partial_kernel<<<nb, OB, 0, s>>>(d, fl, out + 1);
  adj_objective_kernel<<<1, 32, 0, s>>>(d, out + 1, nb, out);
}

// One reversed coupled step (flow on): lbm::coupled_reverse_node per node,
// rows along blockIdx.y.
__global__ void __launch_bounds__(128, 8) adj_coupled_kernel(CoupledStep<float> A) {
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= A.geo.nx) return;
  for (int y = blockIdx.y; y < A.geo.ny; y += gridDim.y) coupled_reverse_node(A, x, y);
}

void adj_coupled_step(const Dev& d, const AdjBuffers& b, const CoupledStep<float>& A, int* list,
                      int* count, int* old_count, int mu_sweeps, cudaStream_t s) {
  adj_band_kernel<<<1, BAND_THREADS, BAND_SMEM, s>>>(d, b, A.fl1, list, count, old_count,
                                                     mu_sweeps);
  const dim3 grid((d.nx + 127) / 128, d.ny < 65535 ? d.ny : 65535);
  adj_coupled_kernel<<<grid, 128, 0, s>>>(A);
}

bool adj_init() {
  return cudaFuncSetAttribute(adj_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BAND_SMEM) == cudaSuccess;
}

void adj_list(const Dev& d, const float* f, int* list, int* count, cudaStream_t s) {
  adj_list_kernel<<<blocks(d.n), AB, 0, s>>>(d, f, list, count);
}

void adj_save(const Dev& d, float* base, unsigned* ctr, cudaStream_t s) {
  long long nb = (d.n + 4LL * AB - 1) / (4LL * AB);
  if (nb > 4 * 152) nb = 4 * 152;
  adj_save_kernel<<<(unsigned)nb, AB, 0, s>>>(d, base, ctr, ctr + 1);
}

void adj_step(const Dev& d, const AdjBuffers& b, const float* f0, const float* f1, int* list,
              int* count, int* old_list, int* old_count, int mu_sweeps, NuSrc nu,
              cudaStream_t s) {
  adj_band_kernel<<<1, BAND_THREADS, BAND_SMEM, s>>>(d, b, f1, list, count, old_count,
                                                     mu_sweeps);
  Mat5 At;
  for (int k = 0; k < 25; ++k) At.m[k] = b.At[k];
  const dim3 grid((d.nx + AB - 1) / AB, d.ny < 65535 ? d.ny : 65535);
  adj_full_kernel<<<grid, AB, 0, s>>>(d, b, At, nu, f0, f1, old_list, old_count);
}

}  // namespace lbm
