// C ABI of liblbm (declared in include/lbm.h): context, parameter derivation,
// workspace layout, step sequencing, outputs.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint.cuh"

using lbm::Dev;

struct lbm_ctx {
  lbm_params p;
  Dev d;
  cudaStream_t stream;
  void* ws;
  size_t ws_bytes;
  bool own_ws;
  int64_t steps;
  int parity;          // layout before the next step: 0 natural (next step even), 1 swapped
  double derived[8];
  float* tmp;          // staging for host inputs/outputs, 9 n floats
  double* partials;
  double* sums;        // 8 doubles
  int* bad;            // validation flag
  int nred;
  bool timing;
  std::vector<cudaEvent_t> ev;   // per step: start, after fused, after enthalpy
  // CUDA graphs of 2..GRAPH_MAX steps from either step parity, captured on a
  // private stream when first needed and replayed on the context stream
  cudaStream_t cap, cap2;         // capture streams (the second one runs the far-tile fused pass)
  cudaEvent_t ev_fork, ev_join;
  cudaGraphExec_t gx[2][65];       // [start parity][steps], GRAPH_MAX = 64
  int gnl[2][65];                  // kernels in each graph
  bool graphs_off;
  int64_t launches;                // kernels launched by lbm_step
  int64_t since_check;             // steps since the last NaN/Inf sentinel
  double adj_ms[2];                // last adjoint call: forward run, reverse sweep (device ms)
  void* trace_buf;                 // lbm_trace records (library-allocated), or null
  lbm::TmaMaps maps;               // tensor maps of the TMA-staged fused kernel
  bool use_tma;
  bool tma_ok;                     // the lattice qualifies for the TMA-staged kernel
  int tpc;                         // its tiles per CTA
  const lbm::TmaMaps* tma() const { return use_tma ? &maps : nullptr; }
};

// longest graph lbm_step replays; a call of n steps launches n / GRAPH_MAX of
// them and one graph of the remainder, so only one graph boundary (where the
// far-tile overlap restarts) falls in every GRAPH_MAX steps
static const int GRAPH_MAX = 64;

namespace {

const double CS2 = 1.0 / 3.0;

int derive(lbm_params* p, double out[8]) {
  if (p->H <= 0) p->H = p->ny;
  if (p->dT <= 0) p->dT = 1;
  if (p->rho0 <= 0) p->rho0 = 1;
  if (p->s_e <= 0) p->s_e = 1.1;
  if (p->s_eps <= 0) p->s_eps = 1.1;
  if (p->s_q <= 0) p->s_q = 1.2;
  if (p->zeta_e <= 0) p->zeta_e = 1.5;
  if (p->zeta_nu <= 0) p->zeta_nu = 1.5;
  if (p->J <= 0) p->J = 1;
  if (p->lambda_ <= 0) p->lambda_ = 1;
  if (p->f_act <= 0) p->f_act = 1e-3;
  if (p->max_inner_iters <= 0) p->max_inner_iters = 1000;
  if (!(p->sigma > 0) || !(p->St > 0)) return LBM_ERR_INVALID_ARG;
  if (!(p->varpi > -4 && p->varpi < 1)) return LBM_ERR_INVALID_ARG;
  if (!(p->T_l >= p->T_s)) return LBM_ERR_INVALID_ARG;
  const double csT2 = (4 + p->varpi) / 10.0;  // Eq. (39)
  double tau_nu = 0, tau_T, nu_e = 0, nu_l = 0, g_beta = 0;
  if (p->flow) {
    if (p->tau_nu > 0) tau_nu = p->tau_nu;
    else if (p->Ra > 0 && p->Pr > 0 && p->Ma > 0)
      tau_nu = 0.5 + p->Ma * p->J * p->H * sqrt(3 * p->Pr) / sqrt(p->Ra);  // Sec. 4.3
    else return LBM_ERR_INVALID_ARG;
    nu_e = CS2 * (tau_nu - 0.5);
    nu_l = nu_e / p->J;
    if (p->tau_T > 0) {
      tau_T = p->tau_T;
    } else {
      if (!(p->Pr > 0)) return LBM_ERR_INVALID_ARG;
      tau_T = 0.5 + p->lambda_ * CS2 * (tau_nu - 0.5) / (p->J * p->sigma * csT2 * p->Pr);
    }
    if (p->g_beta >= 0) {
      g_beta = p->g_beta;
    } else {
      if (!(p->Ra > 0) || !(p->Pr > 0)) return LBM_ERR_INVALID_ARG;
      g_beta = p->Ra * nu_l * (nu_l / p->Pr) / (p->dT * p->H * p->H * p->H);  // Eq. (9)
    }
    if (!(tau_nu > 0.5)) return LBM_ERR_INVALID_ARG;
  } else {
    if (!(p->tau_T > 0)) return LBM_ERR_INVALID_ARG;
    tau_T = p->tau_T;
  }
  if (!(tau_T > 0.5)) return LBM_ERR_INVALID_ARG;
  out[0] = tau_nu;
  out[1] = tau_T;
  out[2] = nu_e;
  out[3] = nu_l;
  out[4] = p->sigma * csT2 * (tau_T - 0.5);  // alpha_e, Eq. (39)
  out[5] = g_beta;
  out[6] = csT2;
  out[7] = p->dT / (p->sigma * p->St);
  return LBM_OK;
}

int check_params(const lbm_params* p) {
  if (!p) return LBM_ERR_INVALID_ARG;
  if (p->nx < 3 || p->ny < 3) return LBM_ERR_INVALID_ARG;
  // 32-bit node offsets address all 14 population planes
  if ((long long)p->nx * p->ny * 14 >= (1LL << 31)) return LBM_ERR_INVALID_ARG;
  for (int k = 0; k < 4; ++k)
    if (p->bc[k] < LBM_BC_PERIODIC || p->bc[k] > LBM_BC_ADIABATIC) return LBM_ERR_INVALID_ARG;
  if ((p->bc[0] == LBM_BC_PERIODIC) != (p->bc[1] == LBM_BC_PERIODIC)) return LBM_ERR_INVALID_ARG;
  if ((p->bc[2] == LBM_BC_PERIODIC) != (p->bc[3] == LBM_BC_PERIODIC)) return LBM_ERR_INVALID_ARG;
  if (p->kernel_variant < 0 || p->kernel_variant > 2) return LBM_ERR_INVALID_ARG;
  if (p->storage < LBM_STORAGE_FP32 || p->storage > LBM_STORAGE_BF16) return LBM_ERR_INVALID_ARG;
  if (!(p->alpha_ratio >= 0)) return LBM_ERR_INVALID_ARG;
  if (!(p->sigma_solid >= 0)) return LBM_ERR_INVALID_ARG;
  if (p->flow_walls < 0 || p->flow_walls > 1) return LBM_ERR_INVALID_ARG;
  if (p->flow_front < 0 || p->flow_front > 1) return LBM_ERR_INVALID_ARG;
  return LBM_OK;
}

struct Layout {
  size_t f, g, fl, phi, K, wallTl, flags, list, lcount, ctr, nearmap, proc, tact, scr, stats,
      tmp, partials, sums, bad, total;
};

size_t up(size_t v) { return (v + 255) & ~(size_t)255; }

Layout layout_of(const lbm_params* p, int nred) {
  const size_t n = (size_t)p->nx * p->ny;
  const size_t tiles = (size_t)((p->nx + lbm::TE - 1) / lbm::TE) * ((p->ny + lbm::TE - 1) / lbm::TE);
  Layout L;
  size_t o = 0;
  const size_t es = p->storage == LBM_STORAGE_FP32 ? sizeof(float) : 2;   // bytes per population
  L.f = o; o += up(9 * n * es);
  L.g = o; o += up(5 * n * es);
  L.fl = o; o += up(n * sizeof(float));
  L.phi = o; o += up(n * sizeof(float));
  L.K = o; o += up(n * sizeof(float));
  L.wallTl = o; o += up((size_t)p->ny * sizeof(float));
  L.flags = o; o += up(2 * tiles * sizeof(int));
  L.list = o; o += up(2 * tiles * sizeof(int));
  L.lcount = o; o += up(2 * sizeof(int));
  L.ctr = o; o += up(2 * sizeof(int));
  L.nearmap = o; o += up(2 * tiles * sizeof(int));
  L.proc = o; o += up(tiles * sizeof(int));
  L.tact = o; o += up(tiles);
  L.scr = o; o += up(n * sizeof(float2));
  L.stats = o; o += up(8 * sizeof(int));
  L.tmp = o; o += up(9 * n * sizeof(float));
  L.partials = o; o += up((size_t)nred * 6 * sizeof(double));
  L.sums = o; o += up(8 * sizeof(double));
  L.bad = o; o += up(sizeof(int));
  L.total = o;
  return L;
}

int nred_of(const lbm_params* p) {
  long long n = (long long)p->nx * p->ny;
  long long b = (n + lbm::RB - 1) / lbm::RB;
  return (int)(b < 1024 ? b : 1024);
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

#define LBM_TRY(call)                     \
  do {                                    \
    int _r = (call);                      \
    if (_r != LBM_OK) return _r;          \
  } while (0)
#define LBM_CUDA(call) LBM_TRY(cuda_err(call))

int layout_now(const lbm_ctx* c) { return c->parity; }

}  // namespace

extern "C" {

const char* lbm_error_string(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NONFINITE: return "non-finite value in the state";
    case LBM_ERR_NOT_CONVERGED: return "inner enthalpy iteration hit its cap";
    case LBM_ERR_OOM: return "out of device memory or workspace too small";
    case LBM_ERR_NO_DEVICE: return "no usable CUDA device";
    case LBM_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    default: return "unknown error";
  }
}

int lbm_workspace_bytes(const lbm_params* p, size_t* bytes) {
  if (!bytes) return LBM_ERR_INVALID_ARG;
  LBM_TRY(check_params(p));
  *bytes = layout_of(p, nred_of(p)).total;
  return LBM_OK;
}

int lbm_create(const lbm_params* pin, void* stream, void* workspace, size_t workspace_bytes,
               lbm_ctx** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  LBM_TRY(check_params(pin));
  lbm_params p = *pin;
  double der[8];
  LBM_TRY(derive(&p, der));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return LBM_ERR_NO_DEVICE;
  }
  const int nred = nred_of(&p);
  const Layout L = layout_of(&p, nred);
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->p = p;
  memcpy(c->derived, der, sizeof der);
  c->stream = (cudaStream_t)stream;
  c->nred = nred;
  if (workspace) {
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 255)) {
      delete c;
      return workspace_bytes < L.total ? LBM_ERR_OOM : LBM_ERR_INVALID_ARG;
    }
    c->ws = workspace;
    c->own_ws = false;
  } else {
    if (cudaMalloc(&c->ws, L.total) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return LBM_ERR_OOM;
    }
    c->own_ws = true;
  }
  c->ws_bytes = L.total;
  char* b = (char*)c->ws;
  Dev& d = c->d;
  memset(&d, 0, sizeof d);
  d.nx = p.nx;
  d.ny = p.ny;
  d.n = (long long)p.nx * p.ny;
  d.per_x = p.bc[0] == LBM_BC_PERIODIC;
  d.per_y = p.bc[2] == LBM_BC_PERIODIC;
  d.wall_l = !d.per_x;
  d.wall_r = !d.per_x;
  d.wall_b = !d.per_y;
  d.wall_t = !d.per_y;
  for (int k = 0; k < 4; ++k) {
    d.bc[k] = p.bc[k];
    d.Tbc[k] = (float)p.T_bc[k];
  }
  d.flow = p.flow ? 1 : 0;
  d.rho0 = (float)p.rho0;
  d.inv_rho0 = (float)(1.0 / p.rho0);
  d.nu_l = (float)der[3];
  d.g_beta = (float)der[5];
  d.T_ref = (float)p.T_ref;
  d.s_e = (float)p.s_e;
  d.s_eps = (float)p.s_eps;
  d.s_q = (float)p.s_q;
  d.s_nu = p.flow ? (float)(1.0 / der[0]) : 0.f;
  d.z_a = (float)(1.0 / der[1]);
  d.alpha_var = (p.alpha_ratio > 0 && p.alpha_ratio != 1.0) ? 1 : 0;
  d.tauT_l = (float)der[1];
  d.inv_aratio = d.alpha_var ? (float)(1.0 / p.alpha_ratio) : 1.f;
  d.sigma_var = (p.sigma_solid > 0 && p.sigma_solid != p.sigma) ? 1 : 0;
  d.flow_walls = (p.flow && p.flow_walls) ? 1 : 0;   // walls carry flow only with a flow lattice
  d.flow_front = (p.flow && p.flow_front) ? 1 : 0;
  d.sigma_s = d.sigma_var ? (float)p.sigma_solid : (float)p.sigma;
  d.z_e = (float)p.zeta_e;
  d.z_nu = (float)p.zeta_nu;
  d.varpi = (float)p.varpi;
  d.csT2 = (float)der[6];
  d.sigma = (float)p.sigma;
  d.conv = p.flow ? (float)(1.0 / (p.sigma * der[6])) : 0.f;
  d.wt0 = (float)((1 - p.varpi) / 5.0);
  d.wt1 = (float)((4 + p.varpi) / 20.0);
  d.lat = (float)der[7];
  d.T_s = (float)p.T_s;
  d.T_l = (float)p.T_l;
  d.dTt = (float)(p.T_l - p.T_s);
  d.f_act = (float)p.f_act;
  {
    double scale = fabs(p.T_s) > fabs(p.T_l) ? fabs(p.T_s) : fabs(p.T_l);
    if (p.dT > scale) scale = p.dT;
    if (scale < 1.0) scale = 1.0;
    d.scr_T = (float)(p.screen_tol > 0 ? p.screen_tol : 1e-7 * scale);
    d.scr_f = 1e-7f;
    d.screen_off = p.screen_tol < 0 ? 1 : 0;
  }
  d.H_over_dT = (float)(p.H / p.dT);
  d.etx = (p.nx + lbm::TE - 1) / lbm::TE;
  d.ety = (p.ny + lbm::TE - 1) / lbm::TE;
  d.ntiles = d.etx * d.ety;
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 1;
    // the solve and the commit walk the step's tile list with up to two CTAs
    // per SM (CTAs without a tile exit at once); inside a batch the grids are
    // capped (lbm_batch_create), so that idle CTAs do not take slots from the
    // lattices beside them
    d.egrid = d.ntiles < 2 * sms ? d.ntiles : 2 * sms;
    d.cgrid = d.ntiles < 2 * sms ? d.ntiles : 2 * sms;
    lbm::enthalpy_setup();
  }
  d.max_inner = p.max_inner_iters;
  d.tol = (float)(p.inner_tol > 1e-6 ? p.inner_tol : 1e-6);
  d.f = b + L.f;
  d.g = b + L.g;
  d.storage = p.storage;
  // reference of the stored g deviations: the melting temperature (the middle
  // of the mushy band), where the phase change needs the finest resolution of
  // T; 0 for FP32 storage
  d.g_ref = p.storage != LBM_STORAGE_FP32 ? (float)(0.5 * (p.T_s + p.T_l)) : 0.f;
  d.fl = (float*)(b + L.fl);
  d.phi = (const float*)(b + L.phi);
  d.K = (const float*)(b + L.K);
  d.wallTl = (const float*)(b + L.wallTl);
  d.flags = (int*)(b + L.flags);
  d.list = (int*)(b + L.list);
  d.lcount = (int*)(b + L.lcount);
  d.ctr = (int*)(b + L.ctr);
  d.nearmap = (int*)(b + L.nearmap);
  d.proc = (int*)(b + L.proc);
  d.tact = (unsigned char*)(b + L.tact);
  d.tskip = 0;
  d.scr = (float2*)(b + L.scr);
  d.stats = (int*)(b + L.stats);
  c->tmp = (float*)(b + L.tmp);
  c->partials = (double*)(b + L.partials);
  c->sums = (double*)(b + L.sums);
  c->bad = (int*)(b + L.bad);
  c->tma_ok = lbm::tma_setup(d, &c->maps);
  c->use_tma = p.kernel_variant != 1 && c->tma_ok;
  c->tpc = lbm::TMA_TPC;
  if (cudaMemsetAsync(c->ws, 0, L.total, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int q = 0; q < 2; ++q)
    for (int k = 0; k <= GRAPH_MAX; ++k)
      if (c->gx[q][k]) cudaGraphExecDestroy(c->gx[q][k]);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->trace_buf) cudaFree(c->trace_buf);
  delete c;
}

int lbm_derived(const lbm_ctx* c, double out[8]) {
  if (!c || !out) return LBM_ERR_INVALID_ARG;
  memcpy(out, c->derived, sizeof c->derived);
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }

// empty work lists and tile flags; tile status words keep old stamps, which
// never equal a later step's stamp
static int reset_lists(lbm_ctx* c) {
  const Dev& d = c->d;
  LBM_CUDA(cudaMemsetAsync(d.flags, 0, 2 * sizeof(int) * d.ntiles, c->stream));
  LBM_CUDA(cudaMemsetAsync(d.lcount, 0, 2 * sizeof(int), c->stream));
  LBM_CUDA(cudaMemsetAsync(d.stats + 5, 0, sizeof(int), c->stream));
  lbm::launch_tile_activity(d, c->stream);   // f_l was just loaded
  c->since_check = 0;
  return cuda_err(cudaGetLastError());
}

static int copy_in(lbm_ctx* c, float* dst, const float* src, size_t count, int device_ptrs) {
  return cuda_err(cudaMemcpyAsync(dst, src, count * sizeof(float),
                                  device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream));
}

int lbm_set_fields(lbm_ctx* c, const float* phi, const float* K, const float* T0,
                   const float* fl0, const float* wall_T_left, int device_ptrs) {
  if (!c || !phi || !K || !T0 || !fl0) return LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)c->d.n;
  Dev& d = c->d;
  // Inputs are validated on the device before anything of the context changes:
  // host arrays are first staged in the scratch buffer (one pinned-to-device
  // copy each), device arrays are read where they are.
  const float* src[4] = {phi, K, T0, fl0};
  if (!device_ptrs) {
    for (int k = 0; k < 4; ++k) {
      LBM_CUDA(cudaMemcpyAsync(c->tmp + k * n, src[k], n * sizeof(float), cudaMemcpyHostToDevice,
                               c->stream));
      src[k] = c->tmp + k * n;
    }
    if (wall_T_left)
      for (int y = 0; y < c->p.ny; ++y)
        if (!isfinite(wall_T_left[y])) return LBM_ERR_INVALID_ARG;
  }
  LBM_CUDA(cudaMemsetAsync(c->bad, 0, sizeof(int), c->stream));
  lbm::launch_validate(d, src[0], src[1], src[2], src[3], c->bad, c->stream);
  int bad = 0;
  LBM_CUDA(cudaMemcpyAsync(&bad, c->bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  if (bad) return LBM_ERR_INVALID_ARG;
  LBM_CUDA(cudaMemcpyAsync((float*)d.phi, src[0], n * sizeof(float), cudaMemcpyDeviceToDevice,
                           c->stream));
  LBM_CUDA(cudaMemcpyAsync((float*)d.K, src[1], n * sizeof(float), cudaMemcpyDeviceToDevice,
                           c->stream));
  LBM_CUDA(cudaMemcpyAsync(d.fl, src[3], n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  if (wall_T_left) {
    LBM_TRY(copy_in(c, (float*)d.wallTl, wall_T_left, (size_t)c->p.ny, device_ptrs));
  } else {
    std::vector<float> w((size_t)c->p.ny, (float)c->p.T_bc[LBM_SIDE_LEFT]);
    LBM_CUDA(cudaMemcpyAsync((float*)d.wallTl, w.data(), w.size() * sizeof(float),
                             cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
  }
  lbm::launch_init(d, src[2], c->stream);
  LBM_CUDA(cudaGetLastError());
  LBM_TRY(reset_lists(c));
  c->steps = 0;
  c->parity = 0;
  if (!device_ptrs) LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

// Streams and events the graph captures use (created on first need).
static bool capture_streams(lbm_ctx* c) {
  // the front kernels (main capture stream) outrank the far-tile fused pass
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (!c->cap && cudaStreamCreateWithPriority(&c->cap, cudaStreamNonBlocking, hi) != cudaSuccess) {
    cudaGetLastError();
    c->cap = nullptr;
    return false;
  }
  if (!c->cap2 && cudaStreamCreateWithPriority(&c->cap2, cudaStreamNonBlocking, lo) != cudaSuccess) {
    cudaGetLastError();
    c->cap2 = nullptr;
    return false;
  }
  if ((!c->ev_fork && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) ||
      (!c->ev_join && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Record `steps` steps starting at parity `start` on c->cap, which is being
// captured (alone, or as one branch of a batch capture); returns the number of
// kernels.  The fused pass of step k+1 is split: its tiles more than one tile
// away from step k's listed tiles run on a second stream concurrently with step
// k's enthalpy solve and commit (which touch only nodes within eight nodes of a
// listed tile); the tiles near the front run after the commit.  Everything
// forked onto the second stream joins back before the last kernel.
// Work an adjoint's forward run adds after every step (all optional): f_l
// into fl_base + fl_ctr[0] n, the whole state into st_base + st_ctr[0] 15 n
// (each counter then advances, so a graph serves every replay), and the
// left-wall Nusselt number added to nu_acc[0].
struct Hooks {
  float* fl_base = nullptr;
  unsigned* fl_ctr = nullptr;
  float* st_base = nullptr;
  unsigned* st_ctr = nullptr;
  double* nu_acc = nullptr;
  bool any() const { return fl_base || st_base || nu_acc; }
};

static int launch_hooks(lbm_ctx* c, const Hooks* h, int layout, cudaStream_t s) {
  if (!h) return 0;
  int nl = 0;
  if (h->fl_base) {
    lbm::adj_save(c->d, h->fl_base, h->fl_ctr, s);   // f_l after the step
    ++nl;
  }
  if (h->st_base) {
    lbm::launch_keep_state(c->d, layout, h->st_base, h->st_ctr, s);   // the state after it
    ++nl;
  }
  if (h->nu_acc) {
    lbm::launch_wall_nusselt(c->d, layout, h->nu_acc, s);   // Nu after the step
    ++nl;
  }
  return nl;
}

static int capture_body(lbm_ctx* c, int steps, int start = 0, const Hooks* hooks = nullptr) {
  int nl = 0;
  for (int k = 0; k < steps; ++k) {
    const int par = (start + k) & 1;
    const int fw = c->d.flow && c->d.flow_walls ? 1 : 0;   // a flow-wall pass before each pass
    if (k == 0) {
      lbm::launch_flow_walls(c->d, par, 0, c->cap);
      lbm::launch_fused(c->d, c->tma(), par, 0, c->cap);
    } else {
      lbm::launch_flow_walls(c->d, par, 2, c->cap);
      lbm::launch_fused(c->d, c->tma(), par, 2, c->cap);       // near tiles, after the last commit
      cudaStreamWaitEvent(c->cap, c->ev_join, 0);    // and the far tiles
    }
    nl += 1 + fw;
    if (k + 1 < steps) {
      cudaEventRecord(c->ev_fork, c->cap);
      cudaStreamWaitEvent(c->cap2, c->ev_fork, 0);
      lbm::launch_flow_walls(c->d, 1 - par, 1, c->cap2);
      nl += fw;
      lbm::launch_fused(c->d, c->tma(), 1 - par, 1, c->cap2);  // next step, far tiles
      cudaEventRecord(c->ev_join, c->cap2);
      nl += 1;
    }
    lbm::launch_enthalpy_solve(c->d, par, c->cap);
    lbm::launch_enthalpy_commit(c->d, par, c->cap);
    nl += 2;
    nl += launch_hooks(c, hooks, 1 - par, c->cap);
  }
  return nl;
}

static cudaGraphExec_t instantiate(cudaGraph_t g) {
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiateWithFlags(&ex, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
    cudaGetLastError();
    ex = nullptr;
  }
  cudaGraphDestroy(g);
  return ex;
}

// A graph of `steps` steps starting at parity `start`, replayed on the
// context stream.
static cudaGraphExec_t capture(lbm_ctx* c, int steps, int start, int* launches) {
  if (!capture_streams(c)) return nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const int nl = capture_body(c, steps, start);
  if (cudaStreamEndCapture(c->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return nullptr;
  }
  *launches = nl;
  return instantiate(g);
}

// Forget the captured graphs (after a change of kernel configuration).
static void drop_graphs(lbm_ctx* c) {
  for (int q = 0; q < 2; ++q)
    for (int k = 0; k <= GRAPH_MAX; ++k) {
      if (c->gx[q][k]) cudaGraphExecDestroy(c->gx[q][k]);
      c->gx[q][k] = nullptr;
    }
}

// The graph of `len` (2..GRAPH_MAX) steps from parity `par`, captured on first
// use; nullptr if capture fails (the caller then steps kernel by kernel).
static cudaGraphExec_t graph_for(lbm_ctx* c, int par, int len) {
  if (!c->gx[par][len]) c->gx[par][len] = capture(c, len, par, &c->gnl[par][len]);
  return c->gx[par][len];
}

// Length of the next chunk lbm_step runs from `left` steps: at most GRAPH_MAX,
// and ending where the next NaN/Inf sentinel is due.
static int chunk_len(const lbm_ctx* c, int64_t left, int64_t since_check) {
  int64_t len = left < GRAPH_MAX ? left : GRAPH_MAX;
  if (c->p.check_every > 0) {
    const int64_t due = c->p.check_every - since_check;
    if (due < len) len = due;
  }
  return (int)(len < 1 ? 1 : len);
}

static const int EV_PER_STEP = 5;

static int step_direct(lbm_ctx* c) {
  cudaEvent_t e[EV_PER_STEP] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  if (c->timing) {
    for (int k = 0; k < EV_PER_STEP; ++k) {
      if (cudaEventCreate(&e[k]) != cudaSuccess) return LBM_ERR_CUDA;
      c->ev.push_back(e[k]);
    }
    cudaEventRecord(e[0], c->stream);
  }
  lbm::launch_flow_walls(c->d, c->parity, 0, c->stream);
  lbm::launch_fused(c->d, c->tma(), c->parity, 0, c->stream);
  if (c->timing) {
    cudaEventRecord(e[1], c->stream);
    cudaEventRecord(e[2], c->stream);   // (no separate prep kernel: slot kept at zero)
  }
  lbm::launch_enthalpy_solve(c->d, c->parity, c->stream);
  if (c->timing) cudaEventRecord(e[3], c->stream);
  lbm::launch_enthalpy_commit(c->d, c->parity, c->stream);
  if (c->timing) cudaEventRecord(e[4], c->stream);
  c->parity ^= 1;
  c->steps++;
  c->launches += 3 + (c->d.flow && c->d.flow_walls ? 1 : 0);
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
  // timed runs launch kernel by kernel so events can bracket each kernel
  const bool graphs = !c->timing && !c->graphs_off;
  while (nsteps > 0) {
    const int len = chunk_len(c, nsteps, c->since_check);
    cudaGraphExec_t g = (graphs && len >= 2) ? graph_for(c, c->parity, len) : nullptr;
    if (g) {
      LBM_CUDA(cudaGraphLaunch(g, c->stream));
      c->launches += c->gnl[c->parity][len];
      c->steps += len;
      c->parity ^= len & 1;
    } else {
      for (int k = 0; k < len; ++k) LBM_TRY(step_direct(c));
    }
    nsteps -= len;
    c->since_check += len;
    if (c->p.check_every > 0 && c->since_check >= c->p.check_every) {
      lbm::launch_nonfinite(c->d, c->nred, c->stream);
      c->launches += 1;
      c->since_check = 0;
    }
  }
  return cuda_err(cudaGetLastError());
}

int lbm_prepare(lbm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return LBM_ERR_INVALID_ARG;
  if (c->timing || c->graphs_off) return LBM_OK;
  int par = c->parity;
  int64_t since = c->since_check;
  while (nsteps > 0) {
    const int len = chunk_len(c, nsteps, since);
    if (len >= 2 && !graph_for(c, par, len)) return LBM_ERR_CUDA;
    par ^= len & 1;
    nsteps -= len;
    since += len;
    if (c->p.check_every > 0 && since >= c->p.check_every) since = 0;
  }
  return LBM_OK;
}

int lbm_check_wait(lbm_ctx* c, int64_t limit_ns) {
  if (!c || limit_ns < 1000 || limit_ns > 1000000000LL) return LBM_ERR_INVALID_ARG;
  lbm::launch_wait_probe(c->d, (long long)limit_ns, c->stream);
  return cuda_err(cudaGetLastError());
}

int64_t lbm_kernel_launches(const lbm_ctx* c) { return c ? c->launches : -1; }

int lbm_kernel_variant(const lbm_ctx* c) { return c ? (c->use_tma ? 2 : 1) : -1; }

int lbm_autotune(lbm_ctx* c, int trial_steps, int32_t* variant, int32_t* tiles_per_cta) {
  if (!c || trial_steps < 2 || (trial_steps & 1) || c->timing) return LBM_ERR_INVALID_ARG;
  struct Cand {
    bool tma;
    int tpc;
  };
  std::vector<Cand> cands{{false, 0}};
  if (c->tma_ok)
    for (int t : {2, 3, 4, 5, 6, 8}) cands.push_back({true, t});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return LBM_ERR_CUDA;
  }
  float best = 0.f;
  Cand pick = {c->use_tma, c->tpc};
  int rc = LBM_OK;
  for (const Cand& k : cands) {
    c->use_tma = k.tma;
    if (k.tma) {
      c->tpc = k.tpc;
      c->d.tgrid = lbm::tma_grid(c->d, k.tpc);
    }
    drop_graphs(c);
    // an even step count, then the trial twice: the first captures the graphs
    // (host work that would idle the GPU inside the timed region), the second is timed
    if (c->parity && (rc = lbm_step(c, 1)) != LBM_OK) break;
    if ((rc = lbm_step(c, trial_steps)) != LBM_OK) break;
    cudaEventRecord(e0, c->stream);
    if ((rc = lbm_step(c, trial_steps)) != LBM_OK) break;
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = LBM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (&k == &cands[0] || ms < best) {
      best = ms;
      pick = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->use_tma = pick.tma;
  if (pick.tma) {
    c->tpc = pick.tpc;
    c->d.tgrid = lbm::tma_grid(c->d, pick.tpc);
  }
  drop_graphs(c);
  if (rc != LBM_OK) return rc;
  if (variant) *variant = c->use_tma ? 2 : 1;
  if (tiles_per_cta) *tiles_per_cta = c->use_tma ? c->tpc : 0;
  return cuda_err(cudaGetLastError());
}

// ---- batches -------------------------------------------------------------------

struct lbm_batch {
  std::vector<lbm_ctx*> ctx;
  cudaStream_t stream;             // where lbm_batch_step launches
  cudaStream_t cap;                // capture origin of the batch graph
  std::vector<cudaEvent_t> ev_in, ev_out;   // per context: fork into / join out of the batch
  cudaEvent_t ev_done;
  cudaGraphExec_t graph;
  std::vector<int> nl;             // kernels per context in one graph replay
  std::vector<int> egrid, cgrid;   // the contexts' own enthalpy grids, restored at destroy
  // Batched launches: when every context runs the TMA-staged FP32 kernel with
  // the same flow setting, each pass of a step is one launch over all of them
  // (plans for the stream-collide, solve and commit passes; the contexts'
  // tensor maps in device memory).
  // The contexts are split into groups of about equal node counts, each group
  // a branch of the graph, so that one group's enthalpy kernels (latency
  // bound) run beside another's stream-collide pass (bandwidth bound).
  bool fused = false;
  struct Group {
    std::vector<int> members;                             // context indices
    lbm::BatchPlan* plan[3] = {nullptr, nullptr, nullptr};  // stream-collide, solve, commit
    int maps0 = 0;                                        // first entry in dmaps
  };
  std::vector<Group> groups;
  lbm::TmaMaps* dmaps = nullptr;
};

static void batch_free_plans(lbm_batch* b) {
  for (auto& g : b->groups)
    for (auto& p : g.plan) {
      delete p;
      p = nullptr;
    }
  b->groups.clear();
  if (b->dmaps) cudaFree(b->dmaps);
  b->dmaps = nullptr;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free_plans(b);
  for (size_t i = 0; i < b->egrid.size(); ++i) {
    lbm_ctx* c = b->ctx[i];
    c->d.egrid = b->egrid[i];
    c->d.cgrid = b->cgrid[i];
    drop_graphs(c);
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaEvent_t e : b->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_out) cudaEventDestroy(e);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

int lbm_batch_create(lbm_ctx* const* ctxs, int count, void* stream, lbm_batch** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || count < 1) return LBM_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return LBM_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return LBM_ERR_INVALID_ARG;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->ctx.assign(ctxs, ctxs + count);
  // a small lattice lists few tiles: beside the others of the batch its
  // enthalpy kernels get at most an eighth of its tiles (at least 32) in CTAs
  for (lbm_ctx* c : b->ctx) {
    b->egrid.push_back(c->d.egrid);
    b->cgrid.push_back(c->d.cgrid);
    const int cap = c->d.ntiles / 8 > 32 ? c->d.ntiles / 8 : 32;
    if (c->d.egrid > cap) c->d.egrid = cap;
    if (c->d.cgrid > cap) c->d.cgrid = cap;
    drop_graphs(c);
  }
  b->stream = (cudaStream_t)stream;
  b->cap = nullptr;
  b->ev_done = nullptr;
  b->graph = nullptr;
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < count; ++i) {
    cudaEvent_t a = nullptr, z = nullptr;
    ok = cudaEventCreateWithFlags(&a, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&z, cudaEventDisableTiming) == cudaSuccess;
    if (a) b->ev_in.push_back(a);
    if (z) b->ev_out.push_back(z);
    ok = ok && capture_streams(ctxs[i]);
  }
  if (!ok) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return LBM_ERR_CUDA;
  }
  // one launch per pass for the whole batch where the contexts allow it
  bool fast = count <= lbm::BATCH_MAX;
  for (lbm_ctx* c : b->ctx)
    fast = fast && c->use_tma && c->p.storage == LBM_STORAGE_FP32 &&
           c->d.flow == b->ctx[0]->d.flow && !c->d.flow_walls && !c->d.flow_front;
  b->fused = fast;
  *out = b;
  return LBM_OK;
}

// The plans of the batched launches, from the contexts' current parameters
// (taken by value into the graph, as a single context's capture does).
static constexpr int BATCH_GROUPS = 4;

static int batch_plans(lbm_batch* b) {
  batch_free_plans(b);
  const int n = (int)b->ctx.size();
  // Stream-collide: a context's own grid spreads its tiles over every SM (one
  // or two tiles per CTA for a small lattice, too few to keep its ring of bulk
  // copies busy).  In a batch the lattices share the GPU: about two waves of
  // CTAs in all, each taking the same number of tiles.
  long long tiles = 0;
  std::vector<long long> nt(n);
  for (int i = 0; i < n; ++i) {
    const lbm::Dev& d = b->ctx[i]->d;
    nt[i] = (long long)((d.nx + lbm::TX - 1) / lbm::TX) * ((d.ny + lbm::TY - 1) / lbm::TY);
    tiles += nt[i];
  }
  const long long slots = b->ctx[0]->d.tslots > 0 ? b->ctx[0]->d.tslots : 1;
  long long tpc = (tiles + 2 * slots - 1) / (2 * slots);
  tpc = tpc < 1 ? 1 : tpc > 32 ? 32 : tpc;
  // groups: largest lattices first, each to the group with the fewest nodes
  const int ng = n < BATCH_GROUPS ? n : BATCH_GROUPS;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    return b->ctx[a]->d.n != b->ctx[c]->d.n ? b->ctx[a]->d.n > b->ctx[c]->d.n : a < c;
  });
  b->groups.assign(ng, lbm_batch::Group());
  std::vector<long long> load(ng, 0);
  for (int i : order) {
    int g = 0;
    for (int k = 1; k < ng; ++k)
      if (load[k] < load[g]) g = k;
    b->groups[g].members.push_back(i);
    load[g] += b->ctx[i]->d.n;
  }
  std::vector<lbm::TmaMaps> maps;
  for (auto& G : b->groups) {
    G.maps0 = (int)maps.size();
    for (int k = 0; k < 3; ++k) {
      G.plan[k] = new (std::nothrow) lbm::BatchPlan();
      if (!G.plan[k]) return LBM_ERR_OOM;
      lbm::BatchPlan& P = *G.plan[k];
      P.count = (int)G.members.size();
      P.start[0] = 0;
      for (int j = 0; j < P.count; ++j) {
        const int i = G.members[j];
        const lbm::Dev& d = b->ctx[i]->d;
        P.d[j] = d;
        P.d[j].tskip = 1;   // batch members are mostly solid early on
        const int grid = k == 0 ? (int)((nt[i] + tpc - 1) / tpc) : k == 1 ? d.egrid : d.cgrid;
        P.start[j + 1] = P.start[j] + grid;
      }
    }
    for (int i : G.members) maps.push_back(b->ctx[i]->maps);
  }
  if (cudaMalloc(&b->dmaps, n * sizeof(lbm::TmaMaps)) != cudaSuccess) {
    cudaGetLastError();
    b->dmaps = nullptr;
    return LBM_ERR_OOM;
  }
  LBM_CUDA(cudaMemcpy(b->dmaps, maps.data(), n * sizeof(lbm::TmaMaps), cudaMemcpyHostToDevice));
  return LBM_OK;
}

// LBM_BATCH_STEPS steps of the whole batch: per group, four launches a step on
// the same schedule as one context's capture (the far tiles of step k + 1 on
// the group's second stream beside the enthalpy kernels of step k), each
// launch over every context of the group; the groups are branches forked from
// the capture's start and joined at its end.
static int batch_capture_fused(lbm_batch* b) {
  LBM_TRY(batch_plans(b));
  lbm::batch_setup();
  const bool flow = b->ctx[0]->d.flow != 0;
  cudaGraph_t gr = nullptr;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  cudaEventRecord(b->ev_done, b->cap);
  int nl = 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const auto& G = b->groups[gi];
    lbm_ctx* c0 = b->ctx[G.members[0]];
    const lbm::BatchPlan &PF = *G.plan[0], &PS = *G.plan[1], &PC = *G.plan[2];
    const lbm::TmaMaps* maps = b->dmaps + G.maps0;
    cudaStreamWaitEvent(c0->cap, b->ev_done, 0);
    for (int k = 0; k < LBM_BATCH_STEPS; ++k) {
      const int par = k & 1;
      if (k == 0) {
        lbm::launch_fused_batch(PF, maps, par, 0, flow, c0->cap);
      } else {
        lbm::launch_fused_batch(PF, maps, par, 2, flow, c0->cap);
        cudaStreamWaitEvent(c0->cap, c0->ev_join, 0);
      }
      if (k + 1 < LBM_BATCH_STEPS) {
        cudaEventRecord(c0->ev_fork, c0->cap);
        cudaStreamWaitEvent(c0->cap2, c0->ev_fork, 0);
        lbm::launch_fused_batch(PF, maps, 1 - par, 1, flow, c0->cap2);
        cudaEventRecord(c0->ev_join, c0->cap2);
        ++nl;
      }
      lbm::launch_enthalpy_solve_batch(PS, par, c0->cap);
      lbm::launch_enthalpy_commit_batch(PC, par, c0->cap);
      nl += 3;
    }
    cudaEventRecord(b->ev_out[gi], c0->cap);
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi) cudaStreamWaitEvent(b->cap, b->ev_out[gi], 0);
  if (cudaStreamEndCapture(b->cap, &gr) != cudaSuccess || !gr) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  b->graph = instantiate(gr);
  // the launches are shared: each group's first context is charged its group's
  b->nl.assign(b->ctx.size(), 0);
  for (const auto& G : b->groups) b->nl[G.members[0]] = nl / (int)b->groups.size();
  return b->graph ? LBM_OK : LBM_ERR_CUDA;
}

// one graph: LBM_BATCH_STEPS steps of every context, one branch per context
static int batch_capture(lbm_batch* b) {
  if (b->fused) return batch_capture_fused(b);
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  b->nl.assign(b->ctx.size(), 0);
  // every branch forks from the start of the capture and joins at its end (a
  // fork recorded after an earlier branch's join would chain the branches)
  cudaEventRecord(b->ev_done, b->cap);
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    lbm_ctx* c = b->ctx[i];
    cudaStreamWaitEvent(c->cap, b->ev_done, 0);
    b->nl[i] = capture_body(c, LBM_BATCH_STEPS, 0);
    cudaEventRecord(b->ev_out[i], c->cap);
  }
  for (size_t i = 0; i < b->ctx.size(); ++i) cudaStreamWaitEvent(b->cap, b->ev_out[i], 0);
  if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  b->graph = instantiate(g);
  return b->graph ? LBM_OK : LBM_ERR_CUDA;
}

int lbm_batch_mode(const lbm_batch* b) {
  if (!b) return LBM_ERR_INVALID_ARG;
  return b->fused ? 1 : 0;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
  if (!b || nsteps < 0) return LBM_ERR_INVALID_ARG;
  const int par = b->ctx[0]->parity;
  for (lbm_ctx* c : b->ctx)
    if (c->timing || c->parity != par) return LBM_ERR_INVALID_ARG;
  // get every context to an even step count first
  if (par && nsteps > 0) {
    for (lbm_ctx* c : b->ctx) LBM_TRY(lbm_step(c, 1));
    --nsteps;
  }
  const int64_t reps = nsteps / LBM_BATCH_STEPS;
  if (reps > 0) {
    if (!b->graph) LBM_TRY(batch_capture(b));
    // the batch runs after what is queued on every context stream ...
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      LBM_CUDA(cudaEventRecord(b->ev_in[i], b->ctx[i]->stream));
      LBM_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in[i], 0));
    }
    for (int64_t r = 0; r < reps; ++r) LBM_CUDA(cudaGraphLaunch(b->graph, b->stream));
    // ... and before what is queued there next
    LBM_CUDA(cudaEventRecord(b->ev_done, b->stream));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      lbm_ctx* c = b->ctx[i];
      LBM_CUDA(cudaStreamWaitEvent(c->stream, b->ev_done, 0));
      c->steps += reps * LBM_BATCH_STEPS;
      c->launches += reps * b->nl[i];
    }
  }
  const int64_t rest = nsteps - reps * LBM_BATCH_STEPS;
  if (rest > 0)
    for (lbm_ctx* c : b->ctx) LBM_TRY(lbm_step(c, rest));
  return cuda_err(cudaGetLastError());
}

int lbm_status(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID_ARG;
  int st[8];
  LBM_CUDA(cudaMemcpyAsync(st, c->d.stats, sizeof st, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  if (st[5]) return LBM_ERR_NONFINITE;   // kept until new fields or a new state are loaded
  if (st[4]) {
    LBM_CUDA(cudaMemsetAsync(c->d.stats + 4, 0, sizeof(int), c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return LBM_ERR_TIMEOUT;
  }
  if (st[0]) {
    LBM_CUDA(cudaMemsetAsync(c->d.stats, 0, sizeof(int), c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return LBM_ERR_NOT_CONVERGED;
  }
  return LBM_OK;
}

int lbm_get_macros(lbm_ctx* c, float* ux, float* uy, float* rho, float* T, float* fl,
                   int device_ptrs) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)c->d.n;
  float* outs[5] = {ux, uy, rho, T, fl};
  float* dst[5];
  for (int k = 0; k < 5; ++k)
    dst[k] = outs[k] ? (device_ptrs ? outs[k] : c->tmp + k * n) : nullptr;
  lbm::launch_macros(c->d, layout_now(c), dst[0], dst[1], dst[2], dst[3], dst[4], c->stream);
  LBM_CUDA(cudaGetLastError());
  if (!device_ptrs) {
    for (int k = 0; k < 5; ++k)
      if (outs[k])
        LBM_CUDA(cudaMemcpyAsync(outs[k], dst[k], n * sizeof(float), cudaMemcpyDeviceToHost,
                                 c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_reduce(lbm_ctx* c, double out[4]) {
  if (!c || !out) return LBM_ERR_INVALID_ARG;
  lbm::launch_reduce(c->d, layout_now(c), c->partials, c->sums, c->nred, c->stream);
  LBM_CUDA(cudaGetLastError());
  double s[4];
  LBM_CUDA(cudaMemcpyAsync(s, c->sums, sizeof s, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(out, s, sizeof s);
  for (int k = 0; k < 4; ++k)
    if (!isfinite(s[k])) return LBM_ERR_NONFINITE;
  return LBM_OK;
}

int lbm_get_state(lbm_ctx* c, float* f, float* g, float* fl, int device_ptrs) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)c->d.n;
  float* df = f ? (device_ptrs ? f : c->tmp) : nullptr;
  float* dg = g ? (device_ptrs ? g : c->tmp) : nullptr;
  if (f) {
    lbm::launch_get_state(c->d, layout_now(c), df, nullptr, c->stream);
    LBM_CUDA(cudaGetLastError());
    if (!device_ptrs) {
      LBM_CUDA(cudaMemcpyAsync(f, df, 9 * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      LBM_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  if (g) {
    lbm::launch_get_state(c->d, layout_now(c), nullptr, dg, c->stream);
    LBM_CUDA(cudaGetLastError());
    if (!device_ptrs) {
      LBM_CUDA(cudaMemcpyAsync(g, dg, 5 * n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      LBM_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  if (fl) {
    LBM_CUDA(cudaMemcpyAsync(fl, c->d.fl, n * sizeof(float),
                             device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    if (!device_ptrs) LBM_CUDA(cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_set_state(lbm_ctx* c, const float* f, const float* g, const float* fl, int device_ptrs) {
  if (!c) return LBM_ERR_INVALID_ARG;
  const size_t n = (size_t)c->d.n;
  const float* sf = f;
  const float* sg = g;
  if (f && !device_ptrs) {
    LBM_CUDA(cudaMemcpyAsync(c->tmp, f, 9 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    sf = c->tmp;
  }
  if (f) {
    lbm::launch_set_state(c->d, sf, nullptr, c->stream);
    LBM_CUDA(cudaGetLastError());
  }
  if (g && !device_ptrs) {
    LBM_CUDA(cudaMemcpyAsync(c->tmp, g, 5 * n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    sg = c->tmp;
  }
  if (g) {
    lbm::launch_set_state(c->d, nullptr, sg, c->stream);
    LBM_CUDA(cudaGetLastError());
  }
  if (fl) LBM_TRY(copy_in(c, c->d.fl, fl, n, device_ptrs));
  LBM_TRY(reset_lists(c));
  c->parity = 0;
  c->steps = 0;
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_trace(lbm_ctx* c, int64_t capacity) {
  if (!c || capacity < 0 || capacity > (1LL << 28)) return LBM_ERR_INVALID_ARG;
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  if (c->trace_buf) cudaFree(c->trace_buf);
  c->trace_buf = nullptr;
  c->d.trace = nullptr;
  c->d.trace_n = nullptr;
  c->d.trace_cap = 0;
  if (capacity > 0) {
    if (cudaMalloc(&c->trace_buf, 256 + (size_t)capacity * 4 * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      c->trace_buf = nullptr;
      return LBM_ERR_OOM;
    }
    LBM_CUDA(cudaMemsetAsync(c->trace_buf, 0, 256, c->stream));
    c->d.trace_n = static_cast<unsigned*>(c->trace_buf);
    c->d.trace = reinterpret_cast<long long*>(static_cast<char*>(c->trace_buf) + 256);
    c->d.trace_cap = (unsigned)capacity;
  }
  drop_graphs(c);   // graphs hold the kernel parameters they were captured with
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_trace_read(lbm_ctx* c, int64_t* records, int64_t max_records, int64_t* count) {
  if (!c || !count || max_records < 0 || (max_records > 0 && !records)) return LBM_ERR_INVALID_ARG;
  *count = 0;
  if (!c->trace_buf) return LBM_OK;
  unsigned n = 0;
  LBM_CUDA(cudaMemcpyAsync(&n, c->d.trace_n, sizeof n, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  int64_t k = n < c->d.trace_cap ? n : c->d.trace_cap;
  if (k > max_records) k = max_records;
  if (k > 0)
    LBM_CUDA(cudaMemcpy(records, c->d.trace, (size_t)k * 4 * sizeof(long long),
                        cudaMemcpyDeviceToHost));
  LBM_CUDA(cudaMemsetAsync(c->d.trace_n, 0, sizeof n, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  *count = k;
  return LBM_OK;
}

int lbm_adjoint_timing(const lbm_ctx* c, double ms[2]) {
  if (!c || !ms) return LBM_ERR_INVALID_ARG;
  ms[0] = c->adj_ms[0];
  ms[1] = c->adj_ms[1];
  return LBM_OK;
}

int lbm_timing(lbm_ctx* c, int enable) {
  if (!c) return LBM_ERR_INVALID_ARG;
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  c->timing = enable != 0;
  static const int zero[2] = {0, 0};
  LBM_CUDA(cudaMemcpyAsync(c->d.stats + 1, zero, 2 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_timing_read(lbm_ctx* c, double ms[4], int64_t* steps_timed, int64_t* tiles_solved,
                    int32_t* max_sweeps) {
  if (!c || !ms) return LBM_ERR_INVALID_ARG;
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  double t[4] = {0, 0, 0, 0};
  for (size_t k = 0; k + EV_PER_STEP - 1 < c->ev.size(); k += EV_PER_STEP) {
    for (int j = 0; j < 4; ++j) {
      float a = 0;
      LBM_CUDA(cudaEventElapsedTime(&a, c->ev[k + j], c->ev[k + j + 1]));
      t[j] += a;
    }
  }
  int st[4];
  LBM_CUDA(cudaMemcpy(st, c->d.stats, sizeof st, cudaMemcpyDeviceToHost));
  memcpy(ms, t, sizeof t);
  if (steps_timed) *steps_timed = (int64_t)(c->ev.size() / EV_PER_STEP);
  if (tiles_solved) *tiles_solved = st[1];
  if (max_sweeps) *max_sweeps = st[2];
  return LBM_OK;
}

}  // extern "C"

// ---- adjoint of the conduction step ------------------------------------------------

namespace {

// CUDA events bracketing the phases of one adjoint call on the context
// stream; their times land in c->adj_ms when it returns
struct PhaseEvents {
  lbm_ctx* c;
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  explicit PhaseEvents(lbm_ctx* ctx) : c(ctx) {
    for (cudaEvent_t& x : e)
      if (cudaEventCreate(&x) != cudaSuccess) {
        cudaGetLastError();
        x = nullptr;
      }
  }
  void mark(int k) {
    if (e[k]) cudaEventRecord(e[k], c->stream);
  }
  ~PhaseEvents() {
    float a = 0.f, b = 0.f;
    if (e[0] && e[1] && e[2] && cudaEventSynchronize(e[2]) == cudaSuccess &&
        cudaEventElapsedTime(&a, e[0], e[1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, e[1], e[2]) == cudaSuccess) {
      c->adj_ms[0] = a;
      c->adj_ms[1] = b;
    }
    cudaGetLastError();
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
};

// device buffers of one adjoint run, freed on scope exit
struct DevMem {
  std::vector<void*> ptrs;
  float* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<float*>(p);
  }
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
};

}  // namespace

// A graph of `steps` steps from parity 0 like capture(), each step followed
// by the hooks.
static cudaGraphExec_t capture_keep(lbm_ctx* c, int steps, const Hooks& h) {
  if (!capture_streams(c)) return nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  capture_body(c, steps, 0, &h);
  if (cudaStreamEndCapture(c->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return nullptr;
  }
  return instantiate(g);
}

// Steps `steps` steps like lbm_step (graphs from parity 0, single steps
// around them), each followed by the hooks; graphs kept in `cache` for later
// calls with the same hooks.
struct HookGraphs {
  cudaGraphExec_t g[2] = {nullptr, nullptr};   // GRAPH_MAX and 2 steps
  ~HookGraphs() {
    for (cudaGraphExec_t x : g)
      if (x) cudaGraphExecDestroy(x);
  }
};

static int step_hooked(lbm_ctx* c, int64_t steps, const Hooks& h, HookGraphs& cache) {
  auto direct = [&]() -> int {
    LBM_TRY(step_direct(c));
    launch_hooks(c, &h, c->parity, c->stream);
    --steps;
    return LBM_OK;
  };
  while (steps > 0 && (c->parity != 0 || c->graphs_off || steps < 2)) LBM_TRY(direct());
  const int lens[2] = {GRAPH_MAX, 2};
  for (int k = 0; k < 2; ++k) {
    if (steps < lens[k]) continue;
    if (!cache.g[k]) cache.g[k] = capture_keep(c, lens[k], h);
    if (!cache.g[k]) break;
    while (steps >= lens[k]) {
      LBM_CUDA(cudaGraphLaunch(cache.g[k], c->stream));
      steps -= lens[k];
      c->steps += lens[k];
    }
  }
  while (steps > 0) LBM_TRY(direct());
  return LBM_OK;
}

int lbm_adjoint_melt(lbm_ctx* c, int64_t nsteps, int32_t checkpoint_every, int32_t mu_sweeps,
                     float* d_phi, float* d_wall_T_left, double* J, int device_ptrs) {
  return lbm_adjoint(c, LBM_OBJ_MELT, nsteps, checkpoint_every, mu_sweeps, d_phi, d_wall_T_left,
                     J, device_ptrs);
}

int lbm_adjoint(lbm_ctx* c, int objective, int64_t nsteps, int32_t checkpoint_every,
                int32_t mu_sweeps, float* d_phi, float* d_wall_T_left, double* J,
                int device_ptrs) {
  if (!c || nsteps < 1 || checkpoint_every < 0 || mu_sweeps < 0 || !d_phi || !d_wall_T_left || !J)
    return LBM_ERR_INVALID_ARG;
  if (objective != LBM_OBJ_MELT && objective != LBM_OBJ_NUSSELT) return LBM_ERR_INVALID_ARG;
  const lbm_params& p = c->p;
  if (p.flow || c->timing || p.storage != LBM_STORAGE_FP32 || c->d.alpha_var || c->d.sigma_var)
    return LBM_ERR_INVALID_ARG;
  if (!c->d.per_y || c->d.per_x || p.bc[0] != LBM_BC_DIRICHLET) return LBM_ERR_INVALID_ARG;
  const bool melt = objective == LBM_OBJ_MELT;
  if (!melt && c->d.nx < 5) return LBM_ERR_INVALID_ARG;   // x = 1, 2 interior
  // Nusselt objective: J = (1/N) sum over the states after steps 1..N of
  // -(-3 T_w + 4 T_1 - T_2)/2 H/dT averaged over the ny rows
  lbm::NuSrc nu{0.f, 0.f, 0.f};
  if (!melt) {
    const double k = (double)c->d.H_over_dT / ((double)c->d.ny * (double)nsteps);
    nu = {(float)(-2.0 * k), (float)(0.5 * k), (float)(1.5 * k)};
  }
  const int sweeps = mu_sweeps > 0 ? mu_sweeps : 64;
  const size_t n = (size_t)c->d.n, st = 6 * n;   // a checkpoint: g (5 planes) and f_l
  if (!lbm::adj_init()) return LBM_ERR_CUDA;
  // Keep f_l of every step when that takes at most half the free memory;
  // otherwise (or when asked for a spacing) keep the whole state every K steps
  // and recompute the steps between.
  size_t free_b = 0, total_b = 0;
  LBM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const bool keep_all =
      checkpoint_every == 0 && (double)(nsteps + 1) * n * sizeof(float) <= 0.5 * (double)free_b;
  const int64_t K = keep_all ? nsteps
                    : checkpoint_every > 0 ? checkpoint_every
                                           : (int64_t)ceil(sqrt((double)nsteps));
  const int64_t ncp = keep_all ? 1 : nsteps / K + 1;
  DevMem mem;
  // f_l per step: all of them (keep_all), else those of one segment (index m:
  // after the segment's m-th step; m = 0: its start)
  float* flS = mem.get((size_t)((keep_all ? nsteps : K) + 1) * n);
  float* cps = keep_all ? nullptr : mem.get((size_t)ncp * st);
  float* fin = keep_all ? nullptr : mem.get(st);
  lbm::AdjBuffers b;
  b.a = mem.get(n);
  b.lamg = mem.get(5 * n);
  b.lamf = mem.get(n);
  b.rhs = mem.get(n);
  b.mu0 = mem.get(n);
  b.mu1 = mem.get(n);
  b.lamgpre = mem.get(5 * n);
  b.lama = mem.get(n);
  b.lamtw = mem.get((size_t)c->d.ny);
  b.pos = reinterpret_cast<int*>(mem.get(n));
  int* lists[2] = {reinterpret_cast<int*>(mem.get(n)), reinterpret_cast<int*>(mem.get(n))};
  int* counts = reinterpret_cast<int*>(mem.get(2));
  unsigned* ctr = reinterpret_cast<unsigned*>(mem.get(2));
  double* nu_acc = reinterpret_cast<double*>(mem.get(2));
  double* dJ = reinterpret_cast<double*>(mem.get(2 * 129));
  if (!flS || (!keep_all && (!cps || !fin)) || !b.a || !b.lamg || !b.lamf || !b.rhs ||
      !b.mu0 || !b.mu1 || !b.lamgpre || !b.lama || !b.lamtw || !b.pos || !lists[0] ||
      !lists[1] || !counts || !ctr || !nu_acc || !dJ)
    return LBM_ERR_OOM;
  // transposed collision matrix with u = 0: g+ = A g,
  // A = N^-1 [(I - Theta) N + Theta e 1^T], e = (1, 0, 0, varpi, 0), Eq. (32)-(37)
  {
    static const double N5[5][5] = {{1, 1, 1, 1, 1}, {0, 1, 0, -1, 0}, {0, 0, 1, 0, -1},
                                    {-4, 1, 1, 1, 1}, {0, 1, -1, 1, -1}};
    const double th[5] = {1.0, c->d.z_a, c->d.z_a, c->d.z_e, c->d.z_nu};
    const double eq[5] = {1.0, 0.0, 0.0, p.varpi, 0.0};
    float* At = b.At;
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        double a = 0.0;
        for (int k = 0; k < 5; ++k) {
          double nk = 0.0;
          for (int m = 0; m < 5; ++m) nk += N5[k][m] * N5[k][m];
          const double ninv = N5[k][i] / nk;   // (N^-1)[i][k]
          a += ninv * ((1.0 - th[k]) * N5[k][j] + th[k] * eq[k]);
        }
        At[j * 5 + i] = (float)a;
      }
  }
  auto save = [&](float* dst) -> int {
    LBM_TRY(lbm_get_state(c, nullptr, dst, dst + 5 * n, 1));
    return LBM_OK;
  };
  auto restore = [&](const float* src) -> int {
    LBM_TRY(lbm_set_state(c, nullptr, src, src + 5 * n, 1));
    return LBM_OK;
  };
  struct Graphs {
    std::vector<cudaGraphExec_t> v;
    ~Graphs() {
      for (cudaGraphExec_t g : v) cudaGraphExecDestroy(g);
    }
  } graphs;
  HookGraphs fwd_graphs;
  const int64_t steps0 = c->steps;
  lbm::adj_seed(c->d, b.lamf, b.lamg, b.a, melt, nu, c->stream);   // a is needed from here on
  PhaseEvents ph(c);
  ph.mark(0);
  LBM_CUDA(cudaMemsetAsync(nu_acc, 0, sizeof(double), c->stream));
  double* const acc = melt ? nullptr : nu_acc;
  if (keep_all) {
    // forward, f_l after every step into flS (its start at index 0)
    LBM_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), c->stream));
    lbm::adj_save(c->d, flS, ctr, c->stream);
    Hooks h;
    h.fl_base = flS;
    h.fl_ctr = ctr;
    h.nu_acc = acc;
    LBM_TRY(step_hooked(c, nsteps, h, fwd_graphs));
  } else {
    // forward, keeping the whole state every K steps
    LBM_TRY(save(cps));
    Hooks h;
    h.nu_acc = acc;
    for (int64_t j = 1; j < ncp; ++j) {
      LBM_TRY(step_hooked(c, K, h, fwd_graphs));
      LBM_TRY(save(cps + (size_t)j * st));
    }
    const int64_t done = (ncp - 1) * K;
    if (nsteps > done) LBM_TRY(step_hooked(c, nsteps - done, h, fwd_graphs));
    LBM_TRY(save(fin));
  }
  const float* fl_end = keep_all ? flS + (size_t)nsteps * n : fin + 5 * n;
  if (melt) lbm::adj_objective(c->d, fl_end, dJ, c->stream);
  ph.mark(1);
  // reverse sweep
  LBM_CUDA(cudaMemsetAsync(b.lama, 0, n * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(b.lamtw, 0, c->d.ny * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(int), c->stream));
  lbm::adj_list(c->d, fl_end, lists[0], counts, c->stream);
  int cur = 0;
  // reversed steps m = hi - 1 .. lo, f_l of step m at F + (m - lo) n
  auto reverse = [&](cudaStream_t sm, const float* F, int64_t lo, int64_t hi) {
    for (int64_t m = hi - 1; m >= lo; --m) {
      const float* f0 = F + (size_t)(m - lo) * n;
      lbm::adj_step(c->d, b, f0, f0 + n, lists[cur], counts + cur, lists[1 - cur],
                    counts + 1 - cur, sweeps, nu, sm);
      std::swap(b.lamg, b.lamgpre);
      cur ^= 1;
    }
  };
  if (keep_all) {
    reverse(c->stream, flS, 0, nsteps);
  } else {
    // One segment after its checkpoint is restored (parity 0): the len steps
    // forward, f_l of each kept, then the len reverse steps; the same
    // launches for every whole segment, so they are captured once per
    // (len, buffer parity) and replayed.
    auto record_segment = [&](cudaStream_t sm, int64_t len) {
      int par = 0;
      for (int64_t m = 1; m <= len; ++m) {
        lbm::launch_fused(c->d, c->tma(), par, 0, sm);
        lbm::launch_enthalpy_solve(c->d, par, sm);
        lbm::launch_enthalpy_commit(c->d, par, sm);
        par ^= 1;
        cudaMemcpyAsync(flS + (size_t)m * n, c->d.fl, n * sizeof(float),
                        cudaMemcpyDeviceToDevice, sm);
      }
      reverse(sm, flS, 0, len);
    };
    struct SegGraph {
      int64_t len;
      float* lamg;
      cudaGraphExec_t ex;
    };
    std::vector<SegGraph> seg_graphs;
    const bool can_capture = capture_streams(c);
    for (int64_t j = ncp - 1; j >= 0; --j) {
      const int64_t first = j * K;
      const int64_t len = (j == ncp - 1) ? nsteps - first : K;
      if (len <= 0) continue;
      LBM_TRY(restore(cps + (size_t)j * st));
      LBM_CUDA(cudaMemcpyAsync(flS, cps + (size_t)j * st + 5 * n, n * sizeof(float),
                               cudaMemcpyDeviceToDevice, c->stream));
      float* const lamg0 = b.lamg;
      float* const lamgpre0 = b.lamgpre;
      const int cur0 = cur;
      cudaGraphExec_t ex = nullptr;
      for (const SegGraph& g : seg_graphs)
        if (g.len == len && g.lamg == lamg0) ex = g.ex;
      if (!ex && can_capture && len == K) {
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          record_segment(c->cap, len);
          if (cudaStreamEndCapture(c->cap, &gr) == cudaSuccess && gr) {
            ex = instantiate(gr);
            if (ex) {
              seg_graphs.push_back({len, lamg0, ex});
              graphs.v.push_back(ex);
            }
          }
        }
        cudaGetLastError();
        b.lamg = lamg0;
        b.lamgpre = lamgpre0;
        cur = cur0;
      }
      if (ex) {
        LBM_CUDA(cudaGraphLaunch(ex, c->stream));
        if (len & 1) {
          std::swap(b.lamg, b.lamgpre);
          cur ^= 1;
        }
      } else {
        record_segment(c->stream, len);
      }
      LBM_CUDA(cudaGetLastError());
    }
    // back to where the forward run ended
    LBM_TRY(restore(fin));
    c->steps = steps0 + nsteps;
  }
  LBM_CUDA(cudaGetLastError());
  ph.mark(2);
  // d J / d phi = (dT / (sigma St)) d J / d a, straight into the caller's arrays
  lbm::adj_scale((long long)n, b.lama, c->d.lat, c->stream);
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  LBM_CUDA(cudaMemcpyAsync(d_phi, b.lama, n * sizeof(float), kind, c->stream));
  LBM_CUDA(cudaMemcpyAsync(d_wall_T_left, b.lamtw, c->d.ny * sizeof(float), kind, c->stream));
  LBM_CUDA(cudaMemcpyAsync(J, melt ? dJ : nu_acc, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  // (the reverse sweep added the Nusselt number's direct term in T_w once per
  // reversed step, for the states 0..N-1 instead of 1..N: the same constant
  // N times)
  if (!melt) *J /= (double)nsteps;
  return LBM_OK;
}

int lbm_adjoint_coupled(lbm_ctx* c, int objective, int64_t nsteps, int32_t checkpoint_every,
                        int32_t mu_sweeps, float* d_phi, float* d_lnK, float* d_wall_T_left,
                        double* J, int device_ptrs) {
  if (!c || nsteps < 1 || checkpoint_every < 0 || mu_sweeps < 0 || !d_phi || !d_lnK ||
      !d_wall_T_left || !J)
    return LBM_ERR_INVALID_ARG;
  if (objective != LBM_OBJ_MELT && objective != LBM_OBJ_NUSSELT) return LBM_ERR_INVALID_ARG;
  const lbm_params& p = c->p;
  const lbm::Dev& d = c->d;
  if (c->timing || p.storage != LBM_STORAGE_FP32 || d.sigma_var || d.flow_walls || d.flow_front)
    return LBM_ERR_INVALID_ARG;
  if (d.per_x || p.bc[0] != LBM_BC_DIRICHLET || d.nx < 5) return LBM_ERR_INVALID_ARG;
  const bool melt = objective == LBM_OBJ_MELT;
  const int sweeps = mu_sweeps > 0 ? mu_sweeps : 64;
  const size_t n = (size_t)d.n, st = 15 * n;   // a kept state: f (9), g (5), f_l
  if (!lbm::adj_init()) return LBM_ERR_CUDA;
  // Every state kept when that takes at most half the free memory (and no
  // spacing is asked for); otherwise the whole state every K steps (K =
  // sqrt(nsteps) by default), each segment recomputed from its checkpoint
  // and reversed from one CUDA graph replay.
  size_t free_b = 0, total_b = 0;
  LBM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const bool keep_all = checkpoint_every == 0 &&
                        (double)(nsteps + 1) * st * sizeof(float) <= 0.5 * (double)free_b;
  const int64_t K = keep_all ? nsteps
                    : checkpoint_every > 0 ? checkpoint_every
                                           : (int64_t)ceil(sqrt((double)nsteps));
  const int64_t ncp = keep_all ? 1 : nsteps / K + 1;
  if (!keep_all && (double)(ncp + 2 * K + 3) * st * sizeof(float) > 0.8 * (double)free_b)
    return LBM_ERR_OOM;
  DevMem mem;
  // states of one segment (index m: after its m-th step; all steps when keep_all)
  float* S = mem.get((size_t)(K + 1) * st);
  float* S2 = keep_all ? nullptr : mem.get((size_t)(K + 1) * st);   // second segment buffer
  float* cps = keep_all ? nullptr : mem.get((size_t)ncp * st);
  float* fin = keep_all ? nullptr : mem.get(st);
  float* lf[2] = {mem.get(9 * n), mem.get(9 * n)};
  float* lg[2] = {mem.get(5 * n), mem.get(5 * n)};
  lbm::AdjBuffers b;
  b.a = mem.get(n);
  b.lamf = mem.get(n);
  b.rhs = mem.get(n);
  b.mu0 = mem.get(n);
  b.mu1 = mem.get(n);
  b.lama = mem.get(n);   // adjoint of phi
  b.lamtw = mem.get((size_t)d.ny);
  b.pos = reinterpret_cast<int*>(mem.get(n));
  float* lK = mem.get(n);
  int* lists[2] = {reinterpret_cast<int*>(mem.get(n)), reinterpret_cast<int*>(mem.get(n))};
  int* counts = reinterpret_cast<int*>(mem.get(2));
  double* nu_acc = reinterpret_cast<double*>(mem.get(2));
  unsigned* ctr = reinterpret_cast<unsigned*>(mem.get(4));   // two counter pairs
  if (!S || (!keep_all && (!cps || !fin || !S2)) || !lf[0] || !lf[1] || !lg[0] || !lg[1] || !b.a ||
      !b.lamf || !b.rhs || !b.mu0 || !b.mu1 || !b.lama || !b.lamtw || !b.pos || !lK ||
      !lists[0] || !lists[1] || !counts || !nu_acc || !ctr)
    return LBM_ERR_OOM;
  // rows of the Nusselt number (lbm_reduce's): all but horizontal wall rows
  const int y0 = d.wall_b ? 1 : 0, y1 = d.wall_t ? d.ny - 1 : d.ny;
  const double kN = melt ? 0.0 : (double)d.H_over_dT / ((double)(y1 - y0) * (double)nsteps);
  const int64_t steps0 = c->steps;
  HookGraphs fwd_graphs;
  Hooks h;
  h.nu_acc = melt ? nullptr : nu_acc;
  PhaseEvents ph(c);
  ph.mark(0);
  LBM_CUDA(cudaMemsetAsync(nu_acc, 0, sizeof(double), c->stream));
  auto save = [&](float* dst) -> int {   // the whole state, natural layout
    lbm::launch_keep_state(c->d, c->parity, dst, nullptr, c->stream);
    return cuda_err(cudaGetLastError());
  };
  if (keep_all) {
    // forward, every state kept (a device counter picks the slot)
    LBM_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), c->stream));
    lbm::launch_keep_state(c->d, c->parity, S, ctr, c->stream);
    h.st_base = S;
    h.st_ctr = ctr;
    LBM_TRY(step_hooked(c, nsteps, h, fwd_graphs));
  } else {
    // forward, the whole state every K steps
    LBM_TRY(save(cps));
    for (int64_t j = 1; j < ncp; ++j) {
      LBM_TRY(step_hooked(c, K, h, fwd_graphs));
      LBM_TRY(save(cps + (size_t)j * st));
    }
    const int64_t done = (ncp - 1) * K;
    if (nsteps > done) LBM_TRY(step_hooked(c, nsteps - done, h, fwd_graphs));
    LBM_TRY(save(fin));
  }
  LBM_CUDA(cudaGetLastError());
  ph.mark(1);
  const float* last = keep_all ? S + (size_t)nsteps * st : fin;
  // objective and seeds (host side: small arrays)
  std::vector<float> hfl(n), seedf(n, 0.f), seedg(5 * n, 0.f);
  LBM_CUDA(cudaMemcpyAsync(hfl.data(), last + 14 * n, n * sizeof(float),
                           cudaMemcpyDeviceToHost, c->stream));
  double accv = 0;
  LBM_CUDA(cudaMemcpyAsync(&accv, nu_acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  auto is_wall = [&](int x, int y) {
    return (d.wall_l && x == 0) || (d.wall_r && x == d.nx - 1) || (d.wall_b && y == 0) ||
           (d.wall_t && y == d.ny - 1);
  };
  size_t cnt = 0;
  double sum = 0;
  for (int y = 0; y < d.ny; ++y)
    for (int x = 0; x < d.nx; ++x)
      if (!is_wall(x, y)) {
        ++cnt;
        sum += hfl[(size_t)y * d.nx + x];
      }
  if (melt) {
    *J = cnt ? sum / (double)cnt : 0.0;
    for (int y = 0; y < d.ny; ++y)
      for (int x = 0; x < d.nx; ++x)
        if (!is_wall(x, y)) seedf[(size_t)y * d.nx + x] = (float)(1.0 / (double)cnt);
  } else {
    *J = accv / (double)nsteps;
    for (int y = y0; y < y1; ++y)
      for (int i = 0; i < 5; ++i) {
        seedg[i * n + (size_t)y * d.nx + 1] = (float)(-2.0 * kN);
        seedg[i * n + (size_t)y * d.nx + 2] = (float)(0.5 * kN);
      }
  }
  LBM_CUDA(cudaMemcpyAsync(b.lamf, seedf.data(), n * sizeof(float), cudaMemcpyHostToDevice,
                           c->stream));
  LBM_CUDA(cudaMemcpyAsync(lg[0], seedg.data(), 5 * n * sizeof(float), cudaMemcpyHostToDevice,
                           c->stream));
  LBM_CUDA(cudaMemsetAsync(lf[0], 0, 9 * n * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(b.lama, 0, n * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(lK, 0, n * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(b.lamtw, 0, d.ny * sizeof(float), c->stream));
  LBM_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(int), c->stream));
  lbm::adj_a(c->d, b.a, c->stream);
  lbm::adj_list(c->d, last + 14 * n, lists[0], counts, c->stream);
  // the step's parameters
  lbm::CoupledStep<float> A;
  A.geo = lbm::CoupledGeo{d.nx, d.ny, d.per_x, d.per_y, {d.bc[0], d.bc[1], d.bc[2], d.bc[3]}};
  A.n = (long long)n;
  A.fp.rho0 = d.rho0;
  A.fp.nu_l = d.nu_l;
  A.fp.g_beta = d.g_beta;
  A.fp.T_ref = d.T_ref;
  const float lam[9] = {1.f, d.s_e, d.s_eps, 1.f, d.s_q, 1.f, d.s_q, d.s_nu, d.s_nu};
  for (int k = 0; k < 9; ++k) A.fp.lam[k] = lam[k];
  A.fp.eps = 1e-30f;
  A.tp.sigma = d.sigma;
  A.tp.csT2 = d.csT2;
  A.tp.varpi = d.varpi;
  const float th[5] = {1.f, d.z_a, d.z_a, d.z_e, d.z_nu};
  for (int k = 0; k < 5; ++k) A.tp.theta[k] = th[k];
  A.tp.w0 = d.wt0;
  A.tp.w1 = d.wt1;
  A.f_act = d.f_act;
  A.T_s = d.T_s;
  A.T_l = d.T_l;
  A.lat = d.lat;
  A.nu_g1 = (float)(-2.0 * kN);
  A.nu_g2 = (float)(0.5 * kN);
  A.nu_tw = (float)(1.5 * kN);
  A.ny0 = y0;
  A.ny1 = y1;
  A.alpha_var = d.alpha_var;   // Sec. 4.1: the flux moments' rate follows f_l(n)
  A.tauT_l = d.tauT_l;
  A.inv_aratio = d.inv_aratio;
  A.flow = d.flow;
  const float w9[9] = {4.f / 9, 1.f / 9, 1.f / 9, 1.f / 9, 1.f / 9,
                       1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36};
  for (int i = 0; i < 9; ++i) A.foff[i] = w9[i] * d.rho0;
  A.phi = d.phi;
  A.K = d.K;
  A.lfl = b.lamf;
  A.lphi = b.lama;
  A.lK = lK;
  A.lTw = b.lamtw;
  // reverse sweep: step m of a stretch whose states sit at F (index m - lo)
  int cur = 0;
  auto reverse = [&](cudaStream_t sm, const float* F, int64_t lo, int64_t hi) {
    for (int64_t m = hi - 1; m >= lo; --m) {
      const float* s0 = F + (size_t)(m - lo) * st;
      const float* s1 = s0 + st;
      A.f0 = s0;
      A.g0 = s0 + 9 * n;
      A.fl0 = s0 + 14 * n;
      A.fl1 = s1 + 14 * n;
      A.lf1 = lf[cur];
      A.lg1 = lg[cur];
      A.lf0 = lf[1 - cur];
      A.lg0 = lg[1 - cur];
      A.next_list = lists[1 - cur];
      A.next_count = counts + 1 - cur;
      b.lamg = lg[cur];
      lbm::adj_coupled_step(c->d, b, A, lists[cur], counts + cur, counts + 1 - cur, sweeps, sm);
      cur ^= 1;
    }
  };
  if (keep_all) {
    reverse(c->stream, S, 0, nsteps);
  } else {
    // Two kinds of work per segment j, on two streams, with the segment's
    // states in one of two buffers (S and S2, alternating):
    //   R(j): its checkpoint copied to the buffer (index 0; a copy outside the
    //         graph), the state set from it (parity 0, empty work lists), len
    //         steps forward with the state after each kept at index m;
    //   B(j): its len reversed steps from the buffer.
    // R(j - 1) runs on a second stream beside B(j): B reads only the buffer
    // and the adjoint arrays, R only the lattice and the other buffer; R(j - 1)
    // waits for B(j + 1), the last reader of its buffer, and B(j) for R(j).
    // Each (kind, len, buffer[, adjoint buffer]) is captured once and replayed.
    float* const Sb[2] = {S, S2};
    auto record_R = [&](cudaStream_t sm, int64_t len, int buf) {
      float* const SS = Sb[buf];
      unsigned* const cc = ctr + 2 * buf;
      lbm::launch_set_state(c->d, SS, SS + 9 * n, sm);
      cudaMemcpyAsync(c->d.fl, SS + 14 * n, n * sizeof(float), cudaMemcpyDeviceToDevice, sm);
      lbm::launch_tile_activity(c->d, sm);
      cudaMemsetAsync(c->d.flags, 0, 2 * sizeof(int) * c->d.ntiles, sm);
      cudaMemsetAsync(c->d.lcount, 0, 2 * sizeof(int), sm);
      if (sm == c->cap) {
        // in a capture: the step sequence of lbm_step's graphs (the next step's
        // far tiles beside each step's enthalpy kernels), the state after each
        // step kept at SS + m st through a counter reset here
        cudaMemsetAsync(cc, 0, 2 * sizeof(unsigned), sm);
        Hooks hk;
        hk.st_base = SS + st;
        hk.st_ctr = cc;
        capture_body(c, (int)len, 0, &hk);
      } else {
        int par = 0;
        for (int64_t m = 1; m <= len; ++m) {
          lbm::launch_flow_walls(c->d, par, 0, sm);
          lbm::launch_fused(c->d, c->tma(), par, 0, sm);
          lbm::launch_enthalpy_solve(c->d, par, sm);
          lbm::launch_enthalpy_commit(c->d, par, sm);
          par ^= 1;
          lbm::launch_keep_state(c->d, par, SS + (size_t)m * st, nullptr, sm);
        }
      }
    };
    struct SegGraph {
      int kind;   // 0 R, 1 B
      int64_t len;
      int buf, cur;
      cudaGraphExec_t ex;
    };
    struct SegGraphs {
      std::vector<SegGraph> v;
      ~SegGraphs() {
        for (SegGraph& g : v) cudaGraphExecDestroy(g.ex);
      }
    } seg_graphs;
    const bool can_capture = !c->graphs_off && capture_streams(c);
    // a captured graph of R (after its checkpoint copy) or B, or nullptr
    auto graph_of = [&](int kind, int64_t len, int buf) -> cudaGraphExec_t {
      for (const SegGraph& g : seg_graphs.v)
        if (g.kind == kind && g.len == len && g.buf == buf && (kind == 0 || g.cur == cur))
          return g.ex;
      if (!can_capture) return nullptr;
      cudaGraphExec_t ex = nullptr;
      cudaGraph_t gr = nullptr;
      const int cur0 = cur;
      if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        if (kind == 0) record_R(c->cap, len, buf);
        else reverse(c->cap, Sb[buf], 0, len);
        if (cudaStreamEndCapture(c->cap, &gr) == cudaSuccess && gr) {
          ex = instantiate(gr);
          if (ex) seg_graphs.v.push_back({kind, len, buf, cur0, ex});
        }
      }
      cudaGetLastError();
      cur = cur0;
      return ex;
    };
    struct Pipe {
      cudaStream_t rs = nullptr;
      cudaEvent_t evR[2] = {nullptr, nullptr}, evB[2] = {nullptr, nullptr};
      ~Pipe() {
        if (rs) cudaStreamDestroy(rs);
        for (cudaEvent_t e : evR)
          if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : evB)
          if (e) cudaEventDestroy(e);
      }
    } pp;
    bool piped = can_capture &&
                 cudaStreamCreateWithFlags(&pp.rs, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; piped && k < 2; ++k)
      piped = cudaEventCreateWithFlags(&pp.evR[k], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&pp.evB[k], cudaEventDisableTiming) == cudaSuccess;
    cudaGetLastError();
    const cudaStream_t rs = piped ? pp.rs : c->stream;
    auto seg_len = [&](int64_t j) { return (j == ncp - 1) ? nsteps - j * K : K; };
    // R runs on rs after everything queued on the context stream so far
    if (piped) {
      LBM_CUDA(cudaEventRecord(pp.evB[1], c->stream));
      LBM_CUDA(cudaStreamWaitEvent(rs, pp.evB[1], 0));
    }
    auto run_R = [&](int64_t j, int buf) -> int {
      const int64_t len = seg_len(j);
      LBM_CUDA(cudaMemcpyAsync(Sb[buf], cps + (size_t)j * st, st * sizeof(float),
                               cudaMemcpyDeviceToDevice, rs));
      cudaGraphExec_t ex = graph_of(0, len, buf);
      if (ex) LBM_CUDA(cudaGraphLaunch(ex, rs));
      else record_R(rs, len, buf);
      if (piped) LBM_CUDA(cudaEventRecord(pp.evR[buf], rs));
      return cuda_err(cudaGetLastError());
    };
    int64_t j = ncp - 1;
    while (j >= 0 && seg_len(j) <= 0) --j;
    int buf = 0;
    if (j >= 0) LBM_TRY(run_R(j, buf));
    bool first = true;
    for (; j >= 0; --j, buf ^= 1, first = false) {
      const int64_t len = seg_len(j);
      if (piped) LBM_CUDA(cudaStreamWaitEvent(c->stream, pp.evR[buf], 0));
      cudaGraphExec_t ex = graph_of(1, len, buf);
      if (ex) {
        LBM_CUDA(cudaGraphLaunch(ex, c->stream));
        if (len & 1) cur ^= 1;
      } else {
        reverse(c->stream, Sb[buf], 0, len);
      }
      if (piped) LBM_CUDA(cudaEventRecord(pp.evB[buf], c->stream));
      if (j > 0) {
        // R(j - 1) into the other buffer, once B(j + 1) is done with it
        if (piped && !first) LBM_CUDA(cudaStreamWaitEvent(rs, pp.evB[buf ^ 1], 0));
        LBM_TRY(run_R(j - 1, buf ^ 1));
      }
      LBM_CUDA(cudaGetLastError());
    }
    // back to where the forward run ended
    LBM_TRY(lbm_set_state(c, fin, fin + 9 * n, fin + 14 * n, 1));
    c->steps = steps0 + nsteps;
  }
  ph.mark(2);
  // d J / d ln K = K d J / d K, then straight into the caller's arrays
  lbm::adj_mul((long long)n, lK, d.K, c->stream);
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  LBM_CUDA(cudaMemcpyAsync(d_phi, b.lama, n * sizeof(float), kind, c->stream));
  LBM_CUDA(cudaMemcpyAsync(d_lnK, lK, n * sizeof(float), kind, c->stream));
  LBM_CUDA(cudaMemcpyAsync(d_wall_T_left, b.lamtw, d.ny * sizeof(float), kind, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  // the context ends where the forward run left it
  return LBM_OK;
}
