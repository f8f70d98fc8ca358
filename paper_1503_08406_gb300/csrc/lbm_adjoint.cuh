// Host entry points of the adjoint of the conduction step (lbm_adjoint.cu).
#pragma once
#include "lbm_flow_adjoint.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// all buffers n floats unless noted
struct AdjBuffers {
  float* a;          // a = phi dT / (sigma St)
  float* lamg;       // 5 n: adjoint of the populations after the step being reversed
  float* lamf;       // adjoint of f_l after the step (in), before it (out)
  float* rhs;        // band nodes (wide bands): right-hand side of mu's equation
  float* mu0;        // mu in global memory (wide bands), ping-pong
  float* mu1;
  float* lamgpre;    // 5 n: adjoint of the populations before the step
  float* lama;       // accumulated adjoint of a
  float* lamtw;      // ny: accumulated adjoint of the left wall profile
  int* pos;          // n: a band node's place in the band list
  float At[25];      // transposed collision matrix (u = 0), passed to kernels by value
};
struct Mat5 {
  float m[25];
};
// Objective terms the reverse sweep adds per state: the adjoint of the
// populations at x = 1 and x = 2 (all five planes) and of the left wall
// profile (the time-averaged left-wall Nusselt number: -2, 1/2 and 3/2 times
// H / (dT rows N)); zero for the melted fraction.
struct NuSrc {
  float g1, g2, tw;
};
// the left-wall Nusselt number of the current state (lbm_reduce's out[3]),
// added to acc[0] (lbm_aux.cu)
void launch_wall_nusselt(const Dev& d, int layout, double* acc, cudaStream_t s);
// a = phi dT / (sigma St); lam_g = the Nusselt terms of the last state; lam_f
// = 1 / (non-wall nodes) on non-wall nodes for the melted fraction (melt),
// else 0
void adj_seed(const Dev& d, float* lamf, float* lamg, float* a, bool melt, NuSrc nu,
              cudaStream_t s);
// v[0..n) *= k
void adj_scale(long long n, float* v, float k, cudaStream_t s);
// v[0..n) *= w[0..n)
void adj_mul(long long n, float* v, const float* w, cudaStream_t s);
// a = phi dT / (sigma St)
void adj_a(const Dev& d, float* a, cudaStream_t s);
// J into out[0]; out holds 129 doubles (the rest: partial sums)
void adj_objective(const Dev& d, const float* fl, double* out, cudaStream_t s);
// the band (non-wall nodes with 0 < f < 1), appended at list[*count]
void adj_list(const Dev& d, const float* f, int* list, int* count, cudaStream_t s);
// d.fl to base + k n, k = ctr[0], which then advances (ctr[1]: scratch, 0)
void adj_save(const Dev& d, float* base, unsigned* ctr, cudaStream_t s);
// One step of the reverse sweep, given f_l before (f0) and after (f1) it and
// the band after it (list, count): from b.lamg / b.lamf (after the step) to
// b.lamgpre / b.lamf (before it), the Nusselt terms (nu) of the state before
// it included.  old_list / old_count hold the band the
// previous call solved on; they are emptied and refilled with the band before
// this step, for the next call.  The caller swaps b.lamg and b.lamgpre and the
// two lists.
void adj_step(const Dev& d, const AdjBuffers& b, const float* f0, const float* f1, int* list,
              int* count, int* old_list, int* old_count, int mu_sweeps, NuSrc nu,
              cudaStream_t s);
// One reversed step of the coupled adjoint (flow on): the band kernel on
// b.lamg / b.lamf (A.lg1 is b.lamg, A.lfl is b.lamf, A.fl1 the band's f_l),
// then lbm::coupled_reverse_node over every node; the band before the step is
// listed at A.next_list (its count at old_count, emptied first).
void adj_coupled_step(const Dev& d, const AdjBuffers& b, const CoupledStep<float>& A, int* list,
                      int* count, int* old_count, int mu_sweeps, cudaStream_t s);
// once per process before adj_step: the band kernel's shared-memory opt-in
bool adj_init();

}  // namespace lbm
