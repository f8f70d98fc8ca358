// Stream-collide kernels instantiated for FP32 population storage.
#include "lbm_fused.cuh"

namespace lbm {

void launch_flow_walls_f32(const Dev& d, int parity, int mode, cudaStream_t s) {
  launch_flow_walls_t<float>(d, parity, mode, s);
}

void launch_fused_f32(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  launch_fused_t<float>(d, m, parity, mode, s);
}

bool tma_setup_f32(Dev& d, TmaMaps* m) { return tma_setup_t<float>(d, m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32); }

void fused_batch_setup() {
  const int s0 = TmaLayout<0, float>::SMEM, s1 = TmaLayout<1, float>::SMEM;
#define LBM_SMEM(P, FL, MO, SM)                                                      \
  cudaFuncSetAttribute(fused_tma_batch_kernel<float, P, FL, MO>,                     \
                       cudaFuncAttributeMaxDynamicSharedMemorySize, SM)
  LBM_SMEM(0, 1, 0, s0); LBM_SMEM(0, 1, 1, s0); LBM_SMEM(0, 1, 2, s0);
  LBM_SMEM(0, 0, 0, s0); LBM_SMEM(0, 0, 1, s0); LBM_SMEM(0, 0, 2, s0);
  LBM_SMEM(1, 1, 0, s1); LBM_SMEM(1, 1, 1, s1); LBM_SMEM(1, 1, 2, s1);
  LBM_SMEM(1, 0, 0, s1); LBM_SMEM(1, 0, 1, s1); LBM_SMEM(1, 0, 2, s1);
#undef LBM_SMEM
}

template <int PAR, int FL, int MO>
static void fused_batch_one(const BatchPlan& P, const TmaMaps* maps, cudaStream_t s) {
  fused_tma_batch_kernel<float, PAR, FL, MO>
      <<<P.start[P.count], dim3(TX, TY), TmaLayout<PAR, float>::SMEM, s>>>(P, maps);
}

template <int PAR, int FL>
static void fused_batch_mode(const BatchPlan& P, const TmaMaps* maps, int mode, cudaStream_t s) {
  if (mode == 0) fused_batch_one<PAR, FL, 0>(P, maps, s);
  else if (mode == 1) fused_batch_one<PAR, FL, 1>(P, maps, s);
  else fused_batch_one<PAR, FL, 2>(P, maps, s);
}

void launch_fused_batch(const BatchPlan& P, const TmaMaps* maps, int parity, int mode, bool flow,
                        cudaStream_t s) {
  if (parity == 0) {
    if (flow) fused_batch_mode<0, 1>(P, maps, mode, s);
    else fused_batch_mode<0, 0>(P, maps, mode, s);
  } else {
    if (flow) fused_batch_mode<1, 1>(P, maps, mode, s);
    else fused_batch_mode<1, 0>(P, maps, mode, s);
  }
}

// Self-check of the bounded wait: one CTA initialises an mbarrier that no copy
// and no thread ever completes, waits on it with mbar_wait's limit, and on
// giving up sets the same timeout flag the stream-collide kernel sets.  Nothing
// is in flight when it returns.
__global__ void wait_probe_kernel(Dev d, long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(b, 0u, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(&d.stats[4], 3);
}

void launch_wait_probe(const Dev& d, long long limit_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(d, limit_ns);
}

}  // namespace lbm
