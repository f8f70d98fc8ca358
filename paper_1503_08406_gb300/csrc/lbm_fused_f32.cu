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
