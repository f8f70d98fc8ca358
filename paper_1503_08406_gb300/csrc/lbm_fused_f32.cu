// Stream-collide kernels instantiated for FP32 population storage.
#include "lbm_fused.cuh"

namespace lbm {

void launch_fused_f32(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  launch_fused_t<float>(d, m, parity, mode, s);
}

bool tma_setup_f32(Dev& d, TmaMaps* m) { return tma_setup_t<float>(d, m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32); }

}  // namespace lbm
