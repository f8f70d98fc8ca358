// Stream-collide kernels instantiated for FP16 population storage.
#include "lbm_fused.cuh"

namespace lbm {

void launch_flow_walls_f16(const Dev& d, int parity, int mode, cudaStream_t s) {
  launch_flow_walls_t<__half>(d, parity, mode, s);
}

void launch_fused_f16(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  launch_fused_t<__half>(d, m, parity, mode, s);
}

bool tma_setup_f16(Dev& d, TmaMaps* m) { return tma_setup_t<__half>(d, m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16); }

}  // namespace lbm
