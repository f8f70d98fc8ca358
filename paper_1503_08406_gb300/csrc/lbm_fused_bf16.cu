// Stream-collide kernels instantiated for BF16 population storage.
#include "lbm_fused.cuh"

namespace lbm {

void launch_flow_walls_bf16(const Dev& d, int parity, int mode, cudaStream_t s) {
  launch_flow_walls_t<__nv_bfloat16>(d, parity, mode, s);
}

void launch_fused_bf16(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  launch_fused_t<__nv_bfloat16>(d, m, parity, mode, s);
}

bool tma_setup_bf16(Dev& d, TmaMaps* m) { return tma_setup_t<__nv_bfloat16>(d, m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16); }

}  // namespace lbm
