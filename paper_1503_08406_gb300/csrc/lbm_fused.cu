// Stream-collide dispatch and tensor-map encoding.  The kernels themselves are
// templates in lbm_fused.cuh, instantiated once per population storage type in
// lbm_fused_f32.cu, lbm_fused_f16.cu and lbm_fused_bf16.cu (compiled in parallel).
#include <cuda.h>

#include "lbm_internal.cuh"

namespace lbm {

void launch_fused_f32(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s);
void launch_fused_f16(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s);
void launch_fused_bf16(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s);
bool tma_setup_f32(Dev& d, TmaMaps* m);
void launch_flow_walls_f32(const Dev& d, int parity, int mode, cudaStream_t s);
void launch_flow_walls_f16(const Dev& d, int parity, int mode, cudaStream_t s);
void launch_flow_walls_bf16(const Dev& d, int parity, int mode, cudaStream_t s);

void launch_flow_walls(const Dev& d, int parity, int mode, cudaStream_t s) {
  if (!d.flow || !d.flow_walls) return;
  if (d.storage == 1) launch_flow_walls_f16(d, parity, mode, s);
  else if (d.storage == 2) launch_flow_walls_bf16(d, parity, mode, s);
  else launch_flow_walls_f32(d, parity, mode, s);
}
bool tma_setup_f16(Dev& d, TmaMaps* m);
bool tma_setup_bf16(Dev& d, TmaMaps* m);

void launch_fused(const Dev& d, const TmaMaps* m, int parity, int mode, cudaStream_t s) {
  if (d.storage == 1) launch_fused_f16(d, m, parity, mode, s);
  else if (d.storage == 2) launch_fused_bf16(d, m, parity, mode, s);
  else launch_fused_f32(d, m, parity, mode, s);
}

int tma_grid(const Dev& d, int tpc) {
  const long long ntile = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
  const long long slots = d.tslots > 0 ? d.tslots : 1;
  if (tpc < 1) tpc = 1;
  long long waves = (ntile + slots * tpc / 2) / (slots * tpc);
  if (waves < 1) waves = 1;
  long long grid = waves * slots;
  if (grid > ntile) grid = ntile;
  if ((ntile + grid - 1) / grid > 32) grid = (ntile + 31) / 32;
  return (int)grid;
}

bool tma_setup(Dev& d, TmaMaps* m) {
  if (d.storage == 1) return tma_setup_f16(d, m);
  if (d.storage == 2) return tma_setup_bf16(d, m);
  return tma_setup_f32(d, m);
}


typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
    else
      cudaGetLastError();
  }
  return fn;
}

bool tma_encode(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, int rank,
                int nx, int ny, int planes, int bx, int by) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)planes};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, dt, rank, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbm
