// Mixed-precision form of the C-GBR interface sweep: FP32 characteristic
// reconstruction, MP5 selection and HLLC on primitives recovered in FP64; the
// flux differences, residual and RK update stay FP64.  This translation unit
// is compiled with FMA contraction (the FP64 parity unit is not).
#include "cg_kernels.cuh"

namespace cgk {

template <int ND, int DIR, bool CART, bool COMPACT>
static int launch_f32(const DevGrid& g, const GbrCfg& q, const StageArgs& A, dim3 grid, cudaStream_t st) {
  size_t smem = sizeof(float) * sweep_smem_doubles<ND, DIR>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gbr_sweep<ND, DIR, CART, COMPACT, float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  k_gbr_sweep<ND, DIR, CART, COMPACT, float><<<grid, 256, smem, st>>>(g, q, A);
  return (int)cudaGetLastError();
}

template <int ND, int DIR>
static int launch_f32_any(bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A, dim3 grid,
                          cudaStream_t st) {
  if (cart) return compact ? launch_f32<ND, DIR, true, true>(g, q, A, grid, st) : launch_f32<ND, DIR, true, false>(g, q, A, grid, st);
  return compact ? launch_f32<ND, DIR, false, true>(g, q, A, grid, st) : launch_f32<ND, DIR, false, false>(g, q, A, grid, st);
}

// Returns a cudaError_t value (0 on success).
int launch_sweep_f32(int nd, int dir, bool cart, bool compact, const DevGrid& g, const GbrCfg& q, const StageArgs& A,
                     dim3 grid, cudaStream_t st) {
#define CGK_CASE(ND_, DIR_) \
  if (nd == ND_ && dir == DIR_) return launch_f32_any<ND_, DIR_>(cart, compact, g, q, A, grid, st);
  CGK_CASE(1, 0)
  CGK_CASE(2, 0)
  CGK_CASE(2, 1)
  CGK_CASE(3, 0)
  CGK_CASE(3, 1)
  CGK_CASE(3, 2)
#undef CGK_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace cgk
