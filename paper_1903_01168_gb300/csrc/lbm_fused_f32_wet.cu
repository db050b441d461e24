// lbm_fused_f32_wet.cu -- the fused step kernel for FP32 deviation storage,
// the four collision variants with wetting walls (free slip, contact angle).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 4)
LBM_INSTANTIATE_FUSED(float, 5)
LBM_INSTANTIATE_FUSED(float, 6)
LBM_INSTANTIATE_FUSED(float, 7)
