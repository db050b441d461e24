// lbm_fused_f16_wet.cu -- the fused step kernel for FP16 deviation storage,
// the four collision variants with wetting walls (free slip, contact angle).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 4)
LBM_INSTANTIATE_FUSED(__half, 5)
LBM_INSTANTIATE_FUSED(__half, 6)
LBM_INSTANTIATE_FUSED(__half, 7)
