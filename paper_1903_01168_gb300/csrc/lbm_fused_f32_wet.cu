// lbm_fused_f32_wet.cu -- the fused step kernel for FP32 deviation storage: BGK and
// MRT with the standard equilibrium and wetting walls (free slip, contact angle), periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 4)
LBM_INSTANTIATE_FUSED(float, 5)
