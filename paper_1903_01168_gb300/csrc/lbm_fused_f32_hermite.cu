// lbm_fused_f32_hermite.cu -- the fused step kernel for FP32 deviation storage: BGK
// and MRT with the Hermite equilibrium and no-slip walls, periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 2)
LBM_INSTANTIATE_FUSED(float, 3)
