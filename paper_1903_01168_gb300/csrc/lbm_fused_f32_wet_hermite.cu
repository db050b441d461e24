// lbm_fused_f32_wet_hermite.cu -- the fused step kernel for FP32 deviation storage:
// BGK and MRT with the Hermite equilibrium and wetting walls, periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 6)
LBM_INSTANTIATE_FUSED(float, 7)
