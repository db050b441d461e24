// lbm_fused_f32_open.cu -- the fused step kernel for FP32 deviation storage: BGK and
// MRT with the standard equilibrium, no-slip walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 8)
LBM_INSTANTIATE_FUSED(float, 9)
