// lbm_fused_f32_open_hermite.cu -- the fused step kernel for FP32 deviation storage:
// BGK and MRT with the Hermite equilibrium, no-slip walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 10)
LBM_INSTANTIATE_FUSED(float, 11)
