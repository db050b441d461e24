// lbm_fused_f32.cu -- the fused step kernel for FP32 deviation storage: BGK and MRT with
// the standard equilibrium and no-slip walls, periodic in x (one
// small translation unit per storage type and variant pair, compiled in parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 0)
LBM_INSTANTIATE_FUSED(float, 1)
