// lbm_fused_f32.cu -- the fused step kernel for FP32 deviation storage, the
// four collision variants with no-slip walls (one translation unit per storage
// type and wall kind, compiled in parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(float, 0)
LBM_INSTANTIATE_FUSED(float, 1)
LBM_INSTANTIATE_FUSED(float, 2)
LBM_INSTANTIATE_FUSED(float, 3)
