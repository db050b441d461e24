// lbm_fused_bf16_open_wet_hermite.cu -- the fused step kernel for BF16 split-form deviation storage:
// BGK and MRT with the Hermite equilibrium, wetting walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 14)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 15)
