// lbm_fused_bf16_open.cu -- the fused step kernel for BF16 split-form deviation storage: BGK and
// MRT with the standard equilibrium, no-slip walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 8)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 9)
