// lbm_fused_bf16_hermite.cu -- the fused step kernel for BF16 split-form deviation storage: BGK
// and MRT with the Hermite equilibrium and no-slip walls, periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 2)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 3)
