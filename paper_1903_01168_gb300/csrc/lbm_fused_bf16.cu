// lbm_fused_bf16.cu -- the fused step kernel for BF16 split-form deviation storage: BGK and MRT with
// the standard equilibrium and no-slip walls, periodic in x (one
// small translation unit per storage type and variant pair, compiled in parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 0)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 1)
