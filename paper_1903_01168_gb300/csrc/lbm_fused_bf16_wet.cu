// lbm_fused_bf16_wet.cu -- the fused step kernel for BF16 split-form deviation storage: BGK and
// MRT with the standard equilibrium and wetting walls (free slip, contact angle), periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 4)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 5)
