// lbm_fused_bf16.cu -- the fused step kernel for BF16 deviation storage, the
// four collision variants with no-slip walls (one translation unit per storage
// type and wall kind, compiled in parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16, 0)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 1)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 2)
LBM_INSTANTIATE_FUSED(__nv_bfloat16, 3)
