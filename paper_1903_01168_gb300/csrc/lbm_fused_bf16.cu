// lbm_fused_bf16.cu -- the fused step kernel for BF16 deviation storage, all
// four collision variants (one translation unit per storage type, compiled in
// parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__nv_bfloat16)
