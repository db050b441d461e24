// lbm_twopass_bf16.cu -- the two-pass step kernels for BF16 deviation storage, all
// four collision variants (one translation unit per storage type, compiled in
// parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_TWOPASS(__nv_bfloat16)
