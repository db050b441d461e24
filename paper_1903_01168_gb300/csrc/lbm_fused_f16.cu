// lbm_fused_f16.cu -- the fused step kernel for FP16 deviation storage, all
// four collision variants (one translation unit per storage type, compiled in
// parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half)
