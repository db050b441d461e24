// lbm_twopass_f32.cu -- the two-pass step kernels for FP32 deviation storage, all
// four collision variants (one translation unit per storage type, compiled in
// parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_TWOPASS(float)
