// lbm_fused_f16.cu -- the fused step kernel for FP16 deviation storage, the
// four collision variants with no-slip walls (one translation unit per storage
// type and wall kind, compiled in parallel).
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 0)
LBM_INSTANTIATE_FUSED(__half, 1)
LBM_INSTANTIATE_FUSED(__half, 2)
LBM_INSTANTIATE_FUSED(__half, 3)
