// lbm_fused_f16_open.cu -- the fused step kernel for FP16 split-form deviation storage: BGK and
// MRT with the standard equilibrium, no-slip walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 8)
LBM_INSTANTIATE_FUSED(__half, 9)
