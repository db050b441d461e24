// lbm_fused_f16_open_wet.cu -- the fused step kernel for FP16 split-form deviation storage: BGK
// and MRT with the standard equilibrium, wetting walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 12)
LBM_INSTANTIATE_FUSED(__half, 13)
