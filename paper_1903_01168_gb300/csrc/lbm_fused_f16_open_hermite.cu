// lbm_fused_f16_open_hermite.cu -- the fused step kernel for FP16 split-form deviation storage:
// BGK and MRT with the Hermite equilibrium, no-slip walls and inlet / outlet columns.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 10)
LBM_INSTANTIATE_FUSED(__half, 11)
