// lbm_fused_f16_wet_hermite.cu -- the fused step kernel for FP16 split-form deviation storage:
// BGK and MRT with the Hermite equilibrium and wetting walls, periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 6)
LBM_INSTANTIATE_FUSED(__half, 7)
