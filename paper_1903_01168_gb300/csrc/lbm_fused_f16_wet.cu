// lbm_fused_f16_wet.cu -- the fused step kernel for FP16 split-form deviation storage: BGK and
// MRT with the standard equilibrium and wetting walls (free slip, contact angle), periodic in x.
#include "lbm_inst.cuh"

LBM_INSTANTIATE_FUSED(__half, 4)
LBM_INSTANTIATE_FUSED(__half, 5)
