// lbm_internal.h -- host helpers shared between the translation units of the
// library (not part of the C ABI).
#pragma once

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Validate a parameter set (message into err, 256 bytes).
lbm_status host_validate(int nx, int ny, const lbm_params *p, char *err);

// Fill a descriptor for a state buffer laid out as by lbm_create (densities
// region followed by deviations region).  Tensor maps are left zero.
void host_fill_desc(SimDesc &h, int nx, int ny, const lbm_params *p, void *state);

// Message returned by lbm_last_error(NULL) on this thread.
void host_set_global_error(const char *msg);

// Launch shape of the fused kernel: columns per strip (= threads per block)
// and shared-memory row slots per block.
#ifndef LBM_FUSED_NSLOT
#define LBM_FUSED_NSLOT 4
#endif
constexpr int FUSED_W = 128;
constexpr int FUSED_NSLOT = LBM_FUSED_NSLOT;

// Launchers of the step kernels.  Each storage type T (float, __half,
// __nv_bfloat16) is instantiated in its own translation units
// (lbm_fused_*.cu, lbm_twopass_*.cu) so that they compile in parallel;
// `variant` is the collision variant (bits CV_MRT, CV_HERMITE).
template <typename T>
cudaError_t fused_launch(int variant, const SimDesc *descs, const WorkItem *items, const int *item_off,
                         int n_blocks, int off, int *err, cudaStream_t st);
template <typename T>
const void *fused_kernel(int variant);
template <typename T>
int fused_smem(int variant);
// Both passes of one two-pass step over `nodes` nodes of the descriptor at
// `desc` (device memory), step `off` of a launch chunk, scratch `aux`.
template <typename T>
cudaError_t twopass_launch(int variant, const SimDesc *desc, int off, float *aux, long long nodes,
                           cudaStream_t st);

}  // namespace lbm
