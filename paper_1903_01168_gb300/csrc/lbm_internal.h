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

// Launchers of the step kernels.  Each (storage type T, variant CV) pair of the
// fused kernel is instantiated explicitly in its own translation unit group
// (lbm_fused_*.cu: variants without and with wetting walls), and the two-pass
// kernels of each T in lbm_twopass_*.cu, so that the units compile in parallel.
// `flags`: FUSED_EARLY_NEXT lets the next step launch as soon as this one starts.
template <typename T, int CV>
cudaError_t fused_launch_cv(const SimDesc *descs, const WorkItem *items, const int *item_off, int n_blocks, int off,
                            int flags, int *err, cudaStream_t st);
template <typename T, int CV>
const void *fused_kernel_cv();
template <typename T, int CV>
int fused_smem_cv();

// Run-time dispatch over the variants (bits CV_MRT, CV_HERMITE, CV_WET, CV_OPEN).
#define LBM_DISPATCH_CV(variant, CALL)          \
    switch (variant) {                           \
    case 0: CALL(0);                             \
    case 1: CALL(1);                             \
    case 2: CALL(2);                             \
    case 3: CALL(3);                             \
    case 4: CALL(4);                             \
    case 5: CALL(5);                             \
    case 6: CALL(6);                             \
    case 7: CALL(7);                             \
    case 8: CALL(8);                             \
    case 9: CALL(9);                             \
    case 10: CALL(10);                           \
    case 11: CALL(11);                           \
    case 12: CALL(12);                           \
    case 13: CALL(13);                           \
    case 14: CALL(14);                           \
    default: CALL(15);                           \
    }

template <typename T>
cudaError_t fused_launch(int variant, const SimDesc *descs, const WorkItem *items, const int *item_off,
                         int n_blocks, int off, int flags, int *err, cudaStream_t st) {
#define LBM_CALL_(cv) return fused_launch_cv<T, cv>(descs, items, item_off, n_blocks, off, flags, err, st)
    LBM_DISPATCH_CV(variant, LBM_CALL_)
#undef LBM_CALL_
}
template <typename T>
const void *fused_kernel(int variant) {
#define LBM_CALL_(cv) return fused_kernel_cv<T, cv>()
    LBM_DISPATCH_CV(variant, LBM_CALL_)
#undef LBM_CALL_
}
template <typename T>
int fused_smem(int variant) {
#define LBM_CALL_(cv) return fused_smem_cv<T, cv>()
    LBM_DISPATCH_CV(variant, LBM_CALL_)
#undef LBM_CALL_
}

// Both passes of one two-pass step over `nodes` nodes of the descriptor at
// `desc` (device memory), step `off` of a launch chunk, scratch `aux`.  The
// two-pass kernels handle wetting walls in every variant (the CV_WET bit is
// ignored).
template <typename T>
cudaError_t twopass_launch(int variant, const SimDesc *desc, int off, float *aux, long long nodes,
                           cudaStream_t st);

}  // namespace lbm
