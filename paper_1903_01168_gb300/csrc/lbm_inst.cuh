// lbm_inst.cuh -- definitions of the step-kernel launchers declared in
// lbm_internal.h.  Included by small translation units that instantiate them
// for one storage type: LBM_INSTANTIATE_FUSED(T, CV) per fused variant, or
// LBM_INSTANTIATE_TWOPASS(T).
#pragma once

#define LBM_DEVICE_HELPERS_ONLY
#include <algorithm>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename T, int CV>
const void *fused_kernel_cv() {
    return reinterpret_cast<const void *>(&k_step_fused<T, CV, FUSED_W, FUSED_NSLOT, 1>);
}

template <typename T, int CV>
int fused_smem_cv() {
    return FusedCfg<T, CV, FUSED_W, FUSED_NSLOT>::SMEM;
}

template <typename T, int CV>
cudaError_t fused_launch_cv(const SimDesc *descs, const WorkItem *items, const int *item_off, int n_blocks, int off,
                            int flags, int *err, cudaStream_t st) {
    constexpr int SMEM = FusedCfg<T, CV, FUSED_W, FUSED_NSLOT>::SMEM;
    static bool attr_done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    // the downward kernel is compiled only where some step uses it
    constexpr bool DOWN = LBM_FUSED_ALTERNATE != 0;
    auto up = k_step_fused<T, CV, FUSED_W, FUSED_NSLOT, 1>;
    auto down = k_step_fused<T, CV, FUSED_W, FUSED_NSLOT, DOWN ? -1 : 1>;
    if (dev < 64 && !attr_done[dev]) {
        cudaError_t e = cudaFuncSetAttribute(up, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e == cudaSuccess && DOWN) e = cudaFuncSetAttribute(down, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    // programmatic dependent launch: the launch of step j+1 overlaps the tail of
    // step j; the kernel waits for its prerequisites before its first access
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3(FUSED_W);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = LBM_FUSED_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool march_down = LBM_FUSED_ALTERNATE == 2 || (LBM_FUSED_ALTERNATE == 1 && (off & 1));
    return cudaLaunchKernelEx(&cfg, march_down ? down : up, descs, items, item_off, n_blocks, off, flags, err);
}

template <typename T, int CV>
cudaError_t twopass_launch_cv(const SimDesc *desc, int off, float *aux, long long nodes, cudaStream_t st) {
    const int g = (int)std::max<long long>(1, std::min<long long>((nodes + 255) / 256, 152LL * 16));
    k_tp_moments<T, CV><<<g, 256, 0, st>>>(desc, off, aux);
    k_tp_collide<T, CV><<<g, 256, 0, st>>>(desc, off, aux);
    return cudaPeekAtLastError();
}

template <typename T>
cudaError_t twopass_launch(int variant, const SimDesc *desc, int off, float *aux, long long nodes, cudaStream_t st) {
    switch (variant & (CV_MRT | CV_HERMITE)) {
    case 0: return twopass_launch_cv<T, 0>(desc, off, aux, nodes, st);
    case CV_MRT: return twopass_launch_cv<T, CV_MRT>(desc, off, aux, nodes, st);
    case CV_HERMITE: return twopass_launch_cv<T, CV_HERMITE>(desc, off, aux, nodes, st);
    default: return twopass_launch_cv<T, CV_MRT | CV_HERMITE>(desc, off, aux, nodes, st);
    }
}

}  // namespace lbm

#define LBM_INSTANTIATE_FUSED(T, CV)                                                                            \
    template cudaError_t lbm::fused_launch_cv<T, CV>(const lbm::SimDesc *, const lbm::WorkItem *, const int *, \
                                                     int, int, int, int *, cudaStream_t);                      \
    template const void *lbm::fused_kernel_cv<T, CV>();                                                        \
    template int lbm::fused_smem_cv<T, CV>();

#define LBM_INSTANTIATE_TWOPASS(T) \
    template cudaError_t lbm::twopass_launch<T>(int, const lbm::SimDesc *, int, float *, long long, cudaStream_t);
