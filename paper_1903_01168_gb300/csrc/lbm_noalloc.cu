// lbm_noalloc.cu -- lbm_step_noalloc: the two-pass step on caller-owned
// state memory with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code running where device allocation is
// forbidden or unavailable (a host that hands out pre-registered memory pools
// only, allocation-free real-time loops, or embedding runtimes whose own
// allocator owns the device).  This entry point lets them advance a
// simulation whose state they own.  The intermediate colour-field pass and the
// simulation descriptor the kernels read live in fixed-size arrays that are
// part of the loaded library; the kernels are the library's two-pass kernels.
#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

// Scratch of the two-pass step (psi, rho_r, rho_b, q u_x, q u_y per node) for
// lattices of up to NOALLOC_MAX_NODES nodes, and the descriptor of the
// simulation being stepped.  Every GPU that loads the library holds these
// 5 * 262144 * 4 bytes (5 MiB) plus one descriptor until the process exits.
constexpr long long NOALLOC_MAX_NODES = 262144;
static __device__ __align__(256) float g_noalloc_scratch[AUX_FIELDS * NOALLOC_MAX_NODES];
static __device__ SimDesc g_noalloc_desc;

// Device addresses of the two arrays, resolved once per device with that
// device current (host code cannot use the symbols themselves as addresses).
constexpr int MAX_DEVICES = 64;
struct StaticAddrs {
    float *scratch = nullptr;
    SimDesc *desc = nullptr;
};
StaticAddrs g_addr[MAX_DEVICES];
std::mutex g_addr_mu;

lbm_status static_addrs_for_device(int dev, StaticAddrs *out, char *err) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        snprintf(err, 256, "lbm_step_noalloc: device %d out of range", dev);
        return LBM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev].scratch) {
        void *ps = nullptr, *pd = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ps, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&pd, g_noalloc_desc);
        if (e != cudaSuccess || !ps || !pd) {
            snprintf(err, 256, "lbm_step_noalloc: cudaGetSymbolAddress of the static arrays failed: %s",
                     cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        g_addr[dev].scratch = static_cast<float *>(ps);
        g_addr[dev].desc = static_cast<SimDesc *>(pd);
    }
    *out = g_addr[dev];
    return LBM_OK;
}

lbm_status fail(lbm_status st, char *err) {
    host_set_global_error(err);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_params *p, int nx, int ny, void *state, size_t bytes, long long t,
                                       long n, void *cuda_stream) {
    char err[256] = "";
    lbm_status v = host_validate(nx, ny, p, err);
    if (v != LBM_OK) return fail(v, err);
    if ((long long)nx * ny > NOALLOC_MAX_NODES) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: %d x %d = %lld nodes exceeds the static scratch limit of %lld nodes",
                 nx, ny, (long long)nx * ny, NOALLOC_MAX_NODES);
        return fail(LBM_EINVAL, err);
    }
    const size_t need = lbm_bytes_required(nx, ny, p);
    if (!state || bytes < need || (reinterpret_cast<uintptr_t>(state) & 255) || t < 0 || n < 0) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: state NULL, unaligned or smaller than %zu bytes, or t / n < 0",
                 need);
        return fail(bytes < need ? LBM_ENOMEM : LBM_EINVAL, err);
    }
    // The state must be device (or managed) memory of the current device: a host
    // pointer or another GPU's buffer would make the kernels fault.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: no usable current CUDA device: %s", cudaGetErrorString(e));
        return fail(LBM_ECUDA, err);
    }
    cudaPointerAttributes attr{};
    e = cudaPointerGetAttributes(&attr, state);
    if (e != cudaSuccess || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
        attr.device != dev) {
        if (e != cudaSuccess) cudaGetLastError();   // the query's own error is the answer, not a fault
        snprintf(err, sizeof(err), "lbm_step_noalloc: state is not device memory of the current device %d", dev);
        return fail(LBM_EINVAL, err);
    }
    if (n == 0) return LBM_OK;
    // An error left pending by earlier, unrelated work would otherwise be
    // reported (and cleared) as a failure of these launches.
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: a CUDA error was pending before the call: %s",
                 cudaGetErrorString(e));
        return fail(LBM_ECUDA, err);
    }
    StaticAddrs a;
    lbm_status st = static_addrs_for_device(dev, &a, err);
    if (st != LBM_OK) return fail(st, err);
    SimDesc h;
    host_fill_desc(h, nx, ny, p, state);
    h.t0 = t;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // The copy is ordered before the kernels on the stream; the host copy of a
    // pageable source is staged before the call returns.
    e = cudaMemcpyAsync(a.desc, &h, sizeof(SimDesc), cudaMemcpyHostToDevice, s);
    const long long nodes = (long long)nx * ny;
    for (long j = 0; j < n && e == cudaSuccess; j++) {
        e = p->storage == ST_F32 ? twopass_launch<float>(h.variant, a.desc, (int)j, a.scratch, nodes, s)
            : p->storage == ST_F16DEV ? twopass_launch<__half>(h.variant, a.desc, (int)j, a.scratch, nodes, s)
                                      : twopass_launch<__nv_bfloat16>(h.variant, a.desc, (int)j, a.scratch, nodes, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(err, sizeof(err), "lbm_step_noalloc: launch failed: %s", cudaGetErrorString(e));
        return fail(LBM_ECUDA, err);
    }
    return LBM_OK;
}
