// lbm_noalloc.cu -- lbm_step_noalloc: the two-pass step on caller-owned
// state memory with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code running where device allocation is
// forbidden or unavailable (a host that hands out pre-registered memory pools
// only, allocation-free real-time loops, or embedding runtimes whose own
// allocator owns the device).  This entry point lets them advance a
// simulation whose state they own, with the intermediate colour-field pass
// kept in a fixed-size scratch array that is part of the loaded library.
#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"
#define LBM_DEVICE_HELPERS_ONLY
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

// Scratch of the two-pass step (psi, rho_r, rho_b, q u_x, q u_y per node) for
// lattices of up to LBM_NOALLOC_MAX_NODES nodes.  Every GPU that loads the
// library holds these 5 * 262144 * 4 bytes (5 MiB) until the process exits.
constexpr long long NOALLOC_MAX_NODES = 262144;
static __device__ __align__(256) float g_noalloc_scratch[AUX_FIELDS * NOALLOC_MAX_NODES];

// Device address of the scratch, resolved once per device with that device current.
constexpr int MAX_DEVICES = 64;
float *g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

lbm_status scratch_for_current_device(float **out, char *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        snprintf(err, 256, "no usable current CUDA device");
        return LBM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            snprintf(err, 256, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<float *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

// Pass 1 of the two-pass step, descriptor passed by value.
template <typename T, int CV>
__global__ void k_na_moments(const __grid_constant__ SimDesc d, int step_offset, float *__restrict__ aux) {
    constexpr bool HERMITE = (CV & CV_HERMITE) != 0, HERMITE_SRC = HERMITE && (CV & CV_MRT);
    const Phys p = d.ph;
    const long long t = d.t0 + step_offset;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L(d, (int)(t & 1));
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        Pulled P;
        pull_node<HERMITE>(p, L, x, y, t, false, 0.0f, 0.0f, P);
        const NodeMoments m = node_moments(p, P);
        aux[k] = m.psi;
        aux[n + k] = m.rr;
        aux[2 * n + k] = m.rb;
        if (HERMITE_SRC) {
            const float q = p.q_r * m.rr + p.q_b * m.rb;
            aux[3 * n + k] = q * m.ux;
            aux[4 * n + k] = q * m.uy;
        }
    }
}

// Pass 2 of the two-pass step, descriptor passed by value.
template <typename T, int CV>
__global__ void k_na_collide(const __grid_constant__ SimDesc d, int step_offset, const float *__restrict__ aux) {
    constexpr bool HERMITE = (CV & CV_HERMITE) != 0, HERMITE_SRC = HERMITE && (CV & CV_MRT);
    const Phys p = d.ph;
    const long long t = d.t0 + step_offset;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const int bsrc = (int)(t & 1);
    const GlobalLoader<T> L(d, bsrc);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        Pulled P;
        pull_node<HERMITE>(p, L, x, y, t, true, aux[n + k], aux[2 * n + k], P);
        float Fx, Fy, dQx = 0.0f, dQy = 0.0f;
        s2i4([&](int dx, int dy) { return aux_at(p, aux, x + dx, y + dy, true); }, Fx, Fy);
        contact_angle_adjust(d.wet, p, y, Fx, Fy);
        if (HERMITE_SRC) {
            float gx_, gy_;
            s2i4([&](int dx, int dy) { return aux_at(p, aux + 3 * n, x + dx, y + dy, false); }, dQx, gy_);
            s2i4([&](int dx, int dy) { return aux_at(p, aux + 4 * n, x + dx, y + dy, false); }, gx_, dQy);
        }
        float dr[9], db[9];
        float sm, sgx, sgy;
        collide_node<CV, SplitStore<T>::value>(p, P, aux[k], Fx, Fy, dQx, dQy, dr, db, sm, sgx, sgy);
        NodeStore<T>(d, p, bsrc ^ 1, x, y).put(P.rr, P.rb, dr, db, sm, sgx, sgy);
    }
}

template <typename T, int CV>
cudaError_t run_na(SimDesc &h, long long t, long n, float *aux, cudaStream_t st) {
    const long long nodes = (long long)h.ph.nx * h.ph.ny;
    const int g = (int)std::max<long long>(1, std::min<long long>((nodes + 255) / 256, 152LL * 16));
    h.t0 = t;
    for (long j = 0; j < n; j++) {
        k_na_moments<T, CV><<<g, 256, 0, st>>>(h, (int)j, aux);
        k_na_collide<T, CV><<<g, 256, 0, st>>>(h, (int)j, aux);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_na_v(SimDesc &h, long long t, long n, float *aux, cudaStream_t st) {
    switch (h.variant) {
    case 0: return run_na<T, 0>(h, t, n, aux, st);
    case CV_MRT: return run_na<T, CV_MRT>(h, t, n, aux, st);
    case CV_HERMITE: return run_na<T, CV_HERMITE>(h, t, n, aux, st);
    default: return run_na<T, CV_MRT | CV_HERMITE>(h, t, n, aux, st);
    }
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_params *p, int nx, int ny, void *state, size_t bytes, long long t,
                                       long n, void *cuda_stream) {
    char err[256] = "";
    lbm_status v = host_validate(nx, ny, p, err);
    if (v != LBM_OK) {
        host_set_global_error(err);
        return v;
    }
    if ((long long)nx * ny > NOALLOC_MAX_NODES) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: %d x %d = %lld nodes exceeds the static scratch limit of %lld nodes",
                 nx, ny, (long long)nx * ny, NOALLOC_MAX_NODES);
        host_set_global_error(err);
        return LBM_EINVAL;
    }
    const size_t need = lbm_bytes_required(nx, ny, p);
    if (!state || bytes < need || (reinterpret_cast<uintptr_t>(state) & 255) || t < 0 || n < 0) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: state NULL, unaligned or smaller than %zu bytes, or t / n < 0",
                 need);
        host_set_global_error(err);
        return bytes < need ? LBM_ENOMEM : LBM_EINVAL;
    }
    if (n == 0) return LBM_OK;
    float *aux = nullptr;
    lbm_status st = scratch_for_current_device(&aux, err);
    if (st != LBM_OK) {
        host_set_global_error(err);
        return st;
    }
    SimDesc h;
    host_fill_desc(h, nx, ny, p, state);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = p->storage == ST_F32 ? run_na_v<float>(h, t, n, aux, s)
                    : p->storage == ST_F16DEV ? run_na_v<__half>(h, t, n, aux, s)
                                              : run_na_v<__nv_bfloat16>(h, t, n, aux, s);
    if (e != cudaSuccess) {
        snprintf(err, sizeof(err), "lbm_step_noalloc: launch failed: %s", cudaGetErrorString(e));
        host_set_global_error(err);
        return LBM_ECUDA;
    }
    return LBM_OK;
}
