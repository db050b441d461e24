// lbm_device.cuh -- device-side building blocks of the GB300 colour-gradient LBM
// library: the per-simulation descriptor, storage codecs, the per-node operators
// of arXiv 1903.01168 Sec. 2 and the inline-PTX TMA / mbarrier helpers.
//
// Node arithmetic is done on the colour-blind distribution N_i = N^r_i + N^b_i.
// omega_eff, the Guo source and the perturbation are the same for both colours
// (Eq. (eq:singleCollision), Eq. (eq:singleCollisionMRT), Eq. (eq:perturbation)),
// so summing the two per-colour collisions gives one collision of N_i towards
// sum_k N^{k(e)}_i; only the moments rho_r, rho_b and the recolouring
// (Eq. (eq:recoloringOperator)) need the colours.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

enum : int { BC_PERIODIC = 0, BC_WALL = 1, BC_INOUT = 2 };
enum : int { ST_F32 = 0, ST_F16DEV = 1, ST_BF16DEV = 2 };

// Error bits written by kernels into the simulation's error word.
enum : int { ERR_TIMEOUT = 1, ERR_BADITEM = 2, ERR_ALIGN = 4 };

// Per-simulation descriptor, resident in device memory.  The tensor map comes
// first so that it keeps the 64-byte alignment TMA requires.
struct alignas(128) SimDesc {
    CUtensorMap tmap;          // 3D map over {pitch, ny, 36 planes} of this simulation
    void *pop;                 // [2 buffers][18 planes][ny][pitch] storage elements
    long long plane_stride;    // elements between planes = ny * pitch
    long long buf_stride;      // elements between the two buffers = 18 * plane_stride
    long long t0;              // time of the state when a launch chunk starts
    int nx, ny, pitch, ghost;  // ghost = columns kept on each side of a row
    int storage, collision, equilibrium, bc_x, bc_y;
    int inlet_mode, inlet_period_r, inlet_period_b, inlet_layer;
    int pad0;
    float inv_gamma;           // 1 / rho_r^0
    float phi_r[3], phi_b[3];  // rest weights phi^k by |c|^2 = 0, 1, 2
    float omega_r, omega_b, chi, eta, kappa, lam, nu, delta;
    float a_coef;              // A = a_coef * omega_eff, a_coef = 9 sigma / 4
    float beta, gx, gy, mrt_lambda, c7;
    float herm_r, herm_b;      // 3 (c_s^k)^2 - 1
    float q_r, q_b;            // 1.8 alpha_k - 0.8
    float cs2_r, cs2_b;        // (c_s^k)^2
    float u_in_r, u_in_b, p_out;
    float ref[18];             // deviation reference per plane (16-bit storage)
};

// One unit of work of a step launch: a strip of w <= W columns starting at x0,
// marching over rows [ya, yb) of simulation `sim`.
struct WorkItem {
    int sim;
    int x0;
    int w;
    int ya;
    int yb;
    int pad[3];
};

// ------------------------------------------------------------------ lattice
__host__ __device__ constexpr int CX(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int CY(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
__host__ __device__ constexpr int C2(int i) { return CX(i) * CX(i) + CY(i) * CY(i); }
__host__ __device__ constexpr float WT(int i) { return C2(i) == 0 ? 4.0f / 9.0f : (C2(i) == 1 ? 1.0f / 9.0f : 1.0f / 36.0f); }
__host__ __device__ constexpr float BP(int i) { return C2(i) == 0 ? -4.0f / 27.0f : (C2(i) == 1 ? 2.0f / 27.0f : 5.0f / 108.0f); }
// S2I4 weights xi_i, Eq. (eq:colorGradient)
__host__ __device__ constexpr float XI(int i) { return C2(i) == 0 ? 0.0f : (C2(i) == 1 ? 1.0f / 3.0f : 1.0f / 12.0f); }

static_assert(OPP(1) == 3 && OPP(2) == 4 && OPP(3) == 1 && OPP(4) == 2, "opposites");
static_assert(OPP(5) == 7 && OPP(6) == 8 && OPP(7) == 5 && OPP(8) == 6, "opposites");

// ---------------------------------------------------------------- storage
template <typename T> struct Codec;
template <> struct Codec<float> {
    static __device__ __forceinline__ float load(const float *p, float ref) { (void)ref; return *p; }
    static __device__ __forceinline__ float dec(float v, float ref) { (void)ref; return v; }
    static __device__ __forceinline__ float enc(float v, float ref) { (void)ref; return v; }
};
template <> struct Codec<__half> {
    static __device__ __forceinline__ float dec(__half v, float ref) { return ref + __half2float(v); }
    static __device__ __forceinline__ __half enc(float v, float ref) { return __float2half_rn(v - ref); }
};
template <> struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float dec(__nv_bfloat16 v, float ref) { return ref + __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float v, float ref) { return __float2bfloat16_rn(v - ref); }
};

// Address of element (buffer b, plane p, row y, column x) with x in [-ghost, nx + ghost).
template <typename T>
__device__ __forceinline__ T *pop_ptr(const SimDesc &d, int b, int p, int x, int y) {
    return reinterpret_cast<T *>(d.pop) + b * d.buf_stride + p * d.plane_stride + (long long)y * d.pitch + (x + d.ghost);
}

// Store the post-collision value of plane p at node (x, y) into buffer b; with
// periodic x the value is mirrored into the ghost columns of the other end.
template <typename T>
__device__ __forceinline__ void store_pop(const SimDesc &d, int b, int p, int x, int y, float v) {
    T e = Codec<T>::enc(v, d.ref[p]);
    T *row = reinterpret_cast<T *>(d.pop) + b * d.buf_stride + p * d.plane_stride + (long long)y * d.pitch + d.ghost;
    row[x] = e;
    if (d.bc_x == BC_PERIODIC) {
        if (x < d.ghost) row[d.nx + x] = e;
        if (x >= d.nx - d.ghost) row[x - d.nx] = e;
    }
}

// ------------------------------------------------------------ boundaries

// Red fraction of the phase injected at inlet row y at time t (Sec. 2.5): the
// inlet alternates red / blue segments in time, or is layered in y.
__device__ __forceinline__ float inlet_red_fraction(const SimDesc &d, int y, long long t) {
    if (d.inlet_mode == 1) return y < d.inlet_layer ? 1.0f : 0.0f;
    long long period = (long long)d.inlet_period_r + d.inlet_period_b;
    if (period <= 0) return 1.0f;
    return (t % period) < d.inlet_period_r ? 1.0f : 0.0f;
}

// Two-phase Zou-He velocity inlet on the west column (Sec. 2.5, the north inlet
// rotated by +90 degrees): unknowns 1, 5, 8, colour split by the injected phase.
__device__ __forceinline__ void zouhe_inlet(const SimDesc &d, float f_r, float (&nr)[9], float (&nb)[9]) {
    float n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const float f_b = 1.0f - f_r;
    const float Vx = f_r * d.u_in_r + f_b * d.u_in_b;
    const float rho = (n[0] + n[2] + n[4] + 2.0f * (n[3] + n[6] + n[7])) / (1.0f - Vx);
    const float H = d.equilibrium ? -rho * (f_r * d.herm_r + f_b * d.herm_b) * Vx * (1.0f / 3.0f) : 0.0f;
    const float n1 = n[3] + (2.0f / 3.0f) * rho * Vx + H;
    const float n5 = n[7] + 0.5f * (n[4] - n[2]) + rho * Vx * (1.0f / 6.0f) - 0.5f * H;
    const float n8 = n[6] + 0.5f * (n[2] - n[4]) + rho * Vx * (1.0f / 6.0f) - 0.5f * H;
    nr[1] = f_r * n1; nb[1] = f_b * n1;
    nr[5] = f_r * n5; nb[5] = f_b * n5;
    nr[8] = f_r * n8; nb[8] = f_b * n8;
}

// Two-phase Zou-He pressure outlet on the east column (the south outlet rotated
// by +90 degrees): unknowns 3, 6, 7; colour fraction from the known populations,
// rho_out = f_b p_out / (c_s^b)^2 + f_r p_out / (c_s^r)^2, v = -1 + (...)/rho_out.
__device__ __forceinline__ void zouhe_outlet(const SimDesc &d, float (&nr)[9], float (&nb)[9]) {
    const float kr = nr[0] + nr[1] + nr[2] + nr[4] + nr[5] + nr[8];
    const float kb = nb[0] + nb[1] + nb[2] + nb[4] + nb[5] + nb[8];
    const float a = kr * d.inv_gamma;
    const float psi = (a - kb) / (a + kb);
    const float f_r = 0.5f * (1.0f + psi), f_b = 1.0f - f_r;
    float n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const float rho = f_b * d.p_out / d.cs2_b + f_r * d.p_out / d.cs2_r;
    const float Vx = -1.0f + (n[0] + n[2] + n[4] + 2.0f * (n[1] + n[5] + n[8])) / rho;
    const float H = d.equilibrium ? rho * (f_r * d.herm_r + f_b * d.herm_b) * Vx * (1.0f / 3.0f) : 0.0f;
    const float n3 = n[1] - (2.0f / 3.0f) * rho * Vx + H;
    const float n6 = n[8] - 0.5f * (n[2] - n[4]) - rho * Vx * (1.0f / 6.0f) - 0.5f * H;
    const float n7 = n[5] + 0.5f * (n[2] - n[4]) - rho * Vx * (1.0f / 6.0f) - 0.5f * H;
    nr[3] = f_r * n3; nb[3] = f_b * n3;
    nr[6] = f_r * n6; nb[6] = f_b * n6;
    nr[7] = f_r * n7; nb[7] = f_b * n7;
}

// Pre-collision populations of node (x, y) at time t by pulling the stored
// post-collision values: Eq. (eq:subop4) with halfway bounce-back across walls
// (the node's own opposite population) and Zou-He on inlet / outlet columns.
// `ld(plane, xs, ys)` returns the decoded stored value of a source node: xs may
// be -1 or nx (ghost column), ys is one of y-1, y, y+1 NOT wrapped (the loader
// wraps periodic rows).  y itself may lie one row outside [0, ny) on a
// periodic lattice.
template <class Loader>
__device__ __forceinline__ void pull_node(const SimDesc &d, const Loader &ld, int x, int y, long long t,
                                          float (&nr)[9], float (&nb)[9]) {
    const bool wall_y = d.bc_y == BC_WALL;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const int ys = y - CY(i);
        const int xs = x - CX(i);
        if (wall_y && (ys < 0 || ys >= d.ny)) {
            nr[i] = ld(OPP(i), x, y);
            nb[i] = ld(9 + OPP(i), x, y);
        } else {
            nr[i] = ld(i, xs, ys);
            nb[i] = ld(9 + i, xs, ys);
        }
    }
    if (d.bc_x == BC_INOUT) {
        const int yw = y < 0 ? y + d.ny : (y >= d.ny ? y - d.ny : y);
        if (x == 0) zouhe_inlet(d, inlet_red_fraction(d, yw, t), nr, nb);
        else if (x == d.nx - 1) zouhe_outlet(d, nr, nb);
    }
}

// ------------------------------------------------------------ node operators

struct NodeMoments {
    float rr, rb, ux, uy, psi;
};

__device__ __forceinline__ NodeMoments node_moments(const SimDesc &d, const float (&nr)[9], const float (&nb)[9]) {
    float rr = 0.0f, rb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; i++) { rr += nr[i]; rb += nb[i]; }
    float n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const float rho = rr + rb;
    const float jx = (n[1] - n[3]) + (n[5] - n[7]) + (n[8] - n[6]);
    const float jy = (n[2] - n[4]) + (n[5] - n[7]) + (n[6] - n[8]);
    NodeMoments m;
    m.rr = rr;
    m.rb = rb;
    m.ux = jx / rho + 0.5f * d.gx;   // Guo half-force shift
    m.uy = jy / rho + 0.5f * d.gy;
    const float a = rr * d.inv_gamma;
    m.psi = (a - rb) / (a + rb);     // Eq. (eq:color_field)
    return m;
}

// omega_eff(psi), Sec. 2.1 interpolation.
__device__ __forceinline__ float omega_eff(const SimDesc &d, float psi) {
    if (psi > d.delta) return d.omega_r;
    if (psi > 0.0f) return d.chi + psi * (d.eta + d.kappa * psi);
    if (psi >= -d.delta) return d.chi + psi * (d.lam + d.nu * psi);
    return d.omega_b;
}

// Collision (BGK or MRT, Guo forcing, Hermite source), perturbation and
// recolouring of one node, in place on the pre-collision colour populations.
// F is the colour gradient; dQx = d_x(q u_x), dQy = d_y(q u_y) with
// q = sum_k (1.8 alpha_k - 0.8) rho_k (the colour sum of the Q^k derivatives).
__device__ __forceinline__ void collide_node(const SimDesc &d, float (&nr)[9], float (&nb)[9],
                                             float Fx, float Fy, float dQx, float dQy) {
    float rr = 0.0f, rb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; i++) { rr += nr[i]; rb += nb[i]; }
    float n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const float rho = rr + rb;
    const float inv_rho = 1.0f / rho;
    const float jx = (n[1] - n[3]) + (n[5] - n[7]) + (n[8] - n[6]);
    const float jy = (n[2] - n[4]) + (n[5] - n[7]) + (n[6] - n[8]);
    const float ux = jx * inv_rho + 0.5f * d.gx;
    const float uy = jy * inv_rho + 0.5f * d.gy;
    const float ca = rr * d.inv_gamma;
    const float psi = (ca - rb) / (ca + rb);
    const float w = omega_eff(d, psi);

    // colour-blind equilibrium sum_k N^{k(e)}_i (Eq. (eq:equilibrium) / (eq:equilibrium_hermite))
    const float usq = ux * ux + uy * uy;
    const float rest[3] = {rr * d.phi_r[0] + rb * d.phi_b[0], rr * d.phi_r[1] + rb * d.phi_b[1],
                           rr * d.phi_r[2] + rb * d.phi_b[2]};
    const float herm = d.equilibrium ? 0.5f * (rr * d.herm_r + rb * d.herm_b) : 0.0f;
    const float Gx = rho * d.gx, Gy = rho * d.gy;   // total body force
    float neq[9], src[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const float cu = CX(i) * ux + CY(i) * uy;
        float lin = rho * 3.0f * cu;
        if (C2(i) > 0) lin += 3.0f * cu * (3.0f * C2(i) - 4.0f) * herm;
        neq[i] = rest[C2(i)] + WT(i) * (lin + rho * (4.5f * cu * cu - 1.5f * usq));
        const float cG = CX(i) * Gx + CY(i) * Gy;
        src[i] = WT(i) * (3.0f * (cG - (ux * Gx + uy * Gy)) + 9.0f * cu * cG);
    }

    if (d.collision == 0) {
        const float fw = 1.0f - 0.5f * w;
#pragma unroll
        for (int i = 0; i < 9; i++) n[i] = n[i] - w * (n[i] - neq[i]) + fw * src[i];
    } else {
        float e[9];
#pragma unroll
        for (int i = 0; i < 9; i++) e[i] = n[i] - neq[i];
        // moments of the non-equilibrium part and of the source, rows of M
        // (appendix "Transformation matrices"); row 0 (mass) is zero for both.
        const float ax = e[1] + e[2] + e[3] + e[4], dg = e[5] + e[6] + e[7] + e[8];
        float m[9], ms[9];
        m[1] = -4.0f * e[0] - ax + 2.0f * dg;
        m[2] = 4.0f * e[0] - 2.0f * ax + dg;
        m[3] = e[1] - e[3] + e[5] - e[6] - e[7] + e[8];
        m[4] = -2.0f * (e[1] - e[3]) + e[5] - e[6] - e[7] + e[8];
        m[5] = e[2] - e[4] + e[5] + e[6] - e[7] - e[8];
        m[6] = -2.0f * (e[2] - e[4]) + e[5] + e[6] - e[7] - e[8];
        m[7] = e[1] - e[2] + e[3] - e[4];
        m[8] = e[5] - e[6] + e[7] - e[8];
        const float sx = src[1] + src[2] + src[3] + src[4], sd = src[5] + src[6] + src[7] + src[8];
        ms[1] = -4.0f * src[0] - sx + 2.0f * sd;
        ms[2] = 4.0f * src[0] - 2.0f * sx + sd;
        ms[3] = src[1] - src[3] + src[5] - src[6] - src[7] + src[8];
        ms[4] = -2.0f * (src[1] - src[3]) + src[5] - src[6] - src[7] + src[8];
        ms[5] = src[2] - src[4] + src[5] + src[6] - src[7] - src[8];
        ms[6] = -2.0f * (src[2] - src[4]) + src[5] + src[6] - src[7] - src[8];
        ms[7] = src[1] - src[2] + src[3] - src[4];
        ms[8] = src[5] - src[6] + src[7] - src[8];
        const float s1 = d.mrt_lambda * w;   // s_0 .. s_6
        float tm[9];
#pragma unroll
        for (int a = 1; a < 9; a++) {
            const float s = a < 7 ? s1 : w;  // s_7 = s_8 = omega_eff
            tm[a] = s * m[a] - (1.0f - 0.5f * s) * ms[a];
        }
        if (d.equilibrium) {
            // + U = M^-1 C, C_1 = 3 (1 - s_1/2)(dQx + dQy), C_7 = 3 (1 - w/2)(dQx + c7 dQy)
            tm[1] -= 3.0f * (1.0f - 0.5f * s1) * (dQx + dQy);
            tm[7] -= 3.0f * (1.0f - 0.5f * w) * (dQx + d.c7 * dQy);
        }
        // n -= M^-1 tm, M^-1 = (1/36) * integer matrix of the appendix (tm[0] = 0)
        const float k36 = 1.0f / 36.0f;
        const float b12 = -tm[1] - 2.0f * tm[2];
        const float d21 = 2.0f * tm[1] + tm[2];
        n[0] -= k36 * (-4.0f * tm[1] + 4.0f * tm[2]);
        n[1] -= k36 * (b12 + 6.0f * tm[3] - 6.0f * tm[4] + 9.0f * tm[7]);
        n[2] -= k36 * (b12 + 6.0f * tm[5] - 6.0f * tm[6] - 9.0f * tm[7]);
        n[3] -= k36 * (b12 - 6.0f * tm[3] + 6.0f * tm[4] + 9.0f * tm[7]);
        n[4] -= k36 * (b12 - 6.0f * tm[5] + 6.0f * tm[6] - 9.0f * tm[7]);
        n[5] -= k36 * (d21 + 6.0f * tm[3] + 3.0f * tm[4] + 6.0f * tm[5] + 3.0f * tm[6] + 9.0f * tm[8]);
        n[6] -= k36 * (d21 - 6.0f * tm[3] - 3.0f * tm[4] + 6.0f * tm[5] + 3.0f * tm[6] - 9.0f * tm[8]);
        n[7] -= k36 * (d21 - 6.0f * tm[3] - 3.0f * tm[4] - 6.0f * tm[5] - 3.0f * tm[6] + 9.0f * tm[8]);
        n[8] -= k36 * (d21 + 6.0f * tm[3] + 3.0f * tm[4] - 6.0f * tm[5] - 3.0f * tm[6] - 9.0f * tm[8]);
    }

    const float F2 = Fx * Fx + Fy * Fy;
    if (F2 > 0.0f) {
        // Eq. (eq:perturbation), one A/2 term per colour: A |F| [W (F.c)^2/|F|^2 - B]
        const float Fn = sqrtf(F2);
        const float invFn = 1.0f / Fn;
        const float A = d.a_coef * w;
        const float pa = A * invFn, pb = A * Fn;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const float Fc = CX(i) * Fx + CY(i) * Fy;
            n[i] += pa * WT(i) * Fc * Fc - pb * BP(i);
        }
        // Eq. (eq:recoloringOperator), cos(phi_i) = c_i.F / (|c_i| |F|)
        const float fr = rr * inv_rho;
        const float kk = d.beta * rr * rb * inv_rho * inv_rho * invFn;
        nr[0] = fr * n[0];
        nb[0] = n[0] - nr[0];
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const float Fc = CX(i) * Fx + CY(i) * Fy;
            const float inv_c = C2(i) == 1 ? 1.0f : 0.70710678118654752f;
            const float term = kk * Fc * inv_c * (C2(i) == 1 ? rest[1] : rest[2]);
            nr[i] = fr * n[i] + term;
            nb[i] = n[i] - nr[i];
        }
    } else {
        const float fr = rr * inv_rho;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            nr[i] = fr * n[i];
            nb[i] = n[i] - nr[i];
        }
    }
}

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tensormap_acquire(const void *tm) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Plain arrival (no transaction bytes): completes the phase of a count-1 barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit_cycles` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit_cycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > limit_cycles) return false;
    }
    return true;
}

// 3D tiled TMA load of one box into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace lbm
