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

// Per-simulation descriptor, resident in device memory.
//
// State layout ("density + deviation" form).  For each node and colour k the
// library stores rho_k (FP32) and the eight deviations
//     d^k_i = N^k_i - phi^k_i rho_k,  i = 1..8
// of the post-collision populations from the rest equilibrium of the node's
// own colour density (the storage type T is FP32, FP16 or BF16).  The rest
// deviation d^k_0 = -sum_{i>=1} d^k_i is implied, so every node's deviations
// sum to zero exactly, a colour that is absent is an exact zero, and all
// quantities the step manipulates are small where a phase is at rest.
//   rho planes: [2 buffers][ny][NS][pitch_r]                 float
//   dev planes: [2 buffers][ny][16 = colour * 8 + (i - 1)][pitch_d]   T
// NS = 2 (rho_r, rho_b) with FP32 deviations.  With 16-bit deviations NS = 5:
// rho_r, rho_b and the node scalars m, G_x, G_y of the split form below.
//
// Split form (16-bit storage).  After recolouring (Eq. (eq:recoloringOperator))
// a node's deviations are
//   d^r_i =  m dphi_c + t_i + (rho_r / rho) E_i,
//   d^b_i = -m dphi_c - t_i + (rho_b / rho) E_i,
// with m = rho_r rho_b / rho, dphi_c = phi^b_c - phi^r_c (c = |c_i|^2),
// t_i = (c_i . G) / |c_i| (rho_r phi^r_c + rho_b phi^b_c), G = beta m / rho F / |F|,
// and E_i the colour-blind non-rest part.  At an interface the first two terms
// are O(m) while E_i is small, so only the residuals r^k_i = d^k_i -+ (m dphi_c
// + t_i) are rounded to 16 bits and m, G stay FP32.  Any state is
// representable: the initial state stores m = G = 0 and r = d.
// i.e. the planes of one lattice row lie next to each other, so that reading
// or writing a row of a strip touches one contiguous stretch of memory per
// array (a planar [plane][ny] layout spreads it over 18 distant pages and
// streams markedly slower).  Rows keep `ghost` columns on each side (periodic
// copies in x).  The tensor
// maps come first so that they keep the 64-byte alignment TMA requires.
// Per-simulation constants the node operators read; kernels copy this struct
// into registers once.
struct Phys {
    int nx, ny, bc_x, bc_y;
    int inlet_mode, inlet_period_r, inlet_period_b, inlet_layer;
    float inv_gamma;           // 1 / rho_r^0
    float gx, gy;              // body acceleration
    float phi_r[3], phi_b[3];  // rest weights phi^k by |c|^2 = 0, 1, 2
    float dphi[3];             // phi_b - phi_r by |c|^2
    float omega_r, omega_b, chi, eta, kappa, lam, nu, delta;
    float a_coef;              // A = a_coef * omega_eff, a_coef = 9 sigma / 4
    float beta, mrt_lambda;
    float c7x, c7y;            // C^k_7 = (1 - omega_eff/2)(c7x d_xQ_x + c7y d_yQ_y)
    float herm_r, herm_b;      // 3 (c_s^k)^2 - 1
    float q_r, q_b;            // 1.8 alpha_k - 0.8
    float cs2_r, cs2_b;        // (c_s^k)^2
    float u_in_r, u_in_b, p_out;
};

// Wetting-wall parameters (free slip, static contact angle).  Kept out of Phys:
// the fused kernel, which holds Phys in registers, never runs such lattices.
struct Wetting {
    int slip;                  // walls: 0 no slip, 1 free slip
    int on;                    // 1: contact-angle adjustment of F next to the walls
    float cos_t, sin_t;        // of the contact angle (measured through the blue phase)
};

// Static contact angle (Sec. "Adjustment of the color gradient for static
// contact angles"): on the fluid rows next to a wall the direction of F is
// replaced by whichever of the two unit normals at angle theta from the wall
// normal n^s (into the fluid) is closer to it (n^s itself on a tie), |F| kept.
__device__ __forceinline__ void contact_angle_adjust(const Wetting &wt, const Phys &p, int y, float &Fx, float &Fy) {
    if (!wt.on || p.bc_y != BC_WALL || (y != 0 && y != p.ny - 1)) return;
    const float nsy = y == 0 ? 1.0f : -1.0f;   // n^s = (0, nsy)
    const float F2 = Fx * Fx + Fy * Fy;
    if (F2 == 0.0f) return;
    const float F = sqrtf(F2), ux = Fx / F, uy = Fy / F;
    // n1 = (-nsy sin, nsy cos), n2 = (nsy sin, nsy cos); compared by squared distance
    const float n1x = -nsy * wt.sin_t, n2x = nsy * wt.sin_t, ny_ = nsy * wt.cos_t;
    const float d1 = (ux - n1x) * (ux - n1x) + (uy - ny_) * (uy - ny_);
    const float d2 = (ux - n2x) * (ux - n2x) + (uy - ny_) * (uy - ny_);
    if (d1 < d2) {
        Fx = F * n1x;
        Fy = F * ny_;
    } else if (d1 > d2) {
        Fx = F * n2x;
        Fy = F * ny_;
    } else {
        Fx = 0.0f;
        Fy = F * nsy;
    }
}

struct alignas(128) SimDesc {
    CUtensorMap tmap_rho;      // 2D {pitch_r, 2 * ny * 2} box {W + 2 halo, 2}: one row's 2 planes
    CUtensorMap tmap_dev;      // 2D {pitch_d, 2 * ny * 16} box {W + 2 halo, 16}: one row's 16 planes
    float *rho;
    void *dev;
    long long rho_plane, rho_row, rho_buf;   // element strides of a plane, a row, a buffer
    long long dev_plane, dev_row, dev_buf;
    long long t0;              // time of the state when a launch chunk starts
    long long t_end;           // steps that would start at t >= t_end are skipped
    int pitch_r, pitch_d, ghost;
    int storage, variant;      // variant: bit 0 MRT, bit 1 Hermite equilibrium
    Phys ph;
    Wetting wet;
};

// Scratch field of the two-pass path: aux[5][ny][nx] = psi, rho_r, rho_b, q u_x, q u_y.
constexpr int AUX_FIELDS = 5;

// Compile-time variants of the step kernels: bit 0 = MRT (else BGK), bit 1 =
// Hermite equilibrium (with the U^k source when combined with MRT), bit 2 =
// wetting walls (free-slip links and the contact-angle adjustment of F; without
// it walls are no-slip and the fused kernel keeps fewer registers), bit 3 =
// inlet / outlet columns in x (else periodic in x).  The fused kernel of a
// periodic lattice carries no open-column code: its mere presence in the loop
// cost the periodic sweep 2 %.
constexpr int CV_MRT = 1, CV_HERMITE = 2, CV_WET = 4, CV_OPEN = 8;
constexpr int N_VARIANTS = 16;
// Launch flag of the fused kernel: the next step may launch as soon as this one
// starts (plans of equal pieces, one launch per step).
constexpr int FUSED_EARLY_NEXT = 1;

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
    static __device__ __forceinline__ float dec(float v) { return v; }
    static __device__ __forceinline__ float enc(float v) { return v; }
};
template <> struct Codec<__half> {
    static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half enc(float v) { return __float2half_rn(v); }
};
template <> struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
};

// 16-bit deviations are stored in the split form; FP32 ones directly.
template <typename T> struct SplitStore { static constexpr bool value = sizeof(T) == 2; };
template <typename T> struct ScalarPlanes { static constexpr int value = SplitStore<T>::value ? 5 : 2; };

// Constants of the split form that a loader needs (by |c|^2 = 1, 2).
struct SplitC {
    float phr1, phr2, phb1, phb2, dph1, dph2;
};

__device__ __forceinline__ SplitC split_consts(const Phys &p) {
    return SplitC{p.phi_r[1], p.phi_r[2], p.phi_b[1], p.phi_b[2], p.dphi[1], p.dphi[2]};
}

// Shift of the split form for direction i (added to red, subtracted from blue):
// m dphi_c + (c_i . G) / |c_i| (rho_r phi^r_c + rho_b phi^b_c).  Every operation is
// rounded explicitly, so that a node's deviation decodes to the same value
// wherever it is read (the puller and the node itself), which keeps the colour
// mass exchanged between nodes balanced.
__device__ __forceinline__ float split_shift(const SplitC &q, int i, float rr, float rb, float m, float gx,
                                             float gy) {
    const bool axis = C2(i) == 1;
    const float rest = __fmaf_rn(rr, axis ? q.phr1 : q.phr2, __fmul_rn(rb, axis ? q.phb1 : q.phb2));
    float gc;
    if (CY(i) == 0) gc = CX(i) > 0 ? gx : -gx;
    else if (CX(i) == 0) gc = CY(i) > 0 ? gy : -gy;
    else gc = __fadd_rn(CX(i) > 0 ? gx : -gx, CY(i) > 0 ? gy : -gy);
    const float inv_c = axis ? 1.0f : 0.70710678118654752f;
    return __fadd_rn(__fmul_rn(m, axis ? q.dph1 : q.dph2), __fmul_rn(__fmul_rn(gc, inv_c), rest));
}

__device__ __forceinline__ float phi_k(const Phys &p, int k, int c2) { return k == 0 ? p.phi_r[c2] : p.phi_b[c2]; }

// Where node (x, y)'s post-collision state goes in buffer b: row pointers of
// the two density planes and of deviation plane 0, the deviation plane stride,
// and the ghost column that mirrors x on a periodic lattice (or INT_MIN).
template <typename T>
struct NodeStore {
    float *rho;        // &rho[b][0][y][x]
    long long rho_plane;
    T *dev;            // &dev[b][0][y][x]
    long long dev_plane;
    int mirror_r;      // +nx when x also lives in the right ghost columns, else 0
    int mirror_l;      // -nx when x also lives in the left ghost columns, else 0

    __device__ __forceinline__ NodeStore(const SimDesc &d, const Phys &p, int b, int x, int y) {
        rho = d.rho + b * d.rho_buf + (long long)y * d.rho_row + d.ghost + x;
        rho_plane = d.rho_plane;
        dev = reinterpret_cast<T *>(d.dev) + b * d.dev_buf + (long long)y * d.dev_row + d.ghost + x;
        dev_plane = d.dev_plane;
        const bool per = p.bc_x == BC_PERIODIC;
        mirror_r = (per && x < d.ghost) ? p.nx : 0;
        mirror_l = (per && x >= p.nx - d.ghost) ? -p.nx : 0;   // both on lattices narrower than 2 ghosts
    }

    __device__ __forceinline__ void store_at(int off, float rr, float rb, const float (&dr)[9],
                                             const float (&db)[9], float m, float gx, float gy) const {
        rho[off] = rr;
        rho[rho_plane + off] = rb;
        if (SplitStore<T>::value) {
            rho[2 * rho_plane + off] = m;
            rho[3 * rho_plane + off] = gx;
            rho[4 * rho_plane + off] = gy;
        }
#pragma unroll
        for (int i = 1; i < 9; i++) {
            dev[(i - 1) * dev_plane + off] = Codec<T>::enc(dr[i]);
            dev[(i + 7) * dev_plane + off] = Codec<T>::enc(db[i]);
        }
    }

    // Post-collision state: with 16-bit storage dr, db are the split-form
    // residuals and (m, gx, gy) its node scalars; with FP32 storage dr, db are
    // the deviations and the scalars are ignored.
    __device__ __forceinline__ void put(float rr, float rb, const float (&dr)[9], const float (&db)[9], float m,
                                        float gx, float gy) const {
        store_at(0, rr, rb, dr, db, m, gx, gy);
        if (mirror_r) store_at(mirror_r, rr, rb, dr, db, m, gx, gy);
        if (mirror_l) store_at(mirror_l, rr, rb, dr, db, m, gx, gy);
    }

    // Any state given by its deviations (split form with m = G = 0).
    __device__ __forceinline__ void store(float rr, float rb, const float (&dr)[9], const float (&db)[9]) const {
        put(rr, rb, dr, db, 0.0f, 0.0f, 0.0f);
    }
};

// ------------------------------------------------------------ boundaries

// Red fraction of the phase injected at inlet row y at time t (Sec. 2.5): the
// inlet alternates red / blue segments in time, or is layered in y.
__device__ __forceinline__ float inlet_red_fraction(const Phys &p, int y, long long t) {
    if (p.inlet_mode == 1) return y < p.inlet_layer ? 1.0f : 0.0f;
    const int period = p.inlet_period_r + p.inlet_period_b;
    if (period <= 0) return 1.0f;
    return (int)(t % period) < p.inlet_period_r ? 1.0f : 0.0f;
}

// Two-phase Zou-He velocity inlet on the west column (Sec. 2.5, the north inlet
// rotated by +90 degrees): unknowns 1, 5, 8, colour split by the injected phase.
// R is the arithmetic type (FP32 on the step path, FP64 for state export).
template <typename R>
__device__ __forceinline__ void zouhe_inlet(const Phys &p, bool hermite, R f_r, R (&nr)[9], R (&nb)[9]) {
    R n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const R f_b = R(1) - f_r;
    const R Vx = f_r * R(p.u_in_r) + f_b * R(p.u_in_b);
    const R rho = (n[0] + n[2] + n[4] + R(2) * (n[3] + n[6] + n[7])) / (R(1) - Vx);
    const R H = hermite ? -rho * (f_r * R(p.herm_r) + f_b * R(p.herm_b)) * Vx / R(3) : R(0);
    const R n1 = n[3] + (R(2) / R(3)) * rho * Vx + H;
    const R n5 = n[7] + R(0.5) * (n[4] - n[2]) + rho * Vx / R(6) - R(0.5) * H;
    const R n8 = n[6] + R(0.5) * (n[2] - n[4]) + rho * Vx / R(6) - R(0.5) * H;
    nr[1] = f_r * n1; nb[1] = f_b * n1;
    nr[5] = f_r * n5; nb[5] = f_b * n5;
    nr[8] = f_r * n8; nb[8] = f_b * n8;
}

// Two-phase Zou-He pressure outlet on the east column (the south outlet rotated
// by +90 degrees): unknowns 3, 6, 7; colour fraction from the known populations,
// rho_out = f_b p_out / (c_s^b)^2 + f_r p_out / (c_s^r)^2, v = -1 + (...)/rho_out.
template <typename R>
__device__ __forceinline__ void zouhe_outlet(const Phys &p, bool hermite, R (&nr)[9], R (&nb)[9]) {
    const R kr = nr[0] + nr[1] + nr[2] + nr[4] + nr[5] + nr[8];
    const R kb = nb[0] + nb[1] + nb[2] + nb[4] + nb[5] + nb[8];
    const R a = kr * R(p.inv_gamma);
    const R psi = (a - kb) / (a + kb);
    const R f_r = R(0.5) * (R(1) + psi), f_b = R(1) - f_r;
    R n[9];
#pragma unroll
    for (int i = 0; i < 9; i++) n[i] = nr[i] + nb[i];
    const R rho = f_b * R(p.p_out) / R(p.cs2_b) + f_r * R(p.p_out) / R(p.cs2_r);
    // v = -1 + S / rho written as (S - rho) / rho
    const R S = n[0] + n[2] + n[4] + R(2) * (n[1] + n[5] + n[8]);
    const R Vx = (S - rho) / rho;
    const R H = hermite ? rho * (f_r * R(p.herm_r) + f_b * R(p.herm_b)) * Vx / R(3) : R(0);
    const R n3 = n[1] - (R(2) / R(3)) * rho * Vx + H;
    const R n6 = n[8] - R(0.5) * (n[2] - n[4]) - rho * Vx / R(6) - R(0.5) * H;
    const R n7 = n[5] + R(0.5) * (n[2] - n[4]) - rho * Vx / R(6) - R(0.5) * H;
    nr[3] = f_r * n3; nb[3] = f_b * n3;
    nr[6] = f_r * n6; nb[6] = f_b * n6;
    nr[7] = f_r * n7; nb[7] = f_b * n7;
}

// Result of pulling one node: its new colour densities and the colour-blind
// non-rest part e_i = N_i - R_i of its pre-collision populations, where
// R_i = rho_r phi^r_i + rho_b phi^b_i is the rest equilibrium of the node.
struct Pulled {
    float rr, rb;
    float e[9];
};

// Where direction i of node (x, y) pulls from: the node x - c_i, or across a
// wall (Sec. 2.5) the node itself in direction OPP(i) (no slip, halfway
// bounce-back), or with free slip the node x - (c_ix, 0) of the same row in the
// mirrored direction (the population travels on along the wall).  Free slip
// falls back to bounce-back where that node is outside an open lattice (the
// Zou-He columns then overwrite the link).
struct Link {
    int xs, ys, ii;
    bool self;   // the source is the node itself
};

__host__ __device__ constexpr int MIRY(int i) { return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i; }

// Link sets a pull is compiled for: no-slip walls only (the fused kernel, which
// never runs lattices with wetting walls: their extra logic would cost the hot
// loop registers on every row), or no-slip and free-slip walls (all others).
constexpr int LINKS_NOSLIP = 1, LINKS_ALL = 2;

template <int LINKS>
__device__ __forceinline__ Link link_of(const Phys &p, int slip, int i, int x, int y, bool bottom, bool top) {
    const bool wall = (CY(i) > 0 && bottom) || (CY(i) < 0 && top);
    if (!wall) return Link{x - CX(i), y - CY(i), i, false};
    if (LINKS == LINKS_NOSLIP) return Link{x, y, OPP(i), true};
    const int xs = x - CX(i);
    if (slip && (p.bc_x == BC_PERIODIC || (xs >= 0 && xs < p.nx))) return Link{xs, y, MIRY(i), CX(i) == 0};
    return Link{x, y, OPP(i), true};
}

// Pull the pre-collision populations of node (x, y) at time t (Eq. (eq:subop4)):
// N^k_i(x) = phi^k_i rho_k(x - c_i) + d^k_i(x - c_i), with halfway bounce-back
// across walls (the node's own opposite population) and two-phase Zou-He on
// the inlet / outlet columns (Sec. 2.5).  The loader provides
//   ld.rho(k, xs, ys), ld.dev(k, i, xs, ys)   (i = 1..8)
// of a source node; xs may be -1 or nx (ghost column); ys is one of y-1, y, y+1
// NOT wrapped (the loader wraps periodic rows); y itself may lie one row
// outside [0, ny) on a periodic lattice.  With have_rho the node's new colour
// densities are already known (rr_new, rb_new) and are not recomputed.
// pull_node for the split form (16-bit storage), away from open columns.  The
// loader gives the stored residual r^k_i and the shift h_i of the split form
// (d^r_i = r^r_i + h_i, d^b_i = r^b_i - h_i).  The shifts cancel in the colour-blind
// parts e_i, and enter the colour densities only through one sum per node,
//   sum_i h_i(source of i) - sum_i h_i(x),
// where the node's own sum is 4 m (dphi_1 + dphi_2) (the flux parts cancel in
// opposite pairs).
template <int LINKS, class Loader>
__device__ __forceinline__ void pull_node_split(const Phys &p, const Loader &ld, int x, int y, bool have_rho,
                                                float rr_new, float rb_new, Pulled &P) {
    const bool wall_y = p.bc_y == BC_WALL;
    const bool bottom = wall_y && y == 0, top = wall_y && y == p.ny - 1;
    float own[2];
    own[0] = ld.rho(0, x, y);
    own[1] = ld.rho(1, x, y);
    // one pass over the links, keeping per direction only
    //   T_i = sum_k phi^k_i (s^k_i - rho_k(x)) + r^r_i + r^b_i
    // (small terms) and the colour sums; then e_i = T_i - sum_k phi^k_i (rho'_k - rho_k(x))
    float T[9], acc[2] = {0.0f, 0.0f}, hsum = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        const Link lk = link_of<LINKS>(p, ld.slip, i, x, y, bottom, top);
        const int xs = lk.xs, ys = lk.ys, ii = lk.ii;
        float ti = 0.0f;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float ds = (lk.self ? own[k] : ld.rho(k, xs, ys)) - own[k];
            const float r = ld.res(k, ii, xs, ys);
            const float f = phi_k(p, k, C2(i)) * ds;
            acc[k] += f + (r - ld.res(k, i, x, y));
            ti += f + r;
        }
        T[i] = ti;
        hsum += ld.shift(ii, xs, ys);
    }
    float rnew[2];
    if (have_rho) {
        rnew[0] = rr_new;
        rnew[1] = rb_new;
    } else {
        const float dh = hsum - ld.own_shift_sum(x, y);
        rnew[0] = own[0] + (acc[0] + dh);
        rnew[1] = own[1] + (acc[1] - dh);
    }
    P.rr = rnew[0];
    P.rb = rnew[1];
    const float dr = rnew[0] - own[0], db = rnew[1] - own[1];
    float e0 = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        P.e[i] = T[i] - (p.phi_r[C2(i)] * dr + p.phi_b[C2(i)] * db);
        e0 += P.e[i];
    }
    P.e[0] = -e0;
}

template <bool HERMITE, int LINKS, class Loader>
__device__ __forceinline__ void pull_node_rows(const Phys &p, const Loader &ld, int x, int y, long long t,
                                               bool have_rho, float rr_new, float rb_new, Pulled &P) {
    const bool wall_y = p.bc_y == BC_WALL;
    const bool open_col = p.bc_x == BC_INOUT && (x == 0 || x == p.nx - 1);
    const bool bottom = wall_y && y == 0, top = wall_y && y == p.ny - 1;
    if (Loader::SPLIT && !open_col) {
        pull_node_split<LINKS>(p, ld, x, y, have_rho, rr_new, rb_new, P);
        return;
    }
    float s[2][9], dl[2][9], own_rho[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        own_rho[k] = ld.rho(k, x, y);
#pragma unroll
        for (int i = 1; i < 9; i++) {
            if (LINKS == LINKS_NOSLIP) {
                // constant plane offsets in both branches (no run-time direction index)
                const bool bounce = (CY(i) > 0 && bottom) || (CY(i) < 0 && top);
                if (bounce) {
                    s[k][i] = own_rho[k];
                    dl[k][i] = ld.dev(k, OPP(i), x, y);
                } else {
                    s[k][i] = ld.rho(k, x - CX(i), y - CY(i));
                    dl[k][i] = ld.dev(k, i, x - CX(i), y - CY(i));
                }
            } else {
                const Link lk = link_of<LINKS>(p, ld.slip, i, x, y, bottom, top);
                s[k][i] = lk.self ? own_rho[k] : ld.rho(k, lk.xs, lk.ys);
                dl[k][i] = ld.dev(k, lk.ii, lk.xs, lk.ys);
            }
        }
    }
    if (!open_col) {
        float rnew[2];
        if (have_rho) {
            rnew[0] = rr_new;
            rnew[1] = rb_new;
        } else {
#pragma unroll
            for (int k = 0; k < 2; k++) {
                float acc = 0.0f;
#pragma unroll
                for (int i = 1; i < 9; i++)
                    acc += phi_k(p, k, C2(i)) * (s[k][i] - own_rho[k]) + (dl[k][i] - ld.dev(k, i, x, y));
                rnew[k] = own_rho[k] + acc;
            }
        }
        P.rr = rnew[0];
        P.rb = rnew[1];
        float e0 = 0.0f;
#pragma unroll
        for (int i = 1; i < 9; i++) {
            P.e[i] = p.phi_r[C2(i)] * (s[0][i] - rnew[0]) + dl[0][i] + p.phi_b[C2(i)] * (s[1][i] - rnew[1]) + dl[1][i];
            e0 += P.e[i];
        }
        P.e[0] = -e0;
        return;
    }
    // open column: full populations, Zou-He, then moments
    float nr[9], nb[9];
    {
        float sr = 0.0f, sb = 0.0f;
#pragma unroll
        for (int i = 1; i < 9; i++) {
            nr[i] = p.phi_r[C2(i)] * s[0][i] + dl[0][i];
            nb[i] = p.phi_b[C2(i)] * s[1][i] + dl[1][i];
            sr += ld.dev(0, i, x, y);
            sb += ld.dev(1, i, x, y);
        }
        nr[0] = p.phi_r[0] * own_rho[0] - sr;
        nb[0] = p.phi_b[0] * own_rho[1] - sb;
    }
    const int yw = y < 0 ? y + p.ny : (y >= p.ny ? y - p.ny : y);
    if (x == 0) zouhe_inlet<float>(p, HERMITE, inlet_red_fraction(p, yw, t), nr, nb);
    else zouhe_outlet<float>(p, HERMITE, nr, nb);
    float rr = 0.0f, rb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; i++) { rr += nr[i]; rb += nb[i]; }
    P.rr = rr;
    P.rb = rb;
#pragma unroll
    for (int i = 0; i < 9; i++) P.e[i] = (nr[i] + nb[i]) - (rr * p.phi_r[C2(i)] + rb * p.phi_b[C2(i)]);
}

// Pull with every kind of wall link.
template <bool HERMITE, class Loader>
__device__ __forceinline__ void pull_node(const Phys &p, const Loader &ld, int x, int y, long long t,
                                          bool have_rho, float rr_new, float rb_new, Pulled &P) {
    pull_node_rows<HERMITE, LINKS_ALL>(p, ld, x, y, t, have_rho, rr_new, rb_new, P);
}

// Moments of the pulled node (x, y) without forming its populations: the new
// colour densities
//   rho_k' = rho_k(x) + sum_{i>=1} [phi^k_i (s^k_i - rho_k(x)) + delta^k_i - d^k_i(x)]
// (s, delta: density and deviation of the source of direction i) and, with
// NEED_J, the momentum sum_i c_i N_i summed over opposite pairs.  Open columns
// take the full pull.
template <bool HERMITE, bool NEED_J, int LINKS, class Loader>
__device__ __forceinline__ void pull_moments_rows(const Phys &p, const Loader &ld, int x, int y, long long t,
                                                  float &rr, float &rb, float &jx, float &jy) {
    if (p.bc_x == BC_INOUT && (x == 0 || x == p.nx - 1)) {
        Pulled P;
        pull_node<HERMITE>(p, ld, x, y, t, false, 0.0f, 0.0f, P);
        rr = P.rr;
        rb = P.rb;
        jx = (P.e[1] - P.e[3]) + (P.e[5] - P.e[7]) + (P.e[8] - P.e[6]);
        jy = (P.e[2] - P.e[4]) + (P.e[5] - P.e[7]) + (P.e[6] - P.e[8]);
        return;
    }
    const bool wall_y = p.bc_y == BC_WALL;
    const bool bottom = wall_y && y == 0, top = wall_y && y == p.ny - 1;
    if (Loader::SPLIT) {
        // split form: residual differences per colour, one shift sum for both
        // (as in pull_node_split)
        float n[2][9], acc[2], own[2];
        float hsum = 0.0f;
        own[0] = ld.rho(0, x, y);
        own[1] = ld.rho(1, x, y);
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const Link lk = link_of<LINKS>(p, ld.slip, i, x, y, bottom, top);
            const int xs = lk.xs, ys = lk.ys, ii = lk.ii;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const float sv = lk.self ? own[k] : ld.rho(k, xs, ys);
                n[k][i] = phi_k(p, k, C2(i)) * (sv - own[k]) + ld.res(k, ii, xs, ys);
            }
            hsum += ld.shift(ii, xs, ys);
        }
        const float dh = hsum - ld.own_shift_sum(x, y);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            float a = 0.0f;
#pragma unroll
            for (int i = 1; i < 9; i++) a += n[k][i] - ld.res(k, i, x, y);
            acc[k] = own[k] + (k == 0 ? a + dh : a - dh);
        }
        rr = acc[0];
        rb = acc[1];
        if (NEED_J) {
            // colour-blind momentum: the shifts cancel between the colours
            float m[9];
#pragma unroll
            for (int i = 1; i < 9; i++) m[i] = n[0][i] + n[1][i];
            jx = (m[1] - m[3]) + (m[5] - m[7]) + (m[8] - m[6]);
            jy = (m[2] - m[4]) + (m[5] - m[7]) + (m[6] - m[8]);
        } else {
            jx = jy = 0.0f;
        }
        return;
    }
    float n[2][9];   // n[k][i] = N^k_i - phi^k_i rho_k(x) for i >= 1 (small)
    float acc[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float own = ld.rho(k, x, y);
        float a = 0.0f;
#pragma unroll
        for (int i = 1; i < 9; i++) {
            float sv, dv;
            if (LINKS == LINKS_NOSLIP) {
                const bool bounce = (CY(i) > 0 && bottom) || (CY(i) < 0 && top);
                if (bounce) {
                    sv = own;
                    dv = ld.dev(k, OPP(i), x, y);
                } else {
                    sv = ld.rho(k, x - CX(i), y - CY(i));
                    dv = ld.dev(k, i, x - CX(i), y - CY(i));
                }
            } else {
                const Link lk = link_of<LINKS>(p, ld.slip, i, x, y, bottom, top);
                sv = lk.self ? own : ld.rho(k, lk.xs, lk.ys);
                dv = ld.dev(k, lk.ii, lk.xs, lk.ys);
            }
            n[k][i] = phi_k(p, k, C2(i)) * (sv - own) + dv;
            a += n[k][i] - ld.dev(k, i, x, y);
        }
        acc[k] = own + a;
    }
    rr = acc[0];
    rb = acc[1];
    if (NEED_J) {
        float m[9];
#pragma unroll
        for (int i = 1; i < 9; i++) m[i] = n[0][i] + n[1][i];
        jx = (m[1] - m[3]) + (m[5] - m[7]) + (m[8] - m[6]);
        jy = (m[2] - m[4]) + (m[5] - m[7]) + (m[6] - m[8]);
    } else {
        jx = jy = 0.0f;
    }
}

template <bool HERMITE, bool NEED_J, class Loader>
__device__ __forceinline__ void pull_moments(const Phys &p, const Loader &ld, int x, int y, long long t,
                                             float &rr, float &rb, float &jx, float &jy) {
    pull_moments_rows<HERMITE, NEED_J, LINKS_ALL>(p, ld, x, y, t, rr, rb, jx, jy);
}

// Pre-collision populations of both colours of node (x, y) at time t in FP64
// (boundary conditions included), for state export.
template <bool HERMITE, class Loader>
__device__ __forceinline__ void pull_populations(const Phys &p, const Loader &ld, int x, int y, long long t,
                                                 double (&nr)[9], double (&nb)[9]) {
    const bool wall_y = p.bc_y == BC_WALL;
    const bool bottom = wall_y && y == 0, top = wall_y && y == p.ny - 1;
    double sr = 0.0, sb = 0.0;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        const Link lk = link_of<LINKS_ALL>(p, ld.slip, i, x, y, bottom, top);
        const int xs = lk.xs, ys = lk.ys, ii = lk.ii;
        nr[i] = (double)p.phi_r[C2(i)] * ld.rho(0, xs, ys) + ld.dev(0, ii, xs, ys);
        nb[i] = (double)p.phi_b[C2(i)] * ld.rho(1, xs, ys) + ld.dev(1, ii, xs, ys);
        sr += ld.dev(0, i, x, y);
        sb += ld.dev(1, i, x, y);
    }
    nr[0] = (double)p.phi_r[0] * ld.rho(0, x, y) - sr;
    nb[0] = (double)p.phi_b[0] * ld.rho(1, x, y) - sb;
    if (p.bc_x == BC_INOUT && (x == 0 || x == p.nx - 1)) {
        if (x == 0) zouhe_inlet<double>(p, HERMITE, inlet_red_fraction(p, y, t), nr, nb);
        else zouhe_outlet<double>(p, HERMITE, nr, nb);
    }
}

// ------------------------------------------------------------ node operators

struct NodeMoments {
    float rr, rb, ux, uy, psi;
};

// Eq. (eq:color_field): psi = (rho_r / rho_r^0 - rho_b / rho_b^0) / (rho_r / rho_r^0 + rho_b / rho_b^0).
__device__ __forceinline__ float colour_field(const Phys &p, float rr, float rb) {
    const float a = rr * p.inv_gamma;
    return (a - rb) / (a + rb);   // IEEE division: exactly +-1 in a pure phase
}

__device__ __forceinline__ NodeMoments node_moments(const Phys &p, const Pulled &P) {
    const float rho = P.rr + P.rb;
    const float jx = (P.e[1] - P.e[3]) + (P.e[5] - P.e[7]) + (P.e[8] - P.e[6]);
    const float jy = (P.e[2] - P.e[4]) + (P.e[5] - P.e[7]) + (P.e[6] - P.e[8]);
    NodeMoments m;
    m.rr = P.rr;
    m.rb = P.rb;
    m.ux = jx / rho + 0.5f * p.gx;   // Guo half-force shift
    m.uy = jy / rho + 0.5f * p.gy;
    m.psi = colour_field(p, P.rr, P.rb);
    return m;
}

// omega_eff(psi), Sec. 2.1 interpolation.
__device__ __forceinline__ float omega_eff(const Phys &p, float psi) {
    if (psi > p.delta) return p.omega_r;
    if (psi > 0.0f) return p.chi + psi * (p.eta + p.kappa * psi);
    if (psi >= -p.delta) return p.chi + psi * (p.lam + p.nu * psi);
    return p.omega_b;
}

// Collision (BGK or MRT, Guo forcing, Hermite source), perturbation and
// recolouring of one pulled node.  F is the colour gradient; dQx = d_x(q u_x),
// dQy = d_y(q u_y) with q = sum_k (1.8 alpha_k - 0.8) rho_k.  Outputs the
// post-collision deviations dr[1..8], db[1..8] of the stored state (the colour
// densities are unchanged by the step's collision part).
template <int CV, bool SPLIT = false>
__device__ __forceinline__ void collide_node(const Phys &p, const Pulled &P, float psi, float Fx, float Fy,
                                             float dQx, float dQy, float (&dr)[9], float (&db)[9], float &o_m,
                                             float &o_gx, float &o_gy) {
    constexpr bool MRT = (CV & CV_MRT) != 0, HERMITE = (CV & CV_HERMITE) != 0;
    const float rr = P.rr, rb = P.rb;
    const float rho = rr + rb;
    const float inv_rho = __fdividef(1.0f, rho);
    float e[9];
#pragma unroll
    for (int i = 0; i < 9; i++) e[i] = P.e[i];
    const float jx = (e[1] - e[3]) + (e[5] - e[7]) + (e[8] - e[6]);
    const float jy = (e[2] - e[4]) + (e[5] - e[7]) + (e[6] - e[8]);
    const float ux = jx * inv_rho + 0.5f * p.gx;
    const float uy = jy * inv_rho + 0.5f * p.gy;
    const float w = omega_eff(p, psi);
    const bool force = (p.gx != 0.0f) || (p.gy != 0.0f);

    // velocity part of the colour-blind equilibrium, sum_k N^{k(e)}_i - R_i
    // (Eq. (eq:equilibrium) / (eq:equilibrium_hermite)), and the Guo source,
    // formed per opposite pair (i, OPP(i)) from the part even in c_i and the
    // part odd in c_i (c_OPP(i) = -c_i)
    const float usq = ux * ux + uy * uy;
    const float herm = HERMITE ? 0.5f * (rr * p.herm_r + rb * p.herm_b) : 0.0f;
    const float Gx = rho * p.gx, Gy = rho * p.gy;
    const float uG = ux * Gx + uy * Gy;
    float weq[9], src[9];
    weq[0] = WT(0) * rho * (-1.5f * usq);
    src[0] = 0.0f;
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int j = OPP(i);
        const float cu = CX(i) * ux + CY(i) * uy;
        const float even = WT(i) * rho * (4.5f * cu * cu - 1.5f * usq);
        float odd = WT(i) * 3.0f * rho * cu;
        if (HERMITE) odd += WT(i) * 3.0f * cu * (3.0f * C2(i) - 4.0f) * herm;
        weq[i] = even + odd;
        weq[j] = even - odd;
        src[i] = src[j] = 0.0f;
    }
    if (force) {
        src[0] = WT(0) * (-3.0f * uG);
#pragma unroll
        for (int i : {1, 2, 5, 6}) {
            const int j = OPP(i);
            const float cu = CX(i) * ux + CY(i) * uy;
            const float cG = CX(i) * Gx + CY(i) * Gy;
            const float even = WT(i) * (9.0f * cu * cG - 3.0f * uG);
            const float odd = WT(i) * 3.0f * cG;
            src[i] = even + odd;
            src[j] = even - odd;
        }
    }

    if (!MRT) {
        const float fw = 1.0f - 0.5f * w;
#pragma unroll
        for (int i = 1; i < 9; i++) e[i] = e[i] - w * (e[i] - weq[i]) + fw * src[i];
    } else {
        float q[9];
#pragma unroll
        for (int i = 0; i < 9; i++) q[i] = e[i] - weq[i];
        // moments of the non-equilibrium part and of the source, rows of M
        // (appendix "Transformation matrices"); row 0 (mass) is zero for both.
        const float ax = q[1] + q[2] + q[3] + q[4], dg = q[5] + q[6] + q[7] + q[8];
        float m[9], ms[9];
        m[1] = -4.0f * q[0] - ax + 2.0f * dg;
        m[2] = 4.0f * q[0] - 2.0f * ax + dg;
        m[3] = q[1] - q[3] + q[5] - q[6] - q[7] + q[8];
        m[4] = -2.0f * (q[1] - q[3]) + q[5] - q[6] - q[7] + q[8];
        m[5] = q[2] - q[4] + q[5] + q[6] - q[7] - q[8];
        m[6] = -2.0f * (q[2] - q[4]) + q[5] + q[6] - q[7] - q[8];
        m[7] = q[1] - q[2] + q[3] - q[4];
        m[8] = q[5] - q[6] + q[7] - q[8];
        const float sx = src[1] + src[2] + src[3] + src[4], sd = src[5] + src[6] + src[7] + src[8];
        ms[1] = -4.0f * src[0] - sx + 2.0f * sd;
        ms[2] = 4.0f * src[0] - 2.0f * sx + sd;
        ms[3] = src[1] - src[3] + src[5] - src[6] - src[7] + src[8];
        ms[4] = -2.0f * (src[1] - src[3]) + src[5] - src[6] - src[7] + src[8];
        ms[5] = src[2] - src[4] + src[5] + src[6] - src[7] - src[8];
        ms[6] = -2.0f * (src[2] - src[4]) + src[5] + src[6] - src[7] - src[8];
        ms[7] = src[1] - src[2] + src[3] - src[4];
        ms[8] = src[5] - src[6] + src[7] - src[8];
        const float s1 = p.mrt_lambda * w;   // s_0 .. s_6
        float tm[9];
#pragma unroll
        for (int a = 1; a < 9; a++) {
            const float sa = a < 7 ? s1 : w;  // s_7 = s_8 = omega_eff
            tm[a] = sa * m[a] - (1.0f - 0.5f * sa) * ms[a];
        }
        if (HERMITE) {
            // + U = M^-1 C, C_1 = 3 (1 - s_1/2)(dQx + dQy), C_7 = (1 - w/2)(dQx - dQy)
            // (C_7's factor and sign from the Chapman-Enskog expansion: the p_xx
            // moment carries d_xQ_x - d_yQ_y of the third-moment error)
            tm[1] -= 3.0f * (1.0f - 0.5f * s1) * (dQx + dQy);
            tm[7] -= (1.0f - 0.5f * w) * (p.c7x * dQx + p.c7y * dQy);
        }
        // e -= M^-1 tm, M^-1 = (1/36) * integer matrix of the appendix (tm[0] = 0)
        const float k36 = 1.0f / 36.0f;
        const float b12 = -tm[1] - 2.0f * tm[2];
        const float d21 = 2.0f * tm[1] + tm[2];
        e[1] -= k36 * (b12 + 6.0f * tm[3] - 6.0f * tm[4] + 9.0f * tm[7]);
        e[2] -= k36 * (b12 + 6.0f * tm[5] - 6.0f * tm[6] - 9.0f * tm[7]);
        e[3] -= k36 * (b12 - 6.0f * tm[3] + 6.0f * tm[4] + 9.0f * tm[7]);
        e[4] -= k36 * (b12 - 6.0f * tm[5] + 6.0f * tm[6] - 9.0f * tm[7]);
        e[5] -= k36 * (d21 + 6.0f * tm[3] + 3.0f * tm[4] + 6.0f * tm[5] + 3.0f * tm[6] + 9.0f * tm[8]);
        e[6] -= k36 * (d21 - 6.0f * tm[3] - 3.0f * tm[4] + 6.0f * tm[5] + 3.0f * tm[6] - 9.0f * tm[8]);
        e[7] -= k36 * (d21 - 6.0f * tm[3] - 3.0f * tm[4] - 6.0f * tm[5] - 3.0f * tm[6] + 9.0f * tm[8]);
        e[8] -= k36 * (d21 + 6.0f * tm[3] + 3.0f * tm[4] - 6.0f * tm[5] - 3.0f * tm[6] - 9.0f * tm[8]);
    }

    // Eq. (eq:recoloringOperator) written for the stored deviations:
    //   d^r_i = rr rb / rho (phi^b_i - phi^r_i) + rr / rho E_i + term_i
    //   d^b_i = rr rb / rho (phi^r_i - phi^b_i) + rb / rho E_i - term_i
    // with E_i the post-collision non-rest part and term_i the recolouring flux.
    // Each colour is formed from its own density, as in the paper, so a colour
    // that is absent stays exactly zero (no rounding-level phantom colour).
    const float fr = rr * inv_rho, fb = rb * inv_rho;
    const float mix = rr * rb * inv_rho;
    const float F2 = Fx * Fx + Fy * Fy;
    o_m = mix;
    o_gx = o_gy = 0.0f;
    // per |c|^2 class: shift of the stored deviations
    const float sh1 = mix * (p.phi_b[1] - p.phi_r[1]), sh2 = mix * (p.phi_b[2] - p.phi_r[2]);
    if (F2 > 0.0f) {
        // Eq. (eq:perturbation), one A/2 term per colour: A |F| [W (F.c)^2/|F|^2 - B]
        // (even in c_i), and the recolouring flux (odd in c_i)
        const float invFn = rsqrtf(F2);
        const float Fn = F2 * invFn;
        const float A = p.a_coef * w;
        const float pa = A * invFn, pb = A * Fn;
        const float kk = p.beta * mix * inv_rho * invFn;   // beta rr rb / rho^2 / |F|
        if (SPLIT) {
            // only the residuals (rho_k / rho) E_i are stored; the shift and the
            // recolouring flux are rebuilt from m and G = kk F (split_shift)
            o_gx = kk * Fx;
            o_gy = kk * Fy;
#pragma unroll
            for (int i : {1, 2, 5, 6}) {
                const int j = OPP(i);
                const float Fc = CX(i) * Fx + CY(i) * Fy;
                const float pert = pa * WT(i) * Fc * Fc - pb * BP(i);
                const float Ei = e[i] + pert, Ej = e[j] + pert;
                dr[i] = fr * Ei;
                dr[j] = fr * Ej;
                db[i] = fb * Ei;
                db[j] = fb * Ej;
            }
            dr[0] = db[0] = 0.0f;
            return;
        }
        // cos(phi_i) = c_i.F / (|c_i| |F|); rest_i = rr phi^r_i + rb phi^b_i
        const float k1 = kk * (rr * p.phi_r[1] + rb * p.phi_b[1]);
        const float k2 = kk * 0.70710678118654752f * (rr * p.phi_r[2] + rb * p.phi_b[2]);
#pragma unroll
        for (int i : {1, 2, 5, 6}) {
            const int j = OPP(i);
            const float Fc = CX(i) * Fx + CY(i) * Fy;
            const float pert = pa * WT(i) * Fc * Fc - pb * BP(i);
            const float term = (C2(i) == 1 ? k1 : k2) * Fc;
            const float sh = C2(i) == 1 ? sh1 : sh2;
            const float Ei = e[i] + pert, Ej = e[j] + pert;
            dr[i] = sh + fr * Ei + term;
            dr[j] = sh + fr * Ej - term;
            db[i] = -sh + fb * Ei - term;
            db[j] = -sh + fb * Ej + term;
        }
    } else if (SPLIT) {
#pragma unroll
        for (int i = 1; i < 9; i++) {
            dr[i] = fr * e[i];
            db[i] = fb * e[i];
        }
    } else {
#pragma unroll
        for (int i = 1; i < 9; i++) {
            const float sh = C2(i) == 1 ? sh1 : sh2;
            dr[i] = sh + fr * e[i];
            db[i] = -sh + fb * e[i];
        }
    }
    dr[0] = 0.0f;
    db[0] = 0.0f;
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

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// 2D tiled TMA load of one box into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
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
