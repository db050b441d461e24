// lbm_kernels.cuh -- CUDA kernels of the GB300 colour-gradient LBM library.
//
//   k_step_fused   one full time step (pull-stream + boundaries, moments, S2I4
//                  colour gradient, omega_eff, collision, perturbation,
//                  recolouring, store) in a single pass.  Each thread block owns
//                  a strip of W columns and marches up a range of rows; source
//                  rows (all 18 planes, with a ghost margin in x) arrive in a
//                  ring of shared-memory slots by 3D TMA loads, so every stored
//                  population is read from HBM once per step.  The colour field
//                  of the row above is computed one row ahead into a small
//                  shared ring, which is what the gradient stencil reads.
//   k_tp_moments / k_tp_collide
//                  the same step as two plain node-parallel kernels with a
//                  global scratch field (psi, q u) in between: the reference
//                  GPU path, bit-identical to the fused one.
//   k_init, k_fields, k_diag_*, k_advance, k_set_times   support kernels.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

// Resident fused-kernel blocks per SM the register allocation is sized for
// (0: the per-variant choice of FusedCfg::MINB).
#ifndef LBM_FUSED_MIN_BLOCKS
#define LBM_FUSED_MIN_BLOCKS 0
#endif
// 1: each fused step is launched as a programmatic dependent of the previous one.
#ifndef LBM_FUSED_PDL
#define LBM_FUSED_PDL 1
#endif
// March direction of the fused steps: 0 every step up, 1 consecutive steps in
// opposite directions, 2 every step down.
#ifndef LBM_FUSED_ALTERNATE
#define LBM_FUSED_ALTERNATE 0
#endif

// ------------------------------------------------------------------ loaders

// Stored values from global memory; ys is wrapped periodically.
template <typename T>
struct GlobalLoader {
    const float *rho0;   // &rho[b][0][0][0] (interior column 0)
    const T *dev0;       // &dev[b][0][0][0]
    long long rho_plane, dev_plane, rho_row, dev_row;
    int ny;
    int slip;   // free-slip walls
    SplitC q;
    __device__ __forceinline__ GlobalLoader(const SimDesc &d, int b) {
        rho0 = d.rho + b * d.rho_buf + d.ghost;
        dev0 = reinterpret_cast<const T *>(d.dev) + b * d.dev_buf + d.ghost;
        rho_plane = d.rho_plane;
        dev_plane = d.dev_plane;
        rho_row = d.rho_row;
        dev_row = d.dev_row;
        ny = d.ph.ny;
        slip = d.wet.slip;
        q = split_consts(d.ph);
    }
    __device__ __forceinline__ int wrap(int ys) const { return ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys); }
    __device__ __forceinline__ float rho(int k, int xs, int ys) const {
        return rho0[k * rho_plane + (long long)wrap(ys) * rho_row + xs];
    }
    static constexpr bool SPLIT = SplitStore<T>::value;
    // stored value r^k_i of node (xs, ys): the deviation itself, or the split-form residual
    __device__ __forceinline__ float res(int k, int i, int xs, int ys) const {
        return Codec<T>::dec(dev0[(k * 8 + i - 1) * dev_plane + (long long)wrap(ys) * dev_row + xs]);
    }
    // split-form shift h_i of node (xs, ys) (0 without the split form)
    __device__ __forceinline__ float shift(int i, int xs, int ys) const {
        if (!SPLIT) return 0.0f;
        return split_shift(q, i, rho(0, xs, ys), rho(1, xs, ys), rho(2, xs, ys), rho(3, xs, ys), rho(4, xs, ys));
    }
    __device__ __forceinline__ float own_shift_sum(int xs, int ys) const {
        return SPLIT ? 4.0f * rho(2, xs, ys) * (q.dph1 + q.dph2) : 0.0f;
    }
    // stored deviation d^k_i of node (xs, ys), decoded from the split form for 16-bit storage
    __device__ __forceinline__ float dev(int k, int i, int xs, int ys) const {
        const float r = res(k, i, xs, ys);
        if (!SPLIT) return r;
        const float sh = shift(i, xs, ys);
        return k == 0 ? __fadd_rn(r, sh) : __fsub_rn(r, sh);
    }
};

// Stored values from the shared-memory row ring (rows y-1, y, y+1 of a strip
// starting at column x0).  A slot holds [NS][BOXW] floats (padded to RHO_BYTES)
// then [16][BOXW] T.
template <typename T, int BOXW, int G, int RHO_BYTES>
struct SmemLoader {
    const unsigned char *r0, *r1, *r2;
    int y, x0;
    SplitC q;
    int slip;   // free-slip walls (read only by the wetting variants' links)
    __device__ __forceinline__ const unsigned char *row(int ys) const {
        const int dy = ys - y;
        return dy < 0 ? r0 : (dy == 0 ? r1 : r2);
    }
    __device__ __forceinline__ float rho(int k, int xs, int ys) const {
        return reinterpret_cast<const float *>(row(ys))[k * BOXW + (xs - x0 + G)];
    }
    static constexpr bool SPLIT = SplitStore<T>::value;
    __device__ __forceinline__ float res(int k, int i, int xs, int ys) const {
        const T *p = reinterpret_cast<const T *>(row(ys) + RHO_BYTES);
        return Codec<T>::dec(p[(k * 8 + i - 1) * BOXW + (xs - x0 + G)]);
    }
    __device__ __forceinline__ float shift(int i, int xs, int ys) const {
        if (!SPLIT) return 0.0f;
        return split_shift(q, i, rho(0, xs, ys), rho(1, xs, ys), rho(2, xs, ys), rho(3, xs, ys), rho(4, xs, ys));
    }
    __device__ __forceinline__ float own_shift_sum(int xs, int ys) const {
        return SPLIT ? 4.0f * rho(2, xs, ys) * (q.dph1 + q.dph2) : 0.0f;
    }
    __device__ __forceinline__ float dev(int k, int i, int xs, int ys) const {
        const float r = res(k, i, xs, ys);
        if (!SPLIT) return r;
        const float sh = shift(i, xs, ys);
        return k == 0 ? __fadd_rn(r, sh) : __fsub_rn(r, sh);
    }
    // same, for direction indices known only at run time
    __device__ __forceinline__ float rho_rt(int k, int xs, int ys) const { return rho(k, xs, ys); }
    __device__ __forceinline__ float dev_rt(int k, int i, int xs, int ys) const { return dev(k, i, xs, ys); }
};

// psi on a solid wall row: W-weighted mean of the in-domain fluid nodes next
// to it on the adjacent fluid row (Sec. 2.4 extrapolation).  `psi_of(X)`
// returns psi of the fluid node in column X of that row.
template <class PsiOf>
__device__ __forceinline__ float wall_psi(const Phys &p, int X, const PsiOf &psi_of) {
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int dx = -1; dx <= 1; dx++) {
        const int Xp = X + dx;
        if (p.bc_x == BC_PERIODIC || (Xp >= 0 && Xp < p.nx)) {
            const float wgt = dx == 0 ? (1.0f / 9.0f) : (1.0f / 36.0f);
            num += wgt * psi_of(Xp);
            den += wgt;
        }
    }
    return den > 0.0f ? num / den : 0.0f;
}

// S2I4 gradient (Eq. (eq:colorGradient)) summed in opposite pairs so that a
// uniform field gives exactly zero.  v(dx, dy) returns the field at x + (dx, dy).
template <class V>
__device__ __forceinline__ void s2i4(const V &v, float &gx, float &gy) {
    const float e = v(1, 0), wv = v(-1, 0), n = v(0, 1), s = v(0, -1);
    const float ne = v(1, 1), nw = v(-1, 1), sw = v(-1, -1), se = v(1, -1);
    const float a = ne - sw, b = se - nw;
    gx = (1.0f / 3.0f) * (e - wv) + (1.0f / 12.0f) * (a + b);
    gy = (1.0f / 3.0f) * (n - s) + (1.0f / 12.0f) * (a - b);
}

// Colour densities of one pulled node computed by 16 lanes of a warp: lane
// j = 8 k + (i - 1) adds colour k's direction-i term of
//   rho_k' = rho_k(x) + sum_{i>=1} [phi^k_i (s^k_i - rho_k(x)) + delta^k_i - d^k_i(x)]
// and the two colour sums are reduced with shuffles inside the 16-lane group.
// No wall link may touch the node (callers use the serial pull next to walls).
template <class Loader>
__device__ __forceinline__ void pull_rho_coop16(const Phys &p, const Loader &ld, int x, int y, int j, float &rr,
                                                float &rb) {
    const int k = j >> 3, i = (j & 7) + 1;
    const int cx = (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    const int cy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    const int c2 = cx * cx + cy * cy;
    const float ph = k == 0 ? (c2 == 1 ? p.phi_r[1] : p.phi_r[2]) : (c2 == 1 ? p.phi_b[1] : p.phi_b[2]);
    const float own = ld.rho_rt(k, x, y);
    float v;
    if (Loader::SPLIT) {
        // split form: residual difference plus the source's shift; the node's own
        // shifts sum to 4 m (dphi_1 + dphi_2), taken off once after the reduction
        const float sg = k == 0 ? 1.0f : -1.0f;
        v = ph * (ld.rho_rt(k, x - cx, y - cy) - own) + (ld.res(k, i, x - cx, y - cy) - ld.res(k, i, x, y)) +
            sg * ld.shift(i, x - cx, y - cy);
    } else {
        v = ph * (ld.rho_rt(k, x - cx, y - cy) - own) + (ld.dev_rt(k, i, x - cx, y - cy) - ld.dev_rt(k, i, x, y));
    }
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    if (Loader::SPLIT) v -= (k == 0 ? 1.0f : -1.0f) * ld.own_shift_sum(x, y);
    const float mine = own + v;                        // colour k's new density
    const float other = __shfl_xor_sync(0xffffffffu, mine, 8);
    rr = k == 0 ? mine : other;
    rb = k == 0 ? other : mine;
}

// ------------------------------------------------------------ fused kernel

template <typename T, int CV, int W, int NSLOT>
struct FusedCfg {
    static constexpr int GMEM = 8;                           // ghost columns kept in memory
    static constexpr int G = 16 / (int)sizeof(T);            // halo columns loaded each side
    static constexpr int BOXW = W + 2 * G;                   // TMA box width (elements)
    static constexpr int NS = ScalarPlanes<T>::value;          // FP32 node planes per row
    static constexpr int RHO_BYTES = ((NS * BOXW * 4 + 127) / 128) * 128;
    static constexpr int DEV_BYTES = 16 * BOXW * (int)sizeof(T);
    static constexpr int SLOT_BYTES = ((RHO_BYTES + DEV_BYTES + 127) / 128) * 128;
    static constexpr int RING = W + 2;                       // ring width (columns x0-1 .. x0+W)
    static constexpr bool QRING = (CV & CV_MRT) && (CV & CV_HERMITE);
    static constexpr bool WET = (CV & CV_WET) != 0;
    static constexpr int LINKS = WET ? LINKS_ALL : LINKS_NOSLIP;
    // shared rings (floats) of what neighbouring threads read: psi and q u over
    // rows y-1..y+1.  Stage A of row y+1 may run while slower threads still do
    // stage B of row y-1, so they hold 4 rows.  The node's own rho_r, rho_b and
    // e_1..8 stay in the registers of the thread that pulled them.
    static constexpr int PSI_OFF = 0;
    static constexpr int QX_OFF = PSI_OFF + 4 * RING;
    static constexpr int QY_OFF = QX_OFF + (QRING ? 4 * RING : 0);
    static constexpr int RING_FLOATS = QY_OFF + (QRING ? 4 * RING : 0);
    static constexpr int DESC_BYTES = ((int)sizeof(SimDesc) + 127) / 128 * 128;
    static constexpr int RING_BYTES = ((RING_FLOATS * 4 + 15) / 16) * 16;
    static constexpr int SMEM = DESC_BYTES + NSLOT * SLOT_BYTES + RING_BYTES + NSLOT * 8 + 16;
    static constexpr uint32_t TX_BYTES = (uint32_t)(NS * BOXW * 4 + DEV_BYTES);
    // Blocks per SM the registers are sized for: 5 (96 registers) for FP32, 6 (80)
    // for 16-bit storage, whose smaller rows let 6 blocks share the SM's shared
    // memory; 4 (128) for MRT + Hermite, whose source term needs them, and for
    // wetting walls (free-slip links, contact-angle adjustment).  Measured
    // on the 40-lattice sweep: 4 -> 5 blocks +2.5 % (FP32), 4 -> 6 +7 % (FP16).
    static constexpr int MINB = LBM_FUSED_MIN_BLOCKS > 0 ? LBM_FUSED_MIN_BLOCKS
                                : ((QRING || WET) ? 4 : (sizeof(T) == 4 ? 5 : 6));
    static_assert(BOXW <= 256, "TMA box dimension limit");
    static_assert((BOXW * sizeof(T)) % 16 == 0 && (BOXW * 4) % 16 == 0, "TMA inner box bytes");
    static_assert(G <= GMEM && G >= 3, "halo must cover the stencil and fit the memory ghost");
    static_assert(NSLOT >= 4, "the prologue waits for rows ya-2 .. ya+1 before any slot is refilled");
};

// Persistent fused step.  Block b processes the work items
// items[item_off[b] .. item_off[b+1]) in order (strip segments, possibly of
// different simulations), so that every block gets an equal share of rows.
//
// Per segment the block marches up rows ya .. yb-1 of a strip of w <= W
// columns.  Source rows arrive by TMA into a ring of NSLOT shared slots.
// Iteration y first pulls row y+1 (stage A: new colour densities, colour field
// and the colour-blind non-rest parts e_i of every node of that row; the colour
// field also one column each side), then collides row y (stage B) from the
// densities and e_i that the same thread pulled one iteration earlier (kept in
// registers) and the colour field of rows y-1..y+1 in a shared ring (S2I4
// gradient).  Stage B reads no source row, so a row's slot is refilled as soon
// as stage A of the row above has used it.  One block runs 4 warps; 5 or 6
// blocks share an SM (FusedCfg::MINB).
//
// DIR = +1 marches up (rows ya .. yb-1), DIR = -1 down (yb-1 .. ya); every node
// is computed the same way in both.  Consecutive steps march in opposite
// directions, so that a step starts on the rows the previous one wrote last,
// while they are still in L2.
template <typename T, int CV, int W, int NSLOT, int DIR>
__global__ void __launch_bounds__(W, (FusedCfg<T, CV, W, NSLOT>::MINB)) k_step_fused(const SimDesc *__restrict__ descs,
                                                     const WorkItem *__restrict__ items,
                                                     const int *__restrict__ item_off, int n_blocks,
                                                     int step_offset, int flags, int *__restrict__ err) {
    static_assert(DIR == 1 || DIR == -1, "march direction");
    using Cfg = FusedCfg<T, CV, W, NSLOT>;
    constexpr int G = Cfg::G, BOXW = Cfg::BOXW, RING = Cfg::RING;
    constexpr bool HERMITE = (CV & CV_HERMITE) != 0;
    constexpr bool HERMITE_SRC = Cfg::QRING;
    constexpr bool WET = Cfg::WET;
    constexpr bool OPEN = (CV & CV_OPEN) != 0;
    constexpr int LINKS = Cfg::LINKS;
    extern __shared__ __align__(128) unsigned char smem[];

    // Launched as a programmatic dependent of the previous step: this block
    // touches no memory that earlier work writes (descriptors, state, error word)
    // before every prerequisite grid has completed and its writes are visible.
    // With FUSED_EARLY_NEXT (plans of equal pieces, one launch per step) the next
    // step may launch at once, its blocks waiting in the slots this grid frees;
    // otherwise only once this block's work is done (below): on uneven batches
    // and concurrent launch groups the early trigger placed waiting blocks on SMs
    // in the order slots freed and cost 5-16 %.
    if (flags & FUSED_EARLY_NEXT) asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if ((int)blockIdx.x >= n_blocks) return;
    const int tid = threadIdx.x;

    SimDesc &d = *reinterpret_cast<SimDesc *>(smem);
    unsigned char *slots = smem + Cfg::DESC_BYTES;
    float *rings = reinterpret_cast<float *>(slots + NSLOT * Cfg::SLOT_BYTES);
    float *ring_psi = rings + Cfg::PSI_OFF;
    float *ring_qx = rings + Cfg::QX_OFF;
    float *ring_qy = rings + Cfg::QY_OFF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(rings) + Cfg::RING_BYTES);
    volatile int &s_bad = *reinterpret_cast<volatile int *>(bars + NSLOT);

    if (smem_u32(slots) & 127) {   // TMA destinations must be 128-byte aligned
        if (tid == 0) atomicOr(err, ERR_ALIGN);
        return;
    }
    if (tid == 0) s_bad = 0;

    const int it_end = item_off[blockIdx.x + 1];
    for (int itx = item_off[blockIdx.x]; itx < it_end; ++itx) {
        const WorkItem it = items[itx];
        const SimDesc *gd = descs + it.sim;
        __syncthreads();   // previous segment fully consumed (all its rows were waited for)
        {
            const int4 *src = reinterpret_cast<const int4 *>(gd);
            int4 *dst = reinterpret_cast<int4 *>(smem);
            for (int j = tid; j < (int)(sizeof(SimDesc) / 16); j += W) dst[j] = src[j];
        }
        if (tid == 0) {
            for (int s = 0; s < NSLOT; s++) {
                if (itx != item_off[blockIdx.x]) mbar_inval(&bars[s]);
                mbar_init(&bars[s], 1);
            }
            fence_mbar_init();
            fence_proxy_async_smem();
            tensormap_acquire(&gd->tmap_rho);
            tensormap_acquire(&gd->tmap_dev);
        }
        __syncthreads();

        const Phys p = d.ph;   // per-simulation constants, in registers from here on
        const SplitC qs = split_consts(p);
        const long long t = d.t0 + step_offset;
        if (t >= d.t_end) continue;   // this simulation has stopped
        const int bsrc = (int)(t & 1), bdst = bsrc ^ 1;
        const int nx = p.nx, ny = p.ny;
        const bool wall_y = p.bc_y == BC_WALL;
        const int x0 = it.x0, w = it.w, ya = it.ya, yb = it.yb;
        if (d.variant != CV || d.ghost != Cfg::GMEM || w <= 0 || w > W || x0 < 0 || x0 + w > nx || (x0 % 8) != 0 ||
            ya < 0 || yb > ny || ya >= yb) {
            if (tid == 0) atomicOr(err, ERR_BADITEM);
            continue;
        }
        const int row_first = ya - 2, row_last = yb + 1, n_rows = row_last - row_first + 1;
        // march index of source row r: the order in which rows are loaded
        auto mi = [&](int r) { return DIR > 0 ? r - row_first : row_last - r; };
        auto row_at = [&](int m) { return DIR > 0 ? row_first + m : row_last - m; };

        auto row_valid = [&](int r) { return !wall_y || (r >= 0 && r < ny); };
        auto slot_of = [&](int r) { return mi(r) % NSLOT; };
        auto parity_of = [&](int r) { return (uint32_t)((mi(r) / NSLOT) & 1); };
        auto row_ptr = [&](int r) { return slots + slot_of(r) * Cfg::SLOT_BYTES; };
        // Load source row r (both colour densities and all 16 deviation planes,
        // columns x0-G .. x0+W+G-1) into its slot.  A row behind a wall is not
        // loaded, but its slot barrier still completes one phase (plain arrival)
        // so that every slot's phase parity stays (use count) & 1.
        auto issue = [&](int r) {
            const int s = slot_of(r);
            if (!row_valid(r)) {
                mbar_arrive(&bars[s]);
                return;
            }
            const int yr = r < 0 ? r + ny : (r >= ny ? r - ny : r);
            unsigned char *dst = slots + s * Cfg::SLOT_BYTES;
            const int xb = x0 + (Cfg::GMEM - G);   // element index of column x0 - G in the padded row
            mbar_arrive_expect_tx(&bars[s], Cfg::TX_BYTES);
            const int brow = bsrc * ny + yr;   // row index over both buffers
            tma_load_2d(dst, &gd->tmap_rho, &bars[s], xb, brow * Cfg::NS);
            tma_load_2d(dst + Cfg::RHO_BYTES, &gd->tmap_dev, &bars[s], xb, brow * 16);
        };
        int next_m = 0;   // march index of the next row to load; meaningful on thread 0 only
        if (tid == 0) {
            for (; next_m < n_rows && next_m < NSLOT; ++next_m) issue(row_at(next_m));
        }

        bool ok = true;
        auto wait_row = [&](int r) {
            if (ok && mi(r) < n_rows && row_valid(r)) {
                if (!mbar_wait_bounded(&bars[slot_of(r)], parity_of(r), WAIT_LIMIT_CYCLES)) {
                    ok = false;
                    s_bad = 1;
                }
            }
        };
        auto loader = [&](int y) {
            SmemLoader<T, BOXW, G, Cfg::RHO_BYTES> L;
            L.r0 = row_ptr(y - 1);
            L.r1 = row_ptr(y);
            L.r2 = row_ptr(y + 1);
            L.y = y;
            L.x0 = x0;
            L.q = qs;
            L.slip = WET ? d.wet.slip : 0;
            return L;
        };

        auto rs_of = [&](int Y) { return ((Y + 4) & 3) * RING; };   // ring row of lattice row Y
        // ring column c (0 or w+1) of row Y by one thread's full pull (next to
        // walls and open columns, or where the node also needs q u)
        auto edge_full = [&](const auto &L, int Y, int c) {
            int X = x0 - 1 + c;
            if (p.bc_x == BC_INOUT) X = X < 0 ? 0 : (X >= nx ? nx - 1 : X);
            Pulled P;
            pull_node_rows<HERMITE, LINKS>(p, L, X, Y, t, false, 0.0f, 0.0f, P);
            ring_psi[rs_of(Y) + c] = colour_field(p, P.rr, P.rb);
            if (HERMITE_SRC) {
                const NodeMoments m = node_moments(p, P);
                const float q = p.q_r * m.rr + p.q_b * m.rb;
                ring_qx[rs_of(Y) + c] = q * m.ux;
                ring_qy[rs_of(Y) + c] = q * m.uy;
            }
        };

        // stage A: ring row Y, columns x0-1 .. x0+w
        auto stageA = [&](int Y, Pulled &out) {
            const int rs = rs_of(Y);
            if (wall_y && (Y < 0 || Y >= ny)) {
                const int Yn = Y < 0 ? 0 : ny - 1;
                const auto L = loader(Yn);
                for (int c = tid; c < w + 2; c += W) {
                    const int X = x0 - 1 + c;
                    const float ps = wall_psi(p, X, [&](int Xp) {
                        float rr, rb, jx, jy;
                        pull_moments_rows<HERMITE, false, LINKS>(p, L, Xp, Yn, t, rr, rb, jx, jy);
                        return colour_field(p, rr, rb);
                    });
                    ring_psi[rs + c] = ps;
                    if (HERMITE_SRC) {
                        ring_qx[rs + c] = 0.0f;
                        ring_qy[rs + c] = 0.0f;
                    }
                }
            } else {
                const auto L = loader(Y);
                // interior ring columns x0 .. x0+w-1: one node per thread, full pull
                if (tid < w) {
                    const int c = tid + 1;
                    const int X = x0 + tid;
                    Pulled P;
                    pull_node_rows<HERMITE, LINKS>(p, L, X, Y, t, false, 0.0f, 0.0f, P);
                    ring_psi[rs + c] = colour_field(p, P.rr, P.rb);
                    out = P;
                    if (HERMITE_SRC) {
                        const NodeMoments m = node_moments(p, P);
                        const float q = p.q_r * m.rr + p.q_b * m.rb;
                        ring_qx[rs + c] = q * m.ux;
                        ring_qy[rs + c] = q * m.uy;
                    }
                }
                // the two edge columns x0-1 and x0+w only need psi (and q u): the
                // last warp computes them 16 lanes per node, unless a boundary
                // touches them (wall row) or the node needs q u
                const int Ye = Y < 0 ? Y + ny : (Y >= ny ? Y - ny : Y);
                const bool wall_row = wall_y && (Ye == 0 || Ye == ny - 1);
                if constexpr (!OPEN) {
                    // bc_x is always periodic here (the variant says so); the
                    // run-time test stays because without it the compiler lays
                    // out this loop 0.9 % slower on the periodic sweep (measured)
                    if (p.bc_x != BC_PERIODIC) {
                    } else if (!HERMITE_SRC && !wall_row) {
                        if (tid >= W - 32) {
                            const int lane = tid & 31, e = lane >> 4;
                            const int X = e == 0 ? x0 - 1 : x0 + w;
                            float rr, rb;
                            pull_rho_coop16(p, L, X, Y, lane & 15, rr, rb);
                            if ((lane & 15) == 0) ring_psi[rs + (e == 0 ? 0 : w + 1)] = colour_field(p, rr, rb);
                        }
                    } else if (tid < 2) {
                        edge_full(L, Y, tid == 0 ? 0 : w + 1);
                    }
                } else {
                    // open lattice: a side beyond the inlet (x = -1) or the outlet
                    // (x = nx) takes the values of the open column itself (zero
                    // gradient, the pull clamps X there), copied by the thread that
                    // wrote that column; the edge next to an open column (x = 0 or
                    // nx - 1, whose pull is the Zou-He one) is pulled in full
                    const bool open_l = x0 == 0, open_r = x0 + w == nx;
                    const int cc = (open_l && tid == 0) ? 0 : ((open_r && tid == w - 1) ? w + 1 : -1);
                    if (cc >= 0) {
                        ring_psi[rs + cc] = ring_psi[rs + tid + 1];
                        if (HERMITE_SRC) {
                            ring_qx[rs + cc] = ring_qx[rs + tid + 1];
                            ring_qy[rs + cc] = ring_qy[rs + tid + 1];
                        }
                    }
                    const bool plain_l = !open_l && x0 - 1 >= 1, plain_r = !open_r && x0 + w <= nx - 2;
                    if (!HERMITE_SRC && !wall_row && (plain_l || plain_r)) {
                        if (tid >= W - 32) {
                            // all 32 lanes take part (full-warp shuffles); a side
                            // that is not plain pulls column x0 and discards it
                            const int lane = tid & 31, e = lane >> 4;
                            const bool plain = e == 0 ? plain_l : plain_r;
                            const int X = plain ? (e == 0 ? x0 - 1 : x0 + w) : x0;
                            float rr, rb;
                            pull_rho_coop16(p, L, X, Y, lane & 15, rr, rb);
                            if ((lane & 15) == 0 && plain) ring_psi[rs + (e == 0 ? 0 : w + 1)] = colour_field(p, rr, rb);
                        }
                    }
                    const bool full_l = !open_l && (HERMITE_SRC || wall_row || !plain_l);
                    const bool full_r = !open_r && (HERMITE_SRC || wall_row || !plain_r);
                    if ((tid == 0 && full_l) || (tid == 1 && full_r)) edge_full(L, Y, tid == 0 ? 0 : w + 1);
                }
            }
        };

        // stage B: collide row y from the rings
        auto stageB = [&](int y, const Pulled &Pin) {
            if (tid >= w) return;
            const int x = x0 + tid;
            const int rm = ((y + 3) & 3) * RING, r0 = ((y + 4) & 3) * RING, rp = ((y + 5) & 3) * RING;
            const int c = tid + 1;
            Pulled P = Pin;
            float e0 = 0.0f;
#pragma unroll
            for (int i = 1; i < 9; i++) e0 += P.e[i];
            P.e[0] = -e0;
            auto ring = [&](const float *f) {
                return [=](int dx, int dy) { return f[(dy < 0 ? rm : (dy == 0 ? r0 : rp)) + c + dx]; };
            };
            float Fx, Fy, dQx = 0.0f, dQy = 0.0f;
            s2i4(ring(ring_psi), Fx, Fy);
            if (WET) contact_angle_adjust(d.wet, p, y, Fx, Fy);
            if (HERMITE_SRC) {
                float gx_, gy_;
                s2i4(ring(ring_qx), dQx, gy_);
                s2i4(ring(ring_qy), gx_, dQy);
            }
            float dr[9], db[9];
            float sm, sgx, sgy;
            collide_node<CV, SplitStore<T>::value>(p, P, ring_psi[r0 + c], Fx, Fy, dQx, dQy, dr, db, sm, sgx, sgy);
            NodeStore<T>(d, p, bdst, x, y).put(P.rr, P.rb, dr, db, sm, sgx, sgy);
        };

        // prologue: ring rows y0 and y0 - DIR, y0 the first row collided
        const int y0 = DIR > 0 ? ya : yb - 1;
        wait_row(y0 - 1);
        wait_row(y0);
        wait_row(y0 + 1);
        Pulled Pc, Pn;   // pulled state of this thread's node in rows y and y + DIR
        stageA(y0, Pc);
        wait_row(y0 - 2 * DIR);
        stageA(y0 - DIR, Pn);
        __syncthreads();   // rows behind y0 are no longer read: refill their slots
        if (tid == 0) {
            for (; next_m < n_rows && next_m <= mi(y0 - DIR) + NSLOT; ++next_m) issue(row_at(next_m));
        }

        for (int k = 0; k < yb - ya; ++k) {
            const int y = y0 + DIR * k;
            wait_row(y + 2 * DIR);
            stageA(y + DIR, Pn);
            __syncthreads();
            if (s_bad) break;
            if (tid == 0) {
                // row y and those behind it are no longer read (stage A(y + DIR)
                // was their last reader)
                for (; next_m < n_rows && next_m <= mi(y) + NSLOT; ++next_m) issue(row_at(next_m));
            }
            stageB(y, Pc);
            Pc = Pn;
        }

        if (s_bad) {
            __syncthreads();
            if (tid == 0) {
                atomicOr(err, ERR_TIMEOUT);
                // wait (bounded) for the copies this block still has in flight, so
                // that none lands after the block's shared memory is released: the
                // latest phase issued into each slot covers the earlier ones
                for (int s = 0; s < NSLOT; s++) {
                    int last = -1;
                    for (int m = 0; m < next_m; ++m)
                        if (m % NSLOT == s) last = m;
                    if (last >= 0) mbar_wait_bounded(&bars[s], (uint32_t)((last / NSLOT) & 1), WAIT_LIMIT_CYCLES / 4);
                }
            }
            __syncthreads();
            return;
        }
    }
    // this block's stores are issued: the next step may launch (it still waits
    // for this grid's completion before it reads anything); a block that
    // triggered at its start does not trigger again
    if (!(flags & FUSED_EARLY_NEXT)) asm volatile("griddepcontrol.launch_dependents;");
}

// --------------------------------------------------------- two-pass kernels

// Pass 1: colour field, colour densities and q u of every node.
template <typename T, int CV>
__global__ void k_tp_moments(const SimDesc *__restrict__ dp, int step_offset, float *__restrict__ aux) {
    constexpr bool HERMITE = (CV & CV_HERMITE) != 0, HERMITE_SRC = HERMITE && (CV & CV_MRT);
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const long long t = d.t0 + step_offset;
    if (t >= d.t_end) return;   // this simulation has stopped
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

// Value of an aux field at lattice position (X, Y) next to the domain.
__device__ __forceinline__ float aux_at(const Phys &p, const float *f, int X, int Y, bool is_psi) {
    const int nx = p.nx, ny = p.ny;
    if (Y < 0 || Y >= ny) {
        if (p.bc_y == BC_WALL) {
            if (!is_psi) return 0.0f;
            const int Yn = Y < 0 ? 0 : ny - 1;
            return wall_psi(p, X, [&](int Xp) {
                const int xw = Xp < 0 ? Xp + nx : (Xp >= nx ? Xp - nx : Xp);
                return f[(long long)Yn * nx + xw];
            });
        }
        Y = Y < 0 ? Y + ny : Y - ny;
    }
    if (X < 0 || X >= nx) {
        if (p.bc_x == BC_PERIODIC) X = X < 0 ? X + nx : X - nx;
        else X = X < 0 ? 0 : nx - 1;
    }
    return f[(long long)Y * nx + X];
}

// Pass 2: gradient from the scratch field, collision, perturbation,
// recolouring and store of every node.
template <typename T, int CV>
__global__ void k_tp_collide(const SimDesc *__restrict__ dp, int step_offset, const float *__restrict__ aux) {
    constexpr bool HERMITE = (CV & CV_HERMITE) != 0, HERMITE_SRC = HERMITE && (CV & CV_MRT);
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const long long t = d.t0 + step_offset;
    if (t >= d.t_end) return;   // this simulation has stopped
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

// ------------------------------------------------------------ init / fields

// Equilibrium state from FP64 fields at t = 0.  The stored state is the one
// whose first pull yields N^k_i(x, 0) = N^{k(e)}_i(x): the slot (i, y) holds
// the equilibrium population of the node that will read it -- node y + c_i,
// or node y itself in direction opp(i) when that link is bounced by a wall.
// The stored colour density of y is the sum of its slots, the deviations are
// taken from it.
// With `pops` non-null the pre-collision populations N^k_i(x, 0) are given
// directly (layout [2][9][ny][nx]) instead of being the equilibria of the fields.
template <typename T>
__global__ void k_init(const SimDesc *__restrict__ dp, const double *__restrict__ rr,
                       const double *__restrict__ rb, const double *__restrict__ ux,
                       const double *__restrict__ uy, const double *__restrict__ pops) {
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const bool hermite = (d.variant & CV_HERMITE) != 0;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const double herm[2] = {p.herm_r, p.herm_b};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        // equilibrium population i of colour kk at node (X, Y) (in the domain)
        auto feq = [&](int kk, int i, int X, int Y) {
            const long long m = (long long)Y * nx + X;
            if (pops) return pops[(long long)(kk * 9 + i) * n + m];
            const double vx = ux[m], vy = uy[m], usq = vx * vx + vy * vy;
            const double rho = kk == 0 ? rr[m] : rb[m];
            const double cu = CX(i) * vx + CY(i) * vy;
            double lin = 3.0 * cu;
            if (hermite) lin = 3.0 * cu * (1.0 + 0.5 * herm[kk] * (3.0 * C2(i) - 4.0));
            return rho * (double)phi_k(p, kk, C2(i)) + rho * WT(i) * (lin + 4.5 * cu * cu - 1.5 * usq);
        };
        double v[2][9];
#pragma unroll
        for (int i = 0; i < 9; i++) {
            int X = x + CX(i), Y = y + CY(i);
            // 0: read by node (X, Y), 1: bounced back to (x, y), 2: unread,
            // 3: sent on along a free-slip wall to node (X, y) in direction MIRY(i)
            int mode = 0;
            if (i != 0) {
                if (Y < 0 || Y >= ny) {
                    if (p.bc_y == BC_WALL) {
                        mode = 1;
                        if (d.wet.slip && (p.bc_x == BC_PERIODIC || (X >= 0 && X < nx))) {
                            mode = 3;
                            Y = y;
                            X = X < 0 ? X + nx : (X >= nx ? X - nx : X);
                        }
                    } else {
                        Y = Y < 0 ? Y + ny : Y - ny;
                    }
                }
                if (mode == 0 && (X < 0 || X >= nx)) {
                    if (p.bc_x == BC_PERIODIC) X = X < 0 ? X + nx : X - nx;
                    else mode = 2;
                }
            }
            for (int kk = 0; kk < 2; kk++) {
                if (mode == 0) v[kk][i] = feq(kk, i, X, Y);
                else if (mode == 3) v[kk][i] = feq(kk, MIRY(i), X, Y);
                else if (mode == 1) v[kk][i] = feq(kk, OPP(i), x, y);
                else v[kk][i] = pops ? pops[(long long)(kk * 9 + i) * n + k]
                                     : (double)phi_k(p, kk, C2(i)) * (kk == 0 ? rr[k] : rb[k]);
            }
        }
        float dr[9], db[9];
        double rs[2];
        for (int kk = 0; kk < 2; kk++) {
            double s = 0.0;
            for (int i = 0; i < 9; i++) s += v[kk][i];
            rs[kk] = s;
            for (int i = 1; i < 9; i++) {
                const float dv = (float)(v[kk][i] - (double)phi_k(p, kk, C2(i)) * s);
                if (kk == 0) dr[i] = dv; else db[i] = dv;
            }
        }
        dr[0] = db[0] = 0.0f;
        NodeStore<T>(d, p, 0, x, y).store((float)rs[0], (float)rs[1], dr, db);
    }
}

// Macroscopic fields of the state at time t (pre-collision moments).
template <typename T, bool HERMITE>
__global__ void k_fields(const SimDesc *__restrict__ dp, long long t, double *__restrict__ out) {
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L(d, (int)(t & 1));
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        Pulled P;
        pull_node<HERMITE>(p, L, x, y, t, false, 0.0f, 0.0f, P);
        const NodeMoments m = node_moments(p, P);
        out[k] = m.rr;
        out[n + k] = m.rb;
        out[2 * n + k] = m.ux;
        out[3 * n + k] = m.uy;
        out[4 * n + k] = (double)m.rr * p.cs2_r + (double)m.rb * p.cs2_b;
    }
}

// Slug-train profile of the state at time t (the measurements of Sec. 5.1), in
// FP64: per column x the light-phase thickness g(x) = sum_y (1 - psi)/2, and the
// colour field psi_c(x) on the channel centreline (the middle row, or the mean
// of the two middle rows when ny is even).  out[0, nx) = g, out[nx, 2 nx) = psi_c.
// One thread per column; the threads of a warp read neighbouring columns.
template <typename T, bool HERMITE>
__global__ void k_slug_profile(const SimDesc *__restrict__ dp, long long t, double *__restrict__ out) {
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const int nx = p.nx, ny = p.ny;
    const GlobalLoader<T> L(d, (int)(t & 1));
    const int ya = (ny - 1) / 2, yb = ny / 2;   // the same row when ny is odd
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
        double g = 0.0, pc = 0.0;
        for (int y = 0; y < ny; y++) {
            Pulled P;
            pull_node<HERMITE>(p, L, x, y, t, false, 0.0f, 0.0f, P);
            const double a = (double)P.rr * p.inv_gamma, b = (double)P.rb;
            const double psi = (a - b) / (a + b);     // Eq. (eq:color_field)
            g += 0.5 * (1.0 - psi);
            if (y == ya || y == yb) pc += psi;
        }
        out[x] = g;
        out[nx + x] = ya == yb ? pc : 0.5 * pc;
    }
}

// Pre-collision populations of every node at time t, layout [2][9][ny][nx].
template <typename T, bool HERMITE>
__global__ void k_read_pops(const SimDesc *__restrict__ dp, long long t, double *__restrict__ out) {
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L(d, (int)(t & 1));
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        double nr[9], nb[9];
        pull_populations<HERMITE>(p, L, x, y, t, nr, nb);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            out[i * n + k] = nr[i];
            out[(9 + i) * n + k] = nb[i];
        }
    }
}

// ---------------------------------------------------------------- diagnostics
constexpr int DIAG_NQ = 16;
constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-reduce DIAG_NQ values (slot 5 is a max, the rest sums) into part[block].
__device__ __forceinline__ void block_reduce_store(double (&acc)[DIAG_NQ], double *part) {
    __shared__ double sh[DIAG_THREADS / 32][DIAG_NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < DIAG_NQ; q++) {
        const double v = q == 5 ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) sh[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_NQ) {
        const int q = threadIdx.x;
        double v = sh[0][q];
        for (int j = 1; j < DIAG_THREADS / 32; j++) v = q == 5 ? fmax(v, sh[j][q]) : v + sh[j][q];
        part[(long long)blockIdx.x * DIAG_NQ + q] = v;
    }
}

// pass 0: mass_r, mass_b, mom_x, mom_y, area_b, max|u| (slot 5), sum x w_b, sum y w_b,
//         sum ux w_b, sum ux w_r, sum w_r, nonfinite
// pass 1: sum p (r < r_in), count, sum p (r > r_out), count around (cx, cy)
template <typename T, bool HERMITE>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(const SimDesc *__restrict__ dp, long long t, int pass,
                                                       double cx, double cy, double r_in, double r_out,
                                                       double *__restrict__ part) {
    const SimDesc &d = *dp;
    const Phys p = d.ph;
    const int nx = p.nx, ny = p.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L(d, (int)(t & 1));
    double acc[DIAG_NQ];
#pragma unroll
    for (int q = 0; q < DIAG_NQ; q++) acc[q] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        Pulled P;
        pull_node<HERMITE>(p, L, x, y, t, false, 0.0f, 0.0f, P);
        const NodeMoments m = node_moments(p, P);
        const double rho = (double)m.rr + m.rb;
        if (pass == 0) {
            const bool bad = !(isfinite(m.rr) && isfinite(m.rb) && isfinite(m.ux) && isfinite(m.uy));
            if (bad) { acc[11] += 1.0; continue; }
            const double wb = 0.5 * (1.0 - m.psi), wr = 1.0 - wb;
            acc[0] += m.rr;
            acc[1] += m.rb;
            acc[2] += rho * m.ux;
            acc[3] += rho * m.uy;
            acc[4] += wb;
            acc[5] = fmax(acc[5], sqrt((double)m.ux * m.ux + (double)m.uy * m.uy));
            acc[6] += wb * x;
            acc[7] += wb * y;
            acc[8] += wb * m.ux;
            acc[9] += wr * m.ux;
            acc[10] += wr;
        } else {
            double dx = fabs(x - cx), dy = fabs(y - cy);
            if (p.bc_x == BC_PERIODIC) dx = fmin(dx, nx - dx);
            if (p.bc_y == BC_PERIODIC) dy = fmin(dy, ny - dy);
            const double r = sqrt(dx * dx + dy * dy);
            const double pr = (double)m.rr * p.cs2_r + (double)m.rb * p.cs2_b;
            if (r < r_in) { acc[0] += pr; acc[1] += 1.0; }
            if (r > r_out) { acc[2] += pr; acc[3] += 1.0; }
        }
    }
    block_reduce_store(acc, part);
}

#ifndef LBM_DEVICE_HELPERS_ONLY   // non-template kernels: defined in one translation unit
// Sum the per-block partials in block order (deterministic) into out[DIAG_NQ].
__global__ void k_diag_final(const double *__restrict__ part, int nblocks, double *__restrict__ out) {
    const int q = threadIdx.x;
    if (q >= DIAG_NQ) return;
    double v = q == 5 ? 0.0 : 0.0;
    for (int b = 0; b < nblocks; b++) {
        const double x = part[(long long)b * DIAG_NQ + q];
        v = q == 5 ? fmax(v, x) : v + x;
    }
    out[q] = v;
}

// ------------------------------------------------------------------- time
__global__ void k_advance(SimDesc *descs, int n, long long k) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) descs[i].t0 += k;
}

// A descriptor's start time and stop time (a batch keeps its own copies of its
// members' descriptors, so both follow the member's logical time and stop here).
__global__ void k_set_times(SimDesc *desc, long long t0, long long t_end) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        desc->t0 = t0;
        desc->t_end = t_end;
    }
}

#endif

}  // namespace lbm
