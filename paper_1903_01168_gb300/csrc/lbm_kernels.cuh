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
//   k_init, k_fields, k_diag_*, k_advance, k_set_t0   support kernels.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

// ------------------------------------------------------------------ loaders

// Decoded stored value from global memory; ys is wrapped periodically.
template <typename T>
struct GlobalLoader {
    const SimDesc *d;
    int b;
    __device__ __forceinline__ float operator()(int p, int xs, int ys) const {
        const int ny = d->ny;
        const int yw = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
        return Codec<T>::dec(*pop_ptr<T>(*d, b, p, xs, yw), d->ref[p]);
    }
};

// Decoded stored value from the shared-memory row ring; rows y-1, y, y+1.
template <typename T, int BOXW, int G>
struct SmemLoader {
    const T *r0, *r1, *r2;
    int y, x0;
    const float *ref;
    __device__ __forceinline__ float operator()(int p, int xs, int ys) const {
        const int dy = ys - y;
        const T *r = dy < 0 ? r0 : (dy == 0 ? r1 : r2);
        return Codec<T>::dec(r[p * BOXW + (xs - x0 + G)], ref[p]);
    }
};

// psi on a solid wall row: W-weighted mean of the in-domain fluid nodes next
// to it on the adjacent fluid row (Sec. 2.4 extrapolation).  `psi_of(X)`
// returns psi of the fluid node in column X of that row.
template <class PsiOf>
__device__ __forceinline__ float wall_psi(const SimDesc &d, int X, const PsiOf &psi_of) {
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int dx = -1; dx <= 1; dx++) {
        const int Xp = X + dx;
        if (d.bc_x == BC_PERIODIC || (Xp >= 0 && Xp < d.nx)) {
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

// ------------------------------------------------------------ fused kernel

template <typename T, int W, int NSLOT>
struct FusedCfg {
    static constexpr int G = 16 / (int)sizeof(T);           // ghost columns each side
    static constexpr int BOXW = W + 2 * G;                   // TMA box width (elements)
    static constexpr int SLOT_BYTES = ((18 * BOXW * (int)sizeof(T) + 127) / 128) * 128;
    static constexpr int RING = W + 2;                       // colour-field ring width
    static constexpr int DESC_BYTES = ((int)sizeof(SimDesc) + 127) / 128 * 128;
    static constexpr int RING_BYTES = 3 * 4 * RING * 4;
    static constexpr int SMEM = DESC_BYTES + NSLOT * SLOT_BYTES + RING_BYTES + NSLOT * 8 + 16;
    static constexpr uint32_t BOX_BYTES = 18u * BOXW * sizeof(T);
    static_assert(BOXW <= 256, "TMA box dimension limit");
    static_assert((BOXW * sizeof(T)) % 16 == 0, "TMA inner box bytes must be a multiple of 16");
};

template <typename T, int W, int NSLOT>
__global__ void __launch_bounds__(W) k_step_fused(const SimDesc *__restrict__ descs,
                                                  const WorkItem *__restrict__ items, int n_items,
                                                  int step_offset, int *__restrict__ err) {
    using Cfg = FusedCfg<T, W, NSLOT>;
    constexpr int G = Cfg::G, BOXW = Cfg::BOXW, RING = Cfg::RING;
    extern __shared__ __align__(128) unsigned char smem[];

    if ((int)blockIdx.x >= n_items) return;
    const int tid = threadIdx.x;
    const WorkItem it = items[blockIdx.x];
    const SimDesc *gd = descs + it.sim;

    SimDesc &d = *reinterpret_cast<SimDesc *>(smem);
    unsigned char *slots = smem + Cfg::DESC_BYTES;
    float *psi_s = reinterpret_cast<float *>(slots + NSLOT * Cfg::SLOT_BYTES);
    float *qux_s = psi_s + 4 * RING;
    float *quy_s = qux_s + 4 * RING;
    uint64_t *bars = reinterpret_cast<uint64_t *>(quy_s + 4 * RING);
    volatile int &s_bad = *reinterpret_cast<volatile int *>(bars + NSLOT);

    if (smem_u32(slots) & 127) {   // TMA destinations must be 128-byte aligned
        if (tid == 0) atomicOr(err, ERR_ALIGN);
        return;
    }
    {
        const int4 *src = reinterpret_cast<const int4 *>(gd);
        int4 *dst = reinterpret_cast<int4 *>(smem);
        for (int j = tid; j < (int)(sizeof(SimDesc) / 16); j += W) dst[j] = src[j];
    }
    if (tid == 0) {
        s_bad = 0;
        for (int s = 0; s < NSLOT; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        tensormap_acquire(&gd->tmap);
    }
    __syncthreads();

    const long long t = d.t0 + step_offset;
    const int bsrc = (int)(t & 1), bdst = bsrc ^ 1;
    const int nx = d.nx, ny = d.ny;
    const bool wall_y = d.bc_y == BC_WALL;
    const bool hermite_src = d.collision == 1 && d.equilibrium == 1;
    const int x0 = it.x0, w = it.w, ya = it.ya, yb = it.yb;
    if (w <= 0 || w > W || x0 < 0 || x0 + w > nx || ya < 0 || yb > ny || ya >= yb) {
        if (tid == 0) atomicOr(err, ERR_BADITEM);
        return;
    }
    const int row_first = ya - 2, row_last = yb + 1;

    auto row_valid = [&](int r) { return !wall_y || (r >= 0 && r < ny); };
    auto slot_of = [&](int r) { return (r - row_first) % NSLOT; };
    auto parity_of = [&](int r) { return (uint32_t)(((r - row_first) / NSLOT) & 1); };
    auto row_ptr = [&](int r) {
        return reinterpret_cast<const T *>(slots + slot_of(r) * Cfg::SLOT_BYTES);
    };
    // Load source row r into its slot.  A row behind a wall is not loaded, but
    // its slot barrier still completes one phase (plain arrival) so that the
    // phase parity of every slot stays (use count) & 1.
    auto issue = [&](int r) {
        const int s = slot_of(r);
        if (!row_valid(r)) {
            mbar_arrive(&bars[s]);
            return;
        }
        const int yr = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        mbar_arrive_expect_tx(&bars[s], Cfg::BOX_BYTES);
        tma_load_3d(slots + s * Cfg::SLOT_BYTES, &gd->tmap, &bars[s], x0, yr, bsrc * 18);
    };
    int next_issue = row_first;   // meaningful on thread 0 only
    if (tid == 0) {
        for (; next_issue <= row_last && next_issue < row_first + NSLOT; ++next_issue) issue(next_issue);
    }

    bool ok = true;
    auto wait_row = [&](int r) {
        if (ok && r <= row_last && row_valid(r)) {
            if (!mbar_wait_bounded(&bars[slot_of(r)], parity_of(r), WAIT_LIMIT_CYCLES)) {
                ok = false;
                s_bad = 1;
            }
        }
    };
    auto loader = [&](int y) {
        SmemLoader<T, BOXW, G> L;
        L.r0 = row_ptr(y - 1);
        L.r1 = row_ptr(y);
        L.r2 = row_ptr(y + 1);
        L.y = y;
        L.x0 = x0;
        L.ref = d.ref;
        return L;
    };

    // colour field (and q u) of ring row Y for ring columns X = x0 - 1 .. x0 + w
    auto stageA = [&](int Y) {
        const int rs = ((Y + 4) & 3) * RING;
        if (wall_y && (Y < 0 || Y >= ny)) {
            const int Yn = Y < 0 ? 0 : ny - 1;
            const auto L = loader(Yn);
            for (int c = tid; c < w + 2; c += W) {
                const int X = x0 - 1 + c;
                const float ps = wall_psi(d, X, [&](int Xp) {
                    float nr[9], nb[9];
                    pull_node(d, L, Xp, Yn, t, nr, nb);
                    return node_moments(d, nr, nb).psi;
                });
                psi_s[rs + c] = ps;
                qux_s[rs + c] = 0.0f;
                quy_s[rs + c] = 0.0f;
            }
        } else {
            const auto L = loader(Y);
            for (int c = tid; c < w + 2; c += W) {
                int X = x0 - 1 + c;
                if (d.bc_x == BC_INOUT) X = X < 0 ? 0 : (X >= nx ? nx - 1 : X);
                float nr[9], nb[9];
                pull_node(d, L, X, Y, t, nr, nb);
                const NodeMoments m = node_moments(d, nr, nb);
                psi_s[rs + c] = m.psi;
                if (hermite_src) {
                    const float q = d.q_r * m.rr + d.q_b * m.rb;
                    qux_s[rs + c] = q * m.ux;
                    quy_s[rs + c] = q * m.uy;
                }
            }
        }
    };

    auto stageB = [&](int y) {
        if (tid >= w) return;
        const int x = x0 + tid;
        float nr[9], nb[9];
        pull_node(d, loader(y), x, y, t, nr, nb);
        const int rm = ((y + 3) & 3) * RING, r0 = ((y + 4) & 3) * RING, rp = ((y + 5) & 3) * RING;
        const int c = tid + 1;
        auto ring = [&](const float *f) {
            return [=](int dx, int dy) { return f[(dy < 0 ? rm : (dy == 0 ? r0 : rp)) + c + dx]; };
        };
        float Fx, Fy, dQx = 0.0f, dQy = 0.0f;
        s2i4(ring(psi_s), Fx, Fy);
        if (hermite_src) {
            float gx_, gy_;
            s2i4(ring(qux_s), dQx, gy_);
            s2i4(ring(quy_s), gx_, dQy);
        }
        collide_node(d, nr, nb, Fx, Fy, dQx, dQy);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            store_pop<T>(d, bdst, i, x, y, nr[i]);
            store_pop<T>(d, bdst, 9 + i, x, y, nb[i]);
        }
    };

    // prologue: colour field of rows ya and ya - 1
    wait_row(ya - 1);
    wait_row(ya);
    wait_row(ya + 1);
    stageA(ya);
    wait_row(ya - 2);
    stageA(ya - 1);

    for (int y = ya; y < yb; ++y) {
        wait_row(y + 2);
        stageA(y + 1);
        __syncthreads();
        if (s_bad) break;
        if (tid == 0) {
            const int r = y - 2 + NSLOT;
            if (r == next_issue && r <= row_last) {
                issue(r);
                ++next_issue;
            }
        }
        stageB(y);
    }

    if (s_bad) {
        __syncthreads();
        if (tid == 0) {
            atomicOr(err, ERR_TIMEOUT);
            // wait (bounded) for the copies this block still has in flight, so
            // that none lands after the block's shared memory is released: the
            // latest phase issued into each slot covers the earlier ones
            for (int s = 0; s < NSLOT; s++) {
                int last = -1 << 30;
                for (int r = row_first; r < next_issue; ++r)
                    if (slot_of(r) == s) last = r;
                if (last > (-1 << 30)) mbar_wait_bounded(&bars[s], parity_of(last), WAIT_LIMIT_CYCLES / 4);
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------- two-pass kernels

// Pass 1: psi and q u of every node into the scratch field aux[3][ny][nx].
template <typename T>
__global__ void k_tp_moments(const SimDesc *__restrict__ dp, long long t, float *__restrict__ aux) {
    const SimDesc &d = *dp;
    const int nx = d.nx, ny = d.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L{dp, (int)(t & 1)};
    const bool hermite_src = d.collision == 1 && d.equilibrium == 1;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        float nr[9], nb[9];
        pull_node(d, L, x, y, t, nr, nb);
        const NodeMoments m = node_moments(d, nr, nb);
        aux[k] = m.psi;
        if (hermite_src) {
            const float q = d.q_r * m.rr + d.q_b * m.rb;
            aux[n + k] = q * m.ux;
            aux[2 * n + k] = q * m.uy;
        }
    }
}

// Value of an aux field at lattice position (X, Y) next to the domain.
__device__ __forceinline__ float aux_at(const SimDesc &d, const float *f, int X, int Y, bool is_psi) {
    const int nx = d.nx, ny = d.ny;
    if (Y < 0 || Y >= ny) {
        if (d.bc_y == BC_WALL) {
            if (!is_psi) return 0.0f;
            const int Yn = Y < 0 ? 0 : ny - 1;
            return wall_psi(d, X, [&](int Xp) {
                const int xw = Xp < 0 ? Xp + nx : (Xp >= nx ? Xp - nx : Xp);
                return f[(long long)Yn * nx + xw];
            });
        }
        Y = Y < 0 ? Y + ny : Y - ny;
    }
    if (X < 0 || X >= nx) {
        if (d.bc_x == BC_PERIODIC) X = X < 0 ? X + nx : X - nx;
        else X = X < 0 ? 0 : nx - 1;
    }
    return f[(long long)Y * nx + X];
}

// Pass 2: gradient from the scratch field, collision, perturbation,
// recolouring and store of every node.
template <typename T>
__global__ void k_tp_collide(const SimDesc *__restrict__ dp, long long t, const float *__restrict__ aux) {
    const SimDesc &d = *dp;
    const int nx = d.nx, ny = d.ny;
    const long long n = (long long)nx * ny;
    const int bsrc = (int)(t & 1);
    const GlobalLoader<T> L{dp, bsrc};
    const bool hermite_src = d.collision == 1 && d.equilibrium == 1;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        float nr[9], nb[9];
        pull_node(d, L, x, y, t, nr, nb);
        float Fx, Fy, dQx = 0.0f, dQy = 0.0f;
        s2i4([&](int dx, int dy) { return aux_at(d, aux, x + dx, y + dy, true); }, Fx, Fy);
        if (hermite_src) {
            float gx_, gy_;
            s2i4([&](int dx, int dy) { return aux_at(d, aux + n, x + dx, y + dy, false); }, dQx, gy_);
            s2i4([&](int dx, int dy) { return aux_at(d, aux + 2 * n, x + dx, y + dy, false); }, gx_, dQy);
        }
        collide_node(d, nr, nb, Fx, Fy, dQx, dQy);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            store_pop<T>(d, bsrc ^ 1, i, x, y, nr[i]);
            store_pop<T>(d, bsrc ^ 1, 9 + i, x, y, nb[i]);
        }
    }
}

// ------------------------------------------------------------ init / fields

// Equilibrium state from FP64 fields, written into the slots the first pull
// reads so that pulling at t = 0 yields N^k_i(x, 0) = N^{k(e)}_i (buffer 0).
template <typename T>
__global__ void k_init(const SimDesc *__restrict__ dp, const double *__restrict__ rr,
                       const double *__restrict__ rb, const double *__restrict__ ux,
                       const double *__restrict__ uy) {
    const SimDesc &d = *dp;
    const int nx = d.nx, ny = d.ny;
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        const double vx = ux[k], vy = uy[k], usq = vx * vx + vy * vy;
        const double rho[2] = {rr[k], rb[k]};
        const double herm[2] = {d.herm_r, d.herm_b};
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const double cu = CX(i) * vx + CY(i) * vy;
            double lin = 3.0 * cu;
            int xs = x - CX(i), ys = y - CY(i), plane = i, xd = x, yd = y;
            for (int kk = 0; kk < 2; kk++) {
                const double phi = kk == 0 ? d.phi_r[C2(i)] : d.phi_b[C2(i)];
                double l = lin;
                if (d.equilibrium) l = 3.0 * cu * (1.0 + 0.5 * herm[kk] * (3.0 * C2(i) - 4.0));
                const double feq = rho[kk] * phi + rho[kk] * WT(i) * (l + 4.5 * cu * cu - 1.5 * usq);
                if (ys < 0 || ys >= ny) {
                    if (d.bc_y == BC_WALL) {
                        store_pop<T>(d, 0, kk * 9 + OPP(i), x, y, (float)feq);
                        continue;
                    }
                    yd = ys < 0 ? ys + ny : ys - ny;
                } else {
                    yd = ys;
                }
                if (xs < 0 || xs >= nx) {
                    if (d.bc_x != BC_PERIODIC) continue;   // unknown at an open boundary
                    xd = xs < 0 ? xs + nx : xs - nx;
                } else {
                    xd = xs;
                }
                store_pop<T>(d, 0, kk * 9 + plane, xd, yd, (float)feq);
            }
        }
    }
}

// Macroscopic fields of the state at time t (pre-collision moments).
template <typename T>
__global__ void k_fields(const SimDesc *__restrict__ dp, long long t, double *__restrict__ out) {
    const SimDesc &d = *dp;
    const int nx = d.nx, ny = d.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L{dp, (int)(t & 1)};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        float nr[9], nb[9];
        pull_node(d, L, x, y, t, nr, nb);
        const NodeMoments m = node_moments(d, nr, nb);
        out[k] = m.rr;
        out[n + k] = m.rb;
        out[2 * n + k] = m.ux;
        out[3 * n + k] = m.uy;
        out[4 * n + k] = (double)m.rr * d.cs2_r + (double)m.rb * d.cs2_b;
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
template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(const SimDesc *__restrict__ dp, long long t, int pass,
                                                       double cx, double cy, double r_in, double r_out,
                                                       double *__restrict__ part) {
    const SimDesc &d = *dp;
    const int nx = d.nx, ny = d.ny;
    const long long n = (long long)nx * ny;
    const GlobalLoader<T> L{dp, (int)(t & 1)};
    double acc[DIAG_NQ];
#pragma unroll
    for (int q = 0; q < DIAG_NQ; q++) acc[q] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        float nr[9], nb[9];
        pull_node(d, L, x, y, t, nr, nb);
        const NodeMoments m = node_moments(d, nr, nb);
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
            if (d.bc_x == BC_PERIODIC) dx = fmin(dx, nx - dx);
            if (d.bc_y == BC_PERIODIC) dy = fmin(dy, ny - dy);
            const double r = sqrt(dx * dx + dy * dy);
            const double p = (double)m.rr * d.cs2_r + (double)m.rb * d.cs2_b;
            if (r < r_in) { acc[0] += p; acc[1] += 1.0; }
            if (r > r_out) { acc[2] += p; acc[3] += 1.0; }
        }
    }
    block_reduce_store(acc, part);
}

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

__global__ void k_set_t0(SimDesc *desc, long long t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) desc->t0 = t;
}

}  // namespace lbm
