// lbm_api.cu -- host implementation of the C ABI declared in include/lbm.h.
//
// Owns parameters, device buffers, streams, TMA descriptors, work tables,
// CUDA graphs and error reporting.  All lattice arithmetic runs in the kernels
// of lbm_kernels.cuh; the host only derives the per-simulation constants of
// arXiv 1903.01168 Sec. 2.1 (alpha_r from gamma, the omega_eff interpolation
// coefficients, A / omega_eff = 9 sigma / 4) and lays out the geometry of the
// initial states.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

thread_local char g_create_err[256] = "";

void set_err(char *buf, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
}

int elem_size(int storage) { return storage == ST_F32 ? 4 : 2; }

// ---- driver entry point for tensor-map encoding (no -lcuda link needed)
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Wetting walls: free-slip links or the contact-angle adjustment of F.
bool wetting(const lbm_params *p) { return p->wall_slip != 0 || p->contact_angle > 0.0; }

int variant_of(const lbm_params *p) {
    return (p->collision == LBM_MRT ? CV_MRT : 0) | (p->equilibrium == LBM_EQ_HERMITE ? CV_HERMITE : 0) |
           (wetting(p) ? CV_WET : 0) | (p->bc_x == LBM_BC_INOUT ? CV_OPEN : 0);
}

}  // namespace

struct lbm_sim {
    int dev = 0;
    int nx = 0, ny = 0;
    lbm_params p{};
    SimDesc h{};                 // host copy of the descriptor
    SimDesc *d_desc = nullptr;   // device copy
    void *pop = nullptr;
    size_t pop_bytes = 0;
    bool own_pop = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long t = 0;
    long long dev_t0 = -1;       // t0 last written into d_desc
    WorkItem *d_items = nullptr;
    int *d_off = nullptr;        // per-block item ranges of the plan
    int n_items = 0, n_blocks = 0;
    int launch_flags = 0;   // fused-kernel flags of the plan (FUSED_EARLY_NEXT)
    int *d_err = nullptr;
    float *d_aux = nullptr;      // two-pass scratch field
    double *d_part = nullptr;    // diagnostic partials + final
    int diag_blocks = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    bool has_center = false;
    double cx = 0.0, cy = 0.0;
    char err[256] = "";
};

struct lbm_batch {
    std::vector<lbm_sim *> sims;
    std::vector<long long> t_mirror;  // t0 of each batch descriptor as last written
    std::vector<long long> t_stop;    // stop time baked into each batch descriptor
    SimDesc *d_descs = nullptr;
    WorkItem *d_items = nullptr;
    int *d_off = nullptr;
    int n_items = 0;
    // one launch per (storage, variant) group: items [item0, ...) and block
    // ranges off[off0 .. off0 + blocks]
    struct Group { int storage, variant, item0, off0, blocks, flags; };
    std::vector<Group> groups;
    // groups beyond the first run concurrently on their own streams (fork / join)
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gjoin;
    cudaEvent_t fork = nullptr;
    int *d_err = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    long graph_steps = 0;
};

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_err(s->err, "%s failed: %s", #call, cudaGetErrorString(e_));              \
            return LBM_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

namespace {

lbm_status validate(int nx, int ny, const lbm_params *p, char *err) {
    if (!p) { set_err(err, "params is NULL"); return LBM_EINVAL; }
    if (nx < 8 || ny < 4 || nx > (1 << 24) || ny > (1 << 24)) {
        set_err(err, "lattice %dx%d out of range (nx >= 8, ny >= 4)", nx, ny);
        return LBM_EINVAL;
    }
    if (!(p->gamma >= 1.0) || !(p->alpha_b > 0.0 && p->alpha_b < 1.0)) {
        set_err(err, "need gamma >= 1 and 0 < alpha_b < 1");
        return LBM_EINVAL;
    }
    if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5) || !(p->delta > 0.0)) {
        set_err(err, "need tau_r, tau_b > 1/2 and delta > 0");
        return LBM_EINVAL;
    }
    if (!(p->beta >= 0.0 && p->beta <= 1.0) || !(p->sigma >= 0.0)) {
        set_err(err, "need 0 <= beta <= 1 and sigma >= 0");
        return LBM_EINVAL;
    }
    if (p->collision < 0 || p->collision > 1 || p->equilibrium < 0 || p->equilibrium > 1) {
        set_err(err, "unknown collision / equilibrium");
        return LBM_EINVAL;
    }
    if (!(p->bc_x == LBM_BC_PERIODIC || p->bc_x == LBM_BC_INOUT) ||
        !(p->bc_y == LBM_BC_PERIODIC || p->bc_y == LBM_BC_WALL)) {
        set_err(err, "bc_x must be PERIODIC or INOUT, bc_y PERIODIC or WALL");
        return LBM_EINVAL;
    }
    if (p->storage < 0 || p->storage > 2) { set_err(err, "unknown storage"); return LBM_EINVAL; }
    if (p->kernel < 0 || p->kernel > 2) { set_err(err, "unknown kernel"); return LBM_EINVAL; }
    if (p->plan_rows < 0 || p->plan_rows > (1 << 20)) { set_err(err, "plan_rows out of range"); return LBM_EINVAL; }
    if (p->plan < LBM_PLAN_AUTO || p->plan > LBM_PLAN_SPLIT) { set_err(err, "unknown plan kind"); return LBM_EINVAL; }
    if (p->wall_slip != 0 && p->wall_slip != 1) { set_err(err, "wall_slip must be 0 or 1"); return LBM_EINVAL; }
    if (!(p->contact_angle >= 0.0 && p->contact_angle < 3.14159265358979)) {
        set_err(err, "contact_angle must be 0 (off) or in (0, pi) radians");
        return LBM_EINVAL;
    }
    if (p->bc_x == LBM_BC_INOUT && !(p->p_out > 0.0)) {
        set_err(err, "inlet/outlet needs p_out > 0");
        return LBM_EINVAL;
    }
    return LBM_OK;
}

// Ghost columns kept on each side of a row: one 32-byte sector of FP32 values,
// so that the interior columns and the periodic copies are stored in whole
// sectors (a 16-byte FP32 ghost moved less DRAM but put every row's stores off
// the sector grid and measured 4 % slower).
constexpr int GHOST = 8;

int pitch_rho(int nx) { return (nx + 2 * GHOST + 3) / 4 * 4; }   // 16-byte rows of floats

int pitch_dev(int nx, int storage) {
    const int align = 16 / elem_size(storage);
    return (nx + 2 * GHOST + align - 1) / align * align;
}

// FP32 node planes per row: rho_r, rho_b, plus the split-form scalars m, G_x, G_y
// for 16-bit deviations.
int scalar_planes(int storage) { return storage == ST_F32 ? 2 : 5; }

size_t rho_region_bytes(int nx, int ny, int storage) {
    const size_t b = 2ull * (size_t)scalar_planes(storage) * (size_t)ny * pitch_rho(nx) * 4ull;
    return (b + 255) / 256 * 256;
}

size_t dev_region_bytes(int nx, int ny, int storage) {
    return 2ull * 16ull * (size_t)ny * pitch_dev(nx, storage) * (size_t)elem_size(storage);
}

// Per-simulation constants of Sec. 2.1 in the descriptor (float).
constexpr long long NO_STOP = 1LL << 62;

void fill_desc(SimDesc &h, int nx, int ny, const lbm_params *p) {
    memset(&h, 0, sizeof(h));
    h.t_end = NO_STOP;
    h.storage = p->storage;
    h.variant = variant_of(p);
    h.ghost = GHOST;
    h.pitch_r = pitch_rho(nx);
    h.pitch_d = pitch_dev(nx, p->storage);
    h.rho_plane = h.pitch_r;
    h.rho_row = (long long)scalar_planes(p->storage) * h.pitch_r;
    h.rho_buf = (long long)ny * h.rho_row;
    h.dev_plane = h.pitch_d;
    h.dev_row = 16LL * h.pitch_d;
    h.dev_buf = (long long)ny * h.dev_row;
    Phys &f = h.ph;
    f.nx = nx;
    f.ny = ny;
    f.bc_x = p->bc_x;
    f.bc_y = p->bc_y;
    f.inlet_mode = p->inlet_mode;
    f.inlet_period_r = p->inlet_period_r;
    f.inlet_period_b = p->inlet_period_b;
    f.inlet_layer = p->inlet_layer;
    const double alpha_b = p->alpha_b;
    const double alpha_r = 1.0 - (1.0 - alpha_b) / p->gamma;     // Eq. (eq:gammaAlphaBeta)
    const double wr = 1.0 / p->tau_r, wb = 1.0 / p->tau_b;
    const double chi = 2.0 * wr * wb / (wr + wb);
    const double eta = 2.0 * (wr - chi) / p->delta;
    const double lam = 2.0 * (chi - wb) / p->delta;
    f.inv_gamma = (float)(1.0 / p->gamma);
    const double ar[3] = {alpha_r, (1.0 - alpha_r) / 5.0, (1.0 - alpha_r) / 20.0};
    const double ab[3] = {alpha_b, (1.0 - alpha_b) / 5.0, (1.0 - alpha_b) / 20.0};
    for (int c = 0; c < 3; c++) {
        f.phi_r[c] = (float)ar[c];
        f.phi_b[c] = (float)ab[c];
        f.dphi[c] = f.phi_b[c] - f.phi_r[c];
    }
    f.omega_r = (float)wr;
    f.omega_b = (float)wb;
    f.chi = (float)chi;
    f.eta = (float)eta;
    f.kappa = (float)(-eta / (2.0 * p->delta));
    f.lam = (float)lam;
    f.nu = (float)(lam / (2.0 * p->delta));
    f.delta = (float)p->delta;
    f.a_coef = (float)(9.0 * p->sigma / 4.0);                     // Eq. (eq:sigmaIsoAllen)
    f.beta = (float)p->beta;
    f.gx = (float)p->gx;
    f.gy = (float)p->gy;
    f.mrt_lambda = (float)p->mrt_lambda;
    f.c7x = (float)p->c7_factor;
    f.c7y = (float)(p->c7_factor * p->c7_sign);
    const double cs2_r = 3.0 * (1.0 - alpha_r) / 5.0, cs2_b = 3.0 * (1.0 - alpha_b) / 5.0;
    f.cs2_r = (float)cs2_r;
    f.cs2_b = (float)cs2_b;
    f.herm_r = (float)(3.0 * cs2_r - 1.0);
    f.herm_b = (float)(3.0 * cs2_b - 1.0);
    f.q_r = (float)(1.8 * alpha_r - 0.8);
    f.q_b = (float)(1.8 * alpha_b - 0.8);
    f.u_in_r = (float)p->u_in_r;
    f.u_in_b = (float)p->u_in_b;
    f.p_out = (float)p->p_out;
    h.wet.slip = p->wall_slip;
    h.wet.on = p->contact_angle > 0.0 ? 1 : 0;
    h.wet.cos_t = (float)cos(p->contact_angle);
    h.wet.sin_t = (float)sin(p->contact_angle);
}

lbm_status encode_tmap(lbm_sim *s) {
    auto enc = get_encode();
    if (!enc) { set_err(s->err, "cuTensorMapEncodeTiled entry point not available"); return LBM_ECUDA; }
    const int es = elem_size(s->p.storage);
    const CUtensorMapDataType dt = s->p.storage == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : s->p.storage == ST_F16DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint32_t box_w = FUSED_W + 2 * (16 / es);   // halo columns loaded: 4 (FP32) or 8 (16-bit)
    // rows of planes over both buffers: [2][ny][planes] -> one 2D row index
    cuuint32_t estr[2] = {1, 1};
    {
        const cuuint32_t ns = (cuuint32_t)scalar_planes(s->p.storage);
        cuuint64_t dims[2] = {(cuuint64_t)s->h.pitch_r, (cuuint64_t)s->ny * 2 * ns};
        cuuint64_t strides[1] = {(cuuint64_t)s->h.pitch_r * 4};
        cuuint32_t box[2] = {box_w, ns};
        CUresult r = enc(&s->h.tmap_rho, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s->h.rho, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { set_err(s->err, "cuTensorMapEncodeTiled (rho) failed (%d)", (int)r); return LBM_ECUDA; }
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)s->h.pitch_d, (cuuint64_t)s->ny * 2 * 16};
        cuuint64_t strides[1] = {(cuuint64_t)s->h.pitch_d * es};
        cuuint32_t box[2] = {box_w, 16};
        CUresult r = enc(&s->h.tmap_dev, dt, 2, s->h.dev, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { set_err(s->err, "cuTensorMapEncodeTiled (dev) failed (%d)", (int)r); return LBM_ECUDA; }
    }
    return LBM_OK;
}

// ---- work plans: which block marches over which rows of which strip

struct StripRef {
    int sim, x0, w, ny;
    int min_piece;   // shortest row range of this strip worth its 4-row halo
};

struct Plan {
    std::vector<WorkItem> items;
    std::vector<int> off;   // block b owns items [off[b], off[b+1])
    int blocks = 0;
};

// Launch flags for a plan run as the only launch of each step: a plan of one
// piece per block, all of the same width and within one row of the same
// height, lets the next step launch early (its blocks then land on whichever
// SMs free first, which only matters where the pieces differ).
int plan_flags(const Plan &P, bool only_launch) {
    if (!only_launch || P.items.empty() || (int)P.items.size() != P.blocks) return 0;
    int lo = 1 << 30, hi = 0, w0 = P.items[0].w;
    for (const WorkItem &it : P.items) {
        if (it.w != w0) return 0;
        lo = std::min(lo, it.yb - it.ya);
        hi = std::max(hi, it.yb - it.ya);
    }
    return hi - lo <= 1 ? FUSED_EARLY_NEXT : 0;
}

constexpr int MIN_PIECE = 8;   // default shortest row range worth a 4-row halo
constexpr double DEFAULT_ROW_OVERHEAD = 1.0;   // fixed cost of a strip row, in busy warps

void strips_of(std::vector<StripRef> &out, int sim, int nx, int ny, int plan_rows) {
    const int mp = plan_rows > 0 ? plan_rows : MIN_PIECE;
    for (int x0 = 0; x0 < nx; x0 += FUSED_W) out.push_back({sim, x0, std::min(FUSED_W, nx - x0), ny, mp});
}

// Balanced persistent plan: the strip rows are cut into nearly equal shares
// of cost, in order, so a block may march over the end of one strip and the
// start of the next.  A row of a strip costs the warps it keeps busy plus a
// fixed row_overhead (barrier, row loads, edge columns: a narrow strip's row is
// not proportionally cheaper).  The share count is max_blocks, or fewer when
// the strips' own shortest pieces would not fill them.
Plan balanced_plan(const std::vector<StripRef> &strips, int max_blocks, double row_overhead) {
    Plan P;
    double total = 0.0, pieces = 0.0;
    for (const auto &s : strips) {
        const int wc = (s.w + 31) / 32;
        total += (double)s.ny * (wc + row_overhead);
        pieces += (double)s.ny * wc / 4.0 / std::max(1, s.min_piece);
    }
    int B = (int)std::min<double>(max_blocks, std::max(1.0, std::floor(pieces)));
    const double quota = total / B;
    P.off.push_back(0);
    int b = 0;
    double acc = 0.0;
    for (const auto &s : strips) {
        const double wc = (s.w + 31) / 32 + row_overhead;
        const int mp = std::max(1, s.min_piece);
        int y = 0;
        while (y < s.ny) {
            const double left = quota * (b + 1) - acc;
            int take = (int)std::floor(left / wc + 1e-9);
            if (take < mp && b < B - 1 && (int)P.items.size() > P.off.back()) {
                P.off.push_back((int)P.items.size());   // close block b, continue in b + 1
                ++b;
                continue;
            }
            take = std::max(take, mp);
            take = std::min(take, s.ny - y);
            if (s.ny - (y + take) < mp) take = s.ny - y;   // no tiny tail pieces
            WorkItem it{};
            it.sim = s.sim;
            it.x0 = s.x0;
            it.w = s.w;
            it.ya = y;
            it.yb = y + take;
            P.items.push_back(it);
            acc += (double)take * wc;
            y += take;
            if (acc >= quota * (b + 1) - 1e-9 && b < B - 1) {
                P.off.push_back((int)P.items.size());
                ++b;
            }
        }
    }
    while ((int)P.off.size() < B + 1) P.off.push_back((int)P.items.size());
    P.off.back() = (int)P.items.size();
    P.blocks = B;
    return P;
}

// Fixed plan: every strip cut into pieces of `rows` rows, one piece per block.
Plan fixed_plan(const std::vector<StripRef> &strips, int rows) {
    Plan P;
    P.off.push_back(0);
    for (const auto &s : strips)
        for (int y = 0; y < s.ny; y += rows) {
            WorkItem it{};
            it.sim = s.sim;
            it.x0 = s.x0;
            it.w = s.w;
            it.ya = y;
            it.yb = std::min(s.ny, y + rows);
            P.items.push_back(it);
            P.off.push_back((int)P.items.size());
        }
    P.blocks = (int)P.items.size();
    return P;
}

// Split plan: every block gets exactly one segment (a block that starts a
// second segment pays a second prologue and a second wait for its first row
// loads, which costs more than it balances).  Each strip is cut into k_s nearly
// equal pieces, with the k_s chosen so that the costliest piece is as cheap as
// possible while sum k_s <= max_blocks and no piece is shorter than its strip's
// min_piece.  Falls back to the balanced plan when there are more strips than
// blocks.
Plan split_plan(const std::vector<StripRef> &strips, int max_blocks, double row_overhead) {
    if ((int)strips.size() > max_blocks || strips.empty()) return balanced_plan(strips, max_blocks, row_overhead);
    const int n = (int)strips.size();
    std::vector<double> cost(n);
    std::vector<int> kmax(n);
    for (int i = 0; i < n; i++) {
        const auto &s = strips[i];
        cost[i] = (double)s.ny * ((s.w + 31) / 32 + row_overhead);
        kmax[i] = std::max(1, s.ny / std::max(1, s.min_piece));
    }
    auto pieces = [&](double C, std::vector<int> *k) {
        long long tot = 0;
        for (int i = 0; i < n; i++) {
            // clamp in floating point: cost / C overflows an int as C -> 0
            const double q = C > 0.0 ? std::ceil(cost[i] / C - 1e-9) : (double)kmax[i];
            const int ki = q >= (double)kmax[i] ? kmax[i] : std::max(1, (int)q);
            tot += ki;
            if (k) (*k)[i] = ki;
        }
        return tot;
    };
    double lo = 0.0, hi = 0.0;
    for (double c : cost) hi = std::max(hi, c);
    if (pieces(hi, nullptr) > max_blocks) return balanced_plan(strips, max_blocks, row_overhead);
    for (int it = 0; it < 60; it++) {   // smallest piece cost whose piece count fits
        const double mid = 0.5 * (lo + hi);
        if (pieces(mid, nullptr) <= max_blocks) hi = mid;
        else lo = mid;
    }
    std::vector<int> k(n);
    pieces(hi, &k);
    Plan P;
    P.off.push_back(0);
    for (int i = 0; i < n; i++) {
        const auto &s = strips[i];
        const int base = s.ny / k[i], extra = s.ny % k[i];
        int y = 0;
        for (int j = 0; j < k[i]; j++) {
            const int rows = base + (j < extra ? 1 : 0);
            WorkItem it{};
            it.sim = s.sim;
            it.x0 = s.x0;
            it.w = s.w;
            it.ya = y;
            it.yb = y + rows;
            y += rows;
            P.items.push_back(it);
            P.off.push_back((int)P.items.size());
        }
    }
    P.blocks = (int)P.items.size();
    return P;
}

// Work plan of the given kind (lbm_plan_kind) over the strips.
Plan make_plan(const std::vector<StripRef> &strips, int kind, int rows_per_item, int max_blocks, double row_overhead) {
    if (rows_per_item > 0) return fixed_plan(strips, rows_per_item);
    if (kind == LBM_PLAN_BALANCED) return balanced_plan(strips, max_blocks, row_overhead);
    return split_plan(strips, max_blocks, row_overhead);
}

cudaError_t launch_fused_any(int storage, int variant, const SimDesc *descs, const WorkItem *items,
                             const int *item_off, int n_blocks, int off, int flags, int *err, cudaStream_t st) {
    switch (storage) {
    case ST_F32: return fused_launch<float>(variant, descs, items, item_off, n_blocks, off, flags, err, st);
    case ST_F16DEV: return fused_launch<__half>(variant, descs, items, item_off, n_blocks, off, flags, err, st);
    default: return fused_launch<__nv_bfloat16>(variant, descs, items, item_off, n_blocks, off, flags, err, st);
    }
}

// Resident fused blocks per SM for a storage type and collision variant
// (occupancy query), times SMs.
int resident_blocks(int storage, int variant) {
    static int cache[3][N_VARIANTS] = {};
    if (storage < 0 || storage > 2 || variant < 0 || variant >= N_VARIANTS) return 1;
    if (cache[storage][variant]) return cache[storage][variant];
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *k = storage == ST_F32 ? fused_kernel<float>(variant)
                    : storage == ST_F16DEV ? fused_kernel<__half>(variant)
                                           : fused_kernel<__nv_bfloat16>(variant);
    const int smem = storage == ST_F32 ? fused_smem<float>(variant)
                     : storage == ST_F16DEV ? fused_smem<__half>(variant)
                                            : fused_smem<__nv_bfloat16>(variant);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, FUSED_W, smem) != cudaSuccess || per < 1) per = 1;
    if (sms < 1) sms = 1;
    cache[storage][variant] = sms * per;
    return cache[storage][variant];
}

int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}

cudaError_t launch_twopass(lbm_sim *s, int off) {
    const long long n = (long long)s->nx * s->ny;
    switch (s->p.storage) {
    case ST_F32: return twopass_launch<float>(s->h.variant, s->d_desc, off, s->d_aux, n, s->stream);
    case ST_F16DEV: return twopass_launch<__half>(s->h.variant, s->d_desc, off, s->d_aux, n, s->stream);
    default: return twopass_launch<__nv_bfloat16>(s->h.variant, s->d_desc, off, s->d_aux, n, s->stream);
    }
}

// Support kernels dispatched on storage type and on the equilibrium (which
// decides the Zou-He correction term of the open boundaries).
template <typename T, bool H>
void launch_fields_t(lbm_sim *s, int g, double *out) {
    k_fields<T, H><<<g, 256, 0, s->stream>>>(s->d_desc, s->t, out);
}

template <typename T>
void launch_fields_s(lbm_sim *s, int g, double *out) {
    if (s->h.variant & CV_HERMITE) launch_fields_t<T, true>(s, g, out);
    else launch_fields_t<T, false>(s, g, out);
}

void launch_fields(lbm_sim *s, int g, double *out) {
    switch (s->p.storage) {
    case ST_F32: launch_fields_s<float>(s, g, out); break;
    case ST_F16DEV: launch_fields_s<__half>(s, g, out); break;
    default: launch_fields_s<__nv_bfloat16>(s, g, out); break;
    }
}

template <typename T>
void launch_read_pops_s(lbm_sim *s, int g, double *out) {
    if (s->h.variant & CV_HERMITE) k_read_pops<T, true><<<g, 256, 0, s->stream>>>(s->d_desc, s->t, out);
    else k_read_pops<T, false><<<g, 256, 0, s->stream>>>(s->d_desc, s->t, out);
}

void launch_read_pops(lbm_sim *s, int g, double *out) {
    switch (s->p.storage) {
    case ST_F32: launch_read_pops_s<float>(s, g, out); break;
    case ST_F16DEV: launch_read_pops_s<__half>(s, g, out); break;
    default: launch_read_pops_s<__nv_bfloat16>(s, g, out); break;
    }
}

template <typename T, bool H>
void launch_diag_t(lbm_sim *s, int pass, double cx, double cy, double rin, double rout) {
    k_diag<T, H><<<s->diag_blocks, DIAG_THREADS, 0, s->stream>>>(s->d_desc, s->t, pass, cx, cy, rin, rout, s->d_part);
}

template <typename T>
void launch_diag_s(lbm_sim *s, int pass, double cx, double cy, double rin, double rout) {
    if (s->h.variant & CV_HERMITE) launch_diag_t<T, true>(s, pass, cx, cy, rin, rout);
    else launch_diag_t<T, false>(s, pass, cx, cy, rin, rout);
}

void launch_diag(lbm_sim *s, int pass, double cx, double cy, double rin, double rout) {
    switch (s->p.storage) {
    case ST_F32: launch_diag_s<float>(s, pass, cx, cy, rin, rout); break;
    case ST_F16DEV: launch_diag_s<__half>(s, pass, cx, cy, rin, rout); break;
    default: launch_diag_s<__nv_bfloat16>(s, pass, cx, cy, rin, rout); break;
    }
}

template <typename T>
void launch_slug_profile_s(lbm_sim *s, double *out) {
    const int g = std::max(1, (s->nx + 127) / 128);
    if (s->h.variant & CV_HERMITE) k_slug_profile<T, true><<<g, 128, 0, s->stream>>>(s->d_desc, s->t, out);
    else k_slug_profile<T, false><<<g, 128, 0, s->stream>>>(s->d_desc, s->t, out);
}

void launch_slug_profile(lbm_sim *s, double *out) {
    switch (s->p.storage) {
    case ST_F32: launch_slug_profile_s<float>(s, out); break;
    case ST_F16DEV: launch_slug_profile_s<__half>(s, out); break;
    default: launch_slug_profile_s<__nv_bfloat16>(s, out); break;
    }
}

// Bubble / slug geometry of lbm_slug from the column profile g and the
// centreline profile pc (both nx values).  Zeros of pc are located on the
// linear interpolant between nodes x and x + 1.
void slug_from_profile(const double *g, const double *pc, int nx, int ny, bool periodic, lbm_slug *o) {
    struct Cross { double x; bool tail; };
    std::vector<Cross> c;
    const int last = periodic ? nx : nx - 1;
    for (int x = 0; x < last; x++) {
        const int x1 = x + 1 == nx ? 0 : x + 1;
        const double a = pc[x], b = pc[x1];
        if ((a >= 0.0) == (b >= 0.0)) continue;
        double pos = x + a / (a - b);
        if (pos >= nx) pos -= nx;
        c.push_back({pos, a >= 0.0});
    }
    size_t start = 0;                  // the walk starts at the first tail
    while (start < c.size() && !c[start].tail) start++;
    if (start == c.size()) return;
    const size_t m = c.size();
    // bubbles: a tail followed by a nose (periodic lines wrap around)
    std::vector<double> tails, noses;
    for (size_t j = 0; j < m; j++) {
        if (!periodic && start + j + 1 >= m) break;
        const Cross &a = c[(start + j) % m], &b = c[(start + j + 1) % m];
        if (a.tail && !b.tail) {
            tails.push_back(a.x);
            noses.push_back(b.x);
        }
    }
    auto fwd = [&](double a, double b) {   // distance from a forward (+x) to b
        const double d = b - a;
        return periodic && d < 0.0 ? d + nx : d;
    };
    auto g_at = [&](double x) {            // g linear between columns
        if (periodic) x = std::fmod(x, (double)nx);
        x = std::min(std::max(x, 0.0), (double)(nx - 1) + (periodic ? 1.0 : 0.0));
        const int i0 = std::min((int)std::floor(x), nx - 1);
        const int i1 = i0 + 1 < nx ? i0 + 1 : (periodic ? 0 : nx - 1);
        const double f = x - i0;
        return (1.0 - f) * g[i0] + f * g[i1];
    };
    const size_t nb = tails.size();
    double sb = 0.0, sf = 0.0, ss = 0.0;
    int ns = 0;
    for (size_t j = 0; j < nb; j++) {
        const double len = fwd(tails[j], noses[j]);
        sb += len;
        sf += 0.5 * (ny - g_at(tails[j] + 0.5 * len));
        if (j + 1 < nb) {
            ss += fwd(noses[j], tails[j + 1]);
            ns++;
        } else if (periodic) {
            ss += fwd(noses[j], tails[0]);   // around the line to the first bubble
            ns++;
        }
        if (j < LBM_SLUG_MAX) {
            o->x_tail[j] = tails[j];
            o->x_nose[j] = noses[j];
        }
    }
    o->n_bubbles = (int)nb;
    o->n_slugs = ns;
    if (nb > 0) {
        o->bubble_len = sb / nb;
        o->film = sf / nb;
    }
    if (ns > 0) o->slug_len = ss / ns;
}

bool use_fused(const lbm_sim *s) { return s->p.kernel != LBM_KERNEL_TWOPASS; }

lbm_status sync_t0(lbm_sim *s) {
    if (s->dev_t0 != s->t) {
        k_set_times<<<1, 32, 0, s->stream>>>(s->d_desc, s->t, s->h.t_end);
        CK(cudaGetLastError());
        s->dev_t0 = s->t;
    }
    return LBM_OK;
}

lbm_status check_err_word(lbm_sim *s, int *d_err) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (h & ERR_TIMEOUT) { set_err(s->err, "a bounded device wait timed out"); return LBM_ETIMEOUT; }
    if (h & ERR_BADITEM) { set_err(s->err, "invalid work item"); return LBM_EINVAL; }
    return LBM_OK;
}

// Launch `n` steps of a single simulation directly (no graph).
lbm_status step_direct(lbm_sim *s, long n) {
    for (long j = 0; j < n; j++) {
        if (use_fused(s)) {
            CK(launch_fused_any(s->p.storage, s->h.variant, s->d_desc, s->d_items, s->d_off, s->n_blocks, (int)j,
                                s->launch_flags, s->d_err, s->stream));
        } else {
            CK(launch_twopass(s, (int)j));
        }
    }
    k_advance<<<1, 32, 0, s->stream>>>(s->d_desc, 1, n);
    CK(cudaGetLastError());
    return LBM_OK;
}

constexpr int GRAPH_CHUNK = 32;

// Upload `nfields` host arrays of n doubles and build the t = 0 state from them:
// 4 fields (rho_r, rho_b, ux, uy) -> equilibria, or 1 array of 18 n populations.
lbm_status init_from_host(lbm_sim *s, const double *const *arrays, int narrays, size_t per_array) {
    double *d = nullptr;
    CK(cudaMallocAsync(&d, narrays * per_array * sizeof(double), s->stream));
    for (int q = 0; q < narrays; q++)
        CK(cudaMemcpyAsync(d + q * per_array, arrays[q], per_array * sizeof(double), cudaMemcpyHostToDevice,
                           s->stream));
    CK(cudaMemsetAsync(s->pop, 0, s->pop_bytes, s->stream));
    s->t = 0;
    lbm_status st = sync_t0(s);
    if (st != LBM_OK) return st;
    const size_t n = (size_t)s->nx * s->ny;
    const int g = grid_for((long long)n, 256);
    const double *f0 = d, *f1 = d + n, *f2 = d + 2 * n, *f3 = d + 3 * n, *pops = nullptr;
    if (narrays == 1) {
        pops = d;
        f0 = f1 = f2 = f3 = nullptr;
    }
    switch (s->p.storage) {
    case ST_F32: k_init<float><<<g, 256, 0, s->stream>>>(s->d_desc, f0, f1, f2, f3, pops); break;
    case ST_F16DEV: k_init<__half><<<g, 256, 0, s->stream>>>(s->d_desc, f0, f1, f2, f3, pops); break;
    default: k_init<__nv_bfloat16><<<g, 256, 0, s->stream>>>(s->d_desc, f0, f1, f2, f3, pops); break;
    }
    CK(cudaGetLastError());
    CK(cudaFreeAsync(d, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status set_fields_from_host(lbm_sim *s, const double *rr, const double *rb, const double *ux,
                                const double *uy) {
    const double *a[4] = {rr, rb, ux, uy};
    return init_from_host(s, a, 4, (size_t)s->nx * s->ny);
}

lbm_status create_common(int nx, int ny, const lbm_params *p, void *buf, size_t bytes, void *stream,
                         bool external, lbm_sim **out) {
    if (!out) { set_err(g_create_err, "out is NULL"); return LBM_EINVAL; }
    *out = nullptr;
    lbm_status v = validate(nx, ny, p, g_create_err);
    if (v != LBM_OK) return v;
    lbm_sim *s = new lbm_sim();
    s->nx = nx;
    s->ny = ny;
    s->p = *p;
    cudaGetDevice(&s->dev);
    fill_desc(s->h, nx, ny, p);
    s->pop_bytes = lbm_bytes_required(nx, ny, p);
    auto fail = [&](lbm_status st) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", s->err);
        lbm_destroy(s);
        return st;
    };
    if (external) {
        if (!buf || bytes < s->pop_bytes || (reinterpret_cast<uintptr_t>(buf) & 255)) {
            set_err(s->err, "caller buffer NULL, smaller than %zu bytes or not 256-byte aligned", s->pop_bytes);
            return fail(bytes < s->pop_bytes ? LBM_ENOMEM : LBM_EINVAL);
        }
        s->pop = buf;
        s->own_pop = false;
        s->stream = reinterpret_cast<cudaStream_t>(stream);
        s->own_stream = false;
    } else {
        if (cudaMalloc(&s->pop, s->pop_bytes) != cudaSuccess) {
            cudaGetLastError();
            set_err(s->err, "cudaMalloc of %zu bytes failed", s->pop_bytes);
            return fail(LBM_ENOMEM);
        }
        s->own_pop = true;
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_err(s->err, "cudaStreamCreate failed");
            return fail(LBM_ECUDA);
        }
        s->own_stream = true;
    }
    s->h.rho = reinterpret_cast<float *>(s->pop);
    s->h.dev = static_cast<char *>(s->pop) + rho_region_bytes(nx, ny, p->storage);
    if (encode_tmap(s) != LBM_OK) return fail(LBM_ECUDA);
    if (cudaMalloc(&s->d_desc, sizeof(SimDesc)) != cudaSuccess || cudaMalloc(&s->d_err, sizeof(int)) != cudaSuccess) {
        set_err(s->err, "cudaMalloc of descriptor failed");
        return fail(LBM_ENOMEM);
    }
    {
        std::vector<StripRef> strips;
        strips_of(strips, 0, nx, ny, p->plan_rows);
        Plan P = make_plan(strips, p->plan, 0, resident_blocks(p->storage, variant_of(p)), DEFAULT_ROW_OVERHEAD);
        s->n_items = (int)P.items.size();
        s->n_blocks = P.blocks;
        s->launch_flags = plan_flags(P, true);
        if (cudaMalloc(&s->d_items, P.items.size() * sizeof(WorkItem)) != cudaSuccess ||
            cudaMalloc(&s->d_off, P.off.size() * sizeof(int)) != cudaSuccess ||
            cudaMemcpy(s->d_items, P.items.data(), P.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(s->d_off, P.off.data(), P.off.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
            set_err(s->err, "work plan upload failed");
            return fail(LBM_ENOMEM);
        }
    }
    const size_t nn = (size_t)nx * ny;
    if (p->kernel == LBM_KERNEL_TWOPASS &&
        cudaMalloc(&s->d_aux, AUX_FIELDS * nn * sizeof(float)) != cudaSuccess) {
        set_err(s->err, "cudaMalloc of scratch field failed");
        return fail(LBM_ENOMEM);
    }
    s->diag_blocks = grid_for((long long)nn, DIAG_THREADS);
    if (cudaMalloc(&s->d_part, ((size_t)s->diag_blocks + 1) * DIAG_NQ * sizeof(double)) != cudaSuccess) {
        set_err(s->err, "cudaMalloc of diagnostic scratch failed");
        return fail(LBM_ENOMEM);
    }
    if (cudaMemcpyAsync(s->d_desc, &s->h, sizeof(SimDesc), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->pop, 0, s->pop_bytes, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        set_err(s->err, "initial uploads failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(LBM_ECUDA);
    }
    s->dev_t0 = 0;
    *out = s;
    return LBM_OK;
}

}  // namespace

namespace lbm {

lbm_status host_validate(int nx, int ny, const lbm_params *p, char *err) { return validate(nx, ny, p, err); }

void host_fill_desc(SimDesc &h, int nx, int ny, const lbm_params *p, void *state) {
    fill_desc(h, nx, ny, p);
    h.rho = reinterpret_cast<float *>(state);
    h.dev = static_cast<char *>(state) + rho_region_bytes(nx, ny, p->storage);
}

void host_set_global_error(const char *msg) { snprintf(g_create_err, sizeof(g_create_err), "%s", msg); }

}  // namespace lbm

extern "C" {

lbm_status lbm_default_params(lbm_params *p) {
    if (!p) return LBM_EINVAL;
    memset(p, 0, sizeof(*p));
    p->gamma = 1.0;
    p->alpha_b = 0.2;
    p->tau_r = 1.0;
    p->tau_b = 1.0;
    p->delta = 0.1;
    p->sigma = 0.005;
    p->beta = 0.99;
    p->mrt_lambda = 0.8;
    p->c7_sign = -1.0;
    p->c7_factor = 1.0;
    return LBM_OK;
}

size_t lbm_bytes_required(int nx, int ny, const lbm_params *p) {
    char tmp[256];
    if (validate(nx, ny, p, tmp) != LBM_OK) return 0;
    return rho_region_bytes(nx, ny, p->storage) + dev_region_bytes(nx, ny, p->storage);
}

lbm_status lbm_create(int nx, int ny, const lbm_params *p, lbm_sim **out) {
    return create_common(nx, ny, p, nullptr, 0, nullptr, false, out);
}

lbm_status lbm_create_ex(int nx, int ny, const lbm_params *p, void *dev_buf, size_t bytes, void *cuda_stream,
                         lbm_sim **out) {
    return create_common(nx, ny, p, dev_buf, bytes, cuda_stream, true, out);
}

lbm_status lbm_init_fields(lbm_sim *s, const double *rho_r, const double *rho_b, const double *ux,
                           const double *uy) {
    if (!s) return LBM_EINVAL;
    if (!rho_r || !rho_b || !ux || !uy) { set_err(s->err, "NULL field"); return LBM_EINVAL; }
    return set_fields_from_host(s, rho_r, rho_b, ux, uy);
}

lbm_status lbm_init_populations(lbm_sim *s, const double *pops) {
    if (!s) return LBM_EINVAL;
    if (!pops) { set_err(s->err, "NULL populations"); return LBM_EINVAL; }
    const double *a[1] = {pops};
    return init_from_host(s, a, 1, 18ull * s->nx * s->ny);
}

lbm_status lbm_init_bubble(lbm_sim *s, double cx, double cy, double R) {
    if (!s) return LBM_EINVAL;
    if (!(R > 0.0)) { set_err(s->err, "R must be > 0"); return LBM_EINVAL; }
    const int nx = s->nx, ny = s->ny;
    std::vector<double> rr((size_t)nx * ny), rb(rr.size()), z(rr.size(), 0.0);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double dx = std::fabs(x - cx), dy = std::fabs(y - cy);
            if (s->p.bc_x == LBM_BC_PERIODIC) dx = std::min(dx, nx - dx);
            if (s->p.bc_y == LBM_BC_PERIODIC) dy = std::min(dy, ny - dy);
            const bool in = dx * dx + dy * dy < R * R;
            rr[(size_t)y * nx + x] = in ? 0.0 : s->p.gamma;
            rb[(size_t)y * nx + x] = in ? 1.0 : 0.0;
        }
    lbm_status st = set_fields_from_host(s, rr.data(), rb.data(), z.data(), z.data());
    if (st == LBM_OK) {
        s->has_center = true;
        s->cx = cx;
        s->cy = cy;
    }
    return st;
}

lbm_status lbm_init_slug(lbm_sim *s, int n_bubbles, double bubble_len, double bubble_h, int poiseuille) {
    if (!s) return LBM_EINVAL;
    if (n_bubbles < 0 || bubble_len < 0 || bubble_h < 0) { set_err(s->err, "negative slug geometry"); return LBM_EINVAL; }
    const int nx = s->nx, ny = s->ny;
    std::vector<double> rr((size_t)nx * ny), rb(rr.size()), ux(rr.size(), 0.0), uy(rr.size(), 0.0);
    const double r = bubble_h / 2.0, yc = (ny - 1) / 2.0, pitch = (double)nx / std::max(n_bubbles, 1);
    const double nu_l = (s->p.tau_r - 0.5) / 3.0;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            bool gas = false;
            for (int b = 0; b < n_bubbles; b++) {
                const double x0 = b * pitch + (pitch - bubble_len) / 2.0;
                const double xs = std::fmod(std::fmod(x - x0, (double)nx) + nx, (double)nx);
                const double dy = y - yc;
                const bool core = xs >= r && xs <= bubble_len - r && std::fabs(dy) < r;
                const bool c1 = (xs - r) * (xs - r) + dy * dy < r * r;
                const bool c2 = (xs - (bubble_len - r)) * (xs - (bubble_len - r)) + dy * dy < r * r;
                gas = gas || core || (xs <= bubble_len && (c1 || c2));
            }
            const size_t k = (size_t)y * nx + x;
            rr[k] = gas ? 0.0 : s->p.gamma;
            rb[k] = gas ? 1.0 : 0.0;
            if (poiseuille && s->p.gx != 0.0) {
                const double Y = y + 0.5;
                ux[k] = s->p.gx / (2.0 * nu_l) * Y * (ny - Y);
            }
        }
    return set_fields_from_host(s, rr.data(), rb.data(), ux.data(), uy.data());
}

lbm_status lbm_step(lbm_sim *s, long n) {
    if (!s) return LBM_EINVAL;
    if (n < 0) { set_err(s->err, "n < 0"); return LBM_EINVAL; }
    if (n == 0) return LBM_OK;
    lbm_status st = sync_t0(s);
    if (st != LBM_OK) return st;
    long done = 0;
    // a captured graph of GRAPH_CHUNK steps (+ time advance), replayed
    if (n >= GRAPH_CHUNK && s->stream != nullptr) {
        if (!s->graph) {
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            lbm_status cs = step_direct(s, GRAPH_CHUNK);
            cudaError_t ce = cudaStreamEndCapture(s->stream, &g);
            if (cs != LBM_OK) return cs;
            CK(ce);
            CK(cudaGraphInstantiate(&s->graph, g, 0));
            cudaGraphDestroy(g);
            s->graph_steps = GRAPH_CHUNK;
        }
        for (; done + GRAPH_CHUNK <= n; done += GRAPH_CHUNK) CK(cudaGraphLaunch(s->graph, s->stream));
    }
    if (done < n) {
        st = step_direct(s, n - done);
        if (st != LBM_OK) return st;
    }
    const long long t_old = s->t;
    s->t = std::min(t_old + n, s->h.t_end);   // steps at or after the stop time were skipped
    s->dev_t0 = t_old + n;                    // what the device descriptor now holds
    return LBM_OK;
}

lbm_status lbm_set_stop(lbm_sim *s, long long t_end) {
    if (!s) return LBM_EINVAL;
    const long long te = t_end < 0 ? NO_STOP : t_end;
    if (te < s->t) { set_err(s->err, "stop time %lld is before the current time %lld", te, s->t); return LBM_EINVAL; }
    s->h.t_end = te;
    CK(cudaMemcpyAsync(&s->d_desc->t_end, &s->h.t_end, sizeof(long long), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->dev_t0 = -1;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_sim *s) {
    if (!s) return LBM_EINVAL;
    CK(cudaStreamSynchronize(s->stream));
    return check_err_word(s, s->d_err);
}

long long lbm_time(const lbm_sim *s) { return s ? s->t : -1; }

lbm_status lbm_read_fields(lbm_sim *s, double *rho_r, double *rho_b, double *ux, double *uy, double *p) {
    if (!s) return LBM_EINVAL;
    const size_t n = (size_t)s->nx * s->ny;
    double *d = nullptr;
    CK(cudaMallocAsync(&d, 5 * n * sizeof(double), s->stream));
    const int g = grid_for((long long)n, 256);
    launch_fields(s, g, d);
    CK(cudaGetLastError());
    double *outs[5] = {rho_r, rho_b, ux, uy, p};
    for (int q = 0; q < 5; q++)
        if (outs[q]) CK(cudaMemcpyAsync(outs[q], d + q * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(d, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return check_err_word(s, s->d_err);
}

lbm_status lbm_read_populations(lbm_sim *s, double *pops) {
    if (!s) return LBM_EINVAL;
    if (!pops) { set_err(s->err, "NULL populations"); return LBM_EINVAL; }
    const size_t n = (size_t)s->nx * s->ny;
    double *d = nullptr;
    CK(cudaMallocAsync(&d, 18 * n * sizeof(double), s->stream));
    launch_read_pops(s, grid_for((long long)n, 256), d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pops, d, 18 * n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(d, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return check_err_word(s, s->d_err);
}

lbm_status lbm_diagnostics(lbm_sim *s, lbm_diag *out) {
    if (!s || !out) return LBM_EINVAL;
    memset(out, 0, sizeof(*out));
    double h[DIAG_NQ];
    double *fin = s->d_part + (size_t)s->diag_blocks * DIAG_NQ;
    auto run = [&](int pass, double cx, double cy, double rin, double rout) -> lbm_status {
        launch_diag(s, pass, cx, cy, rin, rout);
        CK(cudaGetLastError());
        k_diag_final<<<1, 32, 0, s->stream>>>(s->d_part, s->diag_blocks, fin);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h, fin, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        return LBM_OK;
    };
    lbm_status st = run(0, 0, 0, 0, 0);
    if (st != LBM_OK) return st;
    out->t = s->t;
    out->mass_r = h[0];
    out->mass_b = h[1];
    out->mom_x = h[2];
    out->mom_y = h[3];
    out->area_b = h[4];
    out->max_u = h[5];
    out->cx_b = h[4] > 0 ? h[6] / h[4] : 0.0;
    out->cy_b = h[4] > 0 ? h[7] / h[4] : 0.0;
    out->ux_b = h[4] > 0 ? h[8] / h[4] : 0.0;
    out->ux_r = h[10] > 0 ? h[9] / h[10] : 0.0;
    out->nonfinite = (long long)h[11];
    out->r_eff = std::sqrt(std::max(h[4], 0.0) / M_PI);
    const double cx = s->has_center ? s->cx : out->cx_b, cy = s->has_center ? s->cy : out->cy_b;
    st = run(1, cx, cy, out->r_eff / 2.0, out->r_eff + 8.0);
    if (st != LBM_OK) return st;
    out->p_in = h[1] > 0 ? h[0] / h[1] : 0.0;
    out->p_out = h[3] > 0 ? h[2] / h[3] : 0.0;
    out->dp = out->p_in - out->p_out;
    st = check_err_word(s, s->d_err);
    if (st != LBM_OK) return st;
    if (out->nonfinite > 0) {
        set_err(s->err, "%lld non-finite nodes at t = %lld", out->nonfinite, s->t);
        return LBM_EUNSTABLE;
    }
    return LBM_OK;
}

lbm_status lbm_slug_geometry(lbm_sim *s, lbm_slug *out, double *gas) {
    if (!s || !out) return LBM_EINVAL;
    memset(out, 0, sizeof(*out));
    const int nx = s->nx;
    std::vector<double> h(2 * (size_t)nx);
    double *d = nullptr;
    CK(cudaMallocAsync(&d, 2 * (size_t)nx * sizeof(double), s->stream));
    launch_slug_profile(s, d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h.data(), d, 2 * (size_t)nx * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaFreeAsync(d, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    out->t = s->t;
    slug_from_profile(h.data(), h.data() + nx, nx, s->ny, s->p.bc_x == LBM_BC_PERIODIC, out);
    if (gas) memcpy(gas, h.data(), (size_t)nx * sizeof(double));
    return check_err_word(s, s->d_err);
}

size_t lbm_state_bytes(const lbm_sim *s) { return s ? s->pop_bytes + sizeof(long long) : 0; }

lbm_status lbm_save_state(lbm_sim *s, void *host, size_t bytes) {
    if (!s || !host) return LBM_EINVAL;
    if (bytes < lbm_state_bytes(s)) { set_err(s->err, "state buffer too small"); return LBM_ENOMEM; }
    memcpy(host, &s->t, sizeof(long long));
    CK(cudaMemcpyAsync(static_cast<char *>(host) + sizeof(long long), s->pop, s->pop_bytes, cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_sim *s, const void *host, size_t bytes) {
    if (!s || !host) return LBM_EINVAL;
    if (bytes < lbm_state_bytes(s)) { set_err(s->err, "state buffer too small"); return LBM_ENOMEM; }
    long long t;
    memcpy(&t, host, sizeof(long long));
    if (t < 0) { set_err(s->err, "corrupt state (t < 0)"); return LBM_EINVAL; }
    CK(cudaMemcpyAsync(s->pop, static_cast<const char *>(host) + sizeof(long long), s->pop_bytes,
                       cudaMemcpyHostToDevice, s->stream));
    s->t = t;
    lbm_status st = sync_t0(s);
    if (st != LBM_OK) return st;
    CK(cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

const char *lbm_last_error(const lbm_sim *s) { return s ? s->err : g_create_err; }

void lbm_destroy(lbm_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->own_pop && s->pop) cudaFree(s->pop);
    cudaFree(s->d_desc);
    cudaFree(s->d_items);
    cudaFree(s->d_off);
    cudaFree(s->d_err);
    cudaFree(s->d_aux);
    cudaFree(s->d_part);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// ------------------------------------------------------------------ batches

lbm_status lbm_batch_create(lbm_sim *const *sims, int n, int rows_per_item, lbm_batch **out) {
    lbm_batch_opts o{};
    o.rows_per_item = rows_per_item;
    o.row_overhead = -1.0f;
    o.plan = LBM_PLAN_AUTO;
    o.member_plan_rows = nullptr;
    return lbm_batch_create_ex(sims, n, &o, out);
}

lbm_status lbm_plan_preview(const int *nx, const int *ny, const int *plan_rows, int n, const lbm_batch_opts *opts,
                            int max_blocks, int *n_items, int *n_blocks, int *items, int capacity) {
    if (!nx || !ny || n <= 0 || !opts || max_blocks <= 0 || !n_items || !n_blocks || capacity < 0 ||
        (capacity > 0 && !items))
        return LBM_EINVAL;
    if (opts->rows_per_item < 0 || !(opts->row_overhead <= 64.0f) || opts->plan < LBM_PLAN_AUTO ||
        opts->plan > LBM_PLAN_SPLIT)
        return LBM_EINVAL;
    std::vector<StripRef> strips;
    for (int i = 0; i < n; i++) {
        const int pr = opts->member_plan_rows ? opts->member_plan_rows[i] : (plan_rows ? plan_rows[i] : 0);
        if (nx[i] < 1 || ny[i] < 1 || pr < 0 || pr > (1 << 20)) return LBM_EINVAL;
        strips_of(strips, i, nx[i], ny[i], pr);
    }
    const double ovh = opts->row_overhead < 0.0f ? DEFAULT_ROW_OVERHEAD : (double)opts->row_overhead;
    const Plan P = make_plan(strips, opts->plan, opts->rows_per_item, max_blocks, ovh);
    *n_items = (int)P.items.size();
    *n_blocks = P.blocks;
    for (int b = 0; b < P.blocks; b++)
        for (int q = P.off[b]; q < P.off[b + 1]; q++)
            if (q < capacity) {
                const WorkItem &it = P.items[q];
                int *o = items + 6 * q;
                o[0] = it.sim;
                o[1] = it.x0;
                o[2] = it.w;
                o[3] = it.ya;
                o[4] = it.yb;
                o[5] = b;
            }
    return LBM_OK;
}

lbm_status lbm_batch_create_ex(lbm_sim *const *sims, int n, const lbm_batch_opts *opts, lbm_batch **out) {
    if (!out || !sims || n <= 0 || !opts) { set_err(g_create_err, "empty batch or no options"); return LBM_EINVAL; }
    const int rows_per_item = opts->rows_per_item;
    const double row_overhead = opts->row_overhead < 0.0f ? DEFAULT_ROW_OVERHEAD : (double)opts->row_overhead;
    if (rows_per_item < 0 || !(row_overhead <= 64.0) || opts->plan < LBM_PLAN_AUTO || opts->plan > LBM_PLAN_SPLIT) {
        set_err(g_create_err, "batch options out of range");
        return LBM_EINVAL;
    }
    if (opts->member_plan_rows)
        for (int i = 0; i < n; i++)
            if (opts->member_plan_rows[i] < 0 || opts->member_plan_rows[i] > (1 << 20)) {
                set_err(g_create_err, "member_plan_rows[%d] out of range", i);
                return LBM_EINVAL;
            }
    *out = nullptr;
    long long strip_rows = 0;
    for (int i = 0; i < n; i++) {
        if (!sims[i] || sims[i]->dev != sims[0]->dev) {
            set_err(g_create_err, "batch members must exist and share a device");
            return LBM_EINVAL;
        }
        strip_rows += (long long)((sims[i]->nx + FUSED_W - 1) / FUSED_W) * sims[i]->ny;
    }
    lbm_batch *b = new lbm_batch();
    b->sims.assign(sims, sims + n);
    b->stream = sims[0]->stream;
    std::vector<SimDesc> descs(n);
    std::vector<WorkItem> items;
    for (int i = 0; i < n; i++) {
        descs[i] = sims[i]->h;
        descs[i].t0 = sims[i]->t;
        b->t_mirror.push_back(sims[i]->t);
        b->t_stop.push_back(sims[i]->h.t_end);
    }
    // items grouped by (storage, variant): one launch per group and step, each
    // planned for all resident blocks (splitting the blocks between the groups'
    // concurrent launches in proportion to their cost measured 1.8x slower)
    std::vector<int> offs;
    for (int st = 0; st < 3; st++)
        for (int cv = 0; cv < N_VARIANTS; cv++) {
            std::vector<StripRef> strips;
            for (int i = 0; i < n; i++)
                if (sims[i]->p.storage == st && sims[i]->h.variant == cv)
                    strips_of(strips, i, sims[i]->nx, sims[i]->ny,
                              opts->member_plan_rows ? opts->member_plan_rows[i] : sims[i]->p.plan_rows);
            if (strips.empty()) continue;
            Plan P = make_plan(strips, opts->plan, rows_per_item, resident_blocks(st, cv), row_overhead);
            lbm_batch::Group g{st, cv, (int)items.size(), (int)offs.size(), P.blocks, plan_flags(P, true)};
            for (int &o : P.off) o += g.item0;
            items.insert(items.end(), P.items.begin(), P.items.end());
            offs.insert(offs.end(), P.off.begin(), P.off.end());
            b->groups.push_back(g);
        }
    if (b->groups.size() > 1)   // concurrent launch groups: no early launch of the next step
        for (auto &g : b->groups) g.flags = 0;
    b->n_items = (int)items.size();
    if (cudaMalloc(&b->d_descs, n * sizeof(SimDesc)) != cudaSuccess ||
        cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem)) != cudaSuccess ||
        cudaMalloc(&b->d_off, offs.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(b->d_descs, descs.data(), n * sizeof(SimDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_off, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess) {
        set_err(g_create_err, "batch allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
        lbm_batch_destroy(b);
        return LBM_ENOMEM;
    }
    for (size_t g = 1; g < b->groups.size(); g++) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            set_err(g_create_err, "batch stream creation failed");
            lbm_batch_destroy(b);
            return LBM_ECUDA;
        }
        b->gstreams.push_back(st);
        b->gjoin.push_back(ev);
    }
    if (b->groups.size() > 1 && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        set_err(g_create_err, "batch event creation failed");
        lbm_batch_destroy(b);
        return LBM_ECUDA;
    }
    // work queued on member streams must be complete before the batch runs on sims[0]'s stream
    for (int i = 0; i < n; i++) cudaStreamSynchronize(sims[i]->stream);
    *out = b;
    return LBM_OK;
}

int lbm_batch_items(const lbm_batch *b) { return b ? b->n_items : 0; }

lbm_status lbm_batch_step(lbm_batch *b, long n, int use_graph) {
    if (!b) return LBM_EINVAL;
    lbm_sim *s = b->sims[0];
    if (n < 0) { set_err(s->err, "n < 0"); return LBM_EINVAL; }
    if (n == 0) return LBM_OK;
    // resynchronise the descriptors of members stepped outside the batch (their
    // logical time no longer matches the batch descriptor's t0, clamped at the
    // stop) or given a new stop time since the batch last ran
    for (size_t i = 0; i < b->sims.size(); i++) {
        lbm_sim *m = b->sims[i];
        if (std::min(b->t_mirror[i], m->h.t_end) != m->t || b->t_stop[i] != m->h.t_end) {
            k_set_times<<<1, 32, 0, b->stream>>>(b->d_descs + i, m->t, m->h.t_end);
            CK(cudaGetLastError());
            b->t_mirror[i] = m->t;
        }
    }
    const int nsims = (int)b->sims.size();
    // Groups are independent simulations: each runs its k steps on its own stream,
    // forked from and joined back into the batch stream (running them one after
    // another on the batch stream, each with the whole GPU, was 5 % slower).
    auto run = [&](long k) -> lbm_status {
        if (b->groups.size() > 1) CK(cudaEventRecord(b->fork, b->stream));
        for (size_t gi = 0; gi < b->groups.size(); gi++) {
            const auto &g = b->groups[gi];
            cudaStream_t st = gi == 0 ? b->stream : b->gstreams[gi - 1];
            if (gi > 0) CK(cudaStreamWaitEvent(st, b->fork, 0));
            for (long j = 0; j < k; j++)
                CK(launch_fused_any(g.storage, g.variant, b->d_descs, b->d_items, b->d_off + g.off0, g.blocks, (int)j,
                                    g.flags, b->d_err, st));
            if (gi > 0) {
                CK(cudaEventRecord(b->gjoin[gi - 1], st));
                CK(cudaStreamWaitEvent(b->stream, b->gjoin[gi - 1], 0));
            }
        }
        k_advance<<<(nsims + 127) / 128, 128, 0, b->stream>>>(b->d_descs, nsims, k);
        CK(cudaGetLastError());
        return LBM_OK;
    };
    if (use_graph && b->stream != nullptr) {
        if (!b->graph || b->graph_steps != n) {
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            lbm_status cs = run(n);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (cs != LBM_OK) return cs;
            CK(ce);
            CK(cudaGraphInstantiate(&b->graph, g, 0));
            cudaGraphDestroy(g);
            b->graph_steps = n;
        }
        CK(cudaGraphLaunch(b->graph, b->stream));
    } else {
        lbm_status st = run(n);
        if (st != LBM_OK) return st;
    }
    for (size_t i = 0; i < b->sims.size(); i++) {
        lbm_sim *m = b->sims[i];
        const long long tb = b->t_mirror[i] + n;             // batch descriptor's t0 now
        m->t = std::min(m->t + n, m->h.t_end);
        b->t_mirror[i] = tb;
        b->t_stop[i] = m->h.t_end;
    }
    // members' own streams must see the batch's work before their next call
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, b->stream));
    for (size_t i = 1; i < b->sims.size(); i++)
        if (b->sims[i]->stream != b->stream) CK(cudaStreamWaitEvent(b->sims[i]->stream, ev, 0));
    cudaEventDestroy(ev);
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto st : b->gstreams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto ev : b->gjoin) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_descs);
    cudaFree(b->d_items);
    cudaFree(b->d_off);
    cudaFree(b->d_err);
    delete b;
}

}  // extern "C"
