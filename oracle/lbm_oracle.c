/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain, slow, obviously-correct FP64 oracle of the D2Q9 two-phase
 * colour-gradient lattice Boltzmann step of arXiv 1903.01168, Sec. 2.  It
 * follows the paper's operators one by one, in the paper's order and
 * notation, with no fusion and no reordering:
 *
 *   moments and colour field  Sec. 2.1, Eq. (eq:color_field)
 *   colour gradient F         Eq. (eq:colorGradient)
 *   omega_eff, A              Sec. 2.1 (interpolation), Eq. (eq:sigmaIsoAllen)
 *   collision per colour      Eq. (eq:singleCollision) / Eq. (eq:singleCollisionMRT),
 *                             equilibrium Eq. (eq:equilibrium) / Eq. (eq:equilibrium_hermite),
 *                             source U^k = M^-1 C^k (Sec. 2.1, NS recovery),
 *                             Guo body force (not given by the paper; reading below)
 *   perturbation per colour   Eq. (eq:perturbation)
 *   recolouring               Eq. (eq:recoloringOperator)
 *   streaming + boundaries    Eq. (eq:subop4), Sec. 2.5 (bounce-back, periodic,
 *                             two-phase Zou-He inlet / outlet)
 *
 * Rows are processed in parallel (OpenMP) where each node's update reads only
 * the previous pass's arrays, so the result does not depend on the thread count.
 *
 * Readings taken where the paper is silent, garbled or self-contradictory
 * (each is listed in the design notes of the repository):
 *   - direction order is the standard one of the appendix matrices; every
 *     per-direction constant (W, phi, xi, B) is keyed by |c_i|^2, not by the
 *     index parity of the printed velocity formula;
 *   - gamma = (1 - alpha_b) / (1 - alpha_r), i.e. alpha_r = 1 - (1 - alpha_b)/gamma,
 *     so that both pure phases at rest have the same pressure;
 *   - psi = +1 in pure red, as Eq. (eq:color_field) gives;
 *   - the Hermite factor "(3 c_i - 4)" is (3 |c_i|^2 - 4);
 *   - the NS-recovery source: C^k_1 as printed, 3 (1 - s_1/2)(d_x Q_x + d_y Q_y);
 *     C^k_7 = (1 - omega_eff/2)(d_x Q_x - d_y Q_y), not the printed
 *     3 (1 - omega_eff/2)(d_x Q_x + d_y Q_y).  The Chapman-Enskog expansion fixes
 *     both: Q^k_x is the excess of the D2Q9 third moment sum N c_x^3 over that
 *     of a Maxwellian at (c_s^k)^2, and it enters e = sum (3|c|^2 - 4) N as
 *     3 (d_x Q_x + d_y Q_y) but p_xx = sum (c_x^2 - c_y^2) N as d_x Q_x - d_y Q_y;
 *     a source cancels an excess E of a moment relaxed at rate s when it is
 *     (1 - s/2) E.  (c7_factor and c7_sign select the printed form);
 *   - A = 9 sigma omega_eff / 4 per node, from Eq. (eq:sigmaIsoAllen);
 *   - the perturbation term is added to each colour (two colours, one l != k
 *     term each), as Eq. (eq:perturbation) is printed;
 *   - the recolouring term is zero when i = 0 or |F| == 0 exactly;
 *   - Guo-Zheng-Shi forcing with F^k = rho_k g and u = (sum N c + rho g / 2) / rho;
 *   - halfway bounce-back; psi on a solid node is the W-weighted mean of its
 *     in-domain neighbours (the wetting extrapolation of Sec. 2.4 without the
 *     stray c_{i alpha} factor); behind an open inlet / outlet psi and Q^k are
 *     copied from the boundary node (zero normal gradient), Q^k = 0 in walls;
 *   - the paper's north inlet / south outlet are rotated to a west inlet /
 *     east outlet; the inlet phase is prescribed, the outlet colour fraction
 *     comes from the known populations, the outlet velocity is
 *     v = -1 + (...)/rho_out and rho_out mixes the pure-phase densities by
 *     colour fraction.
 */
#include "lbm_oracle.h"

#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

/* The arithmetic type (FP64 unless the header's ORC_REAL is overridden); the
 * parameters are read through (real) casts so that an FP32 build computes in
 * FP32 throughout. */
typedef orc_real real;

/* ---------------------------------------------------------------- lattice */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* mirror images of each direction in a horizontal wall (c_y -> -c_y) and in a
 * vertical one (c_x -> -c_x): where a free-slip wall sends a population */
static const int MIRY[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
static const int MIRX[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};

static int c2(int i) { return CX[i] * CX[i] + CY[i] * CY[i]; }

/* D2Q9 weights W_i (Sec. 2.1). */
static real W(int i) {
    int n = c2(i);
    return n == 0 ? 4.0 / 9.0 : (n == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

/* Rest weights phi^k_i of the density-ratio equilibrium (Sec. 2.1). */
static real phi(real alpha, int i) {
    int n = c2(i);
    return n == 0 ? alpha : (n == 1 ? (1.0 - alpha) / 5.0 : (1.0 - alpha) / 20.0);
}

/* S2I4 gradient weights xi_i, Eq. (eq:colorGradient). */
static real xi(int i) {
    int n = c2(i);
    return n == 0 ? 0.0 : (n == 1 ? 1.0 / 3.0 : 1.0 / 12.0);
}

/* Perturbation constants B_i, Eq. (eq:perturbation). */
static real Bc(int i) {
    int n = c2(i);
    return n == 0 ? -4.0 / 27.0 : (n == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
}

/* ------------------------------------------------------------- parameters */
void orc_derived(const orc_params *p, real *alpha_r, real *omega_r, real *omega_b,
                 real *chi, real *eta, real *kappa, real *lam, real *nu) {
    real ar = 1.0 - (1.0 - (real)p->alpha_b) / (real)p->gamma;    /* Eq. (eq:gammaAlphaBeta) */
    real wr = 1.0 / (real)p->tau_r, wb = 1.0 / (real)p->tau_b;
    real c = 2.0 * wr * wb / (wr + wb);
    real e = 2.0 * (wr - c) / (real)p->delta;
    real l = 2.0 * (c - wb) / (real)p->delta;
    if (alpha_r) *alpha_r = ar;
    if (omega_r) *omega_r = wr;
    if (omega_b) *omega_b = wb;
    if (chi) *chi = c;
    if (eta) *eta = e;
    if (kappa) *kappa = -e / (2.0 * (real)p->delta);
    if (lam) *lam = l;
    if (nu) *nu = l / (2.0 * (real)p->delta);
}

static real alpha_of(const orc_params *p, int k) {
    real ar;
    orc_derived(p, &ar, 0, 0, 0, 0, 0, 0, 0);
    return k == 0 ? ar : (real)p->alpha_b;
}

static real rho0_of(const orc_params *p, int k) { return k == 0 ? (real)p->gamma : 1.0; }

/* (c_s^k)^2 = 3 (1 - alpha_k) / 5, Eq. (eq:pressureRelation). */
static real cs2_of(const orc_params *p, int k) { return 3.0 * (1.0 - alpha_of(p, k)) / 5.0; }

/* --------------------------------------------------------------- operators */

/* Eq. (eq:equilibrium), or Eq. (eq:equilibrium_hermite) with the factor read
 * as (3|c_i|^2 - 4). */
void orc_equilibrium(const orc_params *p, int k, real rho_k, real ux, real uy,
                     real *neq) {
    real alpha = alpha_of(p, k);
    real cs2 = cs2_of(p, k);
    real usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        real cu = CX[i] * ux + CY[i] * uy;
        real lin = 3.0 * cu;
        if (p->equilibrium == ORC_EQ_HERMITE)
            lin = 3.0 * cu * (1.0 + 0.5 * (3.0 * cs2 - 1.0) * (3.0 * c2(i) - 4.0));
        neq[i] = rho_k * phi(alpha, i) + rho_k * W(i) * (lin + 4.5 * cu * cu - 1.5 * usq);
    }
}

/* Piecewise omega_eff(psi) of Sec. 2.1, with f_r and f_b as printed. */
real orc_omega_eff(const orc_params *p, real psi) {
    real wr, wb, chi, eta, kappa, lam, nu;
    orc_derived(p, 0, &wr, &wb, &chi, &eta, &kappa, &lam, &nu);
    if (psi > (real)p->delta) return wr;
    if (psi > 0.0) return chi + eta * psi + kappa * psi * psi;
    if (psi >= -(real)p->delta) return chi + lam * psi + nu * psi * psi;
    return wb;
}

/* One colour's increment (A/2)|F| [W_i (F.c_i)^2/|F|^2 - B_i], Eq. (eq:perturbation).
 * Zero when |F| == 0. */
void orc_perturbation(const orc_params *p, real A, real Fx, real Fy, real *dN) {
    (void)p;
    real F2 = Fx * Fx + Fy * Fy;
    for (int i = 0; i < 9; i++) {
        if (F2 == 0.0) {
            dN[i] = 0.0;
            continue;
        }
        real Fn = sqrt(F2);
        real Fc = Fx * CX[i] + Fy * CY[i];
        dN[i] = 0.5 * A * Fn * (W(i) * Fc * Fc / F2 - Bc(i));
    }
}

/* Eq. (eq:recoloringOperator): N^r_i = rho_r/rho N_i + beta rho_r rho_b/rho^2 cos(phi_i)
 * sum_k N^{k(e)}_i(rho_k, 0, alpha_k); N^b_i = N_i - N^r_i.  The second term is
 * zero for i = 0 or |F| == 0. */
void orc_recolour(const orc_params *p, real rho_r, real rho_b, real Fx, real Fy,
                  const real *N, real *Nr, real *Nb) {
    real rho = rho_r + rho_b;
    real F2 = Fx * Fx + Fy * Fy;
    real ar = alpha_of(p, 0), ab = alpha_of(p, 1);
    for (int i = 0; i < 9; i++) {
        real term = 0.0;
        if (i != 0 && F2 != 0.0) {
            real cosphi = (CX[i] * Fx + CY[i] * Fy) / (sqrt((real)c2(i)) * sqrt(F2));
            real rest = rho_r * phi(ar, i) + rho_b * phi(ab, i); /* N^{k(e)}(rho_k, 0) summed */
            term = (real)p->beta * rho_r * rho_b / (rho * rho) * cosphi * rest;
        }
        Nr[i] = rho_r / rho * N[i] + term;
        Nb[i] = rho_b / rho * N[i] - term;
    }
}

/* The appendix "Transformation matrices": M and M^{-1} = (1/36) * (integer matrix). */
static const int M_INT[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static const int MINV36[9][9] = {
    {4, -4, 4, 0, 0, 0, 0, 0, 0},
    {4, -1, -2, 6, -6, 0, 0, 9, 0},
    {4, -1, -2, 0, 0, 6, -6, -9, 0},
    {4, -1, -2, -6, 6, 0, 0, 9, 0},
    {4, -1, -2, 0, 0, -6, 6, -9, 0},
    {4, 2, 1, 6, 3, 6, 3, 0, 9},
    {4, 2, 1, -6, -3, 6, 3, 0, -9},
    {4, 2, 1, -6, -3, -6, -3, 0, 9},
    {4, 2, 1, 6, 3, -6, -3, 0, -9}};

void orc_mrt_matrices(real *M, real *Minv) {
    for (int a = 0; a < 9; a++)
        for (int b = 0; b < 9; b++) {
            M[a * 9 + b] = (real)M_INT[a][b];
            Minv[a * 9 + b] = (real)MINV36[a][b] / 36.0;
        }
}

static void matvec(const real *A, const real *x, real *y) {
    for (int a = 0; a < 9; a++) {
        real s = 0.0;
        for (int b = 0; b < 9; b++) s += A[a * 9 + b] * x[b];
        y[a] = s;
    }
}

/* Node moments: rho_k, rho, and u = (sum_k sum_i N^k_i c_i + rho g / 2) / rho. */
static void node_moments(const orc_params *p, const real *Nk, real *rho_r, real *rho_b,
                         real *ux, real *uy) {
    real rr = 0.0, rb = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
        rr += Nk[i];
        rb += Nk[9 + i];
        jx += (Nk[i] + Nk[9 + i]) * CX[i];
        jy += (Nk[i] + Nk[9 + i]) * CY[i];
    }
    real rho = rr + rb;
    *rho_r = rr;
    *rho_b = rb;
    *ux = (jx + 0.5 * rho * (real)p->gx) / rho;
    *uy = (jy + 0.5 * rho * (real)p->gy) / rho;
}

static real colour_field(const orc_params *p, real rho_r, real rho_b) {
    real a = rho_r / rho0_of(p, 0), b = rho_b / rho0_of(p, 1);
    return (a - b) / (a + b);                           /* Eq. (eq:color_field) */
}

/* Single-phase collision of each colour (BGK or MRT, + Guo, + U^k) followed by
 * the perturbation of each colour.  Input: pre-collision N^k_i of one node,
 * the colour gradient F and, for the Hermite/MRT source, the divergence parts
 * d_x Q^k_x and d_y Q^k_y of each colour. */
void orc_collide_node(const orc_params *p, const real *Nk, real Fx, real Fy,
                      real divQr_x, real divQr_y, real divQb_x, real divQb_y,
                      real *Nstar) {
    real rho_r, rho_b, ux, uy;
    node_moments(p, Nk, &rho_r, &rho_b, &ux, &uy);
    real psi = colour_field(p, rho_r, rho_b);
    real w = orc_omega_eff(p, psi);
    real A = 9.0 * (real)p->sigma * w / 4.0;                /* Eq. (eq:sigmaIsoAllen) */
    real M[81], Minv[81];
    orc_mrt_matrices(M, Minv);
    real s[9];
    for (int a = 0; a < 9; a++) s[a] = (real)p->mrt_lambda * w; /* s_0..s_6 */
    s[7] = w;
    s[8] = w;

    for (int k = 0; k < 2; k++) {
        const real *N = Nk + 9 * k;
        real *out = Nstar + 9 * k;
        real rho_k = k == 0 ? rho_r : rho_b;
        real neq[9];
        orc_equilibrium(p, k, rho_k, ux, uy, neq);

        /* Guo source of colour k, force F^k = rho_k g. */
        real fx = rho_k * (real)p->gx, fy = rho_k * (real)p->gy;
        real src[9];
        for (int i = 0; i < 9; i++) {
            real cu = CX[i] * ux + CY[i] * uy;
            src[i] = W(i) * (3.0 * ((CX[i] - ux) * fx + (CY[i] - uy) * fy) +
                             9.0 * cu * (CX[i] * fx + CY[i] * fy));
        }

        if (p->collision == ORC_BGK) {
            /* Eq. (eq:singleCollision) + (1 - omega/2) S_i */
            for (int i = 0; i < 9; i++)
                out[i] = N[i] - w * (N[i] - neq[i]) + (1.0 - 0.5 * w) * src[i];
        } else {
            /* Eq. (eq:singleCollisionMRT): N - M^-1 S M (N - Neq) + M^-1 (I - S/2) M src + U^k */
            real d[9], m[9], ms[9], t[9], back[9];
            for (int i = 0; i < 9; i++) d[i] = N[i] - neq[i];
            matvec(M, d, m);
            matvec(M, src, ms);
            for (int a = 0; a < 9; a++) t[a] = s[a] * m[a] - (1.0 - 0.5 * s[a]) * ms[a];
            if (p->equilibrium == ORC_EQ_HERMITE) {
                /* C^k = [0, C_1, 0, 0, 0, 0, 0, C_7, 0]; U^k = M^-1 C^k is ADDED, so it
                 * enters t with a minus sign. */
                real dqx = k == 0 ? divQr_x : divQb_x;
                real dqy = k == 0 ? divQr_y : divQb_y;
                real C1 = 3.0 * (1.0 - 0.5 * s[1]) * (dqx + dqy);
                real C7 = (real)p->c7_factor * (1.0 - 0.5 * w) * (dqx + (real)p->c7_sign * dqy);
                t[1] -= C1;
                t[7] -= C7;
            }
            matvec(Minv, t, back);
            for (int i = 0; i < 9; i++) out[i] = N[i] - back[i];
        }

        /* Eq. (eq:perturbation): one l != k term per colour. */
        if (p->perturb_mode == ORC_PERTURB_PER_COLOUR) {
            real dN[9];
            orc_perturbation(p, A, Fx, Fy, dN);
            for (int i = 0; i < 9; i++) out[i] += dN[i];
        }
    }
    if (p->perturb_mode == ORC_PERTURB_ONCE) {
        /* Alternative reading: one A/2 term on the colour-blind distribution
         * (put on the red set; only the colour-blind sum is used afterwards). */
        real dN[9];
        orc_perturbation(p, A, Fx, Fy, dN);
        for (int i = 0; i < 9; i++) Nstar[i] += dN[i];
    }
}

/* ----------------------------------------------------------- Zou-He (Sec. 2.5) */

/* West velocity inlet, the paper's north inlet rotated by +90 degrees.  On
 * entry Nr/Nb hold the post-streaming populations with the unknowns 1, 5, 8
 * undefined; f_r is the red fraction of the injected phase at this node. */
void orc_zouhe_inlet(const orc_params *p, real f_r, real *Nr, real *Nb) {
    real f_b = 1.0 - f_r;
    real N[9];
    for (int i = 0; i < 9; i++) N[i] = Nr[i] + Nb[i];
    real Vx = f_r * (real)p->u_in_r + f_b * (real)p->u_in_b; /* v^in = v^{b,in} + v^{r,in} */
    real Vy = 0.0;
    real rho = (N[0] + N[2] + N[4] + 2.0 * (N[3] + N[6] + N[7])) / (1.0 - Vx);
    real H = 0.0;
    if (p->equilibrium == ORC_EQ_HERMITE) {
        real amix = f_r * (3.0 * cs2_of(p, 0) - 1.0) + f_b * (3.0 * cs2_of(p, 1) - 1.0);
        H = -rho * amix * Vx / 3.0;
    }
    N[1] = N[3] + 2.0 / 3.0 * rho * Vx + H;
    N[5] = N[7] + 0.5 * (N[4] - N[2]) + 0.5 * rho * Vy + rho * Vx / 6.0 - 0.5 * H;
    N[8] = N[6] + 0.5 * (N[2] - N[4]) - 0.5 * rho * Vy + rho * Vx / 6.0 - 0.5 * H;
    const int unk[3] = {1, 5, 8};
    for (int j = 0; j < 3; j++) {
        Nr[unk[j]] = f_r * N[unk[j]];
        Nb[unk[j]] = f_b * N[unk[j]];
    }
}

/* East pressure outlet, the paper's south outlet rotated by +90 degrees.
 * Unknowns 3, 6, 7.  The colour fraction comes from the known populations. */
void orc_zouhe_outlet(const orc_params *p, real *Nr, real *Nb) {
    const int known[6] = {0, 1, 2, 4, 5, 8};
    real kr = 0.0, kb = 0.0;
    for (int j = 0; j < 6; j++) {
        kr += Nr[known[j]];
        kb += Nb[known[j]];
    }
    real psi = colour_field(p, kr, kb);
    real f_r = 0.5 * (1.0 + psi), f_b = 1.0 - f_r;
    real N[9];
    for (int i = 0; i < 9; i++) N[i] = Nr[i] + Nb[i];
    real rho = f_b * (real)p->p_out / cs2_of(p, 1) + f_r * (real)p->p_out / cs2_of(p, 0);
    real Vx = -1.0 + (N[0] + N[2] + N[4] + 2.0 * (N[1] + N[5] + N[8])) / rho;
    real H = 0.0;
    if (p->equilibrium == ORC_EQ_HERMITE) {
        real amix = f_r * (3.0 * cs2_of(p, 0) - 1.0) + f_b * (3.0 * cs2_of(p, 1) - 1.0);
        H = rho * amix * Vx / 3.0;
    }
    /* tangential outlet velocity is zero (v^out_x = 0 in the paper's frame) */
    N[3] = N[1] - 2.0 / 3.0 * rho * Vx + H;
    N[6] = N[8] - 0.5 * (N[2] - N[4]) - rho * Vx / 6.0 - 0.5 * H;
    N[7] = N[5] + 0.5 * (N[2] - N[4]) - rho * Vx / 6.0 - 0.5 * H;
    const int unk[3] = {3, 6, 7};
    for (int j = 0; j < 3; j++) {
        Nr[unk[j]] = f_r * N[unk[j]];
        Nb[unk[j]] = f_b * N[unk[j]];
    }
}

/* ------------------------------------------------------------------ state */
struct orc_sim {
    orc_params p;
    long t;
    real *N;     /* pre-collision N^k_i(x, t) */
    real *Npost; /* after collision, perturbation and recolouring */
    real *rho_r, *rho_b, *ux, *uy, *psi;
    real *Qx, *Qy; /* Q^k per colour: [k][y][x] */
};

static size_t pidx(const orc_sim *s, int k, int i, int x, int y) {
    return (((size_t)(k * 9 + i) * s->p.ny + y) * s->p.nx) + x;
}

orc_sim *orc_create(const orc_params *p) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    size_t n = (size_t)p->nx * p->ny;
    s->N = (real *)calloc(18 * n, sizeof(real));
    s->Npost = (real *)calloc(18 * n, sizeof(real));
    s->rho_r = (real *)calloc(n, sizeof(real));
    s->rho_b = (real *)calloc(n, sizeof(real));
    s->ux = (real *)calloc(n, sizeof(real));
    s->uy = (real *)calloc(n, sizeof(real));
    s->psi = (real *)calloc(n, sizeof(real));
    s->Qx = (real *)calloc(2 * n, sizeof(real));
    s->Qy = (real *)calloc(2 * n, sizeof(real));
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->N);
    free(s->Npost);
    free(s->rho_r);
    free(s->rho_b);
    free(s->ux);
    free(s->uy);
    free(s->psi);
    free(s->Qx);
    free(s->Qy);
    free(s);
}

long orc_time(const orc_sim *s) { return s->t; }

void orc_set_pops(orc_sim *s, const real *pop) {
    memcpy(s->N, pop, 18 * (size_t)s->p.nx * s->p.ny * sizeof(real));
}

void orc_get_pops(const orc_sim *s, real *pop) {
    memcpy(pop, s->N, 18 * (size_t)s->p.nx * s->p.ny * sizeof(real));
}

static void gather_node(const orc_sim *s, const real *pop, int x, int y, real *Nk) {
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < 9; i++) Nk[9 * k + i] = pop[pidx(s, k, i, x, y)];
}

static void scatter_node(orc_sim *s, real *pop, int x, int y, const real *Nk) {
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < 9; i++) pop[pidx(s, k, i, x, y)] = Nk[9 * k + i];
}

/* Red fraction injected at inlet row y at time t. */
static real inlet_red_fraction(const orc_params *p, int y, long t) {
    if (p->inlet_mode == ORC_INLET_LAYERED) return y < p->inlet_layer ? 1.0 : 0.0;
    long period = (long)p->inlet_period_r + p->inlet_period_b;
    if (period <= 0) return 1.0;
    return (t % period) < p->inlet_period_r ? 1.0 : 0.0;
}

static void apply_inout(orc_sim *s) {
    if (s->p.bc_x != ORC_INOUT) return;
    for (int y = 0; y < s->p.ny; y++) {
        real Nk[18];
        gather_node(s, s->N, 0, y, Nk);
        orc_zouhe_inlet(&s->p, inlet_red_fraction(&s->p, y, s->t), Nk, Nk + 9);
        scatter_node(s, s->N, 0, y, Nk);
        gather_node(s, s->N, s->p.nx - 1, y, Nk);
        orc_zouhe_outlet(&s->p, Nk, Nk + 9);
        scatter_node(s, s->N, s->p.nx - 1, y, Nk);
    }
}

void orc_init_fields(orc_sim *s, const real *rho_r, const real *rho_b, const real *ux,
                     const real *uy) {
    int nx = s->p.nx, ny = s->p.ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)y * nx + x;
            real er[9], eb[9];
            orc_equilibrium(&s->p, 0, rho_r[n], ux[n], uy[n], er);
            orc_equilibrium(&s->p, 1, rho_b[n], ux[n], uy[n], eb);
            for (int i = 0; i < 9; i++) {
                s->N[pidx(s, 0, i, x, y)] = er[i];
                s->N[pidx(s, 1, i, x, y)] = eb[i];
            }
        }
    s->t = 0;
    apply_inout(s);
}

/* Is (X, Y) inside the domain after periodic wrapping?  Writes the wrapped
 * coordinates. */
static int in_domain(const orc_params *p, int X, int Y, int *xw, int *yw) {
    if (X < 0 || X >= p->nx) {
        if (p->bc_x != ORC_PERIODIC) return 0;
        X = ((X % p->nx) + p->nx) % p->nx;
    }
    if (Y < 0 || Y >= p->ny) {
        if (p->bc_y != ORC_PERIODIC) return 0;
        Y = ((Y % p->ny) + p->ny) % p->ny;
    }
    *xw = X;
    *yw = Y;
    return 1;
}

/* psi at any lattice position next to the domain.  Behind a no-slip wall
 * (a solid node) it is the W-weighted mean of the in-domain neighbours
 * (Sec. 2.4 extrapolation); behind an open inlet / outlet column it is the
 * value of the boundary node on the same row (zero normal gradient). */
static real psi_at(const orc_sim *s, int X, int Y) {
    int xw, yw;
    if (in_domain(&s->p, X, Y, &xw, &yw)) return s->psi[(size_t)yw * s->p.nx + xw];
    int out_y = (Y < 0 || Y >= s->p.ny);
    if (!out_y && s->p.bc_x == ORC_INOUT) {
        int xc = X < 0 ? 0 : s->p.nx - 1;
        return s->psi[(size_t)Y * s->p.nx + xc];
    }
    real num = 0.0, den = 0.0;
    for (int i = 1; i < 9; i++)
        if (in_domain(&s->p, X + CX[i], Y + CY[i], &xw, &yw)) {
            num += W(i) * s->psi[(size_t)yw * s->p.nx + xw];
            den += W(i);
        }
    return den > 0.0 ? num / den : 0.0;
}

/* Q^k (component comp: 0 x, 1 y) at any lattice position next to the domain:
 * zero behind a no-slip wall (u = 0 there), the boundary node's value behind
 * an open inlet / outlet column (zero normal gradient). */
static real Q_at(const orc_sim *s, int k, int comp, int X, int Y) {
    const real *Q = comp == 0 ? s->Qx : s->Qy;
    size_t n = (size_t)s->p.nx * s->p.ny;
    int xw, yw;
    if (in_domain(&s->p, X, Y, &xw, &yw)) return Q[k * n + (size_t)yw * s->p.nx + xw];
    int out_y = (Y < 0 || Y >= s->p.ny);
    if (!out_y && s->p.bc_x == ORC_INOUT) {
        int xc = X < 0 ? 0 : s->p.nx - 1;
        return Q[k * n + (size_t)Y * s->p.nx + xc];
    }
    return 0.0;
}

/* Moments, colour field and Q^k of every node of the current state. */
static void moments_pass(orc_sim *s) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    real ar = alpha_of(p, 0), ab = alpha_of(p, 1);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t c = (size_t)y * nx + x;
            real Nk[18];
            gather_node(s, s->N, x, y, Nk);
            node_moments(p, Nk, &s->rho_r[c], &s->rho_b[c], &s->ux[c], &s->uy[c]);
            s->psi[c] = colour_field(p, s->rho_r[c], s->rho_b[c]);
            /* Q^k = (1.8 alpha_k - 0.8) rho_k u (Sec. 2.1, NS recovery) */
            s->Qx[c] = (1.8 * ar - 0.8) * s->rho_r[c] * s->ux[c];
            s->Qy[c] = (1.8 * ar - 0.8) * s->rho_r[c] * s->uy[c];
            s->Qx[n + c] = (1.8 * ab - 0.8) * s->rho_b[c] * s->ux[c];
            s->Qy[n + c] = (1.8 * ab - 0.8) * s->rho_b[c] * s->uy[c];
        }
}

/* Colour gradient F (Eq. (eq:colorGradient)) and the S2I4 derivatives
 * d_x Q^k_x, d_y Q^k_y of one node, from the fields of moments_pass. */
static void gradient_node(const orc_sim *s, int x, int y, real *Fx, real *Fy,
                          real dQ[2][2]) {
    *Fx = 0.0;
    *Fy = 0.0;
    dQ[0][0] = dQ[0][1] = dQ[1][0] = dQ[1][1] = 0.0;
    for (int i = 1; i < 9; i++) {
        real ps = psi_at(s, x + CX[i], y + CY[i]);
        *Fx += xi(i) * CX[i] * ps;
        *Fy += xi(i) * CY[i] * ps;
        for (int k = 0; k < 2; k++) {
            dQ[k][0] += xi(i) * CX[i] * Q_at(s, k, 0, x + CX[i], y + CY[i]);
            dQ[k][1] += xi(i) * CY[i] * Q_at(s, k, 1, x + CX[i], y + CY[i]);
        }
    }
}

/* Static contact angle (Sec. "Adjustment of the color gradient for static
 * contact angles"): at a fluid node next to a wall (class C_fs) the direction
 * n* = F / |F| is replaced by whichever of the two unit normals n1, n2 that make
 * the angle theta with the wall normal n^s (pointing into the fluid) is closer to
 * it, n^s itself on a tie; |F| is kept.  Applied to walls in y (a node next to
 * both walls of a one-row channel takes the bottom one). */
static void contact_angle_adjust(const orc_params *p, int x, int y, real *Fx, real *Fy) {
    (void)x;
    if ((real)p->contact_angle <= 0.0 || p->bc_y != ORC_WALL) return;
    real nsx = 0.0, nsy;
    if (y == 0) nsy = 1.0;
    else if (y == p->ny - 1) nsy = -1.0;
    else return;
    real F = sqrt(*Fx * *Fx + *Fy * *Fy);
    if (F == 0.0) return;
    real ct = cos((real)p->contact_angle), st = sin((real)p->contact_angle);
    real n1x = nsx * ct - nsy * st, n1y = nsy * ct + nsx * st;
    real n2x = nsx * ct + nsy * st, n2y = nsy * ct - nsx * st;
    real ux = *Fx / F, uy = *Fy / F;
    real d1 = sqrt((ux - n1x) * (ux - n1x) + (uy - n1y) * (uy - n1y));
    real d2 = sqrt((ux - n2x) * (ux - n2x) + (uy - n2y) * (uy - n2y));
    real nx_, ny_;
    if (d1 < d2) { nx_ = n1x; ny_ = n1y; }
    else if (d1 > d2) { nx_ = n2x; ny_ = n2y; }
    else { nx_ = nsx; ny_ = nsy; }
    *Fx = F * nx_;
    *Fy = F * ny_;
}

void orc_gradient_fields(orc_sim *s, real *Fx, real *Fy, real *dQ) {
    moments_pass(s);
    int nx = s->p.nx, ny = s->p.ny;
    size_t n = (size_t)nx * ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t c = (size_t)y * nx + x;
            real fx, fy, d[2][2];
            gradient_node(s, x, y, &fx, &fy, d);
            contact_angle_adjust(&s->p, x, y, &fx, &fy);
            if (Fx) Fx[c] = fx;
            if (Fy) Fy[c] = fy;
            if (dQ) {
                dQ[c] = d[0][0];
                dQ[n + c] = d[0][1];
                dQ[2 * n + c] = d[1][0];
                dQ[3 * n + c] = d[1][1];
            }
        }
}

static void step_once(orc_sim *s) {
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;

    /* 1. moments and colour field of every node at time t */
    moments_pass(s);

    /* 2. colour gradient, collision, perturbation, recolouring per node */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t c = (size_t)y * nx + x;
            real Fx, Fy, dQ[2][2];
            gradient_node(s, x, y, &Fx, &Fy, dQ);
            contact_angle_adjust(p, x, y, &Fx, &Fy);
            real Nk[18], Nstar[18], Nsum[9], Nr[9], Nb[9];
            gather_node(s, s->N, x, y, Nk);
            orc_collide_node(p, Nk, Fx, Fy, dQ[0][0], dQ[0][1], dQ[1][0], dQ[1][1], Nstar);
            for (int i = 0; i < 9; i++) Nsum[i] = Nstar[i] + Nstar[9 + i];
            orc_recolour(p, s->rho_r[c], s->rho_b[c], Fx, Fy, Nsum, Nr, Nb);
            for (int i = 0; i < 9; i++) {
                s->Npost[pidx(s, 0, i, x, y)] = Nr[i];
                s->Npost[pidx(s, 1, i, x, y)] = Nb[i];
            }
        }

    /* 3. streaming, Eq. (eq:subop4), with periodic / bounce-back links */
#pragma omp parallel for collapse(3) schedule(static)
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < 9; i++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int X = x - CX[i], Y = y - CY[i];
                    int xw, yw;
                    real v;
                    int out_y = (Y < 0 || Y >= ny), out_x = (X < 0 || X >= nx);
                    int wall_y = out_y && p->bc_y == ORC_WALL, wall_x = out_x && p->bc_x == ORC_WALL;
                    if (in_domain(p, X, Y, &xw, &yw))
                        v = s->Npost[pidx(s, k, i, xw, yw)];
                    else if (p->wall_slip && wall_y && in_domain(p, X, y, &xw, &yw))
                        /* free slip: the population left (X, y) towards the wall and
                         * comes back mirrored, travelling on along the wall */
                        v = s->Npost[pidx(s, k, MIRY[i], xw, yw)];
                    else if (p->wall_slip && wall_x && in_domain(p, x, Y, &xw, &yw))
                        v = s->Npost[pidx(s, k, MIRX[i], xw, yw)];
                    else if (wall_y || wall_x)
                        v = s->Npost[pidx(s, k, OPP[i], x, y)]; /* halfway bounce-back */
                    else
                        v = 0.0; /* unknown, set by Zou-He below */
                    s->N[pidx(s, k, i, x, y)] = v;
                }
    s->t += 1;

    /* 4. two-phase Zou-He columns of the new state */
    apply_inout(s);
}

void orc_step(orc_sim *s, long n) {
    for (long j = 0; j < n; j++) step_once(s);
}

void orc_fields(const orc_sim *s, real *rho_r, real *rho_b, real *ux, real *uy,
                real *p, real *psi) {
    int nx = s->p.nx, ny = s->p.ny;
    real cr = cs2_of(&s->p, 0), cb = cs2_of(&s->p, 1);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t c = (size_t)y * nx + x;
            real Nk[18], rr, rb, vx, vy;
            gather_node(s, s->N, x, y, Nk);
            node_moments(&s->p, Nk, &rr, &rb, &vx, &vy);
            if (rho_r) rho_r[c] = rr;
            if (rho_b) rho_b[c] = rb;
            if (ux) ux[c] = vx;
            if (uy) uy[c] = vy;
            if (p) p[c] = rr * cr + rb * cb;
            if (psi) psi[c] = colour_field(&s->p, rr, rb);
        }
}
