/*
 * lbm_oracle.h -- TEST INFRASTRUCTURE, not part of the product.
 *
 * Plain FP64 CPU oracle of the two-phase colour-gradient lattice Boltzmann
 * step of "Comparison of multiphase SPH and LBM approaches for the simulation
 * of intermittent flows" (arXiv 1903.01168), Sec. 2.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Conventions (the oracle's own):
 *   lattice nx * ny, x fastest; populations N^k_i(x, y) stored as
 *   pop[((k * 9 + i) * ny + y) * nx + x], k = 0 red (heavy), k = 1 blue (light);
 *   direction order 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE
 *   (the order of the MRT matrix in the paper's appendix "Transformation
 *   matrices" and of its Zou-He formulas).
 *   The stored state at time t is the PRE-collision N^k_i(x, t) of
 *   Eq. (eq:evolution); one step applies the four sub-steps of Sec. 2
 *   (collision, perturbation, recolouring, streaming) in the paper's order.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic type of the oracle: FP64 (the default).  The tests also compile
 * the same source with ORC_REAL=float and single-precision constants, to
 * measure what FP32 rounding alone does to a case (the method's FP32 floor);
 * the parameters below stay double either way. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL orc_real;

enum { ORC_BGK = 0, ORC_MRT = 1 };
enum { ORC_EQ_STD = 0, ORC_EQ_HERMITE = 1 };
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_INOUT = 2 };
enum { ORC_INLET_ALTERNATE = 0, ORC_INLET_LAYERED = 1 };
enum { ORC_PERTURB_PER_COLOUR = 0, ORC_PERTURB_ONCE = 1 };

typedef struct {
    int nx, ny;
    double gamma;       /* rho_r^0 / rho_b^0 with rho_b^0 = 1, Eq. (eq:gammaAlphaBeta) */
    double alpha_b;     /* free parameter alpha_b (0.2 in the paper) */
    double tau_r, tau_b;/* omega_k = 1 / tau_k, tau_k = 3 nu_k + 1/2 */
    double delta;       /* interface width of the omega_eff interpolation */
    double sigma;       /* surface tension, Eq. (eq:sigmaIsoAllen) */
    double beta;        /* recolouring parameter, Eq. (eq:recoloringOperator) */
    double gx, gy;      /* body acceleration (Guo forcing) */
    int collision;      /* ORC_BGK / ORC_MRT */
    int equilibrium;    /* ORC_EQ_STD / ORC_EQ_HERMITE (Hermite adds U^k under MRT) */
    double mrt_lambda;  /* s_0..s_6 = lambda * omega_eff */
    double c7_sign;     /* sign of d_y Q_y inside C^k_7 (-1 derived; +1 as printed) */
    double c7_factor;   /* factor of C^k_7 (1 derived; 3 as printed) */
    int perturb_mode;   /* ORC_PERTURB_PER_COLOUR (as printed) or ORC_PERTURB_ONCE */
    int bc_x, bc_y;     /* ORC_PERIODIC / ORC_WALL / ORC_INOUT (x only) */
    double u_in_r, u_in_b; /* inlet speeds of the red / blue phase */
    double p_out;       /* outlet pressure */
    int inlet_mode;     /* ORC_INLET_ALTERNATE (in time) / ORC_INLET_LAYERED (in y) */
    int inlet_period_r, inlet_period_b; /* steps of red then blue injection */
    int inlet_layer;    /* rows y < inlet_layer inject red when layered */
    int wall_slip;      /* walls: 0 no slip (halfway bounce-back), 1 free slip (Sec. 2.5) */
    double contact_angle; /* radians, 0 < theta < pi; 0 = no colour-gradient adjustment
                             (Sec. "Adjustment of the color gradient for static contact
                             angles"); theta is measured through the blue phase */
} orc_params;

typedef struct orc_sim orc_sim;

orc_sim *orc_create(const orc_params *p);
void orc_destroy(orc_sim *s);
long orc_time(const orc_sim *s);

/* State: pre-collision populations N^k_i(x, t). */
void orc_set_pops(orc_sim *s, const orc_real *pop);
void orc_get_pops(const orc_sim *s, orc_real *pop);

/* Equilibrium initial state from macroscopic fields (nx*ny each, x fastest). */
void orc_init_fields(orc_sim *s, const orc_real *rho_r, const orc_real *rho_b,
                     const orc_real *ux, const orc_real *uy);

/* n full time steps. */
void orc_step(orc_sim *s, long n);

/* Macroscopic fields of the current state: rho_r, rho_b, u (Guo half-force
 * included), p = sum_k rho_k (c_s^k)^2 (Eq. (eq:pressureRelation)), psi. Any
 * output pointer may be NULL. */
void orc_fields(const orc_sim *s, orc_real *rho_r, orc_real *rho_b, orc_real *ux,
                orc_real *uy, orc_real *p, orc_real *psi);

/* Colour gradient F and S2I4 derivatives of Q^k for every node of the current
 * state; dQ layout [4][ny][nx] = d_xQ^r_x, d_yQ^r_y, d_xQ^b_x, d_yQ^b_y. */
void orc_gradient_fields(orc_sim *s, orc_real *Fx, orc_real *Fy, orc_real *dQ);

/* ---- single operators, exposed so tests can pin them one by one ---- */
void orc_derived(const orc_params *p, orc_real *alpha_r, orc_real *omega_r, orc_real *omega_b,
                 orc_real *chi, orc_real *eta, orc_real *kappa, orc_real *lam, orc_real *nu);
void orc_equilibrium(const orc_params *p, int k, orc_real rho_k, orc_real ux, orc_real uy,
                     orc_real *neq /* 9 */);
orc_real orc_omega_eff(const orc_params *p, orc_real psi);
void orc_perturbation(const orc_params *p, orc_real A, orc_real Fx, orc_real Fy,
                      orc_real *dN /* 9, increment for one colour */);
void orc_recolour(const orc_params *p, orc_real rho_r, orc_real rho_b, orc_real Fx, orc_real Fy,
                  const orc_real *N /* 9 colour-blind */, orc_real *Nr, orc_real *Nb);
void orc_mrt_matrices(orc_real *M /* 81 */, orc_real *Minv /* 81 */);
void orc_collide_node(const orc_params *p, const orc_real *Nk /* 2*9 */, orc_real Fx, orc_real Fy,
                      orc_real divQr_x, orc_real divQr_y, orc_real divQb_x, orc_real divQb_y,
                      orc_real *Nstar /* 2*9, after collision + perturbation */);
void orc_zouhe_inlet(const orc_params *p, orc_real f_r, orc_real *Nr /* 9 */, orc_real *Nb /* 9 */);
void orc_zouhe_outlet(const orc_params *p, orc_real *Nr /* 9 */, orc_real *Nb /* 9 */);

#ifdef __cplusplus
}
#endif
#endif
