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
void orc_set_pops(orc_sim *s, const double *pop);
void orc_get_pops(const orc_sim *s, double *pop);

/* Equilibrium initial state from macroscopic fields (nx*ny each, x fastest). */
void orc_init_fields(orc_sim *s, const double *rho_r, const double *rho_b,
                     const double *ux, const double *uy);

/* n full time steps. */
void orc_step(orc_sim *s, long n);

/* Macroscopic fields of the current state: rho_r, rho_b, u (Guo half-force
 * included), p = sum_k rho_k (c_s^k)^2 (Eq. (eq:pressureRelation)), psi. Any
 * output pointer may be NULL. */
void orc_fields(const orc_sim *s, double *rho_r, double *rho_b, double *ux,
                double *uy, double *p, double *psi);

/* Colour gradient F and S2I4 derivatives of Q^k for every node of the current
 * state; dQ layout [4][ny][nx] = d_xQ^r_x, d_yQ^r_y, d_xQ^b_x, d_yQ^b_y. */
void orc_gradient_fields(orc_sim *s, double *Fx, double *Fy, double *dQ);

/* ---- single operators, exposed so tests can pin them one by one ---- */
void orc_derived(const orc_params *p, double *alpha_r, double *omega_r, double *omega_b,
                 double *chi, double *eta, double *kappa, double *lam, double *nu);
void orc_equilibrium(const orc_params *p, int k, double rho_k, double ux, double uy,
                     double *neq /* 9 */);
double orc_omega_eff(const orc_params *p, double psi);
void orc_perturbation(const orc_params *p, double A, double Fx, double Fy,
                      double *dN /* 9, increment for one colour */);
void orc_recolour(const orc_params *p, double rho_r, double rho_b, double Fx, double Fy,
                  const double *N /* 9 colour-blind */, double *Nr, double *Nb);
void orc_mrt_matrices(double *M /* 81 */, double *Minv /* 81 */);
void orc_collide_node(const orc_params *p, const double *Nk /* 2*9 */, double Fx, double Fy,
                      double divQr_x, double divQr_y, double divQb_x, double divQb_y,
                      double *Nstar /* 2*9, after collision + perturbation */);
void orc_zouhe_inlet(const orc_params *p, double f_r, double *Nr /* 9 */, double *Nb /* 9 */);
void orc_zouhe_outlet(const orc_params *p, double *Nr /* 9 */, double *Nb /* 9 */);

#ifdef __cplusplus
}
#endif
#endif
