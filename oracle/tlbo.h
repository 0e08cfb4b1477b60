/*
 * tlbo.h -- FP64 CPU oracle for the ternary free-energy, high-density-ratio
 * lattice Boltzmann update of Bala, Pepona, Karlin, Kusumaatmaja & Semprebon,
 * "Wetting boundaries for a ternary high density ratio lattice Boltzmann
 * method" (arXiv:1904.06881).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and tlbo.c are a plain, slow,
 * deliberately unfused restatement of the paper's equations, used to check
 * the CUDA library.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Conventions
 *   - lattices: D2Q9 (lattice = 0) and D3Q27 (lattice = 1), the product
 *     lattices of D1Q3 on which the product-form equilibrium (Sec. II.C,
 *     Eqs. eqrho, A, B) is defined.
 *   - node index n = x + nx*(y + ny*z); every axis is periodic, walls are
 *     given by the solid mask (1 = solid).
 *   - populations are the pre-collision (post-streaming) values f_i(x,t),
 *     stored as f[i*N + n].
 *   - phases: C1 = gas, C2 = liquid with phi = +chi, C3 = liquid with
 *     phi = -chi (Sec. II.A, Eqs. definitionC1-C3).
 *   - contact angles theta[0] = theta_21, theta[1] = theta_31,
 *     theta[2] = theta_23, in degrees; the first index is the phase the
 *     angle is measured in (Sec. IV.A convention).
 */
#ifndef TLBO_H
#define TLBO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { TLBO_D2Q9 = 0, TLBO_D3Q27 = 1 };
enum { TLBO_WET_FORCE = 0, TLBO_WET_GEOM_EXTRAP = 1, TLBO_WET_GEOM_INTERP = 2 };

typedef struct {
    int    lattice;                /* TLBO_D2Q9 or TLBO_D3Q27 */
    int    nx, ny, nz;             /* nz = 1 for D2Q9 */
    double lambda[3], kappa[3];    /* free-energy parameters (Eqs. BulkEnergy, InterfEnergy) */
    double chi;                    /* phi = chi (C2 - C3) */
    double a, b, R;                /* Carnahan-Starling constants before rescaling (Eq. PsiEOS) */
    double rho_l, rho_g;           /* coexistence densities to reach (liquid, gas) */
    double beta;                   /* ELBM beta, nu = (1/beta - 1)/6 */
    double tau_g;                  /* LBGK relaxation time of g */
    double Gamma;                  /* mobility constant of g^eq */
    int    wetting;                /* TLBO_WET_* */
    double theta_deg[3];           /* theta_21, theta_31, theta_23 */
    double kw_rho, kw_phi;         /* force-method strengths (Eq. forceBC) */
    int    eos;                    /* TLBO_EOS_*: Carnahan-Starling (Eq. PsiEOS), van der Waals, Peng-Robinson */
    double omega;                  /* Peng-Robinson acentric factor */
    double nu[3];                  /* kinematic viscosity of C1, C2, C3; all 0: one beta for the fluid */
} tlbo_params;
enum { TLBO_EOS_CS = 0, TLBO_EOS_VDW = 1, TLBO_EOS_PR = 2 };

/* Derived constants of a context (filled by tlbo_create). */
typedef struct {
    double T, a, b, R;             /* temperature and rescaled a, b actually used */
    double rho_l, rho_g;           /* coexistence densities of the rescaled EOS */
    double C, Psi0;                /* constants of Eq. PsiEOS */
    double Tc;                     /* critical temperature of the EOS */
    double kappa_rr, kappa_pp, kappa_rp;   /* gradient mixing coefficients */
} tlbo_derived;

typedef struct tlbo_ctx tlbo_ctx;

/* ---- thermodynamics (Sec. II.A) ---- */
/* Critical temperature of the Carnahan-Starling EOS, found numerically. */
double tlbo_eos_critical_T(double a, double b, double R);
/* The same for the equation of state `kind` (TLBO_EOS_*; omega: the
 * Peng-Robinson acentric factor): free energy Psi, dPsi/drho, pressure
 * p = rho dPsi/drho - Psi, critical temperature, coexistence {rho_g, rho_l,
 * C, Psi0}. */
double tlbo_eos_psi_k(int kind, double omega, double rho, double a, double b, double R, double T, double C);
double tlbo_eos_dpsi_k(int kind, double omega, double rho, double a, double b, double R, double T, double C);
double tlbo_eos_p_k(int kind, double omega, double rho, double a, double b, double R, double T);
double tlbo_eos_critical_T_k(int kind, double omega, double a, double b, double R);
int tlbo_eos_coexistence_k(int kind, double omega, double a, double b, double R, double T, double out[4]);
/* Gas/liquid coexistence densities at temperature T (equal pressure and
 * chemical potential); out = {rho_g, rho_l, C, Psi0}.  Returns 0 or -1. */
int tlbo_eos_coexistence(double a, double b, double R, double T, double out[4]);
/* Psi_eos and its derivative for given constants (Eq. PsiEOS and the
 * printed derivative in Sec. II.B). */
double tlbo_eos_psi(double rho, double a, double b, double R, double T, double C);
double tlbo_eos_dpsi(double rho, double a, double b, double R, double T, double C);

/* ---- lattice kinetics (Sec. II.C) ---- */
/* Lattice tables: c (Q*3 ints, unused components 0), w (Q doubles). Returns Q. */
int tlbo_lattice(int lattice, int *c, double *w);
/* Product-form equilibrium f_i^eq(rho, u) (Eqs. eqrho, A, B); out has Q entries. */
void tlbo_feq(int lattice, double rho, const double *u, double *out);
/* Entropy H(f) = sum_i f_i ln(f_i / w_i) (Eq. EntropyEstimate). */
double tlbo_entropy(int lattice, const double *f);
/* Non-trivial root alpha of H(fp + alpha*delta) = H(fp) (Eq. EntropyEquation).
 * status: 0 root found, 1 near-equilibrium (alpha = 2), 2 no root below the
 * positivity bound (alpha clipped to it). */
double tlbo_alpha(int lattice, const double *fp, const double *delta, int *status);
/* Order-parameter equilibrium g_i^eq(phi, v, mu_phi) (Sec. II.C). */
void tlbo_geq(int lattice, double phi, const double *v, double mu_phi, double Gamma, double *out);

/* ---- simulation context ---- */
int  tlbo_create(const tlbo_params *p, tlbo_ctx **out);
void tlbo_destroy(tlbo_ctx *ctx);
int  tlbo_get_derived(const tlbo_ctx *ctx, tlbo_derived *out);
/* mask: N bytes, 1 = solid. */
int  tlbo_set_solid(tlbo_ctx *ctx, const uint8_t *mask);
/* rho, phi: N doubles; u: D*N doubles (component-major) or NULL for rest. */
int  tlbo_init_fields(tlbo_ctx *ctx, const double *rho, const double *phi, const double *u);
int  tlbo_step(tlbo_ctx *ctx, int nsteps);
/* Any output may be NULL.  u is D*N, C is 3*N.  Solid nodes read 0. */
int  tlbo_get_fields(tlbo_ctx *ctx, double *rho, double *phi, double *u, double *C);
/* Populations: Q*N doubles each (pre-collision, f[i*N+n]). */
int  tlbo_get_populations(tlbo_ctx *ctx, double *f, double *g);
int  tlbo_set_populations(tlbo_ctx *ctx, const double *f, const double *g);

/* Auxiliary fields of the current state, recomputed from the populations:
 * which = 0 p0, 1 mu_rho, 2 mu_phi, 3..5 F_x..F_z (total force incl. wetting
 * force), 6..11 P_xx,P_yy,P_zz,P_xy,P_xz,P_yz, 12 ghost rho, 13 ghost phi
 * (rho/phi including the solid ghost layer). out: N doubles. */
int  tlbo_get_aux(tlbo_ctx *ctx, int which, double *out);

/* Sums over fluid nodes: out = {sum rho, sum phi, sum C1, sum C2, sum C3,
 * kinetic energy 0.5 sum rho |u|^2}. */
int  tlbo_diagnostics(tlbo_ctx *ctx, double out[6]);
/* Count of collisions whose alpha was clipped at the positivity bound. */
long tlbo_alpha_clipped(const tlbo_ctx *ctx);

/* Host threads of the node loops; n <= 0 only reports.  Returns the count in use. */
int  tlbo_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
