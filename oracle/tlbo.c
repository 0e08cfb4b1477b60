/*
 * tlbo.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see tlbo.h).
 *
 * One time step follows the order the paper fixes (Sec. II.C and Sec. IV):
 *   1. moments rho = sum f_i, rho u = sum f_i c_i, phi = sum g_i
 *   2. ghost layer: rho, phi at solid nodes next to fluid (Sec. IV,
 *      method 1 copy, method 2 extrapolation, method 3 interpolation)
 *   3. isotropic stencils for grad and Laplacian of rho and phi
 *   4. concentrations, chemical potentials, pressure tensor (Sec. II.A-B)
 *   5. force F = div(rho c_s^2 I - P) with the wall rules of Sec. IV,
 *      plus the wetting force of method 1 (Eq. forceBC)
 *   6. ELBM collision for f with the exact entropic alpha (Eqs. ELBMequation,
 *      EntropyEquation) and LBGK for g (Eq. CahnHilliardLBM)
 *   7. streaming with halfway bounce-back at solid links
 * Every loop is a plain per-node loop; no blocking, fusion or reordering.
 * OpenMP only distributes independent node loops over threads.
 *
 * Readings of passages the paper leaves open (documented with the project):
 *   - mu_rho^Bulk carries +lambda_2 g(C2)/drho (derivative of Eq. BulkEnergy);
 *   - the rho-phi gradient coefficient is kappa' = (kappa2-kappa3)/(4 chi drho)
 *     in both chemical potentials and in the pressure tensor (derivative of
 *     Eq. InterfEnergy);
 *   - stencils: grad Q = 3 sum w_i c_i Q(x+c_i), lap Q = 6 sum w_i (Q(x+c_i)-Q(x));
 *   - wall rules for div P at a fluid node next to a solid: no P value is
 *     taken from a solid node.  Along an axis with an adjacent solid node the
 *     derivative is one-sided (fluid-side differences, doubled; exact on
 *     linear fields); along the other axes each solid term is replaced by its
 *     mirror image across the wall axes (else by the node itself).  A
 *     literal zero wall-normal derivative leaves sessile drops 17 deg short
 *     of the prescribed geometric angle, against the paper's < 1 deg;
 *   - the wetting force acts on fluid nodes that are not in the first fluid
 *     layer, with s(y) = 1 on first-layer nodes;
 *   - geometric schemes: interface rules in the order 2-3, bulk 1-3, bulk
 *     1-2, sign of grad rho . grad phi, default 1-2; both rho and phi use
 *     the interface geometry of c; the sample point of interpolation lies
 *     at cot(theta) grad c/|grad c| from the first fluid node.
 */
#include "tlbo.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#define MAXQ 27

/* Lattice tables of one lattice type, (c is Q x 3, unused components 0). */
typedef struct { int D, Q; int c[MAXQ * 3]; double w[MAXQ]; } lat_t;

static void lat_init(lat_t *L, int lattice);

struct tlbo_ctx {
    tlbo_params p;
    tlbo_derived d;
    int D, Q;
    long N;
    lat_t L;
    int c[MAXQ][3];
    double w[MAXQ];
    int opp[MAXQ];
    double cot_theta[3];      /* cot(theta_21), cot(theta_31), cot(theta_23) */
    uint8_t *solid;           /* 1 = solid */
    uint8_t *first;           /* fluid node with a solid lattice neighbour */
    uint8_t *ghost;           /* solid node with a fluid lattice neighbour */
    double *f, *g;            /* pre-collision populations, Q*N */
    double *fs, *gs;          /* post-collision populations, Q*N */
    double *rho, *phi;        /* including ghost values at solid nodes */
    double *ux;               /* bare velocity, 3*N */
    double *grho, *gphi;      /* gradients, 3*N */
    double *lrho, *lphi;      /* Laplacians */
    double *mur, *mup, *p0;   /* chemical potentials and bulk pressure */
    double *P;                /* pressure tensor, 6*N: xx yy zz xy xz yz */
    double *F;                /* total force, 3*N */
    long clipped;
};

/* ------------------------------------------------------------------ */
/* Lattice tables.  D2Q9 and D3Q27 are products of D1Q3 with weights   */
/* w(0) = 2/3, w(+-1) = 1/6; the product form of f^eq (Eq. eqrho)      */
/* is defined on these lattices.                                        */
/* ------------------------------------------------------------------ */
int tlbo_lattice(int lattice, int *c, double *w)
{
    int D = (lattice == TLBO_D3Q27) ? 3 : 2;
    int Q = (D == 3) ? 27 : 9;
    static const int digit_to_c[3] = {0, 1, -1};
    for (int i = 0; i < Q; ++i) {
        int rest = i;
        double wi = 1.0;
        for (int a = 0; a < 3; ++a) {
            int ca = 0;
            if (a < D) {
                ca = digit_to_c[rest % 3];
                rest /= 3;
                wi *= (ca == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
            }
            c[3 * i + a] = ca;
        }
        w[i] = wi;
    }
    return Q;
}

static void setup_lattice(tlbo_ctx *ctx)
{
    int ct[MAXQ * 3];
    ctx->D = (ctx->p.lattice == TLBO_D3Q27) ? 3 : 2;
    ctx->Q = tlbo_lattice(ctx->p.lattice, ct, ctx->w);
    lat_init(&ctx->L, ctx->p.lattice);
    for (int i = 0; i < ctx->Q; ++i)
        for (int a = 0; a < 3; ++a) ctx->c[i][a] = ct[3 * i + a];
    for (int i = 0; i < ctx->Q; ++i)
        for (int j = 0; j < ctx->Q; ++j)
            if (ctx->c[j][0] == -ctx->c[i][0] && ctx->c[j][1] == -ctx->c[i][1] &&
                ctx->c[j][2] == -ctx->c[i][2])
                ctx->opp[i] = j;
}

/* ------------------------------------------------------------------ */
/* Equations of state.  Carnahan-Starling: Eq. PsiEOS and its printed   */
/* derivative.  The paper names van der Waals and Peng-Robinson as      */
/* other EOS the model hosts (Sec. II.A); their Psi are the integrals   */
/* Psi/rho = int p/rho^2 drho of the textbook pressures (constant C):    */
/*   vdW: p = rho R T/(1 - b rho) - a rho^2,                              */
/*        Psi = rho (C - a rho + R T ln(rho/(1 - b rho)));                */
/*   PR:  p = rho R T/(1 - b rho) - a A rho^2/(1 + 2 b rho - b^2 rho^2),   */
/*        Psi = rho (C + R T ln(rho/(1 - b rho))                          */
/*              - a A/(2 sqrt2 b) ln((b rho + sqrt2 - 1)/(sqrt2 + 1 - b rho))),*/
/*        A = (1 + k (1 - sqrt(T/T_c)))^2, k = 0.37464 + 1.54226 omega     */
/*        - 0.26992 omega^2, T_c = (0.07780/0.45724) a/(b R).             */
/* ------------------------------------------------------------------ */
static double pr_alpha(double omega, double a, double b, double R, double T)
{
    double k = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
    double Tc = (0.07780 / 0.45724) * a / (b * R);
    double s = 1.0 + k * (1.0 - sqrt(T / Tc));
    return s * s;
}

double tlbo_eos_psi_k(int kind, double omega, double rho, double a, double b, double R, double T, double C)
{
    if (kind == TLBO_EOS_VDW) return rho * (C - a * rho + R * T * log(rho / (1.0 - b * rho)));
    if (kind == TLBO_EOS_PR) {
        double aa = a * pr_alpha(omega, a, b, R, T), r2 = sqrt(2.0);
        return rho * (C + R * T * log(rho / (1.0 - b * rho)) -
                      aa / (2.0 * r2 * b) * log((b * rho + r2 - 1.0) / (r2 + 1.0 - b * rho)));
    }
    double br = b * rho;
    return rho * (C - a * rho - 8.0 * R * T * (br - 6.0) / ((br - 4.0) * (br - 4.0)) +
                  R * T * log(rho));
}

double tlbo_eos_dpsi_k(int kind, double omega, double rho, double a, double b, double R, double T, double C)
{
    if (kind == TLBO_EOS_VDW)
        return C - 2.0 * a * rho + R * T * log(rho / (1.0 - b * rho)) + R * T / (1.0 - b * rho);
    if (kind == TLBO_EOS_PR) {
        double aa = a * pr_alpha(omega, a, b, R, T), r2 = sqrt(2.0), br = b * rho;
        return C + R * T * log(rho / (1.0 - br)) + R * T / (1.0 - br) -
               aa / (2.0 * r2 * b) * log((br + r2 - 1.0) / (r2 + 1.0 - br)) -
               aa * rho / (1.0 + 2.0 * br - br * br);
    }
    double br = b * rho;
    double q = br - 4.0;
    return C - 2.0 * a * rho + R * T * (1.0 + log(rho)) + 16.0 * R * T * (br - 12.0) / (q * q * q);
}

double tlbo_eos_psi(double rho, double a, double b, double R, double T, double C)
{
    return tlbo_eos_psi_k(TLBO_EOS_CS, 0.0, rho, a, b, R, T, C);
}

double tlbo_eos_dpsi(double rho, double a, double b, double R, double T, double C)
{
    return tlbo_eos_dpsi_k(TLBO_EOS_CS, 0.0, rho, a, b, R, T, C);
}

/* p_eos = rho dPsi/drho - Psi (Sec. II.A); independent of C. */
double tlbo_eos_p_k(int kind, double omega, double rho, double a, double b, double R, double T)
{
    return rho * tlbo_eos_dpsi_k(kind, omega, rho, a, b, R, T, 0.0) - tlbo_eos_psi_k(kind, omega, rho, a, b, R, T, 0.0);
}

static double eos_dp(int kind, double om, double rho, double a, double b, double R, double T)
{
    double h = 1e-6 * rho;
    return (tlbo_eos_p_k(kind, om, rho + h, a, b, R, T) - tlbo_eos_p_k(kind, om, rho - h, a, b, R, T)) / (2.0 * h);
}

/* largest density of the EOS (packing limit) */
static double eos_rmax(int kind, double b) { return kind == TLBO_EOS_CS ? 4.0 / b : 1.0 / b; }

/* Spinodal densities: the interval where dp/drho < 0, scanned on a fine grid
 * and refined by bisection.  Returns 0 if the EOS has no unstable branch. */
static int eos_spinodal(int kind, double om, double a, double b, double R, double T, double *s1, double *s2)
{
    const int M = 4000;
    double rmax = eos_rmax(kind, b);
    int first = -1, last = -1;
    for (int k = 1; k < M; ++k) {
        double r = rmax * k / M;
        if (eos_dp(kind, om, r, a, b, R, T) < 0.0) {
            if (first < 0) first = k;
            last = k;
        }
    }
    if (first < 0) return 0;
    double lo = rmax * (first - 1) / M, hi = rmax * first / M;
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (lo + hi);
        if (eos_dp(kind, om, m, a, b, R, T) < 0.0) hi = m; else lo = m;
    }
    *s1 = hi;
    lo = rmax * last / M; hi = rmax * (last + 1) / M;
    for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (lo + hi);
        if (eos_dp(kind, om, m, a, b, R, T) < 0.0) lo = m; else hi = m;
    }
    *s2 = lo;
    return 1;
}

double tlbo_eos_critical_T_k(int kind, double omega, double a, double b, double R)
{
    /* T_c is the largest T with an unstable branch; bracket on a/(bR). */
    double lo = 0.05 * a / (b * R), hi = 1.0 * a / (b * R);
    double s1, s2;
    for (int it = 0; it < 100; ++it) {
        double m = 0.5 * (lo + hi);
        if (eos_spinodal(kind, omega, a, b, R, m, &s1, &s2)) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
}

double tlbo_eos_critical_T(double a, double b, double R) { return tlbo_eos_critical_T_k(TLBO_EOS_CS, 0.0, a, b, R); }

/* Root of p(rho) = P on [lo, hi] by bisection (p monotone there). */
static double eos_root(int kind, double om, double a, double b, double R, double T, double P, double lo, double hi)
{
    double plo = tlbo_eos_p_k(kind, om, lo, a, b, R, T) - P;
    for (int it = 0; it < 300; ++it) {
        double m = 0.5 * (lo + hi);
        double pm = tlbo_eos_p_k(kind, om, m, a, b, R, T) - P;
        if ((pm < 0.0) == (plo < 0.0)) { lo = m; plo = pm; } else hi = m;
        if (hi - lo <= 1e-17 * hi) break;
    }
    return 0.5 * (lo + hi);
}

/* Coexistence: equal pressure and equal chemical potential dPsi/drho of the
 * gas and liquid branches (common tangent, Sec. II.A).  Bisection on the
 * common pressure P between the spinodal pressures. */
int tlbo_eos_coexistence_k(int kind, double om, double a, double b, double R, double T, double out[4])
{
    double s1, s2;
    if (!eos_spinodal(kind, om, a, b, R, T, &s1, &s2)) return -1;
    double Plo = tlbo_eos_p_k(kind, om, s2, a, b, R, T), Phi = tlbo_eos_p_k(kind, om, s1, a, b, R, T);
    if (Plo < 0.0) Plo = 0.0;
    double rg = 0, rl = 0, rtop = eos_rmax(kind, b) * (1.0 - 1e-15);
    for (int it = 0; it < 200; ++it) {
        double P = 0.5 * (Plo + Phi);
        rg = eos_root(kind, om, a, b, R, T, P, 1e-300, s1);
        rl = eos_root(kind, om, a, b, R, T, P, s2, rtop);
        double dmu = tlbo_eos_dpsi_k(kind, om, rl, a, b, R, T, 0.0) - tlbo_eos_dpsi_k(kind, om, rg, a, b, R, T, 0.0);
        /* d mu = dp / rho along each branch (Gibbs-Duhem), so mu(rl) - mu(rg)
         * decreases as the common pressure P rises */
        if (dmu > 0.0) Plo = P; else Phi = P;
        if (Phi - Plo <= 1e-16 * Phi) break;
    }
    double P = 0.5 * (Plo + Phi);
    rg = eos_root(kind, om, a, b, R, T, P, 1e-300, s1);
    rl = eos_root(kind, om, a, b, R, T, P, s2, rtop);
    /* C makes the common tangent horizontal: dPsi/drho = 0 at both phases,
     * so Psi(rho_g) = Psi(rho_l) = Psi0. */
    double C = -0.5 * (tlbo_eos_dpsi_k(kind, om, rl, a, b, R, T, 0.0) + tlbo_eos_dpsi_k(kind, om, rg, a, b, R, T, 0.0));
    out[0] = rg;
    out[1] = rl;
    out[2] = C;
    out[3] = tlbo_eos_psi_k(kind, om, rl, a, b, R, T, C);
    return 0;
}

int tlbo_eos_coexistence(double a, double b, double R, double T, double out[4])
{
    return tlbo_eos_coexistence_k(TLBO_EOS_CS, 0.0, a, b, R, T, out);
}

/* ------------------------------------------------------------------ */
/* Product-form equilibrium (Eqs. eqrho, A, B).                          */
/* ------------------------------------------------------------------ */
static void lat_init(lat_t *L, int lattice)
{
    L->D = (lattice == TLBO_D3Q27) ? 3 : 2;
    L->Q = tlbo_lattice(lattice, L->c, L->w);
}

static void feq_t(const lat_t *L, double rho, const double *u, double *out)
{
    double A[3], B[3];
    for (int a = 0; a < L->D; ++a) {
        double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
        A[a] = 2.0 - s;                          /* Eq. A */
        B[a] = (2.0 * u[a] + s) / (1.0 - u[a]);  /* Eq. B */
    }
    for (int i = 0; i < L->Q; ++i) {
        double v = rho * L->w[i];
        for (int a = 0; a < L->D; ++a) {
            int ca = L->c[3 * i + a];
            /* A(u_a) B(u_a)^{c_ia} with c_ia in {-1, 0, 1} */
            v *= A[a] * (ca == 0 ? 1.0 : (ca > 0 ? B[a] : 1.0 / B[a]));
        }
        out[i] = v;
    }
}

void tlbo_feq(int lattice, double rho, const double *u, double *out)
{
    lat_t L;
    lat_init(&L, lattice);
    feq_t(&L, rho, u, out);
}

static double entropy_t(const lat_t *L, const double *f)
{
    double H = 0.0;
    for (int i = 0; i < L->Q; ++i) H += f[i] * log(f[i] / L->w[i]);
    return H;
}

double tlbo_entropy(int lattice, const double *f)
{
    lat_t L;
    lat_init(&L, lattice);
    return entropy_t(&L, f);
}

/* ------------------------------------------------------------------ */
/* Entropic alpha: the non-trivial root of h(alpha) = H(fp + alpha delta)  */
/* - H(fp) (Eq. EntropyEquation).  h(0) = 0, h is convex, h(1) <= 0        */
/* because fp + delta is the equilibrium with the moments of fp.  The root */
/* is bracketed in [1, alpha_max], alpha_max keeping every population      */
/* positive, and found by Newton's method safeguarded by bisection.        */
/* ------------------------------------------------------------------ */
/* h(alpha) = H(fp + alpha delta) - H(fp). */
static double hfun(const lat_t *L, const double *fp, const double *delta, double al, double H0)
{
    double tmp[MAXQ];
    for (int i = 0; i < L->Q; ++i) tmp[i] = fp[i] + al * delta[i];
    return entropy_t(L, tmp) - H0;
}

static double alpha_t(const lat_t *L, const double *fp, const double *delta, int *status)
{
    int Q = L->Q;
    double xmax = 0.0, amax = INFINITY, Hscale = 0.0;
    for (int i = 0; i < Q; ++i) {
        double x = fabs(delta[i]) / fp[i];
        if (x > xmax) xmax = x;
        if (delta[i] < 0.0) {
            double lim = -fp[i] / delta[i];
            if (lim < amax) amax = lim;
        }
        Hscale += fabs(fp[i] * log(fp[i] / L->w[i])) + fabs(fp[i]);
    }
    /* Near equilibrium the root tends to 2; below this relative deviation the
     * FP64 difference of two entropies no longer resolves h. */
    if (xmax < 1e-6) {
        if (status) *status = 1;
        return 2.0;
    }
    double H0 = entropy_t(L, fp);
    double lo = 1.0, hi;
    if (isfinite(amax)) {
        hi = amax * (1.0 - 1e-12);
        if (hi <= lo || hfun(L, fp, delta, hi, H0) < 0.0) {
            if (status) *status = 2;
            return amax * (1.0 - 1e-6);
        }
    } else {
        hi = 2.0;
        while (hfun(L, fp, delta, hi, H0) < 0.0 && hi < 1e6) hi *= 2.0;
    }
    double tol_h = 1e-15 * Hscale;
    double al = 2.0;
    if (al <= lo || al >= hi) al = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double h = hfun(L, fp, delta, al, H0), dh = 0.0;
        /* h'(alpha) = sum_i delta_i (ln((fp_i + alpha delta_i)/w_i) + 1) */
        for (int i = 0; i < Q; ++i) dh += delta[i] * (log((fp[i] + al * delta[i]) / L->w[i]) + 1.0);
        if (h > 0.0) hi = al; else lo = al;
        if (fabs(h) <= tol_h) break;
        double nxt = (dh != 0.0) ? al - h / dh : 0.5 * (lo + hi);
        /* a Newton step below the resolution of alpha is the root (checked
         * before the bracket test, which a converged step can touch) */
        if (fabs(nxt - al) <= 1e-14 * al) { al = nxt; break; }
        if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);
        al = nxt;
        if (hi - lo <= 1e-15 * hi) break;
    }
    if (status) *status = 0;
    return al;
}

double tlbo_alpha(int lattice, const double *fp, const double *delta, int *status)
{
    lat_t L;
    lat_init(&L, lattice);
    return alpha_t(&L, fp, delta, status);
}

/* Order-parameter equilibrium (Sec. II.C, g_i^eq and g_0^eq). */
static void geq_t(const lat_t *L, double phi, const double *v, double mu_phi, double Gamma, double *out)
{
    const double cs2 = 1.0 / 3.0;
    double sum = 0.0;
    for (int i = 1; i < L->Q; ++i) {
        const int *ci = L->c + 3 * i;
        double cu = 0.0, quad = 0.0;
        for (int a = 0; a < L->D; ++a) cu += v[a] * ci[a];
        for (int a = 0; a < L->D; ++a)
            for (int b = 0; b < L->D; ++b)
                quad += v[a] * v[b] * (ci[a] * ci[b] - cs2 * (a == b));
        out[i] = L->w[i] * (Gamma * mu_phi / cs2 + phi * cu / cs2 + phi * quad / (2.0 * cs2 * cs2));
        sum += out[i];
    }
    out[0] = phi - sum;
}

void tlbo_geq(int lattice, double phi, const double *v, double mu_phi, double Gamma, double *out)
{
    lat_t L;
    lat_init(&L, lattice);
    geq_t(&L, phi, v, mu_phi, Gamma, out);
}

/* ------------------------------------------------------------------ */
/* Context helpers                                                      */
/* ------------------------------------------------------------------ */
static long nb(const tlbo_ctx *ctx, long n, int dx, int dy, int dz)
{
    long nx = ctx->p.nx, ny = ctx->p.ny, nz = ctx->p.nz;
    long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    x = ((x + dx) % nx + nx) % nx;
    y = ((y + dy) % ny + ny) % ny;
    z = ((z + dz) % nz + nz) % nz;
    return x + nx * (y + ny * z);
}

static long nbc(const tlbo_ctx *ctx, long n, int i)
{
    return nb(ctx, n, ctx->c[i][0], ctx->c[i][1], ctx->c[i][2]);
}

static long nbe(const tlbo_ctx *ctx, long n, int axis, int s)
{
    int d[3] = {0, 0, 0};
    d[axis] = s;
    return nb(ctx, n, d[0], d[1], d[2]);
}

static double *dalloc(long n)
{
    double *p = (double *)calloc((size_t)n, sizeof(double));
    return p;
}

int tlbo_create(const tlbo_params *p, tlbo_ctx **out)
{
    if (!p || !out) return -1;
    if (p->lattice != TLBO_D2Q9 && p->lattice != TLBO_D3Q27) return -1;
    if (p->nx < 3 || p->ny < 3 || p->nz < 1) return -1;
    if (p->lattice == TLBO_D2Q9 && p->nz != 1) return -1;
    if (p->lattice == TLBO_D3Q27 && p->nz < 3) return -1;
    if (!(p->rho_l > p->rho_g && p->rho_g > 0.0)) return -1;
    if (p->eos < TLBO_EOS_CS || p->eos > TLBO_EOS_PR) return -1;
    for (int k = 0; k < 3; ++k)
        if (p->nu[k] < 0.0) return -1;
    tlbo_ctx *ctx = (tlbo_ctx *)calloc(1, sizeof(tlbo_ctx));
    ctx->p = *p;
    setup_lattice(ctx);
    ctx->N = (long)p->nx * p->ny * p->nz;

    /* Density ratio r = rho_l/rho_g fixes T (bisection on T/T_c), then a and b
     * are scaled by s = rho_l(T)/rho_l_target, which keeps T_c and the ratio
     * and moves the coexistence densities to the targets. */
    const int K = p->eos;
    const double om = p->omega;
    double Tc = tlbo_eos_critical_T_k(K, om, p->a, p->b, p->R);
    double ratio = p->rho_l / p->rho_g, co[4];
    double lo = 0.05, hi = 0.9999;
    for (int it = 0; it < 60; ++it) {
        double m = 0.5 * (lo + hi);
        if (tlbo_eos_coexistence_k(K, om, p->a, p->b, p->R, m * Tc, co) != 0) { hi = m; continue; }
        if (co[1] / co[0] > ratio) lo = m; else hi = m;
    }
    double T = 0.5 * (lo + hi) * Tc;
    tlbo_eos_coexistence_k(K, om, p->a, p->b, p->R, T, co);
    double s = co[1] / p->rho_l;
    ctx->d.T = T;
    ctx->d.R = p->R;
    ctx->d.a = p->a * s;
    ctx->d.b = p->b * s;
    ctx->d.Tc = Tc;
    tlbo_eos_coexistence_k(K, om, ctx->d.a, ctx->d.b, p->R, T, co);
    ctx->d.rho_g = co[0];
    ctx->d.rho_l = co[1];
    ctx->d.C = co[2];
    ctx->d.Psi0 = co[3];
    /* Gradient coefficients from Eq. InterfEnergy with grad C2 = grad rho/(2 drho)
     * + grad phi/(2 chi) and grad C3 = grad rho/(2 drho) - grad phi/(2 chi). */
    double drho = ctx->d.rho_l - ctx->d.rho_g, chi = p->chi;
    ctx->d.kappa_rr = p->kappa[0] + (p->kappa[1] + p->kappa[2]) / (4.0 * drho * drho);
    ctx->d.kappa_pp = (p->kappa[1] + p->kappa[2]) / (4.0 * chi * chi);
    ctx->d.kappa_rp = (p->kappa[1] - p->kappa[2]) / (4.0 * chi * drho);
    for (int k = 0; k < 3; ++k) ctx->cot_theta[k] = 1.0 / tan(p->theta_deg[k] * M_PI / 180.0);

    long N = ctx->N;
    int Q = ctx->Q;
    ctx->solid = (uint8_t *)calloc((size_t)N, 1);
    ctx->first = (uint8_t *)calloc((size_t)N, 1);
    ctx->ghost = (uint8_t *)calloc((size_t)N, 1);
    ctx->f = dalloc(Q * N); ctx->g = dalloc(Q * N);
    ctx->fs = dalloc(Q * N); ctx->gs = dalloc(Q * N);
    ctx->rho = dalloc(N); ctx->phi = dalloc(N);
    ctx->ux = dalloc(3 * N);
    ctx->grho = dalloc(3 * N); ctx->gphi = dalloc(3 * N);
    ctx->lrho = dalloc(N); ctx->lphi = dalloc(N);
    ctx->mur = dalloc(N); ctx->mup = dalloc(N); ctx->p0 = dalloc(N);
    ctx->P = dalloc(6 * N);
    ctx->F = dalloc(3 * N);
    *out = ctx;
    return 0;
}

void tlbo_destroy(tlbo_ctx *ctx)
{
    if (!ctx) return;
    free(ctx->solid); free(ctx->first); free(ctx->ghost);
    free(ctx->f); free(ctx->g); free(ctx->fs); free(ctx->gs);
    free(ctx->rho); free(ctx->phi); free(ctx->ux);
    free(ctx->grho); free(ctx->gphi); free(ctx->lrho); free(ctx->lphi);
    free(ctx->mur); free(ctx->mup); free(ctx->p0); free(ctx->P); free(ctx->F);
    free(ctx);
}

int tlbo_get_derived(const tlbo_ctx *ctx, tlbo_derived *out)
{
    if (!ctx || !out) return -1;
    *out = ctx->d;
    return 0;
}

int tlbo_set_solid(tlbo_ctx *ctx, const uint8_t *mask)
{
    long N = ctx->N;
    for (long n = 0; n < N; ++n) ctx->solid[n] = mask[n] ? 1 : 0;
    for (long n = 0; n < N; ++n) {
        int touch = 0;
        for (int i = 1; i < ctx->Q; ++i)
            if (ctx->solid[nbc(ctx, n, i)] != ctx->solid[n]) touch = 1;
        ctx->first[n] = (!ctx->solid[n] && touch);
        ctx->ghost[n] = (ctx->solid[n] && touch);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Step 1: moments.                                                     */
/* ------------------------------------------------------------------ */
static void moments(tlbo_ctx *ctx)
{
    long N = ctx->N;
    int Q = ctx->Q, D = ctx->D;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) { ctx->rho[n] = ctx->phi[n] = 0.0; continue; }
        double r = 0.0, ph = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            double fi = ctx->f[i * N + n];
            r += fi;
            ph += ctx->g[i * N + n];
            for (int a = 0; a < D; ++a) j[a] += fi * ctx->c[i][a];
        }
        ctx->rho[n] = r;
        ctx->phi[n] = ph;
        for (int a = 0; a < 3; ++a) ctx->ux[a * N + n] = (a < D) ? j[a] / r : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Step 2: ghost layer (Sec. IV).                                       */
/* ------------------------------------------------------------------ */
static int fluid(const tlbo_ctx *ctx, long n) { return !ctx->solid[n]; }

/* Value of field v at the node y + off_t (in-plane offset k along axis t,
 * and k2 along t2 in 3D); non-fluid samples are replaced by v(y). */
static double sample(const tlbo_ctx *ctx, const double *v, long y, int t, int k, int t2, int k2)
{
    long m = y;
    if (k) m = nbe(ctx, m, t, k);
    if (t2 >= 0 && k2) m = nbe(ctx, m, t2, k2);
    return fluid(ctx, m) ? v[m] : v[y];
}

/* In-plane derivative of v at fluid node y along axis t: central difference
 * between fluid neighbours, one-sided if only one is fluid, else 0. */
static double inplane_grad(const tlbo_ctx *ctx, const double *v, long y, int t)
{
    long yp = nbe(ctx, y, t, +1), ym = nbe(ctx, y, t, -1);
    int fp = fluid(ctx, yp), fm = fluid(ctx, ym);
    if (fp && fm) return 0.5 * (v[yp] - v[ym]);
    if (fp) return v[yp] - v[y];
    if (fm) return v[y] - v[ym];
    return 0.0;
}

/* Plane through three points (x_k, y_k, c_k) evaluated at (px, py)
 * (Eq. interp3D: the plane through the three selected support points). */
static double plane3(const double *xs, const double *ys, const double *cs, double px, double py)
{
    double det = (xs[1] - xs[0]) * (ys[2] - ys[0]) - (xs[2] - xs[0]) * (ys[1] - ys[0]);
    double l1 = ((px - xs[0]) * (ys[2] - ys[0]) - (xs[2] - xs[0]) * (py - ys[0])) / det;
    double l2 = ((xs[1] - xs[0]) * (py - ys[0]) - (px - xs[0]) * (ys[1] - ys[0])) / det;
    return cs[0] + l1 * (cs[1] - cs[0]) + l2 * (cs[2] - cs[0]);
}

/* Ghost value seen from one fluid-facing direction: first fluid node y, wall
 * normal axis a.  Writes rho and phi of the ghost. */
static void ghost_one_axis(const tlbo_ctx *ctx, long y, int a, double *gr, double *gp)
{
    const tlbo_params *p = &ctx->p;
    double r1 = ctx->rho[y], p1 = ctx->phi[y];
    if (p->wetting == TLBO_WET_FORCE) { *gr = r1; *gp = p1; return; }

    int T[2], nt = 0;
    for (int t = 0; t < ctx->D; ++t)
        if (t != a) T[nt++] = t;
    double dr[2] = {0, 0}, dp[2] = {0, 0};
    for (int k = 0; k < nt; ++k) {
        dr[k] = inplane_grad(ctx, ctx->rho, y, T[k]);
        dp[k] = inplane_grad(ctx, ctx->phi, y, T[k]);
    }
    double nr = 0, np = 0, dot = 0;
    for (int k = 0; k < nt; ++k) { nr += dr[k] * dr[k]; np += dp[k] * dp[k]; dot += dr[k] * dp[k]; }
    nr = sqrt(nr);
    np = sqrt(np);

    /* Interface identification (Sec. IV.B rules). pair: 0 = 1-2, 1 = 1-3, 2 = 2-3 */
    double rl = ctx->d.rho_l, rg = ctx->d.rho_g, chi = p->chi;
    int pair;
    if (nr < 0.01 * (rl - rg) / chi * np) pair = 2;
    else if (r1 > 0.5 * rl && p1 < -0.95 * chi) pair = 1;
    else if (r1 > 0.5 * rl && p1 > 0.95 * chi) pair = 0;
    else if (dot < 0.0) pair = 1;
    else pair = 0;
    const double *dc = (pair == 2) ? dp : dr;
    double nc = (pair == 2) ? np : nr;
    double cot = ctx->cot_theta[pair];   /* theta_21, theta_31, theta_23 */
    if (!(nc > 1e-12)) { *gr = r1; *gp = p1; return; }
    double tx = dc[0] / nc, ty = (nt > 1) ? dc[1] / nc : 0.0;

    if (p->wetting == TLBO_WET_GEOM_EXTRAP) {
        /* Eqs. geomamgle, geomding: c_ghost = c_1 + tan(pi/2 - theta)|grad_par c|;
         * the other field uses the same interface direction. */
        double sr = dr[0] * tx + (nt > 1 ? dr[1] * ty : 0.0);
        double sp = dp[0] * tx + (nt > 1 ? dp[1] * ty : 0.0);
        *gr = r1 + cot * sr;
        *gp = p1 + cot * sp;
        return;
    }

    /* Geometric interpolation (Eqs. interp2D, interp3D): sample both fields at
     * the point cot(theta) t_hat of the first fluid layer. */
    if (nt == 1) {
        double l = cot * tx;
        int l0 = (int)floor(l), l1 = l0 + 1;
        double v0r = sample(ctx, ctx->rho, y, T[0], l0, -1, 0), v1r = sample(ctx, ctx->rho, y, T[0], l1, -1, 0);
        double v0p = sample(ctx, ctx->phi, y, T[0], l0, -1, 0), v1p = sample(ctx, ctx->phi, y, T[0], l1, -1, 0);
        *gr = (v1r - v0r) * l + (l1 * v0r - l0 * v1r);
        *gp = (v1p - v0p) * l + (l1 * v0p - l0 * v1p);
        return;
    }
    double lx = cot * tx, ly = cot * ty;
    if (hypot(lx, ly) < 1e-12) { *gr = r1; *gp = p1; return; }
    int X0 = (int)floor(lx), Y0 = (int)floor(ly);
    int cx[4], cy[4];
    double d2[4];
    for (int k = 0; k < 4; ++k) {
        cx[k] = X0 + (k & 1);
        cy[k] = Y0 + (k >> 1);
        d2[k] = (double)cx[k] * cx[k] + (double)cy[k] * cy[k];
    }
    int drop = 0;
    for (int k = 1; k < 4; ++k)
        if (d2[k] < d2[drop]) drop = k;
    double xs[3], ys[3], csr[3], csp[3];
    int m = 0;
    for (int k = 0; k < 4; ++k) {
        if (k == drop) continue;
        xs[m] = cx[k];
        ys[m] = cy[k];
        csr[m] = sample(ctx, ctx->rho, y, T[0], cx[k], T[1], cy[k]);
        csp[m] = sample(ctx, ctx->phi, y, T[0], cx[k], T[1], cy[k]);
        ++m;
    }
    *gr = plane3(xs, ys, csr, lx, ly);
    *gp = plane3(xs, ys, csp, lx, ly);
}

static void ghost_fill(tlbo_ctx *ctx)
{
    long N = ctx->N;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (!ctx->ghost[n]) continue;
        double sr = 0.0, sp = 0.0;
        int cnt = 0;
        /* Average over fluid-facing axis directions (corners, wedges). */
        for (int a = 0; a < ctx->D; ++a)
            for (int s = -1; s <= 1; s += 2) {
                long y = nbe(ctx, n, a, s);
                if (!fluid(ctx, y)) continue;
                double gr, gp;
                ghost_one_axis(ctx, y, a, &gr, &gp);
                sr += gr; sp += gp; ++cnt;
            }
        if (cnt == 0) {
            /* Only diagonal fluid neighbours: mean of their values. */
            for (int i = 1; i < ctx->Q; ++i) {
                long y = nbc(ctx, n, i);
                if (!fluid(ctx, y)) continue;
                sr += ctx->rho[y]; sp += ctx->phi[y]; ++cnt;
            }
        }
        ctx->rho[n] = sr / cnt;
        ctx->phi[n] = sp / cnt;
    }
}

/* ------------------------------------------------------------------ */
/* Steps 3-4: stencils, chemical potentials, pressure tensor.            */
/* ------------------------------------------------------------------ */
static double gfun(double x) { return x * (x - 0.5) * (x - 1.0); }

static void thermo(tlbo_ctx *ctx)
{
    long N = ctx->N;
    int Q = ctx->Q, D = ctx->D;
    const tlbo_params *p = &ctx->p;
    const tlbo_derived *d = &ctx->d;
    double drho = d->rho_l - d->rho_g, chi = p->chi;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) continue;
        double gr[3] = {0, 0, 0}, gp[3] = {0, 0, 0}, lr = 0.0, lp = 0.0;
        double r0 = ctx->rho[n], p0v = ctx->phi[n];
        for (int i = 1; i < Q; ++i) {
            long m = nbc(ctx, n, i);
            for (int a = 0; a < D; ++a) {
                gr[a] += 3.0 * ctx->w[i] * ctx->c[i][a] * ctx->rho[m];
                gp[a] += 3.0 * ctx->w[i] * ctx->c[i][a] * ctx->phi[m];
            }
            lr += 6.0 * ctx->w[i] * (ctx->rho[m] - r0);
            lp += 6.0 * ctx->w[i] * (ctx->phi[m] - p0v);
        }
        for (int a = 0; a < 3; ++a) { ctx->grho[a * N + n] = gr[a]; ctx->gphi[a * N + n] = gp[a]; }
        ctx->lrho[n] = lr;
        ctx->lphi[n] = lp;

        /* Concentrations (Eqs. definitionC1-C3). */
        double C1 = (r0 - d->rho_l) / (d->rho_g - d->rho_l);
        double C2 = 0.5 * (1.0 + p0v / chi - C1);
        double C3 = 0.5 * (1.0 - p0v / chi - C1);
        /* Bulk free energy and chemical potentials (Eq. BulkEnergy and its
         * derivatives with dC2/drho = dC3/drho = 1/(2 drho), dC2/dphi =
         * -dC3/dphi = 1/(2 chi)). */
        double psi = tlbo_eos_psi_k(p->eos, p->omega, r0, d->a, d->b, d->R, d->T, d->C);
        double dpsi = tlbo_eos_dpsi_k(p->eos, p->omega, r0, d->a, d->b, d->R, d->T, d->C);
        double fb = 0.5 * p->lambda[0] * (psi - d->Psi0) +
                    0.5 * p->lambda[1] * C2 * C2 * (1 - C2) * (1 - C2) +
                    0.5 * p->lambda[2] * C3 * C3 * (1 - C3) * (1 - C3);
        double murB = 0.5 * p->lambda[0] * dpsi + (p->lambda[1] * gfun(C2) + p->lambda[2] * gfun(C3)) / drho;
        double mupB = (p->lambda[1] * gfun(C2) - p->lambda[2] * gfun(C3)) / chi;
        double krr = d->kappa_rr, kpp = d->kappa_pp, krp = d->kappa_rp;
        ctx->mur[n] = murB - krr * lr - krp * lp;
        ctx->mup[n] = mupB - kpp * lp - krp * lr;
        double pb = r0 * murB + p0v * mupB - fb;    /* Eq. bulkpressure */
        ctx->p0[n] = pb;

        /* Pressure tensor (Eq. pressuretensor). */
        double g2r = 0, g2p = 0, grp = 0;
        for (int a = 0; a < D; ++a) { g2r += gr[a] * gr[a]; g2p += gp[a] * gp[a]; grp += gr[a] * gp[a]; }
        double iso = pb - krr * (r0 * lr + 0.5 * g2r) - kpp * (p0v * lp + 0.5 * g2p) -
                     krp * (r0 * lp + p0v * lr + grp);
        static const int pa[6] = {0, 1, 2, 0, 0, 1}, pbb[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) {
            int a = pa[k], b = pbb[k];
            double v = krr * gr[a] * gr[b] + kpp * gp[a] * gp[b] + krp * (gr[a] * gp[b] + gp[a] * gr[b]);
            if (a == b) v += iso;
            ctx->P[k * N + n] = v;
        }
    }
}

static int ptens_index(int a, int b)
{
    if (a == b) return a;
    if (a > b) { int t = a; a = b; b = t; }
    return (a == 0) ? (b == 1 ? 3 : 4) : 5;
}

/* Q_ab = rho c_s^2 delta_ab - P_ab at node m. */
static double qtens(const tlbo_ctx *ctx, long m, int a, int b)
{
    double v = -ctx->P[ptens_index(a, b) * ctx->N + m];
    if (a == b) v += ctx->rho[m] / 3.0;
    return v;
}

/* ------------------------------------------------------------------ */
/* Step 5: force (Eq. force) with the wall rules and Eq. forceBC.         */
/* ------------------------------------------------------------------ */
static void force(tlbo_ctx *ctx)
{
    long N = ctx->N;
    int Q = ctx->Q, D = ctx->D;
    const tlbo_params *p = &ctx->p;
    const tlbo_derived *d = &ctx->d;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) continue;
        int wall[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a)
            wall[a] = ctx->solid[nbe(ctx, n, a, +1)] || ctx->solid[nbe(ctx, n, a, -1)];
        double F[3] = {0, 0, 0};
        for (int g = 0; g < D; ++g) {          /* derivative direction */
            if (wall[g]) {
                /* Wall-normal derivative: one-sided stencil that takes no value
                 * from solid nodes -- the isotropic stencil written in
                 * differences Q(x+c_i) - Q(x), solid targets dropped and the
                 * remaining half doubled (exact on linear fields). */
                for (int i = 1; i < Q; ++i) {
                    if (ctx->c[i][g] == 0) continue;
                    long m = nbc(ctx, n, i);
                    if (ctx->solid[m]) continue;
                    for (int a = 0; a < D; ++a)
                        F[a] += 6.0 * ctx->w[i] * ctx->c[i][g] * (qtens(ctx, m, a, g) - qtens(ctx, n, a, g));
                }
                continue;
            }
            for (int i = 1; i < Q; ++i) {
                if (ctx->c[i][g] == 0) continue;
                long m = nbc(ctx, n, i);
                if (ctx->solid[m]) {
                    /* mirror across the wall axes */
                    int cm[3] = {ctx->c[i][0], ctx->c[i][1], ctx->c[i][2]};
                    for (int a = 0; a < D; ++a)
                        if (wall[a]) cm[a] = -cm[a];
                    long mm = nb(ctx, n, cm[0], cm[1], cm[2]);
                    m = ctx->solid[mm] ? n : mm;
                }
                for (int a = 0; a < D; ++a)
                    F[a] += 3.0 * ctx->w[i] * ctx->c[i][g] * qtens(ctx, m, a, g);
            }
        }
        if (p->wetting == TLBO_WET_FORCE && !ctx->first[n] && (p->kw_rho != 0.0 || p->kw_phi != 0.0)) {
            double rrel = (ctx->rho[n] - d->rho_g) / (d->rho_l - d->rho_g);
            double prel = ctx->phi[n] / p->chi;
            double amp = rrel * (p->kw_rho + prel * p->kw_phi);
            for (int i = 1; i < Q; ++i) {
                long m = nbc(ctx, n, i);
                if (!ctx->first[m]) continue;
                for (int a = 0; a < D; ++a) F[a] += amp * ctx->w[i] * ctx->c[i][a];
            }
        }
        for (int a = 0; a < 3; ++a) ctx->F[a * N + n] = F[a];
    }
}

static void macro_pipeline(tlbo_ctx *ctx)
{
    moments(ctx);
    ghost_fill(ctx);
    thermo(ctx);
    force(ctx);
}

/* ------------------------------------------------------------------ */
/* Step 6: collisions.                                                  */
/* ------------------------------------------------------------------ */
static int collide(tlbo_ctx *ctx)
{
    long N = ctx->N;
    int Q = ctx->Q;
    const tlbo_params *p = &ctx->p;
    int bad = 0;
    long clipped = 0;
#pragma omp parallel for schedule(static) reduction(|:bad) reduction(+:clipped)
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) continue;
        double r = ctx->rho[n], u[3], du[3], ud[3], v[3];
        for (int a = 0; a < 3; ++a) {
            u[a] = ctx->ux[a * N + n];
            du[a] = ctx->F[a * N + n] / r;          /* delta u = F dt / rho */
            ud[a] = u[a] + du[a];
            v[a] = u[a] + 0.5 * du[a];              /* actual fluid velocity */
        }
        double feq[MAXQ], feqd[MAXQ], fp[MAXQ], dl[MAXQ];
        feq_t(&ctx->L, r, u, feq);
        feq_t(&ctx->L, r, ud, feqd);
        int nonpos = !(r > 0.0);
        for (int i = 0; i < Q; ++i) {
            double fi = ctx->f[i * N + n];
            double Fi = feqd[i] - feq[i];           /* Eq. ELBMForcingExactDiff */
            fp[i] = fi + Fi;                        /* Eq. mirror_state */
            dl[i] = feqd[i] - fp[i];                /* f^eq(u + du) - f' */
            if (!(fp[i] > 0.0)) nonpos = 1;
        }
        double al = 2.0;
        if (!nonpos) {
            int st = 0;
            al = alpha_t(&ctx->L, fp, dl, &st);
            if (st == 2) ++clipped;
        } else {
            bad = 1;
        }
        double beta = p->beta;
        if (p->nu[0] > 0.0 || p->nu[1] > 0.0 || p->nu[2] > 0.0) {
            /* viscosity of the local mixture: the concentration-weighted mean
             * of the components' kinematic viscosities (concentrations
             * clipped to [0, 1]), nu = (1/beta - 1)/6 */
            const tlbo_derived *d = &ctx->d;
            double C1 = (r - d->rho_l) / (d->rho_g - d->rho_l);
            double C2 = 0.5 * (1.0 + ctx->phi[n] / p->chi - C1), C3 = 0.5 * (1.0 - ctx->phi[n] / p->chi - C1);
            double c[3] = {C1, C2, C3}, ws = 0.0, nu = 0.0;
            for (int k = 0; k < 3; ++k) {
                double ck = c[k] < 0.0 ? 0.0 : (c[k] > 1.0 ? 1.0 : c[k]);
                ws += ck;
                nu += ck * p->nu[k];
            }
            nu /= ws;
            beta = 1.0 / (6.0 * nu + 1.0);
        }
        for (int i = 0; i < Q; ++i) {
            double fi = ctx->f[i * N + n];
            /* Eq. ELBMequation */
            ctx->fs[i * N + n] = fi + al * beta * (feq[i] - fi) + (feqd[i] - feq[i]);
        }
        double geq[MAXQ];
        geq_t(&ctx->L, ctx->phi[n], v, ctx->mup[n], p->Gamma, geq);
        for (int i = 0; i < Q; ++i) {
            double gi = ctx->g[i * N + n];
            ctx->gs[i * N + n] = gi + (geq[i] - gi) / p->tau_g;   /* Eq. CahnHilliardLBM */
        }
    }
    ctx->clipped += clipped;
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* Step 7: streaming with halfway bounce-back.                            */
/* ------------------------------------------------------------------ */
static void stream(tlbo_ctx *ctx)
{
    long N = ctx->N;
    int Q = ctx->Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) continue;
        for (int i = 0; i < Q; ++i) {
            long src = nb(ctx, n, -ctx->c[i][0], -ctx->c[i][1], -ctx->c[i][2]);
            if (ctx->solid[src]) {
                ctx->f[i * N + n] = ctx->fs[ctx->opp[i] * N + n];
                ctx->g[i * N + n] = ctx->gs[ctx->opp[i] * N + n];
            } else {
                ctx->f[i * N + n] = ctx->fs[i * N + src];
                ctx->g[i * N + n] = ctx->gs[i * N + src];
            }
        }
    }
}

int tlbo_step(tlbo_ctx *ctx, int nsteps)
{
    for (int s = 0; s < nsteps; ++s) {
        macro_pipeline(ctx);
        int rc = collide(ctx);
        if (rc) return rc;
        stream(ctx);
    }
    return 0;
}

/* Initial populations.  The velocity given is the fluid velocity
 * v = u + delta u / 2 of Sec. II.C, so the bare velocity of f is
 * u = v - F/(2 rho) with the force F of the initial fields:
 * f = f^eq(rho, u) and g = g^eq(phi, v, mu_phi), with mu_phi and F from one
 * pass of the stencil pipeline over the initial fields. */
int tlbo_init_fields(tlbo_ctx *ctx, const double *rho, const double *phi, const double *u)
{
    long N = ctx->N;
    int Q = ctx->Q, D = ctx->D;
    double *v = dalloc(3 * N);
    for (long n = 0; n < N; ++n) {
        ctx->rho[n] = ctx->solid[n] ? 0.0 : rho[n];
        ctx->phi[n] = ctx->solid[n] ? 0.0 : phi[n];
        for (int a = 0; a < 3; ++a)
            v[a * N + n] = (u && a < D && !ctx->solid[n]) ? u[a * N + n] : 0.0;
    }
    ghost_fill(ctx);
    thermo(ctx);
    force(ctx);
    for (long n = 0; n < N; ++n) {
        double feq[MAXQ], geq[MAXQ], ub[3], vv[3];
        if (ctx->solid[n]) {
            for (int i = 0; i < Q; ++i) ctx->f[i * N + n] = ctx->g[i * N + n] = 0.0;
            continue;
        }
        for (int a = 0; a < 3; ++a) {
            vv[a] = v[a * N + n];
            ub[a] = vv[a] - 0.5 * ctx->F[a * N + n] / ctx->rho[n];
        }
        feq_t(&ctx->L, ctx->rho[n], ub, feq);
        geq_t(&ctx->L, ctx->phi[n], vv, ctx->mup[n], ctx->p.Gamma, geq);
        for (int i = 0; i < Q; ++i) {
            ctx->f[i * N + n] = feq[i];
            ctx->g[i * N + n] = geq[i];
        }
    }
    free(v);
    return 0;
}

int tlbo_get_fields(tlbo_ctx *ctx, double *rho, double *phi, double *u, double *C)
{
    long N = ctx->N;
    int D = ctx->D;
    moments(ctx);
    const tlbo_derived *d = &ctx->d;
    for (long n = 0; n < N; ++n) {
        int s = ctx->solid[n];
        double r = s ? 0.0 : ctx->rho[n], ph = s ? 0.0 : ctx->phi[n];
        if (rho) rho[n] = r;
        if (phi) phi[n] = ph;
        if (u)
            for (int a = 0; a < D; ++a) u[a * N + n] = s ? 0.0 : ctx->ux[a * N + n];
        if (C) {
            double C1 = (r - d->rho_l) / (d->rho_g - d->rho_l);
            double C2 = 0.5 * (1.0 + ph / ctx->p.chi - C1), C3 = 0.5 * (1.0 - ph / ctx->p.chi - C1);
            C[n] = s ? 0.0 : C1;
            C[N + n] = s ? 0.0 : C2;
            C[2 * N + n] = s ? 0.0 : C3;
        }
    }
    return 0;
}

int tlbo_get_populations(tlbo_ctx *ctx, double *f, double *g)
{
    size_t bytes = (size_t)ctx->Q * ctx->N * sizeof(double);
    if (f) memcpy(f, ctx->f, bytes);
    if (g) memcpy(g, ctx->g, bytes);
    return 0;
}

int tlbo_set_populations(tlbo_ctx *ctx, const double *f, const double *g)
{
    size_t bytes = (size_t)ctx->Q * ctx->N * sizeof(double);
    if (f) memcpy(ctx->f, f, bytes);
    if (g) memcpy(ctx->g, g, bytes);
    return 0;
}

int tlbo_get_aux(tlbo_ctx *ctx, int which, double *out)
{
    long N = ctx->N;
    macro_pipeline(ctx);
    const double *src = NULL;
    switch (which) {
    case 0: src = ctx->p0; break;
    case 1: src = ctx->mur; break;
    case 2: src = ctx->mup; break;
    case 3: case 4: case 5: src = ctx->F + (long)(which - 3) * N; break;
    case 6: case 7: case 8: case 9: case 10: case 11: src = ctx->P + (long)(which - 6) * N; break;
    case 12: src = ctx->rho; break;
    case 13: src = ctx->phi; break;
    default: return -1;
    }
    for (long n = 0; n < N; ++n) out[n] = (ctx->solid[n] && which < 12) ? 0.0 : src[n];
    return 0;
}

int tlbo_diagnostics(tlbo_ctx *ctx, double out[6])
{
    long N = ctx->N;
    int D = ctx->D;
    moments(ctx);
    const tlbo_derived *d = &ctx->d;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (long n = 0; n < N; ++n) {
        if (ctx->solid[n]) continue;
        double r = ctx->rho[n], ph = ctx->phi[n];
        double C1 = (r - d->rho_l) / (d->rho_g - d->rho_l);
        s[0] += r;
        s[1] += ph;
        s[2] += C1;
        s[3] += 0.5 * (1.0 + ph / ctx->p.chi - C1);
        s[4] += 0.5 * (1.0 - ph / ctx->p.chi - C1);
        double u2 = 0.0;
        for (int a = 0; a < D; ++a) u2 += ctx->ux[a * N + n] * ctx->ux[a * N + n];
        s[5] += 0.5 * r * u2;
    }
    memcpy(out, s, sizeof(s));
    return 0;
}

long tlbo_alpha_clipped(const tlbo_ctx *ctx) { return ctx->clipped; }

/* Host threads of the node loops (OpenMP); n <= 0 leaves the setting alone.
 * Returns the number of threads the loops use. */
int tlbo_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}
