/*
 * lbhpde_oracle.c -- plain FP64 CPU oracle of the LBGK model for
 *     phi_t + sum_{k=1..m} alpha_k d_x^k Pi_k(phi) = 0,   m <= 6
 * (Shi, He, Guo, "Lattice Boltzmann Model for High-Order Nonlinear Partial
 * Differential Equations", arXiv:0907.1720).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness yardstick for the
 * CUDA library.  Only tests/, __graft_entry__.smoke() and bench.py (its CPU
 * baseline leg and its reference arm) may load it.  It shares no code, header,
 * table or helper with the GPU path, and the GPU path never calls it.
 *
 * Everything is IEEE double precision, evaluated in the order the paper writes
 * it.  Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Steps, in the paper's order:
 *   (1) tau_2..tau_6 from the relaxation time tau                Eq. (taus)
 *   (2) beta_k = alpha_k / (dt^{k-1} tau_k)                       Eqs. (NPDE3)-(NPDE6)
 *   (3) A_40, A_50, A_60                                          Eqs. (Pi4), (Pi5), (Pi6), (A40)-(A60)
 *   (4) auxiliary moments Pi_20..Pi_60 as integrals over phi      Sec. II C-F, Eqs. (Pi4)-(Pi6)
 *   (5) scaled moments Pibar_0..Pibar_{b-1}                       Sec. III A/B
 *   (6) EDF written out component by component                   Eqs. (EDF5), (EDF7)
 *   (7) LBGK collide, then stream                                 Eq. (LBE)
 *   (8) global relative error E                                   Sec. IV
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - integration constants of the auxiliary-moment integrals are zero, i.e.
 *     Pi_k0(phi) = integral from 0 to phi;
 *   - alpha_1 != 1 is folded into Pi_1 (the paper fixes alpha_1 = 1);
 *   - beta_k = 0 when alpha_k = 0 or Pi_k = 0 (Remark 2), and for m < k < b;
 *   - A_40, A_50, A_60 are applied as printed, whatever Pi_2..Pi_4 are; the
 *     model flags "inexact recovery" when the remarks' preconditions fail;
 *   - scheme 2 sets the highest moment Pibar_{b-1} to zero (Sec. IV, before
 *     Examples 4.5 and 4.8);
 *   - scheme | ORACLE_NO_AUX_CORRECTION leaves A_40, A_50, A_60 out (the paper derives them,
 *     but its Kuramoto-Sivashinsky errors of Table I are reproduced only without A_40);
 *   - f is initialised to f^eq(phi_0);
 *   - the grid is periodic with N nodes (oracle_step), or bounded by the non-equilibrium
 *     extrapolation of Guo et al. that Sec. IV cites (oracle_step_nee): after streaming, every
 *     population of the W = max|e| outer nodes at each end is rebuilt as
 *     f^eq(phi_b) + [f(x_f) - f^eq(phi(x_f))], phi_b the prescribed (exact) boundary value and
 *     x_f the node `depth` places inside the outer layer (depth 1: the nearest node that
 *     received all its populations from inside the grid).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_NC 64 /* capacity in powers of phi: i < OR_NC */
#define OR_NA 8  /* capacity in powers of phi^nu: a < OR_NA */

/* A generalised polynomial in phi with one real exponent nu > 0 (Sec. III C, class (1):
 * beta u^n u_x with real n):  p(phi) = sum_{a<na} sum_{i<n} c[a][i] phi^(i + a nu).
 * With na = 1 it is an ordinary polynomial, and nu plays no part. */
typedef struct {
    int n, na;
    double c[OR_NA][OR_NC];
} opoly;

typedef struct {
    int b;        /* number of lattice velocities: 5 or 7                  */
    int m;        /* order of the NPDE                                      */
    int scheme;   /* 1: all b moments; 2: Pibar_{b-1} = 0                   */
    int inexact;  /* 1 if a remark's precondition for exact recovery fails */
    double dx, dt, c, tau;
    double nu;       /* the real exponent of the phi^(i + a nu) terms (0: none) */
    double tk[7];    /* tk[k] = tau_k, k = 2..6                             */
    double alpha[7]; /* alpha[k], k = 1..6                                  */
    double beta[7];  /* beta[k],  k = 2..6                                  */
    double A40, A50, A60;
    opoly Pi[7];     /* Pi[k] = Pi_k(phi), k = 1..6 (alpha_1 folded in)    */
    opoly Pi0[7];    /* Pi0[k] = Pi_k0(phi), k = 2..6                       */
} oracle_model;

/* ---------------------------------------------------------------- polys */

static void op_zero(opoly *p) { memset(p, 0, sizeof(*p)); }

static int op_is_zero(const opoly *p)
{
    for (int a = 0; a < p->na; a++)
        for (int i = 0; i < p->n; i++)
            if (p->c[a][i] != 0.0) return 0;
    return 1;
}

/* dst += s * src */
static int op_axpy(opoly *dst, double s, const opoly *src)
{
    if (src->n > OR_NC || src->na > OR_NA) return -1;
    for (int a = 0; a < src->na; a++)
        for (int i = 0; i < src->n; i++) dst->c[a][i] += s * src->c[a][i];
    if (src->n > dst->n) dst->n = src->n;
    if (src->na > dst->na) dst->na = src->na;
    return 0;
}

/* r = x * y:  phi^(i + a nu) phi^(j + b nu) = phi^(i + j + (a + b) nu) */
static int op_mul(opoly *r, const opoly *x, const opoly *y)
{
    opoly t;
    op_zero(&t);
    if (x->n == 0 || y->n == 0 || x->na == 0 || y->na == 0) { *r = t; return 0; }
    if (x->n + y->n - 1 > OR_NC || x->na + y->na - 1 > OR_NA) return -1;
    t.n = x->n + y->n - 1;
    t.na = x->na + y->na - 1;
    for (int a = 0; a < x->na; a++)
        for (int i = 0; i < x->n; i++) {
            if (x->c[a][i] == 0.0) continue;
            for (int b = 0; b < y->na; b++)
                for (int j = 0; j < y->n; j++) t.c[a + b][i + j] += x->c[a][i] * y->c[b][j];
        }
    *r = t;
    return 0;
}

/* r = x^k, k >= 0 */
static int op_pow(opoly *r, const opoly *x, int k)
{
    opoly t;
    op_zero(&t);
    t.n = 1;
    t.na = 1;
    t.c[0][0] = 1.0;
    for (int i = 0; i < k; i++)
        if (op_mul(&t, &t, x)) return -1;
    *r = t;
    return 0;
}

/* r = d/dphi x:  d phi^(i + a nu) = (i + a nu) phi^(i - 1 + a nu).  A term phi^(a nu) with
 * a >= 1 has no derivative of this form: -1. */
static int op_deriv(opoly *r, const opoly *x, double nu)
{
    opoly t;
    op_zero(&t);
    for (int a = 1; a < x->na; a++)
        if (x->n > 0 && x->c[a][0] != 0.0) return -1;
    for (int a = 0; a < x->na; a++)
        for (int i = 1; i < x->n; i++) t.c[a][i - 1] = ((double)i + (double)a * nu) * x->c[a][i];
    t.n = x->n > 1 ? x->n - 1 : 0;
    t.na = x->na;
    *r = t;
    return 0;
}

/* r = integral_0^phi x(s) ds  (zero integration constant):
 *   phi^(i + a nu) -> phi^(i + 1 + a nu) / (i + 1 + a nu) */
static int op_integ(opoly *r, const opoly *x, double nu)
{
    opoly t;
    op_zero(&t);
    if (x->n + 1 > OR_NC) return -1;
    for (int a = 0; a < x->na; a++)
        for (int i = 0; i < x->n; i++) t.c[a][i + 1] = x->c[a][i] / ((double)(i + 1) + (double)a * nu);
    t.n = x->n + 1;
    t.na = x->na;
    *r = t;
    return 0;
}

/* Plain power-sum evaluation: sum_a (phi^nu)^a sum_i c[a][i] phi^i, powers by repeated
 * products (phi^nu by the C library's pow).  The terms with a >= 1 are taken as zero where
 * phi <= 0: the paper's class (1) has u > 0, and phi^nu -> 0 as phi -> 0+ makes this the
 * continuous extension. */
static double op_eval(const opoly *p, double phi, double nu)
{
    double s = 0.0, wa = 1.0;
    const double w = p->na > 1 ? (phi > 0.0 ? pow(phi, nu) : 0.0) : 1.0;
    for (int a = 0; a < p->na; a++) {
        double pw = 1.0;
        for (int i = 0; i < p->n; i++) {
            s += p->c[a][i] * wa * pw;
            pw *= phi;
        }
        wa *= w;
    }
    return s;
}

/* --------------------------------------------------------------- setup */

/* Step (1): Eq. (taus), the coefficients that the Taylor expansion of the
 * LBGK equation attaches to D^k f (Sec. II B). */
static void oracle_taus(double tau, double tk[7])
{
    double t2 = tau * tau, t3 = t2 * tau, t4 = t3 * tau, t5 = t4 * tau;
    tk[0] = 0.0;
    tk[1] = 1.0;
    tk[2] = -tau + 0.5;
    tk[3] = t2 - tau + 1.0 / 6.0;
    tk[4] = -t3 + 1.5 * t2 - 7.0 / 12.0 * tau + 1.0 / 24.0;
    tk[5] = t4 - 2.0 * t3 + 1.25 * t2 - 0.25 * tau + 1.0 / 120.0;
    tk[6] = -t5 + 2.5 * t4 - 13.0 / 6.0 * t3 + 0.75 * t2 - 31.0 / 360.0 * tau + 1.0 / 720.0;
}

/* Return codes shared with the Python wrapper. */
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_TAU_SINGULAR = 2, OR_ERR_DEGREE = 3 };
#define ORACLE_NO_AUX_CORRECTION 0x100

static int singular(double x) { return fabs(x) < 1e-13; }

/*
 * Build the model.  pi_coef is [m][ncoef] row-major: Pi_k(phi) =
 * sum_p pi_coef[(k-1)*ncoef + p] phi^p + sum_p pi_coef_nu[(k-1)*ncoef + p] phi^(p + nu).
 * pi_coef_nu may be NULL (nu unused); otherwise nu > 0 and pi_coef_nu[.. + 0] = 0, so that
 * every Pi_k' is again of the same form.  lattice: 0 = auto (5 for m <= 4, else 7).
 */
int oracle_model_init_nu(oracle_model *M, int m, const double *alpha, const double *pi_coef,
                         const double *pi_coef_nu, int ncoef, double nu_exp, double dx, double dt, double tau,
                         int lattice, int scheme)
{
    memset(M, 0, sizeof(*M));
    if (m < 1 || m > 6 || ncoef < 1 || ncoef > 16) return OR_ERR_ARG;
    if (pi_coef_nu) {
        if (!(nu_exp > 0.0) || !isfinite(nu_exp)) return OR_ERR_ARG;
        for (int k = 0; k < m; k++)
            if (pi_coef_nu[k * ncoef] != 0.0) return OR_ERR_ARG;
        M->nu = nu_exp;
    }
    if (!(dx > 0.0) || !(dt > 0.0) || !(tau > 0.0) || !isfinite(dx) || !isfinite(dt) ||
        !isfinite(tau))
        return OR_ERR_ARG;
    const int no_aux = (scheme & ORACLE_NO_AUX_CORRECTION) != 0;
    scheme &= ~ORACLE_NO_AUX_CORRECTION;
    if (lattice == 0) lattice = (m <= 4) ? 5 : 7;
    if (lattice != 5 && lattice != 7) return OR_ERR_ARG;
    if (m > lattice - 1) return OR_ERR_ARG;          /* Sec. III: b >= m + 1 */
    if (scheme != 1 && scheme != 2) return OR_ERR_ARG;
    if (scheme == 2 && m >= lattice - 1) return OR_ERR_ARG; /* top moment needed */
    M->b = lattice;
    M->m = m;
    M->scheme = scheme;
    M->dx = dx;
    M->dt = dt;
    M->c = dx / dt;
    M->tau = tau;

    for (int k = 1; k <= m; k++) {
        M->alpha[k] = alpha[k - 1];
        op_zero(&M->Pi[k]);
        M->Pi[k].n = ncoef;
        M->Pi[k].na = pi_coef_nu ? 2 : 1;
        for (int p = 0; p < ncoef; p++) {
            M->Pi[k].c[0][p] = pi_coef[(k - 1) * ncoef + p];
            if (pi_coef_nu) M->Pi[k].c[1][p] = pi_coef_nu[(k - 1) * ncoef + p];
        }
    }
    /* alpha_1 is 1 in Eq. (NPDE); any other value is folded into Pi_1. */
    for (int a = 0; a < M->Pi[1].na; a++)
        for (int p = 0; p < ncoef; p++) M->Pi[1].c[a][p] *= M->alpha[1];
    M->alpha[1] = 1.0;
    for (int k = m + 1; k <= 6; k++) op_zero(&M->Pi[k]);

    /* (1) */
    oracle_taus(tau, M->tk);

    /* (2) alpha_k = dt^{k-1} tau_k beta_k, Eqs. (NPDE3)-(NPDE6); beta_k = 0 when
     * the term is absent (Remark 2). */
    for (int k = 2; k <= 6; k++) {
        M->beta[k] = 0.0;
        if (k > m) continue;
        if (M->alpha[k] == 0.0 || op_is_zero(&M->Pi[k])) continue;
        if (singular(M->tk[k])) return OR_ERR_TAU_SINGULAR;
        M->beta[k] = M->alpha[k] / (pow(dt, (double)(k - 1)) * M->tk[k]);
    }
    double t2 = M->tk[2], t3 = M->tk[3], t4 = M->tk[4], t5 = M->tk[5], t6 = M->tk[6];
    double b2 = M->beta[2], b3 = M->beta[3], b4 = M->beta[4];

    /* (3) The A_k0 corrections, Eqs. (Pi4), (Pi5), (Pi6) and (A40)-(A60).  A moment
     * that the lattice does not carry needs no correction; ORACLE_NO_AUX_CORRECTION leaves
     * all three out (and recovery is then inexact wherever one is needed). */
    const int need4 = M->b - 1 >= 4 && b2 != 0.0;
    const int need5 = M->b - 1 >= 5 && b2 != 0.0 && b3 != 0.0;
    const int need6 = M->b - 1 >= 6 && (b2 != 0.0 || b3 != 0.0);
    M->A40 = M->A50 = M->A60 = 0.0;
    if (need4 && !no_aux) {
        if (singular(t4)) return OR_ERR_TAU_SINGULAR;
        M->A40 = t2 * (3.0 * t3 - t2 * t2) * b2 * b2 / t4;
    }
    if (need5 && !no_aux) {
        if (singular(t5)) return OR_ERR_TAU_SINGULAR;
        M->A50 = (4.0 * t2 * t4 + 3.0 * t3 * t3 - 2.0 * t2 * t2 * t3) * b2 * b3 / t5;
    }
    if (need6 && !no_aux) {
        if (singular(t6)) return OR_ERR_TAU_SINGULAR;
        M->A60 = ((5.0 * t2 * t5 + 3.0 * t3 * t4 - 2.0 * t2 * t2 * t4) * b2 * b4 +
                  (4.0 * t4 - t2 * t3) * t3 * b3 * b3 + (t2 * t3 - 6.0 * t4) * t2 * t2 * b2 * b2 * b2) /
                 t6;
    }
    if (no_aux && (need4 || need5 || need6)) M->inexact = 1;

    /* Preconditions of exact recovery, for the terms that are present: Pi_2 = phi for
     * A_40 (Sec. II D), Pi_2 = Pi_3 = phi for A_50 (Sec. II E), Pi_2 = Pi_3 = Pi_4 = phi
     * for A_60 (Sec. II F), and alpha_2 = 0 on D1Q7 (Remark 5). */
    {
        opoly phi1;
        op_zero(&phi1);
        phi1.n = 2;
        phi1.na = 1;
        phi1.c[0][1] = 1.0;
        int is_phi[7] = {0};
        for (int k = 2; k <= 6; k++) {
            opoly d = M->Pi[k];
            op_axpy(&d, -1.0, &phi1);
            is_phi[k] = op_is_zero(&d);
        }
        if (M->b - 1 >= 4 && b2 != 0.0 && !is_phi[2]) M->inexact = 1;
        if (M->b - 1 >= 5 && b2 != 0.0 && b3 != 0.0 && !(is_phi[2] && is_phi[3])) M->inexact = 1;
        if (M->b - 1 >= 6) {
            if (b3 != 0.0 && !is_phi[3]) M->inexact = 1;
            if (b2 != 0.0 && b4 != 0.0 && !(is_phi[2] && is_phi[4])) M->inexact = 1;
        }
        if (M->b == 7 && b2 != 0.0) M->inexact = 1; /* Remark 5 */
    }

    /* (4) Auxiliary moments, each written as the paper prints its integrand. */
    opoly d1, d2, d3, d4, d5; /* Pi_k' */
    const double nu = M->nu;
    if (op_deriv(&d1, &M->Pi[1], nu) || op_deriv(&d2, &M->Pi[2], nu) || op_deriv(&d3, &M->Pi[3], nu) ||
        op_deriv(&d4, &M->Pi[4], nu) || op_deriv(&d5, &M->Pi[5], nu))
        return OR_ERR_ARG;
    opoly p1[7]; /* (Pi_1')^k */
    for (int k = 0; k <= 6; k++)
        if (op_pow(&p1[k], &d1, k)) return OR_ERR_DEGREE;
    opoly one;
    op_zero(&one);
    one.n = 1;
    one.na = 1;
    one.c[0][0] = 1.0;
    opoly g, t;
    for (int k = 2; k <= 6; k++) op_zero(&M->Pi0[k]);

    /* Pi_20 = int (Pi_1')^2 dphi                                      Sec. II C */
    g = p1[2];
    if (op_integ(&M->Pi0[2], &g, nu)) return OR_ERR_DEGREE;

    /* Pi_30 = int [ (Pi_1')^3 + 3 beta_2 Pi_2' Pi_1' ] dphi              Sec. II C */
    g = p1[3];
    if (op_mul(&t, &d2, &p1[1]) || op_axpy(&g, 3.0 * b2, &t)) return OR_ERR_DEGREE;
    if (op_integ(&M->Pi0[3], &g, nu)) return OR_ERR_DEGREE;

    /* Pi_40 = int [ (Pi_1')^4 + 6 beta_2 Pi_2' (Pi_1')^2
     *             + 4 beta_3 Pi_3' Pi_1' + A_40 ] dphi                   Eq. (Pi4) */
    g = p1[4];
    if (op_mul(&t, &d2, &p1[2]) || op_axpy(&g, 6.0 * b2, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d3, &p1[1]) || op_axpy(&g, 4.0 * b3, &t)) return OR_ERR_DEGREE;
    op_axpy(&g, M->A40, &one);
    if (op_integ(&M->Pi0[4], &g, nu)) return OR_ERR_DEGREE;

    /* Pi_50 = int [ (Pi_1')^5 + 10 beta_2 Pi_2' (Pi_1')^3 + 10 beta_3 Pi_3' (Pi_1')^2
     *             + 5 beta_4 Pi_4' Pi_1' + A_50 ] dphi                   Eq. (Pi5) */
    g = p1[5];
    if (op_mul(&t, &d2, &p1[3]) || op_axpy(&g, 10.0 * b2, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d3, &p1[2]) || op_axpy(&g, 10.0 * b3, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d4, &p1[1]) || op_axpy(&g, 5.0 * b4, &t)) return OR_ERR_DEGREE;
    op_axpy(&g, M->A50, &one);
    if (op_integ(&M->Pi0[5], &g, nu)) return OR_ERR_DEGREE;

    /* Pi_60 = int [ (Pi_1')^6 + 15 beta_2 Pi_2' (Pi_1')^4 + 20 beta_3 Pi_3' (Pi_1')^3
     *             + 15 beta_4 Pi_4' (Pi_1')^2 + 6 beta_5 Pi_5' Pi_1' + A_60 ] dphi
     *                                                                    Eq. (Pi6) */
    g = p1[6];
    if (op_mul(&t, &d2, &p1[4]) || op_axpy(&g, 15.0 * b2, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d3, &p1[3]) || op_axpy(&g, 20.0 * b3, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d4, &p1[2]) || op_axpy(&g, 15.0 * b4, &t)) return OR_ERR_DEGREE;
    if (op_mul(&t, &d5, &p1[1]) || op_axpy(&g, 6.0 * M->beta[5], &t)) return OR_ERR_DEGREE;
    op_axpy(&g, M->A60, &one);
    if (op_integ(&M->Pi0[6], &g, nu)) return OR_ERR_DEGREE;

    return OR_OK;
}

/* The model of an equation whose Pi_k are ordinary polynomials. */
int oracle_model_init(oracle_model *M, int m, const double *alpha, const double *pi_coef,
                      int ncoef, double dx, double dt, double tau, int lattice, int scheme)
{
    return oracle_model_init_nu(M, m, alpha, pi_coef, NULL, ncoef, 0.0, dx, dt, tau, lattice, scheme);
}

/* (5) The scaled moments of Sec. III A (D1Q5) and III B (D1Q7):
 *   Pibar_0 = phi, Pibar_1 = Pi_1 / c, Pibar_k = (Pi_k0 + beta_k Pi_k) / c^k. */
void oracle_moments(const oracle_model *M, double phi, double *pibar)
{
    pibar[0] = phi;
    pibar[1] = op_eval(&M->Pi[1], phi, M->nu) / M->c;
    for (int k = 2; k < M->b; k++) {
        double ck = pow(M->c, (double)k);
        pibar[k] = (op_eval(&M->Pi0[k], phi, M->nu) + M->beta[k] * op_eval(&M->Pi[k], phi, M->nu)) / ck;
    }
    if (M->scheme == 2) pibar[M->b - 1] = 0.0;
}

/* (6) The EDFs, Eq. (EDF5) with e = {0, 1, -1, 2, -2} and Eq. (EDF7) with
 * e = {0, 1, -1, 2, -2, 3, -3}, from the scaled moments. */
void oracle_edf(int b, const double *P, double *feq)
{
    if (b == 5) {
        feq[0] = (4.0 * P[0] - 5.0 * P[2] + P[4]) / 4.0;
        feq[1] = (4.0 * (P[1] + P[2]) - P[3] - P[4]) / 6.0;
        feq[2] = (4.0 * (-P[1] + P[2]) + P[3] - P[4]) / 6.0;
        feq[3] = (-2.0 * (P[1] - P[3]) - P[2] + P[4]) / 24.0;
        feq[4] = (2.0 * (P[1] - P[3]) - P[2] + P[4]) / 24.0;
    } else {
        feq[0] = (36.0 * P[0] - 49.0 * P[2] + 14.0 * P[4] - P[6]) / 36.0;
        feq[1] = (36.0 * (P[1] + P[2]) - 13.0 * (P[3] + P[4]) + P[5] + P[6]) / 48.0;
        feq[2] = (36.0 * (-P[1] + P[2]) + 13.0 * (P[3] - P[4]) - P[5] + P[6]) / 48.0;
        feq[3] = (-18.0 * P[1] - 9.0 * P[2] + 20.0 * P[3] + 10.0 * P[4] - 2.0 * P[5] - P[6]) / 120.0;
        feq[4] = (18.0 * P[1] - 9.0 * P[2] - 20.0 * P[3] + 10.0 * P[4] + 2.0 * P[5] - P[6]) / 120.0;
        feq[5] = (12.0 * P[1] + 4.0 * P[2] - 15.0 * P[3] - 5.0 * P[4] + 3.0 * P[5] + P[6]) / 720.0;
        feq[6] = (-12.0 * P[1] + 4.0 * P[2] + 15.0 * P[3] - 5.0 * P[4] - 3.0 * P[5] + P[6]) / 720.0;
    }
}

void oracle_feq(const oracle_model *M, double phi, double *feq)
{
    double P[7];
    oracle_moments(M, phi, P);
    oracle_edf(M->b, P, feq);
}

/* d f^eq_j / d phi, from the exact derivatives of the moment polynomials; used by
 * the linear (Fourier) analysis in the tests. */
void oracle_dfeq(const oracle_model *M, double phi, double *dfeq)
{
    double P[7];
    opoly d;
    P[0] = 1.0;
    op_deriv(&d, &M->Pi[1], M->nu);
    P[1] = op_eval(&d, phi, M->nu) / M->c;
    for (int k = 2; k < M->b; k++) {
        opoly s = M->Pi0[k];
        op_axpy(&s, M->beta[k], &M->Pi[k]);
        op_deriv(&d, &s, M->nu);
        P[k] = op_eval(&d, phi, M->nu) / pow(M->c, (double)k);
    }
    if (M->scheme == 2) P[M->b - 1] = 0.0;
    oracle_edf(M->b, P, dfeq);
}

/* The lattice velocities in units of c (Sec. III A, III B). */
static const int E7[7] = {0, 1, -1, 2, -2, 3, -3};

/* (7) initial state: f_j(x, 0) = f^eq_j(phi_0(x)).  f is [b][N] row-major. */
void oracle_init(const oracle_model *M, long N, const double *phi0, double *f)
{
    double feq[7];
    for (long i = 0; i < N; i++) {
        oracle_feq(M, phi0[i], feq);
        for (int j = 0; j < M->b; j++) f[(long)j * N + i] = feq[j];
    }
}

/* Right-hand side of Eq. (LBE) at node i: fstar_j = f_j - (f_j - f^eq_j(phi)) / tau with
 * phi = sum_j f_j (Eq. (moments)). */
static void collide(const oracle_model *M, long N, const double *f, long i, double *fstar)
{
    double feq[7];
    double phi = 0.0;
    for (int j = 0; j < M->b; j++) phi += f[(long)j * N + i];
    oracle_feq(M, phi, feq);
    for (int j = 0; j < M->b; j++) {
        double fj = f[(long)j * N + i];
        fstar[j] = fj - (fj - feq[j]) / M->tau;
    }
}

/* (7) nsteps of Eq. (LBE) on a periodic grid: collide at every node, then move
 * each post-collision f_j to node i + e_j (mod N).  tmp has the size of f. */
void oracle_step(const oracle_model *M, long N, double *f, double *tmp, long nsteps)
{
    const int b = M->b;
    double fstar[7];
    for (long n = 0; n < nsteps; n++) {
        for (long i = 0; i < N; i++) {
            collide(M, N, f, i, fstar);
            for (int j = 0; j < b; j++) {
                long dst = ((i + E7[j]) % N + N) % N;
                tmp[(long)j * N + dst] = fstar[j];
            }
        }
        memcpy(f, tmp, sizeof(double) * (size_t)b * (size_t)N);
    }
}

/* nsteps of Eq. (LBE) on a bounded grid of N nodes with the non-equilibrium extrapolation
 * boundary: collide everywhere, stream (populations leaving the grid are dropped), then rebuild
 * the W = max|e| outer nodes at each end from x_f = W - 1 + depth (left) and N - W - depth
 * (right).  phib holds, for step n (time (n + 1) dt), the prescribed phi at the W left nodes
 * 0..W-1 followed by the W right nodes N-W..N-1.  Needs depth >= 1 and N >= 2 (W + depth). */
void oracle_step_nee(const oracle_model *M, long N, double *f, double *tmp, long nsteps, const double *phib,
                     int depth)
{
    const int b = M->b, W = (b - 1) / 2;
    double fstar[7], fb[7], fk[7];
    for (long n = 0; n < nsteps; n++) {
        for (long q = 0; q < (long)b * N; q++) tmp[q] = 0.0;
        for (long i = 0; i < N; i++) {
            collide(M, N, f, i, fstar);
            for (int j = 0; j < b; j++) {
                long dst = i + E7[j];
                if (dst >= 0 && dst < N) tmp[(long)j * N + dst] = fstar[j];
            }
        }
        memcpy(f, tmp, sizeof(double) * (size_t)b * (size_t)N);
        for (int side = 0; side < 2; side++) {
            long k = side == 0 ? W - 1 + depth : N - W - depth;
            double phik = 0.0;
            for (int j = 0; j < b; j++) phik += f[(long)j * N + k];
            oracle_feq(M, phik, fk);
            for (int l = 0; l < W; l++) {
                long i = side == 0 ? l : N - W + l;
                oracle_feq(M, phib[n * 2 * W + side * W + l], fb);
                for (int j = 0; j < b; j++) f[(long)j * N + i] = fb[j] + f[(long)j * N + k] - fk[j];
            }
        }
    }
}

/* phi(x) = sum_j f_j(x)  (first constraint of Eq. (moments)) */
void oracle_phi(const oracle_model *M, long N, const double *f, double *phi)
{
    for (long i = 0; i < N; i++) {
        double s = 0.0;
        for (int j = 0; j < M->b; j++) s += f[(long)j * N + i];
        phi[i] = s;
    }
}

/* (8) E = sum |phi - phi*| / sum |phi*|  (Sec. IV) */
double oracle_error_E(long N, const double *phi, const double *phistar)
{
    double num = 0.0, den = 0.0;
    for (long i = 0; i < N; i++) {
        num += fabs(phi[i] - phistar[i]);
        den += fabs(phistar[i]);
    }
    return num / den;
}

/* One-call driver: phi0 -> phi after nsteps.  Returns an oracle_model_init code. */
int oracle_run(int m, const double *alpha, const double *pi_coef, int ncoef, double dx, double dt,
               double tau, int lattice, int scheme, long N, const double *phi0, long nsteps,
               double *phi_out)
{
    oracle_model *M = (oracle_model *)malloc(sizeof(oracle_model));
    if (!M) return OR_ERR_ARG;
    int rc = oracle_model_init(M, m, alpha, pi_coef, ncoef, dx, dt, tau, lattice, scheme);
    if (rc != OR_OK) { free(M); return rc; }
    double *f = (double *)malloc(sizeof(double) * (size_t)M->b * (size_t)N);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)M->b * (size_t)N);
    if (!f || !tmp) { free(f); free(tmp); free(M); return OR_ERR_ARG; }
    oracle_init(M, N, phi0, f);
    oracle_step(M, N, f, tmp, nsteps);
    oracle_phi(M, N, f, phi_out);
    free(f);
    free(tmp);
    free(M);
    return OR_OK;
}

/* Accessors for the Python wrapper (the struct layout stays private to C). */
size_t oracle_model_size(void) { return sizeof(oracle_model); }
int oracle_model_b(const oracle_model *M) { return M->b; }
int oracle_model_inexact(const oracle_model *M) { return M->inexact; }
void oracle_model_params(const oracle_model *M, double *tk, double *beta, double *A)
{
    for (int k = 0; k < 7; k++) { tk[k] = M->tk[k]; beta[k] = M->beta[k]; }
    A[0] = M->A40;
    A[1] = M->A50;
    A[2] = M->A60;
}
/* Value of Pi_k0(phi), k = 2..6 (0 for other k). */
double oracle_aux_moment(const oracle_model *M, int k, double phi)
{
    if (k < 2 || k > 6) return 0.0;
    return op_eval(&M->Pi0[k], phi, M->nu);
}
