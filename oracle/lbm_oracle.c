/*
 * Plain FP64 CPU oracle of the reactive-mixture lattice Boltzmann step
 * (Sawant, Dorschner, Karlin, "Reactive mixtures with the lattice Boltzmann
 * model", arXiv 2101.01702).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  It is loaded by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the library itself.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * It is deliberately slow and literal: storage is array-of-structures
 * pop[node][set][direction], every step is three separate passes over the
 * lattice (stream + moments, neighbour gradients, collision), and each
 * formula is written in the order and notation of the paper:
 *
 *   D3Q27 velocities c_i in {-1,0,1}^3 ............ Sec. 2, after Eq. (sumfDotc)
 *   product-form Psi_{-1,0,1}(xi, zeta) ............. Eq. (phis)
 *   species equilibria / quasi-equilibria ........... Eqs. (feq), (fstar)
 *   reaction source populations ..................... Eq. (fsource)
 *   species lattice Boltzmann equation .............. Eq. (finalNumericalEquations)
 *   F_ai, beta_a ..................................... Eq. (fStar)
 *   tau_ab, tau_a .................................... Eq. (tauab)
 *   Stefan-Maxwell diffusion-velocity system ........ Eq. (transform1)
 *   U_a, H_a with formation energies ................ Eqs. (specHa), (Umix)
 *   temperature from energy .......................... Eq. (temperature)
 *   mixture f and energy g lattice Boltzmann ......... Eqs. (f), (g)
 *   mixture equilibrium .............................. Eq. (feqmix)
 *   isotropy correction X, A_i ....................... Eqs. (Xalpha), (Ai)
 *   Grad equilibria g^eq, g^* ........................ Eqs. (gieq), (giqeq)
 *   q^eq, R^eq ....................................... Eqs. (geq1mom), (geq2mom)
 *   q^*, q^diff, q^corr .............................. Eqs. (gstareq1mom), (qdiff), (corrFourier)
 *   omega from viscosity, omega_1 from conductivity . Eqs. (mu), (lambda)
 *   slaving of the last species ...................... Eq. (strongest)
 *   heat release rate hdot^c ......................... Sec. 5b (circular flame)
 *
 * Readings where the paper is silent:
 *   - lattice gradients: d_alpha phi(x) = (1/theta) sum_i w_i c_ia phi(x+c_i),
 *     theta = 1/3, applied twice for X (inner derivative, multiply by
 *     (1/omega - 1/2), outer derivative);
 *   - the neighbour fields are those of the same time level (post-stream,
 *     pre-collision moments);
 *   - viscosity either from a constant kinematic viscosity (mu = rho nu, so
 *     1/omega = 1/2 + nu/(R T)) or a constant relaxation (1/omega - 1/2 =
 *     nu); conductivity from a constant Prandtl number, 1/omega_1 - 1/2 =
 *     (1/omega - 1/2)/Pr; or mixture-averaged transport (mixture_transport:
 *     seeded species power laws with the Wilke and Mathur mixing rules);
 *   - chemistry is a mass-action Arrhenius mechanism (third-body and
 *     Lindemann falloff forms, reverse rates from equilibrium constants of
 *     the species Gibbs energies) evaluated with concentrations rho_a/W_a;
 *   - x-faces with bc_x = 1: ghost nodes hold the equilibria of every set at
 *     the post-collision moments of the adjacent boundary node, with zero
 *     velocity on the left ghost (Sec. 5a); macroscopic fields used by the
 *     gradient stencils are continued by zero gradient (nearest interior
 *     node).
 *
 * Direction order: i = (cx+1) + 3*(cy+1) + 9*(cz+1).
 * Set order: species 0..M-2, then the mixture set f, then the energy set g.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 27
#define ORC_MAXM 16
#define ORC_MAXR 64

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NEWTON = -3, ORC_ERR_NONFINITE = -4,
       ORC_ERR_NEGATIVE = -5, ORC_ERR_PIVOT = -6 };
enum { ORC_THERMO_CONST_CP = 0, ORC_THERMO_POLY7 = 1 };
enum { ORC_RXN_ELEMENTARY = 0, ORC_RXN_THIRD_BODY = 1, ORC_RXN_FALLOFF = 2 };

typedef struct {
    int nx, ny, nz, bc_x;
    int M;
    const double *W;        /* [M] */
    int thermo;
    const double *cp_R;     /* [M] */
    const double *h_form;   /* [M] */
    double T0;
    const double *poly7;    /* [M][7] */
    const double *D;        /* [M][M] */
    double nu, Pr, r_lat;
    int visc_model;         /* 0: kinematic viscosity nu; 1: nu = 1/omega - 1/2 */
    int R;
    const int *nu_f, *nu_r; /* [R][M] */
    const double *log_A, *b, *theta; /* [R] */
    const int *rtype;       /* [R] */
    const double *eff;      /* [R][M] */
    const double *low;      /* [R][3] */
    const int *reversible;  /* [R] */
    double T_ref, P0;
    int transport;          /* 0: constant nu, Pr, D_ab; 1: mixture-averaged (below) */
    const double *mu0;      /* [M] species viscosity at T_tr (transport = 1) */
    const double *mu_exp;   /* [M] its temperature exponent */
    double T_tr, D_exp, P_tr;
} orc_params;

typedef struct {
    /* copied parameters */
    int nx, ny, nz, bc_x, N, M, S;
    double W[ORC_MAXM];
    int thermo;
    double cp_R[ORC_MAXM], h_form[ORC_MAXM], T0, poly7[ORC_MAXM][7], D[ORC_MAXM][ORC_MAXM];
    double nu, Pr, r_lat;
    int visc_model;
    int R;
    int nu_f[ORC_MAXR][ORC_MAXM], nu_r[ORC_MAXR][ORC_MAXM];
    double log_A[ORC_MAXR], b[ORC_MAXR], theta[ORC_MAXR];
    int rtype[ORC_MAXR];
    double eff[ORC_MAXR][ORC_MAXM], low[ORC_MAXR][3];
    int reversible[ORC_MAXR];
    double T_ref, P0;
    int transport;
    double mu0[ORC_MAXM], mu_exp[ORC_MAXM], T_tr, D_exp, P_tr;
    /* state */
    double *pop;    /* [N][S][27] post-collision populations, stored at their node */
    double *tmp;    /* [N][S][27] populations after the pull */
    double *Tn;     /* [N] temperature of the last step (Newton starting point) */
    double *ghost;  /* [2][ny*nz][S][27] ghost-node populations (bc_x = 1) */
    /* per-node fields of the current step */
    double *rho_a;  /* [N][M] */
    double *j_a;    /* [N][M][3] */
    double *rho, *j, *rhoE, *q, *Pt; /* [N], [N][3], [N], [N][3], [N][3][3] */
    double *T, *Y, *Phi, *nup, *G, *gradY; /* [N],[N][M],[N][3],[N],[N][3],[N][M][3] */
    int status;
} orc_state;

/* ------------------------------------------------------------------ */
/* Lattice                                                            */
/* ------------------------------------------------------------------ */
static int cx_of(int i) { return i % 3 - 1; }
static int cy_of(int i) { return (i / 3) % 3 - 1; }
static int cz_of(int i) { return i / 9 - 1; }

/* One-dimensional weights w_0 = 1 - theta, w_{+-1} = theta/2, theta = 1/3;
 * w_i is their product over the three axes (Sec. 3, after Eq. (giqeq)). */
static const double THETA = 1.0 / 3.0;
static double w1(int c) { return c == 0 ? 1.0 - THETA : THETA / 2.0; }
static double w_of(int i) { return w1(cx_of(i)) * w1(cy_of(i)) * w1(cz_of(i)); }

/* Eq. (phis). */
static double Psi(int c, double xi, double zeta)
{
    if (c == 0) return 1.0 - (xi * xi + zeta);
    if (c == 1) return (xi + (xi * xi + zeta)) / 2.0;
    return (-xi + (xi * xi + zeta)) / 2.0;
}

/* rho * Psi_cx(v_x) Psi_cy(v_y) Psi_cz(v_z), Eqs. (feq), (fstar), (fsource), (feqmix). */
static double product_form(int i, double rho, const double v[3], double zeta)
{
    return rho * Psi(cx_of(i), v[0], zeta) * Psi(cy_of(i), v[1], zeta) * Psi(cz_of(i), v[2], zeta);
}

void orc_product_form(double rho, const double *v, double zeta, double *out27)
{
    for (int i = 0; i < ORC_Q; ++i) out27[i] = product_form(i, rho, v, zeta);
}

/* Grad's approximation, Eqs. (gieq)/(giqeq): the energy populations with
 * zeroth moment rhoE, first moment qv and second moment Rt. */
static double grad_pop(int i, double rhoE, const double qv[3], const double Rt[3][3])
{
    int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
    double first = 0.0;
    for (int a = 0; a < 3; ++a) first += qv[a] * c[a];
    double second = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double d = (a == b) ? 1.0 : 0.0;
            second += (Rt[a][b] - rhoE * THETA * d) * (c[a] * c[b] - THETA * d);
        }
    return w_of(i) * (rhoE + first / THETA + second / (2.0 * THETA * THETA));
}

void orc_grad_pop(double rhoE, const double *qv, const double *Rt9, double *out27)
{
    double Rt[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Rt[a][b] = Rt9[3 * a + b];
    for (int i = 0; i < ORC_Q; ++i) out27[i] = grad_pop(i, rhoE, qv, Rt);
}

/* ------------------------------------------------------------------ */
/* Thermodynamics, Eqs. (specHa), (Umix)                              */
/* ------------------------------------------------------------------ */
static double R_spec(const orc_state *s, int a) { return s->r_lat / s->W[a]; }

/* Specific internal energy U_a(T) including the energy of formation. */
static double U_spec(const orc_state *s, int a, double T)
{
    double Ra = R_spec(s, a);
    if (s->thermo == ORC_THERMO_CONST_CP) {
        double U0 = s->h_form[a] - Ra * s->T0;          /* U^0 = H^0 - R_a T0 */
        return U0 + (s->cp_R[a] - 1.0) * Ra * (T - s->T0);
    }
    const double *p = s->poly7[a];
    double h_RT = p[0] + p[1] * T / 2.0 + p[2] * T * T / 3.0 + p[3] * T * T * T / 4.0
                + p[4] * T * T * T * T / 5.0 + p[5] / T;
    return Ra * T * h_RT - Ra * T;
}

/* Specific enthalpy H_a(T) = U_a(T) + R_a T (ideal gas). */
static double H_spec(const orc_state *s, int a, double T) { return U_spec(s, a, T) + R_spec(s, a) * T; }

/* Specific heat at constant volume C_{a,v}(T). */
static double Cv_spec(const orc_state *s, int a, double T)
{
    double Ra = R_spec(s, a);
    if (s->thermo == ORC_THERMO_CONST_CP) return (s->cp_R[a] - 1.0) * Ra;
    const double *p = s->poly7[a];
    double cp_R = p[0] + p[1] * T + p[2] * T * T + p[3] * T * T * T + p[4] * T * T * T * T;
    return (cp_R - 1.0) * Ra;
}

/* Standard-state Gibbs energy over R_U T, g_a/(R_U T) = h/(R T) - s/R.
 * With constant cp the entropy is referred to s = 0 at T0. */
static double gRT_spec(const orc_state *s, int a, double T)
{
    if (s->thermo == ORC_THERMO_CONST_CP) {
        double h_RT = H_spec(s, a, T) / (R_spec(s, a) * T);
        double s_R = s->cp_R[a] * log(T / s->T0);
        return h_RT - s_R;
    }
    const double *p = s->poly7[a];
    double h_RT = p[0] + p[1] * T / 2.0 + p[2] * T * T / 3.0 + p[3] * T * T * T / 4.0
                + p[4] * T * T * T * T / 5.0 + p[5] / T;
    double s_R = p[0] * log(T) + p[1] * T + p[2] * T * T / 2.0 + p[3] * T * T * T / 3.0
               + p[4] * T * T * T * T / 4.0 + p[6];
    return h_RT - s_R;
}

/* Eq. (temperature): solve sum_a Y_a U_a(T) = e by Newton's method with
 * derivative C_v = sum_a Y_a C_{a,v}.  Stops when |dT| <= 1e-13 T. */
static int solve_temperature(const orc_state *s, const double *Y, double e, double T_guess, double *T_out)
{
    double T = T_guess;
    for (int it = 0; it < 50; ++it) {
        double F = -e, Fp = 0.0;
        for (int a = 0; a < s->M; ++a) {
            F += Y[a] * U_spec(s, a, T);
            Fp += Y[a] * Cv_spec(s, a, T);
        }
        double dT = F / Fp;
        T -= dT;
        if (!isfinite(T)) { *T_out = T; return ORC_ERR_NONFINITE; }
        if (fabs(dT) <= 1e-13 * fabs(T)) { *T_out = T; return ORC_OK; }
    }
    *T_out = T;
    return ORC_ERR_NEWTON;
}

/* ------------------------------------------------------------------ */
/* Chemistry: production rates rho_dot_a with sum_a rho_dot_a = 0,    */
/* Eq. (sumRhoDot).                                                   */
/* ------------------------------------------------------------------ */
static void production_rates(const orc_state *s, const double *rho_a, double T, double *wdot)
{
    int M = s->M;
    double c[ORC_MAXM], gRT[ORC_MAXM];
    for (int a = 0; a < M; ++a) {
        c[a] = rho_a[a] / s->W[a];
        gRT[a] = gRT_spec(s, a, T);
        wdot[a] = 0.0;
    }
    for (int k = 0; k < s->R; ++k) {
        double kf = exp(s->log_A[k] + s->b[k] * log(T / s->T_ref) - s->theta[k] / T);
        double conc_M = 0.0;
        if (s->rtype[k] != ORC_RXN_ELEMENTARY)
            for (int a = 0; a < M; ++a) conc_M += s->eff[k][a] * c[a];
        if (s->rtype[k] == ORC_RXN_FALLOFF) {
            double k0 = exp(s->low[k][0] + s->low[k][1] * log(T / s->T_ref) - s->low[k][2] / T);
            double Pr = k0 * conc_M / kf;
            kf = kf * Pr / (1.0 + Pr);
        }
        double kr = 0.0;
        if (s->reversible[k]) {
            double dG = 0.0, dn = 0.0;
            for (int a = 0; a < M; ++a) {
                int dnu = s->nu_r[k][a] - s->nu_f[k][a];
                dG += dnu * gRT[a];
                dn += dnu;
            }
            double Kc = exp(-dG) * pow(s->P0 / (s->r_lat * T), dn);
            kr = kf / Kc;
        }
        double qf = kf, qr = kr;
        for (int a = 0; a < M; ++a) {
            for (int n = 0; n < s->nu_f[k][a]; ++n) qf *= c[a];
            for (int n = 0; n < s->nu_r[k][a]; ++n) qr *= c[a];
        }
        double qk = qf - qr;
        if (s->rtype[k] == ORC_RXN_THIRD_BODY) qk *= conc_M;
        for (int a = 0; a < M; ++a) wdot[a] += s->W[a] * (s->nu_r[k][a] - s->nu_f[k][a]) * qk;
    }
}

/* ------------------------------------------------------------------ */
/* Stefan-Maxwell system, Eq. (transform1), by Gaussian elimination   */
/* with partial pivoting; three right-hand sides.                      */
/* ------------------------------------------------------------------ */
static int solve_linear(int M, double A[ORC_MAXM][ORC_MAXM], double rhs[ORC_MAXM][3], double x[ORC_MAXM][3])
{
    for (int k = 0; k < M; ++k) {
        int p = k;
        for (int r = k + 1; r < M; ++r)
            if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
        if (A[p][k] == 0.0) return ORC_ERR_PIVOT;
        if (p != k) {
            for (int cc = 0; cc < M; ++cc) { double t = A[k][cc]; A[k][cc] = A[p][cc]; A[p][cc] = t; }
            for (int d = 0; d < 3; ++d) { double t = rhs[k][d]; rhs[k][d] = rhs[p][d]; rhs[p][d] = t; }
        }
        for (int r = k + 1; r < M; ++r) {
            double l = A[r][k] / A[k][k];
            for (int cc = k; cc < M; ++cc) A[r][cc] -= l * A[k][cc];
            for (int d = 0; d < 3; ++d) rhs[r][d] -= l * rhs[k][d];
        }
    }
    for (int r = M - 1; r >= 0; --r)
        for (int d = 0; d < 3; ++d) {
            double acc = rhs[r][d];
            for (int cc = r + 1; cc < M; ++cc) acc -= A[r][cc] * x[cc][d];
            x[r][d] = acc / A[r][r];
        }
    return ORC_OK;
}

/* 1/omega - 1/2 from Eq. (mu), mu = (1/omega - 1/2) P dt: with a constant
 * kinematic viscosity mu = rho nu gives nu / (R T); the constant-relaxation
 * model takes nu itself. */
static double nu_prime(const orc_state *s, double Rmix, double T)
{
    return s->visc_model == 0 ? s->nu / (Rmix * T) : s->nu;
}

/* 1/tau_ab = m R_U T / (m_a m_b D_ab), Eq. (tauab); dfac scales every
 * binary diffusivity (1 for constant transport). */
static double inv_tau_ab(const orc_state *s, int a, int b, double m, double T)
{
    return m * s->r_lat * T / (s->W[a] * s->W[b] * s->D[a][b]);
}

/* Mixture-averaged transport, the stand-in for the coefficients the paper
 * takes from Cantera (Sec. 3, after Eq. (lambda)): species viscosities
 * mu_a = mu0_a (T/T_tr)^{s_a}; Wilke's mixing rule (Wilke 1950)
 *   mu = sum_a X_a mu_a / sum_b X_b Phi_ab,
 *   Phi_ab = [1 + (mu_a/mu_b)^{1/2} (W_b/W_a)^{1/4}]^2 / [8 (1 + W_a/W_b)]^{1/2};
 * species conductivities by the modified Eucken relation
 * lambda_a = mu_a (C_p,a + 5/4 R_a); the average of Mathur, Tondon and
 * Saxena (1967) lambda = (sum_a X_a lambda_a + 1 / sum_a X_a / lambda_a) / 2;
 * binary diffusivities D_ab (T/T_tr)^{D_exp} (P_tr/P), so every 1/tau_ab
 * is divided by dfac = (T/T_tr)^{D_exp} P_tr / P. */
static void mixture_transport(const orc_state *s, const double *Y, double T, double P, double *mu, double *lambda,
                              double *dfac)
{
    int M = s->M;
    double X[ORC_MAXM], mua[ORC_MAXM], inv_m = 0.0;
    for (int a = 0; a < M; ++a) inv_m += Y[a] / s->W[a];
    for (int a = 0; a < M; ++a) {
        X[a] = Y[a] / s->W[a] / inv_m;
        mua[a] = s->mu0[a] * pow(T / s->T_tr, s->mu_exp[a]);
    }
    double num = 0.0, lsum = 0.0, lrec = 0.0;
    for (int a = 0; a < M; ++a) {
        double den = 0.0;
        for (int b = 0; b < M; ++b) {
            double r = 1.0 + sqrt(mua[a] / mua[b]) * pow(s->W[b] / s->W[a], 0.25);
            den += X[b] * r * r / sqrt(8.0 * (1.0 + s->W[a] / s->W[b]));
        }
        num += X[a] * mua[a] / den;
        double Ra = R_spec(s, a);
        double lam_a = mua[a] * (Cv_spec(s, a, T) + Ra + 1.25 * Ra);
        lsum += X[a] * lam_a;
        lrec += X[a] / lam_a;
    }
    *mu = num;
    *lambda = 0.5 * (lsum + 1.0 / lrec);
    *dfac = pow(T / s->T_tr, s->D_exp) * s->P_tr / P;
}

/* Relaxation parameters: nup = 1/omega - 1/2 from Eq. (mu), mu = nup P dt;
 * nup1 = 1/omega_1 - 1/2 from Eq. (lambda), lambda = nup1 P C_p dt; and the
 * diffusivity factor dfac.  Constant transport: nup from nu_prime,
 * nup1 = nup / Pr, dfac = 1. */
static void relaxation(const orc_state *s, const double *Y, double Rmix, double T, double P, double *nup,
                       double *nup1, double *dfac)
{
    if (!s->transport) {
        *nup = nu_prime(s, Rmix, T);
        *nup1 = *nup / s->Pr;
        *dfac = 1.0;
        return;
    }
    double mu, lambda, Cv = 0.0;
    for (int a = 0; a < s->M; ++a) Cv += Y[a] * Cv_spec(s, a, T);
    mixture_transport(s, Y, T, P, &mu, &lambda, dfac);
    *nup = mu / P;
    *nup1 = lambda / (P * (Cv + Rmix));
}

/* ------------------------------------------------------------------ */
/* Creation                                                           */
/* ------------------------------------------------------------------ */
void orc_destroy(orc_state *s);

orc_state *orc_create(const orc_params *p)
{
    if (!p || p->M < 2 || p->M > ORC_MAXM || p->R < 0 || p->R > ORC_MAXR) return NULL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->nx = p->nx; s->ny = p->ny; s->nz = p->nz; s->bc_x = p->bc_x;
    s->N = p->nx * p->ny * p->nz;
    s->M = p->M; s->S = p->M + 1;
    for (int a = 0; a < p->M; ++a) {
        s->W[a] = p->W[a];
        s->cp_R[a] = p->cp_R ? p->cp_R[a] : 0.0;
        s->h_form[a] = p->h_form ? p->h_form[a] : 0.0;
        for (int k = 0; k < 7; ++k) s->poly7[a][k] = p->poly7 ? p->poly7[7 * a + k] : 0.0;
        for (int b = 0; b < p->M; ++b) s->D[a][b] = p->D[p->M * a + b];
    }
    s->thermo = p->thermo; s->T0 = p->T0;
    s->nu = p->nu; s->Pr = p->Pr; s->r_lat = p->r_lat; s->visc_model = p->visc_model;
    s->R = p->R;
    for (int k = 0; k < p->R; ++k) {
        for (int a = 0; a < p->M; ++a) {
            s->nu_f[k][a] = p->nu_f[p->M * k + a];
            s->nu_r[k][a] = p->nu_r[p->M * k + a];
            s->eff[k][a] = p->eff[p->M * k + a];
        }
        s->log_A[k] = p->log_A[k]; s->b[k] = p->b[k]; s->theta[k] = p->theta[k];
        s->rtype[k] = p->rtype[k]; s->reversible[k] = p->reversible[k];
        for (int d = 0; d < 3; ++d) s->low[k][d] = p->low[3 * k + d];
    }
    s->T_ref = p->T_ref; s->P0 = p->P0;
    s->transport = p->transport;
    if (s->transport && (!p->mu0 || !p->mu_exp || !(p->T_tr > 0.0) || !(p->P_tr > 0.0))) return (free(s), NULL);
    for (int a = 0; a < p->M; ++a) {
        s->mu0[a] = p->mu0 ? p->mu0[a] : 0.0;
        s->mu_exp[a] = p->mu_exp ? p->mu_exp[a] : 0.0;
    }
    s->T_tr = p->T_tr; s->D_exp = p->D_exp; s->P_tr = p->P_tr;
    size_t N = (size_t)s->N, S = (size_t)s->S, M = (size_t)s->M;
    s->pop = (double *)calloc(N * S * ORC_Q, sizeof(double));
    s->tmp = (double *)calloc(N * S * ORC_Q, sizeof(double));
    s->Tn = (double *)calloc(N, sizeof(double));
    s->ghost = (double *)calloc(2 * (size_t)s->ny * s->nz * S * ORC_Q, sizeof(double));
    s->rho_a = (double *)calloc(N * M, sizeof(double));
    s->j_a = (double *)calloc(N * M * 3, sizeof(double));
    s->rho = (double *)calloc(N, sizeof(double));
    s->j = (double *)calloc(N * 3, sizeof(double));
    s->rhoE = (double *)calloc(N, sizeof(double));
    s->q = (double *)calloc(N * 3, sizeof(double));
    s->Pt = (double *)calloc(N * 9, sizeof(double));
    s->T = (double *)calloc(N, sizeof(double));
    s->Y = (double *)calloc(N * M, sizeof(double));
    s->Phi = (double *)calloc(N * 3, sizeof(double));
    s->nup = (double *)calloc(N, sizeof(double));
    s->G = (double *)calloc(N * 3, sizeof(double));
    s->gradY = (double *)calloc(N * M * 3, sizeof(double));
    if (!s->pop || !s->tmp || !s->Tn || !s->ghost || !s->rho_a || !s->j_a || !s->rho || !s->j ||
        !s->rhoE || !s->q || !s->Pt || !s->T || !s->Y || !s->Phi || !s->nup || !s->G || !s->gradY) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->pop); free(s->tmp); free(s->Tn); free(s->ghost); free(s->rho_a); free(s->j_a);
    free(s->rho); free(s->j); free(s->rhoE); free(s->q); free(s->Pt); free(s->T); free(s->Y);
    free(s->Phi); free(s->nup); free(s->G); free(s->gradY);
    free(s);
}

static size_t node_index(const orc_state *s, int x, int y, int z)
{
    return (size_t)x + (size_t)s->nx * ((size_t)y + (size_t)s->ny * (size_t)z);
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* ------------------------------------------------------------------ */
/* Equilibrium populations of every set at a macroscopic state.       */
/* Species a < M-1: Eq. (feq); mixture: Eq. (feqmix); energy: Grad     */
/* equilibrium Eq. (gieq) with q^eq, R^eq of Eqs. (geq1mom), (geq2mom). */
/* ------------------------------------------------------------------ */
static void equilibrium_sets(const orc_state *s, const double *rho_a, const double u[3], double T, double *out)
{
    int M = s->M;
    double rho = 0.0;
    for (int a = 0; a < M; ++a) rho += rho_a[a];
    double Y[ORC_MAXM], inv_m = 0.0;
    for (int a = 0; a < M; ++a) { Y[a] = rho_a[a] / rho; inv_m += Y[a] / s->W[a]; }
    double Rmix = s->r_lat * inv_m;
    for (int a = 0; a < M - 1; ++a)
        for (int i = 0; i < ORC_Q; ++i)
            out[a * ORC_Q + i] = product_form(i, rho_a[a], u, R_spec(s, a) * T);
    for (int i = 0; i < ORC_Q; ++i)
        out[(M - 1) * ORC_Q + i] = product_form(i, rho, u, Rmix * T);
    double Umix = 0.0, Hmix = 0.0;
    for (int a = 0; a < M; ++a) { Umix += Y[a] * U_spec(s, a, T); Hmix += Y[a] * H_spec(s, a, T); }
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double rhoE = rho * (Umix + usq / 2.0);
    double P = rho * Rmix * T;
    double qeq[3], Req[3][3];
    for (int a = 0; a < 3; ++a) qeq[a] = (Hmix + usq / 2.0) * rho * u[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double Peq = (a == b ? P : 0.0) + rho * u[a] * u[b];
            Req[a][b] = (Hmix + usq / 2.0) * Peq + P * u[a] * u[b];
        }
    for (int i = 0; i < ORC_Q; ++i) out[M * ORC_Q + i] = grad_pop(i, rhoE, qeq, Req);
}

/* Initialisation: every set at its equilibrium for the given mole
 * fractions X[M][N], temperature T[N], velocity u[3][N] (or NULL) and
 * uniform pressure P (rho = P / (R T), Eq. (eosIdealGas)). */
int orc_init(orc_state *s, const double *X, const double *T, const double *u, double P)
{
    int M = s->M, S = s->S;
    for (int n = 0; n < s->N; ++n) {
        double m = 0.0;
        for (int a = 0; a < M; ++a) m += X[(size_t)a * s->N + n] * s->W[a];
        double Rmix = s->r_lat / m;
        double rho = P / (Rmix * T[n]);
        double rho_a[ORC_MAXM];
        for (int a = 0; a < M; ++a) rho_a[a] = rho * X[(size_t)a * s->N + n] * s->W[a] / m;
        double v[3] = {0.0, 0.0, 0.0};
        if (u) for (int d = 0; d < 3; ++d) v[d] = u[(size_t)d * s->N + n];
        equilibrium_sets(s, rho_a, v, T[n], s->pop + (size_t)n * S * ORC_Q);
        s->Tn[n] = T[n];
    }
    s->status = ORC_OK;
    return ORC_OK;
}

/* Post-collision moments of a stored node: species densities (slaved last
 * species included), velocity and temperature. */
static int stored_node_state(const orc_state *s, size_t n, double *rho_a, double u[3], double *T)
{
    int M = s->M;
    const double *p = s->pop + n * s->S * ORC_Q;
    double rho = 0.0, j[3] = {0, 0, 0}, rhoE = 0.0;
    double rest = 0.0;
    for (int a = 0; a < M - 1; ++a) {
        rho_a[a] = 0.0;
        for (int i = 0; i < ORC_Q; ++i) rho_a[a] += p[a * ORC_Q + i];
        rest += rho_a[a];
    }
    for (int i = 0; i < ORC_Q; ++i) {
        double f = p[(M - 1) * ORC_Q + i];
        rho += f;
        j[0] += f * cx_of(i); j[1] += f * cy_of(i); j[2] += f * cz_of(i);
        rhoE += p[M * ORC_Q + i];
    }
    rho_a[M - 1] = rho - rest;
    double Y[ORC_MAXM];
    for (int a = 0; a < M; ++a) Y[a] = rho_a[a] / rho;
    for (int d = 0; d < 3; ++d) u[d] = j[d] / rho;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return solve_temperature(s, Y, rhoE / rho - usq / 2.0, s->Tn[n], T);
}

/* Ghost nodes of the x-faces (bc_x = 1), Sec. 5a: equilibrium populations
 * at the moments of the adjacent boundary node; zero velocity on the left. */
static int build_ghosts(orc_state *s)
{
    int st = ORC_OK;
    size_t plane = (size_t)s->ny * s->nz;
    for (int side = 0; side < 2; ++side)
        for (int z = 0; z < s->nz; ++z)
            for (int y = 0; y < s->ny; ++y) {
                int xb = side == 0 ? 0 : s->nx - 1;
                double rho_a[ORC_MAXM], u[3], T;
                int r = stored_node_state(s, node_index(s, xb, y, z), rho_a, u, &T);
                if (r != ORC_OK) st = r;
                if (side == 0) u[0] = u[1] = u[2] = 0.0;
                equilibrium_sets(s, rho_a, u, T,
                                 s->ghost + ((size_t)side * plane + (size_t)y + (size_t)s->ny * z) * s->S * ORC_Q);
            }
    return st;
}

/* Pull streaming: s_i(x) = s_i^post(x - c_i) for every stored set. */
static void stream(orc_state *s)
{
    int S = s->S;
    #pragma omp parallel for schedule(static)
    for (int n = 0; n < s->N; ++n) {
        int x = n % s->nx, y = (n / s->nx) % s->ny, z = n / (s->nx * s->ny);
        for (int i = 0; i < ORC_Q; ++i) {
            int xs = x - cx_of(i);
            int ys = wrap(y - cy_of(i), s->ny), zs = wrap(z - cz_of(i), s->nz);
            const double *src;
            if (xs >= 0 && xs < s->nx) {
                src = s->pop + node_index(s, xs, ys, zs) * S * ORC_Q;
            } else if (s->bc_x == 0) {
                src = s->pop + node_index(s, wrap(xs, s->nx), ys, zs) * S * ORC_Q;
            } else {
                int side = xs < 0 ? 0 : 1;
                src = s->ghost + ((size_t)side * s->ny * s->nz + (size_t)ys + (size_t)s->ny * zs) * S * ORC_Q;
            }
            for (int k = 0; k < S; ++k)
                s->tmp[((size_t)n * S + k) * ORC_Q + i] = src[k * ORC_Q + i];
        }
    }
}

/* Pass 1 at one node: slaving, moments, composition, temperature,
 * isotropy-correction potential Phi and (1/omega - 1/2). */
static int moments_node(orc_state *s, size_t n)
{
    int M = s->M, S = s->S;
    const double *p = s->tmp + n * S * ORC_Q;
    /* Eq. (strongest): f_{M i} = f_i - sum_{a<M} f_{a i} */
    double fM[ORC_Q];
    for (int i = 0; i < ORC_Q; ++i) {
        fM[i] = p[(M - 1) * ORC_Q + i];
        for (int a = 0; a < M - 1; ++a) fM[i] -= p[a * ORC_Q + i];
    }
    /* Eq. (Pa): species densities and momenta */
    for (int a = 0; a < M; ++a) {
        double r = 0.0, ja[3] = {0, 0, 0};
        for (int i = 0; i < ORC_Q; ++i) {
            double f = (a < M - 1) ? p[a * ORC_Q + i] : fM[i];
            r += f;
            ja[0] += f * cx_of(i); ja[1] += f * cy_of(i); ja[2] += f * cz_of(i);
        }
        s->rho_a[n * M + a] = r;
        for (int d = 0; d < 3; ++d) s->j_a[(n * M + a) * 3 + d] = ja[d];
    }
    /* mixture: rho, rho u, pressure tensor P = sum f c c; energy: rho E, q */
    double rho = 0.0, j[3] = {0, 0, 0}, Pt[3][3] = {{0}}, rhoE = 0.0, q[3] = {0, 0, 0};
    for (int i = 0; i < ORC_Q; ++i) {
        double f = p[(M - 1) * ORC_Q + i], g = p[M * ORC_Q + i];
        int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        rho += f;
        rhoE += g;
        for (int a = 0; a < 3; ++a) {
            j[a] += f * c[a];
            q[a] += g * c[a];
            for (int b = 0; b < 3; ++b) Pt[a][b] += f * c[a] * c[b];
        }
    }
    s->rho[n] = rho;
    s->rhoE[n] = rhoE;
    for (int a = 0; a < 3; ++a) {
        s->j[n * 3 + a] = j[a];
        s->q[n * 3 + a] = q[a];
        for (int b = 0; b < 3; ++b) s->Pt[n * 9 + 3 * a + b] = Pt[a][b];
    }
    int st = ORC_OK;
    if (!(rho > 0.0) || !isfinite(rhoE)) st = ORC_ERR_NONFINITE;
    double inv_m = 0.0;
    for (int a = 0; a < M; ++a) {
        double Ya = s->rho_a[n * M + a] / rho;
        s->Y[n * M + a] = Ya;
        inv_m += Ya / s->W[a];
        if (s->rho_a[n * M + a] < -1e-10 * rho && st == ORC_OK) st = ORC_ERR_NEGATIVE;
    }
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double T;
    int r = solve_temperature(s, s->Y + n * M, rhoE / rho - usq / 2.0, s->Tn[n], &T);
    if (r != ORC_OK && st == ORC_OK) st = r;
    s->T[n] = T;
    double Rmix = s->r_lat * inv_m;
    /* Eq. (Xalpha): Phi_alpha = rho u_alpha (1 - 3RT) - rho u_alpha^3 */
    for (int a = 0; a < 3; ++a)
        s->Phi[n * 3 + a] = rho * u[a] * (1.0 - 3.0 * Rmix * T) - rho * u[a] * u[a] * u[a];
    /* Eq. (mu): 1/omega - 1/2 */
    double nup1, dfac;
    relaxation(s, s->Y + n * M, Rmix, T, rho * Rmix * T, &s->nup[n], &nup1, &dfac);
    return st;
}

/* Neighbour index for the gradient stencils: periodic in y, z; periodic or
 * zero-gradient continuation (clamp) in x. */
static size_t stencil_neighbor(const orc_state *s, int x, int y, int z, int i)
{
    int xn = x + cx_of(i), yn = wrap(y + cy_of(i), s->ny), zn = wrap(z + cz_of(i), s->nz);
    if (s->bc_x == 0) xn = wrap(xn, s->nx);
    else { if (xn < 0) xn = 0; if (xn >= s->nx) xn = s->nx - 1; }
    return node_index(s, xn, yn, zn);
}

/* Pass 2: G_alpha = (1/omega - 1/2) d_alpha Phi_alpha and grad Y_a. */
static void gradients_node(orc_state *s, size_t n)
{
    int M = s->M;
    int x = (int)(n % s->nx), y = (int)((n / s->nx) % s->ny), z = (int)(n / ((size_t)s->nx * s->ny));
    double dPhi[3] = {0, 0, 0};
    double gY[ORC_MAXM][3];
    for (int a = 0; a < M; ++a) gY[a][0] = gY[a][1] = gY[a][2] = 0.0;
    for (int i = 0; i < ORC_Q; ++i) {
        size_t nb = stencil_neighbor(s, x, y, z, i);
        int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        double wi = w_of(i);
        for (int a = 0; a < 3; ++a) dPhi[a] += wi * c[a] * s->Phi[nb * 3 + a];
        for (int a = 0; a < M; ++a)
            for (int d = 0; d < 3; ++d) gY[a][d] += wi * c[d] * s->Y[nb * M + a];
    }
    for (int a = 0; a < 3; ++a) s->G[n * 3 + a] = s->nup[n] * dPhi[a] / THETA;
    for (int a = 0; a < M; ++a)
        for (int d = 0; d < 3; ++d) s->gradY[(n * M + a) * 3 + d] = gY[a][d] / THETA;
}

/* Pass 3 at one node: X, relaxation rates, Stefan-Maxwell solve,
 * chemistry and the collisions of all sets; writes pop[n]. */
static int collide_node(orc_state *s, size_t n)
{
    int M = s->M, S = s->S;
    int x = (int)(n % s->nx), y = (int)((n / s->nx) % s->ny), z = (int)(n / ((size_t)s->nx * s->ny));
    const double *p = s->tmp + n * S * ORC_Q;
    double *out = s->pop + n * S * ORC_Q;
    int st = ORC_OK;

    /* Eq. (Xalpha): X_alpha = - d_alpha G_alpha */
    double X[3] = {0, 0, 0};
    for (int i = 0; i < ORC_Q; ++i) {
        size_t nb = stencil_neighbor(s, x, y, z, i);
        int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        for (int a = 0; a < 3; ++a) X[a] += w_of(i) * c[a] * s->G[nb * 3 + a];
    }
    for (int a = 0; a < 3; ++a) X[a] = -X[a] / THETA;

    double rho = s->rho[n], T = s->T[n], rhoE = s->rhoE[n];
    const double *Y = s->Y + n * M, *rho_a = s->rho_a + n * M;
    double u[3] = {s->j[n * 3] / rho, s->j[n * 3 + 1] / rho, s->j[n * 3 + 2] / rho};
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double inv_m = 0.0;
    for (int a = 0; a < M; ++a) inv_m += Y[a] / s->W[a];
    double m = 1.0 / inv_m;
    double Rmix = s->r_lat * inv_m;
    double P = rho * Rmix * T;                                   /* Eq. (eosIdealGas) */

    /* relaxation parameters, Eqs. (mu) and (lambda) */
    double nup, nup1, dfac;
    relaxation(s, Y, Rmix, T, P, &nup, &nup1, &dfac);
    double omega = 1.0 / (0.5 + nup);
    double omega1 = 1.0 / (0.5 + nup1);

    /* Eq. (tauab) and Eq. (fStar): 1/tau_ab, 1/tau_a, beta_a */
    double itab[ORC_MAXM][ORC_MAXM], ita[ORC_MAXM], beta[ORC_MAXM];
    for (int a = 0; a < M; ++a) {
        ita[a] = 0.0;
        for (int b = 0; b < M; ++b) {
            itab[a][b] = (a == b) ? 0.0 : inv_tau_ab(s, a, b, m, T) / dfac;
            if (b != a) ita[a] += Y[b] * itab[a][b];
        }
        double tau_a = 1.0 / ita[a];
        beta[a] = 1.0 / (2.0 * tau_a + 1.0);
    }

    /* Eq. (transform1): (1 + 1/(2 tau_a)) du_a - (1/2) sum_{b!=a} Y_b du_b / tau_ab = u_a - u */
    double A[ORC_MAXM][ORC_MAXM], rhs[ORC_MAXM][3], du[ORC_MAXM][3];
    for (int a = 0; a < M; ++a) {
        for (int b = 0; b < M; ++b)
            A[a][b] = (a == b) ? 1.0 + ita[a] / 2.0 : -0.5 * itab[a][b] * Y[b];
        for (int d = 0; d < 3; ++d) rhs[a][d] = s->j_a[(n * M + a) * 3 + d] / rho_a[a] - u[d];
    }
    int r = solve_linear(M, A, rhs, du);
    if (r != ORC_OK) st = r;

    /* chemistry */
    double wdot[ORC_MAXM];
    production_rates(s, rho_a, T, wdot);

    /* species a < M: Eq. (finalNumericalEquations) with F_ai of Eq. (fStar),
     * quasi-equilibria at u + du_b (Eq. (fstar)) and the source Eq. (fsource) */
    for (int a = 0; a < M - 1; ++a) {
        double zeta_a = R_spec(s, a) * T;
        for (int i = 0; i < ORC_Q; ++i) {
            double feq = product_form(i, rho_a[a], u, zeta_a);
            double F = 0.0;
            for (int b = 0; b < M; ++b) {
                if (b == a) continue;
                double zeta_b = R_spec(s, b) * T;
                double ub[3] = {u[0] + du[b][0], u[1] + du[b][1], u[2] + du[b][2]};
                double fbeq = product_form(i, rho_a[b], u, zeta_b);
                double fbst = product_form(i, rho_a[b], ub, zeta_b);
                F += itab[a][b] * (fbeq - fbst);
            }
            F *= Y[a];
            double src = product_form(i, wdot[a], u, zeta_a);
            double f = p[a * ORC_Q + i];
            out[a * ORC_Q + i] = f + 2.0 * beta[a] * (feq - f) + (beta[a] - 1.0) * F + src;
        }
    }

    /* mixture f: Eq. (f) with Eq. (feqmix) and A_i of Eq. (Ai) */
    for (int i = 0; i < ORC_Q; ++i) {
        int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        double AX = 0.0;
        if (c2 == 1) AX = 0.5 * (c[0] * X[0] + c[1] * X[1] + c[2] * X[2]);
        double f = p[(M - 1) * ORC_Q + i];
        out[(M - 1) * ORC_Q + i] = f + omega * (product_form(i, rho, u, Rmix * T) - f) + AX;
    }

    /* energy g: Eq. (g) with Grad equilibria */
    double H = 0.0, sumHYdu[3] = {0, 0, 0}, sumHgradY[3] = {0, 0, 0};
    for (int a = 0; a < M; ++a) {
        double Ha = H_spec(s, a, T);
        H += Y[a] * Ha;
        for (int d = 0; d < 3; ++d) {
            sumHYdu[d] += Ha * Y[a] * du[a][d];
            sumHgradY[d] += Ha * s->gradY[(n * M + a) * 3 + d];
        }
    }
    double Peq[3][3], Req[3][3], qeq[3], qst[3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Peq[a][b] = (a == b ? P : 0.0) + rho * u[a] * u[b];
            Req[a][b] = (H + usq / 2.0) * Peq[a][b] + P * u[a] * u[b];      /* Eq. (geq2mom) */
        }
    for (int a = 0; a < 3; ++a) qeq[a] = (H + usq / 2.0) * rho * u[a];  /* Eq. (geq1mom) */
    for (int b = 0; b < 3; ++b) {
        double uPdiff = 0.0;
        for (int a = 0; a < 3; ++a) uPdiff += u[a] * (s->Pt[n * 9 + 3 * a + b] - Peq[a][b]);
        double qdiff = (omega1 / (omega - omega1)) * rho * sumHYdu[b];                  /* Eq. (qdiff) */
        double qcorr = 0.5 * ((omega1 - 2.0) / (omega1 - omega)) * P * sumHgradY[b];    /* Eq. (corrFourier) */
        qst[b] = s->q[n * 3 + b] - uPdiff + qdiff + qcorr;                              /* Eq. (gstareq1mom) */
    }
    for (int i = 0; i < ORC_Q; ++i) {
        double geq = grad_pop(i, rhoE, qeq, Req);
        double gst = grad_pop(i, rhoE, qst, Req);
        double g = p[M * ORC_Q + i];
        out[M * ORC_Q + i] = g + omega1 * (geq - g) + (omega - omega1) * (gst - g);
    }

    for (int k = 0; k < S * ORC_Q; ++k)
        if (!isfinite(out[k])) { st = ORC_ERR_NONFINITE; break; }
    s->Tn[n] = T;
    return st;
}

/* Streams the stored state and evaluates the pass-1 fields. */
static int stream_and_moments(orc_state *s)
{
    int st = ORC_OK;
    if (s->bc_x == 1) {
        int r = build_ghosts(s);
        if (r != ORC_OK) st = r;
    }
    stream(s);
    int st1 = ORC_OK;
    #pragma omp parallel for schedule(static) reduction(min:st1)
    for (int n = 0; n < s->N; ++n) {
        int r = moments_node(s, (size_t)n);
        if (r < st1) st1 = r;
    }
    return st != ORC_OK ? st : st1;
}

/* One or more full time steps. Returns the first error met (or 0). */
int orc_step(orc_state *s, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        int st = stream_and_moments(s);
        #pragma omp parallel for schedule(static)
        for (int n = 0; n < s->N; ++n) gradients_node(s, (size_t)n);
        int st3 = ORC_OK;
        #pragma omp parallel for schedule(static) reduction(min:st3)
        for (int n = 0; n < s->N; ++n) {
            int r = collide_node(s, (size_t)n);
            if (r < st3) st3 = r;
        }
        if (st == ORC_OK) st = st3;
        if (st != ORC_OK) { s->status = st; return st; }
    }
    return ORC_OK;
}

/* Macroscopic fields of the current time level (the moments the next
 * collision sees).  Any output may be NULL.  Layouts: rho_a[M][N],
 * rhou[3][N], rhoE[N], T[N], j_a[M][3][N]. */
int orc_moments(orc_state *s, double *rho_a, double *rhou, double *rhoE, double *T, double *j_a)
{
    int st = stream_and_moments(s);
    int M = s->M;
    size_t N = (size_t)s->N;
    for (size_t n = 0; n < N; ++n) {
        for (int a = 0; a < M; ++a) {
            if (rho_a) rho_a[(size_t)a * N + n] = s->rho_a[n * M + a];
            if (j_a) for (int d = 0; d < 3; ++d) j_a[((size_t)a * 3 + d) * N + n] = s->j_a[(n * M + a) * 3 + d];
        }
        if (rhou) for (int d = 0; d < 3; ++d) rhou[(size_t)d * N + n] = s->j[n * 3 + d];
        if (rhoE) rhoE[n] = s->rhoE[n];
        if (T) T[n] = s->T[n];
    }
    return st;
}

/* Raw access to the stored populations, layout [N][S][27]. */
void orc_get_pop(const orc_state *s, double *out)
{
    memcpy(out, s->pop, (size_t)s->N * s->S * ORC_Q * sizeof(double));
}
void orc_set_pop(orc_state *s, const double *in)
{
    memcpy(s->pop, in, (size_t)s->N * s->S * ORC_Q * sizeof(double));
}
void orc_get_T(const orc_state *s, double *out) { memcpy(out, s->Tn, (size_t)s->N * sizeof(double)); }
void orc_set_T(orc_state *s, const double *in) { memcpy(s->Tn, in, (size_t)s->N * sizeof(double)); }

/* ------------------------------------------------------------------ */
/* Point-wise entry points used by the tests that pin the oracle.     */
/* ------------------------------------------------------------------ */
void orc_thermo(const orc_state *s, double T, double *U, double *H, double *Cv, double *gRT)
{
    for (int a = 0; a < s->M; ++a) {
        if (U) U[a] = U_spec(s, a, T);
        if (H) H[a] = H_spec(s, a, T);
        if (Cv) Cv[a] = Cv_spec(s, a, T);
        if (gRT) gRT[a] = gRT_spec(s, a, T);
    }
}

int orc_temperature(const orc_state *s, const double *Y, double e, double T_guess, double *T)
{
    return solve_temperature(s, Y, e, T_guess, T);
}

void orc_rates(const orc_state *s, const double *rho_a, double T, double *wdot)
{
    production_rates(s, rho_a, T, wdot);
}

/* Heat release rate at a node state, Sec. 5b: hdot^c = -sum_a H_a rho_dot_a,
 * with H_a the specific enthalpy (Eq. (specHa)) and rho_dot_a the
 * production rates above. */
double orc_heat_release(const orc_state *s, const double *rho_a, double T)
{
    double wdot[ORC_MAXM];
    production_rates(s, rho_a, T, wdot);
    double h = 0.0;
    for (int a = 0; a < s->M; ++a) h -= H_spec(s, a, T) * wdot[a];
    return h;
}

/* Heat release summed over the lattice at the current time level (the
 * state the next collision sees: pulled populations, their moments and
 * temperature), Sec. 5b.  *status receives the moment pass's status. */
double orc_total_heat_release(orc_state *s, int *status)
{
    int st = stream_and_moments(s);
    if (status) *status = st;
    double J = 0.0;
    for (int n = 0; n < s->N; ++n) J += orc_heat_release(s, s->rho_a + (size_t)n * s->M, s->T[n]);
    return J;
}

/* Diffusion velocities du[M][3] from Eq. (transform1) at a node state. */
int orc_diffusion_velocities(const orc_state *s, const double *Y, const double *ua_minus_u, double T, double *du)
{
    int M = s->M;
    double inv_m = 0.0;
    for (int a = 0; a < M; ++a) inv_m += Y[a] / s->W[a];
    double m = 1.0 / inv_m, A[ORC_MAXM][ORC_MAXM], rhs[ORC_MAXM][3], x[ORC_MAXM][3];
    for (int a = 0; a < M; ++a) {
        double ita = 0.0;
        for (int b = 0; b < M; ++b) if (b != a) ita += Y[b] * inv_tau_ab(s, a, b, m, T);
        for (int b = 0; b < M; ++b)
            A[a][b] = (a == b) ? 1.0 + ita / 2.0 : -0.5 * inv_tau_ab(s, a, b, m, T) * Y[b];
        for (int d = 0; d < 3; ++d) rhs[a][d] = ua_minus_u[3 * a + d];
    }
    int r = solve_linear(M, A, rhs, x);
    for (int a = 0; a < M; ++a)
        for (int d = 0; d < 3; ++d) du[3 * a + d] = x[a][d];
    return r;
}

/* ------------------------------------------------------------------ */
/* Flame diagnostics of the circular expanding flame (Sec. 5b)         */
/* ------------------------------------------------------------------ */
/* Diffusion velocities du[M][3] of node n of the current time level
 * (Eq. (transform1) with the relaxation of this node, as in collide_node). */
static int node_diffusion_velocities(const orc_state *s, size_t n, double du[ORC_MAXM][3])
{
    int M = s->M;
    double rho = s->rho[n], T = s->T[n];
    const double *Y = s->Y + n * M, *rho_a = s->rho_a + n * M;
    double u[3] = {s->j[n * 3] / rho, s->j[n * 3 + 1] / rho, s->j[n * 3 + 2] / rho};
    double inv_m = 0.0;
    for (int a = 0; a < M; ++a) inv_m += Y[a] / s->W[a];
    double m = 1.0 / inv_m, Rmix = s->r_lat * inv_m, P = rho * Rmix * T;
    double nup, nup1, dfac;
    relaxation(s, Y, Rmix, T, P, &nup, &nup1, &dfac);
    double A[ORC_MAXM][ORC_MAXM], rhs[ORC_MAXM][3];
    for (int a = 0; a < M; ++a) {
        double ita = 0.0;
        for (int b = 0; b < M; ++b) if (b != a) ita += Y[b] * inv_tau_ab(s, a, b, m, T) / dfac;
        for (int b = 0; b < M; ++b)
            A[a][b] = (a == b) ? 1.0 + ita / 2.0 : -0.5 * inv_tau_ab(s, a, b, m, T) / dfac * Y[b];
        for (int d = 0; d < 3; ++d) rhs[a][d] = s->j_a[(n * M + a) * 3 + d] / rho_a[a] - u[d];
    }
    return solve_linear(M, A, rhs, du);
}

/* The local displacement speed of Eq. (sd) and the absolute propagation
 * speed at every node of the current time level:
 *   S_d = [ -sum_a H_a rho_dot_a + div(lambda grad T)
 *           - rho (sum_a C_a,p Y_a du_a) . grad T ] / (rho C_p |grad T|),
 *   S_a = S_d + u . n,  n = -grad T / |grad T|,
 * lambda = (1/omega_1 - 1/2) P C_p (Eq. (lambda)), the gradients by the
 * isotropic lattice stencil (the divergence as the sum of the component
 * derivatives of lambda grad T).  Nodes with grad T = 0 get 0. */
int orc_flame_speeds(orc_state *s, double *Sd, double *Sa)
{
    int st = stream_and_moments(s);
    int M = s->M;
    size_t N = (size_t)s->N;
    double *gT = (double *)calloc(3 * N, sizeof(double)), *lg = (double *)calloc(3 * N, sizeof(double));
    double *Cp = (double *)calloc(N, sizeof(double));
    if (!gT || !lg || !Cp) { free(gT); free(lg); free(Cp); return ORC_ERR_ARG; }
    for (size_t n = 0; n < N; ++n) {
        int x = (int)(n % s->nx), y = (int)((n / s->nx) % s->ny), z = (int)(n / ((size_t)s->nx * s->ny));
        for (int i = 0; i < ORC_Q; ++i) {
            size_t nb = stencil_neighbor(s, x, y, z, i);
            int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
            for (int a = 0; a < 3; ++a) gT[n * 3 + a] += w_of(i) * c[a] * s->T[nb] / THETA;
        }
        const double *Y = s->Y + n * M;
        double inv_m = 0.0, Cv = 0.0;
        for (int a = 0; a < M; ++a) { inv_m += Y[a] / s->W[a]; Cv += Y[a] * Cv_spec(s, a, s->T[n]); }
        double Rmix = s->r_lat * inv_m, P = s->rho[n] * Rmix * s->T[n];
        double nup, nup1, dfac;
        relaxation(s, Y, Rmix, s->T[n], P, &nup, &nup1, &dfac);
        Cp[n] = Cv + Rmix;
        double lam = nup1 * P * Cp[n];
        for (int a = 0; a < 3; ++a) lg[n * 3 + a] = lam * gT[n * 3 + a];
    }
    for (size_t n = 0; n < N; ++n) {
        int x = (int)(n % s->nx), y = (int)((n / s->nx) % s->ny), z = (int)(n / ((size_t)s->nx * s->ny));
        double div = 0.0;
        for (int i = 0; i < ORC_Q; ++i) {
            size_t nb = stencil_neighbor(s, x, y, z, i);
            int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
            for (int a = 0; a < 3; ++a) div += w_of(i) * c[a] * lg[nb * 3 + a] / THETA;
        }
        double T = s->T[n], rho = s->rho[n];
        const double *Y = s->Y + n * M;
        double wdot[ORC_MAXM], du[ORC_MAXM][3];
        production_rates(s, s->rho_a + n * M, T, wdot);
        int r = node_diffusion_velocities(s, n, du);
        if (r != ORC_OK && st == ORC_OK) st = r;
        double hdot = 0.0, fl[3] = {0, 0, 0};
        for (int a = 0; a < M; ++a) {
            hdot -= H_spec(s, a, T) * wdot[a];
            double cpa = Cv_spec(s, a, T) + R_spec(s, a);
            for (int d = 0; d < 3; ++d) fl[d] += cpa * Y[a] * du[a][d];
        }
        const double *g = gT + n * 3;
        double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        if (gn == 0.0) { Sd[n] = Sa[n] = 0.0; continue; }
        double num = hdot + div - rho * (fl[0] * g[0] + fl[1] * g[1] + fl[2] * g[2]);
        Sd[n] = num / (rho * Cp[n] * gn);
        double un = -(s->j[n * 3] * g[0] + s->j[n * 3 + 1] * g[1] + s->j[n * 3 + 2] * g[2]) / (rho * gn);
        Sa[n] = Sd[n] + un;
    }
    free(gT); free(lg); free(Cp);
    return st;
}

/* Means along the isoline T = T_iso in the plane z = 0, Eq. (rmean):
 * A^{-1} \int f dA with A the isoline's length.  Marching squares on the
 * cells (x, y)..(x+1, y+1) of the periodic x-y lattice: a crossing on a
 * cell edge where T - T_iso changes sign (T >= T_iso counts as above), at
 * the linear interpolation point, with the fields interpolated alike; the
 * two crossings of a cell make one straight segment; a cell with four
 * crossings is split according to the mean of its corners.  Each segment
 * adds its length times the mean of its ends' values (the trapezoid rule).
 * T [N], fields [K][N]; out = {A, mean R, mean field_0 .. field_{K-1}},
 * R the distance from (cx, cy); positions are not wrapped (the isoline is
 * assumed not to cross the box edge). */
void orc_isoline_means(const orc_state *s, const double *T, double T_iso, double cx, double cy, int K,
                       const double *fields, double *out)
{
    size_t N = (size_t)s->N;
    int nx = s->nx, ny = s->ny;
    double acc[2 + 16] = {0};
    for (int k = 0; k < 2 + K; ++k) acc[k] = 0.0;
    static const int ox[4] = {0, 1, 1, 0}, oy[4] = {0, 0, 1, 1};
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t idx[4];
            double v[4];
            for (int c = 0; c < 4; ++c) {
                idx[c] = (size_t)((x + ox[c]) % nx) + (size_t)nx * ((y + oy[c]) % ny);
                v[c] = T[idx[c]];
            }
            double px[4], py[4], pf[4][16];
            int ne = 0, edge[4];
            for (int e = 0; e < 4; ++e) {
                int a = e, b = (e + 1) % 4;
                if ((v[a] >= T_iso) == (v[b] >= T_iso)) continue;
                double t = (T_iso - v[a]) / (v[b] - v[a]);
                px[ne] = x + ox[a] + t * (ox[b] - ox[a]);
                py[ne] = y + oy[a] + t * (oy[b] - oy[a]);
                for (int k = 0; k < K; ++k)
                    pf[ne][k] = fields[(size_t)k * N + idx[a]] + t * (fields[(size_t)k * N + idx[b]] - fields[(size_t)k * N + idx[a]]);
                edge[ne++] = e;
            }
            int pairs[2][2], np = 0;
            if (ne == 2) { pairs[0][0] = 0; pairs[0][1] = 1; np = 1; }
            else if (ne == 4) {
                double vc = 0.25 * (v[0] + v[1] + v[2] + v[3]);
                /* crossings are on edges 0, 1, 2, 3 in order; corner c lies
                 * between edges c-1 and c */
                if ((vc >= T_iso) == (v[0] >= T_iso)) {      /* corners 1 and 3 cut off */
                    pairs[0][0] = 0; pairs[0][1] = 1; pairs[1][0] = 2; pairs[1][1] = 3;
                } else {                                      /* corners 0 and 2 cut off */
                    pairs[0][0] = 3; pairs[0][1] = 0; pairs[1][0] = 1; pairs[1][1] = 2;
                }
                np = 2;
            }
            (void)edge;
            for (int q = 0; q < np; ++q) {
                int i = pairs[q][0], j = pairs[q][1];
                double L = sqrt((px[i] - px[j]) * (px[i] - px[j]) + (py[i] - py[j]) * (py[i] - py[j]));
                double Ri = sqrt((px[i] - cx) * (px[i] - cx) + (py[i] - cy) * (py[i] - cy));
                double Rj = sqrt((px[j] - cx) * (px[j] - cx) + (py[j] - cy) * (py[j] - cy));
                acc[0] += L;
                acc[1] += L * 0.5 * (Ri + Rj);
                for (int k = 0; k < K; ++k) acc[2 + k] += L * 0.5 * (pf[i][k] + pf[j][k]);
            }
        }
    out[0] = acc[0];
    for (int k = 1; k < 2 + K; ++k) out[k] = acc[0] > 0.0 ? acc[k] / acc[0] : 0.0;
}

/* Transport at a node state (Y [M], T, P): out = {1/omega - 1/2,
 * 1/omega_1 - 1/2, mu, lambda, dfac} (mu and lambda zero for constant
 * transport). */
void orc_transport(const orc_state *s, const double *Y, double T, double P, double *out)
{
    double inv_m = 0.0;
    for (int a = 0; a < s->M; ++a) inv_m += Y[a] / s->W[a];
    relaxation(s, Y, s->r_lat * inv_m, T, P, &out[0], &out[1], &out[4]);
    out[2] = out[3] = 0.0;
    if (s->transport) mixture_transport(s, Y, T, P, &out[2], &out[3], &out[4]);
}

/* Equilibria of every set at a macroscopic state, layout [S][27]. */
void orc_equilibrium_sets(const orc_state *s, const double *rho_a, const double *u, double T, double *out)
{
    equilibrium_sets(s, rho_a, u, T, out);
}

int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
