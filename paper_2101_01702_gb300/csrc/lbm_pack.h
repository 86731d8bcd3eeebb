// Host-side packing of an lbm_species / lbm_mechanism description into the
// constant-memory record the kernels read (MechConst), with validation.
#pragma once

#include <math.h>
#include <string.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

// Returns LBM_OK or LBM_ERR_ARG; fills mc (refs are left zero).
static inline int lbm_pack_tables(const lbm_species *sp, const lbm_mechanism *mech, MechConst &mc)
{
    memset(&mc, 0, sizeof(mc));
    if (!sp || !mech) return LBM_ERR_ARG;
    const int M = sp->M;
    if (M < 2 || M > LBMK_MAXM || !sp->W || !sp->D) return LBM_ERR_ARG;
    if (sp->thermo == LBM_THERMO_CONST_CP && (!sp->cp_R || !sp->h_form)) return LBM_ERR_ARG;
    if (sp->thermo == LBM_THERMO_POLY7 && !sp->poly7) return LBM_ERR_ARG;
    if (sp->thermo != LBM_THERMO_CONST_CP && sp->thermo != LBM_THERMO_POLY7) return LBM_ERR_ARG;
    if (sp->visc_model != LBM_VISC_KINEMATIC && sp->visc_model != LBM_VISC_RELAXATION) return LBM_ERR_ARG;
    if (!(sp->r_lat > 0) || !(sp->nu > 0) || !(sp->Pr > 0)) return LBM_ERR_ARG;
    if (sp->transport != LBM_TRANSPORT_CONSTANT && sp->transport != LBM_TRANSPORT_MIXTURE_AVERAGED) return LBM_ERR_ARG;
    if (sp->transport == LBM_TRANSPORT_MIXTURE_AVERAGED &&
        (!sp->mu0 || !sp->mu_exp || !(sp->T_tr > 0) || !(sp->P_tr > 0) || !isfinite(sp->D_exp)))
        return LBM_ERR_ARG;
    if (sp->thermo == LBM_THERMO_CONST_CP && !(sp->T0 > 0)) return LBM_ERR_ARG;
    if (mech->R < 0 || mech->R > LBMK_MAXR) return LBM_ERR_ARG;
    if (mech->R > 0 && (!mech->nu_f || !mech->nu_r || !mech->log_A || !mech->b || !mech->theta || !mech->rtype ||
                        !mech->reversible || !(mech->T_ref > 0)))
        return LBM_ERR_ARG;
    mc.M = M;
    mc.R = mech->R;
    mc.visc_model = sp->visc_model;
    mc.T0 = sp->T0;
    mc.nu = sp->nu;
    mc.Pr = sp->Pr;
    mc.r_lat = sp->r_lat;
    for (int a = 0; a < M; ++a) {
        if (!(sp->W[a] > 0)) return LBM_ERR_ARG;
        const double R = sp->r_lat / sp->W[a];
        mc.W[a] = sp->W[a];
        mc.invW[a] = 1.0 / sp->W[a];
        mc.Ra[a] = R;
        mc.Ra_f[a] = (float)R;
        if (sp->thermo == LBM_THERMO_CONST_CP) {
            // U_a = U0 + cv (T - T0), U0 = H0 - R T0, H_a = U_a + R T (Eq. (specHa))
            const double cpR = sp->cp_R[a], cv = (cpR - 1.0) * R, U0 = sp->h_form[a] - R * sp->T0;
            const double c0 = U0 - cv * sp->T0;
            const double h[6] = {cv + R, 0, 0, 0, 0, c0};
            const double u[6] = {c0, cv, 0, 0, 0, 0};
            const double g[7] = {cpR, 0, 0, 0, 0, c0 / R, cpR * log(sp->T0)};
            memcpy(mc.hco[a], h, sizeof h);
            memcpy(mc.uco[a], u, sizeof u);
            memcpy(mc.gco[a], g, sizeof g);
        } else {
            const double *p = sp->poly7 + 7 * a;
            const double h[6] = {R * p[0], R * p[1] / 2, R * p[2] / 3, R * p[3] / 4, R * p[4] / 5, R * p[5]};
            const double u[6] = {R * p[5], R * p[0] - R, R * p[1] / 2, R * p[2] / 3, R * p[3] / 4, R * p[4] / 5};
            const double g[7] = {p[0], -p[1] / 2, -p[2] / 6, -p[3] / 12, -p[4] / 20, p[5], -p[6]};
            memcpy(mc.hco[a], h, sizeof h);
            memcpy(mc.uco[a], u, sizeof u);
            memcpy(mc.gco[a], g, sizeof g);
        }
        for (int b = 0; b < M; ++b) {
            if (a == b) continue;
            const double D = sp->D[M * a + b];
            if (!(D > 0) || D != sp->D[M * b + a]) return LBM_ERR_ARG;
            mc.inv_WWD[a][b] = 1.0 / (sp->W[a] * sp->W[b] * D);
            mc.inv_WWD_f[a][b] = (float)mc.inv_WWD[a][b];
        }
    }
    mc.transport = sp->transport;
    if (sp->transport == LBM_TRANSPORT_MIXTURE_AVERAGED) {
        for (int a = 0; a < M; ++a) {
            if (!(sp->mu0[a] > 0) || !isfinite(sp->mu_exp[a])) return LBM_ERR_ARG;
            mc.mu0[a] = sp->mu0[a];
            mc.mu_exp[a] = sp->mu_exp[a];
            mc.eucken[a] = 1.25 * mc.Ra[a];
            for (int b = 0; b < M; ++b) {
                mc.wq[a][b] = pow(sp->W[b] / sp->W[a], 0.25);
                mc.wd[a][b] = 1.0 / sqrt(8.0 * (1.0 + sp->W[a] / sp->W[b]));
            }
        }
        mc.log_T_tr = log(sp->T_tr);
        mc.D_exp = sp->D_exp;
        mc.P_tr = sp->P_tr;
    }
    mc.log_T_ref = mech->R > 0 ? log(mech->T_ref) : 0.0;
    bool need_P0 = false;
    for (int k = 0; k < mech->R; ++k) {
        const int t = mech->rtype[k];
        if (t < 0 || t > 2 || (t != 0 && !mech->eff) || (t == 2 && !mech->low)) return LBM_ERR_ARG;
        mc.rtype[k] = t;
        mc.rev[k] = mech->reversible[k] ? 1 : 0;
        need_P0 |= mc.rev[k] != 0;
        mc.log_A[k] = mech->log_A[k];
        mc.b[k] = mech->b[k];
        mc.theta[k] = mech->theta[k];
        if (t == 2) {
            mc.dlow[k][0] = mech->low[3 * k] - mech->log_A[k];
            mc.dlow[k][1] = mech->low[3 * k + 1] - mech->b[k];
            mc.dlow[k][2] = mech->low[3 * k + 2] - mech->theta[k];
        }
        int nr = 0, np = 0, dn = 0;
        for (int a = 0; a < M; ++a) {
            const int f = mech->nu_f[M * k + a], g = mech->nu_r[M * k + a];
            if (f < 0 || g < 0) return LBM_ERR_ARG;
            for (int j = 0; j < f; ++j) { if (nr >= 3) return LBM_ERR_ARG; mc.reac[k][nr++] = a; }
            for (int j = 0; j < g; ++j) { if (np >= 3) return LBM_ERR_ARG; mc.prod[k][np++] = a; }
            dn += g - f;
            if (t != 0) mc.eff[k][a] = mech->eff[M * k + a];
        }
        if (nr == 0) return LBM_ERR_ARG;
        mc.nreac[k] = nr;
        mc.nprod[k] = np;
        mc.dn[k] = dn;
    }
    if (need_P0 && !(mech->P0 > 0)) return LBM_ERR_ARG;
    mc.P0_over_r = need_P0 ? mech->P0 / sp->r_lat : 1.0;
    return LBM_OK;
}

// Host value of U_a(T) from the packed coefficients.
static inline double lbm_host_U(const MechConst &mc, int a, double T)
{
    const double *u = mc.uco[a];
    return ((((u[5] * T + u[4]) * T + u[3]) * T + u[2]) * T + u[1]) * T + u[0];
}
