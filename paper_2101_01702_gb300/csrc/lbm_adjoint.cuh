// Hand-written adjoint (reverse mode) of the double-precision time step on
// periodic lattices: the transpose of the step's Jacobian applied to an
// adjoint state, plus the gradient of the heat-release objective
// J_t = sum_nodes hdot^c at the state the step's collision sees (Sec. 5b;
// hdot^c = -sum_a H_a rho_dot_a with H_a of Eq. (specHa)).
//
// Forward step at a node (lbm_kernels.cuh), in the variables used here:
//   pull       P_si(x) = F_si(x - c_i)
//   moments    rho_a, j_a (a < M-1), rho, j, P_ab, rho E, q          Eq. (Pa), Sec. 3
//   slaving    rho_{M-1} = rho - sum rho_a, j_{M-1} = j - sum j_a     Eq. (strongest)
//   Y_a = rho_a / rho, u = j / rho, 1/m = sum Y_a / W_a, R = r / m
//   T: sum_a Y_a U_a(T) = rho E / rho - |u|^2 / 2 (Newton)           Eq. (temperature)
//   P = rho R T, 1/omega - 1/2 = nu', omega_1, H_a(T), kappa = m r T  Eqs. (mu), (lambda), (specHa), (tauab)
//   1/tau_a = kappa sum_{b != a} Y_b / (W_a W_b D_ab), beta_a        Eqs. (tauab), (fStar)
//   B du = Y_a (u_a - u)  (B = Y-scaled Stefan-Maxwell matrix)       Eq. (transform1)
//   rho_dot_a(rho, T; ln A)                                          Eq. (sumRhoDot), Sec. 4
//   Phi, G = nu' d Phi, X = -d G, grad Y_a (isotropic stencils)      Eqs. (Xalpha), (corrFourier)
//   collisions of the species, mixture and energy sets              Eqs. (finalNumericalEquations), (f), (g)
//
// The reverse step for one time level runs four passes (after the forward
// moment and gradient passes of the double-precision unit have rebuilt the
// record of that level):
//   A  k_adj_collide  per node: the adjoint of the three collisions with
//      respect to the pulled populations, every node-local quantity, X and
//      sum_a H_a grad Y_a; through the chemistry (the rate-of-progress
//      Jacobian, with the objective's own hdot^c when asked), the
//      Stefan-Maxwell solve (B^T = B), 1/tau_a, the relaxation rates, the
//      enthalpies and the implicit Newton temperature
//      (dT = (de - sum_a U_a dY_a) / C_v) down to the pulled moments;
//   B  k_adj_grad1    per node: adj G = transposed outer stencil of adj X,
//      adj nu' = adj G . d Phi, and nu' adj G;
//   C  k_adj_finish   per node: adj Phi and adj Y from the transposed inner
//      stencils, carried to the moments, and the adjoint of the pulled
//      populations (direct part plus moments);
//   D  k_adj_gather   transposed pull: lam_si(x) = adj P_si(x + c_i).
// The gradient with respect to ln A_k is summed per block (fixed order).
#pragma once
#if LBMK_MIXED
#error "the adjoint is part of the double-precision unit"
#endif

namespace {

// ---------------------------------------------------------------------
// Product-form factors of Eq. (phis) at (v, zeta) with their derivatives:
// P[d][c+1] = Psi_c(v_d, zeta), V = dPsi/dv_d, Z = dPsi/dzeta.
// ---------------------------------------------------------------------
struct PsiTab {
    double P[3][3], V[3][3], Z[3][3];
};

__device__ __forceinline__ void psi_tab(PsiTab &t, const double v[3], double z)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double s = fma(v[d], v[d], z);
        t.P[d][0] = 0.5 * (s - v[d]);
        t.V[d][0] = v[d] - 0.5;
        t.Z[d][0] = 0.5;
        t.P[d][1] = 1.0 - s;
        t.V[d][1] = -2.0 * v[d];
        t.Z[d][1] = -1.0;
        t.P[d][2] = 0.5 * (s + v[d]);
        t.V[d][2] = v[d] + 0.5;
        t.Z[d][2] = 0.5;
    }
}

template <int I>
__device__ __forceinline__ double psi_at(const PsiTab &t)
{
    return t.P[0][CX(I) + 1] * t.P[1][CY(I) + 1] * t.P[2][CZ(I) + 1];
}

// Weights l(I): returns sum_i l_i psi_i and adds sum_i l_i dpsi_i/dv_d to
// dv[d] and sum_i l_i dpsi_i/dzeta to dz.
template <class L>
__device__ __forceinline__ double psi_adj(const PsiTab &t, L &&l, double dv[3], double &dz)
{
    double S = 0.0;
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        constexpr int x = CX(I) + 1, y = CY(I) + 1, z = CZ(I) + 1;
        const double w = l(I);
        const double a = t.P[0][x], b = t.P[1][y], c = t.P[2][z];
        const double bc = b * c;
        S = fma(w * a, bc, S);
        dv[0] = fma(w * t.V[0][x], bc, dv[0]);
        dv[1] = fma(w * a * t.V[1][y], c, dv[1]);
        dv[2] = fma(w * a * b, t.V[2][z], dv[2]);
        dz = fma(w, t.Z[0][x] * bc + a * (t.Z[1][y] * c + b * t.Z[2][z]), dz);
    });
    return S;
}

// ---------------------------------------------------------------------
// Chemistry.  rates_d: the production rates rho_dot_a of the mechanism
// (mass-action, third-body and Lindemann forms, reverse rates from K_c).
// weighted_progress: Q = sum_k c_k q_k with
//   c_k = sum_a wsp_a W_a (nu''_ak - nu'_ak) - (with_hrr ? Delta H_k : 0),
// i.e. sum_a wsp_a rho_dot_a (+ hdot^c), and its derivatives in T and in
// every rho_a (slaved species included); c_k q_k d ln q_k / d ln A_k is
// added to dA[k * stride].  Delta H_k = sum_a W_a (nu''_ak - nu'_ak) H_a
// also enters d ln K_c / dT (van 't Hoff).
// ---------------------------------------------------------------------
template <int M>
__device__ void rates_d(const MechConst &mc, double T, const double *rho_a, double *rho_dot)
{
    const double invT = 1.0 / T, lnTr = log(T) - mc.log_T_ref;
    const double lnc0 = log(mc.P0_over_r * invT);
    double conc[M], g[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        conc[s] = rho_a[s] * mc.invW[s];
        const double *gc = mc.gco[s];
        g[s] = fma(gc[0], 1.0 - log(T),
                   fma(fma(fma(fma(gc[4], T, gc[3]), T, gc[2]), T, gc[1]), T, fma(gc[5], invT, gc[6])));
        rho_dot[s] = 0.0;
    }
    for (int k = 0; k < mc.R; ++k) {
        const int nr = mc.nreac[k], np = mc.nprod[k];
        double dG = 0.0, Pf = 1.0, Pp = 1.0;
        for (int j = 0; j < nr; ++j) {
            dG -= g[mc.reac[k][j]];
            Pf *= conc[mc.reac[k][j]];
        }
        for (int j = 0; j < np; ++j) {
            dG += g[mc.prod[k][j]];
            Pp *= conc[mc.prod[k][j]];
        }
        const double lnkf = fma(mc.b[k], lnTr, fma(-mc.theta[k], invT, mc.log_A[k]));
        const double kf = exp_table(lnkf);
        const double kr = mc.rev[k] ? exp_table(lnkf - fma((double)mc.dn[k], lnc0, -dG)) : 0.0;
        double F = 1.0;
        if (mc.rtype[k] != 0) {
            double cM = 0.0;
#pragma unroll
            for (int s = 0; s < M; ++s) cM = fma(mc.eff[k][s], conc[s], cM);
            if (mc.rtype[k] == 1) {
                F = cM;
            } else {
                const double Pr = exp_table(fma(mc.dlow[k][1], lnTr, fma(-mc.dlow[k][2], invT, mc.dlow[k][0]))) * cM;
                F = Pr / (1.0 + Pr);
            }
        }
        const double q = F * (kf * Pf - kr * Pp);
        for (int j = 0; j < nr; ++j) rho_dot[mc.reac[k][j]] -= mc.W[mc.reac[k][j]] * q;
        for (int j = 0; j < np; ++j) rho_dot[mc.prod[k][j]] += mc.W[mc.prod[k][j]] * q;
    }
}

template <int M>
__device__ double weighted_progress(const MechConst &mc, double T, const double *rho_a, const double *wsp,
                                    bool with_hrr, double *dT_out, double *drho, double *dA, int stride)
{
    const double invT = 1.0 / T, lnTr = log(T) - mc.log_T_ref;
    const double lnc0 = log(mc.P0_over_r * invT);
    const double vhf = invT * invT / mc.r_lat;                 // 1/(r T^2)
    double conc[M], WH[M], Wcp[M], Ww[M], g[M], dc[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        conc[s] = rho_a[s] * mc.invW[s];
        WH[s] = mc.W[s] * H_spec(mc, s, T);
        Wcp[s] = mc.W[s] * cp_spec(mc, s, T);
        Ww[s] = mc.W[s] * wsp[s];
        const double *gc = mc.gco[s];
        g[s] = fma(gc[0], 1.0 - log(T),
                   fma(fma(fma(fma(gc[4], T, gc[3]), T, gc[2]), T, gc[1]), T, fma(gc[5], invT, gc[6])));
        dc[s] = 0.0;
    }
    double Q = 0.0, dT = 0.0;
    for (int k = 0; k < mc.R; ++k) {
        const int nr = mc.nreac[k], np = mc.nprod[k];
        double dH = 0.0, dHdT = 0.0, dG = 0.0, wk = 0.0, Pf = 1.0, Pp = 1.0;
        for (int j = 0; j < nr; ++j) {
            const int s = mc.reac[k][j];
            dH -= WH[s];
            dHdT -= Wcp[s];
            dG -= g[s];
            wk -= Ww[s];
            Pf *= conc[s];
        }
        for (int j = 0; j < np; ++j) {
            const int s = mc.prod[k][j];
            dH += WH[s];
            dHdT += Wcp[s];
            dG += g[s];
            wk += Ww[s];
            Pp *= conc[s];
        }
        const double ck = with_hrr ? wk - dH : wk;
        const double lnkf = fma(mc.b[k], lnTr, fma(-mc.theta[k], invT, mc.log_A[k]));
        const double kf = exp_table(lnkf);
        const double dlnkf = fma(mc.theta[k], invT, mc.b[k]) * invT;
        double kr = 0.0, dlnkr = 0.0;
        if (mc.rev[k]) {
            kr = exp_table(lnkf - fma((double)mc.dn[k], lnc0, -dG));
            dlnkr = dlnkf - fma(dH, vhf, -mc.dn[k] * invT);
        }
        const double qf = kf * Pf, qr = kr * Pp, q0 = qf - qr;
        double F = 1.0, dFdT = 0.0, dFdcM = 0.0, sA = 1.0;
        const int type = mc.rtype[k];
        if (type != 0) {
            double cM = 0.0;
#pragma unroll
            for (int s = 0; s < M; ++s) cM = fma(mc.eff[k][s], conc[s], cM);
            if (type == 1) {
                F = cM;
                dFdcM = 1.0;
            } else {
                const double k0r = exp_table(fma(mc.dlow[k][1], lnTr, fma(-mc.dlow[k][2], invT, mc.dlow[k][0])));
                const double Pr = k0r * cM, i1 = 1.0 / (1.0 + Pr);
                F = Pr * i1;
                dFdcM = k0r * i1 * i1;
                dFdT = F * i1 * fma(mc.dlow[k][2], invT, mc.dlow[k][1]) * invT;
                sA = F;                                     // d ln q / d ln A_k = Pr/(1+Pr)
            }
        }
        const double q = F * q0;
        Q = fma(ck, q, Q);
        dA[k * stride] += ck * q * sA;
        dT += ck * fma(F, qf * dlnkf - qr * dlnkr, q0 * dFdT);
        if (with_hrr) dT -= dHdT * q;
        const double wf = ck * F * kf, wr = -ck * F * kr;
        for (int j = 0; j < nr; ++j) {
            double pj = wf;
            for (int i = 0; i < nr; ++i)
                if (i != j) pj *= conc[mc.reac[k][i]];
            dc[mc.reac[k][j]] += pj;
        }
        if (mc.rev[k])
            for (int j = 0; j < np; ++j) {
                double pj = wr;
                for (int i = 0; i < np; ++i)
                    if (i != j) pj *= conc[mc.prod[k][i]];
                dc[mc.prod[k][j]] += pj;
            }
        if (type != 0) {
            const double wm = ck * q0 * dFdcM;
#pragma unroll
            for (int s = 0; s < M; ++s) dc[s] = fma(wm, mc.eff[k][s], dc[s]);
        }
    }
    *dT_out = dT;
#pragma unroll
    for (int s = 0; s < M; ++s) drho[s] = dc[s] * mc.invW[s];
    return Q;
}

// ---------------------------------------------------------------------
// Node primitives and their adjoints, carried down to the pulled moments:
//   R = r inv_m, inv_m = sum_a Y_a / W_a;
//   T from sum_a Y_a U_a(T) = e:  adj e = adj T / C_v, adj Y_a -= adj T U_a / C_v;
//   e = rho E / rho - |u|^2/2;  u = j / rho;  Y_a = rho_a / rho;
//   slaving rho_{M-1} = rho - sum_a rho_a, j_{M-1} = j - sum_a j_a.
// Output layout: adj_mbar_rows(M) moment adjoints (see AdjBufs).
// ---------------------------------------------------------------------
template <int M>
struct PrimBar {
    double Y[M], rho_a[M], ja[M][3];
    double rho, u[3], T, Rm, inv_m, rhoE, q[3], P6[6];
};

template <int M>
__device__ __forceinline__ void prim_zero(PrimBar<M> &b)
{
#pragma unroll
    for (int s = 0; s < M; ++s) {
        b.Y[s] = b.rho_a[s] = 0.0;
        b.ja[s][0] = b.ja[s][1] = b.ja[s][2] = 0.0;
    }
    b.rho = b.T = b.Rm = b.inv_m = b.rhoE = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) b.u[d] = b.q[d] = 0.0;
#pragma unroll
    for (int d = 0; d < 6; ++d) b.P6[d] = 0.0;
}

template <int M>
__device__ void prim_to_moments(const MechConst &mc, double rho, const double u[3], const double *Y, double T,
                                double rhoE, PrimBar<M> &b, double *mb)
{
    b.inv_m = fma(mc.r_lat, b.Rm, b.inv_m);
#pragma unroll
    for (int s = 0; s < M; ++s) b.Y[s] = fma(b.inv_m, mc.invW[s], b.Y[s]);
    double Cv = 0.0, U[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        U[s] = poly5(mc.uco[s], T);
        Cv = fma(Y[s], dpoly5(mc.uco[s], T), Cv);
    }
    const double be = b.T / Cv, ir = 1.0 / rho;
#pragma unroll
    for (int s = 0; s < M; ++s) b.Y[s] -= be * U[s];
    b.rhoE += be * ir;
    b.rho -= be * rhoE * ir * ir;
    double bj[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        b.u[d] -= be * u[d];
        bj[d] = b.u[d] * ir;
        b.rho -= b.u[d] * u[d] * ir;
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
        b.rho_a[s] += b.Y[s] * ir;
        b.rho -= b.Y[s] * Y[s] * ir;
    }
    b.rho += b.rho_a[M - 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) bj[d] += b.ja[M - 1][d];
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        mb[s] = b.rho_a[s] - b.rho_a[M - 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) mb[M - 1 + 3 * s + d] = b.ja[s][d] - b.ja[M - 1][d];
    }
    const int o = 4 * (M - 1);
    mb[o] = b.rho;
#pragma unroll
    for (int d = 0; d < 3; ++d) mb[o + 1 + d] = bj[d];
#pragma unroll
    for (int d = 0; d < 6; ++d) mb[o + 4 + d] = b.P6[d];
    mb[o + 10] = b.rhoE;
#pragma unroll
    for (int d = 0; d < 3; ++d) mb[o + 11 + d] = b.q[d];
}

// ---------------------------------------------------------------------
// Pass A: adjoint of the collisions at one node.
// ---------------------------------------------------------------------
template <int M>
__device__ void adj_collide_node(const MechConst &mc, const StepArgs &a, const AdjBufs &g, int n, double *dA)
{
    const size_t N = a.N;
    Node nd;
    nd.n = n;
    node_at(nd, a);
    PullIdx p;
    make_pull(p, nd, a);
    const PopView v = view(a.src, a);
    double rho_a[M], ja[M][3];
    Sums sm;
    pull_moments<M, true>(mc, a, p, n, rho_a, ja, sm);
    const double rho = sm.rho, ir = 1.0 / rho;
    {
        double rest = 0.0, js[3] = {sm.j[0], sm.j[1], sm.j[2]};
#pragma unroll
        for (int s = 0; s < M - 1; ++s) {
            rest += rho_a[s];
#pragma unroll
            for (int d = 0; d < 3; ++d) js[d] -= ja[s][d];
        }
        rho_a[M - 1] = rho - rest;
#pragma unroll
        for (int d = 0; d < 3; ++d) ja[M - 1][d] = js[d];
    }
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = rho_a[s] * ir;
        inv_m = fma(Y[s], mc.invW[s], inv_m);
    }
    const double u[3] = {sm.j[0] * ir, sm.j[1] * ir, sm.j[2] * ir};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double T = a.macro[DR_T * N + n];                  // the record's Newton temperature
    const double Rm = mc.r_lat * inv_m, P = rho * Rm * T;
    const double nup = nu_prime(mc, Rm, T);
    const double om = 1.0 / (0.5 + nup), om1 = 1.0 / (0.5 + nup / mc.Pr);
    double Ha[M], H = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Ha[s] = H_spec(mc, s, T);
        H = fma(Y[s], Ha[s], H);
    }
    const double kappa = mc.r_lat * T / inv_m;
    double ita[M], beta[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < M; ++b)
            if (b != s) acc = fma(Y[b], mc.inv_WWD[s][b], acc);
        ita[s] = kappa * acc;
        beta[s] = ita[s] / (2.0 + ita[s]);
    }

    // Stefan-Maxwell system B du = r, B_aa = Y_a (1 + 1/(2 tau_a)),
    // B_ab = -(1/2) kappa Y_a Y_b / (W_a W_b D_ab), r_a = j_a / rho - Y_a u;
    // symmetric, factored L D L^T as in the forward pass.
    double Ln[M][M], Dinv[M], du[M][3];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const double hy = -0.5 * kappa * Y[i];
#pragma unroll
        for (int k = 0; k < i; ++k) Ln[i][k] = hy * mc.inv_WWD[i][k] * Y[k];
        Ln[i][i] = Y[i] * fma(0.5, ita[i], 1.0);
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        double Dk[M];
#pragma unroll
        for (int j = 0; j < k; ++j) Dk[j] = Ln[j][j] * Ln[k][j];
#pragma unroll
        for (int i = k; i < M; ++i) {
            double sacc = Ln[i][k];
#pragma unroll
            for (int j = 0; j < k; ++j) sacc = fma(-Ln[i][j], Dk[j], sacc);
            Ln[i][k] = sacc;
        }
        Dinv[k] = nonzero_bits(Ln[k][k]) ? 1.0 / Ln[k][k] : 0.0;
#pragma unroll
        for (int i = k + 1; i < M; ++i) Ln[i][k] *= Dinv[k];
    }
    // Ln[k][k] now holds D_k; solve B x = rhs for three right-hand sides
    auto ldl_solve = [&](double (*x)[3]) {
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double sacc = x[i][d];
#pragma unroll
                for (int j = 0; j < i; ++j) sacc = fma(-Ln[i][j], x[j][d], sacc);
                x[i][d] = sacc;
            }
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) x[i][d] *= Dinv[i];
#pragma unroll
        for (int i = M - 1; i >= 0; --i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double sacc = x[i][d];
#pragma unroll
                for (int j = i + 1; j < M; ++j) sacc = fma(-Ln[j][i], x[j][d], sacc);
                x[i][d] = sacc;
            }
    };
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) du[i][d] = fma(ja[i][d], ir, -Y[i] * u[d]);
    ldl_solve(du);

    double rdot[M];
    rates_d<M>(mc, T, rho_a, rdot);

    // neighbour fields: X = -d G (Eq. (Xalpha)), grad Y_a, sum_a H_a grad Y_a
    double X[3] = {0.0, 0.0, 0.0}, gY[M][3];
#pragma unroll
    for (int s = 0; s < M; ++s) gY[s][0] = gY[s][1] = gY[s][2] = 0.0;
    {
        const RecRows rr = rec_rows(M);
        const double *Rr = rec(a);
        StencilIdx st;
        make_stencil(st, nd, a);
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            if constexpr (I != REST) {
                const size_t nb = nb_of<I>(st, a);
                constexpr double wx = WI(I) * CX(I), wy = WI(I) * CY(I), wz = WI(I) * CZ(I);
                if (CX(I)) X[0] = fma(wx, Rr[(size_t)rr.g * N + nb], X[0]);
                if (CY(I)) X[1] = fma(wy, Rr[(size_t)(rr.g + 1) * N + nb], X[1]);
                if (CZ(I)) X[2] = fma(wz, Rr[(size_t)(rr.g + 2) * N + nb], X[2]);
#pragma unroll
                for (int s = 0; s < M; ++s) {
                    const double y = Rr[(size_t)(rr.y + s) * N + nb];
                    if (CX(I)) gY[s][0] = fma(wx, y, gY[s][0]);
                    if (CY(I)) gY[s][1] = fma(wy, y, gY[s][1]);
                    if (CZ(I)) gY[s][2] = fma(wz, y, gY[s][2]);
                }
            }
        });
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            X[d] *= -3.0;
#pragma unroll
            for (int s = 0; s < M; ++s) gY[s][d] *= 3.0;
        }
    }
    double HgY[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        HgY[d] = 0.0;
#pragma unroll
        for (int s = 0; s < M; ++s) HgY[d] = fma(Ha[s], gY[s][d], HgY[d]);
    }

    // energy equilibrium moments (Eqs. (geq1mom), (geq2mom)) and Dq
    const double hk = H + 0.5 * usq;
    double Peq[3][3], Req[3][3], qeq[3], Pt[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        qeq[d] = hk * rho * u[d];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            Peq[d][e] = (d == e ? P : 0.0) + rho * u[d] * u[e];
            Req[d][e] = hk * Peq[d][e] + P * u[d] * u[e];
        }
    }
    Pt[0][0] = sm.P[0]; Pt[1][1] = sm.P[1]; Pt[2][2] = sm.P[2];
    Pt[0][1] = Pt[1][0] = sm.P[3];
    Pt[0][2] = Pt[2][0] = sm.P[4];
    Pt[1][2] = Pt[2][1] = sm.P[5];
    double Aq[3], SHYdu[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        double uPd = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) uPd = fma(u[d], Pt[d][e] - Peq[d][e], uPd);
        Aq[e] = sm.q[e] - uPd - qeq[e];
        SHYdu[e] = 0.0;
#pragma unroll
        for (int s = 0; s < M; ++s) SHYdu[e] = fma(Ha[s] * Y[s], du[s][e], SHYdu[e]);
    }

    // ---------------- adjoint accumulators -----------------------------
    const double *Lm = g.lam_next;
    auto lam = [&](int s, int i) { return Lm[((size_t)s * LBMK_Q + i) * N + n]; };
    PrimBar<M> b;
    prim_zero(b);
    double bHa[M], bita[M], bdu[M][3], bz[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        bHa[s] = bita[s] = bz[s] = 0.0;
        bdu[s][0] = bdu[s][1] = bdu[s][2] = 0.0;
    }
    double bkappa = 0.0, bom = 0.0, bom1 = 0.0, bP = 0.0, bzm = 0.0;
    double bPt[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, bPeq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double bReq[3][3], bqeq[3], bDq[3], bX[3], bHgY[3];

    // ---- energy set: g' = (1 - omega) g + omega g^eq + 3 w_i c_i . Dq
    {
        double Lw = 0.0, Lc2 = 0.0, L1[3] = {0, 0, 0}, L2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const double trR = Req[0][0] + Req[1][1] + Req[2][2];
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            constexpr int c[3] = {CX(I), CY(I), CZ(I)};
            constexpr int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
            const double l = lam(M, I), gv = pull_g(v, a, I, p);
            double cq = 0.0, rcc = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cq += c[d] * qeq[d];
#pragma unroll
                for (int e = 0; e < 3; ++e) rcc += c[d] * c[e] * Req[d][e];
            }
            const double geq = WI(I) * (sm.rhoE * (2.5 - 1.5 * c2) + 3.0 * cq + 4.5 * rcc - 1.5 * trR);
            bom = fma(l, geq - gv, bom);
            const double lw = l * WI(I);
            Lw += lw;
            Lc2 += lw * c2;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                L1[d] += lw * c[d];
#pragma unroll
                for (int e = 0; e < 3; ++e) L2[d][e] += lw * (c[d] * c[e]);
            }
        });
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bDq[d] = 3.0 * L1[d];
            bqeq[d] = 3.0 * om * L1[d];
#pragma unroll
            for (int e = 0; e < 3; ++e) bReq[d][e] = 4.5 * om * (L2[d][e] - (d == e ? Lw / 3.0 : 0.0));
        }
        b.rhoE += om * (2.5 * Lw - 1.5 * Lc2);
    }
    // Dq = (omega - omega_1) Aq + omega_1 rho sum_a H_a Y_a du_a + (1/2)(2 - omega_1) P sum_a H_a grad Y_a
    {
        double dAq = 0.0, dS = 0.0, dH = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dAq = fma(bDq[d], Aq[d], dAq);
            dS = fma(bDq[d], SHYdu[d], dS);
            dH = fma(bDq[d], HgY[d], dH);
        }
        bom += dAq;
        bom1 += -dAq + rho * dS - 0.5 * P * dH;
        b.rho += om1 * dS;
        bP += 0.5 * (2.0 - om1) * dH;
        const double c1 = om - om1;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            b.q[e] += c1 * bDq[e];
            bqeq[e] -= c1 * bDq[e];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                b.u[d] -= c1 * bDq[e] * (Pt[d][e] - Peq[d][e]);
                bPt[d][e] -= c1 * u[d] * bDq[e];
                bPeq[d][e] += c1 * u[d] * bDq[e];
            }
        }
        const double orho = om1 * rho;
#pragma unroll
        for (int s = 0; s < M; ++s) {
            double sd = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sd = fma(bDq[d], du[s][d], sd);
                bdu[s][d] = fma(orho * Ha[s] * Y[s], bDq[d], bdu[s][d]);
            }
            bHa[s] += orho * Y[s] * sd;
            b.Y[s] += orho * Ha[s] * sd;
        }
        const double cc = 0.5 * (2.0 - om1) * P;
#pragma unroll
        for (int d = 0; d < 3; ++d) bHgY[d] = cc * bDq[d];
#pragma unroll
        for (int s = 0; s < M; ++s)
#pragma unroll
            for (int d = 0; d < 3; ++d) bHa[s] = fma(bHgY[d], gY[s][d], bHa[s]);
    }
    // R^eq = hk P^eq + P u u;  q^eq = hk rho u;  P^eq = P I + rho u u;  hk = H + |u|^2/2
    {
        double bhk = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                bhk = fma(bReq[d][e], Peq[d][e], bhk);
                bPeq[d][e] = fma(hk, bReq[d][e], bPeq[d][e]);
                bP = fma(bReq[d][e], u[d] * u[e], bP);
                b.u[d] += P * (bReq[d][e] + bReq[e][d]) * u[e];
            }
        double qu = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) qu = fma(bqeq[d], u[d], qu);
        bhk = fma(rho, qu, bhk);
        b.rho = fma(hk, qu, b.rho);
#pragma unroll
        for (int d = 0; d < 3; ++d) b.u[d] = fma(hk * rho, bqeq[d], b.u[d]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bP += bPeq[d][d];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                b.rho = fma(bPeq[d][e], u[d] * u[e], b.rho);
                b.u[d] += rho * (bPeq[d][e] + bPeq[e][d]) * u[e];
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) b.u[d] = fma(bhk, u[d], b.u[d]);
#pragma unroll
        for (int s = 0; s < M; ++s) {
            b.Y[s] = fma(bhk, Ha[s], b.Y[s]);
            bHa[s] = fma(bhk, Y[s], bHa[s]);
        }
    }

    // ---- mixture set: f' = f + omega (rho psi(u, R T) - f) + A_i . X
    {
        PsiTab tm;
        psi_tab(tm, u, Rm * T);
        double dv[3] = {0, 0, 0}, dz = 0.0, Sf = 0.0;
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            Sf = fma(lam(M - 1, I), pull_sf(mc, v, a, M - 1, I, p), Sf);
        });
        const double S = psi_adj(tm, [&](int i) { return lam(M - 1, i); }, dv, dz);
        bom += rho * S - Sf;
        b.rho = fma(om, S, b.rho);
#pragma unroll
        for (int d = 0; d < 3; ++d) b.u[d] = fma(om * rho, dv[d], b.u[d]);
        bzm = om * rho * dz;
        // A_i . X = c_i . X / 2 on the six directions with |c_i| = 1 (Eq. (Ai))
        bX[0] = 0.5 * (lam(M - 1, 14) - lam(M - 1, 12));
        bX[1] = 0.5 * (lam(M - 1, 16) - lam(M - 1, 10));
        bX[2] = 0.5 * (lam(M - 1, 22) - lam(M - 1, 4));
    }

    // ---- species sets a < M-1 (Eq. (finalNumericalEquations)):
    //   f' = f + 2 beta_a (rho_a psi(u, R_a T) - f) + (beta_a - 1) F_a + rho_dot_a psi(u, R_a T),
    //   F_ai = kappa Y_a sum_{b != a} D_bi / (W_a W_b D_ab),
    //   D_bi = rho_b (psi_i(u, R_b T) - psi_i(u + du_b, R_b T)).
    double sF[M];
#pragma unroll
    for (int s = 0; s < M; ++s) sF[s] = 0.0;
#pragma unroll 1
    for (int bb = 0; bb < M; ++bb) {
        const double zb = mc.Ra[bb] * T, rb = rho_a[bb];
        const double vb[3] = {u[0] + du[bb][0], u[1] + du[bb][1], u[2] + du[bb][2]};
        PsiTab te, ts;
        psi_tab(te, u, zb);
        psi_tab(ts, vb, zb);
        double Db[LBMK_Q], Dbar[LBMK_Q];
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            Db[I] = rb * (psi_at<I>(te) - psi_at<I>(ts));
            Dbar[I] = 0.0;
        });
#pragma unroll 1
        for (int s = 0; s < M - 1; ++s) {
            if (s == bb) continue;
            const double iw = mc.inv_WWD[s][bb];
            const double cab = kappa * Y[s] * iw * (beta[s] - 1.0);
            double tsum = 0.0;
            for_dirs<0, LBMK_Q>([&](auto dd) {
                constexpr int I = decltype(dd)::value;
                const double l = lam(s, I);
                tsum = fma(l, Db[I], tsum);
                Dbar[I] = fma(cab, l, Dbar[I]);
            });
            sF[s] = fma(iw, tsum, sF[s]);
        }
        double dve[3] = {0, 0, 0}, dze = 0.0, dvs[3] = {0, 0, 0}, dzs = 0.0;
        const double Se = psi_adj(te, [&](int i) { return Dbar[i]; }, dve, dze);
        const double Ss = psi_adj(ts, [&](int i) { return Dbar[i]; }, dvs, dzs);
        b.rho_a[bb] += Se - Ss;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            b.u[d] = fma(rb, dve[d] - dvs[d], b.u[d]);
            bdu[bb][d] = fma(-rb, dvs[d], bdu[bb][d]);
        }
        bz[bb] = fma(rb, dze - dzs, bz[bb]);
    }
    double bbeta[M], brdot[M];
#pragma unroll
    for (int s = 0; s < M; ++s) bbeta[s] = brdot[s] = 0.0;
#pragma unroll 1
    for (int s = 0; s < M - 1; ++s) {
        bkappa = fma((beta[s] - 1.0) * Y[s], sF[s], bkappa);
        b.Y[s] = fma((beta[s] - 1.0) * kappa, sF[s], b.Y[s]);
        PsiTab ta;
        psi_tab(ta, u, mc.Ra[s] * T);
        double dv[3] = {0, 0, 0}, dz = 0.0, Slf = 0.0;
        const double Sl = psi_adj(ta, [&](int i) { return lam(s, i); }, dv, dz);
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            Slf = fma(lam(s, I), pull_sf(mc, v, a, s, I, p), Slf);
        });
        bbeta[s] = 2.0 * (rho_a[s] * Sl - Slf) + kappa * Y[s] * sF[s];
        b.rho_a[s] = fma(2.0 * beta[s], Sl, b.rho_a[s]);
        brdot[s] = Sl;
        const double cw = fma(2.0 * beta[s], rho_a[s], rdot[s]);
#pragma unroll
        for (int d = 0; d < 3; ++d) b.u[d] = fma(cw, dv[d], b.u[d]);
        bz[s] = fma(cw, dz, bz[s]);
    }

    // ---- chemistry: sum_a adj(rho_dot_a) rho_dot_a (+ hdot^c of the objective)
    {
        double dTc, drc[M];
        weighted_progress<M>(mc, T, rho_a, brdot, g.with_objective != 0, &dTc, drc, dA, LBMK_ADJ_THREADS);
        b.T += dTc;
#pragma unroll
        for (int s = 0; s < M; ++s) b.rho_a[s] += drc[s];
    }
    // beta_a = (1/tau_a) / (2 + 1/tau_a)
#pragma unroll
    for (int s = 0; s < M - 1; ++s) bita[s] = fma(bbeta[s], 2.0 / ((2.0 + ita[s]) * (2.0 + ita[s])), bita[s]);

    // ---- Stefan-Maxwell: adj r = B^{-1} adj du (B symmetric), adj B = -adj r du^T
    {
        ldl_solve(bdu);                                // bdu now holds adj r
#pragma unroll
        for (int s = 0; s < M; ++s) {
#pragma unroll
            for (int t2 = 0; t2 < M; ++t2) {
                const double Bb = -(bdu[s][0] * du[t2][0] + bdu[s][1] * du[t2][1] + bdu[s][2] * du[t2][2]);
                if (s == t2) {
                    b.Y[s] = fma(Bb, fma(0.5, ita[s], 1.0), b.Y[s]);
                    bita[s] = fma(Bb, 0.5 * Y[s], bita[s]);
                } else {
                    const double val = -0.5 * Bb * mc.inv_WWD[s][t2];
                    bkappa = fma(val, Y[s] * Y[t2], bkappa);
                    b.Y[s] = fma(val * kappa, Y[t2], b.Y[s]);
                    b.Y[t2] = fma(val * kappa, Y[s], b.Y[t2]);
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                b.ja[s][d] = fma(bdu[s][d], ir, b.ja[s][d]);
                b.rho -= bdu[s][d] * ja[s][d] * ir * ir;
                b.Y[s] -= bdu[s][d] * u[d];
                b.u[d] -= bdu[s][d] * Y[s];
            }
        }
    }
    // 1/tau_a = kappa sum_{b != a} Y_b / (W_a W_b D_ab)
#pragma unroll
    for (int s = 0; s < M; ++s)
#pragma unroll
        for (int t2 = 0; t2 < M; ++t2)
            if (t2 != s) {
                bkappa = fma(bita[s] * Y[t2], mc.inv_WWD[s][t2], bkappa);
                b.Y[t2] = fma(bita[s] * kappa, mc.inv_WWD[s][t2], b.Y[t2]);
            }
    // omega, omega_1 from nu' (Eqs. (mu), (lambda))
    {
        const double bnup = -bom * om * om - bom1 * om1 * om1 / mc.Pr;
        if (mc.visc_model == 0) {                       // nu' = nu / (R T)
            b.Rm -= bnup * nup / Rm;
            b.T -= bnup * nup / T;
        }
    }
    // H_a(T), zeta_b = R_b T, zeta = R T, P = rho R T, kappa = r T / inv_m
#pragma unroll
    for (int s = 0; s < M; ++s) {
        b.T = fma(bHa[s], cp_spec(mc, s, T), b.T);
        b.T = fma(mc.Ra[s], bz[s], b.T);
    }
    b.T = fma(Rm, bzm, b.T);
    b.Rm = fma(T, bzm, b.Rm);
    b.rho = fma(bP, Rm * T, b.rho);
    b.Rm = fma(bP, rho * T, b.Rm);
    b.T = fma(bP, rho * Rm, b.T);
    b.T = fma(bkappa, kappa / T, b.T);
    b.inv_m -= bkappa * kappa / inv_m;
    // the pressure tensor's six entries (off-diagonal ones appear twice)
    b.P6[0] = bPt[0][0];
    b.P6[1] = bPt[1][1];
    b.P6[2] = bPt[2][2];
    b.P6[3] = bPt[0][1] + bPt[1][0];
    b.P6[4] = bPt[0][2] + bPt[2][0];
    b.P6[5] = bPt[1][2] + bPt[2][1];

    double mb[adj_mbar_rows(M)];
    prim_to_moments<M>(mc, rho, u, Y, T, sm.rhoE, b, mb);
#pragma unroll
    for (int r = 0; r < adj_mbar_rows(M); ++r) g.mbar[(size_t)r * N + n] = mb[r];
#pragma unroll
    for (int s = 0; s < M - 1; ++s) g.coef[(size_t)s * N + n] = 1.0 - 2.0 * beta[s];
    g.coef[(size_t)(M - 1) * N + n] = 1.0 - om;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        g.aux[(size_t)d * N + n] = bX[d];
        g.aux[(size_t)(3 + d) * N + n] = bHgY[d];
    }
}

template <int M>
__global__ void __launch_bounds__(LBMK_ADJ_THREADS) k_adj_collide(StepArgs a, AdjBufs g)
{
    __shared__ double sh_A[LBMK_MAXR * LBMK_ADJ_THREADS];
    const MechConst &mc = c_mech[a.slot];
    const int t = threadIdx.x, R = mc.R;
    for (int k = 0; k < R; ++k) sh_A[k * LBMK_ADJ_THREADS + t] = 0.0;
    const int n = blockIdx.x * LBMK_ADJ_THREADS + t;
    if (n < a.N) adj_collide_node<M>(mc, a, g, n, sh_A + t);
    __syncthreads();
    for (int w = LBMK_ADJ_THREADS / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < R; ++k) sh_A[k * LBMK_ADJ_THREADS + t] += sh_A[k * LBMK_ADJ_THREADS + t + w];
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < R; ++k) g.theta[(size_t)blockIdx.x * R + k] += sh_A[k * LBMK_ADJ_THREADS];
}

// ---------------------------------------------------------------------
// Pass B: X_d(x) = -3 sum_i w_i c_id G_d(x + c_i) transposes to
// adj G_d(y) = 3 sum_i w_i c_id adj X_d(y + c_i); G = nu' d Phi gives
// adj nu' = adj G . d Phi and the weight nu' adj G of the next stencil.
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_adj_grad1(StepArgs a, AdjBufs g)
{
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const RecRows rr = rec_rows(M);
    const double *Rr = rec(a);
    StencilIdx st;
    make_stencil(st, nd, a);
    double Gb[3] = {0, 0, 0}, dPhi[3] = {0, 0, 0};
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        if constexpr (I != REST) {
            const size_t nb = nb_of<I>(st, a);
            constexpr int c[3] = {CX(I), CY(I), CZ(I)};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (c[d]) {
                    Gb[d] = fma(WI(I) * c[d], g.aux[(size_t)d * N + nb], Gb[d]);
                    dPhi[d] = fma(WI(I) * c[d], Rr[(size_t)(rr.phi + d) * N + nb], dPhi[d]);
                }
        }
    });
    const double nup = Rr[(size_t)rr.nup * N + nd.n];
    double nub = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Gb[d] *= 3.0;
        nub = fma(Gb[d], 3.0 * dPhi[d], nub);
        g.aux[(size_t)(6 + d) * N + nd.n] = nup * Gb[d];
    }
    g.aux[(size_t)9 * N + nd.n] = nub;
}

// ---------------------------------------------------------------------
// Pass C: adj Phi_d(z) = -3 sum_i w_i c_id (nu' adj G_d)(z + c_i) and
// adj Y_a(z) = -3 sum_i w_i sum_d c_id adj(HgY)_d(z + c_i) H_a(z + c_i);
// Phi_d = rho u_d (1 - 3 R T) - rho u_d^3 and nu'(R, T) carried to the
// moments; then the adjoint of the pulled populations:
//   species a < M-1:  (1 - 2 beta_a) lam_ai + adj rho_a + c_i . adj j_a
//   mixture f:        (1 - omega) lam_i + adj rho + c_i . adj j + c_i c_i : adj P
//   energy g:         (1 - omega) lam_i + adj rho E + c_i . adj q
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_adj_finish(StepArgs a, AdjBufs g)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const int n = nd.n;
    const RecRows rr = rec_rows(M);
    const double *Rr = rec(a);
    StencilIdx st;
    make_stencil(st, nd, a);
    double Phib[3] = {0, 0, 0}, Yb[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Yb[s] = 0.0;
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        if constexpr (I != REST) {
            const size_t nb = nb_of<I>(st, a);
            constexpr int c[3] = {CX(I), CY(I), CZ(I)};
            double hg = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (c[d]) {
                    Phib[d] = fma(WI(I) * c[d], g.aux[(size_t)(6 + d) * N + nb], Phib[d]);
                    hg = fma((double)c[d], g.aux[(size_t)(3 + d) * N + nb], hg);
                }
            hg *= WI(I);
#pragma unroll
            for (int s = 0; s < M; ++s) Yb[s] = fma(hg, Rr[(size_t)(rr.h + s) * N + nb], Yb[s]);
        }
    });
    const double rho = Rr[(size_t)rr.rho * N + n];
    const double u[3] = {Rr[(size_t)rr.u * N + n], Rr[(size_t)(rr.u + 1) * N + n], Rr[(size_t)(rr.u + 2) * N + n]};
    const double T = a.macro[DR_T * N + n];
    const double rhoE = a.macro[(size_t)dr_ge(M) * N + n];
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = Rr[(size_t)(rr.y + s) * N + n];
        inv_m = fma(Y[s], mc.invW[s], inv_m);
    }
    const double Rm = mc.r_lat * inv_m;
    PrimBar<M> b;
    prim_zero(b);
#pragma unroll
    for (int s = 0; s < M; ++s) b.Y[s] = -3.0 * Yb[s];
    {
        double sPu = 0.0;
        const double RT3 = 1.0 - 3.0 * Rm * T;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double pb = -3.0 * Phib[d];
            b.rho = fma(pb, u[d] * (RT3 - u[d] * u[d]), b.rho);
            b.u[d] = fma(pb * rho, RT3 - 3.0 * u[d] * u[d], b.u[d]);
            sPu = fma(pb * rho, u[d], sPu);
        }
        b.Rm -= 3.0 * T * sPu;
        b.T -= 3.0 * Rm * sPu;
    }
    if (mc.visc_model == 0) {                           // nu' = nu / (R T)
        const double nup = Rr[(size_t)rr.nup * N + n], nub = g.aux[(size_t)9 * N + n];
        b.Rm -= nub * nup / Rm;
        b.T -= nub * nup / T;
    }
    double mb[adj_mbar_rows(M)];
    prim_to_moments<M>(mc, rho, u, Y, T, rhoE, b, mb);
#pragma unroll
    for (int r = 0; r < adj_mbar_rows(M); ++r) mb[r] += g.mbar[(size_t)r * N + n];
    const double *Lm = g.lam_next;
    const int o = 4 * (M - 1);
#pragma unroll 1
    for (int s = 0; s < M - 1; ++s) {
        const double cs = g.coef[(size_t)s * N + n];
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            const size_t k = ((size_t)s * LBMK_Q + I) * N + n;
            g.fbar[k] = fma(cs, Lm[k], mb[s] + CX(I) * mb[M - 1 + 3 * s] + CY(I) * mb[M + 3 * s] +
                                           CZ(I) * mb[M + 1 + 3 * s]);
        });
    }
    const double cm = g.coef[(size_t)(M - 1) * N + n];
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        constexpr int cx = CX(I), cy = CY(I), cz = CZ(I);
        const size_t kf = ((size_t)(M - 1) * LBMK_Q + I) * N + n, kg = ((size_t)M * LBMK_Q + I) * N + n;
        const double mf = mb[o] + cx * mb[o + 1] + cy * mb[o + 2] + cz * mb[o + 3] + (cx * cx) * mb[o + 4] +
                          (cy * cy) * mb[o + 5] + (cz * cz) * mb[o + 6] + (cx * cy) * mb[o + 7] +
                          (cx * cz) * mb[o + 8] + (cy * cz) * mb[o + 9];
        g.fbar[kf] = fma(cm, Lm[kf], mf);
        g.fbar[kg] = fma(cm, Lm[kg], mb[o + 10] + cx * mb[o + 11] + cy * mb[o + 12] + cz * mb[o + 13]);
    });
}

// Pass D: the pull P_si(x) = F_si(x - c_i) transposes to lam_si(y) = adj P_si(y + c_i).
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_adj_gather(StepArgs a, AdjBufs g)
{
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    StencilIdx st;
    make_stencil(st, nd, a);
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        const size_t nb = nb_of<I>(st, a);
#pragma unroll
        for (int s = 0; s <= M; ++s) g.lam[((size_t)s * LBMK_Q + I) * N + nd.n] = g.fbar[((size_t)s * LBMK_Q + I) * N + nb];
    });
}

// ---------------------------------------------------------------------
// dJ/dT(x, 0) from the adjoint lam0 of a state made by lbm_init with zero
// velocity: every set at its equilibrium (Eqs. (feq), (feqmix), (gieq)),
// rho_a = rho Y_a with rho = P / (R T) at fixed mole fractions and P, so
// d rho_a / dT = -rho_a / T, d (rho E) / dT = rho (C_v - U / T) and
// d R^eq / dT = C_p P I.  Reads the node's own populations (a.src).
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_adj_init_T(StepArgs a, const double *lam0, double *out)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const int n = nd.n;
    const double *F = static_cast<const double *>(a.src);
    double rho_a[M], rho = 0.0, rhoE = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        rho_a[s] = 0.0;
        for (int i = 0; i < LBMK_Q; ++i) rho_a[s] += F[((size_t)s * LBMK_Q + i) * N + n];
    }
    for (int i = 0; i < LBMK_Q; ++i) {
        rho += F[((size_t)(M - 1) * LBMK_Q + i) * N + n];
        rhoE += F[((size_t)M * LBMK_Q + i) * N + n];
    }
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) rest += rho_a[s];
    rho_a[M - 1] = rho - rest;
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = rho_a[s] / rho;
        inv_m = fma(Y[s], mc.invW[s], inv_m);
    }
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double T = solve_T(eu, rhoE / rho, a.macro[DR_T * N + n], a.status);
    const double Rm = mc.r_lat * inv_m, P = rho * Rm * T;
    double Cv = dpoly5(eu, T), U = poly5(eu, T), Cp = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) Cp = fma(Y[s], cp_spec(mc, s, T), Cp);
    const double u0[3] = {0.0, 0.0, 0.0};
    double acc = 0.0;
    auto lam = [&](int s, int i) { return lam0[((size_t)s * LBMK_Q + i) * N + n]; };
    for (int s = 0; s < M; ++s) {
        const double z = (s < M - 1 ? mc.Ra[s] : Rm) * T, r = s < M - 1 ? rho_a[s] : rho;
        const double dzdT = s < M - 1 ? mc.Ra[s] : Rm;
        PsiTab t;
        psi_tab(t, u0, z);
        double dv[3] = {0, 0, 0}, dz = 0.0;
        const double S = psi_adj(t, [&](int i) { return lam(s, i); }, dv, dz);
        acc += -r / T * S + r * dzdT * dz;
    }
    const double dE = rho * (Cv - U / T), dR = Cp * P;
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        constexpr int c2 = CX(I) * CX(I) + CY(I) * CY(I) + CZ(I) * CZ(I);
        acc += lam(M, I) * WI(I) * (dE * (2.5 - 1.5 * c2) + 4.5 * dR * (c2 - 1));
    });
    out[n] = acc;
}

// ---------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------
template <int M>
int run_adj_step(const StepArgs &a, const AdjBufs &g)
{
    k_adj_collide<M><<<adj_blocks(a.N), LBMK_ADJ_THREADS, 0, a.stream>>>(a, g);
    k_adj_grad1<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, g);
    k_adj_finish<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, g);
    k_adj_gather<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, g);
    return (int)cudaGetLastError();
}

template <int M>
int run_adj_init_T(const StepArgs &a, const double *lam0, double *out)
{
    k_adj_init_T<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, lam0, out);
    return (int)cudaGetLastError();
}

}  // namespace
