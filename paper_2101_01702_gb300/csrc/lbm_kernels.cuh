// Kernels of the fused reactive-mixture lattice Boltzmann step.
//
// Included once by each precision translation unit after it defines
//   LBMK_MIXED 0 : populations stored and collided in double;
//   LBMK_MIXED 1 : populations stored as float deviations from per-set rest
//                  states and collided in float; moments are accumulated in
//                  float and lifted to double with the rest-state moments.
// In both units the temperature iteration (Eq. (temperature)), the
// Stefan-Maxwell system (Eq. (transform1)) and the reaction rates with
// their equilibrium constants are double precision.
//
// One time step is four launches on one stream:
//   k_ghost  (x-face ghost nodes, Sec. 5a; only for non-periodic x)
//   k_pre    pull + moments + temperature + Phi and 1/omega - 1/2 (Eq. (Xalpha))
//   k_grad   G_alpha = (1/omega - 1/2) d_alpha Phi_alpha
//   k_step   pull + moments + X, grad Y, Stefan-Maxwell, chemistry and the
//            collisions of Eqs. (finalNumericalEquations), (f), (g)
// One thread owns one lattice node; populations are structure-of-arrays
// [set][direction][node] so a warp's pulls are coalesced rows.
#pragma once

#include <math.h>

#include "lbm_internal.h"

#if LBMK_MIXED
typedef float Store;
typedef float Real;
#else
typedef double Store;
typedef double Real;
#endif

#define LBMK_BLOCK 128
#if LBMK_MIXED
#define INVWWD(a_, b_) (mc.inv_WWD_f[a_][b_])
#else
#define INVWWD(a_, b_) (mc.inv_WWD[a_][b_])
#endif

static __constant__ MechConst c_mech[LBMK_SLOTS];

namespace {

// ---------------------------------------------------------------------
// Lattice helpers.  Direction i = (cx+1) + 3 (cy+1) + 9 (cz+1).
// ---------------------------------------------------------------------
__host__ __device__ constexpr int CX(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double W1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double WI(int i) { return W1(CX(i)) * W1(CY(i)) * W1(CZ(i)); }

struct Node {
    int n, x, y, z;
};

template <int I>
struct Dir {
    static constexpr int value = I;
};

// Compile-time loop over directions: f(Dir<0>{}), ..., f(Dir<N-1>{}).
template <int I, int N, class F>
__device__ __forceinline__ void for_dirs(F &&f)
{
    if constexpr (I < N) {
        f(Dir<I>{});
        for_dirs<I + 1, N>(f);
    }
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Source coordinates of the pull s(x) = s_post(x - c): index [c+1].
struct PullIdx {
    int xs[3];    // x - c for c = -1, 0, 1 (may be -1 or nx for ghosts)
    int row[9];   // nx * (y' + ny z') for (cy, cz)
    int yz[9];    // y' + ny z'
};

__device__ __forceinline__ void make_pull(PullIdx &p, const Node &nd, const StepArgs &a)
{
    for (int c = -1; c <= 1; ++c) {
        int xs = nd.x - c;
        if (a.bc_x == 0) xs = wrapi(xs, a.nx);
        p.xs[c + 1] = xs;
    }
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy) {
            int ys = wrapi(nd.y - cy, a.ny), zs = wrapi(nd.z - cz, a.nz);
            int yz = ys + a.ny * zs;
            p.yz[(cy + 1) + 3 * (cz + 1)] = yz;
            p.row[(cy + 1) + 3 * (cz + 1)] = a.nx * yz;
        }
}

// Stored value of set s, direction i pulled to this node.
template <int I>
__device__ __forceinline__ Store pull_raw(const Store *__restrict__ src, const Store *__restrict__ ghost,
                                          int s, int S, const PullIdx &p, const StepArgs &a)
{
    const int xs = p.xs[CX(I) + 1];
    const int k = (CY(I) + 1) + 3 * (CZ(I) + 1);
    if (CX(I) == 0 || a.bc_x == 0 || (xs >= 0 && xs < a.nx))
        return __ldg(src + (size_t)(s * LBMK_Q + I) * a.N + xs + p.row[k]);
    const int side = xs < 0 ? 0 : 1;
    const int plane = a.ny * a.nz;
    return __ldg(ghost + ((size_t)(side * S + s) * LBMK_Q + I) * plane + p.yz[k]);
}

// Stencil neighbour x + c (periodic, or clamped for zero-gradient x faces).
__device__ __forceinline__ int stencil_x(int x, int c, const StepArgs &a)
{
    int xn = x + c;
    if (a.bc_x == 0) return wrapi(xn, a.nx);
    return xn < 0 ? 0 : (xn >= a.nx ? a.nx - 1 : xn);
}

__device__ __forceinline__ void flag(const StepArgs &a, unsigned bit)
{
    atomicOr(a.status, bit);
}

// ---------------------------------------------------------------------
// Thermodynamics (Eqs. (specHa), (Umix), (temperature)).
// Mixture coefficients: U(T) = sum_k u[k] T^k (k = 0..5), C_v = dU/dT.
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void mixture_energy_poly(const MechConst &mc, const double *Y, double u[6])
{
    if (mc.thermo == 0) {
        // sum Y_a (U0_a + cv_a (T - T0))
        double B0 = 0.0, B1 = 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            B0 = fma(Y[a], mc.U0[a], B0);
            B1 = fma(Y[a], mc.cv[a], B1);
        }
        u[0] = B0 - B1 * mc.T0;
        u[1] = B1;
        u[2] = u[3] = u[4] = u[5] = 0.0;
    } else {
        // sum Y_a R_a [a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6 - T]
        double A[6] = {0, 0, 0, 0, 0, 0}, Rm = 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const double yr = Y[a] * mc.Ra[a];
            Rm += yr;
#pragma unroll
            for (int k = 0; k < 6; ++k) A[k] = fma(yr, mc.poly[a][k], A[k]);
        }
        u[0] = A[5];
        u[1] = A[0] - Rm;
        u[2] = A[1] * 0.5;
        u[3] = A[2] * (1.0 / 3.0);
        u[4] = A[3] * 0.25;
        u[5] = A[4] * 0.2;
    }
}

// Newton iteration on U(T) = e from T_guess; stops when |dT| <= 1e-13 T.
__device__ __forceinline__ double solve_T(const double u[6], double e, double T, const StepArgs &a)
{
    for (int it = 0; it < 50; ++it) {
        const double F = fma(fma(fma(fma(fma(u[5], T, u[4]), T, u[3]), T, u[2]), T, u[1]), T, u[0]) - e;
        const double Fp = fma(fma(fma(fma(5.0 * u[5], T, 4.0 * u[4]), T, 3.0 * u[3]), T, 2.0 * u[2]), T, u[1]);
        const double dT = F / Fp;
        T -= dT;
        if (!isfinite(T)) { flag(a, LBMK_BIT_NONFINITE); return T; }
        if (fabs(dT) <= 1e-13 * fabs(T)) return T;
    }
    flag(a, LBMK_BIT_NEWTON);
    return T;
}

// Species specific enthalpy H_a(T).
__device__ __forceinline__ double H_spec(const MechConst &mc, int a, double T)
{
    if (mc.thermo == 0) return mc.U0[a] + mc.cv[a] * (T - mc.T0) + mc.Ra[a] * T;
    const double *p = mc.poly[a];
    // R_a (a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a5 T^5/5 + a6)
    const double h = fma(fma(fma(fma(p[4] * 0.2, T, p[3] * 0.25), T, p[2] * (1.0 / 3.0)), T, p[1] * 0.5), T, p[0]);
    return mc.Ra[a] * fma(h, T, p[5]);
}

// Standard Gibbs energy over R_U T of species a.
__device__ __forceinline__ double gRT_spec(const MechConst &mc, int a, double T, double lnT)
{
    if (mc.thermo == 0) {
        const double h_RT = H_spec(mc, a, T) / (mc.Ra[a] * T);
        return h_RT - mc.cpR[a] * (lnT - log(mc.T0));
    }
    const double *p = mc.poly[a];
    const double h_RT = fma(fma(fma(fma(p[4] * 0.2, T, p[3] * 0.25), T, p[2] * (1.0 / 3.0)), T, p[1] * 0.5), T, p[0]) + p[5] / T;
    const double s_R = fma(p[0], lnT, fma(fma(fma(fma(p[4] * 0.25, T, p[3] * (1.0 / 3.0)), T, p[2] * 0.5), T, p[1]), T, p[6]));
    return h_RT - s_R;
}

__device__ __forceinline__ double nu_prime(const MechConst &mc, double Rm, double T)
{
    return mc.visc_model == 0 ? mc.nu / (Rm * T) : mc.nu;
}

// ---------------------------------------------------------------------
// Production rates rho_dot_a (Eq. (sumRhoDot)) of the mass-action
// mechanism.  Species-indexed scratch lives in shared memory, one column
// per thread, so the reaction tables can index it at run time.
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void production_rates(const MechConst &mc, const double *rho_a, double T,
                                                 double *wdot, double *sh)
{
    double *shc = sh;                         // concentrations
    double *shw = sh + M * LBMK_BLOCK;        // molar production
    double *shg = sh + 2 * M * LBMK_BLOCK;    // g_a / (R_U T)
    const int t = threadIdx.x;
    const double lnT = log(T), invT = 1.0 / T, lnTr = lnT - mc.log_T_ref;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        shc[a * LBMK_BLOCK + t] = rho_a[a] * mc.invW[a];
        shw[a * LBMK_BLOCK + t] = 0.0;
        shg[a * LBMK_BLOCK + t] = gRT_spec(mc, a, T, lnT);
    }
    const double lnc0 = mc.log_P0_over_r - lnT;     // ln(P0 / (r T))
    for (int k = 0; k < mc.R; ++k) {
        const double lk = mc.log_A[k] + mc.b[k] * lnTr - mc.theta[k] * invT;
        double kf = exp(lk);
        double cM = 0.0;
        const int type = mc.rtype[k];
        if (type != 0) {
#pragma unroll
            for (int a = 0; a < M; ++a) cM = fma(mc.eff[k][a], shc[a * LBMK_BLOCK + t], cM);
        }
        if (type == 2) {
            const double k0 = exp(mc.low[k][0] + mc.low[k][1] * lnTr - mc.low[k][2] * invT);
            const double Pr = k0 * cM / kf;
            kf = kf * Pr / (1.0 + Pr);
        }
        double qf = kf;
        for (int j = 0; j < mc.nreac[k]; ++j) qf *= shc[mc.reac[k][j] * LBMK_BLOCK + t];
        double q = qf;
        if (mc.rev[k]) {
            double dG = 0.0;
            for (int j = 0; j < mc.ndnu[k]; ++j) dG += mc.dnu_v[k][j] * shg[mc.dnu_sp[k][j] * LBMK_BLOCK + t];
            // k_r = k_f / K_c, K_c = exp(-dG) (P0/(r T))^dn
            double qr = kf * exp(dG - mc.dn[k] * lnc0);
            for (int j = 0; j < mc.nprod[k]; ++j) qr *= shc[mc.prod[k][j] * LBMK_BLOCK + t];
            q -= qr;
        }
        if (type == 1) q *= cM;
        for (int j = 0; j < mc.nreac[k]; ++j) shw[mc.reac[k][j] * LBMK_BLOCK + t] -= q;
        for (int j = 0; j < mc.nprod[k]; ++j) shw[mc.prod[k][j] * LBMK_BLOCK + t] += q;
    }
#pragma unroll
    for (int a = 0; a < M; ++a) wdot[a] = mc.W[a] * shw[a * LBMK_BLOCK + t];
}

// ---------------------------------------------------------------------
// Product-form factors (Eq. (phis)): P[c+1] = Psi_c(xi, zeta).
// ---------------------------------------------------------------------
__device__ __forceinline__ void psi3(Real xi, Real zeta, Real P[3])
{
    const Real s = xi * xi + zeta;
    P[0] = (Real)0.5 * (s - xi);
    P[1] = (Real)1 - s;
    P[2] = (Real)0.5 * (s + xi);
}

// Store a post-collision value (deviation from the rest state in mixed mode).
template <int I>
__device__ __forceinline__ void put(Store *__restrict__ dst, const MechConst &mc, int s, size_t N, int n, Real v)
{
#if LBMK_MIXED
    dst[(size_t)(s * LBMK_Q + I) * N + n] = v - mc.ref[s][I];
#else
    dst[(size_t)(s * LBMK_Q + I) * N + n] = v;
#endif
}

template <int I>
__device__ __forceinline__ Real absval(const MechConst &mc, int s, Store v)
{
#if LBMK_MIXED
    return v + mc.ref[s][I];
#else
    return v;
#endif
}

// Equilibrium populations of every set at (rho_a, u, T); written as the
// stored representation to out[(s*27+i)*stride + off].
template <int M>
__device__ void write_equilibria(const MechConst &mc, const double *rho_a, const double *u, double T,
                                 Store *out, size_t stride, size_t off)
{
    double rho = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) rho += rho_a[a];
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) { Y[a] = rho_a[a] / rho; inv_m += Y[a] * mc.invW[a]; }
    const double Rm = mc.r_lat * inv_m;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const Real zeta = (Real)((s < M - 1 ? mc.Ra[s] : Rm) * T);
        const Real r = (Real)(s < M - 1 ? rho_a[s] : rho);
        Real Px[3], Py[3], Pz[3];
        psi3((Real)u[0], zeta, Px);
        psi3((Real)u[1], zeta, Py);
        psi3((Real)u[2], zeta, Pz);
#pragma unroll
        for (int i = 0; i < LBMK_Q; ++i) {
            Real v = r * Px[CX(i) + 1] * Py[CY(i) + 1] * Pz[CZ(i) + 1];
#if LBMK_MIXED
            v -= mc.ref[s][i];
#endif
            out[(size_t)(s * LBMK_Q + i) * stride + off] = v;
        }
    }
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double U = fma(fma(fma(fma(fma(eu[5], T, eu[4]), T, eu[3]), T, eu[2]), T, eu[1]), T, eu[0]);
    double H = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) H = fma(Y[a], H_spec(mc, a, T), H);
    const double rhoE = rho * (U + 0.5 * usq);
    const double P = rho * Rm * T;
    const double hk = H + 0.5 * usq;
    double R[3][3];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be)
            R[al][be] = hk * ((al == be ? P : 0.0) + rho * u[al] * u[be]) + P * u[al] * u[be];
    const double tr3 = (R[0][0] + R[1][1] + R[2][2] - rhoE) * (1.0 / 3.0);   // tr(R - rhoE theta I)/3
#pragma unroll
    for (int i = 0; i < LBMK_Q; ++i) {
        const int cx = CX(i), cy = CY(i), cz = CZ(i);
        const double qc = hk * rho * (u[0] * cx + u[1] * cy + u[2] * cz);
        const double rcc = (R[0][0] - rhoE / 3.0) * (cx * cx) + (R[1][1] - rhoE / 3.0) * (cy * cy) +
                           (R[2][2] - rhoE / 3.0) * (cz * cz) +
                           2.0 * (R[0][1] * (cx * cy) + R[0][2] * (cx * cz) + R[1][2] * (cy * cz));
        Real v = (Real)(WI(i) * (rhoE + 3.0 * qc + 4.5 * (rcc - tr3)));
#if LBMK_MIXED
        v -= mc.ref[M][i];
#endif
        out[(size_t)(M * LBMK_Q + i) * stride + off] = v;
    }
}

__device__ __forceinline__ bool node_of(Node &nd, const StepArgs &a)
{
    nd.n = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd.n >= a.N) return false;
    nd.x = nd.n % a.nx;
    const int r = nd.n / a.nx;
    nd.y = r % a.ny;
    nd.z = r / a.ny;
    return true;
}

// ---------------------------------------------------------------------
// Initialisation: every set at equilibrium for X, T, u and pressure P.
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_init(StepArgs a, const double *X, const double *Tf,
                                                     const double *uf, double P)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    const int n = nd.n;
    double m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) m += X[(size_t)s * a.N + n] * mc.W[s];
    const double T = Tf[n];
    const double rho = P / (mc.r_lat / m * T);
    double rho_a[M];
#pragma unroll
    for (int s = 0; s < M; ++s) rho_a[s] = rho * X[(size_t)s * a.N + n] * mc.W[s] / m;
    double u[3] = {0.0, 0.0, 0.0};
    if (uf)
        for (int d = 0; d < 3; ++d) u[d] = uf[(size_t)d * a.N + n];
    write_equilibria<M>(mc, rho_a, u, T, (Store *)a.dst, a.N, n);
    a.macro[(size_t)MAC_T * a.N + n] = T;
}

// ---------------------------------------------------------------------
// Ghost nodes beyond the x faces (Sec. 5a).
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_ghost(StepArgs a)
{
    const MechConst &mc = c_mech[a.slot];
    const int plane = a.ny * a.nz;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * plane) return;
    const int side = t / plane, yz = t % plane;
    const int n = (side ? a.nx - 1 : 0) + a.nx * yz;
    const Store *src = (const Store *)a.src;
    double rho_a[M], rho = 0.0, j[3] = {0, 0, 0}, rhoE = 0.0;
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        Real acc = 0;
#pragma unroll
        for (int i = 0; i < LBMK_Q; ++i) acc += src[(size_t)(s * LBMK_Q + i) * a.N + n];
        rho_a[s] = (double)acc;
#if LBMK_MIXED
        rho_a[s] += mc.ref_m0[s];
#endif
        rest += rho_a[s];
    }
    {
        Real a0 = 0, ax = 0, ay = 0, az = 0, ag = 0;
#pragma unroll
        for (int i = 0; i < LBMK_Q; ++i) {
            const Real f = src[(size_t)((M - 1) * LBMK_Q + i) * a.N + n];
            a0 += f;
            if (CX(i)) ax += CX(i) * f;
            if (CY(i)) ay += CY(i) * f;
            if (CZ(i)) az += CZ(i) * f;
            ag += src[(size_t)(M * LBMK_Q + i) * a.N + n];
        }
        rho = (double)a0;
        rhoE = (double)ag;
#if LBMK_MIXED
        rho += mc.ref_m0[M - 1];
        rhoE += mc.ref_m0[M];
#endif
        j[0] = ax; j[1] = ay; j[2] = az;
    }
    rho_a[M - 1] = rho - rest;
    double Y[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Y[s] = rho_a[s] / rho;
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    const double e = rhoE / rho - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double T = solve_T(eu, e, a.macro[(size_t)MAC_T * a.N + n], a);
    if (side == 0) u[0] = u[1] = u[2] = 0.0;
    write_equilibria<M>(mc, rho_a, u, T, (Store *)a.ghost + (size_t)side * (M + 1) * LBMK_Q * plane, plane, yz);
}

// ---------------------------------------------------------------------
// Pass 1: pull, moments, temperature, Phi, 1/omega - 1/2.  With OUT the
// requested fields go to `out` instead of the macroscopic record.
// ---------------------------------------------------------------------
template <int M, bool OUT>
__global__ void __launch_bounds__(LBMK_BLOCK) k_pre(StepArgs a, unsigned mask, double *out)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    PullIdx p;
    make_pull(p, nd, a);
    const Store *src = (const Store *)a.src;
    const Store *gh = (const Store *)a.ghost;
    constexpr int S = M + 1;
    double rho_a[M], ja[M][3];
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        Real a0 = 0, ax = 0, ay = 0, az = 0;
        for_dirs<0, LBMK_Q>([&](auto d) {
            constexpr int I = decltype(d)::value;
            const Real f = pull_raw<I>(src, gh, s, S, p, a);
            a0 += f;
            if (CX(I)) ax += CX(I) * f;
            if (CY(I)) ay += CY(I) * f;
            if (CZ(I)) az += CZ(I) * f;
        });
        rho_a[s] = (double)a0;
#if LBMK_MIXED
        rho_a[s] += mc.ref_m0[s];
#endif
        ja[s][0] = ax; ja[s][1] = ay; ja[s][2] = az;
        rest += rho_a[s];
    }
    double rho, j[3], rhoE;
    {
        Real a0 = 0, ax = 0, ay = 0, az = 0, ag = 0;
        for_dirs<0, LBMK_Q>([&](auto d) {
            constexpr int I = decltype(d)::value;
            const Real f = pull_raw<I>(src, gh, M - 1, S, p, a);
            const Real g = pull_raw<I>(src, gh, M, S, p, a);
            a0 += f;
            ag += g;
            if (CX(I)) ax += CX(I) * f;
            if (CY(I)) ay += CY(I) * f;
            if (CZ(I)) az += CZ(I) * f;
        });
        rho = (double)a0;
        rhoE = (double)ag;
#if LBMK_MIXED
        rho += mc.ref_m0[M - 1];
        rhoE += mc.ref_m0[M];
#endif
        j[0] = ax; j[1] = ay; j[2] = az;
    }
    rho_a[M - 1] = rho - rest;
    double Y[M], inv_m = 0.0;
    bool neg = false;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = rho_a[s] / rho;
        inv_m += Y[s] * mc.invW[s];
        neg |= rho_a[s] < -1e-10 * rho;      // below rounding noise of trace species
    }
    if (!(rho > 0.0) || !isfinite(rhoE)) flag(a, LBMK_BIT_NONFINITE);
    if (neg) flag(a, LBMK_BIT_NEGATIVE);
    const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const int n = nd.n;
    const size_t N = a.N;
    const double T = solve_T(eu, rhoE / rho - 0.5 * usq, a.macro[MAC_T * N + n], a);
    const double Rm = mc.r_lat * inv_m;
    if (!OUT) {
        a.macro[MAC_T * N + n] = T;
        a.macro[MAC_NUP * N + n] = nu_prime(mc, Rm, T);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            a.macro[(MAC_PHI + d) * N + n] = rho * u[d] * (1.0 - 3.0 * Rm * T) - rho * u[d] * u[d] * u[d];
#pragma unroll
        for (int s = 0; s < M; ++s) a.macro[(MAC_Y + s) * N + n] = Y[s];
    } else {
        size_t row = 0;
        if (mask & 1u) { for (int s = 0; s < M; ++s) out[(row + s) * N + n] = rho_a[s]; row += M; }
        if (mask & 2u) { for (int d = 0; d < 3; ++d) out[(row + d) * N + n] = j[d]; row += 3; }
        if (mask & 4u) { out[row * N + n] = rhoE; row += 1; }
        if (mask & 8u) { out[row * N + n] = T; row += 1; }
        if (mask & 16u) { out[row * N + n] = rho * Rm * T; row += 1; }
        if (mask & 32u) { for (int s = 0; s < M; ++s) out[(row + s) * N + n] = Y[s]; row += M; }
        if (mask & 64u) {
            double jM[3] = {j[0], j[1], j[2]};
            for (int s = 0; s < M - 1; ++s)
                for (int d = 0; d < 3; ++d) { out[(row + 3 * s + d) * N + n] = ja[s][d]; jM[d] -= ja[s][d]; }
            for (int d = 0; d < 3; ++d) out[(row + 3 * (M - 1) + d) * N + n] = jM[d];
        }
    }
}

// ---------------------------------------------------------------------
// Pass 2: G_alpha = (1/omega - 1/2) d_alpha Phi_alpha with the isotropic
// gradient d_alpha phi = (1/theta) sum_i w_i c_ia phi(x + c_i).
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(LBMK_BLOCK) k_grad(StepArgs a)
{
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const double *Phi = a.macro + MAC_PHI * N;
    double d[3] = {0.0, 0.0, 0.0};
    int xs[3], rows[9];
    for (int c = -1; c <= 1; ++c) xs[c + 1] = stencil_x(nd.x, c, a);
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            rows[(cy + 1) + 3 * (cz + 1)] = a.nx * (wrapi(nd.y + cy, a.ny) + a.ny * wrapi(nd.z + cz, a.nz));
#pragma unroll
    for (int i = 0; i < LBMK_Q; ++i) {
        const size_t nb = xs[CX(i) + 1] + rows[(CY(i) + 1) + 3 * (CZ(i) + 1)];
        if (CX(i)) d[0] += (WI(i) * CX(i)) * Phi[nb];
        if (CY(i)) d[1] += (WI(i) * CY(i)) * Phi[N + nb];
        if (CZ(i)) d[2] += (WI(i) * CZ(i)) * Phi[2 * N + nb];
    }
    const double nup = a.macro[MAC_NUP * N + nd.n];
#pragma unroll
    for (int k = 0; k < 3; ++k) a.macro[(MAC_G + k) * N + nd.n] = nup * 3.0 * d[k];
}

// ---------------------------------------------------------------------
// Pass 3: the fused collision.
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_step(StepArgs a)
{
    __shared__ double sh_chem[3 * M * LBMK_BLOCK];
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    const bool live = node_of(nd, a);
    if (!live) return;
    const int n = nd.n;
    const size_t N = a.N;
    const double T = a.macro[MAC_T * N + n];

    // species enthalpies at T (Eq. (specHa))
    double Ha[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Ha[s] = H_spec(mc, s, T);

    // X = -d_alpha G_alpha (Eq. (Xalpha)) and sum_a H_a grad Y_a (Eq. (corrFourier))
    double X[3] = {0, 0, 0}, HgY[3] = {0, 0, 0};
    {
        int xs[3], rows[9];
        for (int c = -1; c <= 1; ++c) xs[c + 1] = stencil_x(nd.x, c, a);
        for (int cz = -1; cz <= 1; ++cz)
            for (int cy = -1; cy <= 1; ++cy)
                rows[(cy + 1) + 3 * (cz + 1)] = a.nx * (wrapi(nd.y + cy, a.ny) + a.ny * wrapi(nd.z + cz, a.nz));
        const double *G = a.macro + MAC_G * N;
        const double *Yf = a.macro + MAC_Y * N;
#pragma unroll
        for (int i = 0; i < LBMK_Q; ++i) {
            if (i == 13) continue;
            const size_t nb = xs[CX(i) + 1] + rows[(CY(i) + 1) + 3 * (CZ(i) + 1)];
            double hy = 0.0;
#pragma unroll
            for (int s = 0; s < M; ++s) hy = fma(Ha[s], Yf[s * N + nb], hy);
            if (CX(i)) { X[0] += (WI(i) * CX(i)) * G[nb]; HgY[0] += (WI(i) * CX(i)) * hy; }
            if (CY(i)) { X[1] += (WI(i) * CY(i)) * G[N + nb]; HgY[1] += (WI(i) * CY(i)) * hy; }
            if (CZ(i)) { X[2] += (WI(i) * CZ(i)) * G[2 * N + nb]; HgY[2] += (WI(i) * CZ(i)) * hy; }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) { X[k] *= -3.0; HgY[k] *= 3.0; }
    }

    PullIdx p;
    make_pull(p, nd, a);
    const Store *src = (const Store *)a.src;
    const Store *gh = (const Store *)a.ghost;
    Store *dst = (Store *)a.dst;
    constexpr int S = M + 1;

    // sweep 1: moments of the pulled populations
    double rho_a[M], ja[M][3];
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        Real a0 = 0, ax = 0, ay = 0, az = 0;
        for_dirs<0, LBMK_Q>([&](auto d) {
            constexpr int I = decltype(d)::value;
            const Real f = pull_raw<I>(src, gh, s, S, p, a);
            a0 += f;
            if (CX(I)) ax += CX(I) * f;
            if (CY(I)) ay += CY(I) * f;
            if (CZ(I)) az += CZ(I) * f;
        });
        rho_a[s] = (double)a0;
#if LBMK_MIXED
        rho_a[s] += mc.ref_m0[s];
#endif
        ja[s][0] = ax; ja[s][1] = ay; ja[s][2] = az;
        rest += rho_a[s];
    }
    double rho, j[3], rhoE, q[3], Pt[6];   // Pt: xx, yy, zz, xy, xz, yz
    {
        Real a0 = 0, ax = 0, ay = 0, az = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
        Real g0 = 0, qx = 0, qy = 0, qz = 0;
        for_dirs<0, LBMK_Q>([&](auto d) {
            constexpr int I = decltype(d)::value;
            const Real f = pull_raw<I>(src, gh, M - 1, S, p, a);
            const Real g = pull_raw<I>(src, gh, M, S, p, a);
            a0 += f;
            g0 += g;
            if (CX(I)) { ax += CX(I) * f; pxx += f; qx += CX(I) * g; }
            if (CY(I)) { ay += CY(I) * f; pyy += f; qy += CY(I) * g; }
            if (CZ(I)) { az += CZ(I) * f; pzz += f; qz += CZ(I) * g; }
            if (CX(I) && CY(I)) pxy += (CX(I) * CY(I)) * f;
            if (CX(I) && CZ(I)) pxz += (CX(I) * CZ(I)) * f;
            if (CY(I) && CZ(I)) pyz += (CY(I) * CZ(I)) * f;
        });
        rho = (double)a0;
        rhoE = (double)g0;
        Pt[0] = pxx; Pt[1] = pyy; Pt[2] = pzz;
#if LBMK_MIXED
        rho += mc.ref_m0[M - 1];
        rhoE += mc.ref_m0[M];
        Pt[0] += mc.ref_m2[M - 1]; Pt[1] += mc.ref_m2[M - 1]; Pt[2] += mc.ref_m2[M - 1];
#endif
        Pt[3] = pxy; Pt[4] = pxz; Pt[5] = pyz;
        j[0] = ax; j[1] = ay; j[2] = az;
        q[0] = qx; q[1] = qy; q[2] = qz;
    }
    rho_a[M - 1] = rho - rest;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double js = j[d];
#pragma unroll
        for (int s = 0; s < M - 1; ++s) js -= ja[s][d];
        ja[M - 1][d] = js;
    }
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) { Y[s] = rho_a[s] / rho; inv_m += Y[s] * mc.invW[s]; }
    const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double m = 1.0 / inv_m;
    const double Rm = mc.r_lat * inv_m;
    const double P = rho * Rm * T;
    const double nup = nu_prime(mc, Rm, T);
    const double omega = 1.0 / (0.5 + nup);
    const double omega1 = 1.0 / (0.5 + nup / mc.Pr);

    // Eq. (tauab): 1/tau_ab = kappa / (W_a W_b D_ab), kappa = m R_U T
    const double kappa = m * mc.r_lat * T;
    double ita[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < M; ++b)
            if (b != s) acc = fma(Y[b], mc.inv_WWD[s][b], acc);
        ita[s] = kappa * acc;
    }

    // Eq. (transform1): Gaussian elimination (the matrix is strictly
    // diagonally dominant, so no pivoting), three right-hand sides.
    double du[M][3];
    {
        double A[M][M], rhs[M][3];
#pragma unroll
        for (int s = 0; s < M; ++s) {
#pragma unroll
            for (int b = 0; b < M; ++b)
                A[s][b] = (s == b) ? 1.0 + 0.5 * ita[s] : -0.5 * kappa * mc.inv_WWD[s][b] * Y[b];
            const double ir = 1.0 / rho_a[s];
#pragma unroll
            for (int d = 0; d < 3; ++d) rhs[s][d] = ja[s][d] * ir - u[d];
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            if (A[k][k] == 0.0) flag(a, LBMK_BIT_PIVOT);
            const double ip = 1.0 / A[k][k];
#pragma unroll
            for (int r = k + 1; r < M; ++r) {
                const double l = A[r][k] * ip;
#pragma unroll
                for (int c = k + 1; c < M; ++c) A[r][c] = fma(-l, A[k][c], A[r][c]);
#pragma unroll
                for (int d = 0; d < 3; ++d) rhs[r][d] = fma(-l, rhs[k][d], rhs[r][d]);
            }
        }
#pragma unroll
        for (int r = M - 1; r >= 0; --r) {
            const double ip = 1.0 / A[r][r];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double acc = rhs[r][d];
#pragma unroll
                for (int c = r + 1; c < M; ++c) acc = fma(-A[r][c], du[c][d], acc);
                du[r][d] = acc * ip;
            }
        }
    }

    // chemistry
    double wdot[M];
    production_rates<M>(mc, rho_a, T, wdot, sh_chem);

    // energy: q^eq, R^eq and the regularised quasi-equilibrium flux change
    // Dq = (omega - omega_1)(q^* - q^eq) (Eqs. (gstareq1mom), (qdiff), (corrFourier))
    double H = 0.0, HYdu[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < M; ++s) {
        H = fma(Y[s], Ha[s], H);
#pragma unroll
        for (int d = 0; d < 3; ++d) HYdu[d] = fma(Ha[s] * Y[s], du[s][d], HYdu[d]);
    }
    const double hk = H + 0.5 * usq;
    double qeq[3], Dq[3];
    {
        double Peq[6] = {P + rho * u[0] * u[0], P + rho * u[1] * u[1], P + rho * u[2] * u[2],
                         rho * u[0] * u[1], rho * u[0] * u[2], rho * u[1] * u[2]};
        double dP[3][3];
        dP[0][0] = Pt[0] - Peq[0]; dP[1][1] = Pt[1] - Peq[1]; dP[2][2] = Pt[2] - Peq[2];
        dP[0][1] = dP[1][0] = Pt[3] - Peq[3];
        dP[0][2] = dP[2][0] = Pt[4] - Peq[4];
        dP[1][2] = dP[2][1] = Pt[5] - Peq[5];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            qeq[b] = hk * rho * u[b];
            const double uP = u[0] * dP[0][b] + u[1] * dP[1][b] + u[2] * dP[2][b];
            Dq[b] = (omega - omega1) * (q[b] - uP - qeq[b]) + omega1 * rho * HYdu[b] +
                    0.5 * (2.0 - omega1) * P * HgY[b];
        }
    }
    // R^eq - rhoE theta I
    const double Rt[6] = {hk * (P + rho * u[0] * u[0]) + P * u[0] * u[0] - rhoE / 3.0,
                          hk * (P + rho * u[1] * u[1]) + P * u[1] * u[1] - rhoE / 3.0,
                          hk * (P + rho * u[2] * u[2]) + P * u[2] * u[2] - rhoE / 3.0,
                          (hk * rho + P) * u[0] * u[1], (hk * rho + P) * u[0] * u[2], (hk * rho + P) * u[1] * u[2]};
    const double tr3 = (Rt[0] + Rt[1] + Rt[2]) * (1.0 / 3.0);

    // sweep 2: collisions, direction by direction
    Real Pe[M][3][3], Ps[M][3][3];
    Real rhoR[M], KY[M], b2[M], bm1[M], wd[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const Real zeta = (Real)(mc.Ra[s] * T);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            psi3((Real)u[d], zeta, Pe[s][d]);
            psi3((Real)(u[d] + du[s][d]), zeta, Ps[s][d]);
        }
        rhoR[s] = (Real)rho_a[s];
        KY[s] = (Real)(kappa * Y[s]);
        const double beta = ita[s] / (2.0 + ita[s]);          // 1/(2 tau_a + 1), Eq. (fStar)
        b2[s] = (Real)(2.0 * beta);
        bm1[s] = (Real)(beta - 1.0);
        wd[s] = (Real)wdot[s];
    }
    Real Pm[3][3];
    {
        const Real zeta = (Real)(Rm * T);
        for (int d = 0; d < 3; ++d) psi3((Real)u[d], zeta, Pm[d]);
    }
    const Real om = (Real)omega, rhoRl = (Real)rho;
    const Real Xr[3] = {(Real)X[0], (Real)X[1], (Real)X[2]};
    const Real gE = (Real)rhoE, gq[3] = {(Real)qeq[0], (Real)qeq[1], (Real)qeq[2]};
    const Real gD[3] = {(Real)Dq[0], (Real)Dq[1], (Real)Dq[2]};
    const Real gR[6] = {(Real)Rt[0], (Real)Rt[1], (Real)Rt[2], (Real)Rt[3], (Real)Rt[4], (Real)Rt[5]};
    const Real gtr = (Real)tr3;
    Real check = 0;

    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        constexpr int ix = CX(I) + 1, iy = CY(I) + 1, iz = CZ(I) + 1;
        Real eqp[M], Dl[M];
#pragma unroll
        for (int s = 0; s < M; ++s) {
            eqp[s] = Pe[s][0][ix] * Pe[s][1][iy] * Pe[s][2][iz];
            Dl[s] = rhoR[s] * (eqp[s] - Ps[s][0][ix] * Ps[s][1][iy] * Ps[s][2][iz]);
        }
        Real fv[S];
#pragma unroll
        for (int s = 0; s < S; ++s) fv[s] = absval<I>(mc, s, pull_raw<I>(src, gh, s, S, p, a));
        Real outv[S];
#pragma unroll
        for (int s = 0; s < M - 1; ++s) {
            Real F = 0;
#pragma unroll
            for (int b = 0; b < M; ++b)
                if (b != s) F += INVWWD(s, b) * Dl[b];
            F *= KY[s];
            const Real feq = rhoR[s] * eqp[s];
            const Real f = fv[s];
            outv[s] = f + b2[s] * (feq - f) + bm1[s] * F + wd[s] * eqp[s];
        }
        {
            const Real feq = rhoRl * Pm[0][ix] * Pm[1][iy] * Pm[2][iz];
            Real AX = 0;
            if (CX(I) * CX(I) + CY(I) * CY(I) + CZ(I) * CZ(I) == 1)
                AX = (Real)0.5 * (CX(I) * Xr[0] + CY(I) * Xr[1] + CZ(I) * Xr[2]);
            outv[M - 1] = fv[M - 1] + om * (feq - fv[M - 1]) + AX;
        }
        {
            const Real qc = CX(I) * gq[0] + CY(I) * gq[1] + CZ(I) * gq[2];
            const Real rcc = gR[0] * (CX(I) * CX(I)) + gR[1] * (CY(I) * CY(I)) + gR[2] * (CZ(I) * CZ(I)) +
                             (Real)2 * (gR[3] * (CX(I) * CY(I)) + gR[4] * (CX(I) * CZ(I)) + gR[5] * (CY(I) * CZ(I)));
            constexpr Real wi = (Real)WI(I);
            const Real geq = wi * (gE + (Real)3 * qc + (Real)4.5 * (rcc - gtr));
            const Real dq = CX(I) * gD[0] + CY(I) * gD[1] + CZ(I) * gD[2];
            outv[M] = fv[M] + om * (geq - fv[M]) + (Real)3 * wi * dq;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            put<I>(dst, mc, s, N, n, outv[s]);
            check += outv[s];
        }
    });
    if (!isfinite(check)) flag(a, LBMK_BIT_NONFINITE);
}

// ---------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------
inline dim3 grid_for(int n) { return dim3((unsigned)((n + LBMK_BLOCK - 1) / LBMK_BLOCK)); }

template <int M>
int run_step(const StepArgs &a, cudaEvent_t *ev)
{
    if (ev) cudaEventRecord(ev[0], a.stream);
    if (a.bc_x == 1) {
        const int plane = a.ny * a.nz;
        k_ghost<M><<<grid_for(2 * plane), LBMK_BLOCK, 0, a.stream>>>(a);
    }
    if (ev) cudaEventRecord(ev[1], a.stream);
    k_pre<M, false><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, 0u, nullptr);
    if (ev) cudaEventRecord(ev[2], a.stream);
    k_grad<<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a);
    if (ev) cudaEventRecord(ev[3], a.stream);
    k_step<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a);
    if (ev) cudaEventRecord(ev[4], a.stream);
    return (int)cudaGetLastError();
}

template <int M>
int run_moments(const StepArgs &a, unsigned mask, double *out)
{
    if (a.bc_x == 1) {
        const int plane = a.ny * a.nz;
        k_ghost<M><<<grid_for(2 * plane), LBMK_BLOCK, 0, a.stream>>>(a);
    }
    k_pre<M, true><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, mask, out);
    return (int)cudaGetLastError();
}

template <int M>
int run_init(const StepArgs &a, const double *X, const double *T, const double *u, double P)
{
    k_init<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, X, T, u, P);
    return (int)cudaGetLastError();
}

}  // namespace

#define LBMK_DISPATCH(M_, CALL)                     \
    switch (M_) {                                   \
    case 2: return CALL(2);                         \
    case 3: return CALL(3);                         \
    case 9: return CALL(9);                         \
    default: return (int)cudaErrorInvalidValue;     \
    }
