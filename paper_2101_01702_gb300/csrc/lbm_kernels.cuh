// Kernels of the fused reactive-mixture lattice Boltzmann step.
//
// Included once by each precision translation unit after it defines
//   LBMK_MIXED 0 : every population stored and collided in double;
//   LBMK_MIXED 1 : the moving populations of the species and mixture sets
//                  stored as float deviations from per-set rest states and
//                  collided in float; their rest populations and the whole
//                  energy set in double (see pop_bytes_for);
//   LBMK_FAST 1  : (with LBMK_MIXED 1) also the relaxation rates, the
//                  Stefan-Maxwell solve and the 2^f of the rate
//                  exponentials in float (see SReal, WReal, exp_rate).
// Otherwise the moments, the temperature iteration (Eq. (temperature)),
// the Stefan-Maxwell system (Eq. (transform1)) and the reaction rates with
// their equilibrium constants are double precision in every unit.
//
// One time step is four launches on one stream (five with x ghosts):
//   k_ghost  x-face ghost nodes (Sec. 5a; only for non-periodic x)
//   k_pre    pull, all moments, Newton temperature, relaxation rates,
//            Stefan-Maxwell diffusion velocities, the local part of the
//            energy-flux correction and the energy equilibrium moments;
//            writes the per-node record.
//   k_grad   G_alpha = (1/omega - 1/2) d_alpha Phi_alpha (Eq. (Xalpha))
//   k_step_g pull of the energy set, sum_a H_a grad Y_a from the neighbours'
//            records, and the collision of Eq. (g) (double)
//   k_step   production rates of the reaction mechanism at the node
//            (double), pull of the species and mixture sets,
//            X = -d_alpha G_alpha from the neighbours' records, and the
//            collisions of Eqs. (finalNumericalEquations), (f), direction
//            by direction
// (k_chem, the production rates as a kernel of their own writing record
// rows, serves builds with LBMK_FUSE_CHEM=0.)
// One thread owns one lattice node; populations are structure-of-arrays
// [set][direction][node] so that a warp's pulls are coalesced rows.
#pragma once

#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "lbm_internal.h"

#ifndef LBMK_FAST
#define LBMK_FAST 0
#endif
// LBMK_CHECKED 1: every index the kernels derive from the lattice geometry
// (pulls from neighbours and ghost planes, stencil neighbours, ghost-node
// sources, batch ranges) is checked against its buffer before use; a bad one
// sets LBMK_BIT_BOUNDS in the status word and is replaced by 0, so that
// nothing traps and no access leaves its buffer.  A testing build.
#ifndef LBMK_CHECKED
#define LBMK_CHECKED 0
#endif

#if LBMK_MIXED
typedef float Real;
#else
typedef double Real;
#endif
// SReal: the relaxation rates, the Stefan-Maxwell factorisation and solve
// and the diffusion part of the energy-flux correction; WReal: the
// accumulation of the reaction contributions.  Double except in the fast
// mixed unit (LBMK_FAST), where these results, stored as floats, are also
// computed in float.
#if LBMK_MIXED && LBMK_FAST
typedef float SReal;
typedef float WReal;
#define INVWWD_S(a_, b_) (mc.inv_WWD_f[a_][b_])
#else
typedef double SReal;
typedef double WReal;
#define INVWWD_S(a_, b_) (mc.inv_WWD[a_][b_])
#endif

// Minimum resident blocks per SM asked of the compiler for the two large
// kernels (register budget 65536 / (LBMK_BLOCK * minB)).  Measured on the
// 256^3 nine-species lattice: the moment pass runs fastest at 5 blocks in
// the fast mixed unit (96 registers, some spilled; latency bound) and at 3
// in the double unit; with its double Stefan-Maxwell solve the mixed unit
// is FP64-bound and nearly insensitive to it (1..5 within 1.4 %, 3 best,
// with the fewest spills of the capped choices).  The species and mixture
// collision runs fastest at 3 blocks in the mixed units (168 registers) and
// unconstrained in the double unit; with the production rates inside it,
// 256^3 mixed: 38.1 ms at 2 blocks (234 registers), 29.5 ms at 3, 31.2 ms
// at 4 (128 registers, 224 B spilled).
#ifndef LBMK_PRE_MINB
#define LBMK_PRE_MINB (LBMK_MIXED && LBMK_FAST ? 5 : 3)
#endif
#ifndef LBMK_STEP_MINB
#define LBMK_STEP_MINB (LBMK_MIXED ? 3 : 1)
#endif
// The moments of lbm_moments (outside the step), 256^3 mixed, T and Y:
// 44.0 ms at 178 registers (2 blocks per SM), 29.3 ms at 4 blocks, 23.8 ms
// at 5 (96 registers, ~200 B spilled); the double unit stays unconstrained
// (a cap of 128 registers spills 600 B there).
#ifndef LBMK_MOM_MINB
#define LBMK_MOM_MINB (LBMK_MIXED ? 5 : 1)
#endif
// Initialisation (equilibria of every set, outside the step; FP64-bound and
// insensitive to occupancy: 43.1-43.5 ms at 4 or 6 blocks per SM): 6 blocks
// (80 registers, ~30 B spilled).
// Production rates formed inside the species collision (k_step) instead of
// a kernel of their own: in the mixed units k_step waits on memory with
// the FP64 pipe idle, and the rates are FP64 work of the same node, so the
// fused kernel overlaps the two (256^3 mixed: k_chem 24.6 ms + k_step
// 11.9 ms -> 29.5 ms; double: 24.0 + 257.7 -> 274.7 ms).  Results are bit
// for bit those of the separate kernels (LBMK_FUSE_CHEM=0).
#ifndef LBMK_FUSE_CHEM
#define LBMK_FUSE_CHEM 1
#endif
// The energy collision inside k_step as well (LBMK_FUSE_ENERGY=1) was
// measured slower (256^3 mixed: species collision 29.5 + energy 4.0 ms ->
// 47.0 ms fused, with more spills at k_step's 168 registers), so k_step_g
// stays a kernel of its own.
#ifndef LBMK_FUSE_ENERGY
#define LBMK_FUSE_ENERGY 0
#endif
#ifndef LBMK_INIT_MINB
#define LBMK_INIT_MINB 6
#endif
#if LBMK_MIXED
#define INVWWD(a_, b_) (mc.inv_WWD_f[a_][b_])
#define RA(a_) (mc.Ra_f[a_])
#else
#define INVWWD(a_, b_) (mc.inv_WWD[a_][b_])
#define RA(a_) (mc.Ra[a_])
#endif

static __constant__ MechConst c_mech[LBMK_SLOTS];

namespace {

// ---------------------------------------------------------------------
// Lattice helpers.  Direction i = (cx+1) + 3 (cy+1) + 9 (cz+1); 13 = rest.
// ---------------------------------------------------------------------
__host__ __device__ constexpr int CX(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double W1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double WI(int i) { return W1(CX(i)) * W1(CY(i)) * W1(CZ(i)); }
constexpr int REST = 13;

// A lattice node and the x range [x0, x1) of the lattice it belongs to
// (lattice k of a batch placed side by side in x).
struct Node {
    int n, x, y, z;
    int x0, x1, k;
};

template <int I>
struct Dir {
    static constexpr int value = I;
};

// Compile-time loop over directions: f(Dir<I>{}), ..., f(Dir<N-1>{}).
template <int I, int N, class F>
__device__ __forceinline__ void for_dirs(F &&f)
{
    if constexpr (I < N) {
        f(Dir<I>{});
        for_dirs<I + 1, N>(f);
    }
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void flag(unsigned *status, unsigned bit) { atomicOr(status, bit); }

// Tests on the bit pattern (integer pipe; the FP64 pipe is the step's
// bottleneck): not Inf or NaN, and not +-0.
__device__ __forceinline__ bool finite_bits(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool finite_bits(float x) { return (__float_as_int(x) & 0x7f800000) != 0x7f800000; }
__device__ __forceinline__ bool nonzero_bits(double x)
{
    return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) != 0;
}
__device__ __forceinline__ bool nonzero_bits(float x) { return (__float_as_int(x) & 0x7fffffff) != 0; }

// Conversions between float and double on the integer pipe.  A hardware
// conversion between the two issues on the FP64 pipe, which bounds the
// moment pass; these give the same IEEE 754 result (binary32 <-> binary64,
// double -> float rounded to nearest, ties to even) with integer
// operations for zeros and normal results.  A warp with a lane outside
// that range (subnormals, overflow, Inf, NaN: rare here) takes the
// hardware conversion for all its lanes; the test is a warp vote, so the
// branch is uniform and the common path issues no FP64 instruction.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f), mag = b & 0x7fffffffu;
    const bool rare = (mag >> 23) - 1u >= 254u && mag != 0u;            // subnormal, Inf, NaN
    if (__builtin_expect(__any_sync(__activemask(), rare), 0)) return (double)f;
    // exponent rebiased by 1023 - 127 = 896; the low 3 mantissa bits move to the low word
    const unsigned hi = (b & 0x80000000u) | (mag ? (mag >> 3) + (896u << 20) : 0u);
    return __hiloint2double((int)hi, (int)(mag << 29));
}

__device__ __forceinline__ float d2f(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned hm = hi & 0x7fffffffu;
    const bool zero = (hm | lo) == 0u;
    // normal float results: biased double exponent in [897, 1150]
    const bool rare = (hm >> 20) - 897u > 253u && !zero;
    if (__builtin_expect(__any_sync(__activemask(), rare), 0)) return __double2float_rn(d);
    const unsigned m = ((hm - (896u << 20)) << 3) | (lo >> 29);     // float exponent and mantissa, truncated
    const unsigned rem = lo & 0x1fffffffu;                          // the 29 bits dropped
    const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & m);
    return __uint_as_float((hi & 0x80000000u) | (zero ? 0u : m + up));   // a carry rounds into the exponent
}

// x converted to To (a plain copy when the types agree).
template <class To, class From>
__device__ __forceinline__ To cvt(From x)
{
    if constexpr (std::is_same<To, From>::value) return x;
    else if constexpr (std::is_same<To, double>::value && std::is_same<From, float>::value) return f2d(x);
    else if constexpr (std::is_same<To, float>::value && std::is_same<From, double>::value) return d2f(x);
    else return (To)x;
}

// Checked builds: records a failed index check; always true otherwise.
__device__ __forceinline__ bool index_ok(bool ok, unsigned *status)
{
#if LBMK_CHECKED
    if (!ok) flag(status, LBMK_BIT_BOUNDS);
    return ok;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}

// Populations and ghost planes are read through the read-only data path
// (__ldg) in the per-phase kernels, none of which reads what it writes.
// The persistent kernel writes, within its one launch, what its later
// phases read, so its units build with LBMK_COHERENT_LOADS=1: plain loads,
// ordered by the grid barrier's fences.
#ifndef LBMK_COHERENT_LOADS
#define LBMK_COHERENT_LOADS 0
#endif
#if LBMK_COHERENT_LOADS
#define LBMK_LDG(p_) (*(p_))
#else
#define LBMK_LDG(p_) __ldg(p_)
#endif

// ---------------------------------------------------------------------
// Population storage (see pop_bytes_for).
// ---------------------------------------------------------------------
struct PopView {
    const void *buf;
    int N, M;
#if LBMK_MIXED
    __device__ const float *mov() const { return static_cast<const float *>(buf); }
    __device__ const double *rest() const
    {
        return reinterpret_cast<const double *>(static_cast<const char *>(buf) + pop_float_bytes(M, N));
    }
    __device__ const double *g() const { return rest() + (size_t)M * N; }
#endif
};

__device__ __forceinline__ PopView view(const void *buf, const StepArgs &a) { return PopView{buf, a.N, a.M}; }

// Value of species/mixture set s (< M), direction i, at buffer node idx;
// absolute (the rest state is added back in mixed precision).
__device__ __forceinline__ Real load_sf(const MechConst &mc, const PopView &v, int s, int i, size_t idx)
{
#if LBMK_MIXED
    if (i == REST) return (Real)v.rest()[(size_t)s * v.N + idx];
    return LBMK_LDG(v.mov() + ((size_t)s * LBMK_Q + i) * v.N + idx) + mc.ref[s][i];
#else
    return LBMK_LDG(static_cast<const double *>(v.buf) + ((size_t)s * LBMK_Q + i) * v.N + idx);
#endif
}

// Stored value of species/mixture set s (< M), moving direction i, at
// buffer node idx: in mixed precision the deviation from the rest state
// RAWREF(s, i); the population is the stored value + RAWREF(s, i).
__device__ __forceinline__ Real load_raw_sf(const PopView &v, int s, int i, size_t idx)
{
#if LBMK_MIXED
    return LBMK_LDG(v.mov() + ((size_t)s * LBMK_Q + i) * v.N + idx);
#else
    return LBMK_LDG(static_cast<const double *>(v.buf) + ((size_t)s * LBMK_Q + i) * v.N + idx);
#endif
}
#if LBMK_MIXED
#define RAWREF(s_, i_) (mc.ref[s_][i_])
#else
#define RAWREF(s_, i_) ((Real)0)
#endif

// The same in double, keeping the double rest population exact.
__device__ __forceinline__ double load_sf_d(const MechConst &mc, const PopView &v, int s, int i, size_t idx)
{
#if LBMK_MIXED
    if (i == REST) return v.rest()[(size_t)s * v.N + idx];
#endif
    return (double)load_sf(mc, v, s, i, idx);
}

// Energy-set value, direction i, at buffer node idx (double in both precisions).
__device__ __forceinline__ double load_g(const PopView &v, int i, size_t idx)
{
#if LBMK_MIXED
    return LBMK_LDG(v.g() + (size_t)i * v.N + idx);
#else
    return LBMK_LDG(static_cast<const double *>(v.buf) + ((size_t)v.M * LBMK_Q + i) * v.N + idx);
#endif
}

// Where a pulled population comes from: s(x) = s_post(x - c).
struct PullIdx {
    int xs[3];    // x - c for c = -1, 0, 1
    int gp[3];    // ghost plane of x - c (2k left, 2k+1 right face of lattice k), -1 inside
    int yz[9];    // y' + ny z' for (cy, cz)
};

__device__ __forceinline__ void make_pull(PullIdx &p, const Node &nd, const StepArgs &a)
{
    for (int c = -1; c <= 1; ++c) {
        int xs = nd.x - c, gp = -1;
        if (a.bc_x == 0) xs = wrapi(xs, a.nx);
        else if (xs < nd.x0) gp = 2 * nd.k;
        else if (xs >= nd.x1) gp = 2 * nd.k + 1;
        p.xs[c + 1] = xs;
        p.gp[c + 1] = gp;
    }
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            p.yz[(cy + 1) + 3 * (cz + 1)] = wrapi(nd.y - cy, a.ny) + a.ny * wrapi(nd.z - cz, a.nz);
}

// Source of direction i: a buffer node, or (ghost plane, index in the plane).
struct Src {
    bool ghost;
    int side;     // ghost plane (see PullIdx::gp)
    size_t idx;
};

__device__ __forceinline__ Src src_of(int i, const PullIdx &p, const StepArgs &a)
{
    const int xs = p.xs[CX(i) + 1];
    const int gp = p.gp[CX(i) + 1];
    const int yz = p.yz[(CY(i) + 1) + 3 * (CZ(i) + 1)];
    if (gp >= 0) {
        const int nlat = a.nseg > 1 ? a.nseg : 1;
        if (!index_ok(gp < 2 * nlat && yz >= 0 && yz < a.ny * a.nz, a.status)) return Src{false, 0, 0};
        return Src{true, gp, (size_t)yz};
    }
    const size_t idx = (size_t)xs + (size_t)a.nx * yz;
    if (!index_ok(xs >= 0 && xs < a.nx && yz >= 0 && idx < (size_t)a.N, a.status)) return Src{false, 0, 0};
    return Src{false, 0, idx};
}

__device__ __forceinline__ double load_ghost(const StepArgs &a, int plane_idx, int s, int i, size_t yz)
{
    const size_t plane = (size_t)a.ny * a.nz;
    return LBMK_LDG(static_cast<const double *>(a.ghost) + ((size_t)(plane_idx * (a.M + 1) + s) * LBMK_Q + i) * plane +
                 yz);
}

__device__ __forceinline__ Real pull_sf(const MechConst &mc, const PopView &v, const StepArgs &a, int s, int i,
                                        const PullIdx &p)
{
    const Src sr = src_of(i, p, a);
    return sr.ghost ? (Real)load_ghost(a, sr.side, s, i, sr.idx) : load_sf(mc, v, s, i, sr.idx);
}

__device__ __forceinline__ double pull_g(const PopView &v, const StepArgs &a, int i, const PullIdx &p)
{
    const Src sr = src_of(i, p, a);
    return sr.ghost ? load_ghost(a, sr.side, a.M, i, sr.idx) : load_g(v, i, sr.idx);
}

// Writers of the post-collision state at node n.  store_raw writes the
// stored value of a moving population of a species/mixture set: in the
// mixed units its deviation from the rest state RAWREF(s, i), in double
// the population; store_sf takes an absolute double value, any direction.
__device__ __forceinline__ void store_raw(void *buf, const StepArgs &a, int s, int i, size_t n, Real v)
{
    static_cast<Real *>(buf)[((size_t)s * LBMK_Q + i) * a.N + n] = v;
}

__device__ __forceinline__ void store_sf(const MechConst &mc, void *buf, const StepArgs &a, int s, int i, size_t n,
                                         double v)
{
#if LBMK_MIXED
    const size_t N = a.N;
    if (i == REST) {
        reinterpret_cast<double *>(static_cast<char *>(buf) + pop_float_bytes(a.M, N))[(size_t)s * N + n] = v;
    } else {
        static_cast<float *>(buf)[((size_t)s * LBMK_Q + i) * N + n] = cvt<float>(v) - mc.ref[s][i];
    }
#else
    static_cast<double *>(buf)[((size_t)s * LBMK_Q + i) * a.N + n] = v;
#endif
}

__device__ __forceinline__ void store_g(void *buf, const StepArgs &a, int i, size_t n, double v)
{
#if LBMK_MIXED
    const size_t N = a.N;
    reinterpret_cast<double *>(static_cast<char *>(buf) + pop_float_bytes(a.M, N))[(size_t)a.M * N + (size_t)i * N + n] = v;
#else
    static_cast<double *>(buf)[((size_t)a.M * LBMK_Q + i) * a.N + n] = v;
#endif
}

// Stencil neighbours x + c (periodic, or clamped to the node's own lattice
// for zero-gradient x faces).
struct StencilIdx {
    int xs[3];
    int row[9];
};

__device__ __forceinline__ void make_stencil(StencilIdx &t, const Node &nd, const StepArgs &a)
{
    for (int c = -1; c <= 1; ++c) {
        int xn = nd.x + c;
        if (a.bc_x == 0) xn = wrapi(xn, a.nx);
        else xn = xn < nd.x0 ? nd.x0 : (xn >= nd.x1 ? nd.x1 - 1 : xn);
        t.xs[c + 1] = xn;
    }
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            t.row[(cy + 1) + 3 * (cz + 1)] = a.nx * (wrapi(nd.y + cy, a.ny) + a.ny * wrapi(nd.z + cz, a.nz));
}

template <int I>
__device__ __forceinline__ size_t nb_of(const StencilIdx &t, const StepArgs &a)
{
    const size_t nb = (size_t)t.xs[CX(I) + 1] + t.row[(CY(I) + 1) + 3 * (CZ(I) + 1)];
    return index_ok(nb < (size_t)a.N, a.status) ? nb : 0;
}

__device__ __forceinline__ Real *rec(const StepArgs &a)
{
    return reinterpret_cast<Real *>(a.macro + (size_t)macro_double_rows(a.M) * a.N);
}

// ---------------------------------------------------------------------
// Thermodynamics (Eqs. (specHa), (Umix), (temperature)).
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void mixture_energy_poly(const MechConst &mc, const double *Y, double u[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) u[k] = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int k = 0; k < 6; ++k) u[k] = fma(Y[a], mc.uco[a][k], u[k]);
}

__device__ __forceinline__ double poly5(const double u[6], double T)
{
    return fma(fma(fma(fma(fma(u[5], T, u[4]), T, u[3]), T, u[2]), T, u[1]), T, u[0]);
}

__device__ __forceinline__ double dpoly5(const double u[6], double T)
{
    return fma(fma(fma(fma(5.0 * u[5], T, 4.0 * u[4]), T, 3.0 * u[3]), T, 2.0 * u[2]), T, u[1]);
}

// Newton iteration on U(T) = e from T.  It stops once a correction is at
// most 1e-7 T: Newton's error after that step is about (C_v'/2C_v) dT^2,
// below 1e-13 T for these polynomials (C_v'/C_v is of order 1/T), so the
// further iteration a 1e-13 test would take changes T by less than that.
__device__ __forceinline__ double solve_T(const double u[6], double e, double T, unsigned *status)
{
    const double d5 = 5.0 * u[5], d4 = 4.0 * u[4], d3 = 3.0 * u[3], d2 = 2.0 * u[2];   // C_v's coefficients
    for (int it = 0; it < 50; ++it) {
        const double F = poly5(u, T) - e;
        const double Fp = fma(fma(fma(fma(d5, T, d4), T, d3), T, d2), T, u[1]);
        const double dT = F / Fp;
        T -= dT;
        if (!finite_bits(T)) { flag(status, LBMK_BIT_NONFINITE); return T; }
        if (fabs(dT) <= 1e-7 * fabs(T)) return T;
    }
    flag(status, LBMK_BIT_NEWTON);
    return T;
}

// Species specific enthalpy H_a(T).
__device__ __forceinline__ double H_spec(const MechConst &mc, int a, double T)
{
    const double *h = mc.hco[a];
    return fma(fma(fma(fma(fma(h[4], T, h[3]), T, h[2]), T, h[1]), T, h[0]), T, h[5]);
}

// Specific heat C_p,a(T) = dH_a/dT.
__device__ __forceinline__ double cp_spec(const MechConst &mc, int a, double T)
{
    const double *h = mc.hco[a];
    return fma(fma(fma(fma(5.0 * h[4], T, 4.0 * h[3]), T, 3.0 * h[2]), T, 2.0 * h[1]), T, h[0]);
}

__device__ __forceinline__ double nu_prime(const MechConst &mc, double Rm, double T)
{
    return mc.visc_model == 0 ? mc.nu / (Rm * T) : mc.nu;
}

// Mixture-averaged transport of a node state (mc.transport = 1; Sec. 3
// after Eq. (lambda), where the paper takes the coefficients from Cantera):
// species viscosities mu_a = mu0_a (T/T_tr)^s_a, Wilke's mixing rule
//   mu = sum_a X_a mu_a / sum_b X_b Phi_ab,
//   Phi_ab = (1 + (mu_a/mu_b)^(1/2) (W_b/W_a)^(1/4))^2 / (8 (1 + W_a/W_b))^(1/2),
// Eucken's lambda_a = mu_a (C_p,a + 5/4 R_a) with the average of Mathur,
// Tondon and Saxena lambda = (sum X_a lambda_a + 1/sum X_a/lambda_a)/2;
// returns 1/omega - 1/2 = mu/P (Eq. (mu)), 1/omega_1 - 1/2 = lambda/(P C_p)
// (Eq. (lambda)) in the storage type, and the factor dfac =
// (T/T_tr)^D_exp P_tr/P of every binary diffusivity (Eq. (tauab)).
template <int M>
__device__ void mixture_transport(const MechConst &mc, const double *Y, double inv_m, double T, double P,
                                  double Cp, Real &nup, Real &nup1, double &dfac)
{
    const double lnT = log(T) - mc.log_T_tr;
    const Real iim = (Real)(1.0 / inv_m);
    Real X[M], mu[M], r[M], ir[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        X[a] = (Real)(Y[a] * mc.invW[a]) * iim;
        mu[a] = (Real)mc.mu0[a] * exp((Real)(mc.mu_exp[a] * lnT));
        r[a] = sqrt(mu[a]);
        ir[a] = (Real)1 / r[a];
    }
    Real num = 0, ls = 0, lr = 0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
        Real den = 0;
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const Real t = fma(r[a] * ir[b], (Real)mc.wq[a][b], (Real)1);
            den = fma(X[b], t * t * (Real)mc.wd[a][b], den);
        }
        num += X[a] * mu[a] / den;
        const Real lam = mu[a] * (Real)(cp_spec(mc, a, T) + mc.eucken[a]);
        ls = fma(X[a], lam, ls);
        lr += X[a] / lam;
    }
    const Real lambda = (Real)0.5 * (ls + (Real)1 / lr);
    nup = num / (Real)P;
    nup1 = lambda / (Real)(P * Cp);
    dfac = exp(mc.D_exp * lnT) * mc.P_tr / P;
}

// Product-form factor Psi_c(xi, zeta) of Eq. (phis) with s = xi^2 + zeta.
template <class V>
__device__ __forceinline__ V psi_c(int c, V xi, V s)
{
    return c == 0 ? (V)1 - s : (V)0.5 * (s + (V)c * xi);
}

// Energy equilibrium moments (Eqs. (geq1mom), (geq2mom)): q^eq, R^eq -
// rhoE theta I (xx yy zz xy xz yz) and a third of its trace.
__device__ __forceinline__ void energy_moments(double rho, const double *u, double P, double hk, double rhoE,
                                               double qeq[3], double Rt[6], double &tr3)
{
    const double hP = hk * rho + P;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        qeq[d] = hk * rho * u[d];
        Rt[d] = hk * P + hP * u[d] * u[d] - rhoE / 3.0;
    }
    Rt[3] = hP * u[0] * u[1];
    Rt[4] = hP * u[0] * u[2];
    Rt[5] = hP * u[1] * u[2];
    tr3 = (Rt[0] + Rt[1] + Rt[2]) * (1.0 / 3.0);
}

// Grad population of direction i (Eqs. (gieq), (giqeq)) for given moments.
__device__ __forceinline__ double grad_dir(int i, double rhoE, const double q[3], const double Rt[6], double tr3)
{
    const int cx = CX(i), cy = CY(i), cz = CZ(i);
    double qc = 0.0, rcc = 0.0;
    if (cx) { qc += cx * q[0]; rcc += Rt[0]; }
    if (cy) { qc += cy * q[1]; rcc += Rt[1]; }
    if (cz) { qc += cz * q[2]; rcc += Rt[2]; }
    if (cx && cy) rcc += 2.0 * (cx * cy) * Rt[3];
    if (cx && cz) rcc += 2.0 * (cx * cz) * Rt[4];
    if (cy && cz) rcc += 2.0 * (cy * cz) * Rt[5];
    return WI(i) * (rhoE + 3.0 * qc + 4.5 * (rcc - tr3));
}

// Equilibrium of every set at (rho_a, u, T), in double, handed to put(s, i, v).
template <int M, class Put>
__device__ void equilibria(const MechConst &mc, const double *rho_a, const double *u, double T, Put &&put)
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
        const double zeta = (s < M - 1 ? mc.Ra[s] : Rm) * T;
        const double r = s < M - 1 ? rho_a[s] : rho;
        double P3[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int c = -1; c <= 1; ++c) P3[d][c + 1] = psi_c(c, u[d], u[d] * u[d] + zeta);
#pragma unroll
        for (int i = 0; i < LBMK_Q; ++i) put(s, i, r * P3[0][CX(i) + 1] * P3[1][CY(i) + 1] * P3[2][CZ(i) + 1]);
    }
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double U = poly5(eu, T);
    double H = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) H = fma(Y[a], H_spec(mc, a, T), H);
    const double rhoE = rho * (U + 0.5 * usq);
    const double P = rho * Rm * T;
    double q[3], Rt[6], tr3;
    energy_moments(rho, u, P, H + 0.5 * usq, rhoE, q, Rt, tr3);
#pragma unroll
    for (int i = 0; i < LBMK_Q; ++i) put(M, i, grad_dir(i, rhoE, q, Rt, tr3));
}

// Coordinates and lattice range of node nd.n (0 <= nd.n < a.N).
__device__ __forceinline__ void node_at(Node &nd, const StepArgs &a)
{
    nd.x = nd.n % a.nx;
    const int r = nd.n / a.nx;
    nd.y = r % a.ny;
    nd.z = r / a.ny;
    if (a.xseg) {
        const int4 e = __ldg(a.xseg + nd.x);
        nd.x0 = e.x;
        nd.x1 = e.y;
        nd.k = e.z;
        if (!index_ok(e.x <= nd.x && nd.x < e.y && e.y <= a.nx && e.z >= 0 && e.z < a.nseg, a.status)) {
            nd.x0 = nd.x;
            nd.x1 = nd.x + 1;
            nd.k = 0;
        }
    } else {
        nd.x0 = 0;
        nd.x1 = a.nx;
        nd.k = 0;
    }
}

__device__ __forceinline__ bool node_of(Node &nd, const StepArgs &a)
{
    nd.n = blockIdx.x * blockDim.x + threadIdx.x;
    if (nd.n >= a.N) return false;
    node_at(nd, a);
    return true;
}

// Moments of one set from its 27 populations, row by row: the directions
// come in 9 rows (cy, cz) of three (cx = -1, 0, 1); per row t = f- + f0 + f+
// and dx = f+ - f-, so that
//   sum f = sum t,  sum c_x f = sum dx,  sum c_y f = sum cy t,  sum c_z f = sum cz t,
//   P_xx = sum (f- + f+), P_yy = sum_{cy != 0} t, P_zz = sum_{cz != 0} t,
//   P_xy = sum cy dx, P_xz = sum cz dx, P_yz = sum cy cz t
// (57 additions for the first four instead of 81 direction by direction).
// ld(Dir<I>{}) returns the population of direction I.
template <bool WITH_P, class V, class LD>
__device__ __forceinline__ void row_moments(LD &&ld, V &s0, V &sx, V &sy, V &sz, V *P6)
{
    for_dirs<0, 9>([&](auto dj) {
        constexpr int j = decltype(dj)::value, cy = j % 3 - 1, cz = j / 3 - 1;
        const V fm = ld(Dir<3 * j>{}), f0 = ld(Dir<3 * j + 1>{}), fp = ld(Dir<3 * j + 2>{});
        const V ac = fm + fp, t = ac + f0, dx = fp - fm;
        if constexpr (j == 0) {                           // cy = cz = -1
            s0 = t;
            sx = dx;
            sy = -t;
            sz = -t;
            if constexpr (WITH_P) {
                P6[0] = ac;
                P6[1] = t;
                P6[2] = t;
                P6[3] = -dx;
                P6[4] = -dx;
                P6[5] = t;
            }
        } else {
            s0 += t;
            sx += dx;
            if constexpr (cy == 1) sy += t;
            if constexpr (cy == -1) sy -= t;
            if constexpr (cz == 1) sz += t;
            if constexpr (cz == -1) sz -= t;
            if constexpr (WITH_P) {
                P6[0] += ac;
                if constexpr (cy != 0) P6[1] += t;
                if constexpr (cz != 0) P6[2] += t;
                if constexpr (cy == 1) P6[3] += dx;
                if constexpr (cy == -1) P6[3] -= dx;
                if constexpr (cz == 1) P6[4] += dx;
                if constexpr (cz == -1) P6[4] -= dx;
                if constexpr (cy * cz == 1) P6[5] += t;
                if constexpr (cy * cz == -1) P6[5] -= t;
            }
        }
    });
}

// Moments of the pulled populations.  Species a < M-1 give rho_a and j_a;
// f gives rho, j and (WITH_P) the pressure tensor; g gives rho E and q.
struct Sums {
    double rho, j[3], P[6], rhoE, q[3];   // P: xx, yy, zz, xy, xz, yz
    Real jr[3];                           // j as summed, in the storage type
};

// In the mixed units the moving populations are summed as the stored float
// deviations from the set's rest state; its moments (ref0, refP: double,
// the first moments vanish) and the double rest population are added once.
#if LBMK_MIXED
__device__ __forceinline__ Real pull_dev(const MechConst &mc, const PopView &v, const StepArgs &a, int s, int i,
                                         const PullIdx &p)
{
    const Src sr = src_of(i, p, a);
    return sr.ghost ? (Real)load_ghost(a, sr.side, s, i, sr.idx) - RAWREF(s, i) : load_raw_sf(v, s, i, sr.idx);
}
#endif

template <int M, bool WITH_P>
__device__ __forceinline__ void pull_moments(const MechConst &mc, const StepArgs &a, const PullIdx &p, int n,
                                             double *rho_a, Real (*ja)[3], Sums &sm)
{
    const PopView v = view(a.src, a);
#pragma unroll
    for (int s = 0; s < M - 1; ++s) {
        Real a0, ax, ay, az;
        row_moments<false, Real>([&](auto d) {
            constexpr int I = decltype(d)::value;
#if LBMK_MIXED
            if (I == REST) return (Real)0;                    // the double rest population: below
            return pull_dev(mc, v, a, s, I, p);
#else
            return pull_sf(mc, v, a, s, I, p);
#endif
        }, a0, ax, ay, az, nullptr);
        rho_a[s] = cvt<double>(a0);
#if LBMK_MIXED
        rho_a[s] += mc.ref0[s] + v.rest()[(size_t)s * a.N + n];
#endif
        ja[s][0] = ax;
        ja[s][1] = ay;
        ja[s][2] = az;
    }
    double g0, qx, qy, qz;
    row_moments<false, double>([&](auto d) { return pull_g(v, a, decltype(d)::value, p); }, g0, qx, qy, qz, nullptr);
    Real a0, ax, ay, az, P6[6];
    row_moments<WITH_P, Real>([&](auto d) {
        constexpr int I = decltype(d)::value;
#if LBMK_MIXED
        if (I == REST) return (Real)0;
        return pull_dev(mc, v, a, M - 1, I, p);
#else
        return pull_sf(mc, v, a, M - 1, I, p);
#endif
    }, a0, ax, ay, az, P6);
    sm.rho = cvt<double>(a0);
    sm.rhoE = g0;
    sm.jr[0] = ax; sm.jr[1] = ay; sm.jr[2] = az;
    sm.j[0] = cvt<double>(ax); sm.j[1] = cvt<double>(ay); sm.j[2] = cvt<double>(az);
    sm.q[0] = qx; sm.q[1] = qy; sm.q[2] = qz;
#pragma unroll
    for (int k = 0; k < 6; ++k) sm.P[k] = WITH_P ? cvt<double>(P6[k]) : 0.0;
#if LBMK_MIXED
    sm.rho += mc.ref0[M - 1] + v.rest()[(size_t)(M - 1) * a.N + n];
    if constexpr (WITH_P)
#pragma unroll
        for (int d = 0; d < 3; ++d) sm.P[d] += mc.refP[M - 1][d];
#endif
}

// ---------------------------------------------------------------------
// Initialisation: every set at equilibrium for X, T, u and pressure P.
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK, LBMK_INIT_MINB) k_init(StepArgs a, const double *X, const double *Tf,
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
    equilibria<M>(mc, rho_a, u, T, [&](int s, int i, double v) {
        if (s < M) store_sf(mc, a.dst, a, s, i, n, v);
        else store_g(a.dst, a, i, n, v);
    });
    a.macro[(size_t)DR_T * a.N + n] = T;
}

// ---------------------------------------------------------------------
// Ghost nodes beyond the x faces (Sec. 5a): equilibria at the
// post-collision moments of the adjacent boundary node, u = 0 on the left.
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void ghost_node(const StepArgs &a, int t)
{
    const MechConst &mc = c_mech[a.slot];
    const int plane = a.ny * a.nz;
    const int nlat = a.nseg > 1 ? a.nseg : 1;
    if (t >= 2 * nlat * plane) return;
    const int gp = t / plane, yz = t % plane;          // ghost plane 2k + side of lattice k
    const int side = gp & 1, k = gp >> 1;
    int x0 = 0, x1 = a.nx;
    if (a.segs) {
        const int2 r = __ldg(a.segs + k);
        x0 = r.x;
        x1 = r.y;
    }
    size_t n = (size_t)(side ? x1 - 1 : x0) + (size_t)a.nx * yz;
    if (!index_ok(x0 >= 0 && x0 < x1 && x1 <= a.nx && n < (size_t)a.N, a.status)) n = 0;
    const PopView v = view(a.src, a);
    double rho_a[M], rho = 0.0, j[3] = {0, 0, 0}, rhoE = 0.0;
    double rest = 0.0;
    for (int s = 0; s < M - 1; ++s) {
        double acc = 0.0;
        for (int i = 0; i < LBMK_Q; ++i) acc += load_sf_d(mc, v, s, i, n);
        rho_a[s] = acc;
        rest += acc;
    }
    for (int i = 0; i < LBMK_Q; ++i) {
        const double f = load_sf_d(mc, v, M - 1, i, n);
        rho += f;
        j[0] += CX(i) * f;
        j[1] += CY(i) * f;
        j[2] += CZ(i) * f;
        rhoE += load_g(v, i, n);
    }
    rho_a[M - 1] = rho - rest;
    double Y[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Y[s] = rho_a[s] / rho;
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    const double e = rhoE / rho - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double T = solve_T(eu, e, a.macro[(size_t)DR_T * a.N + n], a.status);
    if (side == 0) u[0] = u[1] = u[2] = 0.0;
    double *gh = static_cast<double *>(a.ghost) + (size_t)gp * (M + 1) * LBMK_Q * plane;
    equilibria<M>(mc, rho_a, u, T, [&](int s, int i, double val) { gh[((size_t)s * LBMK_Q + i) * plane + yz] = val; });
}

template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_ghost(StepArgs a)
{
    ghost_node<M>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------
// Production rates rho_dot_a (Eq. (sumRhoDot)) of the mass-action
// mechanism.  With E_a = exp(g_a/(R_U T))
// and act_a = c_a E_a, the rate of progress of a reaction is
//   q = k_f / prod_reac E * (prod_reac act - (P0/(r T))^(-dn) prod_prod act),
// which equals k_f prod_reac c - (k_f / K_c) prod_prod c.
// ---------------------------------------------------------------------

// 2^(j/256), j = 0..255, each the double nearest to the exact value
// (60-digit evaluation of 2^(j/256), rounded once).
__device__ const double c_exp2_256[256] = {
    0x1.0000000000000p+0, 0x1.00b1afa5abcbfp+0, 0x1.0163da9fb3335p+0, 0x1.02168143b0281p+0,
    0x1.02c9a3e778061p+0, 0x1.037d42e11bbccp+0, 0x1.04315e86e7f85p+0, 0x1.04e5f72f654b1p+0,
    0x1.059b0d3158574p+0, 0x1.0650a0e3c1f89p+0, 0x1.0706b29ddf6dep+0, 0x1.07bd42b72a836p+0,
    0x1.0874518759bc8p+0, 0x1.092bdf66607e0p+0, 0x1.09e3ecac6f383p+0, 0x1.0a9c79b1f3919p+0,
    0x1.0b5586cf9890fp+0, 0x1.0c0f145e46c85p+0, 0x1.0cc922b7247f7p+0, 0x1.0d83b23395decp+0,
    0x1.0e3ec32d3d1a2p+0, 0x1.0efa55fdfa9c5p+0, 0x1.0fb66affed31bp+0, 0x1.1073028d7233ep+0,
    0x1.11301d0125b51p+0, 0x1.11edbab5e2ab6p+0, 0x1.12abdc06c31ccp+0, 0x1.136a814f204abp+0,
    0x1.1429aaea92de0p+0, 0x1.14e95934f312ep+0, 0x1.15a98c8a58e51p+0, 0x1.166a45471c3c2p+0,
    0x1.172b83c7d517bp+0, 0x1.17ed48695bbc0p+0, 0x1.18af9388c8deap+0, 0x1.1972658375d2fp+0,
    0x1.1a35beb6fcb75p+0, 0x1.1af99f8138a1cp+0, 0x1.1bbe084045cd4p+0, 0x1.1c82f95281c6bp+0,
    0x1.1d4873168b9aap+0, 0x1.1e0e75eb44027p+0, 0x1.1ed5022fcd91dp+0, 0x1.1f9c18438ce4dp+0,
    0x1.2063b88628cd6p+0, 0x1.212be3578a819p+0, 0x1.21f49917ddc96p+0, 0x1.22bdda27912d1p+0,
    0x1.2387a6e756238p+0, 0x1.2451ffb82140ap+0, 0x1.251ce4fb2a63fp+0, 0x1.25e85711ece75p+0,
    0x1.26b4565e27cddp+0, 0x1.2780e341ddf29p+0, 0x1.284dfe1f56381p+0, 0x1.291ba7591bb70p+0,
    0x1.29e9df51fdee1p+0, 0x1.2ab8a66d10f13p+0, 0x1.2b87fd0dad990p+0, 0x1.2c57e39771b2fp+0,
    0x1.2d285a6e4030bp+0, 0x1.2df961f641589p+0, 0x1.2ecafa93e2f56p+0, 0x1.2f9d24abd886bp+0,
    0x1.306fe0a31b715p+0, 0x1.31432edeeb2fdp+0, 0x1.32170fc4cd831p+0, 0x1.32eb83ba8ea32p+0,
    0x1.33c08b26416ffp+0, 0x1.3496266e3fa2dp+0, 0x1.356c55f929ff1p+0, 0x1.36431a2de883bp+0,
    0x1.371a7373aa9cbp+0, 0x1.37f26231e754ap+0, 0x1.38cae6d05d866p+0, 0x1.39a401b7140efp+0,
    0x1.3a7db34e59ff7p+0, 0x1.3b57fbfec6cf4p+0, 0x1.3c32dc313a8e5p+0, 0x1.3d0e544ede173p+0,
    0x1.3dea64c123422p+0, 0x1.3ec70df1c5175p+0, 0x1.3fa4504ac801cp+0, 0x1.40822c367a024p+0,
    0x1.4160a21f72e2ap+0, 0x1.423fb2709468ap+0, 0x1.431f5d950a897p+0, 0x1.43ffa3f84b9d4p+0,
    0x1.44e086061892dp+0, 0x1.45c2042a7d232p+0, 0x1.46a41ed1d0057p+0, 0x1.4786d668b3237p+0,
    0x1.486a2b5c13cd0p+0, 0x1.494e1e192aed2p+0, 0x1.4a32af0d7d3dep+0, 0x1.4b17dea6db7d7p+0,
    0x1.4bfdad5362a27p+0, 0x1.4ce41b817c114p+0, 0x1.4dcb299fddd0dp+0, 0x1.4eb2d81d8abffp+0,
    0x1.4f9b2769d2ca7p+0, 0x1.508417f4531eep+0, 0x1.516daa2cf6642p+0, 0x1.5257de83f4eefp+0,
    0x1.5342b569d4f82p+0, 0x1.542e2f4f6ad27p+0, 0x1.551a4ca5d920fp+0, 0x1.56070dde910d2p+0,
    0x1.56f4736b527dap+0, 0x1.57e27dbe2c4cfp+0, 0x1.58d12d497c7fdp+0, 0x1.59c0827ff07ccp+0,
    0x1.5ab07dd485429p+0, 0x1.5ba11fba87a03p+0, 0x1.5c9268a5946b7p+0, 0x1.5d84590998b93p+0,
    0x1.5e76f15ad2148p+0, 0x1.5f6a320dceb71p+0, 0x1.605e1b976dc09p+0, 0x1.6152ae6cdf6f4p+0,
    0x1.6247eb03a5585p+0, 0x1.633dd1d1929fdp+0, 0x1.6434634ccc320p+0, 0x1.652b9febc8fb7p+0,
    0x1.6623882552225p+0, 0x1.671c1c70833f6p+0, 0x1.68155d44ca973p+0, 0x1.690f4b19e9538p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6b052fa75173ep+0, 0x1.6c012750bdabfp+0, 0x1.6cfdcddd47645p+0,
    0x1.6dfb23c651a2fp+0, 0x1.6ef9298593ae5p+0, 0x1.6ff7df9519484p+0, 0x1.70f7466f42e87p+0,
    0x1.71f75e8ec5f74p+0, 0x1.72f8286ead08ap+0, 0x1.73f9a48a58174p+0, 0x1.74fbd35d7cbfdp+0,
    0x1.75feb564267c9p+0, 0x1.77024b1ab6e09p+0, 0x1.780694fde5d3fp+0, 0x1.790b938ac1cf6p+0,
    0x1.7a11473eb0187p+0, 0x1.7b17b0976cfdbp+0, 0x1.7c1ed0130c132p+0, 0x1.7d26a62ff86f0p+0,
    0x1.7e2f336cf4e62p+0, 0x1.7f3878491c491p+0, 0x1.80427543e1a12p+0, 0x1.814d2add106d9p+0,
    0x1.82589994cce13p+0, 0x1.8364c1eb941f7p+0, 0x1.8471a4623c7adp+0, 0x1.857f4179f5b21p+0,
    0x1.868d99b4492edp+0, 0x1.879cad931a436p+0, 0x1.88ac7d98a6699p+0, 0x1.89bd0a478580fp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8be05bad61778p+0, 0x1.8cf3216b5448cp+0, 0x1.8e06a5e0866d9p+0,
    0x1.8f1ae99157736p+0, 0x1.902fed0282c8ap+0, 0x1.9145b0b91ffc6p+0, 0x1.925c353aa2fe2p+0,
    0x1.93737b0cdc5e5p+0, 0x1.948b82b5f98e5p+0, 0x1.95a44cbc8520fp+0, 0x1.96bdd9a7670b3p+0,
    0x1.97d829fde4e50p+0, 0x1.98f33e47a22a2p+0, 0x1.9a0f170ca07bap+0, 0x1.9b2bb4d53fe0dp+0,
    0x1.9c49182a3f090p+0, 0x1.9d674194bb8d5p+0, 0x1.9e86319e32323p+0, 0x1.9fa5e8d07f29ep+0,
    0x1.a0c667b5de565p+0, 0x1.a1e7aed8eb8bbp+0, 0x1.a309bec4a2d33p+0, 0x1.a42c980460ad8p+0,
    0x1.a5503b23e255dp+0, 0x1.a674a8af46052p+0, 0x1.a799e1330b358p+0, 0x1.a8bfe53c12e59p+0,
    0x1.a9e6b5579fdbfp+0, 0x1.ab0e521356ebap+0, 0x1.ac36bbfd3f37ap+0, 0x1.ad5ff3a3c2774p+0,
    0x1.ae89f995ad3adp+0, 0x1.afb4ce622f2ffp+0, 0x1.b0e07298db666p+0, 0x1.b20ce6c9a8952p+0,
    0x1.b33a2b84f15fbp+0, 0x1.b468415b749b1p+0, 0x1.b59728de5593ap+0, 0x1.b6c6e29f1c52ap+0,
    0x1.b7f76f2fb5e47p+0, 0x1.b928cf22749e4p+0, 0x1.ba5b030a1064ap+0, 0x1.bb8e0b79a6f1fp+0,
    0x1.bcc1e904bc1d2p+0, 0x1.bdf69c3f3a207p+0, 0x1.bf2c25bd71e09p+0, 0x1.c06286141b33dp+0,
    0x1.c199bdd85529cp+0, 0x1.c2d1cd9fa652cp+0, 0x1.c40ab5fffd07ap+0, 0x1.c544778fafb22p+0,
    0x1.c67f12e57d14bp+0, 0x1.c7ba88988c933p+0, 0x1.c8f6d9406e7b5p+0, 0x1.ca3405751c4dbp+0,
    0x1.cb720dcef9069p+0, 0x1.ccb0f2e6d1675p+0, 0x1.cdf0b555dc3fap+0, 0x1.cf3155b5bab74p+0,
    0x1.d072d4a07897cp+0, 0x1.d1b532b08c968p+0, 0x1.d2f87080d89f2p+0, 0x1.d43c8eacaa1d6p+0,
    0x1.d5818dcfba487p+0, 0x1.d6c76e862e6d3p+0, 0x1.d80e316c98398p+0, 0x1.d955d71ff6075p+0,
    0x1.da9e603db3285p+0, 0x1.dbe7cd63a8315p+0, 0x1.dd321f301b460p+0, 0x1.de7d5641c0658p+0,
    0x1.dfc97337b9b5fp+0, 0x1.e11676b197d17p+0, 0x1.e264614f5a129p+0, 0x1.e3b333b16ee12p+0,
    0x1.e502ee78b3ff6p+0, 0x1.e653924676d76p+0, 0x1.e7a51fbc74c83p+0, 0x1.e8f7977cdb740p+0,
    0x1.ea4afa2a490dap+0, 0x1.eb9f4867cca6ep+0, 0x1.ecf482d8e67f1p+0, 0x1.ee4aaa2188510p+0,
    0x1.efa1bee615a27p+0, 0x1.f0f9c1cb6412ap+0, 0x1.f252b376bba97p+0, 0x1.f3ac948dd7274p+0,
    0x1.f50765b6e4540p+0, 0x1.f6632798844f8p+0, 0x1.f7bfdad9cbe14p+0, 0x1.f91d802243c89p+0,
    0x1.fa7c1819e90d8p+0, 0x1.fbdba3692d514p+0, 0x1.fd3c22b8f71f1p+0, 0x1.fe9d96b2a23d9p+0,
};

// exp(x) by the table-driven method of P. T. P. Tang (ACM Trans. Math.
// Softw. 15(2), 1989): x = (256 m + j) ln2/256 + r with |r| <= ln2/512, so
// exp(x) = 2^m 2^(j/256) e^r, and e^r - 1 is its degree-4 Taylor polynomial
// (truncation error below 4e-17).  ln2/256 = L1 + L2 with L1 rounded to 35
// significant bits, so that N L1 is exact for |N| < 2^18 and the reduced
// argument carries no cancellation error (Cody and Waite).  N = rint(x
// 256/ln2) by the 1.5 2^52 rounding constant; 2^m is added to the result's
// binary exponent.  |x| >= 707 (where 2^m would leave the normal range) and
// NaN go to exp(); that test reads the high word of x on the integer pipe.
// About 1 ulp; 9 double operations.
__device__ __forceinline__ double exp_table(double x)
{
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40861800) return exp(x);      // |x| >= 707, inf, NaN
    const double kRound = 6755399441055744.0;                 // 1.5 * 2^52
    const double t = fma(x, 0x1.71547652b82fep+8, kRound);    // x 256/ln2, rounded to an integer
    const int n = __double2loint(t);
    const double N = t - kRound;
    double r = fma(-N, 0x1.62e42fefc0000p-9, x);              // L1
    r = fma(-N, -0x1.c610ca86c3899p-45, r);                   // L2
    const double p = fma(r * r, fma(fma(1.0 / 24.0, r, 1.0 / 6.0), r, 0.5), r);
    const double Tj = __ldg(&c_exp2_256[n & 255]);
    const double y = fma(Tj, p, Tj);
    return __hiloint2double(__double2hiint(y) + (n >> 8) * (1 << 20), __double2loint(y));
}

// Exponential of the rate expressions: exp_table(), except in the fast mixed
// unit, where the rates are stored in float: a base-2 range reduction
// done exactly in double (t = x log2(e) = k + f, k integer, |f| <= 1/2, in
// the manner of Cody and Waite), 2^f from the hardware base-2 exponential
// in float (ex2.approx, relative error about 2^-22), and 2^k added to the
// binary exponent of the result; relative error below 5e-7.
__device__ __forceinline__ double exp_rate(double x)
{
#if LBMK_MIXED && LBMK_FAST
    const double t = x * 1.4426950408889634074;          // log2(e)
    if (!(fabs(t) < 1020.0)) return t > 0.0 ? (double)INFINITY : (t < 0.0 ? 0.0 : t);
    const double k = rint(t);
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"((float)(t - k)));
    const double r = (double)y;                          // in [2^-1/2, 2^1/2]
    return __hiloint2double(__double2hiint(r) + (int)k * (1 << 20), __double2loint(r));
#else
    return exp_table(x);
#endif
}

// Molar production rates sum_k (nu''_ak - nu'_ak) q_k at temperature T and
// concentrations conc, left in sh_w[a * stride + t]; sh_act and sh_g are
// this thread's scratch columns (stride: the block's thread count).
template <int M>
__device__ __forceinline__ void molar_production(const MechConst &mc, double T, const double *conc, double *sh_act,
                                                 double *sh_g, WReal *sh_w, int t, int stride)
{
    const double invT = 1.0 / T, lnT = log(T);
    const double lnTr = lnT - mc.log_T_ref;
    const double om_lnT = 1.0 - lnT;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        const double *gc = mc.gco[s];
        const double g = fma(gc[0], om_lnT,
                             fma(fma(fma(fma(gc[4], T, gc[3]), T, gc[2]), T, gc[1]), T, fma(gc[5], invT, gc[6])));
        sh_g[s * stride + t] = g;
        sh_act[s * stride + t] = conc[s] * exp_rate(g);
        sh_w[s * stride + t] = 0;
    }
    const double c0 = mc.P0_over_r * invT, ic0 = T / mc.P0_over_r;   // P0/(r T) and its inverse
    for (int k = 0; k < mc.R; ++k) {
        const int nr = mc.nreac[k], np = mc.nprod[k];     // nr >= 1 (checked at packing)
        const int s0 = mc.reac[k][0] * stride + t;
        double arg = fma(mc.b[k], lnTr, fma(-mc.theta[k], invT, mc.log_A[k])) - sh_g[s0];
        double pf = sh_act[s0];
        for (int j = 1; j < nr; ++j) {
            const int sidx = mc.reac[k][j] * stride + t;
            arg -= sh_g[sidx];
            pf *= sh_act[sidx];
        }
        double q = pf;
        if (mc.rev[k]) {
            double pr = np > 0 ? sh_act[mc.prod[k][0] * stride + t] : 1.0;
            for (int j = 1; j < np; ++j) pr *= sh_act[mc.prod[k][j] * stride + t];
            const int dn = mc.dn[k];
            for (int j = 0; j < dn; ++j) pr *= ic0;
            for (int j = 0; j < -dn; ++j) pr *= c0;
            q -= pr;
        }
        q *= exp_rate(arg);
        const int type = mc.rtype[k];
        if (type != 0) {
            double cM = 0.0;
#pragma unroll
            for (int s = 0; s < M; ++s) cM = fma(mc.eff[k][s], conc[s], cM);
            if (type == 1) {
                q *= cM;
            } else {
                const double Pr = exp_rate(fma(mc.dlow[k][1], lnTr, fma(-mc.dlow[k][2], invT, mc.dlow[k][0]))) * cM;
                q *= Pr / (1.0 + Pr);
            }
        }
        const WReal qr = cvt<WReal>(q);
        for (int j = 0; j < nr; ++j) sh_w[mc.reac[k][j] * stride + t] -= qr;
        for (int j = 0; j < np; ++j) sh_w[mc.prod[k][j] * stride + t] += qr;
    }
}

// ---------------------------------------------------------------------
// Moments for lbm_moments: the fields of the state in src (no record).
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK, LBMK_MOM_MINB) k_moments(StepArgs a, unsigned mask, double *out)
{
    __shared__ double sh_act[M * LBMK_BLOCK];
    __shared__ double sh_g[M * LBMK_BLOCK];
    __shared__ WReal sh_w[M * LBMK_BLOCK];
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    PullIdx p;
    make_pull(p, nd, a);
    double rho_a[M];
    Real ja[M][3];
    Sums sm;
    pull_moments<M, false>(mc, a, p, nd.n, rho_a, ja, sm);
    const double rho = sm.rho;
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) rest += rho_a[s];
    rho_a[M - 1] = rho - rest;
    double Y[M], inv_m = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) { Y[s] = rho_a[s] / rho; inv_m += Y[s] * mc.invW[s]; }
    const double u[3] = {sm.j[0] / rho, sm.j[1] / rho, sm.j[2] / rho};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const int n = nd.n;
    const size_t N = a.N;
    const double T = solve_T(eu, sm.rhoE / rho - 0.5 * usq, a.macro[DR_T * N + n], a.status);
    const double Rm = mc.r_lat * inv_m;
    size_t row = 0;
    if (mask & 1u) { for (int s = 0; s < M; ++s) out[(row + s) * N + n] = rho_a[s]; row += M; }
    if (mask & 2u) { for (int d = 0; d < 3; ++d) out[(row + d) * N + n] = sm.j[d]; row += 3; }
    if (mask & 4u) { out[row * N + n] = sm.rhoE; row += 1; }
    if (mask & 8u) { out[row * N + n] = T; row += 1; }
    if (mask & 16u) { out[row * N + n] = rho * Rm * T; row += 1; }
    if (mask & 32u) { for (int s = 0; s < M; ++s) out[(row + s) * N + n] = Y[s]; row += M; }
    if (mask & 64u) {
        double jM[3] = {sm.j[0], sm.j[1], sm.j[2]};
        for (int s = 0; s < M - 1; ++s)
            for (int d = 0; d < 3; ++d) { out[(row + 3 * s + d) * N + n] = ja[s][d]; jM[d] -= ja[s][d]; }
        for (int d = 0; d < 3; ++d) out[(row + 3 * (M - 1) + d) * N + n] = jM[d];
        row += 3 * M;
    }
    if (mask & (128u | 256u)) {
        double conc[M];
#pragma unroll
        for (int s = 0; s < M; ++s) conc[s] = rho_a[s] * mc.invW[s];
        molar_production<M>(mc, T, conc, sh_act, sh_g, sh_w, threadIdx.x, LBMK_BLOCK);
        if (mask & 128u) {
            for (int s = 0; s < M; ++s) out[(row + s) * N + n] = mc.W[s] * (double)sh_w[s * LBMK_BLOCK + threadIdx.x];
            row += M;
        }
        if (mask & 256u) {      // heat release rate, -sum_a H_a rho_dot_a
            double h = 0.0;
            for (int s = 0; s < M; ++s)
                h = fma(-H_spec(mc, s, T), mc.W[s] * (double)sh_w[s * LBMK_BLOCK + threadIdx.x], h);
            out[row * N + n] = h;
        }
    }
}

// ---------------------------------------------------------------------
// Pass 1: pull, moments, temperature, relaxation, Stefan-Maxwell solve;
// writes the per-node record (all rows but the production rates).
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void pre_node(const StepArgs &a, const Node &nd)
{
    const MechConst &mc = c_mech[a.slot];
    PullIdx p;
    make_pull(p, nd, a);
    double rho_a[M];
    Real ja[M][3];
    Sums sm;
    pull_moments<M, true>(mc, a, p, nd.n, rho_a, ja, sm);

    // composition and velocity (Eq. (strongest) for the slaved species)
    const double rho = sm.rho, ir = 1.0 / rho;
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) rest += rho_a[s];
    rho_a[M - 1] = rho - rest;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Real js = sm.jr[d];
#pragma unroll
        for (int s = 0; s < M - 1; ++s) js -= ja[s][d];
        ja[M - 1][d] = js;
    }
    double Y[M], inv_m = 0.0;
    bool neg = false;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = rho_a[s] * ir;
        inv_m = fma(Y[s], mc.invW[s], inv_m);
        if (__double2hiint(rho_a[s]) < 0)     // sign bit first: the compare only for negative values
            neg |= rho_a[s] < -1e-10 * rho;  // below rounding noise of trace species
    }
    if (!(rho > 0.0) || !isfinite(sm.rhoE)) flag(a.status, LBMK_BIT_NONFINITE);
    if (neg) flag(a.status, LBMK_BIT_NEGATIVE);
    const double u[3] = {sm.j[0] * ir, sm.j[1] * ir, sm.j[2] * ir};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // temperature, Eq. (temperature)
    const int n = nd.n;
    const size_t N = a.N;
    double T, Cv = 0.0;
    {
        double eu[6];
        mixture_energy_poly<M>(mc, Y, eu);
        T = solve_T(eu, sm.rhoE * ir - 0.5 * usq, a.macro[DR_T * N + n], a.status);
        if (mc.transport) Cv = dpoly5(eu, T);
    }
    const double Rm = mc.r_lat * inv_m;
    const double P = rho * Rm * T;
    // relaxation rates (Eqs. (mu), (lambda)) in the storage type: in the
    // mixed units they are stored and used as floats only; dfac scales the
    // binary diffusivities of mixture-averaged transport
    Real nup, nup1;
    double dfac = 1.0;
    if (mc.transport) {
        mixture_transport<M>(mc, Y, inv_m, T, P, Cv + Rm, nup, nup1, dfac);
    } else {
        nup = cvt<Real>(nu_prime(mc, Rm, T));
        nup1 = nup / cvt<Real>(mc.Pr);
    }
    const Real omega = (Real)1 / ((Real)0.5 + nup);
    const Real omega1 = (Real)1 / ((Real)0.5 + nup1);

    // enthalpies, Eq. (specHa)
    double Ha[M], H = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Ha[s] = H_spec(mc, s, T);
        H = fma(Y[s], Ha[s], H);
    }

    // Eq. (tauab): 1/tau_ab = kappa / (W_a W_b D_ab), kappa = m R_U T;
    // 1/tau_a = sum_b Y_b / tau_ab.  From here to the diffusion velocities
    // the arithmetic is in SReal: double, or float in the fast mixed unit
    // (the results are stored as floats there, and the solve below is well
    // conditioned: B is diagonally dominant after the symmetric scaling by Y).
    const double kappa = mc.transport ? mc.r_lat * T / (inv_m * dfac) : mc.r_lat * T / inv_m;
    const SReal kap = cvt<SReal>(kappa), irr = cvt<SReal>(ir);
    SReal Yr[M], ur[3] = {cvt<SReal>(u[0]), cvt<SReal>(u[1]), cvt<SReal>(u[2])};
#pragma unroll
    for (int s = 0; s < M; ++s) Yr[s] = cvt<SReal>(Y[s]);
    SReal ita[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        SReal acc = 0;
#pragma unroll
        for (int b = 0; b < M; ++b)
            if (b != s) acc = fma(Yr[b], INVWWD_S(s, b), acc);
        ita[s] = kap * acc;
    }

    // Eq. (transform1), multiplied by Y_a so that the matrix is symmetric:
    //   B_aa = Y_a (1 + 1/(2 tau_a)),  B_ab = -(1/2) Y_a Y_b / tau_ab,
    //   rhs_a = Y_a (u_a - u) = j_a / rho - Y_a u.
    // B is symmetric positive definite; L D L^T without pivoting, L unit
    // lower triangular (stored below the diagonal of Ln).
    SReal du[M][3];
    {
        SReal Ln[M][M], D[M], Dinv[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const SReal hy = (SReal)-0.5 * kap * Yr[i];
#pragma unroll
            for (int k = 0; k < i; ++k) Ln[i][k] = hy * INVWWD_S(i, k) * Yr[k];
            Ln[i][i] = Yr[i] * fma((SReal)0.5, ita[i], (SReal)1);
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            SReal tk[M];
#pragma unroll
            for (int j = 0; j < k; ++j) tk[j] = D[j] * Ln[k][j];
#pragma unroll
            for (int i = k; i < M; ++i) {
                SReal sacc = Ln[i][k];
#pragma unroll
                for (int j = 0; j < k; ++j) sacc = fma(-Ln[i][j], tk[j], sacc);
                Ln[i][k] = sacc;
            }
            // D_k = Y_k times the pivot of the unscaled system, which is
            // diagonally dominant: negative where a trace species has dipped
            // to a rounding-level negative density, zero only for an absent
            // species (Y_k = 0), whose row and column vanish and whose
            // diffusion velocity is multiplied by Y_k = 0 wherever it is used.
            D[k] = Ln[k][k];
            if (!finite_bits(D[k])) flag(a.status, LBMK_BIT_PIVOT);
            Dinv[k] = nonzero_bits(D[k]) ? (SReal)1 / D[k] : (SReal)0;
#pragma unroll
            for (int i = k + 1; i < M; ++i) Ln[i][k] *= Dinv[k];
        }
        // L z = rhs, z /= D, L^T x = z
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                SReal sacc = fma(cvt<SReal>(ja[i][d]), irr, -Yr[i] * ur[d]);
#pragma unroll
                for (int j = 0; j < i; ++j) sacc = fma(-Ln[i][j], du[j][d], sacc);
                du[i][d] = sacc;
            }
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) du[i][d] *= Dinv[i];
#pragma unroll
        for (int i = M - 1; i >= 0; --i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                SReal sacc = du[i][d];
#pragma unroll
                for (int j = i + 1; j < M; ++j) sacc = fma(-Ln[j][i], du[j][d], sacc);
                du[i][d] = sacc;
            }
    }

    // energy: equilibrium moments and the local part of
    // Dq = (omega - omega_1)(q^* - q^eq) (Eqs. (gstareq1mom), (qdiff)); the
    // grad-Y part (Eq. (corrFourier)) needs the neighbours and is added in k_step.
    const double hk = H + 0.5 * usq;
    double qeq[3], Rt[6], tr3;
    energy_moments(rho, u, P, hk, sm.rhoE, qeq, Rt, tr3);
    Real dq[3], HaR[M], YR[M], duR[M][3];
    {
        const double dP[6] = {sm.P[0] - (P + rho * u[0] * u[0]), sm.P[1] - (P + rho * u[1] * u[1]),
                              sm.P[2] - (P + rho * u[2] * u[2]), sm.P[3] - rho * u[0] * u[1],
                              sm.P[4] - rho * u[0] * u[2], sm.P[5] - rho * u[1] * u[2]};
        const double uP[3] = {u[0] * dP[0] + u[1] * dP[3] + u[2] * dP[4],
                              u[0] * dP[3] + u[1] * dP[1] + u[2] * dP[5],
                              u[0] * dP[4] + u[1] * dP[5] + u[2] * dP[2]};
        // Dq is stored in the storage type: the differences are formed in
        // double (they cancel), the products with the stored values of
        // omega, omega_1, H_a, Y_a and du_a in the storage type
        Real HY[M];
#pragma unroll
        for (int s = 0; s < M; ++s) {
            HaR[s] = cvt<Real>(Ha[s]);
            YR[s] = cvt<Real>(Yr[s]);
            HY[s] = HaR[s] * YR[s];
#pragma unroll
            for (int d = 0; d < 3; ++d) duR[s][d] = cvt<Real>(du[s][d]);
        }
        const Real orho = omega1 * cvt<Real>(rho);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Real hyd = 0;
#pragma unroll
            for (int s = 0; s < M; ++s) hyd = fma(HY[s], duR[s][d], hyd);
            dq[d] = (omega - omega1) * cvt<Real>(sm.q[d] - uP[d] - qeq[d]) + orho * hyd;
        }
    }

    // the record: double rows
    a.macro[DR_T * N + n] = T;
    a.macro[(size_t)dr_ge(M) * N + n] = sm.rhoE;
#pragma unroll
    for (int d = 0; d < 3; ++d) a.macro[(size_t)(dr_gq(M) + d) * N + n] = qeq[d];
#pragma unroll
    for (int d = 0; d < 6; ++d) a.macro[(size_t)(dr_gr(M) + d) * N + n] = Rt[d];
    a.macro[(size_t)dr_gtr(M) * N + n] = tr3;
#if LBMK_MIXED
    // rest-direction equilibria of the species and mixture sets (Eqs. (feq), (feqmix))
    {
        const double c2[3] = {1.0 - u[0] * u[0], 1.0 - u[1] * u[1], 1.0 - u[2] * u[2]};
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const double z = (s < M - 1 ? mc.Ra[s] : Rm) * T;
            const double r = s < M - 1 ? rho_a[s] : rho;
            a.macro[(size_t)(DR_FEQ0 + s) * N + n] = r * (c2[0] - z) * (c2[1] - z) * (c2[2] - z);
        }
    }
#endif
    // storage-type rows
    const RecRows rr = rec_rows(M);
    Real *R = rec(a);
    R[(size_t)rr.nup * N + n] = nup;
    // Phi (Eq. (Xalpha)), stored in the storage type and formed in it
    const Real rhoR = cvt<Real>(rho), rtR = cvt<Real>(Rm * T), ph = (Real)1 - (Real)3 * rtR;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const Real ud = cvt<Real>(ur[d]);
        R[(size_t)(rr.phi + d) * N + n] = rhoR * ud * (ph - ud * ud);
        R[(size_t)(rr.u + d) * N + n] = ud;
        R[(size_t)(rr.dq + d) * N + n] = dq[d];
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
        R[(size_t)(rr.y + s) * N + n] = YR[s];
#pragma unroll
        for (int d = 0; d < 3; ++d) R[(size_t)(rr.du + 3 * s + d) * N + n] = duR[s][d];
        // beta_a = 1/(2 tau_a + 1), Eq. (fStar): a parameter of the species
        // collision, formed in the storage type it is used in
        const Real it = cvt<Real>(ita[s]);
        R[(size_t)(rr.beta + s) * N + n] = it / ((Real)2 + it);
        R[(size_t)(rr.h + s) * N + n] = HaR[s];
    }
    R[(size_t)rr.rho * N + n] = rhoR;
    R[(size_t)rr.kappa * N + n] = cvt<Real>(kap);
    R[(size_t)rr.rt * N + n] = rtR;
    R[(size_t)rr.om * N + n] = omega;
    R[(size_t)rr.om1 * N + n] = omega1;
    R[(size_t)rr.p * N + n] = cvt<Real>(P);
}

template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK, LBMK_PRE_MINB) k_pre(StepArgs a)
{
    Node nd;
    if (!node_of(nd, a)) return;
    pre_node<M>(a, nd);
}

// ---------------------------------------------------------------------
// Pass 1b: production rates of the record's state (molar_production).
// ---------------------------------------------------------------------
// Shared memory of k_chem for a block of bs threads.
template <int M>
constexpr size_t chem_smem(int bs) { return (size_t)M * bs * (2 * sizeof(double) + sizeof(WReal)); }

template <int M>
__global__ void __launch_bounds__(LBMK_MAXBLOCK) k_chem(StepArgs a)
{
    extern __shared__ double sh_chem[];
    const int bs = blockDim.x;
    double *sh_act = sh_chem;                                   // c_a exp(g_a / R_U T)
    double *sh_g = sh_chem + (size_t)M * bs;                    // g_a / R_U T
    WReal *sh_w = reinterpret_cast<WReal *>(sh_chem + (size_t)2 * M * bs);   // molar production
    const MechConst &mc = c_mech[a.slot];
    const int t = threadIdx.x;
    const int n = blockIdx.x * blockDim.x + t;
    if (n >= a.N) return;
    const size_t N = a.N;
    const RecRows rr = rec_rows(M);
    Real *R = rec(a);
    const double T = a.macro[DR_T * N + n];
    const double rho = (double)R[(size_t)rr.rho * N + n];
    double conc[M];
#pragma unroll
    for (int s = 0; s < M; ++s) conc[s] = rho * (double)R[(size_t)(rr.y + s) * N + n] * mc.invW[s];
    molar_production<M>(mc, T, conc, sh_act, sh_g, sh_w, t, bs);
#pragma unroll
    for (int s = 0; s < M; ++s) R[(size_t)(rr.wd + s) * N + n] = (Real)(mc.W[s] * sh_w[s * bs + t]);
}

// ---------------------------------------------------------------------
// Pass 2: G_alpha = (1/omega - 1/2) d_alpha Phi_alpha with the isotropic
// gradient d_alpha phi = (1/theta) sum_i w_i c_ia phi(x + c_i).
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void grad_node(const StepArgs &a, const Node &nd)
{
    const size_t N = a.N;
    const RecRows rr = rec_rows(M);
    Real *R = rec(a);
    const Real *Phi = R + (size_t)rr.phi * N;
    StencilIdx st;
    make_stencil(st, nd, a);
    Real d[3] = {0, 0, 0};
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        const size_t nb = nb_of<I>(st, a);
        if (CX(I)) d[0] += (Real)(WI(I) * CX(I)) * Phi[nb];
        if (CY(I)) d[1] += (Real)(WI(I) * CY(I)) * Phi[N + nb];
        if (CZ(I)) d[2] += (Real)(WI(I) * CZ(I)) * Phi[2 * N + nb];
    });
    const Real nup = R[(size_t)rr.nup * N + nd.n];
    Real *G = R + (size_t)rr.g * N;
#pragma unroll
    for (int k = 0; k < 3; ++k) G[k * N + nd.n] = nup * (Real)3 * d[k];
}

template <int M>
__global__ void __launch_bounds__(LBMK_MAXBLOCK) k_grad(StepArgs a)
{
    Node nd;
    if (!node_of(nd, a)) return;
    grad_node<M>(a, nd);
}

// ---------------------------------------------------------------------
// Pass 3a: collision of the energy set g, Eq. (g) in the regularised form
//   g + omega (g^eq - g) + w_i (Dq . c_i) / theta,
// with the grad-Y part of Dq (Eq. (corrFourier)) from the neighbours'
// records.  The post-collision value is (1 - omega) g_i + B_i with
//   B_i = omega g_i^eq + 3 w_i c_i . Dq
//       = w_i [A0 + c_i . A1 + sum_d c_id^2 A2_d + sum_{d<e} c_id c_ie A3_de],
//   A0 = omega (rho E - (9/2) tr3),  A1 = 3 (omega q^eq + Dq),
//   A2_d = (9/2) omega R_dd,         A3_de = 9 omega R_de,
// R = R^eq - rho E theta I (Eq. (gieq) expanded in c_i).  Double precision.
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void collide_energy(const StepArgs &a, const Node &nd)
{
    const int n = nd.n;
    const size_t N = a.N;
    const RecRows rr = rec_rows(M);
    const Real *R = rec(a);
    auto ld = [&](int row) { return R[(size_t)row * N + n]; };
    auto ldd = [&](int row) { return a.macro[(size_t)row * N + n]; };

    // sum_a H_a grad Y_a (Eq. (corrFourier)), H_a of this node
    Real Hl[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Hl[s] = ld(rr.h + s);
    Real HgY[3] = {0, 0, 0};
    {
        StencilIdx st;
        make_stencil(st, nd, a);
        const Real *Yf = R + (size_t)rr.y * N;
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            if constexpr (I != REST) {
                const size_t nb = nb_of<I>(st, a);
                Real hy = 0;
#pragma unroll
                for (int s = 0; s < M; ++s) hy += Hl[s] * Yf[s * N + nb];
                constexpr Real wx = (Real)(WI(I) * CX(I)), wy = (Real)(WI(I) * CY(I)), wz = (Real)(WI(I) * CZ(I));
                if (CX(I)) HgY[0] += wx * hy;
                if (CY(I)) HgY[1] += wy * hy;
                if (CZ(I)) HgY[2] += wz * hy;
            }
        });
    }
    const Real om1 = ld(rr.om1), P = ld(rr.p);
    const double omd = (double)ld(rr.om), om1m = 1.0 - omd;
    double gD[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) gD[d] = (double)(ld(rr.dq + d) + (Real)1.5 * ((Real)2 - om1) * P * HgY[d]);
    // energy equilibrium moments (Eqs. (geq1mom), (geq2mom))
    const double gE = ldd(dr_ge(M));
    double gq[3], gR[6];
#pragma unroll
    for (int d = 0; d < 3; ++d) gq[d] = ldd(dr_gq(M) + d);
#pragma unroll
    for (int d = 0; d < 6; ++d) gR[d] = ldd(dr_gr(M) + d);
    const double gtr = ldd(dr_gtr(M));
    const double A0 = omd * (gE - 4.5 * gtr);
    double A1[3], A2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        A1[d] = 3.0 * fma(omd, gq[d], gD[d]);
        A2[d] = 4.5 * omd * gR[d];
    }
    const double A3xy = 9.0 * omd * gR[3], A3xz = 9.0 * omd * gR[4], A3yz = 9.0 * omd * gR[5];

    const PopView v = view(a.src, a);
    PullIdx p;
    make_pull(p, nd, a);
    int bad = 0;     // a non-finite result: all exponent bits set (integer test, no FP64 work)
    // row by row: j = (cy+1) + 3 (cz+1), then cx = -1, 0, 1 (i = (cx+1) + 3 j)
    for_dirs<0, 9>([&](auto dj) {
        constexpr int j = decltype(dj)::value, cy = j % 3 - 1, cz = j / 3 - 1;
        constexpr int nnz = (cy != 0) + (cz != 0);
        double base = A0, lin = A1[0];
        if (cy) { base += cy * A1[1] + A2[1]; lin += cy * A3xy; }
        if (cz) { base += cz * A1[2] + A2[2]; lin += cz * A3xz; }
        if (cy && cz) base += (cy * cz) * A3yz;
        // w_i = w(cx) w(cy) w(cz) with w(0) = 2/3, w(+-1) = 1/6
        constexpr double w0 = nnz == 0 ? 8.0 / 27.0 : (nnz == 1 ? 2.0 / 27.0 : 1.0 / 54.0);
        constexpr double w1 = nnz == 0 ? 2.0 / 27.0 : (nnz == 1 ? 1.0 / 54.0 : 1.0 / 216.0);
        const double bq = base + A2[0];
        const double B[3] = {w1 * (bq - lin), w0 * base, w1 * (bq + lin)};
        for_dirs<0, 3>([&](auto dx) {
            constexpr int k = decltype(dx)::value, I = k + 3 * j;
            const double val = fma(om1m, pull_g(v, a, I, p), B[k]);
            store_g(a.dst, a, I, n, val);
            bad |= (__double2hiint(val) & 0x7ff00000) == 0x7ff00000;
        });
    });
    if (bad) flag(a.status, LBMK_BIT_NONFINITE);
}

template <int M>
__global__ void __launch_bounds__(LBMK_MAXBLOCK) k_step_g(StepArgs a)
{
    Node nd;
    if (!node_of(nd, a)) return;
    collide_energy<M>(a, nd);
}

// ---------------------------------------------------------------------
// Pass 3b: collisions of the species sets (Eq. (finalNumericalEquations)
// with the quasi-equilibria of Eq. (fStar)) and of the mixture set f
// (Eq. (f) with the isotropy correction of Eq. (Ai)), direction by
// direction, in the storage precision.
// ---------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void step_node(const StepArgs &a, const Node &nd)
{
#if !LBMK_MIXED
    // y-z factors of the species equilibria for the current row, this
    // thread's column (kept in registers in the mixed units)
    __shared__ double sh_yz[2 * M * LBMK_BLOCK];
#endif
#if LBMK_FUSE_CHEM
    __shared__ double sh_act[M * LBMK_BLOCK];
    __shared__ double sh_g[M * LBMK_BLOCK];
    __shared__ WReal sh_w[M * LBMK_BLOCK];
#endif
    const MechConst &mc = c_mech[a.slot];
    const int n = nd.n;
    const size_t N = a.N;
    const RecRows rr = rec_rows(M);
    const Real *R = rec(a);
    auto ld = [&](int row) { return R[(size_t)row * N + n]; };
    auto ldd = [&](int row) { return a.macro[(size_t)row * N + n]; };

    // X = -d_alpha G_alpha (Eq. (Xalpha))
    Real X[3] = {0, 0, 0};
    {
        StencilIdx st;
        make_stencil(st, nd, a);
        const Real *G = R + (size_t)rr.g * N;
        for_dirs<0, LBMK_Q>([&](auto dd) {
            constexpr int I = decltype(dd)::value;
            if constexpr (I != REST) {
                const size_t nb = nb_of<I>(st, a);
                constexpr Real wx = (Real)(WI(I) * CX(I)), wy = (Real)(WI(I) * CY(I)), wz = (Real)(WI(I) * CZ(I));
                if (CX(I)) X[0] += wx * G[nb];
                if (CY(I)) X[1] += wy * G[N + nb];
                if (CZ(I)) X[2] += wz * G[2 * N + nb];
            }
        });
#pragma unroll
        for (int k = 0; k < 3; ++k) X[k] *= (Real)-3;
    }

    const Real rho = ld(rr.rho), om = ld(rr.om);
    const Real kappa = ld(rr.kappa), RT = ld(rr.rt);
    const Real u[3] = {ld(rr.u), ld(rr.u + 1), ld(rr.u + 2)};
    const Real T = cvt<Real>(ldd(DR_T));

    // per-species data: mass fraction, quasi-equilibrium velocity u + du_b,
    // beta_b and rho_dot_b (densities, zeta and the products are formed per
    // direction to keep the register footprint small)
    Real Yl[M], xs[M][3], bt[M], wd[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Yl[s] = ld(rr.y + s);
#pragma unroll
        for (int d = 0; d < 3; ++d) xs[s][d] = u[d] + ld(rr.du + 3 * s + d);
        bt[s] = ld(rr.beta + s);
#if !LBMK_FUSE_CHEM
        wd[s] = ld(rr.wd + s);
#endif
    }
#if LBMK_FUSE_CHEM
    {
        // the production rates of this node, as k_chem forms them
        double conc[M];
#pragma unroll
        for (int s = 0; s < M; ++s) conc[s] = cvt<double>(rho) * cvt<double>(Yl[s]) * mc.invW[s];
        molar_production<M>(mc, ldd(DR_T), conc, sh_act, sh_g, sh_w, threadIdx.x, LBMK_BLOCK);
#pragma unroll
        for (int s = 0; s < M; ++s) wd[s] = cvt<Real>(mc.W[s] * sh_w[s * LBMK_BLOCK + threadIdx.x]);
    }
#endif
    const Real u2[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};

    const PopView v = view(a.src, a);
    PullIdx p;
    make_pull(p, nd, a);
    Real check = 0;

    // Directions row by row: j = (cy+1) + 3 (cz+1), then cx = -1, 0, 1
    // (direction i = (cx+1) + 3 j, i.e. i = 0..26 in order).  The y-z
    // factors of the product-form equilibria are formed once per row.  In
    // mixed precision the populations of direction i+1 are loaded while
    // direction i is collided (raw stored values; the rest state is added
    // where they are used).
    constexpr bool kPrefetch = LBMK_MIXED;
    Real fraw[M];
    auto load_raw = [&](int i) {
        const Src sr = src_of(i, p, a);
        if (sr.ghost) {
#pragma unroll
            for (int s = 0; s < M; ++s) fraw[s] = (Real)load_ghost(a, sr.side, s, i, sr.idx) - RAWREF(s, i);
        } else {
            if (LBMK_MIXED && i == REST) return;
#pragma unroll
            for (int s = 0; s < M; ++s) fraw[s] = load_raw_sf(v, s, i, sr.idx);
        }
    };
    if (kPrefetch) load_raw(0);

#if LBMK_MIXED
    Real pe_yz[M], ps_yz[M];
#endif
    Real fe_yz = 0, AXyz = 0;
    int cy = 0, cz = 0;
    auto yz_factors = [&](int s, Real z, Real &pe, Real &ps) {
        pe = psi_c(cy, u[1], u2[1] + z) * psi_c(cz, u[2], u2[2] + z);
        ps = psi_c(cy, xs[s][1], xs[s][1] * xs[s][1] + z) * psi_c(cz, xs[s][2], xs[s][2] * xs[s][2] + z);
    };
#pragma unroll 1
    for (int i = 0; i < LBMK_Q; ++i) {
        const int cx = i % 3 - 1, j = i / 3;
        if (cx < 0) {
            cy = j % 3 - 1;
            cz = j / 3 - 1;
            const int nnz = (cy != 0) + (cz != 0);
            // y-z factors of the species equilibria, shared by the row's three
            // directions: in registers (float) or shared memory (double)
#pragma unroll
            for (int s = 0; s < M; ++s) {
#if LBMK_MIXED
                yz_factors(s, RA(s) * T, pe_yz[s], ps_yz[s]);
#else
                Real pe, ps;
                yz_factors(s, RA(s) * T, pe, ps);
                sh_yz[(2 * s) * LBMK_BLOCK + threadIdx.x] = pe;
                sh_yz[(2 * s + 1) * LBMK_BLOCK + threadIdx.x] = ps;
#endif
            }
            fe_yz = rho * psi_c(cy, u[1], u2[1] + RT) * psi_c(cz, u[2], u2[2] + RT);
            // isotropy correction A_i . X (Eq. (Ai)): only |c_i| = 1
            AXyz = nnz == 1 ? (Real)0.5 * ((Real)cy * X[1] + (Real)cz * X[2]) : (Real)0;
        }
        Real fc[M];
        if (kPrefetch) {
#pragma unroll
            for (int s = 0; s < M; ++s) fc[s] = fraw[s];
            if (i + 1 < LBMK_Q) load_raw(i + 1);
        } else {
            load_raw(i);
#pragma unroll
            for (int s = 0; s < M; ++s) fc[s] = fraw[s];
        }
        if (LBMK_MIXED && i == REST) continue;   // rest of the species and mixture sets: below
        Real eqp[M], Dl[M];
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const Real z = RA(s) * T;
#if LBMK_MIXED
            const Real pyz = pe_yz[s], syz = ps_yz[s];
#else
            const Real pyz = sh_yz[(2 * s) * LBMK_BLOCK + threadIdx.x];
            const Real syz = sh_yz[(2 * s + 1) * LBMK_BLOCK + threadIdx.x];
#endif
            const Real pe = psi_c(cx, u[0], u2[0] + z) * pyz;
            const Real pst = psi_c(cx, xs[s][0], xs[s][0] * xs[s][0] + z) * syz;
            eqp[s] = pe;
            Dl[s] = rho * Yl[s] * (pe - pst);
        }
        // species a < M-1: Eq. (finalNumericalEquations) with F_ai of Eq. (fStar)
#pragma unroll
        for (int s = 0; s < M - 1; ++s) {
            Real F = 0;
#pragma unroll
            for (int b = 0; b < M; ++b)
                if (b != s) F += INVWWD(s, b) * Dl[b];
            F *= kappa * Yl[s];
            // in deviations from the rest state (the stored values; the
            // moments of k_pre are summed from them too): f - r relaxes to
            // feq - r, and the result is stored as it is
            // (explicit fma: the same roundings in every kernel this is inlined into)
            const Real feq = fma(rho * Yl[s], eqp[s], -RAWREF(s, i));
            const Real fd = fc[s];
            const Real val = fma(wd[s], eqp[s], fma(bt[s] - (Real)1, F, fma((Real)2 * bt[s], feq - fd, fd)));
            store_raw(a.dst, a, s, i, n, val);
            check += val;
        }
        // mixture f: Eq. (f) with the isotropy correction A_i . X (Eq. (Ai))
        {
            const Real feq = fma(psi_c(cx, u[0], u2[0] + RT), fe_yz, -RAWREF(M - 1, i));
            const Real AX = cx == 0 ? AXyz : (j == 4 ? (Real)0.5 * (Real)cx * X[0] : (Real)0);
            const Real fd = fc[M - 1];
            const Real val = fma(om, feq - fd, fd) + AX;
            store_raw(a.dst, a, M - 1, i, n, val);
            check += val;
        }
    }
#if LBMK_MIXED
    // Rest direction of the species and mixture sets: populations and
    // equilibria in double, the collision increment (small near
    // equilibrium) in float.
    {
        const double *rs = v.rest();
        Real eqp[M], Dl[M];
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const Real z = RA(s) * T;
            const Real pe = ((Real)1 - (u2[0] + z)) * ((Real)1 - (u2[1] + z)) * ((Real)1 - (u2[2] + z));
            const Real pst = ((Real)1 - (xs[s][0] * xs[s][0] + z)) * ((Real)1 - (xs[s][1] * xs[s][1] + z)) *
                             ((Real)1 - (xs[s][2] * xs[s][2] + z));
            eqp[s] = pe;
            Dl[s] = rho * Yl[s] * (pe - pst);
        }
#pragma unroll
        for (int s = 0; s < M - 1; ++s) {
            Real F = 0;
#pragma unroll
            for (int b = 0; b < M; ++b)
                if (b != s) F += INVWWD(s, b) * Dl[b];
            F *= kappa * Yl[s];
            const double f0 = rs[(size_t)s * N + n];
            const Real diff = cvt<Real>(ldd(DR_FEQ0 + s) - f0);
            const double val = f0 + cvt<double>((Real)2 * bt[s] * diff + (bt[s] - (Real)1) * F + wd[s] * eqp[s]);
            store_sf(mc, a.dst, a, s, REST, n, val);
            check += cvt<Real>(val);
        }
        const double f0 = rs[(size_t)(M - 1) * N + n];
        const double val = f0 + cvt<double>(om * cvt<Real>(ldd(DR_FEQ0 + M - 1) - f0));
        store_sf(mc, a.dst, a, M - 1, REST, n, val);
        check += cvt<Real>(val);
    }
#endif
    if (!isfinite(check)) flag(a.status, LBMK_BIT_NONFINITE);
#if LBMK_FUSE_ENERGY
    collide_energy<M>(a, nd);
#endif
}

template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK, LBMK_STEP_MINB) k_step(StepArgs a)
{
    Node nd;
    if (!node_of(nd, a)) return;
    step_node<M>(a, nd);
}

// ---------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------
inline dim3 grid_for(int n, int bs = LBMK_BLOCK) { return dim3((unsigned)((n + bs - 1) / bs)); }

// Launch of one kernel of the step with the context's block size for it
// (LBMK_K_*; the autotuner times them one at a time).
template <int M>
int launch_one(const StepArgs &a, int k)
{
    const int bs = a.bs[k];
    switch (k) {
    case LBMK_K_GHOST:
        if (a.bc_x == 1) {
            const int plane = a.ny * a.nz;
            k_ghost<M><<<grid_for(2 * (a.nseg > 1 ? a.nseg : 1) * plane), LBMK_BLOCK, 0, a.stream>>>(a);
        }
        break;
    case LBMK_K_PRE: k_pre<M><<<grid_for(a.N, bs), bs, 0, a.stream>>>(a); break;
    case LBMK_K_CHEM: {
        if (LBMK_FUSE_CHEM) break;          // the rates are formed inside k_step
        // blocks needing more than 48 KB of dynamic shared memory opt in,
        // once per device (only tuned block sizes do; the default never)
        if (chem_smem<M>(bs) > 48 * 1024) {
            static std::atomic<unsigned long long> opted{0};   // bit d: device d has opted in
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
            if (!(opted.load() >> dev & 1ull)) {
                // idempotent, so two threads racing here both succeed
                const cudaError_t e = cudaFuncSetAttribute(k_chem<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)chem_smem<M>(LBMK_MAXBLOCK));
                if (e != cudaSuccess) return (int)e;
                opted.fetch_or(1ull << dev);
            }
        }
        k_chem<M><<<grid_for(a.N, bs), bs, chem_smem<M>(bs), a.stream>>>(a);
        break;
    }
    case LBMK_K_GRAD: k_grad<M><<<grid_for(a.N, bs), bs, 0, a.stream>>>(a); break;
    case LBMK_K_STEPG:
        if (LBMK_FUSE_ENERGY) break;        // the energy set collides inside k_step
        k_step_g<M><<<grid_for(a.N, bs), bs, 0, a.stream>>>(a);
        break;
    case LBMK_K_STEP: k_step<M><<<grid_for(a.N, bs), bs, 0, a.stream>>>(a); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------
// Persistent step: nsteps time steps of every node in one cooperative
// launch.  Within a phase each warp takes chunks of `chunk` consecutive
// nodes from a queue (one atomic per chunk), so that SMs whose nodes cost
// less (fewer Newton iterations, no flame) take more of them; the phases
// that read a neighbour's value of the same time level -- ghost planes,
// the record (k_pre), G (k_grad), then both collisions -- are separated by
// grid barriers, whose last arrival also resets the queue, and the two
// population buffers swap every step.  A barrier polls at most `cap`
// times: a block that runs out sets LBMK_BIT_BARRIER and returns, and the
// others then run out at the next barrier, so the launch always ends.
// Built only in the units with coherent loads (LBMK_COHERENT_LOADS).
// ---------------------------------------------------------------------
#if LBMK_COHERENT_LOADS
__device__ __forceinline__ bool grid_barrier(GridBarrier *g, unsigned nblocks, unsigned cap, unsigned *status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = &g->gen;
        const unsigned gen = *vgen;                    // read before arriving: only this barrier's last arrival changes it
        __threadfence();
        if (atomicAdd(&g->count, 1u) == nblocks - 1) {
            atomicExch(&g->count, 0u);
            atomicExch(&g->next, 0u);                  // every block is past its last take
            __threadfence();
            atomicAdd(&g->gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == gen) {
                if (++it > cap) {
                    flag(status, LBMK_BIT_BARRIER);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Each warp takes chunks of `chunk` consecutive nodes (a multiple of 32)
// until the queue passes the last node.
template <int M, class Body>
__device__ __forceinline__ void tile_loop(const StepArgs &a, int chunk, unsigned *next, Body &&body)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(next, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        const long long base = (long long)c * chunk;
        if (base >= a.N) break;
        for (int k = lane; k < chunk; k += 32) {
            Node nd;
            nd.n = (int)(base + k);
            if (nd.n >= a.N) break;
            node_at(nd, a);
            body(nd);
        }
    }
}

// One time step of the persistent kernel over the buffers of b.
template <int M>
__device__ __forceinline__ bool persist_step(const StepArgs &b, int tile, GridBarrier *bar, unsigned nb, unsigned cap)
{
    if (b.bc_x == 1) {
        const int ng = 2 * (b.nseg > 1 ? b.nseg : 1) * b.ny * b.nz;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) ghost_node<M>(b, g);
        if (!grid_barrier(bar, nb, cap, b.status)) return false;
    }
    tile_loop<M>(b, tile, &bar->next, [&](const Node &nd) { pre_node<M>(b, nd); });
    if (!grid_barrier(bar, nb, cap, b.status)) return false;
    tile_loop<M>(b, tile, &bar->next, [&](const Node &nd) { grad_node<M>(b, nd); });
    if (!grid_barrier(bar, nb, cap, b.status)) return false;
    // the two collisions read the same inputs and write disjoint sets; the
    // barrier between them only resets the queue, and separate loops keep
    // each one's arithmetic as in its own kernel (no values shared)
    tile_loop<M>(b, tile, &bar->next, [&](const Node &nd) { collide_energy<M>(b, nd); });
    if (!grid_barrier(bar, nb, cap, b.status)) return false;
    tile_loop<M>(b, tile, &bar->next, [&](const Node &nd) { step_node<M>(b, nd); });
    return grid_barrier(bar, nb, cap, b.status);
}

// a0 steps src -> dst, a1 the same with the buffers swapped: the steps
// alternate between the two parameter blocks, which the phases then read
// in place (no per-step copy of the arguments)
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK, LBMK_PRE_MINB) k_persist(StepArgs a0, StepArgs a1, int nsteps, int tile,
                                                                      GridBarrier *bar, unsigned cap)
{
    const unsigned nb = gridDim.x;
    for (int t = 0; t < nsteps; t += 2) {
        if (!persist_step<M>(a0, tile, bar, nb, cap)) return;
        if (t + 1 < nsteps && !persist_step<M>(a1, tile, bar, nb, cap)) return;
    }
}

template <int M>
int run_persistent(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap)
{
    if (nsteps < 1 || tile_mult < 1) return (int)cudaErrorInvalidValue;
    if (!LBMK_FUSE_CHEM) return (int)cudaErrorNotSupported;     // the rates must form inside the collision
    int per_sm = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<M>, LBMK_BLOCK, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int tile = tile_mult * 32;                   // nodes per warp take
    const long long tiles = ((long long)a.N + LBMK_BLOCK - 1) / LBMK_BLOCK;
    const int blocks = (int)std::min<long long>((long long)per_sm * nsm, tiles);
    if (blocks < 1) return (int)cudaErrorInvalidConfiguration;
    StepArgs a0 = a, a1 = a;
    a1.src = a.dst;
    a1.dst = const_cast<void *>(a.src);
    int ns = nsteps, tl = tile;
    GridBarrier *bb = bar;
    unsigned cc = cap;
    void *args[] = {(void *)&a0, (void *)&a1, (void *)&ns, (void *)&tl, (void *)&bb, (void *)&cc};
    return (int)cudaLaunchCooperativeKernel((const void *)k_persist<M>, dim3(blocks), dim3(LBMK_BLOCK), args, 0,
                                            a.stream);
}
#endif  // LBMK_COHERENT_LOADS

template <int M>
int run_step(const StepArgs &a, cudaEvent_t *ev)
{
    for (int k = 0; k < LBMK_NKERNELS; ++k) {
        if (ev) cudaEventRecord(ev[k], a.stream);
        const int e = launch_one<M>(a, k);
        if (e) return e;
    }
    if (ev) cudaEventRecord(ev[LBMK_NKERNELS], a.stream);
    return (int)cudaGetLastError();
}

template <int M>
int run_moments(const StepArgs &a, unsigned mask, double *out)
{
    if (a.bc_x == 1) {
        const int plane = a.ny * a.nz;
        k_ghost<M><<<grid_for(2 * (a.nseg > 1 ? a.nseg : 1) * plane), LBMK_BLOCK, 0, a.stream>>>(a);
    }
    k_moments<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, mask, out);
    return (int)cudaGetLastError();
}

template <int M>
int run_init(const StepArgs &a, const double *X, const double *T, const double *u, double P)
{
    k_init<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, X, T, u, P);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------
// Statistics of an initial state from which the mixed modes choose their
// rest references: per node rho = P m / (r_lat T) (m = sum_a X_a W_a) and
// rho_a = rho X_a W_a / m; over the lattice the minima of rho_a and rho and
// the sums of rho_a, rho and T.  Record of 2M+3 doubles: min rho_a (M),
// min rho, sum rho_a (M), sum rho, sum T.  Two passes with a fixed
// reduction order (LBMK_STAT_BLOCKS partial records, then one block), so
// that the result -- and every state that depends on it -- is the same
// from run to run.
// ---------------------------------------------------------------------
constexpr int LBMK_STAT_THREADS = 256;

__host__ __device__ constexpr int stat_len(int M) { return 2 * M + 3; }

template <int M>
__device__ __forceinline__ void stat_combine(double *acc, const double *o)
{
#pragma unroll
    for (int k = 0; k <= M; ++k) acc[k] = fmin(acc[k], o[k]);
#pragma unroll
    for (int k = M + 1; k < stat_len(M); ++k) acc[k] += o[k];
}

template <int M>
__device__ __forceinline__ void stat_identity(double *acc)
{
#pragma unroll
    for (int k = 0; k <= M; ++k) acc[k] = INFINITY;
#pragma unroll
    for (int k = M + 1; k < stat_len(M); ++k) acc[k] = 0.0;
}

// Tree reduction of the block's records in shared memory (fixed order);
// thread 0 leaves the block's record in sh[0 .. stat_len(M)).
template <int M>
__device__ __forceinline__ void stat_block_reduce(double *acc, double *sh)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < stat_len(M); ++k) sh[k * LBMK_STAT_THREADS + t] = acc[k];
    __syncthreads();
    for (int w = LBMK_STAT_THREADS / 2; w > 0; w >>= 1) {
        if (t < w) {
            double o[stat_len(M)];
#pragma unroll
            for (int k = 0; k < stat_len(M); ++k) o[k] = sh[k * LBMK_STAT_THREADS + t + w];
            stat_combine<M>(acc, o);
#pragma unroll
            for (int k = 0; k < stat_len(M); ++k) sh[k * LBMK_STAT_THREADS + t] = acc[k];
        }
        __syncthreads();
    }
}

template <int M>
__global__ void __launch_bounds__(LBMK_STAT_THREADS) k_stat_partial(StepArgs a, const double *X, const double *T,
                                                                     double P, double *partial)
{
    __shared__ double sh[stat_len(M) * LBMK_STAT_THREADS];
    const MechConst &mc = c_mech[a.slot];
    double acc[stat_len(M)];
    stat_identity<M>(acc);
    for (int n = blockIdx.x * LBMK_STAT_THREADS + threadIdx.x; n < a.N; n += gridDim.x * LBMK_STAT_THREADS) {
        double m = 0.0;
#pragma unroll
        for (int s = 0; s < M; ++s) m += X[(size_t)s * a.N + n] * mc.W[s];
        const double Tn = T[n];
        const double rho = P * m / (mc.r_lat * Tn);
        double o[stat_len(M)];
#pragma unroll
        for (int s = 0; s < M; ++s) {
            const double ra = rho * X[(size_t)s * a.N + n] * mc.W[s] / m;
            o[s] = ra;
            o[M + 1 + s] = ra;
        }
        o[M] = rho;
        o[2 * M + 1] = rho;
        o[2 * M + 2] = Tn;
        stat_combine<M>(acc, o);
    }
    stat_block_reduce<M>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < stat_len(M); ++k) partial[(size_t)k * gridDim.x + blockIdx.x] = sh[k * LBMK_STAT_THREADS];
}

template <int M>
__global__ void __launch_bounds__(LBMK_STAT_THREADS) k_stat_final(const double *partial, int nblocks, double *out)
{
    __shared__ double sh[stat_len(M) * LBMK_STAT_THREADS];
    double acc[stat_len(M)];
    stat_identity<M>(acc);
    for (int b = threadIdx.x; b < nblocks; b += LBMK_STAT_THREADS) {
        double o[stat_len(M)];
#pragma unroll
        for (int k = 0; k < stat_len(M); ++k) o[k] = partial[(size_t)k * nblocks + b];
        stat_combine<M>(acc, o);
    }
    stat_block_reduce<M>(acc, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < stat_len(M); ++k) out[k] = sh[k * LBMK_STAT_THREADS];
}

// scratch: device, at least LBMK_STAT_BLOCKS * (2M+3) doubles; out: device, 2M+3 doubles.
template <int M>
int run_ref_stats(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out)
{
    const int nb = (int)std::min<long long>(LBMK_STAT_BLOCKS, ((long long)a.N + LBMK_STAT_THREADS - 1) /
                                                                  LBMK_STAT_THREADS);
    k_stat_partial<M><<<nb, LBMK_STAT_THREADS, 0, a.stream>>>(a, X, T, P, scratch);
    k_stat_final<M><<<1, LBMK_STAT_THREADS, 0, a.stream>>>(scratch, nb, out);
    return (int)cudaGetLastError();
}


// ---------------------------------------------------------------------
// Heat release rate hdot^c = -sum_a H_a rho_dot_a (Sec. 5b) of the state in
// src (the state lbm_moments reports) and its partial derivatives there.
// With the reaction enthalpy dH_k = sum_a W_a (nu''_ak - nu'_ak) H_a(T),
// hdot^c = -sum_k dH_k q_k, and q_k = F_k (k_f P_f - k_r P_r) with
//   k_f = A_k (T/T_ref)^b_k exp(-theta_k/T),  P_f, P_r the products of the
//   reactant and product concentrations c_a = rho_a / W_a,
//   k_r = k_f / K_c, ln K_c = -sum_a dnu_a g_a/(R_U T) + dn ln(P0/(r T)),
//   F = 1, [M] = sum_a eff_a c_a (third body) or Pr/(1+Pr) with
//   Pr = (k0/k_inf) [M] (Lindemann falloff; A_k is that of k_inf).
// The derivatives are taken at fixed densities (for d/dT) and at fixed
// temperature (for d/drho_a, every one of the M densities independent):
//   d ln k_f/dT = (b + theta/T)/T,
//   d ln K_c/dT = dH_k/(r T^2) - dn/T          (van 't Hoff; d(g_a/RT)/dT = -h_a/(R T^2)),
//   d ln q_k/d ln A_k = 1, or Pr/(1+Pr) for falloff (Pr scales as 1/k_inf),
//   d dH_k/dT = sum_a W_a dnu_a C_p,a.
// Each block sums hdot^c and d hdot^c/d ln A_k over its nodes (grid-stride,
// then a tree in shared memory, in a fixed order); k_hrr_final sums the
// blocks in a fixed order, so that the totals repeat from run to run.
// ---------------------------------------------------------------------


// hdot^c at one node state (T, rho_a) and its derivatives: d/dT into *dT,
// d/drho_a into drho[M], and d/d ln A_k added to dA[k * stride] (k < R).
template <int M, bool WITH_A = true>
__device__ __forceinline__ double hrr_node(const MechConst &mc, double T, const double *rho_a, double *dT_out,
                                           double *drho, double *dA, int stride)
{
    const double invT = 1.0 / T, lnTr = log(T) - mc.log_T_ref;
    const double lnc0 = log(mc.P0_over_r * invT);              // ln(P0/(r T))
    const double vhf = invT * invT / mc.r_lat;                 // 1/(r T^2), van 't Hoff factor
    double conc[M], WH[M], Wcp[M], g[M], dc[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        conc[s] = rho_a[s] * mc.invW[s];
        WH[s] = mc.W[s] * H_spec(mc, s, T);
        Wcp[s] = mc.W[s] * cp_spec(mc, s, T);
        const double *gc = mc.gco[s];
        g[s] = fma(gc[0], 1.0 - log(T),
                   fma(fma(fma(fma(gc[4], T, gc[3]), T, gc[2]), T, gc[1]), T, fma(gc[5], invT, gc[6])));
        dc[s] = 0.0;
    }
    double hdot = 0.0, dT = 0.0;
    for (int k = 0; k < mc.R; ++k) {
        const int nr = mc.nreac[k], np = mc.nprod[k];
        double dH = 0.0, dHdT = 0.0, dG = 0.0, Pf = 1.0, Pp = 1.0;
        for (int j = 0; j < nr; ++j) {
            const int s = mc.reac[k][j];
            dH -= WH[s];
            dHdT -= Wcp[s];
            dG -= g[s];
            Pf *= conc[s];
        }
        for (int j = 0; j < np; ++j) {
            const int s = mc.prod[k][j];
            dH += WH[s];
            dHdT += Wcp[s];
            dG += g[s];
            Pp *= conc[s];
        }
        const double lnkf = fma(mc.b[k], lnTr, fma(-mc.theta[k], invT, mc.log_A[k]));
        const double kf = exp_table(lnkf);
        const double dlnkf = fma(mc.theta[k], invT, mc.b[k]) * invT;
        double kr = 0.0, dlnkr = 0.0;
        if (mc.rev[k]) {
            kr = exp_table(lnkf - fma((double)mc.dn[k], lnc0, -dG));       // k_f / K_c
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
                sA = F;                                     // Pr/(1+Pr)
            }
        }
        const double q = F * q0;
        hdot -= dH * q;
        if constexpr (WITH_A) dA[k * stride] -= dH * q * sA;
        dT -= fma(dHdT, q, dH * fma(F, qf * dlnkf - qr * dlnkr, q0 * dFdT));
        // d q/d c_b: the reactant and product products with one factor left out
        const double wf = -dH * F * kf, wr = dH * F * kr;
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
            const double wm = -dH * q0 * dFdcM;
#pragma unroll
            for (int s = 0; s < M; ++s) dc[s] = fma(wm, mc.eff[k][s], dc[s]);
        }
    }
    *dT_out = dT;
#pragma unroll
    for (int s = 0; s < M; ++s) drho[s] = dc[s] * mc.invW[s];      // c_a = rho_a / W_a
    return hdot;
}

template <int M>
__global__ void __launch_bounds__(LBMK_HRR_THREADS, 3) k_hrr(StepArgs a, double *dT_out, double *drho_out,
                                                          double *partial)
{
    __shared__ double sh_dA[LBMK_MAXR * LBMK_HRR_THREADS];
    __shared__ double sh_J[LBMK_HRR_THREADS];
    const MechConst &mc = c_mech[a.slot];
    const int t = threadIdx.x, R = mc.R;
    const size_t N = a.N;
    for (int k = 0; k < R; ++k) sh_dA[k * LBMK_HRR_THREADS + t] = 0.0;
    double Jt = 0.0;
    for (int n = blockIdx.x * LBMK_HRR_THREADS + t; n < a.N; n += gridDim.x * LBMK_HRR_THREADS) {
        Node nd;
        nd.n = n;
        node_at(nd, a);
        PullIdx p;
        make_pull(p, nd, a);
        double rho_a[M];
        Real ja[M][3];
        Sums sm;
        pull_moments<M, false>(mc, a, p, n, rho_a, ja, sm);
        // the node state as in k_moments
        const double rho = sm.rho;
        double rest = 0.0;
#pragma unroll
        for (int s = 0; s < M - 1; ++s) rest += rho_a[s];
        rho_a[M - 1] = rho - rest;
        double Y[M];
#pragma unroll
        for (int s = 0; s < M; ++s) Y[s] = rho_a[s] / rho;
        const double u[3] = {sm.j[0] / rho, sm.j[1] / rho, sm.j[2] / rho};
        const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double eu[6];
        mixture_energy_poly<M>(mc, Y, eu);
        const double T = solve_T(eu, sm.rhoE / rho - 0.5 * usq, a.macro[DR_T * N + n], a.status);
        double dT, drho[M];
        Jt += hrr_node<M>(mc, T, rho_a, &dT, drho, sh_dA + t, LBMK_HRR_THREADS);
        if (dT_out) dT_out[n] = dT;
        if (drho_out)
#pragma unroll
            for (int s = 0; s < M; ++s) drho_out[(size_t)s * N + n] = drho[s];
    }
    sh_J[t] = Jt;
    __syncthreads();
    for (int w = LBMK_HRR_THREADS / 2; w > 0; w >>= 1) {
        if (t < w) {
            sh_J[t] += sh_J[t + w];
            for (int k = 0; k < R; ++k) sh_dA[k * LBMK_HRR_THREADS + t] += sh_dA[k * LBMK_HRR_THREADS + t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        double *o = partial + (size_t)blockIdx.x * (1 + R);
        o[0] = sh_J[0];
        for (int k = 0; k < R; ++k) o[1 + k] = sh_dA[k * LBMK_HRR_THREADS];
    }
}

// The chemistry of n given node states (rho_a [M][n], T [n]; device): the
// step's production rates (molar_production, as k_chem evaluates them) and
// hdot^c with its derivatives (hrr_node); each output may be null.
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_chem_at(StepArgs a, int n, const double *rho_in, const double *T_in,
                                                        double *rho_dot, double *hdot, double *dT_out,
                                                        double *drho_out, double *dA_out)
{
    __shared__ double sh_act[M * LBMK_BLOCK];
    __shared__ double sh_g[M * LBMK_BLOCK];
    __shared__ WReal sh_w[M * LBMK_BLOCK];
    const MechConst &mc = c_mech[a.slot];
    const int t = threadIdx.x, i = blockIdx.x * LBMK_BLOCK + t;
    if (i >= n) return;
    double rho_a[M], conc[M];
#pragma unroll
    for (int s = 0; s < M; ++s) {
        rho_a[s] = rho_in[(size_t)s * n + i];
        conc[s] = rho_a[s] * mc.invW[s];
    }
    const double T = T_in[i];
    if (rho_dot) {
        molar_production<M>(mc, T, conc, sh_act, sh_g, sh_w, t, LBMK_BLOCK);
#pragma unroll
        for (int s = 0; s < M; ++s) rho_dot[(size_t)s * n + i] = mc.W[s] * (double)sh_w[s * LBMK_BLOCK + t];
    }
    if (hdot || dT_out || drho_out || dA_out) {
        double dT, drho[M], dA[LBMK_MAXR];
        for (int k = 0; k < mc.R; ++k) dA[k] = 0.0;
        const double h = hrr_node<M>(mc, T, rho_a, &dT, drho, dA, 1);
        if (hdot) hdot[i] = h;
        if (dT_out) dT_out[i] = dT;
        if (drho_out)
#pragma unroll
            for (int s = 0; s < M; ++s) drho_out[(size_t)s * n + i] = drho[s];
        if (dA_out)
            for (int k = 0; k < mc.R; ++k) dA_out[(size_t)k * n + i] = dA[k];
    }
}

// Temperatures of n given node states (Y [M][n], specific internal energy
// e [n], Newton starting points T0 [n]; device) by the step's Newton
// iteration (mixture_energy_poly, solve_T).
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_temperature_at(StepArgs a, int n, const double *Y_in,
                                                               const double *e_in, const double *T0_in,
                                                               double *T_out)
{
    const MechConst &mc = c_mech[a.slot];
    const int i = blockIdx.x * LBMK_BLOCK + threadIdx.x;
    if (i >= n) return;
    double Y[M], eu[6];
#pragma unroll
    for (int s = 0; s < M; ++s) Y[s] = Y_in[(size_t)s * n + i];
    mixture_energy_poly<M>(mc, Y, eu);
    T_out[i] = solve_T(eu, e_in[i], T0_in[i], a.status);
}

// Column c of nb partial records of width w, summed in a fixed order.
__global__ void __launch_bounds__(LBMK_HRR_THREADS) k_hrr_final(const double *partial, int nb, int w, double *out)
{
    __shared__ double sh[LBMK_HRR_THREADS];
    const int t = threadIdx.x, c = blockIdx.x;
    double acc = 0.0;
    for (int b = t; b < nb; b += LBMK_HRR_THREADS) acc += partial[(size_t)b * w + c];
    sh[t] = acc;
    __syncthreads();
    for (int h = LBMK_HRR_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) sh[t] += sh[t + h];
        __syncthreads();
    }
    if (t == 0) out[c] = sh[0];
}

// partial: hrr_blocks(N) (1 + R) doubles; out: 1 + R doubles
// {sum hdot^c, sum d hdot^c/d ln A_k}.
template <int M>
int run_hrr(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out)
{
    if (a.bc_x == 1) {
        const int plane = a.ny * a.nz;
        k_ghost<M><<<grid_for(2 * (a.nseg > 1 ? a.nseg : 1) * plane), LBMK_BLOCK, 0, a.stream>>>(a);
    }
    const int nb = lbmk::hrr_blocks(a.N);
    k_hrr<M><<<nb, LBMK_HRR_THREADS, 0, a.stream>>>(a, dT, drho, partial);
    k_hrr_final<<<1 + R, LBMK_HRR_THREADS, 0, a.stream>>>(partial, nb, 1 + R, out);
    return (int)cudaGetLastError();
}

template <int M>
int run_chem_at(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                double *dT, double *drho, double *dA)
{
    if (n > 0)
        k_chem_at<M><<<grid_for(n), LBMK_BLOCK, 0, a.stream>>>(a, n, rho_a, T, rho_dot, hdot, dT, drho, dA);
    return (int)cudaGetLastError();
}

template <int M>
int run_temperature_at(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T)
{
    if (n > 0) k_temperature_at<M><<<grid_for(n), LBMK_BLOCK, 0, a.stream>>>(a, n, Y, e, T0, T);
    return (int)cudaGetLastError();
}


// ---------------------------------------------------------------------
// Gradient of J = sum_nodes hdot^c with respect to the stored populations
// F of the current state (periodic lattices), the source term of the
// objective in an adjoint of the step.  Node n pulls P_si(n) = F_si(n - c_i)
// and forms rho_a (a < M-1), rho, j and rho E from the pulled sets; the
// slaved density is rho - sum_a rho_a, Y_a = rho_a / rho, and T solves
// sum_a Y_a U_a(T) = e with e = rho E / rho - |j|^2 / (2 rho^2).  By the
// implicit function theorem dT = (de - sum_a U_a dY_a) / C_v.  With
// G_T = d hdot/dT and G_a = d hdot/d rho_a (hrr_node) and l = G_T / C_v:
//   d hdot/d rho_s = G_s - G_{M-1} - l (U_s - U_{M-1}) / rho   (s < M-1)
//   d hdot/d rho   = G_{M-1} + l (de/drho - (U_{M-1} - sum_a Y_a U_a) / rho),
//                    de/drho = -rho E / rho^2 + |j|^2 / rho^3
//   d hdot/d j_d   = -l u_d / rho,      d hdot/d (rho E) = l / rho,
// and dJ/dF_si(x) is the value of node x + c_i for its set (for f:
// d/drho + c_i . d/dj).
// ---------------------------------------------------------------------

// adj [M + 4][N]: d hdot/d rho_s (s < M-1), d/d rho, d/d j (3), d/d rho E.
template <int M>
__global__ void __launch_bounds__(LBMK_HRR_THREADS, 3) k_hrr_adj(StepArgs a, double *adj)
{
    const MechConst &mc = c_mech[a.slot];
    const int n = blockIdx.x * LBMK_HRR_THREADS + threadIdx.x;
    if (n >= a.N) return;
    const size_t N = a.N;
    Node nd;
    nd.n = n;
    node_at(nd, a);
    PullIdx p;
    make_pull(p, nd, a);
    double rho_a[M];
    Real ja[M][3];
    Sums sm;
    pull_moments<M, false>(mc, a, p, n, rho_a, ja, sm);
    const double rho = sm.rho;
    double rest = 0.0;
#pragma unroll
    for (int s = 0; s < M - 1; ++s) rest += rho_a[s];
    rho_a[M - 1] = rho - rest;
    double Y[M];
#pragma unroll
    for (int s = 0; s < M; ++s) Y[s] = rho_a[s] / rho;
    const double u[3] = {sm.j[0] / rho, sm.j[1] / rho, sm.j[2] / rho};
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double eu[6];
    mixture_energy_poly<M>(mc, Y, eu);
    const double T = solve_T(eu, sm.rhoE / rho - 0.5 * usq, a.macro[DR_T * N + n], a.status);
    double GT, G[M];
    hrr_node<M, false>(mc, T, rho_a, &GT, G, nullptr, 0);
    const double l = GT / dpoly5(eu, T), ir = 1.0 / rho;
    double U[M], Umix = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        U[s] = poly5(mc.uco[s], T);
        Umix = fma(Y[s], U[s], Umix);
    }
#pragma unroll
    for (int s = 0; s < M - 1; ++s) adj[(size_t)s * N + n] = G[s] - G[M - 1] - l * (U[s] - U[M - 1]) * ir;
    const double jsq = sm.j[0] * sm.j[0] + sm.j[1] * sm.j[1] + sm.j[2] * sm.j[2];
    const double dedrho = (jsq * ir - sm.rhoE) * ir * ir;
    adj[(size_t)(M - 1) * N + n] = G[M - 1] + l * (dedrho - (U[M - 1] - Umix) * ir);
#pragma unroll
    for (int d = 0; d < 3; ++d) adj[(size_t)(M + d) * N + n] = -l * u[d] * ir;
    adj[(size_t)(M + 3) * N + n] = l * ir;
}

// dJ/dF of set s (0..M), out [27][N]: each direction gathers from x + c_i.
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_hrr_adj_gather(StepArgs a, const double *adj, int s, double *out)
{
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    StencilIdx st;
    make_stencil(st, nd, a);
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        const size_t nb = nb_of<I>(st, a);
        double v;
        if (s < M - 1) {
            v = adj[(size_t)s * N + nb];
        } else if (s == M - 1) {
            v = adj[(size_t)(M - 1) * N + nb];
            if (CX(I)) v += CX(I) * adj[(size_t)M * N + nb];
            if (CY(I)) v += CY(I) * adj[(size_t)(M + 1) * N + nb];
            if (CZ(I)) v += CZ(I) * adj[(size_t)(M + 2) * N + nb];
        } else {
            v = adj[(size_t)(M + 3) * N + nb];
        }
        out[(size_t)I * N + nd.n] = v;
    });
}

template <int M>
int run_hrr_adj(const StepArgs &a, double *adj)
{
    k_hrr_adj<M><<<grid_for(a.N, LBMK_HRR_THREADS), LBMK_HRR_THREADS, 0, a.stream>>>(a, adj);
    return (int)cudaGetLastError();
}

template <int M>
int run_hrr_adj_gather(const StepArgs &a, const double *adj, int s, double *out)
{
    k_hrr_adj_gather<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, adj, s, out);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------
// Flame diagnostics of the circular expanding flame (Sec. 5b), from the
// record k_pre forms for the current state:
//   S_d = [ hdot^c + div(lambda grad T) - rho (sum_a C_a,p Y_a du_a) . grad T ]
//         / (rho C_p |grad T|)                                   (Eq. (sd))
//   S_a = S_d + u . n,  n = -grad T / |grad T|,
// lambda = (1/omega_1 - 1/2) P C_p (Eq. (lambda)), C_p = sum_a Y_a C_a,p,
// the gradients by the isotropic stencil (the divergence as the sum of the
// component derivatives of lambda grad T).  Pass 1 forms grad T and
// lambda grad T (scratch [6][N]); pass 2 the rest.  S_d = S_a = 0 where
// grad T = 0.
// ---------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(LBMK_BLOCK) k_flame1(StepArgs a, double *scr)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const int n = nd.n;
    const RecRows rr = rec_rows(M);
    const Real *R = rec(a);
    const double *Tr = a.macro + (size_t)DR_T * N;
    StencilIdx st;
    make_stencil(st, nd, a);
    double g[3] = {0.0, 0.0, 0.0};
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        if constexpr (I != REST) {
            const double t = Tr[nb_of<I>(st, a)];
            if (CX(I)) g[0] = fma(WI(I) * CX(I), t, g[0]);
            if (CY(I)) g[1] = fma(WI(I) * CY(I), t, g[1]);
            if (CZ(I)) g[2] = fma(WI(I) * CZ(I), t, g[2]);
        }
    });
    const double T = Tr[n];
    double Cp = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) Cp = fma((double)R[(size_t)(rr.y + s) * N + n], cp_spec(mc, s, T), Cp);
    const double lam = (1.0 / (double)R[(size_t)rr.om1 * N + n] - 0.5) * (double)R[(size_t)rr.p * N + n] * Cp;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        scr[(size_t)d * N + n] = 3.0 * g[d];
        scr[(size_t)(3 + d) * N + n] = lam * 3.0 * g[d];
    }
}

template <int M>
__global__ void __launch_bounds__(LBMK_HRR_THREADS) k_flame2(StepArgs a, const double *scr, double *Sd, double *Sa)
{
    const MechConst &mc = c_mech[a.slot];
    Node nd;
    if (!node_of(nd, a)) return;
    const size_t N = a.N;
    const int n = nd.n;
    const RecRows rr = rec_rows(M);
    const Real *R = rec(a);
    StencilIdx st;
    make_stencil(st, nd, a);
    double div = 0.0;
    for_dirs<0, LBMK_Q>([&](auto dd) {
        constexpr int I = decltype(dd)::value;
        if constexpr (I != REST) {
            const size_t nb = nb_of<I>(st, a);
            if (CX(I)) div = fma(WI(I) * CX(I), scr[(size_t)3 * N + nb], div);
            if (CY(I)) div = fma(WI(I) * CY(I), scr[(size_t)4 * N + nb], div);
            if (CZ(I)) div = fma(WI(I) * CZ(I), scr[(size_t)5 * N + nb], div);
        }
    });
    div *= 3.0;
    const double T = a.macro[(size_t)DR_T * N + n];
    const double rho = (double)R[(size_t)rr.rho * N + n];
    double rho_a[M], Y[M], fl[3] = {0.0, 0.0, 0.0}, Cp = 0.0;
#pragma unroll
    for (int s = 0; s < M; ++s) {
        Y[s] = (double)R[(size_t)(rr.y + s) * N + n];
        rho_a[s] = rho * Y[s];
        const double cpy = cp_spec(mc, s, T) * Y[s];
        Cp += cpy;
#pragma unroll
        for (int d = 0; d < 3; ++d) fl[d] = fma(cpy, (double)R[(size_t)(rr.du + 3 * s + d) * N + n], fl[d]);
    }
    double dT, drho[M];
    const double hdot = hrr_node<M, false>(mc, T, rho_a, &dT, drho, nullptr, 0);
    const double g[3] = {scr[n], scr[N + n], scr[2 * N + n]};
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn == 0.0) {
        Sd[n] = Sa[n] = 0.0;
        return;
    }
    const double num = hdot + div - rho * (fl[0] * g[0] + fl[1] * g[1] + fl[2] * g[2]);
    const double sd = num / (rho * Cp * gn);
    double un = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) un -= (double)R[(size_t)(rr.u + d) * N + n] * g[d];
    Sd[n] = sd;
    Sa[n] = sd + un / gn;
}

template <int M>
int run_flame_speeds(const StepArgs &a, double *scr, double *Sd, double *Sa)
{
    int e = 0;
    if (a.bc_x == 1) e = launch_one<M>(a, LBMK_K_GHOST);
    if (!e) e = launch_one<M>(a, LBMK_K_PRE);
    if (e) return e;
    k_flame1<M><<<grid_for(a.N), LBMK_BLOCK, 0, a.stream>>>(a, scr);
    k_flame2<M><<<grid_for(a.N, LBMK_HRR_THREADS), LBMK_HRR_THREADS, 0, a.stream>>>(a, scr, Sd, Sa);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------
// Means along the isoline T = T_iso in the plane z = 0 (Eq. (rmean)):
// marching squares, one thread per cell (x, y)..(x+1, y+1) of the periodic
// x-y lattice: crossings where T - T_iso changes sign (T >= T_iso counts as
// above) at the linear interpolation point along the cell edge, with the K
// fields interpolated alike; two crossings make one straight segment, four
// are split by the mean of the corners; each segment adds its length and
// its length times the mean of its ends' distance from (cx, cy) and field
// values.  Per-block sums in a fixed order: partial [blocks][2 + K].
// ---------------------------------------------------------------------
#define LBMK_ISO_MAXK 8
__global__ void __launch_bounds__(LBMK_HRR_THREADS) k_isoline(int nx, int ny, int N, const double *T, double T_iso,
                                                               double cx, double cy, int K, const double *fields,
                                                               double *partial)
{
    __shared__ double sh[(2 + LBMK_ISO_MAXK) * LBMK_HRR_THREADS];
    const int t = threadIdx.x, W = 2 + K;
    double acc[2 + LBMK_ISO_MAXK];
    for (int k = 0; k < W; ++k) acc[k] = 0.0;
    const int cell = blockIdx.x * LBMK_HRR_THREADS + t;
    if (cell < nx * ny) {
        const int x = cell % nx, y = cell / nx;
        const int ox[4] = {0, 1, 1, 0}, oy[4] = {0, 0, 1, 1};
        int idx[4];
        double v[4];
        for (int c = 0; c < 4; ++c) {
            idx[c] = (x + ox[c]) % nx + nx * ((y + oy[c]) % ny);
            v[c] = T[idx[c]];
        }
        double px[4], py[4], pf[4][LBMK_ISO_MAXK];
        int ne = 0;
        for (int e = 0; e < 4; ++e) {
            const int aa = e, bb = (e + 1) % 4;
            if ((v[aa] >= T_iso) == (v[bb] >= T_iso)) continue;
            const double f = (T_iso - v[aa]) / (v[bb] - v[aa]);
            px[ne] = x + ox[aa] + f * (ox[bb] - ox[aa]);
            py[ne] = y + oy[aa] + f * (oy[bb] - oy[aa]);
            for (int k = 0; k < K; ++k) {
                const double fa = fields[(size_t)k * N + idx[aa]], fb = fields[(size_t)k * N + idx[bb]];
                pf[ne][k] = fa + f * (fb - fa);
            }
            ++ne;
        }
        int pr[2][2] = {{0, 1}, {2, 3}}, np = ne == 2 ? 1 : (ne == 4 ? 2 : 0);
        if (ne == 4) {
            const double vc = 0.25 * (v[0] + v[1] + v[2] + v[3]);
            if ((vc >= T_iso) != (v[0] >= T_iso)) {       // corners 0 and 2 cut off
                pr[0][0] = 3; pr[0][1] = 0; pr[1][0] = 1; pr[1][1] = 2;
            }
        }
        for (int q = 0; q < np; ++q) {
            const int i = pr[q][0], j = pr[q][1];
            const double L = sqrt((px[i] - px[j]) * (px[i] - px[j]) + (py[i] - py[j]) * (py[i] - py[j]));
            const double Ri = sqrt((px[i] - cx) * (px[i] - cx) + (py[i] - cy) * (py[i] - cy));
            const double Rj = sqrt((px[j] - cx) * (px[j] - cx) + (py[j] - cy) * (py[j] - cy));
            acc[0] += L;
            acc[1] += L * 0.5 * (Ri + Rj);
            for (int k = 0; k < K; ++k) acc[2 + k] += L * 0.5 * (pf[i][k] + pf[j][k]);
        }
    }
    for (int k = 0; k < W; ++k) sh[k * LBMK_HRR_THREADS + t] = acc[k];
    __syncthreads();
    for (int h = LBMK_HRR_THREADS / 2; h > 0; h >>= 1) {
        if (t < h)
            for (int k = 0; k < W; ++k) sh[k * LBMK_HRR_THREADS + t] += sh[k * LBMK_HRR_THREADS + t + h];
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < W; ++k) partial[(size_t)blockIdx.x * W + k] = sh[k * LBMK_HRR_THREADS];
}

}  // namespace

#define LBMK_DISPATCH(M_, CALL)                     \
    switch (M_) {                                   \
    case 2: return CALL(2);                         \
    case 3: return CALL(3);                         \
    case 9: return CALL(9);                         \
    default: return (int)cudaErrorInvalidValue;     \
    }
