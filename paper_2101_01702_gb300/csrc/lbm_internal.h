// Internal declarations shared by the C-ABI translation unit and the two
// kernel translation units (double and mixed precision).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#define LBMK_MAXM 12
#define LBMK_MAXS (LBMK_MAXM + 1)
#define LBMK_MAXR 32
#define LBMK_SLOTS 4
#define LBMK_Q 27

// Status bits the kernels set in the device status word.
#define LBMK_BIT_NEWTON 1u
#define LBMK_BIT_NONFINITE 2u
#define LBMK_BIT_NEGATIVE 4u
#define LBMK_BIT_PIVOT 8u

// Row offsets of the per-node macroscopic record (double, [rows][N]).
#define MAC_T 0
#define MAC_NUP 1
#define MAC_PHI 2
#define MAC_G 5
#define MAC_Y 8

// Everything the kernels read from constant memory for one context.
struct MechConst {
    int M, R, thermo, visc_model;
    double T0, nu, Pr, r_lat, log_T_ref, log_P0_over_r;
    double W[LBMK_MAXM], invW[LBMK_MAXM], Ra[LBMK_MAXM];
    double U0[LBMK_MAXM], cv[LBMK_MAXM], cpR[LBMK_MAXM];     // constant-cp thermodynamics
    double poly[LBMK_MAXM][7];                              // polynomial thermodynamics
    double inv_WWD[LBMK_MAXM][LBMK_MAXM];                   // 1 / (W_a W_b D_ab)
    float inv_WWD_f[LBMK_MAXM][LBMK_MAXM];
    int rtype[LBMK_MAXR], rev[LBMK_MAXR];
    int nreac[LBMK_MAXR], nprod[LBMK_MAXR];
    int reac[LBMK_MAXR][3], prod[LBMK_MAXR][3];             // species of each molecule
    int ndnu[LBMK_MAXR], dnu_sp[LBMK_MAXR][6], dnu_v[LBMK_MAXR][6];
    double dn[LBMK_MAXR];
    double log_A[LBMK_MAXR], b[LBMK_MAXR], theta[LBMK_MAXR], low[LBMK_MAXR][3];
    double eff[LBMK_MAXR][LBMK_MAXM];
    // Mixed precision: stored value = population - ref[s][i]; the rest
    // state of set s at (rho_ref, zeta_ref).  m0 = sum_i ref, m2 = sum_i
    // ref c_alpha^2 (first and mixed second moments vanish by symmetry).
    float ref[LBMK_MAXS][LBMK_Q];
    double ref_m0[LBMK_MAXS];
    double ref_m2[LBMK_MAXS];
};

struct StepArgs {
    int slot, M, nx, ny, nz, N, bc_x;
    const void *src;     // populations read (pull)
    void *dst;           // populations written
    double *macro;
    void *ghost;
    unsigned *status;
    cudaStream_t stream;
};

// Kernel translation units (one per storage precision).  Each returns a
// cudaError_t value (0 on success).
namespace lbmk {
int upload_fp64(int slot, const MechConst &mc, cudaStream_t s);
int upload_mixed(int slot, const MechConst &mc, cudaStream_t s);

int init_fp64(const StepArgs &a, const double *X, const double *T, const double *u, double P);
int init_mixed(const StepArgs &a, const double *X, const double *T, const double *u, double P);

// one full time step src -> dst (ghost, moments, gradients, collision);
// with ev != nullptr, events ev[0..4] are recorded around the four phases
int step_fp64(const StepArgs &a, cudaEvent_t *ev = nullptr);
int step_mixed(const StepArgs &a, cudaEvent_t *ev = nullptr);

// macroscopic fields of the state in src, written to out (device)
int moments_fp64(const StepArgs &a, unsigned mask, double *out);
int moments_mixed(const StepArgs &a, unsigned mask, double *out);
}  // namespace lbmk
