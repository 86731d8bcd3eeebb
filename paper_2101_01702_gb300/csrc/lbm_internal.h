// Internal declarations shared by the C-ABI translation unit and the kernel
// translation units (double, mixed precision, fixed scratch).
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
#define LBMK_BIT_BOUNDS 16u     // checked builds: an index derived from the geometry left its buffer
#define LBMK_BIT_BARRIER 32u    // the persistent step: a grid barrier gave up waiting (its poll limit ran out)

// Grid-wide barrier state of the persistent step (device, zeroed before a
// launch): blocks that have arrived, the generation they wait to change,
// and the next chunk of nodes the current phase hands out.
struct GridBarrier {
    unsigned count, gen, next;
};

// Per-node record in the macro buffer: macro_double_rows(M) rows of
// doubles, then rec_rows(M).total rows of the storage type (float in mixed
// precision, double otherwise), each row [N].
// Double rows:
//   DR_T      temperature (Newton starting point and result)
//   DR_FEQ0   rest-direction equilibrium of the species and mixture sets (M)
//   DR_GE     rho E            DR_GQ  q^eq (3)       DR_GR  R^eq - rho E theta I (6: xx yy zz xy xz yz)
//   DR_GTR    tr(R^eq - rho E theta I) / 3
// Storage-type rows:
//   nup  1/omega - 1/2      phi  Phi (3)        g    G (3)
//   y    Y_a (M)            rho  rho            u    u (3)
//   du   du_a (3M, a-major) wd   rho_dot_a (M; written only by k_chem)  beta beta_a (M)
//   kappa m R_U T           rt   R T            om   omega      om1 omega_1
//   p    P                  dq   (omega - omega_1)(q* - q^eq) without the grad-Y part (3)
//   h    H_a (M)
#define DR_T 0
#define DR_FEQ0 1
__host__ __device__ constexpr int dr_ge(int M) { return M + 1; }
__host__ __device__ constexpr int dr_gq(int M) { return M + 2; }
__host__ __device__ constexpr int dr_gr(int M) { return M + 5; }
__host__ __device__ constexpr int dr_gtr(int M) { return M + 11; }
__host__ __device__ constexpr int macro_double_rows(int M) { return M + 12; }
struct RecRows {
    int nup, phi, g, y, rho, u, du, wd, beta, kappa, rt, om, om1, p, dq, h, total;
};
__host__ __device__ constexpr RecRows rec_rows(int M)
{
    return RecRows{0, 1, 4, 7, 7 + M, 8 + M, 11 + M, 11 + 4 * M, 11 + 5 * M, 11 + 6 * M, 12 + 6 * M, 13 + 6 * M,
                   14 + 6 * M, 15 + 6 * M, 16 + 6 * M, 19 + 6 * M, 19 + 7 * M};
}
// Bytes of the macro buffer for N nodes, M species and a storage element size.
__host__ __device__ constexpr size_t macro_bytes_for(int M, size_t N, size_t real_size)
{
    return (size_t)macro_double_rows(M) * N * sizeof(double) + (size_t)rec_rows(M).total * N * real_size;
}

// Population buffer.
//   Double precision: [S][27][N] doubles (S = M + 1 sets: species 0..M-2,
//   mixture f, energy g).
//   Mixed precision: the M species and mixture sets as float deviations
//   [M][27][N] (the rest slot unused), then at a 16-byte boundary their rest
//   populations [M][N] in double, then the energy set g [27][N] in double.
//   On the low-temperature lattice the rest population carries most of a
//   set's mass (a factor 1 - R T per axis), and the energy populations fix
//   the temperature that the Arrhenius rates amplify, so these stay double.
// Ghost planes (x faces): [2 G][S][27][ny nz] doubles in both precisions,
// G lattices side by side in x (plane 2k: left face of lattice k, 2k+1:
// right face).
__host__ __device__ constexpr size_t pop_float_bytes(int M, size_t N) { return ((size_t)M * 27 * N * 4 + 15) & ~(size_t)15; }
__host__ __device__ constexpr size_t pop_bytes_for(int S, size_t N, bool mixed)
{
    return mixed ? pop_float_bytes(S - 1, N) + (size_t)(S - 1) * N * sizeof(double) + (size_t)27 * N * sizeof(double)
                 : (size_t)S * 27 * N * sizeof(double);
}
__host__ __device__ constexpr size_t ghost_bytes_for(int S, size_t plane, int nlat = 1)
{
    return 2 * (size_t)nlat * S * 27 * plane * sizeof(double);
}

// Everything the kernels read from constant memory for one context.
//   H_a(T) = sum_k hco[a][k] T^(k+1) (k = 0..4) + hco[a][5]
//   U_a(T) = sum_k uco[a][k] T^k (k = 0..5)              (U_a = H_a - R_a T)
//   g_a/(R_U T) = gco0 (1 - ln T) + gco1 T + gco2 T^2 + gco3 T^3 + gco4 T^4
//                 + gco5 / T + gco6
// Both the constant-cp and the 7-coefficient thermodynamics map onto these.
struct MechConst {
    int M, R;
    int visc_model;
    double T0, nu, Pr, r_lat, log_T_ref, P0_over_r;
    double W[LBMK_MAXM], invW[LBMK_MAXM], Ra[LBMK_MAXM];
    float Ra_f[LBMK_MAXM];
    double hco[LBMK_MAXM][6], uco[LBMK_MAXM][6], gco[LBMK_MAXM][7];
    double inv_WWD[LBMK_MAXM][LBMK_MAXM];                   // 1 / (W_a W_b D_ab), 0 on the diagonal
    float inv_WWD_f[LBMK_MAXM][LBMK_MAXM];
    int rtype[LBMK_MAXR], rev[LBMK_MAXR];
    int nreac[LBMK_MAXR], nprod[LBMK_MAXR];
    int reac[LBMK_MAXR][3], prod[LBMK_MAXR][3];             // species of each molecule
    int dn[LBMK_MAXR];                                      // sum of product minus reactant coefficients
    double log_A[LBMK_MAXR], b[LBMK_MAXR], theta[LBMK_MAXR];
    double dlow[LBMK_MAXR][3];                              // falloff: ln(A0/A), b0 - b, theta0 - theta
    double eff[LBMK_MAXR][LBMK_MAXM];
    // Mixture-averaged transport (transport = 1): species viscosity law,
    // Wilke's mass factors wq[a][b] = (W_b/W_a)^(1/4) and
    // wd[a][b] = (8 (1 + W_a/W_b))^(-1/2), 5/4 R_a for Eucken's relation, and
    // the diffusivity law (T/T_tr)^D_exp (P_tr/P).
    int transport;
    double mu0[LBMK_MAXM], mu_exp[LBMK_MAXM], eucken[LBMK_MAXM];
    double wq[LBMK_MAXM][LBMK_MAXM], wd[LBMK_MAXM][LBMK_MAXM];
    double log_T_tr, D_exp, P_tr;
    // Mixed precision: stored float value = population - ref[s][i] for the
    // moving directions of the species and mixture sets (s < M); ref is a
    // rest state of set s (zero in the rest slot, which is not used).
    float ref[LBMK_MAXS][LBMK_Q];
    // Moments of each set's rest state ref (exact sums in double): the
    // zeroth moment and the diagonal of the second; the first moments and
    // the off-diagonal second moments vanish by symmetry.  The mixed units
    // sum the stored deviations and add these once.
    double ref0[LBMK_MAXS], refP[LBMK_MAXS][3];
};

// Fills mc.ref0 and mc.refP from mc.ref (M species and mixture sets).
inline void lbmk_reference_moments(MechConst &mc, int M)
{
    for (int s = 0; s < M; ++s) {
        double z = 0.0, p[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < LBMK_Q; ++i) {
            const double r = (double)mc.ref[s][i];
            const int c[3] = {i % 3 - 1, (i / 3) % 3 - 1, i / 9 - 1};
            z += r;
            for (int d = 0; d < 3; ++d) p[d] += c[d] * c[d] * r;
        }
        mc.ref0[s] = z;
        for (int d = 0; d < 3; ++d) mc.refP[s][d] = p[d];
    }
}

#define LBMK_BLOCK 128      // default block; the block of k_pre and k_step is at most this
#define LBMK_MAXBLOCK 256   // largest block of the kernels tuned up to it (k_grad, k_step_g; k_chem)

// The kernels of one step, in launch order (timing phases and autotuned
// block sizes are indexed alike).
enum { LBMK_K_GHOST = 0, LBMK_K_PRE, LBMK_K_CHEM, LBMK_K_GRAD, LBMK_K_STEPG, LBMK_K_STEP, LBMK_NKERNELS };

struct StepArgs {
    int slot, M, nx, ny, nz, N, bc_x;
    int bs[LBMK_NKERNELS];   // threads per block of each kernel
    // Lattices side by side in x (nseg >= 2): per x coordinate its lattice's
    // x range and index {x0, x1, k, 0}; per lattice its range {x0, x1}.
    // Null for one lattice (x0 = 0, x1 = nx, k = 0).
    int nseg;
    const int4 *xseg;
    const int2 *segs;
    const void *src;     // populations read (pull)
    void *dst;           // populations written
    double *macro;       // double rows, then the storage-type record rows
    void *ghost;
    unsigned *status;
    cudaStream_t stream;
};

// Kernel translation units (one per storage precision).  Each returns a
// cudaError_t value (0 on success).
namespace lbmk {
int upload_fp64(int slot, const MechConst &mc, cudaStream_t s);
int upload_mixed(int slot, const MechConst &mc, cudaStream_t s);
int upload_mixed_fast(int slot, const MechConst &mc, cudaStream_t s);

int init_fp64(const StepArgs &a, const double *X, const double *T, const double *u, double P);
int init_mixed(const StepArgs &a, const double *X, const double *T, const double *u, double P);
int init_mixed_fast(const StepArgs &a, const double *X, const double *T, const double *u, double P);

// one full time step src -> dst (ghost, moments, production rates,
// gradients, energy collision, species/mixture collision); with ev !=
// nullptr, events ev[0..6] are recorded around the six phases
int step_fp64(const StepArgs &a, cudaEvent_t *ev = nullptr);
int step_mixed(const StepArgs &a, cudaEvent_t *ev = nullptr);
int step_mixed_fast(const StepArgs &a, cudaEvent_t *ev = nullptr);

// macroscopic fields of the state in src, written to out (device)
int moments_fp64(const StepArgs &a, unsigned mask, double *out);
int moments_mixed(const StepArgs &a, unsigned mask, double *out);
int moments_mixed_fast(const StepArgs &a, unsigned mask, double *out);

// statistics of an initial state (X [M][N], T [N], pressure P; device) for
// the rest references: out = {min rho_a (M), min rho, sum rho_a (M), sum rho,
// sum T}; scratch holds LBMK_STAT_SCRATCH(M) doubles
#define LBMK_STAT_BLOCKS 1024
#define LBMK_STAT_SCRATCH(M_) (LBMK_STAT_BLOCKS * (2 * (M_) + 3))
int ref_stats_fp64(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out);
int ref_stats_mixed(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out);
int ref_stats_mixed_fast(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out);

// heat release rate and its sensitivities of the state in src (lbm_heat_release):
// dT [N] and drho [M][N] (device, or null), partial hrr_blocks(N) (1 + R)
// doubles of scratch, out {sum hdot^c, sum d hdot^c/d ln A_k (R)}
#define LBMK_HRR_BLOCKS 912     // 6 per SM of 152: whole waves at 2 or 3 resident blocks per SM
#define LBMK_HRR_THREADS 128
// blocks of the heat-release kernel for N nodes (grid-stride beyond)
inline int hrr_blocks(long long N)
{
    const long long b = (N + LBMK_HRR_THREADS - 1) / LBMK_HRR_THREADS;
    return (int)(b < LBMK_HRR_BLOCKS ? b : LBMK_HRR_BLOCKS);
}
int hrr_fp64(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out);
int hrr_mixed(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out);
int hrr_mixed_fast(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out);

// the step's chemistry and Newton temperature at n given node states
// (lbm_chemistry_at, lbm_temperature_at; device arrays, outputs may be null)
int chem_at_fp64(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                 double *dT, double *drho, double *dA);
int chem_at_mixed(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                  double *dT, double *drho, double *dA);
int chem_at_mixed_fast(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot,
                       double *hdot, double *dT, double *drho, double *dA);
int temperature_at_fp64(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T);
int temperature_at_mixed(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T);
int temperature_at_mixed_fast(const StepArgs &a, int n, const double *Y, const double *e, const double *T0,
                              double *T);

// gradient of sum hdot^c with respect to the populations of src (periodic
// lattices; lbm_heat_release_adjoint): adj [M + 4][N] per-node moment
// derivatives, then per set s (0..M) the gathered rows out [27][N]
int hrr_adj_fp64(const StepArgs &a, double *adj);
int hrr_adj_mixed(const StepArgs &a, double *adj);
int hrr_adj_mixed_fast(const StepArgs &a, double *adj);
int hrr_adj_gather_fp64(const StepArgs &a, const double *adj, int s, double *out);
int hrr_adj_gather_mixed(const StepArgs &a, const double *adj, int s, double *out);
int hrr_adj_gather_mixed_fast(const StepArgs &a, const double *adj, int s, double *out);

// flame diagnostics of the state in src (lbm_flame_speeds): the record
// pass, then S_d and S_a [N] (device); scratch holds 6 N doubles
int flame_fp64(const StepArgs &a, double *scratch, double *Sd, double *Sa);
int flame_mixed(const StepArgs &a, double *scratch, double *Sd, double *Sa);
int flame_mixed_fast(const StepArgs &a, double *scratch, double *Sd, double *Sa);
// isoline means in the plane z = 0 (lbm_isoline_means): T [N] and fields
// [K][N] (device, K <= 8), partial isoline_blocks(nx ny) (2 + K) doubles of
// scratch, out 2 + K doubles (device) {length, sum L R, sum L f_k}
inline int isoline_blocks(long long cells) { return (int)((cells + LBMK_HRR_THREADS - 1) / LBMK_HRR_THREADS); }
int isoline_fp64(int nx, int ny, int N, const double *T, double T_iso, double cx, double cy, int K,
                 const double *fields, double *partial, double *out, cudaStream_t s);

// nsteps full time steps in one cooperative launch (lbm_step_persistent):
// every node in tiles of tile_mult blocks' worth of nodes, the phases
// separated by grid barriers that poll at most cap times; bar: device
int persistent_fp64(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap);
int persistent_mixed(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap);
int persistent_mixed_fast(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap);
// the persistent units' constant tables (called by upload_fp64 and the like)
int upload_persistent_fp64(int slot, const MechConst &mc, cudaStream_t s);
int upload_persistent_mixed(int slot, const MechConst &mc, cudaStream_t s);
int upload_persistent_mixed_fast(int slot, const MechConst &mc, cudaStream_t s);

// one kernel of the step (LBMK_K_*) with the block size a.bs[kernel]
int launch_one_fp64(const StepArgs &a, int kernel);
int launch_one_mixed(const StepArgs &a, int kernel);
int launch_one_mixed_fast(const StepArgs &a, int kernel);

// The kernel unit of one storage/arithmetic precision.
struct PrecisionOps {
    int (*upload)(int slot, const MechConst &mc, cudaStream_t s);
    int (*init)(const StepArgs &a, const double *X, const double *T, const double *u, double P);
    int (*step)(const StepArgs &a, cudaEvent_t *ev);
    int (*moments)(const StepArgs &a, unsigned mask, double *out);
    int (*ref_stats)(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out);
    int (*launch_one)(const StepArgs &a, int kernel);
    int (*hrr)(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out);
    int (*chem_at)(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                   double *dT, double *drho, double *dA);
    int (*temperature_at)(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T);
    int (*hrr_adj)(const StepArgs &a, double *adj);
    int (*hrr_adj_gather)(const StepArgs &a, const double *adj, int s, double *out);
    int (*flame)(const StepArgs &a, double *scratch, double *Sd, double *Sa);
    int (*persistent)(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap);
};
}  // namespace lbmk

// Hand-written adjoint of the double-precision step (periodic lattices).
// One reverse step takes lam_next, the adjoint of the post-collision state
// the step writes, and returns lam, the adjoint of the state it pulls from
// (plus, with with_objective, the gradient of sum_nodes hdot^c at the
// state the step's collision sees).  The per-node record of the step must
// have been recomputed first (the moment and gradient passes of the
// forward step, launch_one_fp64 LBMK_K_PRE and LBMK_K_GRAD, on the same
// state and Newton starting temperatures).  The adjoint kernels live in a
// unit of their own (k_adjoint.cu) whose constant-memory tables adj_upload
// fills, in the context's slot, before each adjoint call.
//   mbar  [adj_mbar_rows(M)][N]: adjoint of the pulled moments (rho_a and
//         j_a of the M-1 stored species, rho, j, the pressure tensor's six
//         entries, rho E, q)
//   coef  [M][N]: 1 - 2 beta_a (a < M-1) and 1 - omega
//   aux   [10][N]: adjoints of X (3) and of sum_a H_a grad Y_a (3), then
//         (1/omega - 1/2) times the adjoint of G (3) and the adjoint of
//         1/omega - 1/2 (1)
//   theta [adj_blocks(N)][R]: per-block sums of the ln A_k gradient, which
//         every reverse step adds to
#define LBMK_ADJ_THREADS 128
__host__ __device__ constexpr int adj_mbar_rows(int M) { return 4 * (M - 1) + 14; }
inline int adj_blocks(long long N) { return (int)((N + LBMK_ADJ_THREADS - 1) / LBMK_ADJ_THREADS); }
struct AdjBufs {
    const double *lam_next;
    double *lam, *fbar, *mbar, *coef, *aux, *theta;
    int with_objective;
};
namespace lbmk {
int adj_upload(int slot, const MechConst &mc, cudaStream_t s);
int adj_step_fp64(const StepArgs &a, const AdjBufs &g);
// d J / d T(x, 0) of a state made by lbm_init (every set at equilibrium at
// zero velocity, fixed mole fractions and pressure) from the adjoint lam0 of
// that state: out [N]
int adj_init_T_fp64(const StepArgs &a, const double *lam0, double *out);
// column sums of nb partial records of width w (fixed order)
int column_sums_fp64(const double *partial, int nb, int w, double *out, cudaStream_t s);
}  // namespace lbmk
