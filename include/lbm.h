/*
 * lbm.h - C ABI of the GB300 (sm_103a) reactive-mixture lattice Boltzmann
 * library.
 *
 * The library advances the fully kinetic reactive-mixture lattice Boltzmann
 * model of Sawant, Dorschner and Karlin, "Reactive mixtures with the lattice
 * Boltzmann model" (arXiv 2101.01702), on a D3Q27 lattice: M species
 * population sets of which the last is slaved to the mixture (Eq. (strongest),
 * so M-1 species sets are stored), the mixture mass/momentum set f (Eq. (f))
 * and the total-energy set g (Eq. (g)).  One time step is pull streaming,
 * moments, temperature from energy (Eq. (temperature)), the per-node
 * Stefan-Maxwell system (Eq. (transform1)), the reaction source
 * (Eqs. (sumfDotc), (fsource)), and the collisions of
 * Eqs. (finalNumericalEquations), (f) and (g).
 *
 * Conventions (all entry points):
 *   - Every call returns an int status (LBM_OK or a negative LBM_ERR_*); no
 *     call aborts, traps or prints.  lbm_strerror() names a status.
 *   - Lattice units: grid spacing and time step are 1.  Node index
 *     n = x + nx * (y + ny * z); directions i = (cx+1) + 3 (cy+1) + 9 (cz+1)
 *     with c in {-1,0,1}^3.  Set order: species 0..M-2, then f, then g.
 *   - Device buffers are owned by the caller (for example torch tensors) and
 *     are never freed by the library.  Host arrays passed to lbm_create are
 *     copied; the library keeps no pointer to them.
 *   - All GPU work is ordered on the CUDA stream given to lbm_create.
 *   - A context belongs to the CUDA device that is current when lbm_create
 *     is called; every later call on it that touches the GPU must be made
 *     with that device current, else it returns LBM_ERR_ARG.  Contexts on
 *     different devices of one process share no state.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,          /* NULL pointer, bad size, unsupported value        */
    LBM_ERR_CUDA = -2,         /* a CUDA runtime call failed                       */
    LBM_ERR_NEWTON = -3,       /* temperature iteration did not converge (50 its)  */
    LBM_ERR_NONFINITE = -4,    /* a density, energy or population became NaN/Inf   */
    LBM_ERR_NEGATIVE = -5,     /* a species density fell below -1e-10 rho           */
    LBM_ERR_PIVOT = -6,        /* non-finite pivot in the Stefan-Maxwell elimination */
    LBM_ERR_BOUNDS = -7,       /* checked builds: an index left its buffer (a bug)  */
    LBM_ERR_UNSUPPORTED = -8,  /* valid request this build does not provide        */
    LBM_ERR_BARRIER = -9       /* lbm_step_persistent: a grid barrier gave up waiting */
};

enum { LBM_BC_PERIODIC = 0, LBM_BC_EQ_ZEROGRAD_U0LEFT = 1 };
enum { LBM_FP64 = 0, LBM_MIXED = 1, LBM_MIXED_FAST = 2 };
enum { LBM_THERMO_CONST_CP = 0, LBM_THERMO_POLY7 = 1 };
enum { LBM_VISC_KINEMATIC = 0, LBM_VISC_RELAXATION = 1 };
enum { LBM_TRANSPORT_CONSTANT = 0, LBM_TRANSPORT_MIXTURE_AVERAGED = 1 };
enum { LBM_RXN_ELEMENTARY = 0, LBM_RXN_THIRD_BODY = 1, LBM_RXN_FALLOFF = 2 };

/* Lattice.  y and z are periodic.  bc_x = LBM_BC_PERIODIC wraps x;
 * LBM_BC_EQ_ZEROGRAD_U0LEFT places ghost nodes beyond both x faces holding
 * the equilibria of every set at the post-collision moments of the adjacent
 * boundary node, with zero velocity on the left (paper Sec. 5a, the 1D
 * flame setup); macroscopic fields used by the gradient stencils continue
 * with zero gradient.  precision:
 *   LBM_FP64        stores and collides every population in double;
 *   LBM_MIXED       stores the 26 moving populations of the species and
 *                   mixture sets as float deviations from per-set rest
 *                   states and collides them in float; their rest
 *                   populations and the energy set stay double, and so do
 *                   the moments, the temperature iteration, the
 *                   Stefan-Maxwell solve, the reaction rates and the
 *                   equilibrium constants;
 *   LBM_MIXED_FAST  as LBM_MIXED, but the relaxation rates and the
 *                   Stefan-Maxwell solve run in float and the exponentials
 *                   of the rate expressions take a double range reduction
 *                   with a float 2^f (relative error ~3e-7); its results
 *                   are stored as floats in both mixed modes.  Same
 *                   storage layout and accuracy bar as LBM_MIXED. */
typedef struct {
    int nx, ny, nz;
    int bc_x;
    int precision;
    /* Batches of independent lattices (the paper's 1D flame setup of Sec. 5a
     * repeated): nseg >= 2 places nseg lattices of seg_nx[k] x ny x nz
     * nodes side by side along x (sum of seg_nx = nx; bc_x must be
     * LBM_BC_EQ_ZEROGRAD_U0LEFT).  Each has its own ghost nodes on both x
     * faces, and no population, gradient stencil or ghost crosses from one
     * to the next: every lattice evolves exactly as it would alone.
     * nseg = 0 or 1: one lattice (seg_nx unused).  seg_nx is read during
     * lbm_buffer_sizes and lbm_create only. */
    int nseg;
    const int *seg_nx;
} lbm_lattice;

/* Species, thermodynamics and transport (paper Secs. 2-3).
 *   M            number of species, 2 <= M <= 12; species M-1 is slaved.
 *   W[M]         molar masses; R_a = r_lat / W[a] (paper Sec. 2, after Eq. (eosIdealGas)).
 *   thermo       LBM_THERMO_CONST_CP: U_a(T) = h_form[a] - R_a T0 + (cp_R[a]-1) R_a (T-T0)
 *                (Eq. (specHa) with constant heat capacity; h_form is the
 *                mass-specific formation enthalpy at T0).
 *                LBM_THERMO_POLY7: single-range 7-coefficient polynomials
 *                poly7[M][7]: cp/R = a1 + a2 T + ... + a5 T^4,
 *                h/(R T) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
 *                s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
 *   D[M][M]      binary diffusivities D_ab (Eq. (tauab)), symmetric.
 *   nu, visc_model   LBM_VISC_KINEMATIC: kinematic viscosity nu, so
 *                1/omega - 1/2 = nu / (R T) (Eq. (mu) with mu = rho nu);
 *                LBM_VISC_RELAXATION: 1/omega - 1/2 = nu (mu = nu P).
 *   Pr           Prandtl number: 1/omega_1 - 1/2 = (1/omega - 1/2) / Pr (Eq. (lambda)).
 *   r_lat        universal gas constant in lattice units.
 *   transport    LBM_TRANSPORT_CONSTANT: nu, visc_model, Pr and D as above.
 *                LBM_TRANSPORT_MIXTURE_AVERAGED: the viscosity, conductivity
 *                and diffusivities of each node's state, the stand-in for
 *                the coefficients the paper takes from Cantera (Sec. 3,
 *                after Eq. (lambda)):
 *                  mu_a = mu0[a] (T/T_tr)^mu_exp[a]  (species viscosities),
 *                  mu by Wilke's mixing rule (Wilke 1950),
 *                  lambda_a = mu_a (C_p,a + 5/4 R_a) (modified Eucken),
 *                  lambda by the average of Mathur, Tondon and Saxena (1967),
 *                  D_ab(T, P) = D[a][b] (T/T_tr)^D_exp (P_tr/P);
 *                then 1/omega - 1/2 = mu / P (Eq. (mu)),
 *                1/omega_1 - 1/2 = lambda / (P C_p) (Eq. (lambda)) and tau_ab
 *                from D_ab(T, P) (Eq. (tauab)); nu and Pr are not used.
 *                mu0, mu_exp [M]; T_tr, P_tr > 0.
 * Unused arrays (cp_R/h_form for POLY7, poly7 for CONST_CP, mu0/mu_exp for
 * constant transport) may be NULL. */
typedef struct {
    int M;
    const double *W;
    int thermo;
    const double *cp_R;
    const double *h_form;
    double T0;
    const double *poly7;
    const double *D;
    double nu, Pr, r_lat;
    int visc_model;
    int transport;
    const double *mu0;
    const double *mu_exp;
    double T_tr, D_exp, P_tr;
} lbm_species;

/* Reaction mechanism giving the production rates rho_dot_a of Eq. (sumRhoDot)
 * (the paper obtains them from Cantera, Sec. 4).  R <= 32 reactions, each
 * with at most 3 reactant and 3 product molecules.
 *   nu_f[R][M], nu_r[R][M]   reactant / product stoichiometric coefficients
 *   k = exp(log_A + b ln(T/T_ref) - theta/T), concentrations c_a = rho_a/W_a
 *   rtype: ELEMENTARY, THIRD_BODY (rate of progress times [M] = sum eff[k][a] c_a),
 *          FALLOFF (Lindemann: k = k_inf P_r/(1+P_r), P_r = k0 [M]/k_inf,
 *          k0 from low[k] = {log_A0, b0, theta0})
 *   reversible[k] != 0: reverse rate k / K_c with
 *          K_c = exp(-sum_a dnu_a g_a/(R_U T)) (P0/(r_lat T))^(sum_a dnu_a).
 * eff and low may be NULL when no reaction needs them. */
typedef struct {
    int R;
    const int *nu_f, *nu_r;
    const double *log_A, *b, *theta;
    const int *rtype;
    const double *eff;
    const double *low;
    const int *reversible;
    double T_ref, P0;
} lbm_mechanism;

/* Caller-owned device memory, sized by lbm_buffer_sizes():
 *   pop_a, pop_b  two population buffers that swap roles every step; node
 *                 n = x + nx (y + ny z); sets 0..M-2 the stored species,
 *                 M-1 the mixture f, M the energy set g.
 *                 LBM_FP64: double [M+1][27][N].
 *                 mixed modes: float [M][27][N] (sets 0..M-1 as deviations
 *                 from their rest states; the rest slot 13 unused), then at
 *                 the next 16-byte boundary double [M][N] (their rest
 *                 populations), then double [27][N] (the energy set).
 *                 Must be distinct and 16-byte aligned.
 *   macro         per-node record of the current step, [rows][N]: M+12
 *                 rows of double (temperature first: the Newton starting
 *                 point, which lbm_init writes), then 19+7M rows of the
 *                 storage type (float in the mixed modes): moments,
 *                 relaxation rates, diffusion velocities, production rates
 *                 and the inputs of the gradient stencils.
 *   ghost         x-face ghost populations, double [2 G][M+1][27][ny*nz]
 *                 with G = max(nseg, 1) lattices (left then right face of
 *                 each); may be NULL for periodic x. */
typedef struct {
    void *pop_a, *pop_b, *macro, *ghost;
    size_t pop_bytes, macro_bytes, ghost_bytes;
} lbm_buffers;

/* Bytes each buffer needs for the lattice and species count. */
int lbm_buffer_sizes(const lbm_lattice *lat, const lbm_species *sp,
                     size_t *pop_bytes, size_t *macro_bytes, size_t *ghost_bytes);

/* Validates the description, copies the tables to the device, binds the
 * buffers and the stream (a cudaStream_t, or NULL for the default stream).
 * Allocates host state and a 4-byte device status word. */
int lbm_create(const lbm_lattice *lat, const lbm_species *sp, const lbm_mechanism *mech,
               const lbm_buffers *bufs, void *cuda_stream, lbm_ctx **out);

/* Sets every set to its equilibrium (Eqs. (feq), (feqmix), (gieq)) for mole
 * fractions X[M][N], temperature T[N], velocity u[3][N] (NULL: at rest) and
 * a uniform pressure P, with rho = P / (R T) (Eq. (eosIdealGas)).  Pointers
 * may be host or device memory; host data is staged through pop_b. */
int lbm_init(lbm_ctx *ctx, const double *X, const double *T, const double *u, double P);

/* Enqueues n time steps on the stream, then waits for them and returns the
 * first error the kernels recorded (LBM_ERR_NEWTON ... LBM_ERR_PIVOT). */
int lbm_step(lbm_ctx *ctx, int n);

/* Enqueues n time steps without waiting; errors surface at lbm_sync(). */
int lbm_step_async(lbm_ctx *ctx, int n);

/* lbm_step_async through a CUDA graph.  The first call captures two time
 * steps (A -> B -> A) on the context's stream and instantiates the graph;
 * each call then launches it n/2 times, plus one ordinary step when n is
 * odd or the current state is not in the graph's starting buffer.  Cuts
 * the per-step launch cost of small lattices and batches; the results are
 * those of lbm_step_async.  The stream must not be the legacy default
 * stream (LBM_ERR_UNSUPPORTED).  Errors surface at lbm_sync(). */
int lbm_step_graph(lbm_ctx *ctx, int n);

/* n time steps in ONE persistent, cooperative kernel launch (the paper has
 * no counterpart: a launch structure for batches of small lattices, such as
 * the quasi-1D flames of Sec. 5a side by side).  The blocks stay resident;
 * in each phase of a step (ghost planes, the per-node record, G, the
 * energy collision, the species collision) their warps take chunks of
 * tile_mult x 32 consecutive nodes from a queue, and all meet at a grid
 * barrier before the next phase.  Results agree with lbm_step to rounding
 * (the compiler may fuse a multiply and an add in this kernel where it does
 * not in the separate ones: about one unit in the last place per step).
 * Each barrier polls a device word at most spin_cap times
 * (0: 1 << 24, about two seconds); a block that runs out records
 * LBM_ERR_BARRIER and returns, the others then run out at the next barrier,
 * so the launch always ends -- the state is then partly stepped and must be
 * re-initialised or restored.  tile_mult >= 1.  Waits for the stream and
 * returns like lbm_sync (LBM_ERR_BARRIER after a timeout); LBM_ERR_ARG for
 * n < 0 or tile_mult < 1; LBM_ERR_UNSUPPORTED in a build whose production
 * rates run in a kernel of their own (LBMK_FUSE_CHEM=0); LBM_ERR_CUDA when
 * the device cannot hold the grid's blocks at once. */
int lbm_step_persistent(lbm_ctx *ctx, int n, int tile_mult, unsigned spin_cap);

/* Picks the tile length of lbm_step_persistent (tile_mult in 1, 2, 4, 8)
 * by timing `steps` persistent steps of each on a copy of the current state
 * (kept aside and put back, with the temperature row: the state is
 * unchanged); *tile_mult_out receives the fastest.  Allocates a copy of the
 * state for the duration of the call.  Waits for the stream. */
int lbm_autotune_persistent(lbm_ctx *ctx, int steps, int *tile_mult_out);

/* Autotuner of the launch shapes (the paper has no counterpart): times
 * each kernel of the step on the context's current state with every
 * candidate block size -- 64 or 128 threads for the moment and species-
 * collision kernels, whose register budgets are set for 128, and 64, 128
 * or 256 for the production-rate, gradient and energy-collision kernels --
 * over `trials` launches (1..1000) after two untimed ones, and keeps the
 * fastest for every later step of this context.  The state is left as it
 * was (the kernels write only the per-node record and the other buffer;
 * the temperature row, the next Newton start, is restored), so results
 * are bit for bit those of the untuned context.  Allocates and frees one
 * temporary row of N doubles.  block_out (NULL or 6 ints) receives the
 * chosen blocks in launch order: ghost nodes, moments, production rates,
 * gradients, energy collision, species/mixture collision (the production-
 * rate entry has no effect: the rates are formed inside the species
 * collision).  Waits for the stream; returns like lbm_sync. */
int lbm_autotune(lbm_ctx *ctx, int trials, int *block_out);

/* Sets the block sizes of the six kernels directly (for instance a choice
 * lbm_autotune made in an earlier run): blocks[6] in the order of
 * block_out above, each 64, 128 or 256, at most 128 for the moment and
 * species-collision kernels, and 128 for the ghost-node kernel; else
 * LBM_ERR_ARG.  Results do not depend on the choice. */
int lbm_set_blocks(lbm_ctx *ctx, const int *blocks);

/* lbm_step_async with CUDA events recorded on the stream between the
 * kernels of each step (all steps enqueued back to back, one wait at the
 * end).  phase_ms must hold LBM_PHASES + 1 doubles: phase_ms[0..5] receive
 * the summed device time of the ghost-node, moment, production-rate,
 * gradient, energy-collision and species/mixture-collision kernels over
 * the n steps, phase_ms[LBM_PHASES] the device time from the first launch
 * to the end of the last.  The production rates are formed inside the
 * species/mixture-collision kernel (no kernel of their own), so their phase
 * is empty and their time is in phase_ms[5].  Returns like lbm_step. */
#define LBM_PHASES 6
int lbm_step_timed(lbm_ctx *ctx, int n, double *phase_ms);

/* Waits for the stream and returns (then clears) the recorded error. */
int lbm_sync(lbm_ctx *ctx);

/* Macroscopic fields of the current time level (the moments the next
 * collision sees), double, written to out (host or device) as consecutive
 * [N] rows in this order for the bits set in mask:
 *   LBM_F_RHO_A  rho_a, M rows        LBM_F_RHOU  rho u, 3 rows
 *   LBM_F_RHOE   rho E, 1 row         LBM_F_T     T, 1 row
 *   LBM_F_P      P = rho R T, 1 row   LBM_F_Y     Y_a, M rows
 *   LBM_F_J_A    species momenta rho_a u_a, 3M rows (a-major)
 *   LBM_F_RHO_DOT  mass production rates rho_dot_a of the mechanism at
 *                (rho_a, T), M rows (Eq. (sumRhoDot); per lattice time unit)
 *   LBM_F_HRR    heat release rate hdot^c = -sum_a H_a rho_dot_a, 1 row
 *                (Sec. 5b; H_a the specific enthalpy of Eq. (specHa))
 * Waits for the stream before returning. */
enum { LBM_F_RHO_A = 1, LBM_F_RHOU = 2, LBM_F_RHOE = 4, LBM_F_T = 8, LBM_F_P = 16,
       LBM_F_Y = 32, LBM_F_J_A = 64, LBM_F_RHO_DOT = 128, LBM_F_HRR = 256 };
int lbm_moments(lbm_ctx *ctx, unsigned mask, double *out);

/* Number of doubles lbm_moments writes for mask. */
size_t lbm_moments_count(const lbm_ctx *ctx, unsigned mask);

/* Heat-release objective and its sensitivities at the current time level
 * (the state lbm_moments reports).  The heat release rate of Sec. 5b,
 * hdot^c = -sum_a H_a rho_dot_a, is written per reaction as
 * -sum_k dH_k q_k with dH_k = sum_a W_a (nu''_ak - nu'_ak) H_a(T) and the
 * rate of progress q_k of the mechanism (Eqs. (sumRhoDot), (specHa)).
 *   J         host, double: the sum of hdot^c over the nodes (required)
 *   dJ_dlogA  host, double [R], or NULL: dJ/d ln A_k, A_k the
 *             pre-exponential factor of reaction k (that of the
 *             high-pressure rate for a falloff reaction), all else fixed
 *   dJ_dT     host or device, double [N], or NULL: d hdot^c/dT at each node
 *             with its densities fixed
 *   dJ_drho   host or device, double [M][N], or NULL: d hdot^c/d rho_a at
 *             each node with T and the other densities fixed (all M
 *             densities independent, the slaved one included)
 * J and dJ_dlogA are summed on the GPU in a fixed order, so that they
 * repeat from run to run.  These are the chemistry terms of an adjoint of
 * the step (the paper has none; the transposed step is not part of this
 * library).  The second population buffer serves as scratch, as in
 * lbm_moments.  Waits for the stream; returns like lbm_sync, or
 * LBM_ERR_ARG for a NULL ctx or J.  The transposed step is
 * lbm_adjoint_step and the gradient through time
 * lbm_heat_release_gradient. */
int lbm_heat_release(lbm_ctx *ctx, double *J, double *dJ_dlogA, double *dJ_dT, double *dJ_drho);

/* Gradient of the same objective J = sum over the nodes of hdot^c with
 * respect to the stored populations of the current state: the source term
 * that J contributes to an adjoint of the step.  Node n pulls
 * P_si(n) = F_si(n - c_i) and forms rho_a, rho, rho u and rho E; the
 * temperature depends on them through Eq. (temperature) (implicit function:
 * dT = (de - sum_a U_a dY_a) / C_v), the slaved density through
 * Eq. (strongest), and hdot^c on (rho_a, T) as in lbm_heat_release.
 *   dJ_dF  host or device, double [M+1][27][N] (the layout of
 *          lbm_get_populations): dJ/dF_si(x) for every set, direction and
 *          node, with respect to the absolute population values
 * Periodic lattices only (LBM_ERR_UNSUPPORTED for ghost-node faces or
 * batches).  The second population buffer serves as scratch.  Waits for
 * the stream; returns like lbm_sync. */
int lbm_heat_release_adjoint(lbm_ctx *ctx, double *dJ_dF);

/* Hand-written adjoint of the double-precision step (the paper has no
 * adjoint; the objective is its heat release rate of Sec. 5b).  Both calls
 * below take a caller-owned device workspace of at least the size this
 * call reports, for nsteps steps with a checkpoint every checkpoint_every
 * steps (nsteps = 0: the size lbm_adjoint_step needs; checkpoint_every = 0:
 * the size of the objective alone, without gradients).  LBM_ERR_ARG for a
 * NULL ctx or bytes, negative counts, or both counts 0. */
int lbm_adjoint_workspace_bytes(const lbm_ctx *ctx, int nsteps, int checkpoint_every, size_t *bytes);

/* One reverse step at the current state F (the state the next lbm_step
 * would pull from): given lam_next = dL/dF' for the state F' = step(F)
 * that lbm_step would produce, returns
 *   lam = (dF'/dF)^T lam_next  (+ dJ_t/dF with with_objective != 0)
 * where J_t is the sum over the nodes of hdot^c at the state the step's
 * collision sees (as lbm_heat_release at F).  The transpose covers every
 * dependence of F' on F: the pull (Eqs. (finalNumericalEquations), (f),
 * (g) left-hand sides), the moments and slaving (Eqs. (Pa), (strongest)),
 * the Newton temperature (Eq. (temperature), implicit-function adjoint),
 * the relaxation rates (Eqs. (mu), (lambda), (tauab), (fStar)), the
 * Stefan-Maxwell solve (Eq. (transform1); B is symmetric after the
 * Y-scaling, so its adjoint solve is with B itself), the production rates
 * (Sec. 4), the isotropy correction and the interdiffusion heat flux with
 * their lattice gradients (Eqs. (Xalpha), (Ai), (qdiff), (corrFourier))
 * and the three collisions.
 *   lam_next, lam  device, double [M+1][27][N] (lbm_get_populations layout);
 *                  distinct, and neither inside the workspace
 *   dJ_dlogA       host, double [R], or NULL: (dF'/d ln A_k)^T lam_next
 *                  (+ dJ_t/d ln A_k)
 *   workspace      device, at least lbm_adjoint_workspace_bytes(ctx, 0, 1)
 * The state is not changed.  LBM_FP64 periodic lattices only
 * (LBM_ERR_UNSUPPORTED otherwise).  Waits for the stream; returns like
 * lbm_sync. */
int lbm_adjoint_step(lbm_ctx *ctx, const double *lam_next, double *lam, double *dJ_dlogA, int with_objective,
                     void *workspace, size_t workspace_bytes);

/* The objective integrated over time, J = sum_{t=0}^{nsteps-1} J_t with
 * J_t = sum over the nodes of hdot^c at the state step t's collision sees,
 * starting from the current state, which must be one lbm_init made with
 * zero velocity; and its gradients through the dynamics:
 *   J          host, double: the objective
 *   dJ_dlogA   host, double [R], or NULL: dJ/d ln A_k (A_k as in
 *              lbm_heat_release)
 *   dJ_dT0     host or device, double [N], or NULL: dJ/dT(x, 0), the
 *              initial temperature of each node at fixed mole fractions,
 *              pressure and zero velocity (the inputs of lbm_init)
 * The forward sweep keeps the state every checkpoint_every steps; the
 * reverse sweep recomputes each segment's states from its checkpoint and
 * applies lbm_adjoint_step's transpose step by step, last step first.  With
 * dJ_dlogA and dJ_dT0 both NULL only the forward sweep runs (J alone,
 * without checkpoints; the workspace needs only
 * lbm_adjoint_workspace_bytes(ctx, nsteps, 0)).  The
 * context ends at the state after nsteps steps, as lbm_step(nsteps) leaves
 * it.  LBM_FP64 periodic lattices only (LBM_ERR_UNSUPPORTED otherwise);
 * LBM_ERR_ARG for nsteps < 1, checkpoint_every < 1 or a workspace smaller
 * than lbm_adjoint_workspace_bytes(ctx, nsteps, checkpoint_every).  Waits
 * for the stream; returns like lbm_sync. */
int lbm_heat_release_gradient(lbm_ctx *ctx, int nsteps, int checkpoint_every, double *J, double *dJ_dlogA,
                              double *dJ_dT0, void *workspace, size_t workspace_bytes);

/* The step's chemistry at n given node states, for checks of the node
 * functions on inputs of the caller's choice.  Inputs, device:
 *   rho_a [M][n] species densities, T [n] temperatures.
 * Outputs, device, each NULL to skip:
 *   rho_dot     [M][n]  mass production rates, evaluated as the step does
 *                       (Eq. (sumRhoDot); in the precision unit's arithmetic)
 *   hdot        [n]     heat release rate -sum_a H_a rho_dot_a (Sec. 5b)
 *   dhdot_dT    [n]     its derivative in T at fixed densities
 *   dhdot_drho  [M][n]  its derivatives in rho_a at fixed T
 *   dhdot_dlogA [R][n]  its derivatives in ln A_k (as in lbm_heat_release)
 * Waits for the stream; LBM_ERR_ARG for n < 0, a NULL input or a host
 * pointer; else returns like lbm_sync. */
int lbm_chemistry_at(lbm_ctx *ctx, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                     double *dhdot_dT, double *dhdot_drho, double *dhdot_dlogA);

/* The step's Newton temperature (Eq. (temperature)) at n given node states:
 * mass fractions Y [M][n], specific internal energy e [n] (including the
 * energies of formation; e = rho E / rho - u^2/2) and starting points
 * T_guess [n]; temperatures to T [n].  All device.  Waits for the stream;
 * LBM_ERR_ARG for n < 0, NULL or host pointers; LBM_ERR_NEWTON when an
 * iteration did not converge. */
int lbm_temperature_at(lbm_ctx *ctx, int n, const double *Y, const double *e, const double *T_guess, double *T);

/* Current post-collision populations as absolute doubles, layout
 * [M+1][27][N], copied to host memory out.  Diagnostic accessor. */
int lbm_get_populations(lbm_ctx *ctx, double *host_out);

/* Device pointer of the buffer that holds the current state (pop_a or
 * pop_b); with the T row of macro (and, in the mixed modes, the rest
 * references below) it is everything a checkpoint needs. */
void *lbm_state_buffer(lbm_ctx *ctx);

/* Mixed modes: the rest references the stored float deviations are taken
 * from, float [M][27] (set s = 0..M-1, direction i; the rest direction 13
 * is unused and reads 0).  lbm_init chooses them from the initial fields
 * (each set's rest equilibrium at its smallest initial density and the
 * mean initial temperature); lbm_set_references fixes them instead, so
 * that a later lbm_init keeps them -- for restarting from a checkpoint
 * written with those references, or for giving several contexts the same
 * tables (contexts with identical mechanism and references share one
 * constant-memory slot; each precision has 4 slots).  Set before lbm_init
 * or before restoring a state.  LBM_ERR_UNSUPPORTED for LBM_FP64,
 * LBM_ERR_ARG for NULL or non-finite values. */
int lbm_get_references(const lbm_ctx *ctx, float *ref);
int lbm_set_references(lbm_ctx *ctx, const float *ref);

/* One double-precision time step that allocates nothing (the paper has no
 * counterpart; this is a service for callers).  Some callers cannot call
 * cudaMalloc where they need to step the lattice: a plugin or callback
 * running inside another framework that owns every device allocation, or
 * a process whose device allocator is capped or exhausted.  They can still
 * pass their own population buffers, so this entry point takes
 *   pop_in   device, double [M+1][27][N]: post-collision state (input)
 *   pop_out  device, double [M+1][27][N]: the state one step later (output,
 *            distinct from pop_in)
 *   T_io     device, double [N]: starting temperatures for the Newton
 *            iteration on input; the temperatures of the step's moments on
 *            output (must not overlap either population buffer)
 * and keeps the per-node macroscopic record, the x-face ghost planes and the
 * status word in a fixed device array of LBM_FIXED_SCRATCH_BYTES compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.  No context (lbm_create) is needed; the species and
 * mechanism tables are copied to constant memory on every call.
 * Limits: precision LBM_FP64 only (else LBM_ERR_UNSUPPORTED); the lattice
 * must fit, 256 + (31 + 8M) N 8 bytes plus, for non-periodic x,
 * 2 (M+1) 27 ny nz 8 bytes <= LBM_FIXED_SCRATCH_BYTES (up to 43^3 nodes
 * with M = 9, 53^3 with M = 3), else LBM_ERR_ARG; pop_in, pop_out and
 * T_io must not overlap one another (LBM_ERR_ARG).  The first call on a
 * device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call uses the same array and it keeps the previous call's
 * contents (the call clears its status word itself), so calls that overlap
 * on the GPU -- on different streams or host threads -- race and must be
 * serialised by the caller.  Every call waits for the stream (it reads
 * the status word back) and returns like lbm_step. */
#define LBM_FIXED_SCRATCH_BYTES (64u << 20)
int lbm_step_fixed_scratch(const lbm_lattice *lat, const lbm_species *sp, const lbm_mechanism *mech,
                           const double *pop_in, double *pop_out, double *T_io, void *cuda_stream);

/* Diagnostic (the paper has no counterpart): evaluates the kernels' own
 * double-precision exponential -- the table-driven method of P. T. P. Tang
 * (ACM Trans. Math. Softw. 15(2), 1989) used for the Arrhenius factors and
 * equilibrium constants -- into y and the CUDA math library's exp into
 * y_ref, for n arguments x.  x, y, y_ref: device, double [n].  Waits for
 * the stream; LBM_ERR_ARG for NULL pointers or n < 0. */
int lbm_exp_check(const double *x, double *y, double *y_ref, int n, void *cuda_stream);

/* Diagnostic (the paper has no counterpart): the kernels convert between
 * float and double with integer operations (the hardware conversion issues
 * on the FP64 pipe).  Writes those conversions of f [n] to fd and of d [n]
 * to df, and the hardware conversions (round to nearest even) to fd_ref
 * and df_ref.  All pointers device; waits for the stream; LBM_ERR_ARG for
 * NULL pointers or n < 0. */
int lbm_convert_check(const float *f, double *fd, double *fd_ref, const double *d, float *df, float *df_ref,
                      int n, void *cuda_stream);

/* Flame diagnostics of the circular expanding flame (paper Sec. 5b) at the
 * current state (the state the next collision sees): per node the local
 * displacement speed of Eq. (sd),
 *   S_d = [hdot^c + div(lambda grad T) - rho (sum_a C_a,p Y_a du_a) . grad T]
 *         / (rho C_p |grad T|),
 * with hdot^c = -sum_a H_a rho_dot_a, lambda = (1/omega_1 - 1/2) P C_p
 * (Eq. (lambda)), the diffusion velocities du_a of Eq. (transform1) and the
 * isotropic lattice gradients; and the absolute propagation speed
 * S_a = S_d + u . n with n = -grad T / |grad T| (0 where grad T = 0).
 *   Sd, Sa  host or device (both alike), double [N]
 * The second population buffer serves as scratch; the state and the
 * temperature row are unchanged.  Waits for the stream; returns like
 * lbm_sync. */
int lbm_flame_speeds(lbm_ctx *ctx, double *Sd, double *Sa);

/* Means along the isoline T = T_iso in the plane z = 0, Eq. (rmean):
 * A^{-1} int f dA over the isoline of length A, found by marching squares
 * on the periodic x-y cells (crossings interpolated linearly along cell
 * edges; a cell with four crossings split by the mean of its corners).
 *   T        device, double [N]: the field whose isoline is taken
 *   cx, cy   the centre for the distance R
 *   fields   device, double [K][N] (K <= 8), or NULL for K = 0
 *   out      host, double [2 + K]: {A, mean R, mean field_0 .. field_{K-1}}
 * Positions are not wrapped: the isoline must not cross the box edge.
 * Sums in a fixed order.  The second population buffer serves as scratch.
 * Waits for the stream; LBM_ERR_ARG for NULL or host arrays, K > 8. */
int lbm_isoline_means(lbm_ctx *ctx, const double *T, double T_iso, double cx, double cy, int K,
                      const double *fields, double *out);

/* Diagnostic (the paper has no counterpart): throughput of the GPU's
 * double-precision arithmetic, the peak the step's FP64-bound kernels are
 * measured against.  kind: LBM_PROBE_DFMA (independent fused multiply-add
 * chains; rate in flops/s, 2 per FMA), LBM_PROBE_EXP or LBM_PROBE_LOG
 * (independent chains of CUDA's double exp or log; rate in calls/s).
 * blocks: grid size (256 threads each; a multiple of the SM count fills the
 * GPU evenly); iters: loop trips per thread (32 FMA or 4 calls each).
 * sink: device, double [blocks], never written in practice (it keeps the
 * compiler from removing the chains).  out: host, double [2]: elapsed
 * milliseconds (CUDA events on the stream) and the rate.  Waits for the
 * stream; LBM_ERR_ARG for a bad kind, NULL or host pointers, or
 * non-positive sizes. */
#define LBM_PROBE_DFMA 0
#define LBM_PROBE_EXP 1
#define LBM_PROBE_LOG 2
int lbm_fp64_probe(int kind, int blocks, int iters, double *sink, double *out, void *cuda_stream);

/* Frees host state and the status word; never the caller's buffers. */
int lbm_destroy(lbm_ctx *ctx);

const char *lbm_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
