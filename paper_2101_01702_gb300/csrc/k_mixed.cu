// Kernels of the reactive-mixture lattice Boltzmann step, float populations stored as deviations (mixed precision).
#define LBMK_MIXED 1
#include "lbm_kernels.cuh"

namespace lbmk {

int upload_mixed(int slot, const MechConst &mc, cudaStream_t s)
{
    // this unit's tables and those of its persistent kernel's unit
    const int e = (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                               cudaMemcpyHostToDevice, s);
    return e ? e : upload_persistent_mixed(slot, mc, s);
}

int init_mixed(const StepArgs &a, const double *X, const double *T, const double *u, double P)
{
#define CALL(M_) run_init<M_>(a, X, T, u, P)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int step_mixed(const StepArgs &a, cudaEvent_t *ev)
{
#define CALL(M_) run_step<M_>(a, ev)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int ref_stats_mixed(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out)
{
#define CALL(M_) run_ref_stats<M_>(a, X, T, P, scratch, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int launch_one_mixed(const StepArgs &a, int kernel)
{
#define CALL(M_) launch_one<M_>(a, kernel)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int moments_mixed(const StepArgs &a, unsigned mask, double *out)
{
#define CALL(M_) run_moments<M_>(a, mask, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_mixed(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out)
{
#define CALL(M_) run_hrr<M_>(a, R, dT, drho, partial, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int chem_at_mixed(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                 double *dT, double *drho, double *dA)
{
#define CALL(M_) run_chem_at<M_>(a, n, rho_a, T, rho_dot, hdot, dT, drho, dA)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int temperature_at_mixed(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T)
{
#define CALL(M_) run_temperature_at<M_>(a, n, Y, e, T0, T)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_adj_mixed(const StepArgs &a, double *adj)
{
#define CALL(M_) run_hrr_adj<M_>(a, adj)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_adj_gather_mixed(const StepArgs &a, const double *adj, int s, double *out)
{
#define CALL(M_) run_hrr_adj_gather<M_>(a, adj, s, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int flame_mixed(const StepArgs &a, double *scratch, double *Sd, double *Sa)
{
#define CALL(M_) run_flame_speeds<M_>(a, scratch, Sd, Sa)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

}  // namespace lbmk
