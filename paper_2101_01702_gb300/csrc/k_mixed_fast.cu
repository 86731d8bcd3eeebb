// Kernels of the reactive-mixture lattice Boltzmann step, float populations stored as deviations, with the Stefan-Maxwell solve, the relaxation rates and the exponentials of the rates in float as well (fast mixed precision).
#define LBMK_MIXED 1
#define LBMK_FAST 1
#include "lbm_kernels.cuh"

namespace lbmk {

int upload_mixed_fast(int slot, const MechConst &mc, cudaStream_t s)
{
    return (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                        cudaMemcpyHostToDevice, s);
}

int init_mixed_fast(const StepArgs &a, const double *X, const double *T, const double *u, double P)
{
#define CALL(M_) run_init<M_>(a, X, T, u, P)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int step_mixed_fast(const StepArgs &a, cudaEvent_t *ev)
{
#define CALL(M_) run_step<M_>(a, ev)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int ref_stats_mixed_fast(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out)
{
#define CALL(M_) run_ref_stats<M_>(a, X, T, P, scratch, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int launch_one_mixed_fast(const StepArgs &a, int kernel)
{
#define CALL(M_) launch_one<M_>(a, kernel)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int moments_mixed_fast(const StepArgs &a, unsigned mask, double *out)
{
#define CALL(M_) run_moments<M_>(a, mask, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

}  // namespace lbmk
