// Kernels of the reactive-mixture lattice Boltzmann step, double-precision populations.
#define LBMK_MIXED 0
#include "lbm_kernels.cuh"

namespace lbmk {

int upload_fp64(int slot, const MechConst &mc, cudaStream_t s)
{
    return (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                        cudaMemcpyHostToDevice, s);
}

int init_fp64(const StepArgs &a, const double *X, const double *T, const double *u, double P)
{
#define CALL(M_) run_init<M_>(a, X, T, u, P)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int step_fp64(const StepArgs &a, cudaEvent_t *ev)
{
#define CALL(M_) run_step<M_>(a, ev)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int moments_fp64(const StepArgs &a, unsigned mask, double *out)
{
#define CALL(M_) run_moments<M_>(a, mask, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

}  // namespace lbmk
