// The hand-written adjoint of the double-precision step (lbm_adjoint.cuh)
// in a translation unit of its own.  Its kernels read the species and
// mechanism tables from this unit's constant memory, which the C-ABI layer
// fills (adj_upload) with the context's record, in the context's slot,
// before every adjoint call; the forward kernels it relies on (the record
// pass, the step) run in the double-precision unit.
#define LBMK_MIXED 0
#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_adjoint.cuh"

namespace lbmk {

int adj_upload(int slot, const MechConst &mc, cudaStream_t s)
{
    return (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                        cudaMemcpyHostToDevice, s);
}

int adj_step_fp64(const StepArgs &a, const AdjBufs &g)
{
#define CALL(M_) run_adj_step<M_>(a, g)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int adj_init_T_fp64(const StepArgs &a, const double *lam0, double *out)
{
#define CALL(M_) run_adj_init_T<M_>(a, lam0, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int column_sums_fp64(const double *partial, int nb, int w, double *out, cudaStream_t s)
{
    if (w > 0) k_hrr_final<<<w, LBMK_HRR_THREADS, 0, s>>>(partial, nb, w, out);
    return (int)cudaGetLastError();
}

}  // namespace lbmk
