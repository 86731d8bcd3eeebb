// The persistent step (lbm_step_persistent) for double-precision populations, in a
// translation unit of its own: its one launch writes what its later phases
// read, so populations and ghost planes are read with plain loads, which
// the grid barrier's fences order, instead of the read-only path the
// per-phase kernels use.  The unit keeps its own copy of the constant
// tables, which the unit of the per-phase kernels fills beside its own.
#define LBMK_MIXED 0
#define LBMK_COHERENT_LOADS 1
#include "lbm_kernels.cuh"

namespace lbmk {

int upload_persistent_fp64(int slot, const MechConst &mc, cudaStream_t s)
{
    return (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                        cudaMemcpyHostToDevice, s);
}

int persistent_fp64(const StepArgs &a, int nsteps, int tile_mult, GridBarrier *bar, unsigned cap)
{
#define CALL(M_) run_persistent<M_>(a, nsteps, tile_mult, bar, cap)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

}  // namespace lbmk
