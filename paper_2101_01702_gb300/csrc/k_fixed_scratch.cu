// One double-precision time step whose working memory is a fixed array
// compiled into this library, for callers that cannot allocate GPU memory.
//
// Who needs this: code that runs where cudaMalloc is not available or not
// allowed at the point of the call -- for example a host callback or a
// plugin inside another framework that owns every device allocation, or a
// process whose allocator is capped or already exhausted.  Such callers can
// pass their own population buffers (inputs and outputs) but cannot hand the
// library the per-node macroscopic record and ghost planes that lbm_step keeps
// in caller-provided scratch buffers.  Here that scratch lives in
// g_fixed_scratch, a file-scope device array of LBM_FIXED_SCRATCH_BYTES that
// every GPU which loads the library keeps until the process exits.
//
// The kernels are the same templates as the double-precision unit
// (lbm_kernels.cuh); this translation unit has its own constant-memory copy
// of the tables, so it never touches the contexts created by lbm_create.
#define LBMK_MIXED 0
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_pack.h"

// Device-side scratch.  Layout of one call: [0, 256) status word, then the
// macroscopic record (8 N (31 + 8M) bytes), then the x-face ghost planes.
static __device__ __align__(256) unsigned char g_fixed_scratch[LBM_FIXED_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_fixed_scratch on the current device.  In host code
// the symbol name only stands for the array; the address a kernel may use
// comes from cudaGetSymbolAddress, looked up once per device.
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fixed_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int lbm_step_fixed_scratch(const lbm_lattice *lat, const lbm_species *sp, const lbm_mechanism *mech,
                                      const double *pop_in, double *pop_out, double *T_io, void *cuda_stream)
{
    if (!lat || !sp || !mech || !pop_in || !pop_out || !T_io || pop_in == pop_out) return LBM_ERR_ARG;
    if (lat->precision != LBM_FP64) return LBM_ERR_UNSUPPORTED;
    if (lat->bc_x != LBM_BC_PERIODIC && lat->bc_x != LBM_BC_EQ_ZEROGRAD_U0LEFT) return LBM_ERR_ARG;
    if (lat->nseg > 1) return LBM_ERR_UNSUPPORTED;   // batches of lattices: lbm_create
    if (lat->nx < 1 || lat->ny < 1 || lat->nz < 1 || sp->M < 2 || sp->M > LBMK_MAXM) return LBM_ERR_ARG;
    if (sp->M != 2 && sp->M != 3 && sp->M != 9) return LBM_ERR_UNSUPPORTED;
    const size_t N = (size_t)lat->nx * lat->ny * lat->nz;
    const size_t S = (size_t)sp->M + 1;
    const size_t macro_bytes = macro_bytes_for(sp->M, N, sizeof(double));
    const size_t ghost_bytes = lat->bc_x == LBM_BC_PERIODIC ? 0 : 2 * S * LBMK_Q * (size_t)lat->ny * lat->nz * sizeof(double);
    if (N > (size_t)0x7fffffff || 256 + macro_bytes + ghost_bytes > (size_t)LBM_FIXED_SCRATCH_BYTES)
        return LBM_ERR_ARG;     // lattice too large for the fixed scratch array
    // T_io is copied into the array before the step and back after it, and
    // pop_out is written while pop_in is read: overlapping ranges would
    // corrupt the state silently, so they are rejected.
    const size_t pop_bytes = S * LBMK_Q * N * sizeof(double);
    if (ranges_overlap(pop_in, pop_bytes, pop_out, pop_bytes) ||
        ranges_overlap(T_io, N * sizeof(double), pop_in, pop_bytes) ||
        ranges_overlap(T_io, N * sizeof(double), pop_out, pop_bytes))
        return LBM_ERR_ARG;
    MechConst mc;
    int st = lbm_pack_tables(sp, mech, mc);
    if (st != LBM_OK) return st;
    void *base = nullptr;
    st = scratch_address(&base);
    if (st != LBM_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned char *scratch = (unsigned char *)base;

    StepArgs a;
    a.slot = 0;
    a.M = sp->M;
    a.nx = lat->nx;
    a.ny = lat->ny;
    a.nz = lat->nz;
    a.N = (int)N;
    a.bc_x = lat->bc_x;
    a.nseg = 0;
    a.xseg = nullptr;
    a.segs = nullptr;
    for (int k = 0; k < LBMK_NKERNELS; ++k) a.bs[k] = LBMK_BLOCK;
    a.src = pop_in;
    a.dst = pop_out;
    a.status = (unsigned *)scratch;
    a.macro = (double *)(scratch + 256);
    a.ghost = ghost_bytes ? (void *)(scratch + 256 + macro_bytes) : nullptr;
    a.stream = stream;

    // The array keeps the previous call's contents: clear the status word;
    // the temperature row is the Newton starting point and comes from T_io;
    // every other row and the ghost planes are written before they are read.
    if (cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), 0, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaMemsetAsync(a.status, 0, 256, stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(a.macro + (size_t)DR_T * N, T_io, N * sizeof(double), cudaMemcpyDeviceToDevice, stream) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    int e;
    switch (sp->M) {
    case 2: e = run_step<2>(a, nullptr); break;
    case 3: e = run_step<3>(a, nullptr); break;
    default: e = run_step<9>(a, nullptr); break;
    }
    if (e) return LBM_ERR_CUDA;
    if (cudaMemcpyAsync(T_io, a.macro + (size_t)DR_T * N, N * sizeof(double), cudaMemcpyDeviceToDevice, stream) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    unsigned bits = 0;
    if (cudaMemcpyAsync(&bits, a.status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (bits & LBMK_BIT_NONFINITE) return LBM_ERR_NONFINITE;
    if (bits & LBMK_BIT_NEWTON) return LBM_ERR_NEWTON;
    if (bits & LBMK_BIT_NEGATIVE) return LBM_ERR_NEGATIVE;
    if (bits & LBMK_BIT_PIVOT) return LBM_ERR_PIVOT;
    if (bits & LBMK_BIT_BOUNDS) return LBM_ERR_BOUNDS;
    return LBM_OK;
}
