// Kernels of the reactive-mixture lattice Boltzmann step, double-precision populations.
#define LBMK_MIXED 0
#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

namespace {
__global__ void k_exp_check(const double *x, double *y, double *y_ref, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = exp_table(x[i]);
    y_ref[i] = exp(x[i]);
}

__global__ void k_convert_check(const float *f, double *fd, double *fd_ref, const double *d, float *df, float *df_ref,
                                int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    fd[i] = f2d(f[i]);
    fd_ref[i] = (double)f[i];
    df[i] = d2f(d[i]);
    df_ref[i] = __double2float_rn(d[i]);
}
}  // namespace

extern "C" int lbm_convert_check(const float *f, double *fd, double *fd_ref, const double *d, float *df,
                                 float *df_ref, int n, void *cuda_stream)
{
    if (!f || !fd || !fd_ref || !d || !df || !df_ref || n < 0) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    k_convert_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, fd, fd_ref, d, df, df_ref, n);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

extern "C" int lbm_exp_check(const double *x, double *y, double *y_ref, int n, void *cuda_stream)
{
    if (!x || !y || !y_ref || n < 0) return LBM_ERR_ARG;
    if (n == 0) return LBM_OK;
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    k_exp_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, y_ref, n);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

namespace lbmk {

int upload_fp64(int slot, const MechConst &mc, cudaStream_t s)
{
    // this unit's tables and those of its persistent kernel's unit
    const int e = (int)cudaMemcpyToSymbolAsync(c_mech, &mc, sizeof(MechConst), (size_t)slot * sizeof(MechConst),
                                               cudaMemcpyHostToDevice, s);
    return e ? e : upload_persistent_fp64(slot, mc, s);
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

int ref_stats_fp64(const StepArgs &a, const double *X, const double *T, double P, double *scratch, double *out)
{
#define CALL(M_) run_ref_stats<M_>(a, X, T, P, scratch, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int launch_one_fp64(const StepArgs &a, int kernel)
{
#define CALL(M_) launch_one<M_>(a, kernel)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int moments_fp64(const StepArgs &a, unsigned mask, double *out)
{
#define CALL(M_) run_moments<M_>(a, mask, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_fp64(const StepArgs &a, int R, double *dT, double *drho, double *partial, double *out)
{
#define CALL(M_) run_hrr<M_>(a, R, dT, drho, partial, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int chem_at_fp64(const StepArgs &a, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                double *dT, double *drho, double *dA)
{
#define CALL(M_) run_chem_at<M_>(a, n, rho_a, T, rho_dot, hdot, dT, drho, dA)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int temperature_at_fp64(const StepArgs &a, int n, const double *Y, const double *e, const double *T0, double *T)
{
#define CALL(M_) run_temperature_at<M_>(a, n, Y, e, T0, T)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_adj_fp64(const StepArgs &a, double *adj)
{
#define CALL(M_) run_hrr_adj<M_>(a, adj)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int hrr_adj_gather_fp64(const StepArgs &a, const double *adj, int s, double *out)
{
#define CALL(M_) run_hrr_adj_gather<M_>(a, adj, s, out)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int flame_fp64(const StepArgs &a, double *scratch, double *Sd, double *Sa)
{
#define CALL(M_) run_flame_speeds<M_>(a, scratch, Sd, Sa)
    LBMK_DISPATCH(a.M, CALL)
#undef CALL
}

int isoline_fp64(int nx, int ny, int N, const double *T, double T_iso, double cx, double cy, int K,
                 const double *fields, double *partial, double *out, cudaStream_t s)
{
    if (K < 0 || K > LBMK_ISO_MAXK) return (int)cudaErrorInvalidValue;
    const int nb = isoline_blocks((long long)nx * ny);
    k_isoline<<<nb, LBMK_HRR_THREADS, 0, s>>>(nx, ny, N, T, T_iso, cx, cy, K, fields, partial);
    k_hrr_final<<<2 + K, LBMK_HRR_THREADS, 0, s>>>(partial, nb, 2 + K, out);
    return (int)cudaGetLastError();
}

}  // namespace lbmk
