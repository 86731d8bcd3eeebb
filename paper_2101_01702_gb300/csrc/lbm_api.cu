// C ABI of the reactive-mixture lattice Boltzmann library (include/lbm.h).
//
// Host side only: argument validation, packing of the species and mechanism
// tables into the constant-memory record the kernels read (slots shared by
// identical tables), buffer binding, the A/B swap of the population buffers,
// CUDA-graph replay, and status reporting.  Every step of the numerical
// method runs in the kernels of k_fp64.cu, k_mixed.cu and k_mixed_fast.cu.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_pack.h"

struct lbm_ctx {
    lbm_lattice lat;
    int M, S, N, slot;
    cudaStream_t stream;
    void *buf[2];
    int cur;                 // index of the buffer holding the current state
    double *macro;
    void *ghost;
    size_t pop_bytes;
    unsigned *status;        // device status word
    MechConst mc;            // host copy of the constant-memory record
    int nseg;                // lattices side by side in x (>= 2), else 0
    int4 *xseg;              // device [nx]: {x0, x1, k, 0} of the lattice at x
    int2 *segs;              // device [nseg]: {x0, x1} of lattice k
    cudaGraphExec_t graph;   // two captured steps (lbm_step_graph), or null
    int graph_cur;           // value of cur the graph starts from
    bool refs_fixed;         // rest references set by lbm_set_references
    int bs[LBMK_NKERNELS];   // threads per block of each kernel (lbm_autotune)
    int dev;                 // CUDA device current at lbm_create
};

namespace {

// Constant-memory slots of each kernel unit (precision) on each device.
// Contexts on one device whose packed tables are identical -- the same
// mechanism and, in the mixed modes, the same rest references -- share a
// slot; a slot is uploaded when it is taken and reused once no context
// refers to it.  Constant memory is per device, so each device keeps its
// own table: a slot uploaded on one device holds nothing on another.
struct SlotTable {
    int refs[LBMK_SLOTS];
    MechConst mc[LBMK_SLOTS];
};
std::mutex g_slot_mutex;
std::map<int, std::array<SlotTable, 3>> g_slots;    // device -> precision -> slots

bool supported_M(int M) { return M == 2 || M == 3 || M == 9; }

bool is_mixed(int precision) { return precision == LBM_MIXED || precision == LBM_MIXED_FAST; }
bool valid_precision(int precision) { return precision == LBM_FP64 || is_mixed(precision); }
size_t store_size(int precision) { return is_mixed(precision) ? sizeof(float) : sizeof(double); }

const lbmk::PrecisionOps kOps[3] = {
    {lbmk::upload_fp64, lbmk::init_fp64, lbmk::step_fp64, lbmk::moments_fp64, lbmk::ref_stats_fp64,
     lbmk::launch_one_fp64, lbmk::hrr_fp64,
     lbmk::chem_at_fp64, lbmk::temperature_at_fp64,
     lbmk::hrr_adj_fp64, lbmk::hrr_adj_gather_fp64, lbmk::flame_fp64, lbmk::persistent_fp64},
    {lbmk::upload_mixed, lbmk::init_mixed, lbmk::step_mixed, lbmk::moments_mixed, lbmk::ref_stats_mixed,
     lbmk::launch_one_mixed, lbmk::hrr_mixed,
     lbmk::chem_at_mixed, lbmk::temperature_at_mixed,
     lbmk::hrr_adj_mixed, lbmk::hrr_adj_gather_mixed, lbmk::flame_mixed, lbmk::persistent_mixed},
    {lbmk::upload_mixed_fast, lbmk::init_mixed_fast, lbmk::step_mixed_fast, lbmk::moments_mixed_fast,
     lbmk::ref_stats_mixed_fast, lbmk::launch_one_mixed_fast, lbmk::hrr_mixed_fast,
     lbmk::chem_at_mixed_fast, lbmk::temperature_at_mixed_fast,
     lbmk::hrr_adj_mixed_fast, lbmk::hrr_adj_gather_mixed_fast, lbmk::flame_mixed_fast,
     lbmk::persistent_mixed_fast},
};
const lbmk::PrecisionOps &ops(int precision) { return kOps[precision]; }

// A slot of precision p on device dev (the current device) holding mc
// (shared or newly uploaded on stream and waited for); -1 when every slot
// holds other tables.
int acquire_slot(int dev, int p, const MechConst &mc, cudaStream_t stream, int *err)
{
    *err = LBM_OK;
    std::lock_guard<std::mutex> lk(g_slot_mutex);
    SlotTable &t = g_slots[dev][p];
    for (int s = 0; s < LBMK_SLOTS; ++s)
        if (t.refs[s] > 0 && memcmp(&t.mc[s], &mc, sizeof(MechConst)) == 0) {
            ++t.refs[s];
            return s;
        }
    for (int s = 0; s < LBMK_SLOTS; ++s)
        if (t.refs[s] == 0) {
            if (ops(p).upload(s, mc, stream) != 0 || cudaStreamSynchronize(stream) != cudaSuccess) {
                *err = LBM_ERR_CUDA;
                return -1;
            }
            t.mc[s] = mc;
            t.refs[s] = 1;
            return s;
        }
    *err = LBM_ERR_UNSUPPORTED;
    return -1;
}

void release_slot(int dev, int p, int s)
{
    if (s < 0 || s >= LBMK_SLOTS) return;
    std::lock_guard<std::mutex> lk(g_slot_mutex);
    auto it = g_slots.find(dev);
    if (it != g_slots.end() && it->second[p].refs[s] > 0) --it->second[p].refs[s];
}

// LBM_OK when the calling thread's current device is the one c was created
// on; its buffers, stream and constant-memory slot live there.
int on_ctx_device(const lbm_ctx *c)
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return LBM_ERR_CUDA;
    return d == c->dev ? LBM_OK : LBM_ERR_ARG;
}

// Moves context c to a slot holding c->mc (after its stream has drained,
// so that none of its kernels still reads the old slot).
int reslot(lbm_ctx *c)
{
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LBM_ERR_CUDA;
    int err;
    const int s = acquire_slot(c->dev, c->lat.precision, c->mc, c->stream, &err);
    if (s < 0) return err;
    release_slot(c->dev, c->lat.precision, c->slot);
    c->slot = s;
    if (c->graph) {                      // captured with the old slot
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LBM_OK;
}

int map_status(unsigned bits)
{
    if (bits & LBMK_BIT_NONFINITE) return LBM_ERR_NONFINITE;
    if (bits & LBMK_BIT_NEWTON) return LBM_ERR_NEWTON;
    if (bits & LBMK_BIT_NEGATIVE) return LBM_ERR_NEGATIVE;
    if (bits & LBMK_BIT_PIVOT) return LBM_ERR_PIVOT;
    if (bits & LBMK_BIT_BOUNDS) return LBM_ERR_BOUNDS;
    if (bits & LBMK_BIT_BARRIER) return LBM_ERR_BARRIER;
    return LBM_OK;
}

// Lattices side by side in x: LBM_OK when lat describes one lattice or a
// valid batch (lengths >= 1 summing to nx, equilibrium ghost faces).
int check_segments(const lbm_lattice *lat)
{
    if (lat->nseg < 0) return LBM_ERR_ARG;
    if (lat->nseg <= 1) return LBM_OK;
    if (!lat->seg_nx || lat->bc_x != LBM_BC_EQ_ZEROGRAD_U0LEFT || lat->nseg > lat->nx) return LBM_ERR_ARG;
    long long sum = 0;
    for (int k = 0; k < lat->nseg; ++k) {
        if (lat->seg_nx[k] < 1) return LBM_ERR_ARG;
        sum += lat->seg_nx[k];
    }
    return sum == lat->nx ? LBM_OK : LBM_ERR_ARG;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

StepArgs args_of(const lbm_ctx *c)
{
    StepArgs a;
    a.slot = c->slot;
    a.M = c->M;
    a.nx = c->lat.nx;
    a.ny = c->lat.ny;
    a.nz = c->lat.nz;
    a.N = c->N;
    a.bc_x = c->lat.bc_x;
    for (int k = 0; k < LBMK_NKERNELS; ++k) a.bs[k] = c->bs[k];
    a.nseg = c->nseg;
    a.xseg = c->xseg;
    a.segs = c->segs;
    a.src = c->buf[c->cur];
    a.dst = c->buf[1 - c->cur];
    a.macro = c->macro;
    a.ghost = c->ghost;
    a.status = c->status;
    a.stream = c->stream;
    return a;
}

double psi_host(int c, double zeta) { return c == 0 ? 1.0 - zeta : 0.5 * zeta; }

// Rest states subtracted by mixed-precision storage of the moving
// populations of the species and mixture sets: each set's rest equilibrium
// at the mean initial temperature and at the smallest initial density of
// that set, so that the stored deviations of positive populations stay
// non-negative and trace species keep float's relative precision.
// st: the statistics of the initial state from lbmk::ref_stats_* (min
// rho_a (M), min rho, sum rho_a (M), sum rho, sum T) over N nodes.
void references_from_stats(MechConst &mc, int M, const double *st, size_t N)
{
    const double rho_tmin = st[M];
    const double rho_t = st[2 * M + 1] / (double)N;
    const double T_m = st[2 * M + 2] / (double)N;
    double inv_m = 0.0;
    for (int a = 0; a < M; ++a) inv_m += st[M + 1 + a] / (double)N / rho_t / mc.W[a];
    const double Rm = mc.r_lat * inv_m;
    for (int s = 0; s < M; ++s)
        for (int i = 0; i < LBMK_Q; ++i) {
            const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
            const double zeta = (s < M - 1 ? mc.Ra[s] : Rm) * T_m;
            const double r = s < M - 1 ? st[s] : rho_tmin;
            const double v = r * psi_host(cx, zeta) * psi_host(cy, zeta) * psi_host(cz, zeta);
            mc.ref[s][i] = i == 13 ? 0.0f : (float)v;     // rest populations are stored in double
        }
    lbmk_reference_moments(mc, M);
}

int check_cuda(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

// Workspace of the adjoint calls, in doubles from a 256-byte aligned base:
// every region starts on a 256-byte boundary.
struct AdjLayout {
    size_t tkeep, fbar, mbar, coef, aux, theta, theta_out;     // one reverse step
    size_t lamA, lamB, ck, ckT, seg, segT, jpart, hrrpart, dT0;  // gradient through time
    size_t total;                                                // bytes
    int nck;
};

AdjLayout adj_layout(const lbm_ctx *c, int nsteps, int every)
{
    const size_t N = (size_t)c->N, pop = (size_t)c->S * LBMK_Q * N, R = (size_t)std::max(c->mc.R, 1);
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t at = off;
        off += (n + 31) & ~(size_t)31;
        return at;
    };
    AdjLayout L;
    L.tkeep = take(N);
    L.fbar = take(pop);
    L.mbar = take((size_t)adj_mbar_rows(c->M) * N);
    L.coef = take((size_t)c->M * N);
    L.aux = take(10 * N);
    L.theta = take((size_t)adj_blocks(c->N) * R);
    L.theta_out = take(R);
    // every = 0: the objective alone (no checkpoints, no reverse sweep)
    L.nck = nsteps > 0 && every > 0 ? (nsteps + every - 1) / every : 0;
    L.lamA = L.lamB = L.ck = L.ckT = L.seg = L.segT = L.jpart = L.hrrpart = L.dT0 = 0;
    if (nsteps > 0) {
        L.jpart = take((size_t)nsteps * (1 + R));
        L.hrrpart = take((size_t)lbmk::hrr_blocks(c->N) * (1 + R));
    }
    if (nsteps > 0 && every > 0) {
        L.lamA = take(pop);
        L.lamB = take(pop);
        L.ck = take((size_t)L.nck * pop);
        L.ckT = take((size_t)L.nck * N);
        L.seg = take((size_t)every * pop);
        L.segT = take((size_t)every * N);
        L.dT0 = take(N);
    }
    L.total = off * sizeof(double);
    return L;
}

// LBM_OK when the adjoint supports context c (double precision, one
// periodic lattice, constant transport).
int adjoint_supported(const lbm_ctx *c)
{
    if (c->lat.precision != LBM_FP64 || c->lat.bc_x != LBM_BC_PERIODIC || c->nseg > 1 || c->mc.transport)
        return LBM_ERR_UNSUPPORTED;
    return LBM_OK;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

int copy_d2d(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
}

// The record of the step at a.src (moments, temperature, relaxation,
// Stefan-Maxwell solve; then G), as the forward step's first passes form it.
int adj_record(const StepArgs &a)
{
    int e = lbmk::launch_one_fp64(a, LBMK_K_PRE);
    if (!e) e = lbmk::launch_one_fp64(a, LBMK_K_GRAD);
    return e;
}

}  // namespace

extern "C" {

int lbm_buffer_sizes(const lbm_lattice *lat, const lbm_species *sp, size_t *pop_bytes, size_t *macro_bytes,
                     size_t *ghost_bytes)
{
    if (!lat || !sp || lat->nx < 1 || lat->ny < 1 || lat->nz < 1 || sp->M < 2 || sp->M > LBMK_MAXM)
        return LBM_ERR_ARG;
    if (!valid_precision(lat->precision)) return LBM_ERR_ARG;
    if (lat->bc_x != LBM_BC_PERIODIC && lat->bc_x != LBM_BC_EQ_ZEROGRAD_U0LEFT) return LBM_ERR_ARG;
    if (check_segments(lat) != LBM_OK) return LBM_ERR_ARG;
    const size_t N = (size_t)lat->nx * lat->ny * lat->nz;
    const size_t S = (size_t)sp->M + 1;
    const size_t st = store_size(lat->precision);
    if (pop_bytes) *pop_bytes = pop_bytes_for((int)S, N, is_mixed(lat->precision));
    if (macro_bytes) *macro_bytes = macro_bytes_for(sp->M, N, st);
    if (ghost_bytes)
        *ghost_bytes = lat->bc_x == LBM_BC_PERIODIC
                           ? 0
                           : ghost_bytes_for((int)S, (size_t)lat->ny * lat->nz, lat->nseg > 1 ? lat->nseg : 1);
    return LBM_OK;
}

int lbm_create(const lbm_lattice *lat, const lbm_species *sp, const lbm_mechanism *mech, const lbm_buffers *bufs,
               void *cuda_stream, lbm_ctx **out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!lat || !sp || !mech || !bufs) return LBM_ERR_ARG;
    if (lat->bc_x != LBM_BC_PERIODIC && lat->bc_x != LBM_BC_EQ_ZEROGRAD_U0LEFT) return LBM_ERR_ARG;
    size_t need_pop, need_mac, need_gh;
    int r = lbm_buffer_sizes(lat, sp, &need_pop, &need_mac, &need_gh);
    if (r != LBM_OK) return r;
    const size_t N = (size_t)lat->nx * lat->ny * lat->nz;
    if (N > (size_t)0x7fffffff) return LBM_ERR_ARG;
    const int M = sp->M;
    if (!supported_M(M)) return LBM_ERR_UNSUPPORTED;
    if (!bufs->pop_a || !bufs->pop_b || bufs->pop_a == bufs->pop_b || !bufs->macro) return LBM_ERR_ARG;
    if (bufs->pop_bytes < need_pop || bufs->macro_bytes < need_mac) return LBM_ERR_ARG;
    if (need_gh && (!bufs->ghost || bufs->ghost_bytes < need_gh)) return LBM_ERR_ARG;
    if (((uintptr_t)bufs->pop_a | (uintptr_t)bufs->pop_b | (uintptr_t)bufs->macro) & 15u) return LBM_ERR_ARG;

    MechConst mc;
    r = lbm_pack_tables(sp, mech, mc);
    if (r != LBM_OK) return r;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    int err = LBM_OK;
    const int slot = acquire_slot(dev, lat->precision, mc, (cudaStream_t)cuda_stream, &err);
    if (slot < 0) return err;

    lbm_ctx *c = (lbm_ctx *)calloc(1, sizeof(lbm_ctx));
    if (!c) {
        release_slot(dev, lat->precision, slot);
        return LBM_ERR_ARG;
    }
    c->dev = dev;
    c->lat = *lat;
    c->M = M;
    c->S = M + 1;
    c->N = (int)N;
    c->slot = slot;
    c->stream = (cudaStream_t)cuda_stream;
    c->buf[0] = bufs->pop_a;
    c->buf[1] = bufs->pop_b;
    c->cur = 0;
    c->macro = (double *)bufs->macro;
    c->ghost = bufs->ghost;
    c->pop_bytes = need_pop;
    c->mc = mc;
    c->lat.seg_nx = nullptr;     // read here only
    for (int k = 0; k < LBMK_NKERNELS; ++k) c->bs[k] = LBMK_BLOCK;
    // the status word, then (at byte 16) the persistent step's barrier state
    int st = check_cuda(cudaMalloc((void **)&c->status, 16 + sizeof(GridBarrier)));
    if (st == LBM_OK) st = check_cuda(cudaMemsetAsync(c->status, 0, 16 + sizeof(GridBarrier), c->stream));
    if (st == LBM_OK && lat->nseg > 1) {
        // per-x and per-lattice ranges of the batch
        const int nx = lat->nx, ns = lat->nseg;
        int4 *hx = (int4 *)malloc((size_t)nx * sizeof(int4));
        int2 *hs = (int2 *)malloc((size_t)ns * sizeof(int2));
        if (!hx || !hs) st = LBM_ERR_ARG;
        for (int k = 0, x0 = 0; st == LBM_OK && k < ns; x0 += lat->seg_nx[k], ++k) {
            hs[k] = make_int2(x0, x0 + lat->seg_nx[k]);
            for (int x = x0; x < x0 + lat->seg_nx[k]; ++x) hx[x] = make_int4(x0, x0 + lat->seg_nx[k], k, 0);
        }
        if (st == LBM_OK) st = check_cuda(cudaMalloc((void **)&c->xseg, (size_t)nx * sizeof(int4)));
        if (st == LBM_OK) st = check_cuda(cudaMalloc((void **)&c->segs, (size_t)ns * sizeof(int2)));
        if (st == LBM_OK) st = check_cuda(cudaMemcpy(c->xseg, hx, (size_t)nx * sizeof(int4), cudaMemcpyHostToDevice));
        if (st == LBM_OK) st = check_cuda(cudaMemcpy(c->segs, hs, (size_t)ns * sizeof(int2), cudaMemcpyHostToDevice));
        if (st == LBM_OK) c->nseg = ns;
        free(hx);
        free(hs);
    }
    if (st == LBM_OK) st = check_cuda(cudaStreamSynchronize(c->stream));
    if (st != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

int lbm_init(lbm_ctx *c, const double *X, const double *T, const double *u, double P)
{
    if (!c || !X || !T || !(P > 0)) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const size_t N = (size_t)c->N, M = (size_t)c->M;
    const bool dX = is_device_ptr(X), dT = is_device_ptr(T), du = u ? is_device_ptr(u) : dX;
    if (dX != dT || dX != du) return LBM_ERR_ARG;     // all host or all device
    int st = LBM_OK;
    // The second population buffer is free until the first step: host fields
    // are staged there, followed by the scratch of the reference statistics.
    double *stage = (double *)c->buf[1 - c->cur];
    const size_t stage_doubles = dX ? 0 : (M + 4) * N;
    if (stage_doubles * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
    const double *dXp = X, *dTp = T, *dup = u;
    if (!dX) {
        st = check_cuda(cudaMemcpyAsync(stage, X, M * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (st == LBM_OK)
            st = check_cuda(cudaMemcpyAsync(stage + M * N, T, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (st == LBM_OK && u)
            st = check_cuda(cudaMemcpyAsync(stage + (M + 1) * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice,
                                            c->stream));
        if (st != LBM_OK) return st;
        dXp = stage;
        dTp = stage + M * N;
        dup = u ? stage + (M + 1) * N : nullptr;
    }
    if (is_mixed(c->lat.precision) && !c->refs_fixed) {
        // rest references from statistics of the initial state, reduced on
        // the GPU in a fixed order
        const size_t len = 2 * M + 3;
        const size_t nb = std::min<size_t>(LBMK_STAT_BLOCKS, (N + 255) / 256);
        const size_t off = (stage_doubles + 31) & ~(size_t)31;
        if ((off + (nb + 1) * len) * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
        double *scratch = stage + off, *dstat = scratch + nb * len;
        if (ops(c->lat.precision).ref_stats(args_of(c), dXp, dTp, P, scratch, dstat)) return LBM_ERR_CUDA;
        double hstat[2 * LBMK_MAXM + 3];
        st = check_cuda(cudaMemcpyAsync(hstat, dstat, len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (st == LBM_OK) st = check_cuda(cudaStreamSynchronize(c->stream));
        if (st != LBM_OK) return st;
        for (size_t k = 0; k < len; ++k)
            if (!isfinite(hstat[k])) return LBM_ERR_ARG;      // a non-finite or non-positive initial state
        references_from_stats(c->mc, c->M, hstat, N);
        st = reslot(c);
        if (st != LBM_OK) return st;
    }
    StepArgs a = args_of(c);
    a.dst = c->buf[c->cur];
    const int e = ops(c->lat.precision).init(a, dXp, dTp, dup, P);
    if (e) return LBM_ERR_CUDA;
    st = check_cuda(cudaMemsetAsync(c->status, 0, 16, c->stream));
    if (st == LBM_OK) st = check_cuda(cudaStreamSynchronize(c->stream));
    return st;
}

int lbm_step_async(lbm_ctx *c, int n)
{
    if (!c || n < 0) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    for (int t = 0; t < n; ++t) {
        StepArgs a = args_of(c);
        const int e = ops(c->lat.precision).step(a, nullptr);
        if (e) return LBM_ERR_CUDA;
        c->cur = 1 - c->cur;
    }
    return LBM_OK;
}

int lbm_step_graph(lbm_ctx *c, int n)
{
    if (!c || n < 0) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (c->stream == nullptr) return LBM_ERR_UNSUPPORTED;   // the legacy default stream cannot be captured
    if (!c->graph) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
        const int cur0 = c->cur;
        int e = 0;
        for (int t = 0; t < 2 && !e; ++t) {
            StepArgs a = args_of(c);
            e = ops(c->lat.precision).step(a, nullptr);
            c->cur = 1 - c->cur;
        }
        c->cur = cur0;
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        if (e || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        cudaGraphExec_t x = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return LBM_ERR_CUDA;
        c->graph = x;
        c->graph_cur = cur0;
    }
    int left = n;
    if (left > 0 && c->cur != c->graph_cur) {
        const int st = lbm_step_async(c, 1);
        if (st != LBM_OK) return st;
        --left;
    }
    for (; left >= 2; left -= 2)          // two steps leave cur where it was
        if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) return LBM_ERR_CUDA;
    return left == 1 ? lbm_step_async(c, 1) : LBM_OK;
}

int lbm_step_persistent(lbm_ctx *c, int n, int tile_mult, unsigned spin_cap)
{
    if (!c || n < 0 || tile_mult < 1) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (n == 0) return lbm_sync(c);
    // the barrier state follows the status word's 16 bytes
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(c->status + 4);
    int st = check_cuda(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), c->stream));
    if (st != LBM_OK) return st;
    const int e = ops(c->lat.precision).persistent(args_of(c), n, tile_mult, bar, spin_cap ? spin_cap : (1u << 24));
    if (e == (int)cudaErrorNotSupported) return LBM_ERR_UNSUPPORTED;
    if (e) return LBM_ERR_CUDA;
    if (n & 1) c->cur = 1 - c->cur;
    return lbm_sync(c);
}

int lbm_autotune_persistent(lbm_ctx *c, int steps, int *tile_mult_out)
{
    if (!c || steps < 1 || !tile_mult_out) return LBM_ERR_ARG;
    int st = lbm_sync(c);
    if (st != LBM_OK) return st;
    const size_t Tb = (size_t)c->N * sizeof(double);
    const int cur0 = c->cur;
    void *keep = nullptr;
    if (cudaMalloc(&keep, c->pop_bytes + Tb) != cudaSuccess) return LBM_ERR_CUDA;
    double *Trow = c->macro + (size_t)DR_T * c->N;
    st = copy_d2d(keep, c->buf[cur0], c->pop_bytes, c->stream);
    if (st == LBM_OK) st = copy_d2d((char *)keep + c->pop_bytes, Trow, Tb, c->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = LBM_ERR_CUDA;
    static const int cand[4] = {1, 2, 4, 8};
    float best = 0.f;
    int best_t = 1;
    for (int j = 0; j < 4 && st == LBM_OK; ++j) {
        for (int rep = 0; rep < 2 && st == LBM_OK; ++rep) {    // once to warm up, once timed
            c->cur = cur0;
            st = copy_d2d(c->buf[cur0], keep, c->pop_bytes, c->stream);
            if (st == LBM_OK) st = copy_d2d(Trow, (char *)keep + c->pop_bytes, Tb, c->stream);
            if (st == LBM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = LBM_ERR_CUDA;
            if (st == LBM_OK) st = lbm_step_persistent(c, steps, cand[j], 0);
            if (st == LBM_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = LBM_ERR_CUDA;
        }
        float ms = 0.f;
        if (st == LBM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = LBM_ERR_CUDA;
        if (st == LBM_OK && (best == 0.f || ms < best)) {
            best = ms;
            best_t = cand[j];
        }
    }
    c->cur = cur0;
    const int st2 = copy_d2d(c->buf[cur0], keep, c->pop_bytes, c->stream);
    const int st3 = copy_d2d(Trow, (char *)keep + c->pop_bytes, Tb, c->stream);
    const int st4 = check_cuda(cudaStreamSynchronize(c->stream));
    cudaFree(keep);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st == LBM_OK) st = st2 != LBM_OK ? st2 : (st3 != LBM_OK ? st3 : st4);
    if (st == LBM_OK) *tile_mult_out = best_t;
    return st;
}

int lbm_autotune(lbm_ctx *c, int trials, int *block_out)
{
    if (!c || trials < 1 || trials > 1000) return LBM_ERR_ARG;
    int st = lbm_sync(c);
    if (st != LBM_OK) return st;
    // Candidate blocks per kernel: k_pre and k_step carry register caps for
    // 128-thread blocks, so at most 128; the others up to LBMK_MAXBLOCK.
    static const int cand[3] = {64, 128, 256};
    const int maxbs[LBMK_NKERNELS] = {LBMK_BLOCK, LBMK_BLOCK, LBMK_MAXBLOCK, LBMK_MAXBLOCK, LBMK_MAXBLOCK,
                                      LBMK_BLOCK};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return LBM_ERR_CUDA;
    }
    const lbmk::PrecisionOps &op = ops(c->lat.precision);
    // Every kernel of the step reads the current state (and the record the
    // earlier kernels write from it) and writes only the record and the other
    // buffer, so repeating any of them leaves the state as it was -- except
    // the temperature row, the Newton start of the next step, which repeated
    // iterations may move by a rounding: it is kept aside and put back.
    double *t_keep = nullptr;
    const size_t tbytes = (size_t)c->N * sizeof(double);
    if (cudaMalloc((void **)&t_keep, tbytes) != cudaSuccess ||
        cudaMemcpyAsync(t_keep, c->macro + (size_t)DR_T * c->N, tbytes, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess) {
        if (t_keep) cudaFree(t_keep);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return LBM_ERR_CUDA;
    }
    for (int k = 0; k < LBMK_NKERNELS && st == LBM_OK; ++k) {
        StepArgs a = args_of(c);
        if (op.launch_one(a, k)) { st = LBM_ERR_CUDA; break; }     // the kernel's inputs, at the current choice
        if (k == LBMK_K_GHOST) continue;
        float best = 0.f;
        for (int j = 0; j < 3 && st == LBM_OK; ++j) {
            if (cand[j] > maxbs[k]) continue;
            a.bs[k] = cand[j];
            for (int w = 0; w < 2 + trials && st == LBM_OK; ++w) {   // 2 untimed, then trials timed
                if (w == 2 && cudaEventRecord(e0, c->stream) != cudaSuccess) st = LBM_ERR_CUDA;
                if (op.launch_one(a, k)) st = LBM_ERR_CUDA;
            }
            if (st != LBM_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = LBM_ERR_CUDA;
                break;
            }
            if (best == 0.f || ms < best) {
                best = ms;
                c->bs[k] = cand[j];
            }
        }
        a = args_of(c);
        if (st == LBM_OK && op.launch_one(a, k)) st = LBM_ERR_CUDA;   // leave its outputs from the choice
    }
    if (cudaMemcpyAsync(c->macro + (size_t)DR_T * c->N, t_keep, tbytes, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        st = LBM_ERR_CUDA;
    cudaFree(t_keep);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (c->graph) {                      // captured with the previous blocks
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (block_out)
        for (int k = 0; k < LBMK_NKERNELS; ++k) block_out[k] = c->bs[k];
    if (st != LBM_OK) return st;
    return lbm_sync(c);
}

int lbm_set_blocks(lbm_ctx *c, const int *blocks)
{
    if (!c || !blocks) return LBM_ERR_ARG;
    const int maxbs[LBMK_NKERNELS] = {LBMK_BLOCK, LBMK_BLOCK, LBMK_MAXBLOCK, LBMK_MAXBLOCK, LBMK_MAXBLOCK,
                                      LBMK_BLOCK};
    for (int k = 0; k < LBMK_NKERNELS; ++k) {
        const int b = blocks[k];
        if ((b != 64 && b != 128 && b != 256) || b > maxbs[k] || (k == LBMK_K_GHOST && b != LBMK_BLOCK))
            return LBM_ERR_ARG;
    }
    for (int k = 0; k < LBMK_NKERNELS; ++k) c->bs[k] = blocks[k];
    if (c->graph) {                      // captured with the previous blocks
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LBM_OK;
}

int lbm_step_timed(lbm_ctx *c, int n, double *phase_ms)
{
    if (!c || n < 0 || !phase_ms) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    for (int k = 0; k <= LBM_PHASES; ++k) phase_ms[k] = 0.0;
    if (n == 0) return lbm_sync(c);
    // LBM_PHASES + 1 events per step, all recorded before the one wait, so
    // that the timed steps run back to back as in lbm_step_async.
    const size_t nev = (size_t)n * (LBM_PHASES + 1);
    cudaEvent_t *ev = (cudaEvent_t *)calloc(nev, sizeof(cudaEvent_t));
    if (!ev) return LBM_ERR_ARG;
    int st = LBM_OK;
    size_t made = 0;
    for (; made < nev; ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) { st = LBM_ERR_CUDA; break; }
    for (int t = 0; t < n && st == LBM_OK; ++t) {
        StepArgs a = args_of(c);
        cudaEvent_t *e = ev + (size_t)t * (LBM_PHASES + 1);
        const int r = ops(c->lat.precision).step(a, e);
        if (r) { st = LBM_ERR_CUDA; break; }
        c->cur = 1 - c->cur;
    }
    if (st == LBM_OK && cudaEventSynchronize(ev[nev - 1]) != cudaSuccess) st = LBM_ERR_CUDA;
    for (int t = 0; t < n && st == LBM_OK; ++t) {
        cudaEvent_t *e = ev + (size_t)t * (LBM_PHASES + 1);
        for (int k = 0; k < LBM_PHASES; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e[k], e[k + 1]);
            phase_ms[k] += ms;
        }
    }
    if (st == LBM_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[nev - 1]);
        phase_ms[LBM_PHASES] = ms;
    }
    for (size_t k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    free(ev);
    if (st != LBM_OK) return st;
    return lbm_sync(c);
}

int lbm_sync(lbm_ctx *c)
{
    if (!c) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    unsigned bits = 0;
    int st = check_cuda(cudaMemcpyAsync(&bits, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    if (st == LBM_OK) st = check_cuda(cudaStreamSynchronize(c->stream));
    if (st != LBM_OK) return st;
    if (bits) {
        st = check_cuda(cudaMemsetAsync(c->status, 0, 16, c->stream));
        if (st != LBM_OK) return st;
    }
    return map_status(bits);
}

int lbm_step(lbm_ctx *c, int n)
{
    int st = lbm_step_async(c, n);
    if (st != LBM_OK) return st;
    return lbm_sync(c);
}

size_t lbm_moments_count(const lbm_ctx *c, unsigned mask)
{
    if (!c) return 0;
    size_t rows = 0;
    if (mask & LBM_F_RHO_A) rows += c->M;
    if (mask & LBM_F_RHOU) rows += 3;
    if (mask & LBM_F_RHOE) rows += 1;
    if (mask & LBM_F_T) rows += 1;
    if (mask & LBM_F_P) rows += 1;
    if (mask & LBM_F_Y) rows += c->M;
    if (mask & LBM_F_J_A) rows += 3 * (size_t)c->M;
    if (mask & LBM_F_RHO_DOT) rows += c->M;
    if (mask & LBM_F_HRR) rows += 1;
    return rows * (size_t)c->N;
}

int lbm_moments(lbm_ctx *c, unsigned mask, double *out)
{
    if (!c || !out || mask == 0 || (mask & ~511u)) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const size_t count = lbm_moments_count(c, mask);
    const bool dev = is_device_ptr(out);
    double *target = out;
    if (!dev) {
        if (count * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
        target = (double *)c->buf[1 - c->cur];
    }
    StepArgs a = args_of(c);
    const int e = ops(c->lat.precision).moments(a, mask, target);
    if (e) return LBM_ERR_CUDA;
    if (!dev) {
        int st = check_cuda(cudaMemcpyAsync(out, target, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (st != LBM_OK) return st;
    }
    return lbm_sync(c);
}

int lbm_heat_release(lbm_ctx *c, double *J, double *dJ_dlogA, double *dJ_dT, double *dJ_drho)
{
    if (!c || !J) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const size_t N = (size_t)c->N, M = (size_t)c->M;
    const int R = c->mc.R;
    const bool dT_dev = dJ_dT && is_device_ptr(dJ_dT), dr_dev = dJ_drho && is_device_ptr(dJ_drho);
    // Scratch in the free population buffer: the rows bound for host
    // memory, then the per-block partial sums and the totals.
    double *stage = (double *)c->buf[1 - c->cur];
    size_t off = 0;
    double *dT = dJ_dT, *dr = dJ_drho;
    if (dJ_dT && !dT_dev) { dT = stage + off; off += N; }
    if (dJ_drho && !dr_dev) { dr = stage + off; off += M * N; }
    off = (off + 31) & ~(size_t)31;
    double *partial = stage + off;
    off += (size_t)lbmk::hrr_blocks(c->N) * (1 + R);
    double *tot = stage + off;
    off += 1 + R;
    if (off * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
    if (ops(c->lat.precision).hrr(args_of(c), R, dT, dr, partial, tot)) return LBM_ERR_CUDA;
    double htot[1 + LBMK_MAXR];
    int st = check_cuda(cudaMemcpyAsync(htot, tot, (1 + R) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (st == LBM_OK && dJ_dT && !dT_dev)
        st = check_cuda(cudaMemcpyAsync(dJ_dT, dT, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (st == LBM_OK && dJ_drho && !dr_dev)
        st = check_cuda(cudaMemcpyAsync(dJ_drho, dr, M * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (st == LBM_OK) st = lbm_sync(c);
    if (st != LBM_OK) return st;
    *J = htot[0];
    if (dJ_dlogA)
        for (int k = 0; k < R; ++k) dJ_dlogA[k] = htot[1 + k];
    return LBM_OK;
}

int lbm_heat_release_adjoint(lbm_ctx *c, double *dJ_dF)
{
    if (!c || !dJ_dF) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (c->lat.bc_x != LBM_BC_PERIODIC || c->nseg > 1) return LBM_ERR_UNSUPPORTED;
    const size_t N = (size_t)c->N, S = (size_t)c->S, M = (size_t)c->M;
    const bool dev = is_device_ptr(dJ_dF);
    // scratch in the free population buffer: the per-node moment
    // derivatives, then (host output) one set's rows at a time
    double *adj = (double *)c->buf[1 - c->cur];
    double *rows = adj + (M + 4) * N;
    if (((M + 4) * N + (dev ? 0 : LBMK_Q * N)) * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
    const StepArgs a = args_of(c);
    if (ops(c->lat.precision).hrr_adj(a, adj)) return LBM_ERR_CUDA;
    for (size_t s = 0; s < S; ++s) {
        double *target = dev ? dJ_dF + s * LBMK_Q * N : rows;
        if (ops(c->lat.precision).hrr_adj_gather(a, adj, (int)s, target)) return LBM_ERR_CUDA;
        if (!dev) {
            const int st = check_cuda(cudaMemcpyAsync(dJ_dF + s * LBMK_Q * N, rows, LBMK_Q * N * sizeof(double),
                                                      cudaMemcpyDeviceToHost, c->stream));
            if (st != LBM_OK) return st;
        }
    }
    return lbm_sync(c);
}

int lbm_adjoint_workspace_bytes(const lbm_ctx *c, int nsteps, int every, size_t *bytes)
{
    if (!c || !bytes || nsteps < 0 || every < 0 || (every == 0 && nsteps == 0)) return LBM_ERR_ARG;
    *bytes = adj_layout(c, nsteps, every).total + 256;      // room to align the caller's base
    return LBM_OK;
}

namespace {
double *ws_base(void *ws) { return (double *)(((uintptr_t)ws + 255) & ~(uintptr_t)255); }

AdjBufs adj_bufs(double *w, const AdjLayout &L)
{
    AdjBufs g;
    g.lam_next = nullptr;
    g.lam = nullptr;
    g.fbar = w + L.fbar;
    g.mbar = w + L.mbar;
    g.coef = w + L.coef;
    g.aux = w + L.aux;
    g.theta = w + L.theta;
    g.with_objective = 1;
    return g;
}
}  // namespace

int lbm_adjoint_step(lbm_ctx *c, const double *lam_next, double *lam, double *dJ_dlogA, int with_objective,
                     void *workspace, size_t workspace_bytes)
{
    if (!c || !lam_next || !lam || !workspace || lam_next == lam) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const int sup = adjoint_supported(c);
    if (sup != LBM_OK) return sup;
    const AdjLayout L = adj_layout(c, 0, 1);
    const size_t N = (size_t)c->N, popb = (size_t)c->S * LBMK_Q * N * sizeof(double);
    const int R = c->mc.R;
    if (workspace_bytes < L.total + 256 || !is_device_ptr(workspace) || !is_device_ptr(lam_next) ||
        !is_device_ptr(lam))
        return LBM_ERR_ARG;
    if (ranges_overlap(lam_next, popb, lam, popb) || ranges_overlap(lam_next, popb, workspace, workspace_bytes) ||
        ranges_overlap(lam, popb, workspace, workspace_bytes))
        return LBM_ERR_ARG;
    double *w = ws_base(workspace);
    double *Trow = c->macro + (size_t)DR_T * N;
    const cudaStream_t s = c->stream;
    // The record pass overwrites the temperature row (the Newton starting
    // point of the next step); it is kept aside and put back.
    int st = copy_d2d(w + L.tkeep, Trow, N * sizeof(double), s);
    const int nb = adj_blocks(c->N);
    if (st == LBM_OK) st = check_cuda(cudaMemsetAsync(w + L.theta, 0, (size_t)nb * std::max(R, 1) * sizeof(double), s));
    if (st != LBM_OK) return st;
    if (lbmk::adj_upload(c->slot, c->mc, s)) return LBM_ERR_CUDA;
    const StepArgs a = args_of(c);
    AdjBufs g = adj_bufs(w, L);
    g.lam_next = lam_next;
    g.lam = lam;
    g.with_objective = with_objective ? 1 : 0;
    if (adj_record(a) || lbmk::adj_step_fp64(a, g)) return LBM_ERR_CUDA;
    if (lbmk::column_sums_fp64(w + L.theta, nb, R, w + L.theta_out, s)) return LBM_ERR_CUDA;
    double hA[LBMK_MAXR];
    if (dJ_dlogA && R > 0) st = check_cuda(cudaMemcpyAsync(hA, w + L.theta_out, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (st == LBM_OK) st = copy_d2d(Trow, w + L.tkeep, N * sizeof(double), s);
    if (st == LBM_OK) st = lbm_sync(c);
    if (st != LBM_OK) return st;
    if (dJ_dlogA)
        for (int k = 0; k < R; ++k) dJ_dlogA[k] = hA[k];
    return LBM_OK;
}

int lbm_heat_release_gradient(lbm_ctx *c, int nsteps, int every, double *J, double *dJ_dlogA, double *dJ_dT0,
                              void *workspace, size_t workspace_bytes)
{
    if (!c || !J || !workspace || nsteps < 1 || every < 1) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const int sup = adjoint_supported(c);
    if (sup != LBM_OK) return sup;
    const bool grads = dJ_dlogA || dJ_dT0;
    const AdjLayout L = adj_layout(c, nsteps, grads ? every : 0);
    if (workspace_bytes < L.total + 256 || !is_device_ptr(workspace)) return LBM_ERR_ARG;
    const bool T0_dev = dJ_dT0 && is_device_ptr(dJ_dT0);
    const size_t N = (size_t)c->N, pop = (size_t)c->S * LBMK_Q * N, popb = pop * sizeof(double);
    if (T0_dev && ranges_overlap(dJ_dT0, N * sizeof(double), workspace, workspace_bytes)) return LBM_ERR_ARG;
    const int R = c->mc.R, W = 1 + R;
    const lbmk::PrecisionOps &op = ops(c->lat.precision);
    const cudaStream_t s = c->stream;
    double *w = ws_base(workspace);
    double *Trow = c->macro + (size_t)DR_T * N;
    const size_t Tb = N * sizeof(double);
    int st = LBM_OK;

    // Forward sweep: J_t at every step, the state and temperature row every
    // checkpoint_every steps (no checkpoints and no reverse sweep when no
    // gradient is asked for).
    for (int t = 0; t < nsteps && st == LBM_OK; ++t) {
        if (grads && t % every == 0) {
            const int k = t / every;
            st = copy_d2d(w + L.ck + (size_t)k * pop, c->buf[c->cur], popb, s);
            if (st == LBM_OK) st = copy_d2d(w + L.ckT + (size_t)k * N, Trow, Tb, s);
            if (st != LBM_OK) break;
        }
        if (op.hrr(args_of(c), R, nullptr, nullptr, w + L.hrrpart, w + L.jpart + (size_t)t * W)) st = LBM_ERR_CUDA;
        if (st == LBM_OK && op.step(args_of(c), nullptr)) st = LBM_ERR_CUDA;
        c->cur = 1 - c->cur;
    }
    if (st == LBM_OK) st = copy_d2d(w + L.tkeep, Trow, Tb, s);
    if (st == LBM_OK) st = lbm_sync(c);                  // a failed forward sweep stops here
    if (st != LBM_OK) return st;
    if (!grads) {
        double *hJ = (double *)malloc((size_t)nsteps * W * sizeof(double));
        if (!hJ) return LBM_ERR_ARG;
        st = check_cuda(cudaMemcpy(hJ, w + L.jpart, (size_t)nsteps * W * sizeof(double), cudaMemcpyDeviceToHost));
        if (st == LBM_OK) {
            double acc = 0.0;
            for (int t = 0; t < nsteps; ++t) acc += hJ[(size_t)t * W];
            *J = acc;
        }
        free(hJ);
        return st;
    }

    // Reverse sweep, segment by segment from the last.
    if (lbmk::adj_upload(c->slot, c->mc, s)) return LBM_ERR_CUDA;
    double *lamA = w + L.lamA, *lamB = w + L.lamB;
    const int nb = adj_blocks(c->N);
    st = check_cuda(cudaMemsetAsync(lamA, 0, popb, s));
    if (st == LBM_OK) st = check_cuda(cudaMemsetAsync(w + L.theta, 0, (size_t)nb * std::max(R, 1) * sizeof(double), s));
    AdjBufs g = adj_bufs(w, L);
    for (int k = L.nck - 1; k >= 0 && st == LBM_OK; --k) {
        const int t0 = k * every, len = std::min(every, nsteps - t0);
        double *seg = w + L.seg, *segT = w + L.segT;
        st = copy_d2d(seg, w + L.ck + (size_t)k * pop, popb, s);
        if (st == LBM_OK) st = copy_d2d(segT, w + L.ckT + (size_t)k * N, Tb, s);
        for (int j = 0; j + 1 < len && st == LBM_OK; ++j) {      // the segment's states, recomputed
            st = copy_d2d(Trow, segT + (size_t)j * N, Tb, s);
            StepArgs a = args_of(c);
            a.src = seg + (size_t)j * pop;
            a.dst = seg + (size_t)(j + 1) * pop;
            if (st == LBM_OK && op.step(a, nullptr)) st = LBM_ERR_CUDA;
            if (st == LBM_OK) st = copy_d2d(segT + (size_t)(j + 1) * N, Trow, Tb, s);
        }
        for (int j = len - 1; j >= 0 && st == LBM_OK; --j) {       // last step first
            st = copy_d2d(Trow, segT + (size_t)j * N, Tb, s);
            StepArgs a = args_of(c);
            a.src = seg + (size_t)j * pop;
            g.lam_next = lamA;
            g.lam = lamB;
            if (st == LBM_OK && (adj_record(a) || lbmk::adj_step_fp64(a, g))) st = LBM_ERR_CUDA;
            std::swap(lamA, lamB);
        }
    }
    // lamA is now dJ/dF of the initial state: carry it to T(x, 0)
    double *dT0 = T0_dev ? dJ_dT0 : w + L.dT0;
    if (st == LBM_OK && dJ_dT0) {
        st = copy_d2d(Trow, w + L.ckT, Tb, s);
        StepArgs a = args_of(c);
        a.src = w + L.ck;
        if (st == LBM_OK && lbmk::adj_init_T_fp64(a, lamA, dT0)) st = LBM_ERR_CUDA;
        if (st == LBM_OK && !T0_dev)
            st = check_cuda(cudaMemcpyAsync(dJ_dT0, dT0, Tb, cudaMemcpyDeviceToHost, s));
    }
    if (st == LBM_OK && lbmk::column_sums_fp64(w + L.theta, nb, R, w + L.theta_out, s)) st = LBM_ERR_CUDA;
    double hA[LBMK_MAXR];
    double *hJ = (double *)malloc((size_t)nsteps * W * sizeof(double));
    if (!hJ) st = st == LBM_OK ? LBM_ERR_ARG : st;
    if (st == LBM_OK && R > 0)
        st = check_cuda(cudaMemcpyAsync(hA, w + L.theta_out, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (st == LBM_OK)
        st = check_cuda(cudaMemcpyAsync(hJ, w + L.jpart, (size_t)nsteps * W * sizeof(double),
                                        cudaMemcpyDeviceToHost, s));
    const int st_r = copy_d2d(Trow, w + L.tkeep, Tb, s);      // the temperature row after the forward sweep
    if (st == LBM_OK) st = st_r;
    if (st == LBM_OK) st = lbm_sync(c);
    if (st == LBM_OK) {
        double acc = 0.0;
        for (int t = 0; t < nsteps; ++t) acc += hJ[(size_t)t * W];
        *J = acc;
        if (dJ_dlogA)
            for (int k = 0; k < R; ++k) dJ_dlogA[k] = hA[k];
    }
    free(hJ);
    return st;
}

int lbm_flame_speeds(lbm_ctx *c, double *Sd, double *Sa)
{
    if (!c || !Sd || !Sa || Sd == Sa) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const size_t N = (size_t)c->N;
    const bool dev = is_device_ptr(Sd);
    if (dev != is_device_ptr(Sa)) return LBM_ERR_ARG;                // both host or both device
    // scratch in the free population buffer: the kept temperature row, the
    // gradients, then (host outputs) the two rows
    double *stage = (double *)c->buf[1 - c->cur];
    double *tkeep = stage, *scr = stage + N, *dSd = dev ? Sd : stage + 7 * N, *dSa = dev ? Sa : stage + 8 * N;
    if ((dev ? 7 : 9) * N * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
    double *Trow = c->macro + (size_t)DR_T * N;
    // the record pass overwrites the temperature row (the Newton starting
    // point of the next step): kept aside and put back
    int st = copy_d2d(tkeep, Trow, N * sizeof(double), c->stream);
    if (st != LBM_OK) return st;
    if (ops(c->lat.precision).flame(args_of(c), scr, dSd, dSa)) return LBM_ERR_CUDA;
    if (!dev) {
        st = check_cuda(cudaMemcpyAsync(Sd, dSd, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (st == LBM_OK) st = check_cuda(cudaMemcpyAsync(Sa, dSa, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (st != LBM_OK) return st;
    }
    st = copy_d2d(Trow, tkeep, N * sizeof(double), c->stream);
    if (st != LBM_OK) return st;
    return lbm_sync(c);
}

int lbm_isoline_means(lbm_ctx *c, const double *T, double T_iso, double cx, double cy, int K, const double *fields,
                      double *out)
{
    if (!c || !T || !out || K < 0 || K > 8 || (K > 0 && !fields) || !isfinite(T_iso)) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (!is_device_ptr(T) || (K > 0 && !is_device_ptr(fields))) return LBM_ERR_ARG;
    const int nb = lbmk::isoline_blocks((long long)c->lat.nx * c->lat.ny);
    double *partial = (double *)c->buf[1 - c->cur], *dout = partial + (size_t)nb * (2 + K);
    if (((size_t)nb * (2 + K) + 2 + K) * sizeof(double) > c->pop_bytes) return LBM_ERR_ARG;
    if (lbmk::isoline_fp64(c->lat.nx, c->lat.ny, c->N, T, T_iso, cx, cy, K, fields, partial, dout, c->stream))
        return LBM_ERR_CUDA;
    double h[2 + 8];
    int st = check_cuda(cudaMemcpyAsync(h, dout, (2 + K) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (st == LBM_OK) st = lbm_sync(c);
    if (st != LBM_OK) return st;
    out[0] = h[0];
    for (int k = 1; k < 2 + K; ++k) out[k] = h[0] > 0.0 ? h[k] / h[0] : 0.0;
    return LBM_OK;
}

int lbm_chemistry_at(lbm_ctx *c, int n, const double *rho_a, const double *T, double *rho_dot, double *hdot,
                     double *dhdot_dT, double *dhdot_drho, double *dhdot_dlogA)
{
    if (!c || n < 0 || (n > 0 && (!rho_a || !T))) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (n == 0) return LBM_OK;
    const double *ptrs[7] = {rho_a, T, rho_dot, hdot, dhdot_dT, dhdot_drho, dhdot_dlogA};
    for (const double *q : ptrs)
        if (q && !is_device_ptr(q)) return LBM_ERR_ARG;
    if (ops(c->lat.precision).chem_at(args_of(c), n, rho_a, T, rho_dot, hdot, dhdot_dT, dhdot_drho, dhdot_dlogA))
        return LBM_ERR_CUDA;
    return lbm_sync(c);
}

int lbm_temperature_at(lbm_ctx *c, int n, const double *Y, const double *e, const double *T_guess, double *T)
{
    if (!c || n < 0 || (n > 0 && (!Y || !e || !T_guess || !T))) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    if (n == 0) return LBM_OK;
    if (!is_device_ptr(Y) || !is_device_ptr(e) || !is_device_ptr(T_guess) || !is_device_ptr(T)) return LBM_ERR_ARG;
    if (ops(c->lat.precision).temperature_at(args_of(c), n, Y, e, T_guess, T)) return LBM_ERR_CUDA;
    return lbm_sync(c);
}

int lbm_get_populations(lbm_ctx *c, double *host_out)
{
    if (!c || !host_out) return LBM_ERR_ARG;
    const int od = on_ctx_device(c);
    if (od != LBM_OK) return od;
    const size_t cnt = (size_t)c->S * LBMK_Q * c->N;
    int st = check_cuda(cudaStreamSynchronize(c->stream));
    if (st != LBM_OK) return st;
    if (c->lat.precision == LBM_FP64)
        return check_cuda(cudaMemcpy(host_out, c->buf[c->cur], cnt * sizeof(double), cudaMemcpyDeviceToHost));
    const size_t M = (size_t)c->M, N = (size_t)c->N;
    float *mov = (float *)malloc(M * LBMK_Q * N * sizeof(float));
    double *dbl = (double *)malloc((M + LBMK_Q) * N * sizeof(double));   // rest [M][N], then g [27][N]
    if (!mov || !dbl) { free(mov); free(dbl); return LBM_ERR_ARG; }
    st = check_cuda(cudaMemcpy(mov, c->buf[c->cur], M * LBMK_Q * N * sizeof(float), cudaMemcpyDeviceToHost));
    if (st == LBM_OK)
        st = check_cuda(cudaMemcpy(dbl, (const char *)c->buf[c->cur] + pop_float_bytes(c->M, N),
                                   (M + LBMK_Q) * N * sizeof(double), cudaMemcpyDeviceToHost));
    if (st == LBM_OK)
        for (size_t s = 0; s <= M; ++s)
            for (int i = 0; i < LBMK_Q; ++i) {
                double *o = host_out + (s * LBMK_Q + i) * N;
                for (size_t n = 0; n < N; ++n) {
                    if (s == M) o[n] = dbl[M * N + (size_t)i * N + n];
                    else if (i == 13) o[n] = dbl[s * N + n];
                    else o[n] = (double)mov[(s * LBMK_Q + i) * N + n] + (double)c->mc.ref[s][i];
                }
            }
    free(mov);
    free(dbl);
    return st;
}

void *lbm_state_buffer(lbm_ctx *c) { return c ? c->buf[c->cur] : nullptr; }

int lbm_get_references(const lbm_ctx *c, float *ref)
{
    if (!c || !ref) return LBM_ERR_ARG;
    if (!is_mixed(c->lat.precision)) return LBM_ERR_UNSUPPORTED;
    for (int s = 0; s < c->M; ++s)
        for (int i = 0; i < LBMK_Q; ++i) ref[s * LBMK_Q + i] = c->mc.ref[s][i];
    return LBM_OK;
}

int lbm_set_references(lbm_ctx *c, const float *ref)
{
    if (!c || !ref) return LBM_ERR_ARG;
    if (!is_mixed(c->lat.precision)) return LBM_ERR_UNSUPPORTED;
    for (int s = 0; s < c->M; ++s)
        for (int i = 0; i < LBMK_Q; ++i) {
            if (!isfinite(ref[s * LBMK_Q + i])) return LBM_ERR_ARG;
            c->mc.ref[s][i] = i == 13 ? 0.0f : ref[s * LBMK_Q + i];   // rest populations are stored in double
        }
    lbmk_reference_moments(c->mc, c->M);
    c->refs_fixed = true;
    return reslot(c);
}

int lbm_destroy(lbm_ctx *c)
{
    if (!c) return LBM_ERR_ARG;
    if (c->status || c->xseg || c->segs || c->graph) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->status) cudaFree(c->status);
    if (c->xseg) cudaFree(c->xseg);
    if (c->segs) cudaFree(c->segs);
    release_slot(c->dev, c->lat.precision, c->slot);
    free(c);
    return LBM_OK;
}

const char *lbm_strerror(int s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_NEWTON: return "temperature iteration did not converge";
    case LBM_ERR_NONFINITE: return "non-finite density, energy or population";
    case LBM_ERR_NEGATIVE: return "negative species density";
    case LBM_ERR_PIVOT: return "non-finite pivot in the Stefan-Maxwell solve";
    case LBM_ERR_BOUNDS: return "index out of bounds (checked build)";
    case LBM_ERR_UNSUPPORTED: return "unsupported configuration";
    case LBM_ERR_BARRIER: return "a grid barrier of the persistent step gave up waiting";
    default: return "unknown status";
    }
}

}  // extern "C"
