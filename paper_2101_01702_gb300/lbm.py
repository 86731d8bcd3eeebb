"""Thin ctypes binding of liblbm.so (include/lbm.h).

The functions below carry the C names and only marshal arguments; every
step of the lattice Boltzmann method runs in the library's CUDA kernels.
PyTorch provides the device buffers and the stream.  Importing this module
fails with ImportError when the compiled library is absent: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

import os

# LBM_LIBRARY may name another build of the same library (same ABI).
_LIB_PATH = Path(os.environ.get("LBM_LIBRARY", Path(__file__).resolve().parent / "_build" / "liblbm.so"))
if not _LIB_PATH.exists():
    raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2101_01702_gb300.build.build()")
_lib = C.CDLL(str(_LIB_PATH))

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_NEWTON = -3
LBM_ERR_NONFINITE = -4
LBM_ERR_NEGATIVE = -5
LBM_ERR_BOUNDS = -7
LBM_ERR_PIVOT = -6
LBM_ERR_UNSUPPORTED = -8
LBM_ERR_BARRIER = -9
LBM_BC_PERIODIC = 0
LBM_BC_EQ_ZEROGRAD_U0LEFT = 1
LBM_FP64 = 0
LBM_MIXED = 1
LBM_MIXED_FAST = 2
LBM_F_RHO_A, LBM_F_RHOU, LBM_F_RHOE, LBM_F_T, LBM_F_P, LBM_F_Y, LBM_F_J_A = 1, 2, 4, 8, 16, 32, 64
LBM_F_RHO_DOT = 128
LBM_F_HRR = 256
LBM_PHASES = 6
LBM_TRANSPORT_CONSTANT, LBM_TRANSPORT_MIXTURE_AVERAGED = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class lbm_lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc_x", C.c_int), ("precision", C.c_int),
                ("nseg", C.c_int), ("seg_nx", C.POINTER(C.c_int))]


class lbm_species(C.Structure):
    _fields_ = [("M", C.c_int), ("W", _dp), ("thermo", C.c_int), ("cp_R", _dp), ("h_form", _dp),
                ("T0", C.c_double), ("poly7", _dp), ("D", _dp), ("nu", C.c_double), ("Pr", C.c_double),
                ("r_lat", C.c_double), ("visc_model", C.c_int), ("transport", C.c_int), ("mu0", _dp),
                ("mu_exp", _dp), ("T_tr", C.c_double), ("D_exp", C.c_double), ("P_tr", C.c_double)]


class lbm_mechanism(C.Structure):
    _fields_ = [("R", C.c_int), ("nu_f", _ip), ("nu_r", _ip), ("log_A", _dp), ("b", _dp), ("theta", _dp),
                ("rtype", _ip), ("eff", _dp), ("low", _dp), ("reversible", _ip), ("T_ref", C.c_double),
                ("P0", C.c_double)]


class lbm_buffers(C.Structure):
    _fields_ = [("pop_a", C.c_void_p), ("pop_b", C.c_void_p), ("macro", C.c_void_p), ("ghost", C.c_void_p),
                ("pop_bytes", C.c_size_t), ("macro_bytes", C.c_size_t), ("ghost_bytes", C.c_size_t)]


_sz = C.c_size_t
_lib.lbm_buffer_sizes.argtypes = [C.POINTER(lbm_lattice), C.POINTER(lbm_species), C.POINTER(_sz),
                                  C.POINTER(_sz), C.POINTER(_sz)]
_lib.lbm_create.argtypes = [C.POINTER(lbm_lattice), C.POINTER(lbm_species), C.POINTER(lbm_mechanism),
                            C.POINTER(lbm_buffers), C.c_void_p, C.POINTER(C.c_void_p)]
_lib.lbm_init.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]
_lib.lbm_step.argtypes = [C.c_void_p, C.c_int]
_lib.lbm_step_async.argtypes = [C.c_void_p, C.c_int]
_lib.lbm_step_graph.argtypes = [C.c_void_p, C.c_int]
_lib.lbm_autotune.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
_lib.lbm_set_blocks.argtypes = [C.c_void_p, C.c_void_p]
_lib.lbm_get_references.argtypes = [C.c_void_p, C.c_void_p]
_lib.lbm_set_references.argtypes = [C.c_void_p, C.c_void_p]
_lib.lbm_sync.argtypes = [C.c_void_p]
_lib.lbm_step_timed.argtypes = [C.c_void_p, C.c_int, _dp]
_lib.lbm_moments.argtypes = [C.c_void_p, C.c_uint, C.c_void_p]
_lib.lbm_moments_count.argtypes = [C.c_void_p, C.c_uint]
_lib.lbm_moments_count.restype = C.c_size_t
_lib.lbm_get_populations.argtypes = [C.c_void_p, _dp]
_lib.lbm_heat_release.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p, C.c_void_p]
_lib.lbm_heat_release_adjoint.argtypes = [C.c_void_p, C.c_void_p]
_lib.lbm_chemistry_at.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 7
_lib.lbm_temperature_at.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 4
_lib.lbm_state_buffer.argtypes = [C.c_void_p]
_lib.lbm_state_buffer.restype = C.c_void_p
_lib.lbm_destroy.argtypes = [C.c_void_p]
_lib.lbm_step_fixed_scratch.argtypes = [C.POINTER(lbm_lattice), C.POINTER(lbm_species), C.POINTER(lbm_mechanism),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
_lib.lbm_strerror.argtypes = [C.c_int]
_lib.lbm_strerror.restype = C.c_char_p

EXPORTED = ["lbm_buffer_sizes", "lbm_create", "lbm_init", "lbm_step", "lbm_step_async", "lbm_step_graph",
            "lbm_step_timed", "lbm_sync",
            "lbm_moments", "lbm_moments_count", "lbm_get_populations", "lbm_state_buffer", "lbm_destroy",
            "lbm_strerror", "lbm_step_fixed_scratch", "lbm_exp_check", "lbm_convert_check", "lbm_get_references",
            "lbm_set_references", "lbm_autotune", "lbm_set_blocks", "lbm_heat_release",
            "lbm_chemistry_at", "lbm_temperature_at", "lbm_heat_release_adjoint", "lbm_fp64_probe",
            "lbm_adjoint_workspace_bytes", "lbm_adjoint_step", "lbm_heat_release_gradient",
            "lbm_flame_speeds", "lbm_isoline_means", "lbm_step_persistent", "lbm_autotune_persistent"]


def library_path() -> str:
    return str(_LIB_PATH)


class LBMError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {lbm_strerror(status)} ({status})" if what else lbm_strerror(status))


def _check(st: int, what: str) -> int:
    if st != LBM_OK:
        raise LBMError(st, what)
    return st


# ---------------------------------------------------------------------------
# C-named wrappers (argument marshalling only)
# ---------------------------------------------------------------------------
def lbm_buffer_sizes(lat: lbm_lattice, sp: lbm_species):
    a, b, c = _sz(), _sz(), _sz()
    _check(_lib.lbm_buffer_sizes(C.byref(lat), C.byref(sp), C.byref(a), C.byref(b), C.byref(c)), "lbm_buffer_sizes")
    return a.value, b.value, c.value


def lbm_create(lat, sp, mech, bufs, stream: int):
    h = C.c_void_p()
    st = _lib.lbm_create(C.byref(lat), C.byref(sp), C.byref(mech), C.byref(bufs), C.c_void_p(stream), C.byref(h))
    _check(st, "lbm_create")
    return h


def lbm_init(ctx, X_ptr: int, T_ptr: int, u_ptr, P: float) -> int:
    return _lib.lbm_init(ctx, C.c_void_p(X_ptr), C.c_void_p(T_ptr), C.c_void_p(u_ptr) if u_ptr else None,
                         float(P))


def lbm_step(ctx, n: int) -> int:
    return _lib.lbm_step(ctx, int(n))


def lbm_step_async(ctx, n: int) -> int:
    return _lib.lbm_step_async(ctx, int(n))


def lbm_step_graph(ctx, n: int) -> int:
    return _lib.lbm_step_graph(ctx, int(n))


def lbm_autotune(ctx, trials: int, block_out: np.ndarray = None) -> int:
    if block_out is not None:
        assert block_out.dtype == np.int32 and block_out.size >= 6
    return _lib.lbm_autotune(ctx, int(trials), block_out.ctypes.data if block_out is not None else None)


def lbm_set_blocks(ctx, blocks) -> int:
    b = np.ascontiguousarray(blocks, dtype=np.int32)
    assert b.size == 6
    return _lib.lbm_set_blocks(ctx, b.ctypes.data)


def lbm_get_references(ctx, ref: np.ndarray) -> int:
    assert ref.dtype == np.float32 and ref.flags.c_contiguous
    return _lib.lbm_get_references(ctx, ref.ctypes.data)


def lbm_set_references(ctx, ref: np.ndarray) -> int:
    ref = np.ascontiguousarray(ref, dtype=np.float32)
    return _lib.lbm_set_references(ctx, ref.ctypes.data)


def lbm_step_timed(ctx, n: int, phase_ms: np.ndarray) -> int:
    assert phase_ms.dtype == np.float64 and phase_ms.size >= LBM_PHASES + 1
    return _lib.lbm_step_timed(ctx, int(n), phase_ms.ctypes.data_as(_dp))


def lbm_sync(ctx) -> int:
    return _lib.lbm_sync(ctx)


def lbm_moments(ctx, mask: int, out_ptr: int) -> int:
    return _lib.lbm_moments(ctx, C.c_uint(mask), C.c_void_p(out_ptr))


def lbm_moments_count(ctx, mask: int) -> int:
    return _lib.lbm_moments_count(ctx, C.c_uint(mask))


def lbm_heat_release(ctx, J: np.ndarray, dlogA, dT_ptr, drho_ptr) -> int:
    """J: float64 [1] host; dlogA: float64 [R] host or None; dT_ptr,
    drho_ptr: host or device addresses, or None."""
    assert J.dtype == np.float64 and J.size >= 1
    if dlogA is not None:
        assert dlogA.dtype == np.float64 and dlogA.flags.c_contiguous
    return _lib.lbm_heat_release(ctx, J.ctypes.data_as(_dp), dlogA.ctypes.data_as(_dp) if dlogA is not None else None,
                                 C.c_void_p(dT_ptr) if dT_ptr else None, C.c_void_p(drho_ptr) if drho_ptr else None)


def lbm_heat_release_adjoint(ctx, out_ptr: int) -> int:
    """out_ptr: host or device address of double [M+1][27][N]."""
    return _lib.lbm_heat_release_adjoint(ctx, C.c_void_p(out_ptr) if out_ptr else None)


def lbm_chemistry_at(ctx, n: int, rho_a_ptr: int, T_ptr: int, rho_dot_ptr=None, hdot_ptr=None, dT_ptr=None,
                     drho_ptr=None, dlogA_ptr=None) -> int:
    """Device addresses; outputs may be None."""
    v = [C.c_void_p(p) if p else None for p in (rho_a_ptr, T_ptr, rho_dot_ptr, hdot_ptr, dT_ptr, drho_ptr, dlogA_ptr)]
    return _lib.lbm_chemistry_at(ctx, int(n), *v)


def lbm_temperature_at(ctx, n: int, Y_ptr: int, e_ptr: int, T0_ptr: int, T_ptr: int) -> int:
    return _lib.lbm_temperature_at(ctx, int(n), *[C.c_void_p(p) if p else None for p in (Y_ptr, e_ptr, T0_ptr, T_ptr)])


def lbm_get_populations(ctx, out: np.ndarray) -> int:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    return _lib.lbm_get_populations(ctx, out.ctypes.data_as(_dp))


def lbm_state_buffer(ctx) -> int:
    return _lib.lbm_state_buffer(ctx)


def lbm_destroy(ctx) -> int:
    return _lib.lbm_destroy(ctx)


_lib.lbm_exp_check.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
_lib.lbm_exp_check.restype = C.c_int


_lib.lbm_convert_check.argtypes = [C.c_void_p] * 6 + [C.c_int, C.c_void_p]
_lib.lbm_convert_check.restype = C.c_int


def lbm_convert_check(f_ptr: int, fd_ptr: int, fd_ref_ptr: int, d_ptr: int, df_ptr: int, df_ref_ptr: int, n: int,
                      stream: int) -> int:
    return _lib.lbm_convert_check(*(C.c_void_p(p) for p in (f_ptr, fd_ptr, fd_ref_ptr, d_ptr, df_ptr, df_ref_ptr)),
                                  int(n), C.c_void_p(stream))


def lbm_exp_check(x_ptr: int, y_ptr: int, y_ref_ptr: int, n: int, stream: int) -> int:
    """The kernels' exponential into y and CUDA's exp into y_ref (device)."""
    return _lib.lbm_exp_check(C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.c_void_p(y_ref_ptr), int(n),
                              C.c_void_p(stream))


_lib.lbm_adjoint_workspace_bytes.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
_lib.lbm_adjoint_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, _dp, C.c_int, C.c_void_p, C.c_size_t]
_lib.lbm_heat_release_gradient.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp, C.c_void_p, C.c_void_p,
                                           C.c_size_t]


def lbm_adjoint_workspace_bytes(ctx, nsteps: int, checkpoint_every: int) -> int:
    out = C.c_size_t(0)
    _check(_lib.lbm_adjoint_workspace_bytes(ctx, int(nsteps), int(checkpoint_every), C.byref(out)),
           "lbm_adjoint_workspace_bytes")
    return int(out.value)


def lbm_adjoint_step(ctx, lam_next_ptr: int, lam_ptr: int, dlogA, with_objective: bool, ws_ptr: int,
                     ws_bytes: int) -> int:
    """One reverse step at the current state (see include/lbm.h); dlogA: numpy [R] or None."""
    return _lib.lbm_adjoint_step(ctx, C.c_void_p(lam_next_ptr), C.c_void_p(lam_ptr),
                                 dlogA.ctypes.data_as(_dp) if dlogA is not None else None,
                                 1 if with_objective else 0, C.c_void_p(ws_ptr), int(ws_bytes))


def lbm_heat_release_gradient(ctx, nsteps: int, checkpoint_every: int, J: np.ndarray, dlogA, dT0_ptr,
                              ws_ptr: int, ws_bytes: int) -> int:
    """Time-integrated heat release and its gradients (see include/lbm.h)."""
    return _lib.lbm_heat_release_gradient(ctx, int(nsteps), int(checkpoint_every), J.ctypes.data_as(_dp),
                                          dlogA.ctypes.data_as(_dp) if dlogA is not None else None,
                                          C.c_void_p(dT0_ptr) if dT0_ptr else None, C.c_void_p(ws_ptr),
                                          int(ws_bytes))


_lib.lbm_step_persistent.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint]
_lib.lbm_autotune_persistent.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]


def lbm_step_persistent(ctx, n: int, tile_mult: int = 1, spin_cap: int = 0) -> int:
    return _lib.lbm_step_persistent(ctx, int(n), int(tile_mult), C.c_uint(spin_cap))


def lbm_autotune_persistent(ctx, steps: int):
    out = C.c_int(0)
    st = _lib.lbm_autotune_persistent(ctx, int(steps), C.byref(out))
    return st, int(out.value)


_lib.lbm_flame_speeds.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
_lib.lbm_isoline_means.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                   _dp]


def lbm_flame_speeds(ctx, Sd_ptr: int, Sa_ptr: int) -> int:
    return _lib.lbm_flame_speeds(ctx, C.c_void_p(Sd_ptr), C.c_void_p(Sa_ptr))


def lbm_isoline_means(ctx, T_ptr: int, T_iso: float, cx: float, cy: float, K: int, fields_ptr, out: np.ndarray) -> int:
    return _lib.lbm_isoline_means(ctx, C.c_void_p(T_ptr), float(T_iso), float(cx), float(cy), int(K),
                                  C.c_void_p(fields_ptr) if fields_ptr else None, out.ctypes.data_as(_dp))


_lib.lbm_fp64_probe.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, _dp, C.c_void_p]
_lib.lbm_fp64_probe.restype = C.c_int
LBM_PROBE_DFMA, LBM_PROBE_EXP, LBM_PROBE_LOG = 0, 1, 2


def lbm_fp64_probe(kind: int, blocks: int, iters: int, sink_ptr: int, stream: int):
    """(status, milliseconds, rate) of one probe launch (see include/lbm.h)."""
    out = np.zeros(2)
    st = _lib.lbm_fp64_probe(int(kind), int(blocks), int(iters), C.c_void_p(sink_ptr),
                             out.ctypes.data_as(_dp), C.c_void_p(stream))
    return st, float(out[0]), float(out[1])


def lbm_step_fixed_scratch(lat, sp, mech, pop_in_ptr: int, pop_out_ptr: int, T_io_ptr: int, stream: int) -> int:
    """One double-precision step with the library's fixed device scratch
    array (no allocation); see include/lbm.h for the limits."""
    return _lib.lbm_step_fixed_scratch(C.byref(lat), C.byref(sp), C.byref(mech), C.c_void_p(pop_in_ptr),
                                       C.c_void_p(pop_out_ptr), C.c_void_p(T_io_ptr), C.c_void_p(stream))


def lbm_strerror(st: int) -> str:
    return _lib.lbm_strerror(int(st)).decode()


# ---------------------------------------------------------------------------
# Convenience: a problem description plus torch-owned device buffers
# ---------------------------------------------------------------------------
def _on_device(method):
    """Runs a Solver method with the solver's device current: the library
    binds a context to the device current at lbm_create and rejects calls
    made from another."""

    def wrapped(self, *args, **kw):
        with self.torch.cuda.device(self.device):
            return method(self, *args, **kw)

    wrapped.__name__ = method.__name__
    wrapped.__doc__ = method.__doc__
    return wrapped


class Solver:
    """Owns torch buffers for one lattice and drives the C ABI.

    lattice/species/mech follow workload.problem (numpy arrays).  The
    tables are passed to lbm_create, which copies them.  Every call runs
    with the solver's device current, whichever device the caller has.
    """

    def __init__(self, lattice, species, mech, precision: int = LBM_FP64, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.M = species.M
        self.R = mech.R
        self.S = self.M + 1
        self.N = lattice.nx * lattice.ny * lattice.nz
        self.precision = precision
        self._keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(_dp)

        def i(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(_ip)

        seg = getattr(lattice, "seg_nx", None)
        if seg is not None and len(seg) > 1:
            self.lat = lbm_lattice(lattice.nx, lattice.ny, lattice.nz, lattice.bc_x, precision, len(seg), i(seg))
        else:
            self.lat = lbm_lattice(lattice.nx, lattice.ny, lattice.nz, lattice.bc_x, precision, 0, None)
        tr = getattr(species, "transport", 0)
        self.sp = lbm_species(self.M, d(species.W), species.thermo, d(species.cp_R), d(species.h_form),
                              species.T0, d(species.poly7), d(species.D), species.nu, species.Pr,
                              species.r_lat, species.visc_model, tr,
                              d(species.mu0) if tr else None, d(species.mu_exp) if tr else None,
                              getattr(species, "T_tr", 1.0), getattr(species, "D_exp", 1.5),
                              getattr(species, "P_tr", 1.0))
        R = mech.R
        self.mech = lbm_mechanism(R, i(mech.nu_f.reshape(R, -1)) if R else None,
                                  i(mech.nu_r.reshape(R, -1)) if R else None,
                                  d(mech.log_A) if R else None, d(mech.b) if R else None,
                                  d(mech.theta) if R else None, i(mech.rtype) if R else None,
                                  d(mech.eff) if R else None, d(mech.low) if R else None,
                                  i(mech.reversible) if R else None, mech.T_ref, mech.P0)
        pop_b, mac_b, gh_b = lbm_buffer_sizes(self.lat, self.sp)
        with torch.cuda.device(self.device):
            self.pop = [torch.empty(pop_b, dtype=torch.uint8, device=self.device) for _ in range(2)]
            self.macro = torch.zeros(mac_b // 8, dtype=torch.float64, device=self.device)
            self.ghost = torch.empty(max(gh_b, 16), dtype=torch.uint8, device=self.device)
        self.bufs = lbm_buffers(self.pop[0].data_ptr(), self.pop[1].data_ptr(), self.macro.data_ptr(),
                                self.ghost.data_ptr() if gh_b else None, pop_b, mac_b, gh_b)
        with torch.cuda.device(self.device):
            self.ctx = lbm_create(self.lat, self.sp, self.mech, self.bufs, self.stream.cuda_stream)

    @classmethod
    def from_problem(cls, prob, precision: int = LBM_FP64, init: bool = True, **kw):
        s = cls(prob.lattice, prob.species, prob.mech, precision, **kw)
        if init:
            s.init(prob.init.X, prob.init.T, prob.init.u, prob.init.P)
        return s

    @_on_device
    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @_on_device
    def init(self, X, T, u, P):
        """X[M,N], T[N], u[3,N] or None: numpy (host) or torch (device) arrays."""
        torch = self.torch
        if isinstance(X, torch.Tensor):
            Xt = X.contiguous().to(torch.float64)
            Tt = T.contiguous().to(torch.float64)
            ut = None if u is None else u.contiguous().to(torch.float64)
            keep = (Xt, Tt, ut)
            st = lbm_init(self.ctx, Xt.data_ptr(), Tt.data_ptr(), ut.data_ptr() if ut is not None else None, P)
            del keep
        else:
            Xh = np.ascontiguousarray(X, dtype=np.float64)
            Th = np.ascontiguousarray(T, dtype=np.float64)
            uh = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
            st = lbm_init(self.ctx, Xh.ctypes.data, Th.ctypes.data, uh.ctypes.data if uh is not None else None, P)
        _check(st, "lbm_init")

    @_on_device
    def step(self, n: int = 1, check: bool = True) -> int:
        st = lbm_step(self.ctx, n)
        if check:
            _check(st, "lbm_step")
        return st

    @_on_device
    def step_async(self, n: int = 1):
        _check(lbm_step_async(self.ctx, n), "lbm_step_async")

    @_on_device
    def autotune(self, trials: int = 3) -> dict:
        """Picks each kernel's block size by timing it on the current state
        (results unchanged); returns the choice per kernel."""
        bs = np.zeros(6, dtype=np.int32)
        _check(lbm_autotune(self.ctx, trials, bs), "lbm_autotune")
        return dict(zip(("ghost", "moments", "rates", "gradients", "energy_collision", "species_collision"),
                        bs.tolist()))

    @_on_device
    def set_blocks(self, blocks):
        """Block sizes of the six kernels in launch order (see autotune)."""
        _check(lbm_set_blocks(self.ctx, blocks), "lbm_set_blocks")

    def references(self) -> np.ndarray:
        """Rest references of the mixed modes, float32 [M, 27]."""
        ref = np.zeros((self.M, 27), dtype=np.float32)
        _check(lbm_get_references(self.ctx, ref), "lbm_get_references")
        return ref

    @_on_device
    def set_references(self, ref):
        _check(lbm_set_references(self.ctx, ref), "lbm_set_references")

    @_on_device
    def step_graph(self, n: int = 1):
        """n steps through the captured two-step CUDA graph (no wait)."""
        _check(lbm_step_graph(self.ctx, n), "lbm_step_graph")

    @_on_device
    def step_persistent(self, n: int = 1, tile_mult: int = 1, spin_cap: int = 0, check: bool = True) -> int:
        """n steps in one persistent cooperative launch (see lbm_step_persistent)."""
        st = lbm_step_persistent(self.ctx, n, tile_mult, spin_cap)
        if check:
            _check(st, "lbm_step_persistent")
        return st

    @_on_device
    def autotune_persistent(self, steps: int = 4) -> int:
        """The fastest tile_mult of lbm_step_persistent on the current state (unchanged)."""
        st, t = lbm_autotune_persistent(self.ctx, steps)
        _check(st, "lbm_autotune_persistent")
        return t

    @_on_device
    def step_timed(self, n: int = 1):
        """Runs n steps; returns per-phase device milliseconds summed over
        them (ghost, moments, production rates, gradients, energy collision,
        species/mixture collision) and, last, the device milliseconds of the
        whole run."""
        ph = np.zeros(LBM_PHASES + 1)
        _check(lbm_step_timed(self.ctx, n, ph), "lbm_step_timed")
        return ph

    @_on_device
    def sync(self) -> int:
        return lbm_sync(self.ctx)

    @_on_device
    def moments(self, mask: int = LBM_F_RHO_A | LBM_F_RHOU | LBM_F_RHOE | LBM_F_T, device: bool = False):
        """Dictionary of fields (numpy on host, or torch on the device)."""
        torch = self.torch
        count = lbm_moments_count(self.ctx, mask)
        if device:
            out = torch.empty(count, dtype=torch.float64, device=self.device)
            _check(lbm_moments(self.ctx, mask, out.data_ptr()), "lbm_moments")
        else:
            out = np.empty(count, dtype=np.float64)
            _check(lbm_moments(self.ctx, mask, out.ctypes.data), "lbm_moments")
        res, row, N, M = {}, 0, self.N, self.M
        for bit, name, rows in ((LBM_F_RHO_A, "rho_a", M), (LBM_F_RHOU, "rhou", 3), (LBM_F_RHOE, "rhoE", 1),
                                (LBM_F_T, "T", 1), (LBM_F_P, "P", 1), (LBM_F_Y, "Y", M), (LBM_F_J_A, "j_a", 3 * M),
                                (LBM_F_RHO_DOT, "rho_dot", M), (LBM_F_HRR, "hrr", 1)):
            if mask & bit:
                blk = out[row * N:(row + rows) * N]
                res[name] = blk.reshape(rows, N) if rows > 1 else blk.reshape(N)
                row += rows
        if "j_a" in res:
            res["j_a"] = res["j_a"].reshape(M, 3, N)
        return res

    @_on_device
    def heat_release(self, gradients: bool = True, device: bool = False):
        """J = sum over nodes of the heat release rate at the current state,
        and (gradients) dJ/d ln A_k [R], d hdot^c/dT [N], d hdot^c/d rho_a
        [M, N] there (see lbm_heat_release); the per-node fields as numpy
        arrays, or torch tensors on the device with device=True."""
        J = np.zeros(1)
        if not gradients:
            _check(lbm_heat_release(self.ctx, J, None, None, None), "lbm_heat_release")
            return float(J[0])
        R = self.R
        dA = np.zeros(R)
        if device:
            torch = self.torch
            dT = torch.empty(self.N, dtype=torch.float64, device=self.device)
            dr = torch.empty((self.M, self.N), dtype=torch.float64, device=self.device)
            _check(lbm_heat_release(self.ctx, J, dA, dT.data_ptr(), dr.data_ptr()), "lbm_heat_release")
        else:
            dT = np.empty(self.N)
            dr = np.empty((self.M, self.N))
            _check(lbm_heat_release(self.ctx, J, dA, dT.ctypes.data, dr.ctypes.data), "lbm_heat_release")
        return float(J[0]), dA, dT, dr

    @_on_device
    def heat_release_adjoint(self, device: bool = False):
        """dJ/dF [M+1, 27, N] of J = sum of hdot^c at the current state (see
        lbm_heat_release_adjoint); numpy, or a torch tensor on the device."""
        if device:
            out = self.torch.empty((self.S, 27, self.N), dtype=self.torch.float64, device=self.device)
            _check(lbm_heat_release_adjoint(self.ctx, out.data_ptr()), "lbm_heat_release_adjoint")
        else:
            out = np.empty((self.S, 27, self.N))
            _check(lbm_heat_release_adjoint(self.ctx, out.ctypes.data), "lbm_heat_release_adjoint")
        return out

    def _workspace(self, nsteps: int, every: int):
        """A device workspace for the adjoint calls (see lbm_adjoint_workspace_bytes)."""
        nb = lbm_adjoint_workspace_bytes(self.ctx, nsteps, every)
        return self.torch.empty(nb, dtype=self.torch.uint8, device=self.device), nb

    @_on_device
    def adjoint_step(self, lam_next, with_objective: bool = True):
        """One reverse step at the current state: lam_next, a float64 device
        tensor [M+1, 27, N] (the adjoint of the state the next step would
        produce), gives (lam [M+1, 27, N] on the device, d/d ln A_k [R] numpy)
        -- see lbm_adjoint_step.  The state is not changed."""
        torch = self.torch
        lam_next = lam_next.contiguous().to(device=self.device, dtype=torch.float64)
        lam = torch.empty_like(lam_next)
        ws, nb = self._workspace(0, 1)
        dA = np.zeros(max(self.R, 1))
        _check(lbm_adjoint_step(self.ctx, lam_next.data_ptr(), lam.data_ptr(), dA, with_objective, ws.data_ptr(), nb),
               "lbm_adjoint_step")
        return lam, dA[:self.R]

    @_on_device
    def heat_release_total(self, steps: int):
        """J alone: the forward sweep of lbm_heat_release_gradient."""
        ws, nb = self._workspace(steps, 0)
        J = np.zeros(1)
        _check(lbm_heat_release_gradient(self.ctx, steps, steps, J, None, None, ws.data_ptr(), nb),
               "lbm_heat_release_gradient")
        return float(J[0])

    @_on_device
    def heat_release_gradient(self, steps: int, checkpoint_every: int = 64):
        """J = sum over steps and nodes of hdot^c from the current (freshly
        initialised) state, with dJ/d ln A_k [R] (numpy) and dJ/dT(x, 0) [N]
        (float64 device tensor); see lbm_heat_release_gradient.  Also returns
        the workspace size in bytes."""
        torch = self.torch
        ws, nb = self._workspace(steps, checkpoint_every)
        J = np.zeros(1)
        dA = np.zeros(max(self.R, 1))
        dT0 = torch.empty(self.N, dtype=torch.float64, device=self.device)
        _check(lbm_heat_release_gradient(self.ctx, steps, checkpoint_every, J, dA, dT0.data_ptr(), ws.data_ptr(), nb),
               "lbm_heat_release_gradient")
        del ws
        return float(J[0]), dA[:self.R], dT0, nb

    @_on_device
    def flame_speeds(self, device: bool = False):
        """(S_d, S_a) [N] of the current state (see lbm_flame_speeds)."""
        if device:
            Sd = self.torch.empty(self.N, dtype=self.torch.float64, device=self.device)
            Sa = self.torch.empty_like(Sd)
            _check(lbm_flame_speeds(self.ctx, Sd.data_ptr(), Sa.data_ptr()), "lbm_flame_speeds")
        else:
            Sd, Sa = np.empty(self.N), np.empty(self.N)
            _check(lbm_flame_speeds(self.ctx, Sd.ctypes.data, Sa.ctypes.data), "lbm_flame_speeds")
        return Sd, Sa

    @_on_device
    def isoline_means(self, T, T_iso: float, cx: float, cy: float, fields=()):
        """{A, mean R, means of fields} along T = T_iso (see lbm_isoline_means);
        T and fields: float64 device tensors [N]."""
        torch = self.torch
        K = len(fields)
        Td = T.contiguous().to(device=self.device, dtype=torch.float64)
        F = torch.stack([f.to(device=self.device, dtype=torch.float64) for f in fields]).contiguous() if K else None
        out = np.zeros(2 + K)
        _check(lbm_isoline_means(self.ctx, Td.data_ptr(), T_iso, cx, cy, K, F.data_ptr() if K else None, out),
               "lbm_isoline_means")
        return out

    @_on_device
    def chemistry_at(self, rho_a, T):
        """The step's chemistry at given node states: rho_a [M, n], T [n]
        (numpy).  Returns a dict of numpy arrays: rho_dot [M, n], hdot [n],
        dT [n], drho [M, n], dlogA [R, n]."""
        torch = self.torch
        rho_a = np.ascontiguousarray(rho_a, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        n = T.size
        dev = self.device
        ri = torch.from_numpy(rho_a).to(dev)
        ti = torch.from_numpy(T).to(dev)
        out = {"rho_dot": torch.empty((self.M, n), dtype=torch.float64, device=dev),
               "hdot": torch.empty(n, dtype=torch.float64, device=dev),
               "dT": torch.empty(n, dtype=torch.float64, device=dev),
               "drho": torch.empty((self.M, n), dtype=torch.float64, device=dev),
               "dlogA": torch.empty((max(self.R, 1), n), dtype=torch.float64, device=dev)}
        _check(lbm_chemistry_at(self.ctx, n, ri.data_ptr(), ti.data_ptr(), out["rho_dot"].data_ptr(),
                                out["hdot"].data_ptr(), out["dT"].data_ptr(), out["drho"].data_ptr(),
                                out["dlogA"].data_ptr()), "lbm_chemistry_at")
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["dlogA"] = res["dlogA"][:self.R]
        return res

    @_on_device
    def temperature_at(self, Y, e, T_guess):
        """The step's Newton temperature at given (Y [M, n], e [n]) from T_guess [n]."""
        torch = self.torch
        dev = self.device
        Yt = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float64)).to(dev)
        et = torch.from_numpy(np.ascontiguousarray(e, dtype=np.float64)).to(dev)
        t0 = torch.from_numpy(np.ascontiguousarray(T_guess, dtype=np.float64)).to(dev)
        T = torch.empty_like(et)
        _check(lbm_temperature_at(self.ctx, et.numel(), Yt.data_ptr(), et.data_ptr(), t0.data_ptr(), T.data_ptr()),
               "lbm_temperature_at")
        return T.cpu().numpy()

    @_on_device
    def populations(self) -> np.ndarray:
        out = np.empty((self.S, 27, self.N), dtype=np.float64)
        _check(lbm_get_populations(self.ctx, out), "lbm_get_populations")
        return out


# ---------------------------------------------------------------------------
# Gradients of the time-integrated heat release as a torch.autograd.Function
# ---------------------------------------------------------------------------
def _heat_release_function():
    import torch

    class HeatReleaseObjective(torch.autograd.Function):
        """J(ln A, T0) = sum_{t < steps} sum_nodes hdot^c (Sec. 5b) of a
        periodic double-precision lattice started by lbm_init from the
        problem's mole fractions, pressure and zero velocity at T(x, 0) = T0.
        forward runs lbm_heat_release_gradient (forward sweep with
        checkpoints every checkpoint_every steps, then the hand-written
        reverse sweep); backward scales the stored gradients by the incoming
        gradient.  Inputs: log_A [R] and T0 [N] float64 tensors."""

        @staticmethod
        def forward(ctx, log_A, T0, problem, steps, checkpoint_every):
            import copy
            mech = copy.deepcopy(problem.mech)
            mech.log_A = log_A.detach().cpu().numpy().astype(np.float64)
            dev = T0.device if T0.is_cuda else torch.device("cuda", torch.cuda.current_device())
            s = Solver(problem.lattice, problem.species, mech, LBM_FP64, device=dev)
            try:
                s.init(problem.init.X, T0.detach().cpu().numpy().astype(np.float64), None, problem.init.P)
                J, dA, dT0, _ = s.heat_release_gradient(int(steps), int(checkpoint_every))
            finally:
                s.close()
            ctx.save_for_backward(torch.from_numpy(dA).to(log_A.device), dT0.to(T0.device))
            return torch.tensor(J, dtype=torch.float64, device=T0.device)

        @staticmethod
        def backward(ctx, gJ):
            dA, dT0 = ctx.saved_tensors
            return gJ.to(dA.device) * dA, gJ.to(dT0.device) * dT0, None, None, None

    return HeatReleaseObjective


_HRO = None


def heat_release_objective(log_A, T0, problem, steps: int, checkpoint_every: int = 64):
    """Differentiable time-integrated heat release (HeatReleaseObjective.apply)."""
    global _HRO
    if _HRO is None:
        _HRO = _heat_release_function()
    return _HRO.apply(log_A, T0, problem, steps, checkpoint_every)
