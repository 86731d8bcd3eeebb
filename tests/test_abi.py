"""The C ABI library builds for sm_103a, loads, and exports every entry
point include/lbm.h declares; host-side argument validation (no GPU)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm
    return lbm


def _declared():
    text = (ROOT / "include" / "lbm.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:int|size_t|void \*|const char \*)\s*(lbm_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    raw = C.CDLL(lib.library_path())
    for n in names:
        assert hasattr(raw, n), n
    assert set(lib.EXPORTED) == set(names)


def test_buffer_sizes_and_validation(lib):
    import workload as w
    p = w.sphere3d_problem(n=8, radius=2)
    lat = lib.lbm_lattice(8, 8, 8, 0, lib.LBM_MIXED)
    W = np.ascontiguousarray(p.species.W)
    sp = lib.lbm_species(9, W.ctypes.data_as(C.POINTER(C.c_double)), 1, None, None, 298.15, None, None,
                         0.8, 0.71, p.species.r_lat, 1)
    pop, mac, gh = lib.lbm_buffer_sizes(lat, sp)
    # species and mixture sets: float moving + double rest; energy set: double
    assert pop == 9 * 27 * 512 * 4 + 9 * 512 * 8 + 27 * 512 * 8
    assert mac == (9 + 12) * 512 * 8 + (19 + 7 * 9) * 512 * 4
    assert gh == 0
    lat.precision = lib.LBM_MIXED_FAST           # same layout as LBM_MIXED
    assert lib.lbm_buffer_sizes(lat, sp) == (pop, mac, gh)
    lat.precision = 3
    with pytest.raises(lib.LBMError) as e:
        lib.lbm_buffer_sizes(lat, sp)
    assert e.value.status == lib.LBM_ERR_ARG
    lat.bc_x = 1
    lat.precision = lib.LBM_FP64
    pop, mac, gh = lib.lbm_buffer_sizes(lat, sp)
    assert pop == 10 * 27 * 512 * 8 and gh == 2 * 10 * 27 * 64 * 8
    lat.nx = 0
    with pytest.raises(lib.LBMError) as e:
        lib.lbm_buffer_sizes(lat, sp)
    assert e.value.status == lib.LBM_ERR_ARG


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    raw = C.CDLL(lib.library_path())
    raw.lbm_create.argtypes = [C.c_void_p] * 6
    out = C.c_void_p()
    assert raw.lbm_create(None, None, None, None, None, C.byref(out)) == lib.LBM_ERR_ARG
    assert raw.lbm_create(None, None, None, None, None, None) == lib.LBM_ERR_ARG
    assert lib.lbm_strerror(lib.LBM_ERR_NEGATIVE) == "negative species density"
    assert lib.lbm_strerror(12345) == "unknown status"


def test_context_calls_reject_a_null_context_without_touching_the_gpu(lib):
    raw = C.CDLL(lib.library_path())
    for name, nargs in (("lbm_heat_release", 5), ("lbm_heat_release_adjoint", 2), ("lbm_chemistry_at", 9), ("lbm_temperature_at", 6),
                        ("lbm_step", 2), ("lbm_step_async", 2), ("lbm_step_graph", 2), ("lbm_sync", 1),
                        ("lbm_moments", 3), ("lbm_get_populations", 2), ("lbm_destroy", 1)):
        f = getattr(raw, name)
        f.argtypes = [C.c_void_p] * nargs
        f.restype = C.c_int
        assert f(*([None] * nargs)) == lib.LBM_ERR_ARG, name


def test_buffer_sizes_of_a_batch_of_lattices(lib):
    import workload as w
    p = w.sphere3d_problem(n=8, radius=2)
    W = np.ascontiguousarray(p.species.W)
    sp = lib.lbm_species(9, W.ctypes.data_as(C.POINTER(C.c_double)), 1, None, None, 298.15, None, None,
                         0.8, 0.71, p.species.r_lat, 1)
    seg = (C.c_int * 3)(37, 64, 129)
    lat = lib.lbm_lattice(230, 4, 4, 1, lib.LBM_FP64, 3, C.cast(seg, C.POINTER(C.c_int)))
    pop, mac, gh = lib.lbm_buffer_sizes(lat, sp)
    N = 230 * 16
    assert pop == 10 * 27 * N * 8
    assert gh == 2 * 3 * 10 * 27 * 16 * 8           # two ghost faces per lattice
    bad = []
    seg_short = (C.c_int * 3)(37, 64, 128)          # lengths must add up to nx
    bad.append(lib.lbm_lattice(230, 4, 4, 1, lib.LBM_FP64, 3, C.cast(seg_short, C.POINTER(C.c_int))))
    bad.append(lib.lbm_lattice(230, 4, 4, 0, lib.LBM_FP64, 3, C.cast(seg, C.POINTER(C.c_int))))  # periodic x
    seg_zero = (C.c_int * 3)(0, 101, 129)
    bad.append(lib.lbm_lattice(230, 4, 4, 1, lib.LBM_FP64, 3, C.cast(seg_zero, C.POINTER(C.c_int))))
    bad.append(lib.lbm_lattice(230, 4, 4, 1, lib.LBM_FP64, 3, None))
    for b in bad:
        with pytest.raises(lib.LBMError) as e:
            lib.lbm_buffer_sizes(b, sp)
        assert e.value.status == lib.LBM_ERR_ARG



class _Tables:
    """Valid lbm_* descriptors of the nine-species flame tube, with fake
    (never dereferenced) device pointers: every case below is rejected by
    lbm_create's host-side validation before any CUDA call."""

    def __init__(self, lib):
        import workload as w
        prob = w.flame1d_problem(nx=64)
        sp, mech = prob.species, prob.mech
        self.keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self.keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_double))

        def i(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self.keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_int))

        self.d, self.i = d, i
        L = prob.lattice
        self.lat = lib.lbm_lattice(L.nx, L.ny, L.nz, L.bc_x, lib.LBM_FP64, 0, None)
        self.W = np.array(sp.W, dtype=np.float64)
        self.D = np.array(sp.D, dtype=np.float64)
        self.sp = lib.lbm_species(sp.M, d(self.W), sp.thermo, d(sp.cp_R), d(sp.h_form), sp.T0, d(sp.poly7),
                                  d(self.D), sp.nu, sp.Pr, sp.r_lat, sp.visc_model)
        R = mech.R
        self.nu_f = np.array(mech.nu_f, dtype=np.int32).reshape(R, -1)
        self.rtype = np.array(mech.rtype, dtype=np.int32)
        self.mech = lib.lbm_mechanism(R, i(self.nu_f), i(mech.nu_r.reshape(R, -1)), d(mech.log_A), d(mech.b),
                                      d(mech.theta), i(self.rtype), d(mech.eff), d(mech.low), i(mech.reversible),
                                      mech.T_ref, mech.P0)
        pop, mac, gh = lib.lbm_buffer_sizes(self.lat, self.sp)
        self.sizes = (pop, mac, gh)
        fake = 1 << 40                                   # aligned, never dereferenced
        self.bufs = lib.lbm_buffers(fake, fake + (1 << 36), fake + (2 << 36), fake + (3 << 36), pop, mac, gh)

    def create(self, lib):
        raw = C.CDLL(lib.library_path())
        raw.lbm_create.argtypes = [C.c_void_p] * 6
        out = C.c_void_p()
        st = raw.lbm_create(C.addressof(self.lat), C.addressof(self.sp), C.addressof(self.mech),
                            C.addressof(self.bufs), None, C.byref(out))
        assert not out.value
        return st


def _expect_rejected(lib, t):
    assert t.create(lib) == lib.LBM_ERR_ARG


def test_create_rejects_undersized_and_misaligned_buffers(lib):
    t = _Tables(lib)
    t.bufs.pop_bytes = t.sizes[0] - 1
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.bufs.macro_bytes = t.sizes[1] - 8
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.bufs.ghost_bytes = t.sizes[2] - 8                  # ghost faces of the flame tube
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.bufs.pop_b = t.bufs.pop_a                          # the two population buffers must differ
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.bufs.macro = t.bufs.macro + 8                      # 16-byte alignment
    _expect_rejected(lib, t)


def test_create_rejects_bad_species(lib):
    t = _Tables(lib)
    t.W[3] = 0.0                                         # zero molar mass
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.D[1, 2] *= 1.5                                     # asymmetric binary diffusivity
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.D[0, 4] = t.D[4, 0] = -0.01                        # negative diffusivity
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.sp.nu = 0.0
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.sp.thermo = 7
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.sp.transport = 1                                   # mixture-averaged transport without its tables
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.sp.transport = 4                                   # unknown transport model
    _expect_rejected(lib, t)


def test_create_rejects_bad_mechanisms(lib):
    t = _Tables(lib)
    t.rtype[0] = 5                                       # unknown reaction type
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.nu_f[2, :] = 0
    t.nu_f[2, 0] = 4                                     # more than three reactant molecules
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.nu_f[3, :] = 0                                     # a reaction without reactants
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.mech.log_A = None                                  # missing rate table
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.mech.R = 33                                        # more reactions than the build holds
    _expect_rejected(lib, t)
    t = _Tables(lib)
    t.lat.precision = 9
    _expect_rejected(lib, t)


def test_valid_tables_pass_host_validation(lib):
    """The unmodified descriptors get past every host-side check: without a
    GPU the call then fails at its first CUDA call (LBM_ERR_CUDA); with one
    it creates a context (no kernel touches the placeholder buffers) that is
    destroyed at once."""
    t = _Tables(lib)
    raw = C.CDLL(lib.library_path())
    raw.lbm_create.argtypes = [C.c_void_p] * 6
    raw.lbm_destroy.argtypes = [C.c_void_p]
    out = C.c_void_p()
    st = raw.lbm_create(C.addressof(t.lat), C.addressof(t.sp), C.addressof(t.mech), C.addressof(t.bufs), None,
                        C.byref(out))
    if out.value:
        raw.lbm_destroy(out)
    assert st in (lib.LBM_OK, lib.LBM_ERR_CUDA), st
