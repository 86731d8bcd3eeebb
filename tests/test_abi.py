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

