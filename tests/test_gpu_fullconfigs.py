"""Parity at the full sizes of the quasi-1D workloads, in the launch
configuration the library uses for them:

* the 4096x4x4 flame tube (ghost-node faces) against the oracle after 200
  steps, every node of every moment field (double path, 1e-10);
* the 512x4x4 flame tube against the oracle after 2000 steps (double path);
* the full batch of 48 ragged flames (1.69 M nodes) against the same 48
  flames stepped one per context: bit for bit, in double precision and in
  mixed precision with the batch's rest references given to every context.
"""
import numpy as np
import pytest

import workload as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _fields(m):
    out = {"rhou": m["rhou"], "rhoE": m["rhoE"], "T": m["T"]}
    for a in range(m["rho_a"].shape[0]):
        out[f"rho_a{a}"] = m["rho_a"][a]
        out[f"Y{a}"] = m["Y"][a]
    return out


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("nx,steps,tol", [(4096, 200, 1e-10), (512, 2000, 1e-10)])
def test_flame_tube_full_size_against_oracle(orc, lbm, nx, steps, tol):
    prob = w.flame1d_problem(nx=nx)
    o = orc.Oracle.from_problem(prob)
    assert o.step(steps) == 0
    ref = _fields(o.moments())
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.step(steps)
    got = _fields(s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_RHOU | lbm.LBM_F_RHOE | lbm.LBM_F_T | lbm.LBM_F_Y))
    s.close()
    err = {k: _rel(got[k], ref[k]) for k in ref}
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, bad


def _segment_slices(prob):
    lat = prob.lattice
    xs = np.arange(lat.n_nodes) % lat.nx
    x0 = 0
    for L in lat.seg_nx:
        yield (xs >= x0) & (xs < x0 + L)
        x0 += L


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_full_batch_of_48_flames_equals_single_flames(lbm, mode):
    steps = 30
    prob = w.batched_flames_problem()
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    b = lbm.Solver.from_problem(prob, precision=p)
    refs = b.references() if mode != "fp64" else None
    b.step(steps)
    mask = lbm.LBM_F_RHO_A | lbm.LBM_F_RHOU | lbm.LBM_F_RHOE | lbm.LBM_F_T
    mb = b.moments(mask)
    b.close()
    for k, sel in enumerate(_segment_slices(prob)):
        fk = w.flame_of_batch(prob, k)
        s = lbm.Solver.from_problem(fk, precision=p, init=False)
        if refs is not None:
            s.set_references(refs)
        s.init(fk.init.X, fk.init.T, fk.init.u, fk.init.P)
        s.step(steps)
        m1 = s.moments(mask)
        s.close()
        for name in ("rho_a", "rhou", "rhoE", "T"):
            assert np.array_equal(mb[name][..., sel], m1[name]), (k, name)
