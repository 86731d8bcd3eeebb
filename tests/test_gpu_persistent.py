"""The persistent step (lbm_step_persistent): n time steps in one
cooperative launch, the phases of each step separated by grid barriers with
a poll limit.

* On a ragged batch of quasi-1D flames (per-flame ghost faces, lengths not
  multiples of the 128-thread block) and on a periodic lattice, the
  populations and the temperature row equal those of lbm_step, for several
  tile lengths and odd step counts (the buffer parity), to rounding: the
  compiler may fuse a multiply and an add inside the combined kernel where
  it does not in a phase's own kernel (one rounding of difference per
  step).  Bounds: 1e-12 of each set's largest value in double, 1e-6 in the
  float units; the temperature row 1e-13 and 1e-7 of its maximum.
* A poll limit of one makes a barrier give up: the call returns
  LBM_ERR_BARRIER, returns at all (no hang), and the context steps
  correctly again once re-initialised.
* The tile-length autotuner leaves the state as it found it and returns
  one of its candidates.
"""
import numpy as np
import pytest

import workload as w

pytestmark = pytest.mark.gpu

LENGTHS = [37, 64, 129, 200, 83]
PHIS = [0.6, 1.0, 2.5, 0.8, 1.4]


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _precision(L, mode):
    return {"fp64": L.LBM_FP64, "mixed": L.LBM_MIXED, "fast": L.LBM_MIXED_FAST}[mode]


def _state(s, n_nodes):
    assert s.sync() == 0
    return s.populations(), s.macro[:n_nodes].cpu().numpy().copy()


def _same(mode, pa, pb, ta, tb):
    tp, tt = (1e-12, 1e-13) if mode == "fp64" else (1e-6, 1e-7)
    scale = np.abs(pa).max(axis=(1, 2), keepdims=True)
    assert (np.abs(pa - pb) <= tp * scale).all(), float((np.abs(pa - pb) / scale).max())
    assert np.abs(ta - tb).max() <= tt * np.abs(ta).max(), float(np.abs(ta - tb).max())


def _pair(L, prob, mode):
    p = _precision(L, mode)
    return L.Solver.from_problem(prob, precision=p), L.Solver.from_problem(prob, precision=p)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fast"])
@pytest.mark.parametrize("tile_mult,steps", [(1, 25), (3, 24), (8, 7)])
def test_batch_persistent_equals_plain_steps(lbm, mode, tile_mult, steps):
    prob = w.batched_flames_problem(lengths=LENGTHS, phis=PHIS)
    n = prob.lattice.n_nodes
    a, b = _pair(lbm, prob, mode)
    a.step(steps)
    b.step_persistent(steps, tile_mult=tile_mult)
    pa, ta = _state(a, n)
    pb, tb = _state(b, n)
    _same(mode, pa, pb, ta, tb)
    # a second call continues from the buffer the first one left
    a.step(5)
    b.step_persistent(5, tile_mult=tile_mult)
    pa, ta = _state(a, n)
    pb, tb = _state(b, n)
    _same(mode, pa, pb, ta, tb)
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fast"])
def test_periodic_persistent_equals_plain_steps(lbm, mode):
    prob = w.small_periodic_problem(n=12)
    n = prob.lattice.n_nodes
    a, b = _pair(lbm, prob, mode)
    a.step(9)
    b.step_persistent(9, tile_mult=2)
    pa, ta = _state(a, n)
    pb, tb = _state(b, n)
    _same(mode, pa, pb, ta, tb)
    a.close()
    b.close()


def test_poll_limit_runs_out_and_the_context_recovers(lbm):
    prob = w.batched_flames_problem(lengths=[4096] * 24, phis=[1.0] * 24)
    n = prob.lattice.n_nodes
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED)
    ref.step(4)
    want = _state(ref, n)
    ref.close()
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED)
    st = s.step_persistent(20, tile_mult=1, spin_cap=1, check=False)
    assert st == lbm.LBM_ERR_BARRIER, lbm.lbm_strerror(st)
    assert s.sync() == lbm.LBM_OK            # the status word was cleared
    s.init(prob.init.X, prob.init.T, prob.init.u, prob.init.P)
    s.step_persistent(4)
    pb, tb = _state(s, n)
    _same("mixed", want[0], pb, want[1], tb)
    s.close()


def test_autotune_keeps_the_state(lbm):
    prob = w.batched_flames_problem(lengths=LENGTHS, phis=PHIS)
    n = prob.lattice.n_nodes
    a, b = _pair(lbm, prob, "mixed")
    a.step(3)
    b.step(3)
    t = b.autotune_persistent(steps=3)
    assert t in (1, 2, 4, 8)
    a.step(4)
    b.step_persistent(4, tile_mult=t)
    pa, ta = _state(a, n)
    pb, tb = _state(b, n)
    _same("mixed", pa, pb, ta, tb)
    a.close()
    b.close()


def test_arguments(lbm):
    prob = w.flame_of_batch(w.batched_flames_problem(lengths=LENGTHS, phis=PHIS), 0)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    assert lbm.lbm_step_persistent(s.ctx, -1, 1, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_persistent(s.ctx, 1, 0, 0) == lbm.LBM_ERR_ARG
    before = s.populations()
    assert lbm.lbm_step_persistent(s.ctx, 0, 1, 0) == lbm.LBM_OK
    assert np.array_equal(s.populations(), before)
    s.close()
