"""Batches of independent quasi-1D flames side by side in x (one lattice,
per-flame ghost faces), and stepping through a captured CUDA graph.

* A batch evolves each flame exactly as that flame alone: bitwise in double
  precision against single-flame GPU runs, and within the parity bars
  against the FP64 oracle run flame by flame (1e-10 for the double path,
  1e-4 in Y and T for the mixed path).
* lbm_step_graph gives the same populations, bit for bit, as lbm_step.
Flame lengths are ragged (not multiples of the 128-thread block) and the
equivalence ratios differ per flame."""
import numpy as np
import pytest

import workload as w

pytestmark = pytest.mark.gpu

LENGTHS = [37, 64, 129]
PHIS = [0.6, 1.0, 2.5]


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _batch():
    return w.batched_flames_problem(lengths=LENGTHS, phis=PHIS)


def _segment(field, prob, k):
    lat = prob.lattice
    x0 = sum(lat.seg_nx[:k])
    xs = np.arange(lat.n_nodes) % lat.nx
    sel = (xs >= x0) & (xs < x0 + lat.seg_nx[k])
    return field[..., sel]


MASK_NAMES = ("rho_a", "rhou", "rhoE", "T", "Y")


def _moments(s, L):
    return s.moments(L.LBM_F_RHO_A | L.LBM_F_RHOU | L.LBM_F_RHOE | L.LBM_F_T | L.LBM_F_Y)


def test_batch_equals_single_flames_bitwise_fp64(lbm):
    prob = _batch()
    sb = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    sb.step(60)
    mb = _moments(sb, lbm)
    sb.close()
    for k in range(len(LENGTHS)):
        fk = w.flame_of_batch(prob, k)
        s1 = lbm.Solver.from_problem(fk, precision=lbm.LBM_FP64)
        s1.step(60)
        m1 = _moments(s1, lbm)
        s1.close()
        for name in MASK_NAMES:
            assert np.array_equal(_segment(mb[name], prob, k), m1[name]), (k, name)


def test_batch_heat_release_equals_single_flames(lbm):
    """lbm_heat_release on a batch: the per-node derivatives of each flame
    are those of the flame alone, bit for bit (double precision), and J and
    dJ/d ln A_k are the sums over the flames (up to the order of the sums)."""
    prob = _batch()
    sb = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    sb.step(60)
    Jb, dAb, dTb, drb = sb.heat_release()
    sb.close()
    Js, dAs, habs = 0.0, 0.0, 0.0
    for k in range(len(LENGTHS)):
        s1 = lbm.Solver.from_problem(w.flame_of_batch(prob, k), precision=lbm.LBM_FP64)
        s1.step(60)
        J1, dA1, dT1, dr1 = s1.heat_release()
        h1 = s1.moments(lbm.LBM_F_HRR)["hrr"]
        s1.close()
        assert np.array_equal(_segment(dTb, prob, k), dT1), k
        assert np.array_equal(_segment(drb, prob, k), dr1), k
        Js, dAs, habs = Js + J1, dAs + dA1, habs + np.abs(h1).sum()
    assert habs > 0 and abs(Jb - Js) <= 1e-12 * habs
    assert np.abs(dAb - dAs).max() <= 1e-10 * np.abs(dAs).max()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("mode,steps,tol", [("fp64", 60, 1e-10), ("mixed", 100, 1e-4)])
def test_batch_against_oracle_flame_by_flame(orc, lbm, mode, steps, tol):
    prob = _batch()
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    sb = lbm.Solver.from_problem(prob, precision=p)
    sb.step(steps)
    mb = _moments(sb, lbm)
    sb.close()
    for k in range(len(LENGTHS)):
        o = orc.Oracle.from_problem(w.flame_of_batch(prob, k))
        assert o.step(steps) == 0
        ref = o.moments()
        keys = ("T",) if mode == "mixed" else ("T", "rhoE")
        for name in keys:
            assert _rel(_segment(mb[name], prob, k), ref[name]) <= tol, (k, name)
        for a in range(9):
            assert _rel(_segment(mb["Y"][a], prob, k), ref["Y"][a]) <= tol, (k, "Y", a)
            if mode == "fp64":
                assert _rel(_segment(mb["rho_a"][a], prob, k), ref["rho_a"][a]) <= tol, (k, "rho_a", a)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_graph_steps_equal_plain_steps(lbm, mode):
    import torch
    prob = _batch()
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    stream = torch.cuda.Stream()
    a = lbm.Solver.from_problem(prob, precision=p, stream=stream)
    b = lbm.Solver.from_problem(prob, precision=p, stream=stream)
    a.step(7)
    b.step_graph(3)          # captured from buffer A; odd count leaves the state in B
    b.step_graph(4)          # one aligning plain step, one graph launch, one plain step
    assert b.sync() == lbm.LBM_OK
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_contexts_with_equal_tables_share_constant_slots(lbm):
    """Eight double-precision contexts of one mechanism (more than the four
    constant-memory slots) and eight mixed contexts given the same rest
    references all create, and each steps like a lone context."""
    prob = w.flame_of_batch(_batch(), 0)
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    ref.step(5)
    want = ref.populations()
    ref.close()
    many = [lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64) for _ in range(8)]
    for s in many:
        s.step(5)
    for s in many:
        assert np.array_equal(s.populations(), want)
        s.close()
    first = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED)
    refs = first.references()
    mixed = [first]
    for _ in range(7):
        s = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED, init=False)
        s.set_references(refs)
        s.init(prob.init.X, prob.init.T, prob.init.u, prob.init.P)
        mixed.append(s)
    for s in mixed:
        s.step(5)
    want = mixed[0].populations()
    for s in mixed[1:]:
        assert np.array_equal(s.references(), refs)
        assert np.array_equal(s.populations(), want)
    for s in mixed:
        s.close()


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_restart_from_state_buffer_and_references(lbm, mode):
    """A checkpoint is the state buffer, the temperature row of the record
    and (mixed modes) the rest references: a new context restored from them
    continues bit for bit."""
    import torch
    prob = _batch()
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    a = lbm.Solver.from_problem(prob, precision=p)
    a.step(30)
    nbytes = a.pop[0].numel()
    state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    src = a.pop[0] if a.pop[0].data_ptr() == lbm.lbm_state_buffer(a.ctx) else a.pop[1]
    state.copy_(src)
    T_row = a.macro[:prob.lattice.n_nodes].clone()
    refs = a.references() if mode != "fp64" else None
    b = lbm.Solver.from_problem(prob, precision=p, init=False)
    if refs is not None:
        b.set_references(refs)
    dst = b.pop[0] if b.pop[0].data_ptr() == lbm.lbm_state_buffer(b.ctx) else b.pop[1]
    dst.copy_(state)
    b.macro[:prob.lattice.n_nodes].copy_(T_row)
    torch.cuda.synchronize()
    a.step(20)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()
