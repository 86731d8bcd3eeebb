"""A context belongs to the device current at lbm_create.  The constant-
memory tables of each device are kept apart (two contexts with the same
tables on two devices each get an uploaded slot on their own device), and a
call made with another device current is rejected with LBM_ERR_ARG instead
of launching on the wrong device.  The Solver binding makes its own device
current around every call."""
import numpy as np
import pytest

import workload as w
from workload.problem import InitFields, LatticeSpec, Problem, BC_PERIODIC

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


def _problem():
    sp, mech = w.mech3()
    lat = LatticeSpec(9, 5, 4, BC_PERIODIC)
    N = 9 * 5 * 4
    rng = np.random.default_rng(5)
    X = np.array([[0.3], [0.5], [0.2]]) + rng.uniform(-0.02, 0.02, (3, N))
    X /= X.sum(axis=0, keepdims=True)
    T = 1.0 + rng.uniform(0.0, 0.2, N)
    return Problem("three_gas_9x5x4", lat, sp, mech, InitFields(X=X, T=T, u=None, P=sp.r_lat / 23.4))


def test_solver_binds_the_current_device(lbm):
    import torch
    s = lbm.Solver.from_problem(_problem(), precision=lbm.LBM_FP64)
    assert s.device.index == torch.cuda.current_device()
    assert s.step(2) == lbm.LBM_OK
    s.close()


def test_contexts_on_two_devices_keep_their_own_tables(lbm):
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    prob = _problem()
    torch.cuda.set_device(0)
    s0 = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64, device="cuda:0")
    s1 = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64, device="cuda:1")
    assert s0.step(3) == lbm.LBM_OK and s1.step(3) == lbm.LBM_OK
    m0, m1 = s0.moments(), s1.moments()
    for k in m0:
        np.testing.assert_array_equal(m0[k], m1[k])   # same tables, same kernels, same order
    # a raw call with device 0 current on the device-1 context is refused
    assert torch.cuda.current_device() == 0
    assert lbm.lbm_step(s1.ctx, 1) == lbm.LBM_ERR_ARG
    assert s1.sync() == lbm.LBM_OK
    s0.close()
    s1.close()
