"""Failure detection through the device status word, without any GPU
fault: bad states are planted in the initial fields on the host, the
kernels record them in the status word, and the call that waits returns
the matching LBM_ERR_* -- the same status the oracle returns for the same
state.  Afterwards the context still answers (moments, sync) and steps on.
No value here feeds an index or a size: every access stays in bounds."""
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


def _three_gas(X, T):
    sp, mech = w.mech3()
    lat = LatticeSpec(9, 5, 4, BC_PERIODIC)
    return Problem("three_gas_9x5x4", lat, sp, mech, InitFields(X=X, T=T, u=None, P=sp.r_lat / 23.4))


def _fields(N, seed=11):
    rng = np.random.default_rng(seed)
    X = np.array([[0.3], [0.5], [0.2]]) + rng.uniform(-0.02, 0.02, (3, N))
    X /= X.sum(axis=0, keepdims=True)
    T = 1.0 + rng.uniform(0.0, 0.2, N)
    return X, T


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_negative_species_density_is_reported_like_the_oracle(orc, lbm, mode):
    N = 9 * 5 * 4
    X, T = _fields(N)
    slab = (np.arange(N) % 9 >= 3) & (np.arange(N) % 9 <= 5)
    X[0, slab] = -0.05                                # a slab with a negative species fraction
    X[1, slab] += 0.05                                # (one node alone is outweighed after streaming)
    prob = _three_gas(X, T)
    o = orc.Oracle.from_problem(prob)
    assert o.step(1) == lbm.LBM_ERR_NEGATIVE          # the oracle's own status code
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    s = lbm.Solver.from_problem(prob, precision=p)
    assert s.step(1, check=False) == lbm.LBM_ERR_NEGATIVE
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_T)      # the state stays readable
    assert np.isfinite(m["T"]).all() and m["rho_a"][0, slab].min() < 0
    assert s.sync() == lbm.LBM_OK                     # the status was cleared when it was returned
    s.close()


def test_non_finite_temperature_is_reported(lbm):
    N = 9 * 5 * 4
    X, T = _fields(N)
    T[5] = np.nan
    prob = _three_gas(X, T)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    assert s.step(1, check=False) == lbm.LBM_ERR_NONFINITE
    assert s.sync() == lbm.LBM_OK
    # a fresh valid state in the same context steps cleanly again
    X2, T2 = _fields(N, seed=12)
    s.init(X2, T2, None, prob.init.P)
    assert s.step(3, check=False) == lbm.LBM_OK
    s.close()


def test_mixed_init_rejects_a_non_finite_state_before_any_step(lbm):
    N = 9 * 5 * 4
    X, T = _fields(N)
    T[5] = np.inf
    prob = _three_gas(X, T)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED, init=False)
    with pytest.raises(lbm.LBMError) as e:
        s.init(prob.init.X, prob.init.T, None, prob.init.P)
    assert e.value.status == lbm.LBM_ERR_ARG
    s.close()
