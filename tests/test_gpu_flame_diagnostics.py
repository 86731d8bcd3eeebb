"""Flame diagnostics of the circular expanding flame (Sec. 5b) on the GPU
against the FP64 oracle (the same state: both step the perturbed flame of
Eq. (cflamePerturbation) on a 64 x 64 x 1 periodic box):

* S_d (Eq. (sd)) and S_a = S_d + u . n of the double path after 20 steps at
  the nodes of the flame zone (400 K < T < 1700 K): 1e-9 of the largest
  there;
* the isoline means of Eq. (rmean) of T = 3 T_u -- length, mean radius and
  the means of S_a and of rho S_d -- from the same arrays: 1e-12;
* the mixed path's speeds against the double path's: 1e-3.
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


def _problem():
    return w.circular_flame_problem(n=64, R_ig=14.0, A0=0.1, n0=1, width=2.0)


@pytest.fixture(scope="module")
def oracle_state(orc):
    p = _problem()
    o = orc.Oracle.from_problem(p)
    assert o.step(20) == 0
    Sd, Sa = o.flame_speeds()
    m = o.moments()
    return p, o, Sd, Sa, m


def test_flame_speeds_against_oracle(lbm, oracle_state):
    p, o, Sd_o, Sa_o, m = oracle_state
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP64)
    s.step(20)
    T_before = s.macro[: s.N].clone()
    Sd, Sa = s.flame_speeds()
    assert bool((s.macro[: s.N] == T_before).all())               # the temperature row is kept
    s.close()
    zone = (m["T"] > 400.0) & (m["T"] < 1700.0)
    assert zone.sum() > 100
    for got, ref in ((Sd, Sd_o), (Sa, Sa_o)):
        scale = np.abs(ref[zone]).max()
        assert scale > 0
        assert np.abs(got[zone] - ref[zone]).max() <= 1e-9 * scale


def test_isoline_means_against_oracle(lbm, oracle_state):
    import torch
    p, o, Sd_o, Sa_o, m = oracle_state
    c = (p.lattice.nx - 1) / 2.0
    T_iso = 3 * 298.0
    ref = o.isoline_means(m["T"], T_iso, c, c, [Sa_o, m["rho"] * Sd_o])
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP64)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = s.isoline_means(dev(m["T"]), T_iso, c, c, [dev(Sa_o), dev(m["rho"] * Sd_o)])
    s.close()
    assert ref[0] > 50 and abs(ref[1] - 14.0) < 2.0                 # the perturbed circle is there
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref))


def test_mixed_speeds_against_double(lbm):
    p = _problem()
    out = {}
    for name, prec in (("fp64", lbm.LBM_FP64), ("mixed", lbm.LBM_MIXED)):
        s = lbm.Solver.from_problem(p, precision=prec)
        s.step(20)
        out[name] = s.flame_speeds() + (s.moments(lbm.LBM_F_T)["T"],)
        s.close()
    T = out["fp64"][2]
    zone = (T > 400.0) & (T < 1700.0)
    for k in (0, 1):
        ref = out["fp64"][k][zone]
        assert np.abs(out["mixed"][k][zone] - ref).max() <= 1e-3 * np.abs(ref).max()
