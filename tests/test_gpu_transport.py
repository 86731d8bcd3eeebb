"""Mixture-averaged transport (LBM_TRANSPORT_MIXTURE_AVERAGED: the viscosity,
conductivity and binary diffusivities of each node's composition,
temperature and pressure, the stand-in for the coefficients the paper takes
from Cantera, Sec. 3 after Eq. (lambda)) against the FP64 oracle:

* the double path on the nine-species expanding flame (20 x 18 x 16,
  radius 5, seeded transport of workload.with_mixture_transport) after
  100 steps: 1e-10 in every moment field;
* the mixed paths (transport coefficients in float, like the relaxation
  rates they set): 1e-4 in mass fractions and temperature;
* the three-gas workload with transport after 200 steps: 1e-10;
* the adjoint refuses contexts with this transport (not built for it).
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


def _sphere():
    p = w.sphere3d_problem(shape=(20, 18, 16), radius=5.0)
    p.species = w.with_mixture_transport(p.species, w.configs.PHI1_X + 1e-12, p.mech.P0, 300.0)
    return p


def _config1():
    p = w.config1_problem()
    X0 = np.array([0.3, 0.5, 0.2])
    p.species = w.with_mixture_transport(p.species, X0, p.init.P, 1.0, nup_ref=0.5)
    return p


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def sphere_ref(orc):
    p = _sphere()
    o = orc.Oracle.from_problem(p)
    assert o.step(100) == 0
    return p, o.moments()


def test_fp64_against_oracle_nine_species(lbm, sphere_ref):
    p, ref = sphere_ref
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP64)
    s.step(100)
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_RHOU | lbm.LBM_F_RHOE | lbm.LBM_F_T | lbm.LBM_F_Y)
    s.close()
    worst = {"rhou": _rel(m["rhou"], ref["rhou"]), "rhoE": _rel(m["rhoE"], ref["rhoE"]), "T": _rel(m["T"], ref["T"])}
    for a in range(p.species.M):
        worst[f"rho_a{a}"] = _rel(m["rho_a"][a], ref["rho_a"][a])
        worst[f"Y{a}"] = _rel(m["Y"][a], ref["Y"][a])
    bad = {k: v for k, v in worst.items() if not v <= 1e-10}
    assert not bad, bad


@pytest.mark.parametrize("mode", ["mixed", "mixed_fast"])
def test_mixed_against_oracle_nine_species(lbm, sphere_ref, mode):
    p, ref = sphere_ref
    prec = lbm.LBM_MIXED if mode == "mixed" else lbm.LBM_MIXED_FAST
    s = lbm.Solver.from_problem(p, precision=prec)
    s.step(100)
    m = s.moments(lbm.LBM_F_T | lbm.LBM_F_Y)
    s.close()
    err = [_rel(m["T"], ref["T"])] + [_rel(m["Y"][a], ref["Y"][a]) for a in range(p.species.M)]
    assert max(err) <= 1e-4, err


def test_fp64_against_oracle_three_gas(orc, lbm):
    p = _config1()
    o = orc.Oracle.from_problem(p)
    assert o.step(200) == 0
    ref = o.moments()
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP64)
    s.step(200)
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_RHOU | lbm.LBM_F_RHOE | lbm.LBM_F_T)
    s.close()
    for k in ("rhou", "rhoE", "T"):
        assert _rel(m[k], ref[k]) <= 1e-10, k
    for a in range(3):
        assert _rel(m["rho_a"][a], ref["rho_a"][a]) <= 1e-10, a


def test_adjoint_refuses_mixture_averaged_transport(lbm):
    import torch
    p = w.sphere3d_problem(shape=(8, 6, 5), radius=2.0)
    p.species = w.with_mixture_transport(p.species, w.configs.PHI1_X + 1e-12, p.mech.P0, 300.0)
    s = lbm.Solver.from_problem(p, precision=lbm.LBM_FP64)
    lam = torch.zeros((s.S, 27, s.N), dtype=torch.float64, device="cuda")
    ws = torch.empty(lbm.lbm_adjoint_workspace_bytes(s.ctx, 0, 1), dtype=torch.uint8, device="cuda")
    assert lbm.lbm_adjoint_step(s.ctx, lam.data_ptr(), torch.empty_like(lam).data_ptr(), None, True,
                                ws.data_ptr(), ws.numel()) == lbm.LBM_ERR_UNSUPPORTED
    s.close()
