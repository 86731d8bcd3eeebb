"""The 256^3 nine-species expanding-flame lattice that bench.py times, in
the same launch configuration, checked where the oracle can check it:

* lattice totals after three steps: mass, the mass of each element (H, O,
  N; reactions only move them between species), momentum and total energy
  including formation enthalpy are conserved (1e-12 double, 1e-7 mixed);
* 600 sampled nodes (uniform over the box plus the hot kernel and its
  edge), right after initialisation: the moments, the temperature and the
  production rates of the GPU state equal those of the oracle's own state
  of the node (a 3x3x3 oracle patch of the initial fields,
  tests/oracle_patch.py); densities 1e-13 of each species' largest,
  temperature 1e-11, rates 1e-10 of each species' largest in double, and
  1e-5, 1e-5, 1e-4 in the mixed modes, whose stored state carries the
  float rounding of the moving populations.

Also: a uniform state (at rest or moving, chemistry off) is a fixed point
of the GPU step: exactly in double, and in the mixed modes up to the float
rounding of the stored moving populations (at most ~1e-8 of the largest
population per step)."""
import numpy as np
import pytest

import oracle_patch
import workload as w
from workload.problem import LatticeSpec, BC_PERIODIC

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


def _mode(lbm, name):
    return {"fp64": lbm.LBM_FP64, "mixed": lbm.LBM_MIXED, "mixed_fast": lbm.LBM_MIXED_FAST}[name]


def _totals(s, lbm, species):
    import torch
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_RHOU | lbm.LBM_F_RHOE, device=True)
    rho_a = m["rho_a"]                                     # [M, N]
    mol = rho_a / torch.tensor(species.W, dtype=torch.float64, device=rho_a.device)[:, None]
    elem = torch.tensor(species.elements, dtype=torch.float64, device=rho_a.device)   # [E, M]
    out = {"mass": float(rho_a.sum().item()),
           "elements": (elem @ mol.sum(dim=1)).cpu().numpy(),
           "momentum": m["rhou"].sum(dim=1).cpu().numpy(),
           "energy": float(m["rhoE"].sum().item())}
    del m, rho_a, mol
    return out


def _sample_nodes(prob, count=600, seed=5):
    n = prob.lattice.nx
    rng = np.random.default_rng(seed)
    N = prob.lattice.n_nodes
    uniform = rng.choice(N, count // 2, replace=False)
    hot = np.flatnonzero(prob.init.T > 0.5 * (prob.init.T.max() + prob.init.T.min()))
    # the hot kernel and a shell around it: x, y, z near the centre
    c = n // 2
    idx = np.arange(N)
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    shell = np.flatnonzero(r < 0.15 * n)
    near = rng.choice(np.union1d(hot, shell), count - count // 2, replace=False)
    return np.concatenate([uniform, near])


@pytest.mark.parametrize("mode", ["mixed", "mixed_fast", "fp64"])
def test_fullsize_conservation_and_sampled_nodes(orc, lbm, mode):
    import torch
    prob = w.sphere3d_problem(n=256, radius=20.0)
    sp = prob.species
    s = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
    nodes_np = _sample_nodes(prob)
    nodes = torch.from_numpy(nodes_np).cuda()
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_RHOE | lbm.LBM_F_T | lbm.LBM_F_RHO_DOT, device=True)
    pick = {k: (v[..., nodes] if v.dim() > 1 else v[nodes]).cpu().numpy() for k, v in m.items()}
    del m
    t0 = _totals(s, lbm, sp)
    s.step(3)
    t1 = _totals(s, lbm, sp)
    s.close()
    del s
    torch.cuda.empty_cache()
    tol = 1e-12 if mode == "fp64" else 1e-7
    assert abs(t1["mass"] - t0["mass"]) <= tol * t0["mass"]
    assert np.all(np.abs(t1["elements"] - t0["elements"]) <= tol * np.abs(t0["elements"]))
    assert abs(t1["energy"] - t0["energy"]) <= tol * abs(t0["energy"])
    assert np.abs(t1["momentum"] - t0["momentum"]).max() <= tol * t0["mass"]

    one = orc.Oracle(LatticeSpec(1, 1, 1, BC_PERIODIC), sp, prob.mech)
    T_tol, rate_tol, rho_tol = (1e-11, 1e-10, 1e-13) if mode == "fp64" else (1e-5, 1e-4, 1e-5)
    ref = {"rho_a": [], "rhoE": [], "T": [], "rho_dot": []}
    for n in nodes_np:
        st = oracle_patch.node_state_after_init(orc, prob, int(n))
        for k in ("rho_a", "rhoE", "T"):
            ref[k].append(st[k])
        ref["rho_dot"].append(one.rates(st["rho_a"], st["T"]))
    ref = {k: np.array(v) for k, v in ref.items()}
    ref["rho_a"], ref["rho_dot"] = ref["rho_a"].T, ref["rho_dot"].T
    for a in range(sp.M):
        scale = np.abs(ref["rho_a"][a]).max()
        assert np.abs(pick["rho_a"][a] - ref["rho_a"][a]).max() <= rho_tol * scale, a
    assert np.abs(pick["rhoE"] - ref["rhoE"]).max() <= rho_tol * np.abs(ref["rhoE"]).max()
    assert np.all(np.abs(pick["T"] - ref["T"]) <= T_tol * ref["T"])
    assert np.abs(ref["rho_dot"]).max() > 0
    for a in range(sp.M):
        scale = np.abs(ref["rho_dot"][a]).max()
        if scale == 0.0:                        # a species no reaction involves (N2)
            assert np.abs(pick["rho_dot"][a]).max() == 0.0, a
            continue
        assert np.abs(pick["rho_dot"][a] - ref["rho_dot"][a]).max() <= rate_tol * scale, a


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_fast"])
def test_uniform_states_are_fixed_points(lbm, mode):
    sp, mech = w.mech3()
    mech.log_A[:] = -800.0                      # chemistry off
    from workload.problem import InitFields, Problem
    lat = LatticeSpec(13, 6, 5, BC_PERIODIC)
    N = lat.n_nodes
    X = np.tile(np.array([[0.3], [0.5], [0.2]]), (1, N))
    T = np.full(N, 1.3)
    P = sp.r_lat / 23.4
    for u0 in (np.zeros(3), np.array([0.02, -0.01, 0.005])):
        prob = Problem("uniform", lat, sp, mech, InitFields(X=X, T=T, u=np.tile(u0[:, None], (1, N)), P=P))
        s = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
        p0 = s.populations()
        s.step(100)
        p1 = s.populations()
        s.step(100)
        p2 = s.populations()
        s.close()
        scale = np.abs(p0).max()
        if mode == "fp64":
            assert np.abs(p1 - p0).max() <= 1e-14 * scale
        else:
            # the moving populations are rounded to float at every store; on a
            # uniform state every node rounds alike, so the state moves by at
            # most about one float rounding (6e-8 of the scale) per step
            assert np.abs(p1 - p0).max() <= 100 * 1e-8 * scale, mode
            assert np.abs(p2 - p1).max() <= 100 * 1e-8 * scale, mode
