"""Heat release rate hdot^c = -sum_a H_a rho_dot_a (Sec. 5b) and its
sensitivities on the GPU, against the oracle.

* Node functions (lbm_chemistry_at) on seeded node states that both sides
  receive unchanged (workload.node_states: 700-2600 K, trace species over
  six decades, some species absent): the step's production rates against
  the oracle's rate function, hdot^c against the oracle's, and the
  derivatives in T, rho_a and ln A_k against central differences of the
  oracle (tests/hrr_fd.py).  Bars: rates 1e-10 of each species' largest
  (2e-6 with the fast mixed unit's float exponentials), hdot^c 1e-10 of the
  largest, derivatives 1e-6 of the largest of each kind (the differences
  carry ~1e-9).
* The state entry point (lbm_heat_release): its per-node derivatives equal
  the node functions at the state's own moments, its totals equal the sums
  of the per-node values and of the LBM_F_HRR moment row, and they repeat
  bit for bit.
* Against the oracle's own lattice after steps (FP64): J and dJ/d ln A_k.
* At the 256^3 size that bench.py times, after initialisation: sampled
  nodes against the oracle's state of the same node (tests/oracle_patch.py).
"""
import numpy as np
import pytest

import hrr_fd
import oracle_patch
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


def _mode(lbm, name):
    return {"fp64": lbm.LBM_FP64, "mixed": lbm.LBM_MIXED, "mixed_fast": lbm.LBM_MIXED_FAST}[name]


def _tiny_solver(lbm, sp, mech, mode):
    from workload.problem import InitFields, LatticeSpec, Problem
    lat = LatticeSpec(5, 4, 3)
    N = lat.n_nodes
    X = np.tile((w.configs.PHI1_X + 1e-3)[:, None] / (1 + 9e-3), (1, N))
    prob = Problem("tiny", lat, sp, mech, InitFields(X=X, T=np.full(N, 1200.0), u=None, P=mech.P0))
    return lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))


def _max_rel(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("mode,rate_tol", [("fp64", 1e-10), ("mixed", 1e-10), ("mixed_fast", 2e-6)])
def test_node_functions_against_oracle(orc, lbm, mode, rate_tol):
    sp, mech = w.mech9()
    rho_a, T = w.node_states(sp.M, 700, seed=11)
    s = _tiny_solver(lbm, sp, mech, mode)
    g = s.chemistry_at(rho_a, T)
    s.close()
    o = hrr_fd.oracle_of(orc, sp, mech)
    rates = np.array([o.rates(rho_a[:, i], T[i]) for i in range(T.size)]).T
    for a in range(sp.M):
        scale = np.abs(rates[a]).max()
        if scale == 0.0:                       # a species no reaction involves
            assert np.abs(g["rho_dot"][a]).max() == 0.0
            continue
        assert np.abs(g["rho_dot"][a] - rates[a]).max() <= rate_tol * scale, a
    h = hrr_fd.hdot(o, rho_a, T)
    assert np.abs(h).max() > 0 and _max_rel(g["hdot"], h) <= 1e-10
    assert _max_rel(g["dT"], hrr_fd.d_dT(o, rho_a, T)) <= 1e-6
    fd = hrr_fd.d_drho(o, rho_a, T)
    for a in range(sp.M):
        scale = max(np.abs(fd[a]).max(), 1e-300)
        assert np.abs(g["drho"][a] - fd[a]).max() <= 1e-6 * scale, a
    fdA = hrr_fd.d_dlogA(orc, sp, mech, rho_a, T)
    assert np.abs(g["dlogA"] - fdA).max() <= 1e-6 * np.abs(fdA).max()


def test_log_A_derivatives_sum_to_hdot_without_falloff(lbm):
    """With every reaction elementary or third-body, hdot^c is a sum of
    terms each proportional to one A_k, so sum_k d hdot^c/d ln A_k =
    hdot^c (Euler's relation for homogeneous functions)."""
    sp, mech = w.mech9()
    fall = mech.rtype == 2
    mech.rtype = np.where(fall, 1, mech.rtype).astype(np.int32)
    rho_a, T = w.node_states(sp.M, 300, seed=12)
    s = _tiny_solver(lbm, sp, mech, "fp64")
    g = s.chemistry_at(rho_a, T)
    s.close()
    assert fall.any()
    terms = np.abs(g["dlogA"]).sum(axis=0)                 # sum_k |dH_k q_k| per state
    assert np.all(np.abs(g["dlogA"].sum(axis=0) - g["hdot"]) <= 1e-13 * terms)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_fast"])
def test_state_entry_point_matches_node_functions(lbm, mode):
    prob = w.sphere3d_problem(shape=(21, 18, 17), radius=5.0)
    s = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
    s.step(3)
    J, dA, dT, dr = s.heat_release()
    J2, dA2, dT2, dr2 = s.heat_release()
    assert J == J2 and np.array_equal(dA, dA2) and np.array_equal(dT, dT2) and np.array_equal(dr, dr2)
    dTd = s.heat_release(device=True)[2]
    assert np.array_equal(dTd.cpu().numpy(), dT)
    assert s.heat_release(gradients=False) == J
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_T | lbm.LBM_F_HRR)
    g = s.chemistry_at(m["rho_a"], m["T"])
    s.close()
    np.testing.assert_allclose(dT, g["dT"], rtol=1e-13, atol=1e-13 * np.abs(g["dT"]).max())
    np.testing.assert_allclose(dr, g["drho"], rtol=1e-13, atol=1e-13 * np.abs(g["drho"]).max())
    habs = np.abs(g["hdot"]).sum()
    assert abs(J - g["hdot"].sum()) <= 1e-12 * habs
    np.testing.assert_allclose(dA, g["dlogA"].sum(axis=1), rtol=0, atol=1e-12 * np.abs(g["dlogA"]).sum())
    # the moment row evaluates the rates as the step does (float accumulation
    # of the reaction contributions in the fast mixed unit)
    tol = 1e-6 if mode == "mixed_fast" else 1e-10
    assert abs(m["hrr"].sum() - J) <= tol * habs
    assert np.abs(m["hrr"] - g["hdot"]).max() <= tol * np.abs(g["hdot"]).max()


def test_fp64_lattice_against_oracle(orc, lbm):
    """J and dJ/d ln A_k of the state after 4 steps, each side from its own
    run of the same problem."""
    prob = w.sphere3d_problem(shape=(14, 12, 10), radius=4.0)
    o = orc.Oracle.from_problem(prob)
    assert o.step(4) == 0
    m = o.moments()
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.step(4)
    J, dA, _, _ = s.heat_release()
    s.close()
    one = hrr_fd.oracle_of(orc, prob.species, prob.mech)
    h = hrr_fd.hdot(one, m["rho_a"], m["T"])
    assert abs(J - h.sum()) <= 1e-9 * np.abs(h).sum()
    fdA = hrr_fd.d_dlogA(orc, prob.species, prob.mech, m["rho_a"], m["T"]).sum(axis=1)
    assert np.abs(dA - fdA).max() <= 1e-6 * np.abs(fdA).max()


@pytest.mark.parametrize("mode,tol", [("mixed", 1e-4), ("fp64", 1e-9)])
def test_fullsize_sampled_nodes_after_init(orc, lbm, mode, tol):
    """256^3, nine species, right after lbm_init: hdot^c (LBM_F_HRR) and
    d hdot^c/dT at 300 sampled nodes (uniform, plus the hot kernel and its
    edge) against the oracle's own state of each node.  In the mixed mode
    the stored state carries the float rounding of the moving populations,
    hence its bar."""
    import torch
    prob = w.sphere3d_problem(n=256, radius=20.0)
    s = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
    rng = np.random.default_rng(21)
    N = prob.lattice.n_nodes
    is_hot = prob.init.T > 1000.0
    hot = np.flatnonzero(is_hot)
    edge = np.flatnonzero(~is_hot & (np.roll(is_hot, 1) | np.roll(is_hot, -1)))   # beside the kernel in x
    nodes = np.concatenate([rng.choice(N, 100, replace=False), rng.choice(hot, 100, replace=False),
                            rng.choice(edge, 100, replace=False)])
    J, dA, dT, _ = s.heat_release(device=True)
    m = s.moments(lbm.LBM_F_HRR, device=True)
    idx = torch.from_numpy(nodes).to(dT.device)
    got_h = m["hrr"][idx].cpu().numpy()
    got_dT = dT[idx].cpu().numpy()
    hsum = float(m["hrr"].sum().item())
    habs = float(m["hrr"].abs().sum().item())
    del m, dT
    s.close()
    del s
    torch.cuda.empty_cache()
    assert abs(hsum - J) <= 1e-10 * habs
    one = hrr_fd.oracle_of(orc, prob.species, prob.mech)
    ref_h, ref_dT = [], []
    for n in nodes:
        st = oracle_patch.node_state_after_init(orc, prob, int(n))
        R1, T1 = st["rho_a"][:, None], np.array([st["T"]])
        ref_h.append(hrr_fd.hdot(one, R1, T1)[0])
        ref_dT.append(hrr_fd.d_dT(one, R1, T1)[0])
    ref_h, ref_dT = np.array(ref_h), np.array(ref_dT)
    assert np.abs(ref_h).max() > 0
    assert _max_rel(got_h, ref_h) <= tol
    assert _max_rel(got_dT, ref_dT) <= max(tol, 1e-6)


def test_node_functions_argument_checks(lbm):
    """Host pointers and negative counts are rejected before any launch;
    n = 0 does nothing; the context stays usable."""
    import torch
    sp, mech = w.mech9()
    s = _tiny_solver(lbm, sp, mech, "fp64")
    rho_h = np.ones((sp.M, 4))
    T_h = np.full(4, 1000.0)
    T_d = torch.full((4,), 1000.0, dtype=torch.float64, device="cuda")
    rho_d = torch.ones((sp.M, 4), dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    assert lbm.lbm_chemistry_at(s.ctx, 4, rho_h.ctypes.data, T_d.data_ptr(), None, out.data_ptr()) == lbm.LBM_ERR_ARG
    assert lbm.lbm_chemistry_at(s.ctx, -1, rho_d.data_ptr(), T_d.data_ptr()) == lbm.LBM_ERR_ARG
    assert lbm.lbm_chemistry_at(s.ctx, 0, None, None) == lbm.LBM_OK
    assert lbm.lbm_temperature_at(s.ctx, 4, rho_d.data_ptr(), T_h.ctypes.data, T_d.data_ptr(),
                                  out.data_ptr()) == lbm.LBM_ERR_ARG
    assert lbm.lbm_chemistry_at(s.ctx, 4, rho_d.data_ptr(), T_d.data_ptr(), None, out.data_ptr()) == lbm.LBM_OK
    assert np.isfinite(out.cpu().numpy()).all()
    assert s.step(1) == lbm.LBM_OK
    # a 60-node lattice: one block of partial sums fits the scratch
    J, dA, dT, dr = s.heat_release()
    m = s.moments(lbm.LBM_F_RHO_A | lbm.LBM_F_T)
    g = s.chemistry_at(m["rho_a"], m["T"])
    assert abs(J - g["hdot"].sum()) <= 1e-12 * np.abs(g["hdot"]).sum()
    s.close()


def _near_hot(prob, count, seed):
    rng = np.random.default_rng(seed)
    hot = np.flatnonzero(prob.init.T > 1000.0)
    lat = prob.lattice
    idx = np.arange(lat.n_nodes)
    x, y, z = idx % lat.nx, (idx // lat.nx) % lat.ny, idx // (lat.nx * lat.ny)
    cx, cy, cz = lat.nx // 2, lat.ny // 2, lat.nz // 2
    near = np.flatnonzero((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= 9)
    return rng.choice(np.union1d(hot, near), count, replace=False)


def test_population_gradient_against_oracle(orc, lbm):
    """dJ/dF (lbm_heat_release_adjoint, double) against central differences
    of the oracle's J with respect to single populations of its own state
    after 2 steps: the H2 and O2 sets, the mixture set f and the energy set
    g, rest and moving directions; 1e-5 of the largest sampled value, 1e-4
    of each.  The trace H radical's set separately: its populations are
    ~1e-13 of the density, so its difference step is 1e-2 of them (a step
    of 1e-6 moves hdot^c by less than its rounding), and its bar 1e-3."""
    prob = w.sphere3d_problem(shape=(10, 8, 6), radius=2.5)
    M = prob.species.M
    o = orc.Oracle.from_problem(prob)
    assert o.step(2) == 0
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.step(2)
    G = s.heat_release_adjoint()
    Gd = s.heat_release_adjoint(device=True).cpu().numpy()
    s.close()
    assert np.array_equal(G, Gd)
    rng = np.random.default_rng(31)
    nodes = _near_hot(prob, 8, 32)
    samples = []
    for k, x in enumerate(nodes):
        for st in (0, 1, M - 1, M):
            samples.append((int(x), st, int(rng.integers(27))))
    one = hrr_fd.oracle_of(orc, prob.species, prob.mech)
    fd = hrr_fd.d_dpop(o, one, samples)
    got = np.array([G[st, i, x] for (x, st, i) in samples])
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(got - fd).max() <= 1e-5 * scale
    big = np.abs(fd) > 1e-3 * scale
    assert np.all(np.abs(got - fd)[big] <= 1e-4 * np.abs(fd)[big])
    radical = [(int(x), 3, int(rng.integers(27))) for x in nodes]
    fd_r = hrr_fd.d_dpop(o, one, radical, rel=1e-2)
    got_r = np.array([G[st, i, x] for (x, st, i) in radical])
    assert np.abs(fd_r).max() > 0
    assert np.all(np.abs(got_r - fd_r) <= 1e-3 * np.abs(fd_r) + 1e-5 * scale)


def test_population_gradient_is_the_directional_derivative(lbm):
    """<dJ/dF, delta> equals (J(F + eps delta) - J(F - eps delta)) / (2 eps)
    with J from lbm_heat_release, perturbing the double state in place
    (48 x 40 x 36 nodes, a seeded relative perturbation of every
    population): 1e-6."""
    import torch
    prob = w.sphere3d_problem(shape=(48, 40, 36), radius=8.0)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.step(3)
    G = s.heat_release_adjoint(device=True)
    n_pop = s.S * 27 * s.N
    ptr = lbm.lbm_state_buffer(s.ctx)
    buf = s.pop[0] if s.pop[0].data_ptr() == ptr else s.pop[1]
    F = buf.view(torch.float64)[:n_pop].view(s.S, 27, s.N)
    gen = torch.Generator(device=G.device).manual_seed(41)
    delta = F * (2 * torch.rand(F.shape, generator=gen, device=G.device, dtype=torch.float64) - 1)
    eps = 1e-6
    F0 = F.clone()
    F.add_(eps * delta)
    Jp = s.heat_release(gradients=False)
    F.copy_(F0)
    F.sub_(eps * delta)
    Jm = s.heat_release(gradients=False)
    F.copy_(F0)
    fd = (Jp - Jm) / (2 * eps)
    ad = float((G * delta).sum().item())
    s.close()
    assert ad != 0.0 and abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
def test_population_gradient_mixed_units_match_double(lbm, precision):
    """lbm_heat_release_adjoint in the mixed units (float deviations plus
    double rest and energy populations, summed by their own moment pass)
    against the double unit on the same initial state after 2 steps
    (10 x 8 x 6): per set, 1e-5 of that set's largest |dJ/dF| -- float
    storage moves the state by ~1e-7 relative, and the gradient is smooth
    in the state; the fast unit's float exponential adds ~2e-7."""
    prob = w.sphere3d_problem(shape=(10, 8, 6), radius=2.5)
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    ref.step(2)
    G_ref = ref.heat_release_adjoint()
    ref.close()
    p = {"mixed": lbm.LBM_MIXED, "mixed_fast": lbm.LBM_MIXED_FAST}[precision]
    s = lbm.Solver.from_problem(prob, precision=p)
    s.step(2)
    G = s.heat_release_adjoint()
    s.close()
    assert G.shape == G_ref.shape
    for st in range(G.shape[0]):
        scale = np.abs(G_ref[st]).max()
        assert scale > 0, st
        err = np.abs(G[st] - G_ref[st]).max() / scale
        assert err <= 1e-5, (precision, st, err)
