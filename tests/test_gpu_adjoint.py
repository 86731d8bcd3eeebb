"""The hand-written adjoint of the double-precision step and the gradients
of the time-integrated heat release through the dynamics.

* One reverse step (lbm_adjoint_step) is the transpose of the step's
  Jacobian: for L(F) = <lam, step(F)> (+ J_t(F), the heat release the
  step's collision sees), <lbm_adjoint_step(lam), delta> equals the central
  difference (L(F + eps delta) - L(F - eps delta)) / (2 eps) of the forward
  step itself, on a nine-species 12 x 10 x 8 lattice a few steps into an
  expanding flame (every term of the step is active: flow, diffusion
  velocities, reactions, the isotropy correction, the interdiffusion heat
  flux); likewise for ln A_k along a seeded direction (Richardson-
  extrapolated differences of the post-step states).  Three-gas lattices
  (constant heat capacities, kinematic viscosity) too.
* The gradient through time (lbm_heat_release_gradient, checkpoints with
  recomputation) of J = sum_{t<K} sum_nodes hdot^c on the 64 x 4 x 4
  periodic flame: against central differences (step 1e-6) of the GPU's own
  forward J, and against central differences of the FP64 oracle's J
  (tests/hrr_time_fd.py): 1e-4 relative.  Checkpoint spacing does not
  change the result (bit for bit), and the torch.autograd.Function returns
  the same gradients.
"""
import copy

import numpy as np
import pytest

import hrr_time_fd
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


def _state(s, L):
    import torch
    ptr = L.lbm_state_buffer(s.ctx)
    buf = s.pop[0] if s.pop[0].data_ptr() == ptr else s.pop[1]
    return buf.view(torch.float64)[: s.S * 27 * s.N].view(s.S, 27, s.N)


def _L_of(s, L, F, Trow, lam, with_objective):
    """<lam, step(F)> (+ J_t(F)) with the solver's forward step, from state F
    and Newton starting temperatures Trow; leaves s at state F."""
    _state(s, L).copy_(F)
    s.macro[: s.N].copy_(Trow)
    J = s.heat_release(gradients=False) if with_objective else 0.0
    s.step(1)
    val = float((lam * _state(s, L)).sum().item()) + J
    _state(s, L).copy_(F)                  # the step swapped buffers: put F back as the current state
    s.macro[: s.N].copy_(Trow)
    return val


def _solver_at(lbm, prob, F, Trow, log_A=None):
    mech = copy.deepcopy(prob.mech)
    if log_A is not None:
        mech.log_A = np.array(log_A, dtype=float)
    s = lbm.Solver(prob.lattice, prob.species, mech, precision=lbm.LBM_FP64)
    s.init(prob.init.X, prob.init.T, prob.init.u, prob.init.P)
    _state(s, lbm).copy_(F)
    s.macro[: s.N].copy_(Trow)
    return s


def _problems():
    # the expanding flame with 1 % of each of H, O and OH mixed in, so that
    # the chain reactions run from the first step
    sph = w.sphere3d_problem(shape=(12, 10, 8), radius=3.0)
    X = sph.init.X.copy()
    X[3:6] += 0.01
    sph.init.X = X / X.sum(axis=0, keepdims=True)
    return {"nine_species_sphere": (sph, 3),
            "three_gas_periodic": (w.small_periodic_problem(n=6, seed=3, M3_rate_A=20.0), 2)}


def _post(s, L, F, Trow, with_objective):
    """step(F) and J_t(F) (or 0) with the solver's forward step; leaves s at F."""
    _state(s, L).copy_(F)
    s.macro[: s.N].copy_(Trow)
    J = s.heat_release(gradients=False) if with_objective else 0.0
    s.step(1)
    out = _state(s, L).clone()
    _state(s, L).copy_(F)
    s.macro[: s.N].copy_(Trow)
    return out, J


@pytest.mark.parametrize("with_objective", [False, True])
@pytest.mark.parametrize("case", ["nine_species_sphere", "three_gas_periodic"])
def test_reverse_step_is_the_transposed_step(lbm, case, with_objective):
    import torch
    prob, warm = _problems()[case]
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    s.step(warm)
    F = _state(s, lbm).clone()
    Trow = s.macro[: s.N].clone()
    gen = torch.Generator(device=F.device).manual_seed(7)
    lam = torch.randn(F.shape, generator=gen, device=F.device, dtype=torch.float64)
    lam_out, dA = s.adjoint_step(lam, with_objective=with_objective)
    # the state and temperature row are left as they were
    assert torch.equal(_state(s, lbm), F) and torch.equal(s.macro[: s.N], Trow)
    delta = F * (2 * torch.rand(F.shape, generator=gen, device=F.device, dtype=torch.float64) - 1)
    eps = 1e-6
    Lp = _L_of(s, lbm, F + eps * delta, Trow, lam, with_objective)
    Lm = _L_of(s, lbm, F - eps * delta, Trow, lam, with_objective)
    fd = (Lp - Lm) / (2 * eps)
    ad = float((lam_out * delta).sum().item())
    assert ad != 0.0 and abs(fd - ad) <= 2e-6 * abs(ad), (fd, ad)
    # per set: the transpose restricted to one set's populations
    for st in range(s.S):
        d1 = torch.zeros_like(delta)
        d1[st] = delta[st]
        Lp = _L_of(s, lbm, F + eps * d1, Trow, lam, with_objective)
        Lm = _L_of(s, lbm, F - eps * d1, Trow, lam, with_objective)
        fd1 = (Lp - Lm) / (2 * eps)
        ad1 = float((lam_out[st] * delta[st]).sum().item())
        assert abs(fd1 - ad1) <= 1e-5 * abs(ad) + 2e-6 * abs(ad1), (st, fd1, ad1)
    # ln A_k along a seeded direction: the post-step states of two solvers
    # with ln A -+ h dth, differenced element by element before the
    # contraction with lam (the chemistry moves each population by far less
    # than the rounding of a sum over the whole state)
    # (one population's rounding, ~3e-17, over 2h would already be 3e-4 of
    # the nine-species signal at h = 1e-4, so a larger step with Richardson
    # extrapolation: error O(h^4))
    R = prob.mech.R
    dth = np.random.default_rng(11).uniform(-1, 1, R)

    def central(h):
        sp_ = _solver_at(lbm, prob, F, Trow, prob.mech.log_A + h * dth)
        sm_ = _solver_at(lbm, prob, F, Trow, prob.mech.log_A - h * dth)
        Fp, Jp = _post(sp_, lbm, F, Trow, with_objective)
        Fm, Jm = _post(sm_, lbm, F, Trow, with_objective)
        sp_.close()
        sm_.close()
        return float((lam * (Fp - Fm)).sum().item()) / (2 * h) + (Jp - Jm) / (2 * h)

    h = 2e-2
    fdA = (4.0 * central(h / 2) - central(h)) / 3.0
    adA = float(dA @ dth)
    s.close()
    assert adA != 0.0 and abs(fdA - adA) <= 2e-5 * abs(adA), (fdA, adA)


# ---------------------------------------------------------------------------
# Gradients through time
# ---------------------------------------------------------------------------
K_STEPS = 100


def _gpu_J(lbm, prob, steps, log_A=None, T0=None):
    mech = copy.deepcopy(prob.mech)
    if log_A is not None:
        mech.log_A = np.array(log_A, dtype=float)
    s = lbm.Solver(prob.lattice, prob.species, mech, precision=lbm.LBM_FP64)
    s.init(prob.init.X, prob.init.T if T0 is None else T0, None, prob.init.P)
    J = 0.0
    for _ in range(steps):
        J += s.heat_release(gradients=False)
        s.step(1)
    s.close()
    return J


@pytest.fixture(scope="module")
def flame64(lbm):
    prob = w.adjoint_flame_problem(nx=64)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    J, dA, dT0, _ = s.heat_release_gradient(K_STEPS, 16)
    s.close()
    return prob, J, dA, dT0.cpu().numpy()


def _sample_nodes(prob):
    nx = prob.lattice.nx
    xs = [0, 10, 49, 50, 51, 52, 60, 63]                     # cold, the hot slab's two fronts, hot
    return [x + nx * (1 + 4 * 2) for x in xs]


def _check_grad(got, ref, tol=1e-4):
    scale = np.abs(ref).max()
    assert scale > 0
    err = np.abs(got - ref)
    assert err.max() <= tol * scale, (err.max() / scale)
    big = np.abs(ref) > 1e-2 * scale
    assert np.all(err[big] <= tol * np.abs(ref[big])), (err[big] / np.abs(ref[big])).max()


def test_gradient_through_time_against_gpu_differences(lbm, flame64):
    prob, J, dA, dT0 = flame64
    assert abs(J - _gpu_J(lbm, prob, K_STEPS)) <= 1e-13 * abs(J)
    R = prob.mech.R
    fdA = np.empty(R)
    h = 1e-6
    for k in range(R):
        up = np.array(prob.mech.log_A, dtype=float)
        dn = up.copy()
        up[k] += h
        dn[k] -= h
        fdA[k] = (_gpu_J(lbm, prob, K_STEPS, log_A=up) - _gpu_J(lbm, prob, K_STEPS, log_A=dn)) / (2 * h)
    _check_grad(dA, fdA)
    nodes = _sample_nodes(prob)
    fdT = np.empty(len(nodes))
    for j, x in enumerate(nodes):
        hT = 1e-6 * prob.init.T[x]
        up = np.array(prob.init.T, dtype=float)
        dn = up.copy()
        up[x] += hT
        dn[x] -= hT
        fdT[j] = (_gpu_J(lbm, prob, K_STEPS, T0=up) - _gpu_J(lbm, prob, K_STEPS, T0=dn)) / (2 * hT)
    _check_grad(dT0[nodes], fdT)


def test_gradient_through_time_against_oracle_differences(orc, lbm, flame64):
    prob, J, dA, dT0 = flame64
    Jo = hrr_time_fd.objective(orc, prob, K_STEPS)
    assert abs(J - Jo) <= 1e-10 * abs(Jo), (J, Jo)
    fdA = hrr_time_fd.d_dlogA(orc, prob, K_STEPS, range(prob.mech.R))
    _check_grad(dA, fdA)
    nodes = _sample_nodes(prob)
    fdT = hrr_time_fd.d_dT0(orc, prob, K_STEPS, nodes)
    _check_grad(dT0[nodes], fdT)


def test_checkpoint_spacing_does_not_change_the_gradient(lbm, flame64):
    prob, J, dA, dT0 = flame64
    for every in (7, K_STEPS, 1):
        s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
        J2, dA2, dT2, _ = s.heat_release_gradient(K_STEPS, every)
        s.close()
        assert J2 == J and np.array_equal(dA2, dA) and np.array_equal(dT2.cpu().numpy(), dT0), every


def test_autograd_function_returns_the_gradients(lbm, flame64):
    import torch
    prob, J, dA, dT0 = flame64
    log_A = torch.tensor(prob.mech.log_A, dtype=torch.float64, requires_grad=True)
    T0 = torch.tensor(prob.init.T, dtype=torch.float64, device="cuda", requires_grad=True)
    out = lbm.heat_release_objective(log_A, T0, prob, K_STEPS, 16)
    assert float(out.item()) == J
    (2.0 * out).backward()
    assert np.array_equal(log_A.grad.numpy(), 2.0 * dA)
    assert np.array_equal(T0.grad.cpu().numpy(), 2.0 * dT0)


def test_adjoint_rejects_unsupported_contexts(lbm):
    import torch
    prob = w.flame1d_problem(nx=32)                          # ghost-node x faces
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    lam = torch.zeros((s.S, 27, s.N), dtype=torch.float64, device="cuda")
    ws = torch.empty(lbm.lbm_adjoint_workspace_bytes(s.ctx, 0, 1), dtype=torch.uint8, device="cuda")
    assert lbm.lbm_adjoint_step(s.ctx, lam.data_ptr(), torch.empty_like(lam).data_ptr(), None, True,
                                ws.data_ptr(), ws.numel()) == lbm.LBM_ERR_UNSUPPORTED
    s.close()
    prob = w.sphere3d_problem(shape=(8, 6, 5), radius=2.0)
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_MIXED)
    J = np.zeros(1)
    wsb = lbm.lbm_adjoint_workspace_bytes(s.ctx, 4, 2)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert lbm.lbm_heat_release_gradient(s.ctx, 4, 2, J, None, None, ws.data_ptr(), wsb) == lbm.LBM_ERR_UNSUPPORTED
    s.close()
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    assert lbm.lbm_heat_release_gradient(s.ctx, 4, 2, J, None, None, ws.data_ptr(), 1024) == lbm.LBM_ERR_ARG
    assert lbm.lbm_heat_release_gradient(s.ctx, 0, 2, J, None, None, ws.data_ptr(), wsb) == lbm.LBM_ERR_ARG
    assert lbm.lbm_adjoint_step(s.ctx, lam.data_ptr(), lam.data_ptr(), None, True, ws.data_ptr(),
                                wsb) == lbm.LBM_ERR_ARG
    s.close()
