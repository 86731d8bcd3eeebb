"""Pins of the oracle's time-integrated heat release (tests/hrr_time_fd.py),
the objective whose gradients the adjoint of the step computes, against a
homogeneous reactor written out directly.

On a single periodic node at rest the step is the forward Euler update of
the production rates (Eq. (fsource)) with the temperature of constant heat
capacities in closed form (Eqs. (specHa), (temperature)); the node starts
at rho = P / (R T0) with the given mole fractions.  So
  J(A, T0) = sum_{t<K} -sum_a H_a(T^t) rho_dot_a^t
is a short scalar recursion, and its central differences in ln A and T0
must equal the oracle's.  A wrong time window, a dropped enthalpy, or an
initial state at the wrong density fails here."""
import math

import numpy as np

import hrr_time_fd
import workload as w
from workload.problem import BC_PERIODIC, InitFields, LatticeSpec, Problem


def _reactor_problem(A, T0=3.0):
    sp, mech = w.mech3(rate_A=A)
    X = np.array([[0.45], [0.45], [0.10]])
    P = sp.r_lat / 23.4
    return Problem("reactor", LatticeSpec(1, 1, 1, BC_PERIODIC), sp, mech,
                   InitFields(X=X, T=np.array([T0]), u=None, P=P))


def _reactor_J(prob, steps, log_A=None, T0=None):
    """The same objective by the scalar recursion (three-gas thermodynamics:
    c_p/R = 3.5, H^0 = 0, 0, -30 R_P T0; R + O -> P with q = A e^{-10/T} c_R c_O)."""
    sp = prob.species
    W = np.array(sp.W, dtype=float)
    Ra = sp.r_lat / W
    Tref = sp.T0
    U0 = np.array(sp.h_form, dtype=float) - Ra * Tref
    cv = (np.array(sp.cp_R) - 1.0) * Ra
    A = math.exp(prob.mech.log_A[0] if log_A is None else log_A[0])
    T = prob.init.T[0] if T0 is None else T0[0]
    X = prob.init.X[:, 0]
    m = X @ W
    rho = prob.init.P / (sp.r_lat / m * T)
    rho_a = rho * X * W / m
    E = (rho_a / rho) @ (U0 + cv * (T - Tref))
    J = 0.0
    for _ in range(steps):
        Y = rho_a / rho_a.sum()
        T = Tref + (E - Y @ U0) / (Y @ cv)
        H = U0 + cv * (T - Tref) + Ra * T
        q = A * math.exp(-prob.mech.theta[0] / T) * (rho_a[0] / W[0]) * (rho_a[1] / W[1])
        rdot = np.array([-W[0], -W[1], W[2]]) * q
        J += -H @ rdot
        rho_a = rho_a + rdot
    return J


def test_time_objective_of_the_homogeneous_reactor(orc):
    prob = _reactor_problem(400.0)
    for K in (1, 5, 40):
        Jo = hrr_time_fd.objective(orc, prob, K)
        Jr = _reactor_J(prob, K)
        assert Jr != 0.0
        assert abs(Jo - Jr) <= 1e-11 * abs(Jr), (K, Jo, Jr)


def test_time_objective_differences_of_the_homogeneous_reactor(orc):
    prob = _reactor_problem(400.0)
    K = 40
    gA = hrr_time_fd.d_dlogA(orc, prob, K, [0])[0]
    gT = hrr_time_fd.d_dT0(orc, prob, K, [0])[0]
    h = 1e-6
    la = np.array(prob.mech.log_A, dtype=float)
    rA = (_reactor_J(prob, K, log_A=la + h) - _reactor_J(prob, K, log_A=la - h)) / (2 * h)
    hT = 1e-6 * prob.init.T[0]
    rT = (_reactor_J(prob, K, T0=prob.init.T + hT) - _reactor_J(prob, K, T0=prob.init.T - hT)) / (2 * hT)
    assert abs(gA - rA) <= 1e-6 * abs(rA), (gA, rA)
    assert abs(gT - rT) <= 1e-6 * abs(rT), (gT, rT)
