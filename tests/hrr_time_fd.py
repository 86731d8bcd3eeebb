"""The oracle-side objective of the gradients through time and its
central finite differences (never of the CUDA path):

  J(ln A, T0) = sum_{t=0}^{K-1} sum_nodes hdot^c(state step t's collision sees)

with hdot^c = -sum_a H_a rho_dot_a (Sec. 5b), the oracle initialised at
the problem's mole fractions and pressure, zero velocity and temperatures
T0.  Steps: ln A_k by h = 1e-6; T0 at a node by 1e-6 of its value."""
import copy

import numpy as np


def objective(orc, prob, steps, log_A=None, T0=None):
    mech = copy.deepcopy(prob.mech)
    if log_A is not None:
        mech.log_A = np.array(log_A, dtype=float)
    o = orc.Oracle(prob.lattice, prob.species, mech)
    T = prob.init.T if T0 is None else T0
    assert o.init(prob.init.X, T, None, prob.init.P) == 0
    J = 0.0
    for _ in range(steps):
        J += o.total_heat_release()
        assert o.step(1) == 0
    return J


def d_dlogA(orc, prob, steps, ks, h=1e-6):
    out = []
    for k in ks:
        up = np.array(prob.mech.log_A, dtype=float)
        dn = up.copy()
        up[k] += h
        dn[k] -= h
        out.append((objective(orc, prob, steps, log_A=up) - objective(orc, prob, steps, log_A=dn)) / (2 * h))
    return np.array(out)


def d_dT0(orc, prob, steps, nodes, rel=1e-6):
    out = []
    for x in nodes:
        h = rel * prob.init.T[x]
        up = np.array(prob.init.T, dtype=float)
        dn = up.copy()
        up[x] += h
        dn[x] -= h
        out.append((objective(orc, prob, steps, T0=up) - objective(orc, prob, steps, T0=dn)) / (2 * h))
    return np.array(out)
