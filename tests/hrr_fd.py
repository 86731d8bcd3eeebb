"""The oracle-side gradient of the heat release rate hdot^c = -sum_a H_a
rho_dot_a (Sec. 5b): central finite differences of the oracle's own
function, never of the CUDA path.

Steps: ln A_k by h = 1e-6 (hdot^c depends on A_k through exp(ln A_k) only);
T by 1e-6 T; each density by 1e-6 times the node's total density (hdot^c is
a polynomial of degree at most three in each density at fixed T, except
through a falloff factor, so the truncation error is of order h^2).
"""
import copy

import numpy as np

from workload.problem import LatticeSpec


def oracle_of(orc, species, mech):
    return orc.Oracle(LatticeSpec(1, 1, 1), species, mech)


def hdot(o, rho_a, T):
    """hdot^c at each of n states (rho_a [M, n], T [n])."""
    return np.array([o.heat_release(rho_a[:, i], T[i]) for i in range(T.size)])


def d_dT(o, rho_a, T, rel=1e-6):
    h = rel * T
    return (hdot(o, rho_a, T + h) - hdot(o, rho_a, T - h)) / (2 * h)


def d_drho(o, rho_a, T, rel=1e-6):
    M, n = rho_a.shape
    h = rel * rho_a.sum(axis=0)
    out = np.empty((M, n))
    for b in range(M):
        up, dn = rho_a.copy(), rho_a.copy()
        up[b] += h
        dn[b] -= h
        out[b] = (hdot(o, up, T) - hdot(o, dn, T)) / (2 * h)
    return out


def d_dlogA(orc, species, mech, rho_a, T, h=1e-6):
    """[R, n]: d hdot^c / d ln A_k at each state."""
    out = np.empty((mech.R, T.size))
    for k in range(mech.R):
        hi, lo = copy.deepcopy(mech), copy.deepcopy(mech)
        hi.log_A = np.array(mech.log_A, dtype=float)
        lo.log_A = np.array(mech.log_A, dtype=float)
        hi.log_A[k] += h
        lo.log_A[k] -= h
        out[k] = (hdot(oracle_of(orc, species, hi), rho_a, T) - hdot(oracle_of(orc, species, lo), rho_a, T)) / (2 * h)
    return out


def hdot_of_state(o, one):
    """hdot^c at every node of the oracle lattice o's current state (its
    moments and Newton temperatures), evaluated by the one-node oracle one."""
    m = o.moments()
    assert m["status"] == 0
    return hdot(one, m["rho_a"], m["T"])


def d_dpop(o, one, samples, rel=1e-6):
    """dJ/dF at samples (node, set, direction) of o's state, J = sum of
    hdot^c: central differences with a step of rel times the largest
    population of that set at that node.  Only the node that pulls the
    perturbed population changes, so the per-node differences are summed."""
    pop = o.get_pop()
    out = []
    for (x, s, i) in samples:
        h = rel * np.abs(pop[x, s]).max()
        p1 = pop.copy()
        p1[x, s, i] += h
        o.set_pop(p1)
        hp = hdot_of_state(o, one)
        p1[x, s, i] -= 2 * h
        o.set_pop(p1)
        hm = hdot_of_state(o, one)
        out.append(float((hp - hm).sum() / (2 * h)))
    o.set_pop(pop)
    return np.array(out)
