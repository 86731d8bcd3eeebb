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
