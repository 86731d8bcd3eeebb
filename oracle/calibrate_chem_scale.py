"""Calibrates the global rate scale of the nine-species synthetic mechanism.

Test/input infrastructure, run by hand: it prints the largest rate scale for
which the explicit source term of the species lattice Boltzmann equation
(Eq. (finalNumericalEquations), delta_t * rho_dot_a) stays well resolved.
The printed value is frozen as MECH9_CHEM_SCALE in workload/configs.py.

Criterion, over temperatures 300-2500 K and a set of compositions (unburnt
phi = 0.5 .. 3 mixtures, and partially burnt mixtures carrying radicals):
  * the self-consumption frequency |d rho_dot_a / d rho_a| <= 0.2 per step
    for every species (explicit-Euler stability of the stiffest species);
  * |rho_dot_a| <= 0.02 rho per step.
Rates are linear in the scale, so one evaluation at a unit scale suffices.
Only the oracle's production-rate routine is used.

    python -m oracle.calibrate_chem_scale
"""
from __future__ import annotations

import numpy as np

import oracle
import workload.configs as wc
from workload.problem import LatticeSpec


def states():
    mixes = []
    for phi in (0.5, 1.0, 2.0, 3.0):
        mixes.append(np.maximum(wc.phi_mixture(phi), 1e-12))
    burnt = np.array([0.05, 0.02, 0.25, 0.01, 0.01, 0.01, 0.005, 0.005, 0.64])
    half = 0.5 * (np.maximum(wc.phi_mixture(1.0), 1e-12) + burnt)
    mixes += [burnt, half]
    for X in mixes:
        X = X / X.sum()
        for T in np.linspace(300.0, 2500.0, 23):
            yield X, T


def main(scale: float = 1.0):
    sp, mech = wc.mech9(chem_scale=scale)
    o = oracle.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    worst_J = 0.0
    worst_w = 0.0
    for X, T in states():
        m = float(np.dot(X, sp.W))
        rho = mech.P0 / (sp.r_lat / m * T)
        rho_a = rho * X * sp.W / m
        w0 = o.rates(rho_a, T)
        worst_w = max(worst_w, float(np.abs(w0).max() / rho))
        for a in range(sp.M):
            eps = 1e-6
            r1 = rho_a.copy()
            r1[a] *= 1.0 + eps
            J = (o.rates(r1, T)[a] - w0[a]) / (rho_a[a] * eps)
            worst_J = max(worst_J, abs(J))
    s = scale * min(0.2 / worst_J, 0.02 / worst_w)
    print(f"max |J_aa| = {worst_J:.3e}, max |rho_dot|/rho = {worst_w:.3e} at scale {scale:.3e}")
    print(f"chem_scale = {s:.3e}")
    return s


if __name__ == "__main__":
    main()
