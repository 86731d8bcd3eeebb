"""Pins of the oracle's flame diagnostics of the circular expanding flame
(Sec. 5b): the isoline means of Eq. (rmean) and the displacement speed of
Eq. (sd) with S_a = S_d + u . n.

* isoline of a radial field: a circle of radius r0 -- its length tends to
  2 pi r0, the mean radius to r0 and the mean of r^2 to r0^2, at second
  order in the lattice spacing; a perturbed circle
  R(theta) = R0 (1 + A0 cos(4 n0 theta)) (Eq. (cflamePerturbation)): the
  mean radius is the length-weighted one of Eq. (rmean), against a dense
  quadrature of the curve;
* S_d on a state at rest with uniform composition and a temperature sine
  T0 + a sin(k x) (constant relaxation, so that lambda is uniform): the
  lattice gradient d_h sin(kx) = sin(k) cos(kx) and its nested application
  give
      S_d = (hdot^c - lambda sin^2(k) sin(kx)) / (rho C_p |sin(k) cos(kx)|),
  with hdot^c = 0 without reactions, and the closed form of the
  single-step three-gas heat release (q Delta H) with them; u = 0, so
  S_a = S_d.
"""
import math

import numpy as np
import pytest

import workload as w
from workload.problem import BC_PERIODIC, InitFields, LatticeSpec, Problem


def _plane_oracle(orc, n):
    p = w.sphere3d_problem(shape=(n, n, 1), radius=2.0)
    return orc.Oracle.from_problem(p), p


@pytest.mark.parametrize("n,r0", [(64, 16.0), (128, 32.0)])
def test_isoline_of_a_circle(orc, n, r0):
    o, _ = _plane_oracle(orc, n)
    idx = np.arange(n * n)
    x, y = idx % n, idx // n
    c = n / 2 - 0.3
    r2 = (x - c) ** 2 + (y - c) ** 2
    T = 300 + 1000 * np.exp(-r2 / (r0 * r0))
    A, R, mr2 = o.isoline_means(T, 300 + 1000 * math.exp(-1.0), c, c, [r2])
    tol = 2e-4 * (64 / n) ** 2
    assert abs(A / (2 * math.pi * r0) - 1) < tol
    assert abs(R / r0 - 1) < 2 * tol
    assert abs(mr2 / r0 ** 2 - 1) < 8 * tol


def test_isoline_of_a_perturbed_circle_is_length_weighted(orc):
    n, R0, A0, n0 = 192, 60.0, 0.1, 4
    o, _ = _plane_oracle(orc, n)
    idx = np.arange(n * n)
    x, y = idx % n, idx // n
    c = n / 2 - 0.37
    th = np.arctan2(y - c, x - c)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2)
    T = R0 * (1 + A0 * np.cos(4 * n0 * th)) - r            # zero on the curve, positive inside
    A, R = o.isoline_means(T, 0.0, c, c)[:2]
    t = np.linspace(0, 2 * np.pi, 200001)[:-1]
    Rt = R0 * (1 + A0 * np.cos(4 * n0 * t))
    dRt = -R0 * A0 * 4 * n0 * np.sin(4 * n0 * t)
    ds = np.sqrt(Rt ** 2 + dRt ** 2)                        # arc length per unit angle
    A_ref = ds.mean() * 2 * np.pi
    R_ref = (Rt * ds).mean() / ds.mean()
    assert abs(A / A_ref - 1) < 4e-3, (A, A_ref)           # polygon through a wavy curve: a little short
    assert abs(R / R_ref - 1) < 5e-4, (R, R_ref)
    assert abs(R_ref / Rt.mean() - 1) > 2e-3                  # the weighting matters here


def _sine_state(orc, rate_A, n=48, a=0.2):
    """Uniform composition at rest with T = 2 + a sin(k x) in the state a
    collision sees: every node's equilibrium (Eqs. (feq), (feqmix), (gieq))
    stored pre-shifted, direction i at x - c_i, so that the pull returns
    exactly the node's own equilibrium."""
    sp, mech = w.mech3(rate_A=rate_A if rate_A > 0 else 1.0)
    if rate_A == 0.0:
        mech.log_A[:] = -800.0
    # constant relaxation: lambda = (1/omega_1 - 1/2) P C_p is uniform at
    # uniform pressure and composition
    from workload.problem import VISC_RELAXATION
    sp.visc_model, sp.nu = VISC_RELAXATION, 0.8
    lat = LatticeSpec(n, 2, 1, BC_PERIODIC)
    N = lat.n_nodes
    k = 2 * math.pi / n
    x = np.arange(N) % n
    yy = (np.arange(N) // n) % 2
    T = 2.0 + a * np.sin(k * x)
    X0 = np.array([0.3, 0.5, 0.2])
    P = sp.r_lat / 23.4
    m = X0 @ sp.W
    rho = P / (sp.r_lat / m * T)
    rho_a = rho[None, :] * (X0 * sp.W / m)[:, None]
    prob = Problem("sine", lat, sp, mech, InitFields(X=np.tile(X0[:, None], (1, N)), T=T, u=None, P=P))
    o = orc.Oracle.from_problem(prob)
    pop = np.empty((N, 4, 27))
    for nd in range(N):
        eq = o.equilibrium_sets(rho_a[:, nd], np.zeros(3), T[nd])
        for i in range(27):
            cx, cy = orc.C_VEL[i][0], orc.C_VEL[i][1]
            src = (x[nd] - cx) % n + n * ((yy[nd] - cy) % 2)
            pop[src, :, i] = eq[:, i]
    o.set_pop(pop)
    o.set_T(T)
    return o, prob, k, x, a, rho_a, T


@pytest.mark.parametrize("rate_A", [0.0, 50.0])
def test_displacement_speed_closed_form(orc, rate_A):
    o, prob, k, x, a, rho_a, Tf = _sine_state(orc, rate_A)
    Sd, Sa = o.flame_speeds()
    sp = prob.species
    one = orc.Oracle(LatticeSpec(1, 1, 1, BC_PERIODIC), sp, prob.mech)
    pick = np.flatnonzero(np.abs(np.cos(k * x)) > 0.3)[:40]
    cp = sp.cp_R * sp.r_lat / sp.W
    refs = []
    for nd in pick:
        T, rho = Tf[nd], rho_a[:, nd].sum()
        Y = rho_a[:, nd] / rho
        Rm = sp.r_lat * (Y / sp.W).sum()
        P = rho * Rm * T
        Cp = float(Y @ cp)
        lam = one.transport(Y, T, P)["nup1"] * P * Cp
        # three-gas single step R + O -> P: hdot = q (W_R H_R + W_O H_O - W_P H_P)
        W = sp.W
        H = sp.h_form + cp * (T - sp.T0)
        c = rho_a[:, nd] / W
        q = math.exp(prob.mech.log_A[0]) * math.exp(-prob.mech.theta[0] / T) * c[0] * c[1]
        hdot = q * (W[0] * H[0] + W[1] * H[1] - W[2] * H[2])
        gT = a * math.sin(k) * math.cos(k * x[nd])
        lapT = -a * math.sin(k) ** 2 * math.sin(k * x[nd])
        refs.append((hdot + lam * lapT) / (rho * Cp * abs(gT)))
    refs = np.array(refs)
    scale = np.abs(refs).max()
    assert np.abs(Sd[pick] - refs).max() <= 1e-9 * scale
    assert np.abs(Sa[pick] - Sd[pick]).max() <= 1e-12 * scale    # at rest: S_a = S_d
    if rate_A > 0:
        assert np.abs(hdot) > 1e-3 * np.abs(lam * lapT)               # the reaction term is really there
