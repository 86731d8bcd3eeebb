"""Pins of the oracle's heat release rate hdot^c = -sum_a H_a rho_dot_a
(Sec. 5b) and of its finite-difference gradient (tests/hrr_fd.py), against
what the mathematics fixes for the single irreversible step R + O -> P of
the three-gas mechanism:

  q = A exp(-theta/T) c_R c_O,   H_a = h_a^0 + c_p,a (T - T0)   (constant c_p),
  hdot^c = q (W_R H_R + W_O H_O - W_P H_P),
  d hdot^c/d ln A = hdot^c,
  d hdot^c/dT = q (theta/T^2) dH + q (W_R c_p,R + W_O c_p,O - W_P c_p,P),
  d hdot^c/d rho_R = hdot^c / rho_R,  d hdot^c/d rho_P = 0.

A dropped enthalpy term, a wrong sign or a swapped species fails one of
these."""
import math

import numpy as np
import pytest

import workload as w
import hrr_fd


def _closed_form(sp, mech, rho_a, T):
    W = sp.W
    Ra = sp.r_lat / W
    H = sp.h_form + sp.cp_R * Ra * (T - sp.T0)
    cp = sp.cp_R * Ra
    A, theta = math.exp(mech.log_A[0]), mech.theta[0]
    c = rho_a / W
    q = A * math.exp(-theta / T) * c[0] * c[1]
    dH = W[0] * H[0] + W[1] * H[1] - W[2] * H[2]
    dcp = W[0] * cp[0] + W[1] * cp[1] - W[2] * cp[2]
    return q * dH, q * dH, q * theta / T ** 2 * dH + q * dcp, np.array([q * dH / rho_a[0], q * dH / rho_a[1], 0.0])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_heat_release_single_step_closed_form(orc, seed):
    sp, mech = w.mech3()
    rng = np.random.default_rng(seed)
    rho_a = rng.uniform(0.05, 0.6, 3)
    T = rng.uniform(0.8, 4.0)
    o = hrr_fd.oracle_of(orc, sp, mech)
    h, dA, dT, drho = _closed_form(sp, mech, rho_a, T)
    assert h > 0                                          # P lies 30 R_P T0 below R + O
    assert abs(o.heat_release(rho_a, T) - h) <= 1e-13 * abs(h)
    R1, T1 = rho_a[:, None], np.array([T])
    assert abs(hrr_fd.d_dlogA(orc, sp, mech, R1, T1)[0, 0] - dA) <= 1e-8 * abs(dA)
    assert abs(hrr_fd.d_dT(o, R1, T1)[0] - dT) <= 1e-7 * abs(dT)
    fd = hrr_fd.d_drho(o, R1, T1)[:, 0]
    assert np.all(np.abs(fd - drho) <= 1e-7 * np.abs(drho).max())


def test_heat_release_vanishes_without_reactions(orc):
    sp, mech = w.mech3()
    mech.log_A[:] = -800.0
    o = hrr_fd.oracle_of(orc, sp, mech)
    assert o.heat_release(np.array([0.3, 0.4, 0.3]), 2.0) == 0.0


def test_node_states_cover_absent_and_trace_species():
    rho_a, T = w.node_states(9, 400, seed=3)
    assert rho_a.shape == (9, 400) and T.shape == (400,)
    assert (rho_a == 0).any() and (rho_a > 0).sum(axis=0).min() >= 1
    Y = rho_a / rho_a.sum(axis=0)
    assert Y[Y > 0].min() < 1e-5 and T.min() >= 700.0 and T.max() <= 2600.0


def test_energy_population_gradient_is_the_temperature_derivative(orc):
    """Perturbing an energy population g_i(x) moves only rho E of the node
    n = x + c_i that pulls it, hence only its temperature, by
    dT = d(rho E) / (rho C_v): the finite-difference population gradient
    (tests/hrr_fd.py) equals d hdot^c/dT / (rho C_v) at n."""
    prob = w.sphere3d_problem(shape=(6, 5, 4), radius=1.5)
    o = orc.Oracle.from_problem(prob)
    assert o.step(1) == 0
    one = hrr_fd.oracle_of(orc, prob.species, prob.mech)
    m = o.moments()
    M, nx, ny, nz = prob.species.M, 6, 5, 4
    x0, y0, z0 = 3, 2, 2
    for i in (13, 14, 22):          # c = (0,0,0), (1,0,0), (0,0,1); i = (cx+1) + 3 (cy+1) + 9 (cz+1)
        cx, cy, cz = i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1
        x = x0 + nx * (y0 + ny * z0)
        n = (x0 + cx) % nx + nx * ((y0 + cy) % ny + ny * ((z0 + cz) % nz))
        fd = hrr_fd.d_dpop(o, one, [(x, M, i)])[0]
        rho_a, T = m["rho_a"][:, n], m["T"][n]
        rho = rho_a.sum()
        Cv = float((rho_a / rho * one.thermo(T)["Cv"]).sum())
        ref = hrr_fd.d_dT(one, rho_a[:, None], np.array([T]))[0] / (rho * Cv)
        assert ref != 0.0 and abs(fd - ref) <= 1e-5 * abs(ref), (i, fd, ref)
