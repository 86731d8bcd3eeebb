"""Pins of the oracle's mixture-averaged transport (the stand-in for the
coefficients the paper takes from Cantera, Sec. 3 after Eq. (lambda)):
Wilke's mixing rule for the viscosity, the modified Eucken relation and the
Mathur-Tondon-Saxena average for the conductivity, and binary diffusivities
D_ab (T/T_tr)^{D_exp} (P_tr/P); and of their use in the relaxation rates
(Eqs. (mu), (lambda), (tauab)).

* a pure species has the mixture viscosity mu_a and conductivity
  lambda_a = mu_a (C_p,a + 5/4 R_a) (Phi_aa = 1, the average of equal means);
* a mixture of two copies of one species has that species' coefficients at
  every composition (Phi_ab = 1);
* Wilke's coefficients obey Phi_ba = Phi_ab (mu_b W_a) / (mu_a W_b): read off
  from the dilute-limit slopes of the binary viscosity,
  d mu/d X_2 |_{X_2=0} = -mu_1 Phi_12 + mu_2 / Phi_21 (and 1 <-> 2);
* a transverse shear wave in a uniform mixture decays at mu / rho k^2
  (Eq. (mu)) with the oracle's own mixture viscosity;
* a binary composition mode at rest decays at D_12(T) k^2 with
  D_12(T) = D_12 (T/T_tr)^{D_exp} at the reference pressure (Eq. (tauab)).
"""
import copy
import math

import numpy as np
import pytest

import workload as w
from workload.problem import BC_PERIODIC, LatticeSpec, TRANSPORT_MIXTURE_AVERAGED


def _species3(mu0, mu_exp, W=(2.0, 32.0, 34.0)):
    sp, mech = w.mech3()
    sp = copy.deepcopy(sp)
    sp.W = np.array(W, dtype=float)
    sp.transport = TRANSPORT_MIXTURE_AVERAGED
    sp.mu0 = np.array(mu0, dtype=float)
    sp.mu_exp = np.array(mu_exp, dtype=float)
    sp.T_tr, sp.P_tr, sp.D_exp = 1.0, 0.02, 1.5
    return sp, mech


def _one(orc, sp, mech):
    return orc.Oracle(LatticeSpec(1, 1, 1, BC_PERIODIC), sp, mech)


def test_pure_species_and_identical_species(orc):
    sp, mech = _species3([0.01, 0.03, 0.02], [0.6, 0.7, 0.5])
    o = _one(orc, sp, mech)
    T, P = 1.7, 0.03
    for a in range(3):
        Y = np.zeros(3)
        Y[a] = 1.0
        t = o.transport(Y, T, P)
        mu_a = sp.mu0[a] * (T / sp.T_tr) ** sp.mu_exp[a]
        R_a = sp.r_lat / sp.W[a]
        cv_a = o.thermo(T)["Cv"][a]
        assert abs(t["mu"] - mu_a) <= 1e-15 * mu_a
        assert abs(t["lam"] - mu_a * (cv_a + R_a + 1.25 * R_a)) <= 1e-14 * t["lam"]
        assert abs(t["nup"] - mu_a / P) <= 1e-14 * t["nup"]
    # two copies of species 0 (same W, viscosity law): coefficients of species 0
    sp2, mech2 = _species3([0.01, 0.01, 0.02], [0.6, 0.6, 0.5], W=(2.0, 2.0, 34.0))
    o2 = _one(orc, sp2, mech2)
    ref = o2.transport(np.array([1.0, 0.0, 0.0]), T, P)
    for x in (0.1, 0.5, 0.83):
        t = o2.transport(np.array([x, 1 - x, 0.0]), T, P)
        assert abs(t["mu"] - ref["mu"]) <= 1e-14 * ref["mu"]
        assert abs(t["lam"] - ref["lam"]) <= 1e-14 * ref["lam"]


def test_wilke_coefficients_obey_their_symmetry(orc):
    """Phi_12 and Phi_21 from the dilute-limit slopes of mu(X_2) in a binary
    of very unequal molar masses and viscosities; then
    Phi_21 mu_1 W_2 = Phi_12 mu_2 W_1 (a swapped mass ratio or a wrong power
    of the viscosity ratio breaks it)."""
    sp, mech = _species3([0.004, 0.03, 0.02], [0.6, 0.6, 0.6], W=(2.0, 32.0, 34.0))
    o = _one(orc, sp, mech)
    T, P = 1.0, 0.02
    W1, W2 = sp.W[0], sp.W[1]

    def mu_of_X2(x2):                 # X_2 = x2, X_1 = 1 - x2, X_3 = 0
        X = np.array([1 - x2, x2, 0.0])
        Y = X * sp.W / (X @ sp.W)
        return o.transport(Y, T, P)["mu"]

    h = 1e-6
    s0 = (mu_of_X2(h) - mu_of_X2(-h)) / (2 * h)                    # at X_2 = 0
    s1 = (mu_of_X2(1 + h) - mu_of_X2(1 - h)) / (2 * h)              # at X_1 = 0 (slope in X_2)
    mu1, mu2 = sp.mu0[0], sp.mu0[1]
    # s0 = -mu1 Phi12 + mu2 / Phi21 and s1 = mu2 Phi21 - mu1 / Phi12.  With the
    # symmetry Phi21 = Phi12 mu2 W1 / (mu1 W2), s0 fixes Phi12 through
    # mu1 Phi12^2 + s0 Phi12 - mu1 W2 / W1 = 0; the symmetry then predicts s1.
    P12 = (-s0 + math.sqrt(s0 * s0 + 4 * mu1 * mu1 * W2 / W1)) / (2 * mu1)
    P21 = P12 * mu2 * W1 / (mu1 * W2)
    s1_pred = mu2 * P21 - mu1 / P12
    assert abs(s1 - s1_pred) <= 1e-6 * abs(s1), (s1, s1_pred)
    assert abs(P21 / P12 - 1.0) > 0.3                                # far from the trivial case


def _mode_amplitude(field, nx):
    return abs(np.fft.rfft(field[:nx])[1]) * 2 / nx


def test_shear_wave_decays_with_the_mixture_viscosity(orc):
    nx = 64
    sp, mech = _species3([0.01, 0.03, 0.02], [0.6, 0.7, 0.5])
    mech = copy.deepcopy(mech)
    mech.log_A[:] = -800.0
    X0 = np.array([0.3, 0.5, 0.2])
    rho0 = 1.0
    m = X0 @ sp.W
    P = rho0 * sp.r_lat / m * 1.0
    sp.P_tr = P
    # 1/omega - 1/2 = mu / P near 0.8 in this mixture
    o1 = _one(orc, sp, mech)
    Y0 = X0 * sp.W / m
    scale = 0.8 / o1.transport(Y0, 1.0, P)["nup"]
    sp.mu0 = sp.mu0 * scale
    lat = LatticeSpec(nx, 1, 1, BC_PERIODIC)
    k = 2 * math.pi / nx
    u = np.zeros((3, nx))
    u[1] = 1e-3 * np.sin(k * np.arange(nx))
    o = orc.Oracle(lat, sp, mech)
    o.init(np.tile(X0[:, None], (1, nx)), np.ones(nx), u, P)
    amps = {}
    for t in range(1001):
        if t:
            assert o.step(1) == 0
        if t in (200, 1000):
            mm = o.moments()
            amps[t] = _mode_amplitude(mm["rhou"][1] / mm["rho"], nx)
    rate = math.log(amps[200] / amps[1000]) / 800
    nu = _one(orc, sp, mech).transport(Y0, 1.0, P)["mu"] / rho0
    assert abs(rate / (nu * k * k) - 1) < 0.02, (rate, nu * k * k)


@pytest.mark.parametrize("T", [1.0, 1.6])
def test_binary_diffusion_follows_the_temperature_law(orc, T):
    """Equal molar masses at rest, uniform T and P = P_tr: a Y_1 mode decays
    at D_12 (T/T_tr)^{D_exp} k^2."""
    nx = 64
    D = 0.01
    W0 = 20.0
    r_lat = 0.4
    R = r_lat / W0
    from workload.problem import MechanismSpec, SpeciesSpec, THERMO_CONST_CP, VISC_KINEMATIC
    sp = SpeciesSpec(names=["A", "B"], W=np.array([W0, W0]), thermo=THERMO_CONST_CP, cp_R=np.full(2, 3.5),
                     h_form=np.zeros(2), T0=1.0, poly7=np.zeros((2, 7)), D=np.full((2, 2), D), nu=R, Pr=0.71,
                     r_lat=r_lat, elements=np.eye(2, dtype=np.int32), element_names=["A", "B"],
                     visc_model=VISC_KINEMATIC, transport=TRANSPORT_MIXTURE_AVERAGED,
                     mu0=np.full(2, 0.8 * R), mu_exp=np.full(2, 0.0), T_tr=1.0, D_exp=1.5, P_tr=R)
    mech = MechanismSpec(nu_f=np.zeros((0, 2), np.int32), nu_r=np.zeros((0, 2), np.int32), log_A=np.zeros(0),
                         b=np.zeros(0), theta=np.zeros(0), rtype=np.zeros(0, np.int32), eff=np.zeros((0, 2)),
                         low=np.zeros((0, 3)), reversible=np.zeros(0, np.int32), T_ref=1.0, P0=1.0)
    lat = LatticeSpec(nx, 1, 1, BC_PERIODIC)
    x = np.arange(nx)
    k = 2 * math.pi / nx
    X1 = 0.5 + 0.02 * np.sin(k * x)
    o = orc.Oracle(lat, sp, mech)
    o.init(np.stack([X1, 1 - X1]), np.full(nx, T), None, R)          # P = P_tr
    amps = []
    t1 = int(round(0.4 / (D * T ** 1.5 * k * k)))
    for t in range(t1 + 1):
        if t:
            assert o.step(1) == 0
        if t in (t1 // 5, t1):
            amps.append(_mode_amplitude(o.moments()["Y"][0], nx))
    rate = math.log(amps[0] / amps[1]) / (t1 - t1 // 5)
    assert abs(rate / (D * T ** 1.5 * k * k) - 1) < 0.02, (rate, D * T ** 1.5 * k * k)
