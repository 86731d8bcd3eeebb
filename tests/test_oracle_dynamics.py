"""Pins of the oracle's time stepping against what the paper fixes (no GPU).

* exact conservation of total mass, species mass up to the reaction source,
  element mass, momentum and total energy with formation enthalpy
  (Eqs. (sumRhoDot), (finalNumericalEquations), (f), (g), (strongest))
* homogeneous reactor = forward Euler of the production rates with the
  closed-form temperature of constant heat capacities (Eqs. (specHa),
  (temperature), (fsource))
* uniform rest state and uniform flow are fixed points
* Fick's law for a binary mixture of equal molar masses (Eq. (constit2))
* shear viscosity and thermal diffusivity from the relaxation rates
  (Eqs. (mu), (lambda))
* sound attenuation with the paper's bulk viscosity, which holds only with
  the isotropy correction X of Eq. (Xalpha)
* slaving of the last species (Eq. (strongest))
"""
import math

import numpy as np
import pytest

import workload as w
from workload.problem import (BC_PERIODIC, LatticeSpec, MechanismSpec, InitFields,
                              Problem, SpeciesSpec, THERMO_CONST_CP, VISC_KINEMATIC)


def _reacting_config1(nx=16, ny=4, nz=4, rate_A=50.0):
    p = w.config1_problem(nx=nx, ny=ny, nz=nz, slab=(5, 9))
    sp, mech = w.mech3(rate_A=rate_A)
    p.species, p.mech = sp, mech
    return p


def _totals(m, sp):
    rho_a = m["rho_a"]
    return dict(mass=rho_a.sum(), species=rho_a.sum(axis=1),
                elements=sp.elements @ (rho_a.sum(axis=1) / sp.W),
                mom=m["rhou"].sum(axis=1), energy=m["rhoE"].sum())


def test_conservation_config1_gases(orc):
    p = _reacting_config1()
    o = orc.Oracle.from_problem(p)
    sp = p.species
    m = o.moments()
    tot0 = _totals(m, sp)
    reacted = 0.0
    for step in range(30):
        # production rates at every node from the moments of this time level
        wsum = np.zeros(sp.M)
        for n in range(o.N):
            wsum += o.rates(m["rho_a"][:, n], m["T"][n])
        before = _totals(m, sp)
        assert o.step(1) == 0
        m = o.moments()
        after = _totals(m, sp)
        scale = before["mass"]
        assert abs(after["mass"] - before["mass"]) <= 1e-14 * scale
        assert np.allclose(after["species"] - before["species"], wsum, rtol=0, atol=1e-14 * scale)
        assert np.allclose(after["elements"], before["elements"], rtol=1e-14, atol=0)
        assert np.abs(after["mom"] - before["mom"]).max() <= 1e-15 * scale
        assert abs(after["energy"] - before["energy"]) <= 1e-14 * abs(before["energy"])
        reacted += abs(wsum[2])
    assert reacted > 1e-4 * tot0["mass"]       # the reaction really ran
    # slaving, Eq. (strongest): species momenta add up to the mixture momentum
    assert np.allclose(m["j_a"].sum(axis=0), m["rhou"], rtol=0, atol=1e-15)


def test_conservation_nine_species_sphere(orc):
    p = w.sphere3d_problem(n=12, radius=3.5, seed=11)
    o = orc.Oracle.from_problem(p)
    sp = p.species
    m0 = o.moments()
    t0 = _totals(m0, sp)
    assert o.step(20) == 0
    m = o.moments()
    t1 = _totals(m, sp)
    assert abs(t1["mass"] - t0["mass"]) <= 1e-13 * t0["mass"]
    assert np.allclose(t1["elements"], t0["elements"], rtol=1e-13, atol=0)
    assert np.abs(t1["mom"] - t0["mom"]).max() <= 1e-15 * t0["mass"]
    assert abs(t1["energy"] - t0["energy"]) <= 1e-13 * abs(t0["energy"])
    # composition changed by chemistry (water formed)
    assert t1["species"][2] > t0["species"][2] * (1 + 1e-7)


def _forward_euler_config1(rho_a, E, steps, A, theta, r_lat, T0=1.0):
    """Homogeneous reactor R + O -> P written out directly: constant heat
    capacities give T = T0 + (e - sum Y U0) / sum Y cv in closed form."""
    W = np.array([2.0, 32.0, 34.0])
    Ra = r_lat / W
    U0 = np.array([0.0, 0.0, -30.0 * Ra[2] * T0]) - Ra * T0
    cv = 2.5 * Ra
    rho_a = rho_a.copy()
    out = []
    for _ in range(steps):
        rho = rho_a.sum()
        Y = rho_a / rho
        T = T0 + (E - Y @ U0) / (Y @ cv)
        q = A * math.exp(-theta / T) * (rho_a[0] / 2.0) * (rho_a[1] / 32.0)
        out.append((rho_a.copy(), T))
        rho_a = rho_a + np.array([-2.0, -32.0, 34.0]) * q
    return out


def test_homogeneous_reactor_is_forward_euler(orc):
    sp, mech = w.mech3(rate_A=400.0)
    lat = LatticeSpec(1, 1, 1, BC_PERIODIC)
    X = np.array([[0.45], [0.45], [0.10]])
    T = np.array([3.0])
    P = sp.r_lat / 23.4
    o = orc.Oracle(lat, sp, mech)
    o.init(X, T, None, P)
    m = o.moments()
    E = m["rhoE"][0] / m["rho"][0]
    ref = _forward_euler_config1(m["rho_a"][:, 0], E, 60, 400.0, 10.0, sp.r_lat)
    for k in range(60):
        rho_ref, T_ref = ref[k]
        assert np.allclose(m["rho_a"][:, 0], rho_ref, rtol=1e-12, atol=1e-16)
        assert abs(m["T"][0] - T_ref) <= 1e-12 * T_ref
        assert o.step(1) == 0
        m = o.moments()
    # heat release: temperature rise equals 30 R_U T0 per mole of P formed
    # over the mixture's molar heat capacity (formation enthalpy, Eq. (specHa))
    assert ref[-1][1] > ref[0][1] + 0.1


def test_uniform_states_are_fixed_points(orc):
    sp, mech = w.mech3()
    mech.log_A[:] = -800.0                      # chemistry off
    lat = LatticeSpec(6, 5, 4, BC_PERIODIC)
    N = lat.n_nodes
    X = np.tile(np.array([[0.3], [0.5], [0.2]]), (1, N))
    T = np.full(N, 1.3)
    P = sp.r_lat / 23.4
    for u0 in (np.zeros(3), np.array([0.02, -0.01, 0.005])):
        o = orc.Oracle(lat, sp, mech)
        o.init(X, T, np.tile(u0[:, None], (1, N)), P)
        p0 = o.get_pop()
        assert o.step(100) == 0
        p1 = o.get_pop()
        assert np.abs(p1 - p0).max() <= 1e-14 * np.abs(p0).max()
        assert np.abs(p1 - p1[:1]).max() <= 1e-15 * np.abs(p0).max()


def _binary_equal_mass(nx, D=0.02, nu_prime=1.0, r_lat=0.4, W0=20.0):
    W = np.array([W0, W0])
    R = r_lat / W0
    sp = SpeciesSpec(names=["A", "B"], W=W, thermo=THERMO_CONST_CP, cp_R=np.full(2, 3.5),
                     h_form=np.zeros(2), T0=1.0, poly7=np.zeros((2, 7)), D=np.full((2, 2), D),
                     nu=nu_prime * R, Pr=0.71, r_lat=r_lat, elements=np.eye(2, dtype=np.int32),
                     element_names=["A", "B"], visc_model=VISC_KINEMATIC)
    mech = MechanismSpec(nu_f=np.zeros((0, 2), np.int32), nu_r=np.zeros((0, 2), np.int32),
                         log_A=np.zeros(0), b=np.zeros(0), theta=np.zeros(0),
                         rtype=np.zeros(0, np.int32), eff=np.zeros((0, 2)), low=np.zeros((0, 3)),
                         reversible=np.zeros(0, np.int32), T_ref=1.0, P0=1.0)
    return sp, mech, LatticeSpec(nx, 1, 1, BC_PERIODIC)


def _mode_amplitude(field, nx):
    return abs(np.fft.rfft(field[:nx])[1]) * 2 / nx


def _decay_rate(series, t0, t1):
    return math.log(series[t0] / series[t1]) / (t1 - t0)


@pytest.mark.parametrize("nx", [64, 128])
def test_fick_limit_binary(orc, nx):
    """Binary mixture of equal molar masses at rest, uniform T and P: the
    Stefan-Maxwell law reduces to Fick's law with D_12, so a sine mode of
    Y_1 decays at D_12 k^2."""
    D = 0.02
    sp, mech, lat = _binary_equal_mass(nx, D=D)
    x = np.arange(nx)
    k = 2 * math.pi / nx
    X1 = 0.5 + 0.02 * np.sin(k * x)
    o = orc.Oracle(lat, sp, mech)
    o.init(np.stack([X1, 1 - X1]), np.ones(nx), None, sp.r_lat / 20.0)
    amps = []
    for t in range(1501):
        if t:
            assert o.step(1) == 0
        if t in (300, 1500):
            m = o.moments()
            amps.append(_mode_amplitude(m["Y"][0], nx))
    rate = math.log(amps[0] / amps[1]) / 1200
    rel = abs(rate / (D * k * k) - 1)
    assert rel < (0.02 if nx == 64 else 0.006), (rate, D * k * k)


def test_shear_wave_viscosity(orc):
    """Transverse wave u_y = U sin(k x): decays at nu k^2 with the kinematic
    viscosity nu = (1/omega - 1/2) R T of Eq. (mu)."""
    nx = 64
    sp, mech = w.mech3()
    mech.log_A[:] = -800.0
    lat = LatticeSpec(nx, 1, 1, BC_PERIODIC)
    k = 2 * math.pi / nx
    u = np.zeros((3, nx))
    u[1] = 1e-3 * np.sin(k * np.arange(nx))
    X = np.tile(np.array([[0.3], [0.5], [0.2]]), (1, nx))
    o = orc.Oracle(lat, sp, mech)
    o.init(X, np.ones(nx), u, sp.r_lat / 23.4)
    amps = {}
    for t in range(1001):
        if t:
            assert o.step(1) == 0
        if t in (200, 1000):
            m = o.moments()
            amps[t] = _mode_amplitude(m["rhou"][1] / m["rho"], nx)
    rate = math.log(amps[200] / amps[1000]) / 800
    assert abs(rate / (sp.nu * k * k) - 1) < 0.02, (rate, sp.nu * k * k)


def _thermal_rate(orc, nx, steps):
    sp, mech = w.mech3()
    mech.log_A[:] = -800.0
    lat = LatticeSpec(nx, 1, 1, BC_PERIODIC)
    k = 2 * math.pi / nx
    T = 1.0 + 0.01 * np.sin(k * np.arange(nx))
    X = np.tile(np.array([[0.3], [0.5], [0.2]]), (1, nx))
    o = orc.Oracle(lat, sp, mech)
    o.init(X, T, None, sp.r_lat / 23.4)
    ts, la = [], []
    for t in range(steps + 1):
        if t:
            assert o.step(1) == 0
        if t >= 200 and t % 5 == 0:
            m = o.moments()
            ts.append(t)
            la.append(math.log(_mode_amplitude(m["T"], nx)))
    rate = -np.polyfit(ts, la, 1)[0]
    RT = sp.r_lat / 23.4
    chi = (sp.nu / RT / sp.Pr) * RT           # (1/omega_1 - 1/2) R T
    return rate / (chi * k * k)


def test_thermal_diffusivity(orc):
    """Entropy mode at uniform pressure: the temperature wave decays at
    lambda/(rho C_p) k^2 = (1/omega_1 - 1/2) R T k^2 (Eq. (lambda)); the
    finite-k deviation falls like k^2."""
    r64 = _thermal_rate(orc, 64, 3000)
    r128 = _thermal_rate(orc, 128, 6000)
    assert abs(r128 - 1) < 0.03, r128
    assert abs(r64 - 1) / abs(r128 - 1) > 3.0, (r64, r128)


def _sound_attenuation_ratio(orc, nx, steps):
    """Amplitude decay rate of a standing sound wave in a binary mixture of
    equal molar masses (no barodiffusion), over the Navier-Stokes-Fourier
    value k^2/2 [ (4/3) mu/rho + varsigma/rho + (gamma - 1) lambda/(rho C_p) ]
    with mu, varsigma of Eq. (mu) and lambda of Eq. (lambda)."""
    sp, mech, lat = _binary_equal_mass(nx)
    R = sp.r_lat / sp.W[0]
    k = 2 * math.pi / nx
    u = np.zeros((3, nx))
    u[0] = 1e-4 * np.sin(k * np.arange(nx))
    X = np.tile(np.array([[0.4], [0.6]]), (1, nx))
    o = orc.Oracle(lat, sp, mech)
    o.init(X, np.ones(nx), u, R)
    gamma = 3.5 / 2.5
    c = math.sqrt(gamma * R)
    ts, la = [], []
    for t in range(steps + 1):
        if t:
            assert o.step(1) == 0
        if t >= 100 and t % 2 == 0:
            m = o.moments()
            a = np.fft.rfft(m["rhou"][0] / m["rho"])[1]
            b = np.fft.rfft(m["rho"] * R * m["T"])[1] / c
            ts.append(t)
            la.append(0.5 * math.log(abs(a) ** 2 + abs(b) ** 2))
    G = -np.polyfit(ts, la, 1)[0]
    nu = sp.nu                                   # mu / rho
    bulk = nu * (2.0 / 3.0 - 1.0 / 2.5)          # varsigma / rho, D = 3
    chi = nu / sp.Pr
    return G / (k * k / 2 * (4.0 / 3.0 * nu + bulk + (gamma - 1) * chi))


def test_sound_attenuation_bulk_viscosity(orc):
    r128 = _sound_attenuation_ratio(orc, 128, 3840)
    r256 = _sound_attenuation_ratio(orc, 256, 7680)
    assert abs(r256 - 1) < 0.02, r256
    assert abs(r128 - 1) / abs(r256 - 1) > 3.0, (r128, r256)


# ---------------------------------------------------------------------------
# Interdiffusion heat flux (Eqs. (qdiff), (corrFourier), (qneq), (dtE))
# ---------------------------------------------------------------------------
def _binary_unequal_enthalpy(nx, dh=10.0, cp_R=(2.5, 4.5), D=0.02, r_lat=0.4, W0=20.0):
    """Two species of equal molar mass (equal R_a, no barodiffusion) whose
    enthalpies differ: different heat capacities and a formation enthalpy
    difference of dh R T0 (Eq. (specHa))."""
    sp, mech, lat = _binary_equal_mass(nx, D=D, r_lat=r_lat, W0=W0)
    R = r_lat / W0
    sp.cp_R = np.array(cp_R, dtype=float)
    sp.h_form = np.array([0.0, -dh * R * sp.T0])
    return sp, mech, lat


def _interdiffusion_run(nx, library=None, dY=0.02, dh=10.0, D=0.02):
    """Y_1 = 1/2 + dY sin(k x) at rest, uniform T = T0 and P.  Returns the
    largest temperature-mode amplitude over the first 1/(D k^2) steps in
    units of (Delta H / C_v) dY, and the decay rate of the Y mode over D k^2.

    With q = -lambda grad T + rho sum_a H_a Y_a V_a (Eq. (qneq)) the energy
    equation at rest, uniform T and P reduces to
        rho C_v dT/dt = -sum_a R_a T div(rho_a V_a) = -R T div(sum_a rho_a V_a) = 0
    for equal R_a, so T stays uniform to leading order in k.  A wrong
    q^diff or q^corr leaves a flux ~ Delta H rho D grad Y_1 in the energy
    equation and drives a T mode of order (Delta H / C_v) dY."""
    import oracle
    sp, mech, lat = _binary_unequal_enthalpy(nx, dh=dh, D=D)
    x = np.arange(nx)
    k = 2 * math.pi / nx
    X1 = 0.5 + dY * np.sin(k * x)
    o = oracle.Oracle(lat, sp, mech, library=library)
    o.init(np.stack([X1, 1 - X1]), np.ones(nx), None, sp.r_lat / sp.W[0])
    R = sp.r_lat / sp.W[0]
    Cv = 0.5 * (sp.cp_R[0] - 1 + sp.cp_R[1] - 1) * R
    scale = dh * R / Cv * dY
    steps = int(round(1.0 / (D * k * k)))
    chunk = max(1, steps // 40)
    t, tmax, ys = 0, 0.0, []
    while True:
        m = o.moments()
        assert m["status"] == 0
        tmax = max(tmax, _mode_amplitude(m["T"], nx))
        ys.append((t, _mode_amplitude(m["Y"][0], nx)))
        if t >= steps:
            break
        assert o.step(chunk) == 0
        t += chunk
    (t0, a0), (t1, a1) = ys[len(ys) // 4], ys[-1]
    rate = math.log(a0 / a1) / (t1 - t0)
    return tmax / scale, rate / (D * k * k)


def test_interdiffusion_heat_flux_keeps_temperature_uniform(orc):
    """Binary mixture of equal molar masses but unequal enthalpies: Y decays
    at D_12 k^2 (Eq. (constit2)) while T stays uniform; the residual
    temperature mode is below 1 % of (Delta H / C_v) dY and falls as k^2.
    Every other hydrodynamic pin uses species of equal enthalpy, for which
    q^diff and q^corr vanish identically."""
    r32, d32 = _interdiffusion_run(32)
    r64, d64 = _interdiffusion_run(64)
    assert r32 < 0.01 and r64 < 0.004, (r32, r64)
    assert r32 / r64 > 3.0, (r32, r64)                 # second order in k
    assert abs(d64 - 1) < 0.02, (d32, d64)              # Fick decay D_12 k^2 ...
    assert abs(d32 - 1) / abs(d64 - 1) > 3.0, (d32, d64)  # ... reached at second order


_QDIFF = "double qdiff = (omega1 / (omega - omega1)) * rho * sumHYdu[b];"
_QCORR = "double qcorr = 0.5 * ((omega1 - 2.0) / (omega1 - omega)) * P * sumHgradY[b];"
_GRADY = "s->gradY[(n * M + a) * 3 + d] = gY[a][d] / THETA;"


@pytest.mark.parametrize("mutant,old,new", [
    ("q^diff dropped", _QDIFF, "double qdiff = 0.0;"),
    ("q^corr prefactor sign flipped", _QCORR, _QCORR.replace("0.5 *", "-0.5 *")),
    ("q^corr half dropped", _QCORR, _QCORR.replace("0.5 * ", "")),
    ("grad Y sign flipped", _GRADY, _GRADY.replace("gY[a][d] / THETA", "-gY[a][d] / THETA")),
])
def test_interdiffusion_pin_catches_planted_mistakes(orc, tmp_path, mutant, old, new):
    """The pin above fails for an oracle with a plausible mistake planted in
    q^diff (Eq. (qdiff)), q^corr (Eq. (corrFourier)) or the lattice
    gradient of Y that feeds it: the temperature mode then reaches 20-60 %
    of (Delta H / C_v) dY, against 0.75 % for the oracle as written."""
    src = orc.SRC.read_text()
    assert src.count(old) == 1, mutant
    lib = orc.load_variant(src.replace(old, new), tmp_path)
    r32, _ = _interdiffusion_run(32, library=lib)
    assert r32 > 0.1, (mutant, r32)
