"""Pins of the oracle's point-wise pieces against what the paper and the
mathematics fix (no GPU).

* golden D3Q27 weights (Sec. 3, 1D weights 1 - theta, theta/2, theta = 1/3)
* product-form moments (Eq. (phis), Eqs. (feq)/(fstar)/(feqmix)):
  every 1D moment sum_c Psi_c c^p is 1, xi, xi^2 + zeta, so the 27 product
  moments of a set are products of those
* Grad equilibrium moments, Eqs. (gieq), (geq1mom), (geq2mom)
* Stefan-Maxwell system, Eq. (transform1): sum_a Y_a du_a = 0 and the binary
  closed form
* thermodynamic identities of Eqs. (specHa), (temperature)
* zero net production at chemical equilibrium, Eq. (sumRhoDot) and the
  mass-action/equilibrium-constant construction
"""
import math
from pathlib import Path

import mpmath
import numpy as np
import pytest

import workload as w
from workload.problem import LatticeSpec

GOLDEN = Path(__file__).parent / "golden"


def _cvel(orc):
    return orc.C_VEL


def test_golden_d3q27_weights(orc):
    rows = [l.split() for l in (GOLDEN / "d3q27_weights.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    table = {int(r[0]): (int(r[1]) / int(r[2]), int(r[3])) for r in rows}
    # the weights are the zero-velocity rest populations of Grad's form with
    # rhoE = 1 and no flux, and the product form at zeta = theta = 1/3
    g = orc.grad_pop(1.0, np.zeros(3), np.eye(3) / 3.0)
    f = orc.product_form(1.0, np.zeros(3), 1.0 / 3.0)
    c2 = (_cvel(orc) ** 2).sum(axis=1)
    for k, (wk, mult) in table.items():
        assert (c2 == k).sum() == mult
        assert np.allclose(g[c2 == k], wk, rtol=0, atol=2e-16)
        assert np.allclose(f[c2 == k], wk, rtol=0, atol=2e-16)
    assert abs(sum(wk * m for wk, m in table.values()) - 1.0) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_product_form_moments(orc, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 3.0)
    v = rng.uniform(-0.2, 0.2, 3)
    zeta = rng.uniform(0.01, 0.6)
    f = orc.product_form(rho, v, zeta)
    c = _cvel(orc)

    def m1(p, xi):
        return [1.0, xi, xi * xi + zeta][p]

    for p in range(3):
        for q in range(3):
            for r in range(3):
                got = np.sum(f * c[:, 0] ** p * c[:, 1] ** q * c[:, 2] ** r)
                want = rho * m1(p, v[0]) * m1(q, v[1]) * m1(r, v[2])
                assert abs(got - want) <= 1e-15 * rho * 10
    # 27 moments determine the populations: the moment matrix is invertible
    Mm = np.array([[c[i, 0] ** p * c[i, 1] ** q * c[i, 2] ** r for i in range(27)]
                   for p in range(3) for q in range(3) for r in range(3)])
    assert np.linalg.matrix_rank(Mm) == 27


@pytest.mark.parametrize("seed", range(5))
def test_grad_equilibrium_moments(orc, seed):
    rng = np.random.default_rng(100 + seed)
    rhoE = rng.uniform(-2.0, 5.0)
    q = rng.uniform(-1, 1, 3)
    A = rng.uniform(-1, 1, (3, 3))
    R = A + A.T + 3 * np.eye(3)
    g = orc.grad_pop(rhoE, q, R)
    c = _cvel(orc).astype(float)
    assert abs(g.sum() - rhoE) < 1e-14 * (1 + abs(rhoE))
    assert np.allclose(c.T @ g, q, atol=1e-14)
    second = np.einsum("i,ia,ib->ab", g, c, c)
    assert np.allclose(second, R, atol=1e-14)


def test_mixture_equilibrium_sets_moments(orc):
    """Every set at equilibrium: species densities, mixture momentum, energy
    with formation enthalpy (Eq. (g0momTotalEnergy)), q^eq and R^eq."""
    sp, mech = w.mech3()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    rho_a = np.array([0.05, 0.6, 0.35])
    u = np.array([0.03, -0.01, 0.02])
    T = 1.7
    eq = o.equilibrium_sets(rho_a, u, T)
    c = _cvel(orc).astype(float)
    rho = rho_a.sum()
    for a in range(2):
        assert abs(eq[a].sum() - rho_a[a]) < 1e-15
        assert np.allclose(c.T @ eq[a], rho_a[a] * u, atol=1e-16)
    assert abs(eq[2].sum() - rho) < 1e-15
    assert np.allclose(c.T @ eq[2], rho * u, atol=1e-15)
    th = o.thermo(T)
    Y = rho_a / rho
    U = float(Y @ th["U"])
    H = float(Y @ th["H"])
    usq = float(u @ u)
    assert abs(eq[3].sum() - rho * (U + usq / 2)) < 1e-14
    assert np.allclose(c.T @ eq[3], (H + usq / 2) * rho * u, atol=1e-15)
    Rmix = sp.r_lat * float(Y @ (1 / sp.W))
    P = rho * Rmix * T
    Peq = P * np.eye(3) + rho * np.outer(u, u)
    Req = (H + usq / 2) * Peq + P * np.outer(u, u)
    assert np.allclose(np.einsum("i,ia,ib->ab", eq[3], c, c), Req, atol=1e-15)
    # ideal-gas enthalpy: H_a - U_a = R_a T
    assert np.allclose(th["H"] - th["U"], sp.r_lat / sp.W * T, rtol=1e-14)


def _random_sm_state(rng, M):
    Y = rng.uniform(0.01, 1.0, M)
    Y /= Y.sum()
    ua = rng.uniform(-0.05, 0.05, (M, 3))
    u = (Y[:, None] * ua).sum(axis=0)       # sum_a rho_a u_a = rho u (Sec. 2)
    return Y, ua - u


@pytest.mark.parametrize("seed", range(4))
def test_stefan_maxwell_mass_weighted_sum_vanishes(orc, seed):
    rng = np.random.default_rng(seed)
    sp, mech = w.mech9()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    Y, r = _random_sm_state(rng, 9)
    du, st = o.diffusion_velocities(Y, r, T=rng.uniform(300, 2500))
    assert st == 0
    assert np.abs((Y[:, None] * du).sum(axis=0)).max() < 1e-15
    # relaxation: the transformed velocities are smaller than the raw ones
    assert np.abs(du).max() <= np.abs(r).max()


def test_stefan_maxwell_binary_closed_form(orc):
    """For M = 2 Eq. (transform1) gives du_1 = (u_1 - u)/(1 + 1/(2 tau_12)),
    with tau_12 = m_1 m_2 D_12 / (m R_U T) (Eq. (tauab))."""
    W = np.array([4.0, 20.0])
    sp, mech = w.mech3()
    sp.W = W
    sp.D = np.full((2, 2), 0.03)
    sp.cp_R = np.full(2, 3.5)
    sp.h_form = np.zeros(2)
    sp.poly7 = np.zeros((2, 7))
    mech.nu_f = np.zeros((0, 2), dtype=np.int32)
    mech.nu_r = np.zeros((0, 2), dtype=np.int32)
    for k in ("log_A", "b", "theta"):
        setattr(mech, k, np.zeros(0))
    mech.rtype = np.zeros(0, dtype=np.int32)
    mech.reversible = np.zeros(0, dtype=np.int32)
    mech.eff = np.zeros((0, 2))
    mech.low = np.zeros((0, 3))
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    Y = np.array([0.3, 0.7])
    r1 = np.array([0.01, -0.02, 0.005])
    r = np.stack([r1, -Y[0] * r1 / Y[1]])
    T = 1.3
    du, st = o.diffusion_velocities(Y, r, T)
    m = 1.0 / (Y[0] / W[0] + Y[1] / W[1])
    tau12 = W[0] * W[1] * 0.03 / (m * sp.r_lat * T)
    assert np.allclose(du[0], r1 / (1.0 + 1.0 / (2.0 * tau12)), rtol=1e-14, atol=0)


def test_thermo_identities_poly7(orc):
    """U_a, H_a, C_{a,v} and g_a/(R_U T) of the polynomial thermodynamics obey
    dU_a/dT = C_{a,v}, H_a - U_a = R_a T, and d(g/RT)/dT = -h/(R T^2)."""
    sp, mech = w.mech9()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    Ra = sp.r_lat / sp.W
    for T in (300.0, 900.0, 1800.0, 2700.0):
        h = 1e-3
        tp, tm = o.thermo(T + h), o.thermo(T - h)
        t0 = o.thermo(T)
        dU = (tp["U"] - tm["U"]) / (2 * h)
        assert np.allclose(dU, t0["Cv"], rtol=1e-7)
        assert np.allclose(t0["H"] - t0["U"], Ra * T, rtol=1e-13)
        dg = (tp["gRT"] - tm["gRT"]) / (2 * h)
        assert np.allclose(dg, -(t0["H"] / (Ra * T)) / T, rtol=1e-6, atol=1e-9)


def test_temperature_constant_cv_closed_form(orc):
    """Eq. (temperature) with constant C_{a,v}: T = T0 + (e - sum Y U0)/sum Y cv."""
    sp, mech = w.mech3()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    Ra = sp.r_lat / sp.W
    U0 = sp.h_form - Ra * sp.T0
    cv = (sp.cp_R - 1.0) * Ra
    rng = np.random.default_rng(3)
    for _ in range(20):
        Y = rng.uniform(0.05, 1, 3)
        Y /= Y.sum()
        T_true = rng.uniform(0.5, 6.0)
        e = float(Y @ (U0 + cv * (T_true - sp.T0)))
        T, st = o.temperature(Y, e, T_guess=1.0)
        assert st == 0
        assert abs(T - T_true) <= 1e-13 * T_true


def test_temperature_poly7_against_bisection(orc):
    """Polynomial thermodynamics: Newton's T against a 40-digit bisection of
    sum_a Y_a U_a(T) = e with U_a from the single-range 7-coefficient form."""
    sp, mech = w.mech9()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    mpmath.mp.dps = 40
    P = [[mpmath.mpf(float(x)) for x in row] for row in sp.poly7]
    r = mpmath.mpf(sp.r_lat)

    def U(a, T):
        p = P[a]
        hRT = p[0] + p[1] * T / 2 + p[2] * T ** 2 / 3 + p[3] * T ** 3 / 4 + p[4] * T ** 4 / 5 + p[5] / T
        return r / mpmath.mpf(float(sp.W[a])) * T * (hRT - 1)

    rng = np.random.default_rng(5)
    for _ in range(4):
        Y = rng.uniform(0.01, 1, 9)
        Y /= Y.sum()
        Ym = [mpmath.mpf(float(y)) for y in Y]
        T_true = mpmath.mpf(float(rng.uniform(300, 2800)))
        e = sum(Ym[a] * U(a, T_true) for a in range(9))
        lo, hi = mpmath.mpf(100), mpmath.mpf(5000)
        for _ in range(200):
            mid = (lo + hi) / 2
            if sum(Ym[a] * U(a, mid) for a in range(9)) < e:
                lo = mid
            else:
                hi = mid
        T_ref = float((lo + hi) / 2)
        T, st = o.temperature(Y, float(e), T_guess=1000.0)
        assert st == 0
        assert abs(T - T_ref) <= 1e-13 * T_ref


@pytest.mark.parametrize("T", [400.0, 900.0, 1500.0, 2400.0])
def test_zero_production_at_chemical_equilibrium(orc, T):
    """Concentrations c_a = (P0/(R_U T)) exp(-g_a/RT + sum_e lambda_e n_ea)
    make every element-balanced reaction's forward and reverse rates equal,
    whatever its rate law (elementary, third body, falloff)."""
    sp, mech = w.mech9()
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    g = o.thermo(T)["gRT"]
    rng = np.random.default_rng(int(T))
    lam = rng.uniform(-3, 3, 3)
    c = mech.P0 / (sp.r_lat * T) * np.exp(-g + lam @ sp.elements)
    rho_a = c * sp.W
    wdot = o.rates(rho_a, T)
    # scale of the individual forward terms
    kmax = 0.0
    for k in range(mech.R):
        kf = math.exp(mech.log_A[k] + mech.b[k] * math.log(T / mech.T_ref) - mech.theta[k] / T)
        conc_M = float(mech.eff[k] @ c) if mech.rtype[k] == 1 else 1.0
        kmax = max(kmax, kf * np.prod(c ** mech.nu_f[k]) * conc_M * sp.W.max())
    assert np.abs(wdot).max() <= 1e-10 * kmax
    # mass conservation, Eq. (sumRhoDot), away from equilibrium
    rho_b = rho_a * rng.uniform(0.5, 2.0, 9)
    wb = o.rates(rho_b, T)
    assert abs(wb.sum()) <= 1e-13 * np.abs(wb).max()
    # element conservation
    assert np.allclose(sp.elements @ (wb / sp.W), 0.0, atol=1e-13 * np.abs(wb / sp.W).max())


def _single_reaction_mech(rtype, log_A, b, theta, eff=None, low=None, reversible=0):
    sp, mech = w.mech9()
    k = 4 if rtype == 2 else 0          # H + HO2 <=> H2O2 (falloff) / O + OH <=> HO2 (third body)
    sel = slice(k, k + 1)
    mech.nu_f, mech.nu_r = mech.nu_f[sel].copy(), mech.nu_r[sel].copy()
    mech.log_A = np.array([log_A])
    mech.b = np.array([b])
    mech.theta = np.array([theta])
    mech.rtype = np.array([rtype], dtype=np.int32)
    mech.eff = np.ones((1, 9)) if eff is None else np.asarray(eff, dtype=float)[None]
    mech.low = np.zeros((1, 3)) if low is None else np.asarray(low, dtype=float)[None]
    mech.reversible = np.array([reversible], dtype=np.int32)
    return sp, mech


def test_arrhenius_third_body_and_falloff_limits(orc):
    """Rate laws used for the synthetic mechanism: irreversible rate of
    progress k c_A c_B with k = A (T/T_ref)^b exp(-theta/T); a third body
    multiplies it by [M] = sum eff_a c_a; the Lindemann falloff tends to the
    high-pressure k_inf when k0 [M] >> k_inf and to k0 [M] when k0 [M] << k_inf."""
    T = 1300.0
    rho_a = np.array([0.02, 0.2, 0.05, 1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 0.7])
    c = rho_a / w.configs.W9
    sp, mech = _single_reaction_mech(0, 1.5, 0.7, 3000.0)
    o = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech)
    base = o.rates(rho_a, T)
    k = math.exp(1.5) * (T / 1000.0) ** 0.7 * math.exp(-3000.0 / T)
    # O + OH -> HO2: O consumed at W_O * k c_O c_OH
    assert abs(-base[4] / (16.0 * k * c[4] * c[5]) - 1) < 1e-13
    # third body: linear in each efficiency
    eff = np.zeros(9)
    eff[8] = 2.0
    sp, mech = _single_reaction_mech(1, 1.5, 0.7, 3000.0, eff=eff)
    r2 = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech).rates(rho_a, T)
    assert abs(r2[4] / base[4] - 2.0 * c[8]) < 1e-13 * 2.0 * c[8]
    # falloff limits
    sp, mech = _single_reaction_mech(2, 1.5, 0.7, 3000.0, low=(60.0, 0.0, 0.0))
    hi = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech).rates(rho_a, T)
    kinf = math.exp(1.5) * (T / 1000.0) ** 0.7 * math.exp(-3000.0 / T)
    # H + HO2 -> H2O2: H consumed at W_H * k c_H c_HO2
    assert abs(-hi[3] / (1.0 * kinf * c[3] * c[6]) - 1) < 1e-12
    sp, mech = _single_reaction_mech(2, 1.5, 0.7, 3000.0, low=(-40.0, 0.3, 100.0))
    lo = orc.Oracle(LatticeSpec(1, 1, 1), sp, mech).rates(rho_a, T)
    k0 = math.exp(-40.0) * (T / 1000.0) ** 0.3 * math.exp(-100.0 / T)
    assert abs(-lo[3] / (1.0 * k0 * c.sum() * c[3] * c[6]) - 1) < 1e-9
