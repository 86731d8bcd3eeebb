"""Seeded problem instances.

Config names follow the workloads they stand in for:

* ``config1_problem``   64x4x4 periodic, three ideal gases R, O, P, one
                        irreversible step R + O -> P (plain FP64 scale).
* ``flame1d_problem``   quasi-1D premixed flame nx x 4 x 4 with equilibrium
                        zero-gradient ghost nodes in x (u = 0 on the left),
                        the nine-species synthetic mechanism.  Stand-in for
                        the paper's 1D hydrogen/air flame-speed runs (Sec. 5a).
* ``sphere3d_problem``  periodic cube with a hot spherical kernel, the same
                        mechanism.  Stand-in for the paper's expanding
                        circular flame (Sec. 5b), lifted to 3D.
* ``small_periodic_problem``  4^3 / 8^3 perturbed states for brute-force checks.

The real hydrogen/air mechanism, Cantera and the paper's data are not
available; the nine-species mechanism is a seeded synthetic one with the
paper's species set and sizes (9 species, 21 reactions).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .problem import (
    TRANSPORT_MIXTURE_AVERAGED,
    BC_EQ_ZEROGRAD_U0LEFT,
    BC_PERIODIC,
    RXN_ELEMENTARY,
    RXN_FALLOFF,
    RXN_THIRD_BODY,
    THERMO_CONST_CP,
    THERMO_POLY7,
    VISC_KINEMATIC,
    VISC_RELAXATION,
    InitFields,
    LatticeSpec,
    MechanismSpec,
    Problem,
    SpeciesSpec,
)

X_FLOOR = 1e-12

# --------------------------------------------------------------------------
# Config-1 gases: R (W=2), O (W=32), P (W=34), cp/R = 3.5, T0 = 1 (lattice).
# --------------------------------------------------------------------------
# Universal gas constant in lattice units.  With the stated kinematic
# viscosity 0.02 this puts 1/omega - 1/2 = nu/(R T) at 1.17 (T0) and 0.29
# (4 T0), inside the range where the coupled f/g collisions stay stable, and
# keeps R_a T below 1 for the lightest gas up to T = 5 T0.
MECH3_R_LAT = 0.4
MECH3_T0 = 1.0


def mech3(D: float = 0.02, nu: float = 0.02, Pr: float = 0.71, rate_A: float = 0.05,
          rate_theta: float = 10.0):
    """Three ideal gases R, O, P and the irreversible step R + O -> P.

    Formation enthalpy (mass specific, at T0): 0 for R and O, -30 R_P T0 for P.
    Rate of progress q = rate_A * exp(-rate_theta*T0/T) * c_R * c_O.
    """
    names = ["R", "O", "P"]
    W = np.array([2.0, 32.0, 34.0])
    r = MECH3_R_LAT
    h_form = np.array([0.0, 0.0, -30.0 * (r / W[2]) * MECH3_T0])
    sp = SpeciesSpec(
        names=names, W=W, thermo=THERMO_CONST_CP, cp_R=np.full(3, 3.5), h_form=h_form,
        T0=MECH3_T0, poly7=np.zeros((3, 7)), D=np.full((3, 3), D), nu=nu, Pr=Pr,
        r_lat=r, elements=np.array([[1, 0, 1], [0, 1, 1]], dtype=np.int32),
        element_names=["R", "O"], visc_model=VISC_KINEMATIC)
    mech = MechanismSpec(
        nu_f=np.array([[1, 1, 0]], dtype=np.int32),
        nu_r=np.array([[0, 0, 1]], dtype=np.int32),
        log_A=np.array([math.log(rate_A)]), b=np.zeros(1), theta=np.array([rate_theta * MECH3_T0]),
        rtype=np.zeros(1, dtype=np.int32), eff=np.ones((1, 3)), low=np.zeros((1, 3)),
        reversible=np.zeros(1, dtype=np.int32), T_ref=1.0, P0=1.0)
    return sp, mech


def _normalise_with_noise(X0: np.ndarray, N: int, seed, amp: float = 1e-3) -> np.ndarray:
    """X0 [M] mean mole fractions -> [M,N] with per-node uniform noise.

    Draw order: one array of shape [N, M] (node-major, x fastest, then
    species) from numpy's PCG64 with the given seed.  The noise perturbs the
    species present in X0; absent species stay at X_FLOOR (noise on them
    would make trace densities jump by nine orders of magnitude between
    neighbouring nodes).  Clip at X_FLOOR and renormalise each node.
    """
    M = X0.shape[0]
    X = np.repeat(X0[:, None], N, axis=1)
    if seed is not None:
        rng = np.random.Generator(np.random.PCG64(seed))
        noise = rng.uniform(-amp, amp, size=(N, M))
        X = X + noise.T * (X0 > 0)[:, None]
    X = np.maximum(X, X_FLOOR)
    X = X / X.sum(axis=0, keepdims=True)
    return np.ascontiguousarray(X)


def _pressure_for_unit_density(X_mean: np.ndarray, W: np.ndarray, r_lat: float, T: float) -> float:
    """Uniform pressure level at which the mean mixture at T has unit density.

    This is the unit convention of the inputs ("1 atm" maps to the pressure
    of the cold mixture at unit lattice density).
    """
    m = float(np.dot(X_mean, W))
    return r_lat / m * T


def config1_problem(nx: int = 64, ny: int = 4, nz: int = 4, seed: int = 1702,
                    slab=(28, 36), T_hot: float = 4.0) -> Problem:
    sp, mech = mech3()
    N = nx * ny * nz
    X0 = np.array([0.3, 0.5, 0.2])
    X = _normalise_with_noise(X0, N, seed)
    T = np.full(N, MECH3_T0)
    xs = np.arange(N) % nx
    T[(xs >= slab[0]) & (xs < slab[1])] = T_hot * MECH3_T0
    P = _pressure_for_unit_density(X0, sp.W, sp.r_lat, MECH3_T0)
    return Problem("config1_64x4x4_M3", LatticeSpec(nx, ny, nz, BC_PERIODIC), sp, mech,
                   InitFields(X=X, T=T, u=None, P=P), steps=200)


def small_periodic_problem(n: int = 4, seed: int = 7, M3_rate_A: float = 0.05,
                           du: float = 0.02, dT: float = 0.5) -> Problem:
    """n^3 periodic, config-1 gases, random composition, temperature and velocity."""
    sp, mech = mech3(rate_A=M3_rate_A)
    N = n ** 3
    rng = np.random.Generator(np.random.PCG64(seed))
    X0 = np.array([0.3, 0.5, 0.2])
    X = X0[:, None] + rng.uniform(-0.1, 0.1, size=(3, N))
    X = np.maximum(X, X_FLOOR)
    X /= X.sum(axis=0, keepdims=True)
    T = MECH3_T0 * (1.0 + rng.uniform(0.0, dT, size=N))
    u = rng.uniform(-du, du, size=(3, N))
    P = _pressure_for_unit_density(X0, sp.W, sp.r_lat, MECH3_T0)
    return Problem(f"periodic_{n}^3_M3", LatticeSpec(n, n, n, BC_PERIODIC), sp, mech,
                   InitFields(X=np.ascontiguousarray(X), T=T, u=np.ascontiguousarray(u), P=P))


# --------------------------------------------------------------------------
# Nine-species synthetic mechanism (H, O, N elements; hydrogen/air species).
# --------------------------------------------------------------------------
SPECIES9 = ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N2"]
W9 = np.array([2.0, 32.0, 18.0, 1.0, 16.0, 17.0, 33.0, 34.0, 28.0])
ELEM9 = np.array([  # rows: H, O, N
    [2, 0, 2, 1, 0, 1, 1, 2, 0],
    [0, 2, 1, 0, 1, 1, 2, 2, 0],
    [0, 0, 0, 0, 0, 0, 0, 0, 2],
], dtype=np.int32)
MECH9_SEED = 2101
MECH9_R_LAT = 0.5 / 3000.0     # R_U in lattice units per kelvin: R_H * 3000 K = 0.5
MECH9_T_REF = 1000.0           # rate coefficients use (T / 1000 K)^b
MECH9_T_UNBURNT = 300.0
# Global rate scale applied to every pre-exponential factor.  Chosen once for
# this seeded mechanism (oracle/calibrate_chem_scale.py prints the value) so
# that no species is consumed faster than a fixed fraction of its own mass per
# lattice time step anywhere in the temperature range 300-2500 K.
MECH9_CHEM_SCALE = 1.8e-21
# Constant relaxation 1/omega - 1/2 (viscosity mu = 0.8 P).  A constant
# kinematic viscosity would move 1/omega - 1/2 by the temperature ratio
# (8x between 300 K and 2500 K), beyond the range where the coupled
# collisions stay stable.
MECH9_NU_PRIME = 0.8
PHI1_X = np.array([0.296, 0.148, 0, 0, 0, 0, 0, 0, 0.556])   # H2/O2/N2, phi = 1


def phi_mixture(phi: float) -> np.ndarray:
    """Unburnt H2/O2/N2 mole fractions 2 phi : 1 : 3.76, normalised."""
    X = np.zeros(9)
    X[0], X[1], X[8] = 2.0 * phi, 1.0, 3.76
    return X / X.sum()


def _enumerate_reactions():
    """All element-balanced reactions among the 8 reactive species with at
    most two reactants and two products and no species on both sides.
    Returns (association list [(A,B)->(C,)], exchange list [(A,B)->(C,D)])."""
    reactive = range(8)
    el = ELEM9[:2]
    sides2 = [(a, b) for a in reactive for b in reactive if a <= b]
    sides1 = [(c,) for c in reactive]

    def comp(s):
        return tuple(int(sum(el[e, i] for i in s)) for e in range(2))

    assoc = [(s2, s1) for s2 in sides2 for s1 in sides1
             if comp(s2) == comp(s1) and set(s2).isdisjoint(s1)]
    exch = []
    for i, s in enumerate(sides2):
        for t in sides2[i + 1:]:
            if comp(s) == comp(t) and set(s).isdisjoint(t):
                exch.append((s, t))
    return assoc, exch


def _draw_poly7(rng, h_f_R: float, s_R: float) -> np.ndarray:
    """Seeded 7-coefficient polynomial with cp/R in [2.5, 8] on [200, 4000] K,
    h/R(298.15) = h_f_R and s/R(298.15) = s_R."""
    Ts = np.linspace(200.0, 4000.0, 400)
    while True:
        a1 = rng.uniform(2.5, 4.5)
        a2 = rng.uniform(0.0, 1.0e-3)
        a3 = rng.uniform(-2.0e-7, 2.0e-7)
        a4 = rng.uniform(-2.0e-11, 2.0e-11)
        a5 = rng.uniform(-1.0e-15, 1.0e-15)
        cp = a1 + a2 * Ts + a3 * Ts ** 2 + a4 * Ts ** 3 + a5 * Ts ** 4
        if cp.min() >= 2.5 and cp.max() <= 8.0:
            break
    t = 298.15
    a6 = h_f_R - (a1 * t + a2 * t ** 2 / 2 + a3 * t ** 3 / 3 + a4 * t ** 4 / 4 + a5 * t ** 5 / 5)
    a7 = s_R - (a1 * math.log(t) + a2 * t + a3 * t ** 2 / 2 + a4 * t ** 3 / 3 + a5 * t ** 4 / 4)
    return np.array([a1, a2, a3, a4, a5, a6, a7])


# Formation-enthalpy ranges h_f / R_U [K] at 298.15 K: zero for the reference
# molecules, strongly negative for the product, positive for radicals.
_HF_RANGES = {
    "H2": (0.0, 0.0), "O2": (0.0, 0.0), "N2": (0.0, 0.0),
    "H2O": (-26000.0, -22000.0), "H": (24000.0, 28000.0), "O": (27000.0, 31000.0),
    "OH": (3000.0, 5000.0), "HO2": (0.0, 2000.0), "H2O2": (-18000.0, -14000.0),
}


def mech9(chem_scale: float = MECH9_CHEM_SCALE, seed: int = MECH9_SEED):
    """The seeded nine-species, 21-reaction synthetic mechanism.

    Draw order from PCG64(seed): association picks, exchange picks (redrawn
    until H2 and O2 each appear as a reactant), per-species formation
    enthalpies h_f/R_U [K] and entropies s/R at 298.15 K, log10 A, b, Ea/R,
    third-body efficiencies, falloff low-pressure parameters, then the
    polynomial coefficients species by species.  Association reactions are
    written A + B -> C; exchange reactions in their exothermic direction
    (by the drawn formation enthalpies).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    assoc, exch = _enumerate_reactions()
    while True:
        ia = rng.choice(len(assoc), 6, replace=False)
        ie = rng.choice(len(exch), 15, replace=False)
        chosen = [assoc[i] for i in ia] + [exch[i] for i in ie]
        reactant_species = set(itertools.chain.from_iterable(r[0] for r in chosen))
        if 0 in reactant_species and 1 in reactant_species:
            break
    # Formation enthalpies are drawn here (before the rate parameters) so
    # that every exchange reaction can be written in its exothermic direction:
    # the Arrhenius parameters below belong to that direction, and the reverse
    # rate follows from the equilibrium constant.
    h_f = np.array([rng.uniform(*_HF_RANGES[name]) if _HF_RANGES[name][1] > _HF_RANGES[name][0]
                    else _HF_RANGES[name][0] for name in SPECIES9])
    s_R = rng.uniform(13.0, 30.0, size=9)
    rxns = [assoc[i] for i in ia]
    for i in ie:
        s_, t_ = exch[i]
        dh = sum(h_f[j] for j in t_) - sum(h_f[j] for j in s_)
        rxns.append((s_, t_) if dh <= 0.0 else (t_, s_))
    R = len(rxns)
    nu_f = np.zeros((R, 9), dtype=np.int32)
    nu_r = np.zeros((R, 9), dtype=np.int32)
    for k, (lhs, rhs) in enumerate(rxns):
        for s in lhs:
            nu_f[k, s] += 1
        for s in rhs:
            nu_r[k, s] += 1
    log10A = rng.uniform(10.0, 18.0, size=R)
    b = rng.uniform(-1.0, 2.0, size=R)
    theta = rng.uniform(0.0, 25000.0, size=R)
    rtype = np.zeros(R, dtype=np.int32)
    rtype[0:4] = RXN_THIRD_BODY
    rtype[4:6] = RXN_FALLOFF
    eff = np.ones((R, 9))
    eff[0:6] = rng.uniform(0.5, 12.0, size=(6, 9))
    low = np.zeros((R, 3))
    low[4:6, 0] = rng.uniform(12.0, 20.0, size=2) * math.log(10.0) + math.log(chem_scale)
    low[4:6, 1] = rng.uniform(-1.0, 2.0, size=2)
    low[4:6, 2] = rng.uniform(0.0, 25000.0, size=2)
    poly7 = np.zeros((9, 7))
    for a in range(9):
        poly7[a] = _draw_poly7(rng, h_f[a], s_R[a])

    W = W9.copy()
    D = 0.02 * np.sqrt(14.0 * (1.0 / W[:, None] + 1.0 / W[None, :]))
    X_cold = np.maximum(PHI1_X, X_FLOOR)
    X_cold = X_cold / X_cold.sum()
    P0 = _pressure_for_unit_density(X_cold, W, MECH9_R_LAT, MECH9_T_UNBURNT)
    sp = SpeciesSpec(
        names=list(SPECIES9), W=W, thermo=THERMO_POLY7, cp_R=np.zeros(9), h_form=np.zeros(9),
        T0=298.15, poly7=poly7, D=D, nu=MECH9_NU_PRIME, Pr=0.71, r_lat=MECH9_R_LAT,
        elements=ELEM9.copy(), element_names=["H", "O", "N"], visc_model=VISC_RELAXATION)
    mech = MechanismSpec(
        nu_f=nu_f, nu_r=nu_r, log_A=log10A * math.log(10.0) + math.log(chem_scale), b=b,
        theta=theta, rtype=rtype, eff=eff, low=low, reversible=np.ones(R, dtype=np.int32),
        T_ref=MECH9_T_REF, P0=P0)
    return sp, mech


def flame1d_problem(nx: int = 4096, ny: int = 4, nz: int = 4, phi: float = 1.0,
                    T_u: float = MECH9_T_UNBURNT, T_slab: float = 1500.0,
                    slab_frac: float = 0.2, chem_scale: float = MECH9_CHEM_SCALE,
                    X_override=None) -> Problem:
    """Quasi-1D flame tube: unburnt mixture at T_u, the rightmost slab_frac of
    x at T_slab with the same composition, uniform pressure, at rest."""
    sp, mech = mech9(chem_scale)
    N = nx * ny * nz
    X0 = phi_mixture(phi) if X_override is None else np.asarray(X_override, dtype=float)
    X = _normalise_with_noise(X0, N, None)
    T = np.full(N, T_u)
    xs = np.arange(N) % nx
    T[xs >= int(round((1.0 - slab_frac) * nx))] = T_slab
    return Problem(f"flame1d_{nx}x{ny}x{nz}_M9", LatticeSpec(nx, ny, nz, BC_EQ_ZEROGRAD_U0LEFT),
                   sp, mech, InitFields(X=X, T=T, u=None, P=mech.P0), steps=20000)


def adjoint_flame_problem(nx: int = 512, ny: int = 4, nz: int = 4, T_slab: float = 1500.0,
                          chem_scale: float = MECH9_CHEM_SCALE) -> Problem:
    """The quasi-1D flame tube of flame1d_problem (phi = 1 unburnt mixture
    at 300 K, the rightmost fifth at T_slab) with periodic x faces: the
    workload of the heat-release gradients through time."""
    p = flame1d_problem(nx=nx, ny=ny, nz=nz, T_slab=T_slab, chem_scale=chem_scale)
    p.lattice.bc_x = BC_PERIODIC
    p.name = f"adjoint_flame_{nx}x{ny}x{nz}_M9_periodic"
    p.steps = 2000
    return p


def circular_flame_problem(n: int = 512, nz: int = 1, R_ig: float = 48.0, A0: float = 0.05, n0: int = 4,
                           phi: float = 0.6, T_u: float = 298.0, T_b: float = 1844.27, width: float = 1.5,
                           chem_scale: float = MECH9_CHEM_SCALE) -> Problem:
    """The circular expanding flame of Sec. 5b on a periodic quasi-2D box
    n x n x nz: the mixture of equivalence ratio phi at T_u, and inside
    R(theta) = R_ig (1 + A0 cos(4 n0 theta)) around the box centre
    (Eq. (cflamePerturbation)) the same composition at T_b, joined by a
    tanh profile of the given width (nodes); uniform pressure, at rest."""
    sp, mech = mech9(chem_scale)
    N = n * n * nz
    X = _normalise_with_noise(phi_mixture(phi), N, None)
    idx = np.arange(N)
    x = (idx % n).astype(float)
    y = ((idx // n) % n).astype(float)
    c = (n - 1) / 2.0
    th = np.arctan2(y - c, x - c)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2)
    Rt = R_ig * (1.0 + A0 * np.cos(4 * n0 * th))
    T = T_u + (T_b - T_u) * 0.5 * (1.0 - np.tanh((r - Rt) / width))
    return Problem(f"circular_flame_{n}x{n}x{nz}_M9", LatticeSpec(n, n, nz, BC_PERIODIC), sp, mech,
                   InitFields(X=X, T=T, u=None, P=mech.P0), steps=1000)


def sphere3d_problem(n: int = 256, radius: float = 20.0, T_u: float = MECH9_T_UNBURNT,
                     T_hot: float = 2000.0, seed: int = 1703,
                     chem_scale: float = MECH9_CHEM_SCALE, shape=None) -> Problem:
    """Periodic box (n^3, or shape = (nx, ny, nz)), phi = 1 mixture with seeded
    composition noise, hot sphere |x - c| < radius (c = box centre, integer
    division) at T_hot, at rest."""
    sp, mech = mech9(chem_scale)
    nx, ny, nz = (n, n, n) if shape is None else shape
    N = nx * ny * nz
    X = _normalise_with_noise(PHI1_X, N, seed)
    idx = np.arange(N)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    r2 = (x - nx // 2) ** 2 + (y - ny // 2) ** 2 + (z - nz // 2) ** 2
    T = np.full(N, T_u)
    T[r2 < radius * radius] = T_hot
    name = f"sphere3d_{n}^3_M9" if shape is None else f"sphere3d_{nx}x{ny}x{nz}_M9"
    return Problem(name, LatticeSpec(nx, ny, nz, BC_PERIODIC), sp, mech,
                   InitFields(X=X, T=T, u=None, P=mech.P0), steps=1000)


def batched_flames_lengths(count: int = 48, seed: int = 48):
    """Lengths L ~ U{256..4096} and equivalence ratios phi ~ U[0.5, 3.0]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = rng.integers(256, 4097, size=count)
    phi = rng.uniform(0.5, 3.0, size=count)
    return L, phi


def batched_flames_problem(count: int = 48, seed: int = 48, ny: int = 4, nz: int = 4, lengths=None, phis=None,
                           T_u: float = MECH9_T_UNBURNT, T_slab: float = 1500.0, slab_frac: float = 0.2,
                           chem_scale: float = MECH9_CHEM_SCALE) -> Problem:
    """Independent quasi-1D flames side by side along x in one lattice.

    Flame k has L_k x ny x nz nodes (lengths and equivalence ratios from
    batched_flames_lengths(count, seed) unless given), each set up as
    flame1d_problem: its unburnt mixture at T_u, the rightmost slab_frac of
    its own x range at T_slab, uniform pressure, at rest, with ghost-node
    faces of its own on both x ends.  lattice.seg_nx holds the lengths.
    """
    if lengths is None or phis is None:
        L, ph = batched_flames_lengths(count, seed)
        lengths = L if lengths is None else lengths
        phis = ph if phis is None else phis
    lengths = [int(v) for v in lengths]
    phis = [float(v) for v in phis]
    sp, mech = mech9(chem_scale)
    nx = sum(lengths)
    N = nx * ny * nz
    xs = np.arange(N) % nx
    X = np.empty((9, N))
    T = np.full(N, T_u)
    x0 = 0
    for Lk, phk in zip(lengths, phis):
        sel = (xs >= x0) & (xs < x0 + Lk)
        X[:, sel] = _normalise_with_noise(phi_mixture(phk), 1, None)[:, :1]
        T[sel & (xs >= x0 + int(round((1.0 - slab_frac) * Lk)))] = T_slab
        x0 += Lk
    return Problem(f"flames{len(lengths)}_{nx}x{ny}x{nz}_M9",
                   LatticeSpec(nx, ny, nz, BC_EQ_ZEROGRAD_U0LEFT, seg_nx=lengths),
                   sp, mech, InitFields(X=np.ascontiguousarray(X), T=T, u=None, P=mech.P0), steps=5000)


def flame_of_batch(prob: Problem, k: int) -> Problem:
    """Flame k of a batched_flames_problem as a lattice of its own."""
    lat = prob.lattice
    x0 = sum(lat.seg_nx[:k])
    Lk = lat.seg_nx[k]
    N = lat.nx * lat.ny * lat.nz
    xs = np.arange(N) % lat.nx
    sel = (xs >= x0) & (xs < x0 + Lk)
    X = np.ascontiguousarray(prob.init.X[:, sel])
    T = np.ascontiguousarray(prob.init.T[sel])
    return Problem(f"{prob.name}_flame{k}", LatticeSpec(Lk, lat.ny, lat.nz, lat.bc_x), prob.species, prob.mech,
                   InitFields(X=X, T=T, u=None, P=prob.init.P), steps=prob.steps)



def node_states(M: int, n: int, seed: int = 2101, T_range=(700.0, 2600.0), rho_range=(0.2, 1.2),
                absent_frac: float = 0.1):
    """n seeded node states (rho_a [M, n], T [n]) for checks of the node
    functions (production rates, heat release and its derivatives).

    Draw order (numpy PCG64, one generator): T [n] uniform in T_range; total
    density [n] uniform in rho_range; log10 weights [n, M] uniform in
    [-6, 0]; absence flags [n, M] (uniform < absent_frac).  A species flagged
    absent gets weight 0, except the largest-weight species of each state;
    the weights are normalised per state to mass fractions and scaled by the
    total density.  Trace species span six decades and about one species in
    ten is exactly absent, so that products of concentrations with a zero
    factor occur.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.uniform(T_range[0], T_range[1], size=n)
    rho = rng.uniform(rho_range[0], rho_range[1], size=n)
    wts = 10.0 ** rng.uniform(-6.0, 0.0, size=(n, M))
    absent = rng.uniform(size=(n, M)) < absent_frac
    absent[np.arange(n), np.argmax(wts, axis=1)] = False
    wts[absent] = 0.0
    Y = wts / wts.sum(axis=1, keepdims=True)
    rho_a = np.ascontiguousarray((Y * rho[:, None]).T)
    return rho_a, np.ascontiguousarray(T)


def with_mixture_transport(species, X_ref, P_ref: float, T_ref: float, seed: int = 342,
                           nup_ref: float = 0.45, D_exp: float = 1.5):
    """A copy of species with seeded mixture-averaged transport (the stand-in
    for the paper's Cantera transport): species viscosities
    mu0_a = c sqrt(W_a) U[0.8, 1.2] at T_ref with exponents U[0.55, 0.65],
    c set so that their mole-fraction average over X_ref equals
    nup_ref * P_ref (so that 1/omega - 1/2 is near nup_ref in the reference
    mixture); binary diffusivities D_ab (T/T_ref)^D_exp (P_ref/P) from the
    species' constant D.  The exponents keep 1/omega - 1/2 within the
    scheme's stable window (about 0.4 to 1.5) over 300-2000 K."""
    import copy
    rng = np.random.Generator(np.random.PCG64(seed))
    sp = copy.deepcopy(species)
    W = np.asarray(sp.W, dtype=float)
    raw = np.sqrt(W) * rng.uniform(0.8, 1.2, size=W.size)
    X = np.asarray(X_ref, dtype=float)
    X = X / X.sum()
    sp.mu0 = raw * (nup_ref * P_ref / float(X @ raw))
    sp.mu_exp = rng.uniform(0.55, 0.65, size=W.size)
    sp.transport = TRANSPORT_MIXTURE_AVERAGED
    sp.T_tr = float(T_ref)
    sp.P_tr = float(P_ref)
    sp.D_exp = float(D_exp)
    return sp
