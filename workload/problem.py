"""Plain containers describing one lattice Boltzmann problem instance.

Everything is stored in lattice units (grid spacing and time step equal to
one).  Arrays are numpy, float64 or int32, C-contiguous.  Node index
convention used by every array of length N: n = x + nx * (y + ny * z).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

BC_PERIODIC = 0
BC_EQ_ZEROGRAD_U0LEFT = 1

THERMO_CONST_CP = 0
THERMO_POLY7 = 1

VISC_KINEMATIC = 0
VISC_RELAXATION = 1

TRANSPORT_CONSTANT = 0
TRANSPORT_MIXTURE_AVERAGED = 1

RXN_ELEMENTARY = 0
RXN_THIRD_BODY = 1
RXN_FALLOFF = 2


@dataclass
class LatticeSpec:
    nx: int
    ny: int
    nz: int
    bc_x: int = BC_PERIODIC  # y and z are always periodic
    # independent lattices side by side in x (lengths summing to nx), each
    # with its own boundary faces; None for a single lattice
    seg_nx: Optional[list] = None

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class SpeciesSpec:
    """Species, thermodynamics and transport.

    The last species (index M-1) is the one slaved to the mixture set.
    thermo == THERMO_CONST_CP: U_a(T) = h_form[a] - R_a*T0 + (cp_R[a]-1)*R_a*(T-T0)
    thermo == THERMO_POLY7:    single-range 7-coefficient cp/R, h/RT, s/R form.
    D[a][b] are the binary diffusivities, nu the kinematic viscosity and Pr
    the Prandtl number, all constant in lattice units.  r_lat is the universal
    gas constant in lattice units, so R_a = r_lat / W[a].
    visc_model == VISC_KINEMATIC: nu is a constant kinematic viscosity,
        mu = rho nu, so 1/omega - 1/2 = nu / (R T).
    visc_model == VISC_RELAXATION: nu is the constant 1/omega - 1/2, i.e.
        mu = nu P (a constant-relaxation-time gas).
    transport == TRANSPORT_MIXTURE_AVERAGED replaces nu, Pr and the
        constant D by mixture-averaged coefficients: species viscosities
        mu0[a] (T/T_tr)^mu_exp[a], Wilke's rule for the mixture viscosity,
        modified Eucken species conductivities with the Mathur-Tondon-Saxena
        average, and binary diffusivities D[a][b] (T/T_tr)^D_exp (P_tr/P).
    """
    names: list
    W: np.ndarray          # [M] molar masses
    thermo: int
    cp_R: np.ndarray       # [M] (CONST_CP)
    h_form: np.ndarray     # [M] mass-specific formation enthalpy at T0 (CONST_CP)
    T0: float
    poly7: np.ndarray      # [M,7] (POLY7)
    D: np.ndarray          # [M,M]
    nu: float
    Pr: float
    r_lat: float
    elements: np.ndarray   # [E,M] element counts per species (test bookkeeping)
    element_names: list
    visc_model: int = 0
    transport: int = 0
    mu0: Optional[np.ndarray] = None      # [M]
    mu_exp: Optional[np.ndarray] = None   # [M]
    T_tr: float = 1.0
    D_exp: float = 1.5
    P_tr: float = 1.0

    @property
    def M(self) -> int:
        return int(self.W.shape[0])


@dataclass
class MechanismSpec:
    """Reaction mechanism.

    Forward rate coefficient k = exp(log_A + b*ln(T/T_ref) - theta/T) in
    lattice units (concentrations c_a = rho_a / W_a).  rtype 1 multiplies the
    rate of progress by [M] = sum_a eff[k,a] c_a; rtype 2 is a Lindemann
    falloff whose low-pressure coefficient uses low[k] = (log_A0, b0, theta0).
    Reversible reactions use K_c from the species Gibbs energies at the
    standard pressure P0 (lattice units).
    """
    nu_f: np.ndarray       # [R,M] int32 reactant stoichiometry
    nu_r: np.ndarray       # [R,M] int32 product stoichiometry
    log_A: np.ndarray      # [R]
    b: np.ndarray          # [R]
    theta: np.ndarray      # [R]
    rtype: np.ndarray      # [R] int32
    eff: np.ndarray        # [R,M]
    low: np.ndarray        # [R,3]
    reversible: np.ndarray  # [R] int32
    T_ref: float
    P0: float

    @property
    def R(self) -> int:
        return int(self.log_A.shape[0])


@dataclass
class InitFields:
    """Initial primitive fields; populations start at their equilibria."""
    X: np.ndarray          # [M,N] mole fractions
    T: np.ndarray          # [N]
    u: Optional[np.ndarray]  # [3,N] or None (fluid at rest)
    P: float               # uniform pressure


@dataclass
class Problem:
    name: str
    lattice: LatticeSpec
    species: SpeciesSpec
    mech: MechanismSpec
    init: InitFields
    steps: int = 0
    notes: dict = field(default_factory=dict)
