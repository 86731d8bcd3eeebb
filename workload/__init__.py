"""Seeded synthetic inputs for the reactive-mixture lattice Boltzmann step.

This package is the single source of inputs shared by the CPU oracle and the
CUDA path.  It holds no arithmetic of the method itself: it draws mechanism
parameters, thermodynamic polynomial coefficients and initial primitive
fields (mole fractions, temperature, velocity, pressure) from fixed seeds.
Turning those fields into populations, moments, rates or temperatures is left
to each implementation.
"""
from .problem import Problem, LatticeSpec, SpeciesSpec, MechanismSpec, InitFields  # noqa: F401
from .configs import (  # noqa: F401
    config1_problem,
    flame1d_problem,
    adjoint_flame_problem,
    circular_flame_problem,
    sphere3d_problem,
    small_periodic_problem,
    batched_flames_lengths,
    batched_flames_problem,
    flame_of_batch,
    mech9,
    mech3,
    node_states,
    with_mixture_transport,
)
