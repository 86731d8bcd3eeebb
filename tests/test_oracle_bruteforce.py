"""Brute-force agreement on 4^3 lattices: the oracle's step against an
independent multi-precision restatement (tests/bruteforce_lbm.py) of the
same equations, on random perturbed states of the three-gas workload."""
import numpy as np
import pytest

import workload as w
from bruteforce_lbm import BruteForce, VELS

import mpmath as mp


def _to_dict(pop, shape):
    nx, ny, nz = shape
    out = {}
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                n = x + nx * (y + ny * z)
                sets = []
                for s in range(pop.shape[1]):
                    sets.append({c: mp.mpf(float(pop[n, s, (c[0] + 1) + 3 * (c[1] + 1) + 9 * (c[2] + 1)]))
                                 for c in VELS})
                out[(x, y, z)] = sets
    return out


def _to_array(d, shape, S):
    nx, ny, nz = shape
    a = np.zeros((nx * ny * nz, S, 27))
    for (x, y, z), sets in d.items():
        n = x + nx * (y + ny * z)
        for s in range(S):
            for c, v in sets[s].items():
                a[n, s, (c[0] + 1) + 3 * (c[1] + 1) + 9 * (c[2] + 1)] = float(v)
    return a


@pytest.mark.parametrize("seed", [7, 8])
def test_bruteforce_4cubed(orc, seed):
    p = w.small_periodic_problem(n=4, seed=seed, M3_rate_A=20.0)
    sp, mech = p.species, p.mech
    o = orc.Oracle.from_problem(p)
    params = dict(W=sp.W, cp_R=sp.cp_R, h_form=sp.h_form, T0=sp.T0, D=sp.D, nu=sp.nu, Pr=sp.Pr,
                  r_lat=sp.r_lat,
                  reactions=[(mech.log_A[k], mech.b[k], mech.theta[k], mech.nu_f[k], mech.nu_r[k],
                              mech.T_ref) for k in range(mech.R)])
    shape = (4, 4, 4)
    bf = BruteForce(shape, params)
    state = _to_dict(o.get_pop(), shape)
    for _ in range(2):
        state = bf.step(state)
        assert o.step(1) == 0
        ref = _to_array(state, shape, o.S)
        got = o.get_pop()
        for s in range(o.S):
            scale = np.abs(ref[:, s]).max()
            assert np.abs(got[:, s] - ref[:, s]).max() <= 1e-13 * scale, s


def test_bruteforce_ghost_boundaries(orc):
    """Equilibrium zero-gradient ghost nodes at both x ends, zero velocity on
    the left (Sec. 5a), on a 5x3x3 lattice."""
    p = w.small_periodic_problem(n=3, seed=9, M3_rate_A=20.0)
    from workload.problem import LatticeSpec, BC_EQ_ZEROGRAD_U0LEFT
    nx = 5
    rng = np.random.default_rng(9)
    N = nx * 9
    X = np.array([[0.3], [0.5], [0.2]]) + rng.uniform(-0.1, 0.1, (3, N))
    X /= X.sum(axis=0, keepdims=True)
    T = 1.0 + rng.uniform(0, 0.5, N)
    u = rng.uniform(-0.02, 0.02, (3, N))
    sp, mech = p.species, p.mech
    lat = LatticeSpec(nx, 3, 3, BC_EQ_ZEROGRAD_U0LEFT)
    o = orc.Oracle(lat, sp, mech)
    o.init(X, T, u, p.init.P)
    params = dict(W=sp.W, cp_R=sp.cp_R, h_form=sp.h_form, T0=sp.T0, D=sp.D, nu=sp.nu, Pr=sp.Pr,
                  r_lat=sp.r_lat,
                  reactions=[(mech.log_A[k], mech.b[k], mech.theta[k], mech.nu_f[k], mech.nu_r[k],
                              mech.T_ref) for k in range(mech.R)])
    shape = (nx, 3, 3)
    bf = BruteForce(shape, params, bc_x=1)
    state = _to_dict(o.get_pop(), shape)
    for _ in range(2):
        state = bf.step(state)
        assert o.step(1) == 0
        ref = _to_array(state, shape, o.S)
        got = o.get_pop()
        for s in range(o.S):
            scale = np.abs(ref[:, s]).max()
            assert np.abs(got[:, s] - ref[:, s]).max() <= 1e-13 * scale, s
