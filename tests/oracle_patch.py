"""The state that a collision sees at one node of a periodic lattice,
right after initialisation or after a few steps, computed by the oracle
alone.

A (2h+1)^3 periodic oracle lattice is initialised with the node's
neighbourhood of the initial fields (with the periodic wrap of the full
lattice).  One step at a node reads the initial fields within 3 nodes (the
pull, the gradient of Phi at the neighbours, X = -grad G), so after k steps
the patch nodes within h - 3k of the centre hold exactly the full
lattice's post-collision state, and the moments the next collision sees at
the centre (one more pull) are the node's when h >= 3k + 1."""
import numpy as np

from workload.problem import BC_PERIODIC, LatticeSpec


def neighbourhood(lat, node, h=1):
    """Full-lattice indices of the (2h+1)^3 patch nodes, patch order x fastest."""
    nx, ny, nz = lat.nx, lat.ny, lat.nz
    x, y, z = node % nx, (node // nx) % ny, node // (nx * ny)
    r = range(-h, h + 1)
    idx = []
    for dz in r:
        for dy in r:
            for dx in r:
                idx.append((x + dx) % nx + nx * ((y + dy) % ny + ny * ((z + dz) % nz)))
    return np.array(idx)


def node_state_after_init(orc, prob, node):
    """dict rho_a [M], rhou [3], rhoE, T of the node (oracle moments)."""
    assert prob.lattice.bc_x == BC_PERIODIC
    idx = neighbourhood(prob.lattice, node)
    o = orc.Oracle(LatticeSpec(3, 3, 3, BC_PERIODIC), prob.species, prob.mech)
    ini = prob.init
    u = None if ini.u is None else ini.u[:, idx]
    assert o.init(ini.X[:, idx], ini.T[idx], u, ini.P) == 0
    m = o.moments()
    assert m["status"] == 0
    c = 13
    return {"rho_a": m["rho_a"][:, c].copy(), "rhou": m["rhou"][:, c].copy(), "rhoE": float(m["rhoE"][c]),
            "T": float(m["T"][c])}


def node_state_after_steps(orc, prob, node, steps):
    """Moments rho_a [M], rhou [3], rhoE, T that the collision of step
    steps + 1 sees at the node, from a (6 steps + 3)^3 periodic patch."""
    assert prob.lattice.bc_x == BC_PERIODIC
    h = 3 * steps + 1
    idx = neighbourhood(prob.lattice, node, h)
    w = 2 * h + 1
    o = orc.Oracle(LatticeSpec(w, w, w, BC_PERIODIC), prob.species, prob.mech)
    ini = prob.init
    u = None if ini.u is None else ini.u[:, idx]
    assert o.init(ini.X[:, idx], ini.T[idx], u, ini.P) == 0
    assert o.step(steps) == 0
    m = o.moments()
    assert m["status"] == 0
    c = (w * w * w) // 2
    return {"rho_a": m["rho_a"][:, c].copy(), "rhou": m["rhou"][:, c].copy(), "rhoE": float(m["rhoE"][c]),
            "T": float(m["T"][c])}
