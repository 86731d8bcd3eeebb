"""The state that the first collision sees at one node of a periodic
lattice right after initialisation, computed by the oracle alone.

A 3x3x3 periodic oracle lattice is initialised with the node's
neighbourhood of the initial fields (with the periodic wrap of the full
lattice); its centre pulls exactly the populations that the node pulls in
the full lattice, so the oracle's moments at the centre are the node's."""
import numpy as np

from workload.problem import BC_PERIODIC, LatticeSpec


def neighbourhood(lat, node):
    """Full-lattice indices of the 27 patch nodes, patch order x fastest."""
    nx, ny, nz = lat.nx, lat.ny, lat.nz
    x, y, z = node % nx, (node // nx) % ny, node // (nx * ny)
    idx = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
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
