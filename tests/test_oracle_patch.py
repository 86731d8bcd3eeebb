"""The 3x3x3 neighbourhood patch (tests/oracle_patch.py) reproduces the
full oracle lattice's moments at a node after initialisation, including
nodes on the periodic wrap."""
import numpy as np

import oracle_patch
import workload as w


def test_patch_equals_full_lattice(orc):
    prob = w.sphere3d_problem(shape=(11, 7, 6), radius=3.0)
    full = orc.Oracle.from_problem(prob).moments()
    for node in (0, 5, 11 * 7 * 6 - 1, 3 + 11 * (6 + 7 * 2), 10 + 11 * 3):
        st = oracle_patch.node_state_after_init(orc, prob, node)
        assert np.array_equal(st["rho_a"], full["rho_a"][:, node])
        assert np.array_equal(st["rhou"], full["rhou"][:, node])
        assert st["rhoE"] == full["rhoE"][node] and st["T"] == full["T"][node]
