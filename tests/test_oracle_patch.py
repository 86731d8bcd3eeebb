"""The neighbourhood patches (tests/oracle_patch.py) reproduce the full
oracle lattice's moments at a node -- after initialisation (3x3x3) and
after two steps (15^3) -- bit for bit, including nodes on the periodic
wrap."""
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


def test_patch_after_two_steps_equals_full_lattice(orc):
    prob = w.sphere3d_problem(shape=(20, 19, 17), radius=5.0)
    o = orc.Oracle.from_problem(prob)
    assert o.step(2) == 0
    full = o.moments()
    c = 10 + 20 * (9 + 19 * 8)
    for node in (c, c + 4, c - 20 * 3 + 2, 0, 20 * 19 * 17 - 1):
        st = oracle_patch.node_state_after_steps(orc, prob, node, 2)
        assert np.array_equal(st["rho_a"], full["rho_a"][:, node]), node
        assert np.array_equal(st["rhou"], full["rhou"][:, node]), node
        assert st["rhoE"] == full["rhoE"][node] and st["T"] == full["T"][node], node
