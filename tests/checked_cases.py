"""Small lattices covering every index path of the kernels (periodic wrap,
ghost-node faces, ragged boxes, a batch of lattices side by side, two,
three and nine species), stepped through whichever library LBM_LIBRARY
names; writes the final populations and the step status of every case to
an .npz file.  Run as a script by tests/test_gpu_checked.py (once with the
bounds-checked build) and imported by it (the ordinary build)."""
import sys

import numpy as np

import workload as w
from workload.problem import InitFields, LatticeSpec, Problem, BC_EQ_ZEROGRAD_U0LEFT


def _ragged_three_gas():
    base = w.small_periodic_problem(n=3, seed=4, M3_rate_A=20.0)
    nx, ny, nz = 37, 5, 3
    N = nx * ny * nz
    rng = np.random.default_rng(4)
    X = np.array([[0.3], [0.5], [0.2]]) + rng.uniform(-0.1, 0.1, (3, N))
    X /= X.sum(axis=0, keepdims=True)
    T = 1.0 + rng.uniform(0, 0.5, N)
    u = rng.uniform(-0.01, 0.01, (3, N))
    return Problem("ragged", LatticeSpec(nx, ny, nz, BC_EQ_ZEROGRAD_U0LEFT), base.species, base.mech,
                   InitFields(X=X, T=T, u=u, P=base.init.P))


def cases():
    return {
        "sphere_periodic": (lambda: w.sphere3d_problem(shape=(20, 18, 17), radius=5.0), 8),
        "small_periodic": (lambda: w.small_periodic_problem(n=4, seed=3, M3_rate_A=20.0), 20),
        "ragged_ghost": (_ragged_three_gas, 20),
        "flame_ghost": (lambda: w.flame1d_problem(nx=200, ny=3, nz=2), 20),
        "batch": (lambda: w.batched_flames_problem(lengths=[5, 37, 64, 2, 129], phis=[0.6, 1.0, 2.5, 1.2, 0.8]), 20),
    }


def run(lbm):
    out = {}
    for name, (make, steps) in cases().items():
        prob = make()
        for mode, p in (("fp64", lbm.LBM_FP64), ("mixed", lbm.LBM_MIXED), ("fast", lbm.LBM_MIXED_FAST)):
            s = lbm.Solver.from_problem(prob, precision=p)
            out[f"{name}_{mode}_status"] = np.array([s.step(steps, check=False)])
            out[f"{name}_{mode}_pop"] = s.populations()
            s.close()
    return out


if __name__ == "__main__":
    from paper_2101_01702_gb300 import lbm
    np.savez(sys.argv[1], **run(lbm))
