"""Error of the mixed-precision steps (float moving populations; double
rest and energy populations, temperature, and -- in LBM_MIXED -- Stefan-
Maxwell solve and chemistry) after 1000 steps, against the double
GPU path on the 1D flame (4096x4x4, ghost nodes) and against the FP64 CPU
oracle on the 32^3 expanding-flame instance.  Target: 1e-4 relative error
in mass fractions (each species normalised by its maximum) and
temperature."""
import json
import os

import numpy as np
import pytest

import workload as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _errors(m, ref, M):
    err = {"T": float(np.abs(m["T"] - ref["T"]).max() / np.abs(ref["T"]).max())}
    for a in range(M):
        err[f"Y{a}"] = float(np.abs(m["Y"][a] - ref["Y"][a]).max() / np.abs(ref["Y"][a]).max())
    return err


def _report(name, err):
    out = os.environ.get("LBM_ERROR_REPORT")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({"case": name, "errors": err}) + "\n")


MODES = ["mixed", "mixed_fast"]


def _mode(lbm, name):
    return lbm.LBM_MIXED if name == "mixed" else lbm.LBM_MIXED_FAST


@pytest.mark.parametrize("mode", MODES)
def test_mixed_vs_double_flame1d_1000_steps(lbm, mode):
    prob = w.flame1d_problem(nx=4096)
    mask = lbm.LBM_F_T | lbm.LBM_F_Y
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    ref.step(1000)
    r = ref.moments(mask)
    ref.close()
    mix = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
    mix.step(1000)
    m = mix.moments(mask)
    mix.close()
    err = _errors(m, r, 9)
    _report(f"flame1d_4096x4x4_1000_{mode}_vs_fp64gpu", err)
    assert max(err.values()) <= 1e-4, err


@pytest.fixture(scope="module")
def oracle_sphere32_1000(orc):
    prob = w.sphere3d_problem(n=32, radius=8.0)
    o = orc.Oracle.from_problem(prob)
    assert o.step(1000) == 0
    return prob, o.moments()


@pytest.mark.parametrize("mode", MODES)
def test_mixed_vs_oracle_sphere32_1000_steps(oracle_sphere32_1000, lbm, mode):
    prob, ref = oracle_sphere32_1000
    mix = lbm.Solver.from_problem(prob, precision=_mode(lbm, mode))
    mix.step(1000)
    m = mix.moments(lbm.LBM_F_T | lbm.LBM_F_Y)
    mix.close()
    err = _errors(m, ref, 9)
    _report(f"sphere3d_32^3_1000_{mode}_vs_oracle", err)
    assert max(err.values()) <= 1e-4, err
