"""Launch shapes do not change results: the autotuner (lbm_autotune) and
explicitly set block sizes (lbm_set_blocks, every candidate, including the
256-thread production-rate kernel with more than 48 KB of shared memory)
give populations bit for bit equal to the default blocks, and tuning leaves
the current state untouched.  Periodic box and a batch of ragged flames
with ghost faces, in double and mixed precision."""
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


PROBLEMS = {
    "sphere": lambda: w.sphere3d_problem(shape=(25, 23, 21), radius=6.0),
    "flames": lambda: w.batched_flames_problem(lengths=[37, 64, 129], phis=[0.6, 1.0, 2.5]),
}


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["sphere", "flames"])
def test_autotune_and_set_blocks_keep_results(lbm, mode, case):
    prob = PROBLEMS[case]()
    p = lbm.LBM_FP64 if mode == "fp64" else lbm.LBM_MIXED
    ref = lbm.Solver.from_problem(prob, precision=p)
    ref.step(12)
    want = ref.populations()
    ref.close()

    a = lbm.Solver.from_problem(prob, precision=p)
    a.step(5)
    before = a.populations()
    chosen = a.autotune(trials=2)
    assert np.array_equal(a.populations(), before)       # tuning leaves the state as it was
    assert chosen["ghost"] == 128 and chosen["moments"] in (64, 128) and chosen["species_collision"] in (64, 128)
    assert all(chosen[k] in (64, 128, 256) for k in ("rates", "gradients", "energy_collision"))
    a.step(7)
    assert np.array_equal(a.populations(), want)
    a.close()

    for blocks in ([128, 64, 64, 64, 64, 64], [128, 128, 256, 256, 256, 128]):
        b = lbm.Solver.from_problem(prob, precision=p)
        b.set_blocks(blocks)
        b.step(12)
        assert np.array_equal(b.populations(), want), blocks
        b.close()


def test_set_blocks_rejects_invalid_shapes(lbm):
    prob = PROBLEMS["sphere"]()
    s = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    for bad in ([128, 256, 128, 128, 128, 128], [128, 128, 96, 128, 128, 128], [64, 128, 128, 128, 128, 128],
                [128, 128, 128, 128, 128, 256]):
        with pytest.raises(lbm.LBMError) as e:
            s.set_blocks(bad)
        assert e.value.status == lbm.LBM_ERR_ARG
    s.close()
