"""Index safety: the library rebuilt with LBMK_CHECKED=1 checks every index
its kernels derive from the lattice geometry (pulls from neighbours and
ghost planes, stencil neighbours, ghost-node sources, batch ranges) and
reports LBM_ERR_BOUNDS instead of reading outside a buffer.  On small
lattices that exercise every index path (periodic, ghost faces, ragged
boxes, a batch including one- and two-node-long lattices; three and nine
species; all precisions) it must report no error and give populations bit
for bit equal to the ordinary build's: the checks change no arithmetic."""
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def test_checked_build_reports_no_bounds_error_and_matches(lbm, tmp_path):
    from paper_2101_01702_gb300 import build
    checked = build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, LBM_LIBRARY=str(checked), PYTHONPATH=str(ROOT) + os.pathsep + str(ROOT / "tests"))
    r = subprocess.run([sys.executable, str(ROOT / "tests" / "checked_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    sys.path.insert(0, str(ROOT / "tests"))
    import checked_cases
    plain = checked_cases.run(lbm)
    got = np.load(out)
    for key in plain:
        if key.endswith("_status"):
            assert int(got[key][0]) == lbm.LBM_OK, (key, int(got[key][0]))
            assert int(plain[key][0]) == lbm.LBM_OK, key
        else:
            assert np.array_equal(got[key], plain[key]), key
