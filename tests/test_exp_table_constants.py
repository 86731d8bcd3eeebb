"""The constants of the kernels' table-driven exponential, re-derived from
the mathematics: 2^(j/256) rounded to the nearest double for j = 0..255,
the split ln2/256 = L1 + L2 with L1 of at most 35 significant bits (so that
N L1 is exact for |N| < 2^18, i.e. |x| < 707), and the high word of 707
used by the range test.  Read from the kernel source as text."""
import math
import re
from pathlib import Path

import pytest

mp = pytest.importorskip("mpmath")

SRC = Path(__file__).resolve().parents[1] / "paper_2101_01702_gb300" / "csrc" / "lbm_kernels.cuh"


def _table():
    text = SRC.read_text()
    body = text[text.index("c_exp2_256[256] = {"):]
    body = body[:body.index("};")]
    return [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", body)]


def test_table_is_two_to_the_j_over_256_correctly_rounded():
    mp.mp.dps = 50
    tab = _table()
    assert len(tab) == 256
    for j, v in enumerate(tab):
        exact = mp.mpf(2) ** (mp.mpf(j) / 256)
        assert v == float(exact), j
        assert abs(mp.mpf(v) - exact) <= mp.mpf(2) ** -53 * exact


def test_reduction_constants():
    import struct
    mp.mp.dps = 50
    text = SRC.read_text()
    fn = text[text.index("double exp_table(double x)"):]
    fn = fn[:fn.index("\n}\n")]
    consts = [float.fromhex(h) for h in re.findall(r"-?0x[0-9a-f.]+p[+-]\d+", fn)]
    inv, L1, L2 = consts[0], consts[1], consts[2]
    assert inv == float(256 / mp.log(2))
    ln2_256 = mp.log(2) / 256
    # L2 is ln2/256 - L1 rounded once: within half an ulp of L2 (2^-97)
    assert abs(mp.mpf(L1) + mp.mpf(L2) - ln2_256) <= mp.mpf(2) ** -98
    m, e = mp.frexp(mp.mpf(L1))
    assert (m * 2 ** 35) == int(m * 2 ** 35)          # at most 35 significant bits
    assert 707 * 256 / math.log(2) < 2 ** 18           # N L1 exact over the table's range
    hi = struct.unpack(">Q", struct.pack(">d", 707.0))[0] >> 32
    assert "0x%08x" % hi in fn.lower()
