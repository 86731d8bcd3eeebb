"""The kernels' float <-> double conversions on the integer pipe against
the hardware conversions, bit for bit: every float exponent with random
mantissas, zeros of both signs, subnormals, the largest and smallest
normals, Inf and NaN; doubles across the whole exponent range, at the
edges of the float range, and at exact rounding ties of both parities
(ties round to even) and one unit either side of them."""
import numpy as np
import pytest

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


def _floats(rng):
    exps = np.repeat(np.arange(256, dtype=np.uint32), 400)
    mant = rng.integers(0, 1 << 23, exps.size, dtype=np.uint32)
    mant[::400] = 0
    mant[1::400] = (1 << 23) - 1
    sign = rng.integers(0, 2, exps.size, dtype=np.uint32) << 31
    bits = sign | (exps << 23) | mant
    special = np.array([0, 0x80000000, 1, 0x80000001, 0x007fffff, 0x00800000, 0x7f7fffff, 0xff7fffff,
                        0x7f800000, 0xff800000, 0x7fc00000, 0x7f800001, 0x3f800000], dtype=np.uint32)
    return np.concatenate([bits, special]).view(np.float32)


def _doubles(rng):
    parts = []
    e = rng.integers(0, 2047, 400000).astype(np.uint64)
    m = rng.integers(0, 1 << 52, e.size, dtype=np.uint64)
    s = rng.integers(0, 2, e.size).astype(np.uint64) << np.uint64(63)
    parts.append(s | (e << np.uint64(52)) | m)
    # the float range and its edges: biased exponents 880..1170
    e = rng.integers(880, 1171, 400000).astype(np.uint64)
    m = rng.integers(0, 1 << 52, e.size, dtype=np.uint64)
    parts.append((e << np.uint64(52)) | m)
    # exact ties (dropped 29 bits = 1 followed by zeros) and their neighbours, both parities
    e = rng.integers(890, 1155, 100000).astype(np.uint64)
    hi = rng.integers(0, 1 << 23, e.size, dtype=np.uint64) << np.uint64(29)
    tie = (e << np.uint64(52)) | hi | np.uint64(1 << 28)
    parts += [tie, tie + np.uint64(1), tie - np.uint64(1), tie | np.uint64(1 << 29)]
    # carries into the exponent and overflow to Inf
    parts.append(np.array([(e_ << 52) | ((1 << 52) - 1) for e_ in (895, 896, 897, 1149, 1150, 1151)],
                          dtype=np.uint64))
    parts.append(np.array([0, 1 << 63, 1, (2047 << 52), (2047 << 52) | 1, (4095 << 52), (1023 << 52)],
                          dtype=np.uint64))
    return np.concatenate(parts).view(np.float64)


def _same_bits(a, b):
    an, bn = np.isnan(a), np.isnan(b)
    ok = an == bn
    both = ~an & ~bn
    ok[both] = a[both].view(np.uint64 if a.dtype == np.float64 else np.uint32)[...] == \
        b[both].view(np.uint64 if b.dtype == np.float64 else np.uint32)[...]
    return ok


def test_integer_conversions_equal_the_hardware_ones(lbm):
    import torch
    rng = np.random.default_rng(754)
    f = _floats(rng)
    d = _doubles(rng)
    n = max(f.size, d.size)
    f = np.resize(f, n)
    d = np.resize(d, n)
    fdev = torch.from_numpy(f.copy()).cuda()
    ddev = torch.from_numpy(d.copy()).cuda()
    fd = torch.empty(n, dtype=torch.float64, device="cuda")
    fd_ref = torch.empty_like(fd)
    df = torch.empty(n, dtype=torch.float32, device="cuda")
    df_ref = torch.empty_like(df)
    stream = torch.cuda.current_stream().cuda_stream
    st = lbm.lbm_convert_check(fdev.data_ptr(), fd.data_ptr(), fd_ref.data_ptr(), ddev.data_ptr(), df.data_ptr(),
                               df_ref.data_ptr(), n, stream)
    assert st == lbm.LBM_OK
    a, b = fd.cpu().numpy(), fd_ref.cpu().numpy()
    bad = ~_same_bits(a, b)
    assert not bad.any(), (f[bad][:5], a[bad][:5], b[bad][:5])
    a, b = df.cpu().numpy(), df_ref.cpu().numpy()
    bad = ~_same_bits(a, b)
    assert not bad.any(), (d[bad][:5], a[bad][:5], b[bad][:5])
    # the hardware reference is IEEE rounding: spot-check it against numpy's
    assert np.array_equal(b[np.isfinite(b)], d[np.isfinite(b)].astype(np.float32))
