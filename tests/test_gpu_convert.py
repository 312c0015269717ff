"""The FP32 kernels' integer FP32 <-> FP64 conversions (hfv_convert) against
the hardware conversion and numpy's IEEE 754 round-to-nearest-even, bit for
bit, on random bit patterns (every exponent, NaN, infinity, subnormals) and
on the cases a rounding mistake shows first: exact ties with an even and an
odd kept fraction, one unit either side of a tie, all-ones fractions whose
rounding carries into the exponent (up to infinity past the largest float)
and the boundary to the FP32 subnormals."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25906_gb300 import hfv
    hfv.load()
    return hfv


def _doubles(rng):
    n = 1 << 20
    parts = [rng.integers(0, 2**64, n, dtype=np.uint64)]                  # any bit pattern
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    frac = rng.integers(0, 2**52, n, dtype=np.uint64)
    exp = rng.integers(890, 1160, n, dtype=np.uint64) << np.uint64(52)   # around the float range
    parts.append(sign | exp | frac)
    # ties and their neighbours: the 29 dropped bits are 0x10000000 (+-1)
    hi = (sign | exp | (frac & ~np.uint64(0x1FFFFFFF)))
    for d in (0, 1, -1):
        parts.append(hi | np.uint64(0x10000000 + d))
    # all-ones kept fractions with a round-up remainder: carries into the exponent
    ones = sign | exp | np.uint64(0xFFFFFFFFFFFFF)
    parts.append(ones)
    edge = []
    for e in (896, 897, 898, 1149, 1150, 1151, 0, 2047):
        for f in (0, 1, 0x10000000, 0x10000001, 0xFFFFFFFFFFFFF, 0xFFFFFE0000000, 0xFFFFFF0000000, 0xFFFFFEFFFFFFF):
            for s in (0, 1):
                edge.append((s << 63) | (e << 52) | f)
    parts.append(np.array(edge, dtype=np.uint64))
    return np.concatenate(parts).view(np.float64)


def _floats(rng):
    n = 1 << 22
    parts = [rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)]
    edge = []
    for e in (0, 1, 2, 126, 127, 253, 254, 255):
        for f in (0, 1, 2, 0x400000, 0x7FFFFF):
            for s in (0, 1):
                edge.append((s << 31) | (e << 23) | f)
    parts.append(np.array(edge, dtype=np.uint32))
    return np.concatenate(parts).view(np.float32)


def test_fp64_to_fp32_matches_the_hardware_and_ieee_rounding(H):
    x = _doubles(np.random.default_rng(20251029))
    xd = torch.from_numpy(x).cuda()
    ours = H.convert(xd)
    hw = xd.to(torch.float32)
    torch.cuda.synchronize()
    a = ours.view(torch.int32).cpu().numpy()
    b = hw.view(torch.int32).cpu().numpy()
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, [(x.view(np.uint64)[i], a[i], b[i]) for i in bad[:8]]
    with np.errstate(over="ignore", invalid="ignore"):   # signalling NaNs raise "invalid" on some hosts
        ref = x.astype(np.float32)
    fin = ~np.isnan(x)
    assert np.array_equal(a[fin], ref.view(np.int32)[fin])


def test_fp32_to_fp64_is_exact(H):
    x = _floats(np.random.default_rng(20251030))
    xf = torch.from_numpy(x).cuda()
    ours = H.convert(xf)
    hw = xf.to(torch.float64)
    torch.cuda.synchronize()
    a = ours.view(torch.int64).cpu().numpy()
    b = hw.view(torch.int64).cpu().numpy()
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, [(x.view(np.uint32)[i], a[i], b[i]) for i in bad[:8]]
    fin = ~np.isnan(x)
    with np.errstate(invalid="ignore"):
        ref = x.astype(np.float64)
    assert np.array_equal(a[fin], ref.view(np.int64)[fin])


def test_convert_rejects_bad_arguments(H):
    lib = H.load()
    assert lib.hfv_convert(2, 4, None, None, None) == H.HFV_ERR_ARG
    assert lib.hfv_convert(1, -1, None, None, None) == H.HFV_ERR_ARG
    assert lib.hfv_convert(1, 4, None, None, None) == H.HFV_ERR_ARG
    assert lib.hfv_convert(1, 0, None, None, None) == H.HFV_OK


def test_fp64_reciprocal_within_one_ulp(H):
    """The FP64 kernels' reciprocal (hardware seed and two Newton-Raphson
    steps) against numpy's correctly rounded 1/x: at most one ulp apart over
    normal inputs of either sign whose reciprocals are normal, and exact on
    powers of two."""
    rng = np.random.default_rng(20251031)
    n = 1 << 20
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-1000, 1000, n)
    sign = np.where(rng.integers(0, 2, n) == 1, -1.0, 1.0)
    x = sign * np.ldexp(mant, expo)
    x = np.concatenate([x, np.ldexp(1.0, np.arange(-1000, 1001)), -np.ldexp(1.0, np.arange(-1000, 1001)),
                        [1.0, 3.0, 7.0, 0.1, 1.0 / 3.0, 1.4, 0.4]])
    got = H.rcp64(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    ulps = np.abs(got - ref) / np.spacing(np.abs(ref))
    worst = int(np.argmax(ulps))
    assert ulps.max() <= 1.0, (x[worst], got[worst], ref[worst], ulps.max())
    p2 = np.abs(np.log2(np.abs(x)) - np.round(np.log2(np.abs(x)))) == 0
    assert np.array_equal(got[p2], ref[p2])
    print(f"reciprocal: max {ulps.max():.2f} ulp, {np.mean(ulps > 0) * 100:.2f} % not correctly rounded")
