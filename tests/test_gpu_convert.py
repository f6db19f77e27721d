"""The FP32 <-> FP64 conversions of the step kernels (bh_prim_split2).

Every step splits each body's FP64 coordinates into a float pair and widens
each FP32 acceleration to FP64 (the FP64 state of §3.1 with FP32 arithmetic
in cell-relative coordinates, §3.2).  The library does both on the integer
units, written from the IEEE 754 formats, because GB300's FP64 pipe bounds
the step kernels otherwise.  This test holds them to IEEE 754 as numpy
implements it: hi = x rounded to the nearest float with ties to even,
lo = (x - hi) rounded the same way, and the exact widening of a float.
Bit for bit in the normal float range, at ties and next to them, at the
overflow threshold, for zeros and for floats that are exactly
representable.  Results that are subnormal floats may be flushed to a zero of
the same sign (the library is built with flush-to-zero).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _x_cases(rng):
    f32 = np.float32
    xs = []
    # magnitudes over the whole float range and past it, both signs
    e = rng.uniform(-160.0, 140.0, 40000)
    xs.append(np.sign(rng.uniform(-1, 1, e.size)) * np.exp2(e))
    # coordinates like the bodies' (|x| up to a few hundred), float-exact ones too
    xs.append(rng.normal(0.0, 30.0, 40000))
    xs.append(rng.normal(0.0, 30.0, 5000).astype(f32).astype(np.float64))
    # exact ties between neighbouring floats, and one FP64 ulp either side
    f = rng.normal(0.0, 10.0, 5000).astype(f32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2
    xs += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf)]
    # the largest float, the overflow threshold (half an ulp above it) and beyond
    fmax = float(np.finfo(f32).max)
    half_ulp = 2.0 ** (127 - 24)
    xs.append(np.array([fmax, -fmax, fmax + half_ulp, np.nextafter(fmax + half_ulp, 0.0),
                        fmax + 2 * half_ulp, 1e39, -1e39]))
    # the smallest normal float and below; zeros; infinities
    tiny = float(np.finfo(f32).tiny)
    xs.append(np.array([tiny, -tiny, np.nextafter(tiny, 0.0), tiny / 2, 1e-40, -1e-45, 1e-50, 0.0, -0.0,
                        np.inf, -np.inf]))
    return np.concatenate(xs)


def _f_cases(rng, n):
    # float bit patterns of every kind (normals, subnormals, zeros, infinities, NaNs), n of them
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x807fffff, 0x00400000, 0x7f7fffff, 0x7f800000,
                        0xff800000, 0x00800000, 0x3f800000], dtype=np.uint32)
    bits = rng.integers(0, 1 << 32, n - special.size, dtype=np.uint64).astype(np.uint32)
    return np.concatenate([bits, special]).view(np.float32)


def _subnormal32(v):
    v = np.asarray(v, dtype=np.float32)
    return (v != 0) & (np.abs(v) < np.finfo(np.float32).tiny)


def test_split_and_widen_match_ieee(cuda_lib):
    import torch

    rng = np.random.default_rng(17)
    x = _x_cases(rng)
    f = _f_cases(rng, x.size)
    hi, lo, wide = cuda_lib.split2(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    hi, lo, wide = hi.cpu().numpy(), lo.cpu().numpy(), wide.cpu().numpy()

    with np.errstate(over="ignore", invalid="ignore"):
        hi_ref = x.astype(np.float32)
    # hi: bit for bit, except that a subnormal float may come back as a signed zero
    flushed = _subnormal32(hi_ref) & (hi == 0) & (np.signbit(hi) == np.signbit(hi_ref))
    same_hi = hi.view(np.uint32) == hi_ref.view(np.uint32)
    assert np.all(same_hi | flushed), x[~(same_hi | flushed)][:5]
    # the normal range is exact: no flush allowed there
    normal = np.isfinite(hi_ref) & ~_subnormal32(hi_ref) & (hi_ref != 0)
    assert np.all(same_hi[normal])
    assert normal.sum() > 50000
    # lo: the rest x - hi (exact in FP64) rounded, where hi is finite
    fin = np.isfinite(hi)
    with np.errstate(over="ignore", invalid="ignore"):
        lo_ref = (x[fin] - hi[fin].astype(np.float64)).astype(np.float32)
    got = lo[fin]
    ok = (got.view(np.uint32) == lo_ref.view(np.uint32)) | (_subnormal32(lo_ref) & (got == 0))
    assert np.all(ok), x[fin][~ok][:5]
    # hi + lo carries x to about 2^-48 relative; above 2^-60 a flushed
    # subnormal lo (below 2^-126) stays inside that bound too
    both = normal & (np.abs(x) > 2.0 ** -60)
    r = np.abs(hi[both].astype(np.float64) + lo[both].astype(np.float64) - x[both])
    assert np.all(r <= 2.0 ** -47 * np.abs(x[both]))

    # widening: exact for every float, subnormals included; NaN stays NaN
    with np.errstate(invalid="ignore"):
        wide_ref = f.astype(np.float64)
    nan = np.isnan(f)
    assert np.array_equal(np.isnan(wide), nan)
    assert np.array_equal(wide[~nan].view(np.uint64), wide_ref[~nan].view(np.uint64))
    assert np.count_nonzero(_subnormal32(f)) > 0


def test_split2_argument_checks(cuda_lib):
    import torch

    lib = cuda_lib.load()
    assert lib.bh_prim_split2(None, None, 0, None, None, None, None) == 0
    assert lib.bh_prim_split2(None, None, -1, None, None, None, None) == 1
    assert lib.bh_prim_split2(None, None, 5, None, None, None, None) == 1
    with pytest.raises(ValueError):
        cuda_lib.split2(torch.zeros(4, dtype=torch.float32, device="cuda"),
                        torch.zeros(4, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        cuda_lib.split2(torch.zeros(4, dtype=torch.float64, device="cuda"),
                        torch.zeros(3, dtype=torch.float32, device="cuda"))
