"""The set-up's cube root (CIE companding): Newton-Raphson on the reciprocal
cube root from a bit-pattern start, two steps and one correction, emulated
step by step in FP32 (products and fused multiply-adds rounded as the device
rounds them) and compared with the exact root on a dense sample of its range
[(6/29)^3, 1]: less than one ulp everywhere."""
import numpy as np

START = 0x54A232A0


def _fma(a, b, c):
    # a*b is exact in FP64 for FP32 inputs; one rounding to FP32 after the sum
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _cube_root_fp32(t):
    third = np.float32(1.0) / np.float32(3.0)
    y = (np.uint32(START) - t.view(np.uint32) // np.uint32(3)).view(np.float32)
    for _ in range(2):
        y = (y * _fma(-t, (y * y) * y, np.float32(4.0))) * third
    y2 = y * y
    c = t * y2
    return _fma(_fma(-c, c * c, t), y2 * third, c)


def _range_sample(step):
    lo = np.float32((6.0 / 29.0) ** 3).view(np.uint32)
    hi = np.float32(1.0001).view(np.uint32)
    bits = np.concatenate([np.arange(lo, hi, step, dtype=np.uint32), np.array([lo, hi], np.uint32)])
    return bits.view(np.float32)


def test_cube_root_within_one_ulp():
    t = _range_sample(5)
    exact = np.cbrt(t.astype(np.float64))
    got = _cube_root_fp32(t).astype(np.float64)
    ulp = np.spacing(exact.astype(np.float32)).astype(np.float64)
    err = np.abs(got - exact) / ulp
    assert err.max() < 1.0, err.max()
    # most results are the correctly rounded root
    assert (err <= 0.5).mean() > 0.9


def test_start_error_bound():
    """The start constant keeps the first guess within 3.5% of t^(-1/3), the
    error two quadratic steps take below FP32 resolution."""
    t = _range_sample(97)
    y0 = (np.uint32(START) - t.view(np.uint32) // np.uint32(3)).view(np.float32).astype(np.float64)
    rel = np.abs(y0 * np.cbrt(t.astype(np.float64)) - 1.0)
    assert rel.max() < 0.035, rel.max()
