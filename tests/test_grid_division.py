"""The set-up's grid column, floor(x * nx / W), as a multiply-high: with
m = ceil(2^32 / W), the high word of (x * nx) * m equals the floor division
whenever (W - 1) * nx * W < 2^32 (the condition the library checks before it
uses the reciprocal).  Checked for every column of many widths and cell
counts that meet the condition, including widths near the limit."""
import numpy as np


def _reciprocal(length, cells):
    # the library's rule: 0 (divide instead) unless (length - 1) * cells * length < 2^32
    if length < 2:
        return 0
    num = (length - 1) * cells
    if num > 0xFFFFFFFF // length:
        return 0
    return (2**32 + length - 1) // length


def _check(W, nx):
    m = _reciprocal(W, nx)
    if m == 0:
        return False
    x = np.arange(W, dtype=np.uint64)
    num = x * np.uint64(nx)
    assert num.max() < 2**32
    hi = (num * np.uint64(m)) >> np.uint64(32)
    assert np.array_equal(hi, num // np.uint64(W)), (W, nx)
    return True


def test_grid_reciprocal_exact():
    rng = np.random.default_rng(7)
    checked = 0
    # common image widths and grid sizes
    for W in (2, 3, 7, 9, 31, 32, 33, 320, 481, 1080, 1920, 3840, 4096, 7680):
        for nx in {1, 2, 3, max(1, W // 30), max(1, W // 12), max(1, W // 5), W}:
            checked += _check(W, nx)
    # random (W, nx) pairs, and pairs at the edge of the condition
    for _ in range(400):
        W = int(rng.integers(2, 20000))
        limit = max(1, min(W, (0xFFFFFFFF // W) // (W - 1)))  # nx the condition admits
        nx = int(rng.integers(1, limit + 1))
        assert _check(W, nx)
        checked += 1
    for W in (1000, 4000, 16000, 40000):
        nx = (0xFFFFFFFF // W) // (W - 1)  # the largest nx the condition admits
        assert _check(W, nx)
        assert _reciprocal(W, nx + 1) == 0
        checked += 1
    assert checked > 300


def test_reciprocal_refuses_outside_condition():
    assert _reciprocal(1, 1) == 0
    assert _reciprocal(70000, 70000) == 0  # (W-1)*nx*W far above 2^32
