"""Host check of the row index that the second CGS2 pass uses to place an
element of the newest basis vector in its binary16 copy (rows of mx values
padded to mx4): row = (e * mul) >> (32 + s) with s = ceil(log2 mx) and
mul = ceil(2^(32+s) / mx) must equal e // mx for every e below 2^31 (the
workspace takes that route only for N < 2^31).  The check runs the same
unsigned 64-bit arithmetic on numpy's uint64, at every multiple of mx
(and one either side of it) in sampled ranges, and at the top of the range."""
import numpy as np
import pytest


def _mul_shift(mx):
    s = 0
    while (1 << s) < mx:
        s += 1
    return ((1 << (32 + s)) + mx - 1) // mx, 32 + s


@pytest.mark.parametrize("mx", [32, 33, 63, 64, 95, 126, 127, 255, 511, 1023, 1025, 4095, 8191, 46340])
def test_row_by_multiply_shift(mx):
    mul, shift = _mul_shift(mx)
    assert mul < (1 << 33)            # e * mul stays below 2^64 for e < 2^31
    top = (1 << 31) - 1
    rng = np.random.default_rng(mx)
    qs = np.concatenate([np.arange(0, 4096), rng.integers(0, top // mx, 20000), [top // mx - 1, top // mx]])
    e = np.concatenate([qs * mx - 1, qs * mx, qs * mx + 1, qs * mx + mx - 1, [top, top - 1]])
    e = e[(e >= 0) & (e <= top)].astype(np.uint64)
    row = (e * np.uint64(mul)) >> np.uint64(shift)
    np.testing.assert_array_equal(row, e // np.uint64(mx))


@pytest.mark.parametrize("mx", [32, 33, 63, 95, 127, 255, 256, 511, 1023, 1025, 4095])
def test_quad_row_by_multiply_shift(mx):
    """The binary16 basis passes walk a slot in quads of 4 pairs (rows of mx4
    = 4 mq pairs): row = (quad * mulq) >> (32 + s), s = ceil(log2 mq), mulq =
    ceil(2^(32+s) / mq), must equal quad // mq for every quad of a slot
    below 2^31 pairs; a quad's first column 4 (quad - row mq) then never
    reaches mx4."""
    mq = (mx + 3) // 4
    mul, shift = _mul_shift(mq)
    top = (1 << 29) - 1                 # quads of a slot of < 2^31 pairs
    rng = np.random.default_rng(mx + 1)
    qs = np.concatenate([np.arange(0, 2048), rng.integers(0, top // mq, 20000), [top // mq - 1, top // mq]])
    quad = np.concatenate([qs * mq - 1, qs * mq, qs * mq + 1, qs * mq + mq - 1, [top]])
    quad = quad[(quad >= 0) & (quad <= top)].astype(np.uint64)
    row = (quad * np.uint64(mul)) >> np.uint64(shift)
    np.testing.assert_array_equal(row, quad // np.uint64(mq))
    col0 = 4 * (quad - row * np.uint64(mq))
    assert int(col0.max()) <= 4 * mq - 4
