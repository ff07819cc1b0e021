"""The contrast kernel's integer map (no GPU): round-half-up((c) * maxv / q) for
0 <= c <= q = hi - lo, computed as a binary32 estimate
    est = trunc(fl32(c * fl32(maxv / q) + 1/2))        (one fused multiply-add)
and one correction by the exact remainder.  The kernel relies on the estimate
being off by at most one; this checks that claim exhaustively for 8 and 12
bits and on a large random sample (plus the extreme spans) for 16 bits,
emulating each binary32 rounding exactly: c * s + 1/2 is exact in binary64
for c < 2^16 and a binary32 s, so one rounding to binary32 is the FMA's."""
import numpy as np
import pytest


def exact(c, q, maxv):
    return (2 * c * maxv + q) // (2 * q)


def estimate(c, q, maxv):
    scale = (np.float32(maxv) / np.float32(q)).astype(np.float32)     # correctly rounded binary32 divide
    x = c.astype(np.float64) * scale.astype(np.float64) + 0.5         # exact in binary64
    return np.trunc(x.astype(np.float32)).astype(np.int64)             # one rounding, then truncation


def corrected(c, q, maxv):
    est = estimate(c, q, maxv)
    r = 2 * c * maxv + q - 2 * est * q
    return est - (r < 0) + (r >= 2 * q)


@pytest.mark.parametrize("bits", [8, 12])
def test_exhaustive(bits):
    maxv = (1 << bits) - 1
    for q in range(1, maxv + 1):
        c = np.arange(q + 1, dtype=np.int64)
        qa = np.full_like(c, q)
        e = exact(c, qa, maxv)
        est = estimate(c, qa, maxv)
        assert np.abs(est - e).max() <= 1, q
        np.testing.assert_array_equal(corrected(c, qa, maxv), e)


def test_sixteen_bit_sample_and_extremes():
    maxv = 65535
    rng = np.random.default_rng(5)
    q = rng.integers(1, maxv + 1, size=2_000_000)
    c = (rng.random(q.size) * (q + 1)).astype(np.int64)
    for qq in (1, 2, 3, 255, 4095, 65534, 65535):           # whole spans at the extremes
        cc = np.arange(qq + 1, dtype=np.int64)
        q = np.concatenate([q, np.full_like(cc, qq)])
        c = np.concatenate([c, cc])
    e = exact(c, q, maxv)
    assert np.abs(estimate(c, q, maxv) - e).max() <= 1
    np.testing.assert_array_equal(corrected(c, q, maxv), e)
