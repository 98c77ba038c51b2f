"""Host checks of the binary32 identities the FP32 cell kernel relies on.

The kernel avoids integer<->float conversions (they issue on GB300's narrow FP64
pipe) by building values from bits.  Each identity is restated here in numpy
binary32 arithmetic, whose round-to-nearest operations match the device's, and
checked against its plain definition:

* the FP32 uniform ((w >> 8) + 1) 2^-24 equals (w >> 9) 2^-23 + (((w >> 8) & 1) + 1) 2^-24
  built as (float with mantissa w >> 9 in [1, 2)) - 1 plus 2^-24 or 2^-23, for
  every one of the 2^24 values of w >> 8;
* the null-collision candidate threshold H(p) -- the number of 16-bit prefixes
  h whose smallest uniform (256 h + 1) 2^-24 is below p -- equals
  ceil((p 2^24 - 1) / 256) evaluated in binary32, over random and boundary p.
"""
import numpy as np


def _f32(bits):
    return np.asarray(bits, dtype=np.uint32).view(np.float32)


def test_fp32_uniform_from_bits_all_inputs():
    u24 = np.arange(1 << 24, dtype=np.uint32)
    hi = _f32(np.uint32(0x3F800000) | (u24 >> np.uint32(1))) - np.float32(1.0)
    lo = _f32(np.uint32(0x33800000) + ((u24 & np.uint32(1)) << np.uint32(23)))
    built = (hi + lo).astype(np.float32)
    want = (u24.astype(np.float64) + 1.0) * 2.0 ** -24       # exact, then exactly representable
    assert np.array_equal(built.astype(np.float64), want)
    assert built.min() > 0 and built.max() == 1.0


def _threshold_f32(p):
    p = np.float32(p)
    h = np.ceil((p * np.float32(16777216.0) - np.float32(1.0)) * np.float32(0.00390625)).astype(np.float32)
    if not h > 0:
        return 0
    if h >= 65536:
        return 65536
    return int(h)


def _threshold_def(p):
    lo = (np.arange(65536, dtype=np.float64) * 256.0 + 1.0) * 2.0 ** -24   # smallest uniform of prefix h
    return int(np.count_nonzero(lo < np.float64(np.float32(p))))


def test_candidate_threshold_binary32():
    rng = np.random.default_rng(5)
    ps = list(rng.random(3000, dtype=np.float32))
    ps += list((rng.integers(0, 65536, 1000) * 256.0 + 1.0) * 2.0 ** -24)        # exactly at a boundary
    ps += list(np.nextafter(np.float32(ps[-1]), np.float32(2)) for _ in range(1))
    ps += [0.0, 1.0, 2.0 ** -24, 2.0 ** -23, 1.0 - 2.0 ** -24, 0.02, 0.5]
    ps += list(_f32(rng.integers(0, 0x3F800001, 2000, dtype=np.uint32)))           # all magnitudes
    for p in ps:
        assert _threshold_f32(p) == _threshold_def(p), p
