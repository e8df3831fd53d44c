"""Pins of the block floating-point format reference (oracle/bfp.py) against what its definition
fixes by arithmetic: worked values, the 16-bit headroom at the exponent boundary, the error bound,
exact round trips of representable values, zero and non-finite blocks, and the gain over FP16 on
smooth data.  CPU only."""
import numpy as np
import pytest

from oracle import bfp


def f32(x):
    return np.asarray(x, dtype=np.float32)


def test_worked_block():
    # M = 1.0: b = 127, mantissa 0 -> e = 113, scale 2^14; u = v 2^14 + 32768
    v = f32([1.0, 0.5, -0.25, 0.0, 2.0 ** -14, -1.0, 0.75, 3.0 * 2.0 ** -13])
    u, e = bfp.encode(v)
    assert e.tolist() == [113]
    assert u.tolist() == [49152, 40960, 28672, 32768, 32769, 16384, 45056, 32774]
    assert np.array_equal(bfp.decode(u, e), v.astype(np.float64))


def test_exponent_bump_keeps_headroom():
    # just below the bump: M 2^14 = 32766.5 - 2^-9 rounds to 32766 at e = b - 14
    below = np.float32((8388608 + bfp.BUMP_MANTISSA - 1) / 2.0 ** 23)
    at = np.float32((8388608 + bfp.BUMP_MANTISSA) / 2.0 ** 23)  # M 2^14 = 32766.5 -> next exponent
    top = np.nextafter(np.float32(2.0), np.float32(0.0))         # largest float below 2
    for m, want_e, want_k in ((below, 113, 32766), (at, 114, 16383), (top, 114, 16384)):
        u, e = bfp.encode(f32([m] + [0.0] * 7))
        assert e.tolist() == [want_e], m
        assert int(u[0]) - 32768 == want_k, m


@pytest.mark.parametrize("seed", range(4))
def test_error_bound_and_bit_usage(seed):
    rng = np.random.default_rng(seed)
    # blocks of very different magnitudes, signs and spreads
    v = (rng.normal(size=(7, 4096)) * 10.0 ** rng.uniform(-30, 5, size=(7, 512)).repeat(8, axis=1)).astype(np.float32)
    u, e = bfp.encode(v)
    got = bfp.decode(u, e)
    k = u.astype(np.int64) - 32768
    assert np.abs(k).max() <= 32766
    blocks = np.abs(v.astype(np.float64)).reshape(7, 512, 8)
    M = blocks.max(axis=-1)
    err = np.abs(got - v.astype(np.float64)).reshape(7, 512, 8).max(axis=-1)
    assert np.all(err <= 2.0 ** -15 * M * (1 + 2.0 ** -14))
    # the largest value of every non-zero block keeps at least 15 bits
    kmax = np.abs(k).reshape(7, 512, 8).max(axis=-1)
    assert np.all(kmax[M > 0] >= 16383)


def test_decoded_values_encode_back_to_themselves():
    rng = np.random.default_rng(7)
    v = (rng.normal(size=(5, 8192)) * 1e-3).astype(np.float32)
    once = bfp.round_trip(v)
    assert np.array_equal(bfp.round_trip(once.astype(np.float32)), once)
    # values that are multiples of the block unit within 32766 units are kept exactly
    e = 120
    unit = 2.0 ** (e - 127)
    ks = rng.integers(-32766, 32767, size=(3, 64))
    ks[:, ::8] = 32766  # the block maximum fixes e = 120 exactly (32766 < 32766.5)
    vals = (ks * unit).astype(np.float32)
    assert np.array_equal(bfp.round_trip(vals), ks * unit)


def test_zero_and_nonfinite_blocks():
    z = np.zeros(16, dtype=np.float32)
    u, e = bfp.encode(z)
    assert e.tolist() == [0, 0] and np.all(u == 32768)
    assert np.array_equal(bfp.decode(u, e), np.zeros(16))
    tiny = f32([1e-40] + [0.0] * 7)  # below 2^-112: the block flushes to zero
    assert bfp.block_exponents(tiny).tolist() == [0]
    for bad in (np.nan, np.inf, -np.inf):
        v = np.ones(16, dtype=np.float32)
        v[3] = bad
        u, e = bfp.encode(v)
        assert e.tolist() == [255, 113]
        out = bfp.decode(u, e)
        assert np.isnan(out[:8]).all() and np.array_equal(out[8:], np.ones(8))


def test_more_accurate_than_fp16_on_smooth_fields():
    x = np.arange(1 << 16)
    v = (1e-3 * np.exp(-((x - 30000.0) / 3000.0) ** 2) + 1e-4 * np.cos(2 * np.pi * x / 97.0)).astype(np.float32)
    e_bfp = np.linalg.norm(bfp.round_trip(v) - v) / np.linalg.norm(v)
    S = 2.0 ** 20
    f16 = (v.astype(np.float64) * S).astype(np.float16).astype(np.float64) / S
    e_f16 = np.linalg.norm(f16 - v) / np.linalg.norm(v)
    assert e_bfp * 8 < e_f16, (e_bfp, e_f16)
